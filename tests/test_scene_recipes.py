"""The seeded synthetic workloads are what the documentation states: sizes,
cameras and the distributions of every parameter (checked statistically,
with bounds several standard errors wide), deterministic per seed."""
import math

import numpy as np
import pytest

from paper_2604_02120_gb300 import scenes


def _check_common(sc, n, sh_degree):
    k = (sh_degree + 1) ** 2
    assert sc.means.shape == (n, 3) and sc.scales.shape == (n, 3) and sc.quats.shape == (n, 4)
    assert sc.opacities.shape == (n,) and sc.sh.shape == (n, k, 3) and sc.sh_degree == sh_degree
    for a in (sc.means, sc.scales, sc.quats, sc.opacities, sc.sh):
        assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    np.testing.assert_allclose(np.linalg.norm(sc.quats.astype(np.float64), axis=1), 1.0, atol=1e-6)
    assert np.all(sc.opacities > 0) and np.all(sc.opacities < 1)


def _camera_at_origin_view(cam, w, h):
    assert (cam.width, cam.height) == (w, h)
    f = (h / 2) / math.tan(math.radians(30.0))  # 60 degree vertical field of view
    assert cam.fx == pytest.approx(f) and cam.fy == pytest.approx(f)
    assert (cam.cx, cam.cy) == (w / 2, h / 2)
    np.testing.assert_allclose(cam.position(), [0.0, 0.0, -3.0], atol=1e-12)


def test_uniform_workloads():
    for k, (w, h, n, deg) in {0: (256, 256, 10_000, 0), 1: (1280, 720, 200_000, 3)}.items():
        sc = scenes.make_config(k)
        _check_common(sc, n, deg)
        assert len(sc.cameras) == 1
        _camera_at_origin_view(sc.cameras[0], w, h)
        m = sc.means.astype(np.float64)
        assert m.min() >= -1 and m.max() <= 1 and abs(m.mean()) < 0.02
        ls = np.log(sc.scales.astype(np.float64))
        assert abs(ls.mean() + 4.0) < 0.02 and abs(ls.std() - 0.5) < 0.02
        logit = np.log(sc.opacities / (1 - sc.opacities.astype(np.float64)))
        assert abs(logit.mean()) < 0.05 and abs(logit.std() - 1.0) < 0.05
        dc = sc.sh[:, 0, :].astype(np.float64)
        assert abs(dc.std() - 0.3) < 0.01
        if deg == 3:
            assert abs(sc.sh[:, 1:, :].astype(np.float64).std() - 0.05) < 0.002


def test_clustered_workload():
    sc = scenes.make_config(2, n=200_000)
    _check_common(sc, 200_000, 0)
    _camera_at_origin_view(sc.cameras[0], 1920, 1080)
    ls = np.log(sc.scales.astype(np.float64))
    # one axis of each Gaussian shifted by -2 in log space: the per-Gaussian mean
    # log-scale is N(-4.5, 0.8) averaged over 3 axes, minus 2/3
    assert abs(ls.mean() - (-4.5 - 2.0 / 3.0)) < 0.02
    # 64 clusters: every mean lies within a few 0.2-sigma offsets of one of 64 centres
    m = sc.means.astype(np.float64)
    assert m.min() > -2 - 6 * 0.2 and m.max() < 2 + 6 * 0.2

    def occupied(p):  # cells of 0.1 holding at least one mean
        g = np.floor((p + 3.2) / 0.1).astype(np.int64)
        return len(np.unique(g[:, 0] * 10**6 + g[:, 1] * 10**3 + g[:, 2]))

    uniform = np.random.default_rng(1).uniform(m.min(0), m.max(0), m.shape)
    assert occupied(m) < 0.5 * occupied(uniform)  # measured: 37.6k cells against 107k
    assert scenes.make_config(2).means.shape == (1_000_000, 3)


def test_ring_workload_cameras():
    sc = scenes.make_config(3, n=1000)
    assert len(sc.cameras) == 16 and sc.sh_degree == 0
    allowed = {(640, 480), (1280, 720), (1600, 900), (1920, 1080)}
    assert {(c.width, c.height) for c in sc.cameras} <= allowed
    for i, c in enumerate(sc.cameras):
        p = c.position()
        assert abs(p[1]) < 1e-12 and math.hypot(p[0], p[2]) == pytest.approx(3.0)
        a = 2 * math.pi * i / 16
        np.testing.assert_allclose(p, [3 * math.sin(a), 0.0, -3 * math.cos(a)], atol=1e-9)
        # the view axis points at the origin
        np.testing.assert_allclose(c.R[2], -p / np.linalg.norm(p), atol=1e-12)


def test_heavy_tailed_workload():
    n = 300_000
    sc = scenes.make_config(4, n=n)
    _check_common(sc, n, 3)
    _camera_at_origin_view(sc.cameras[0], 3840, 2160)
    o = sc.opacities.astype(np.float64)
    # Beta(0.5, 0.5): P(o < x) = (2/pi) asin(sqrt(x)), U-shaped
    for x in (0.01, 0.1, 0.5):
        assert abs((o < x).mean() - 2 / math.pi * math.asin(math.sqrt(x))) < 0.005
    ls = np.log(sc.scales.astype(np.float64)[np.isfinite(sc.scales).all(1)])
    t = (ls + 4.5) / 0.7
    # Student t with 3 degrees of freedom: median 0, P(|t| > 3) = 0.0577
    assert abs(np.median(t)) < 0.01 and abs((np.abs(t) > 3).mean() - 0.0577) < 0.003


def test_seeded_and_deterministic():
    a, b, c = scenes.make_config(0, seed=5), scenes.make_config(0, seed=5), scenes.make_config(0, seed=6)
    assert scenes.scene_digest(a) == scenes.scene_digest(b) != scenes.scene_digest(c)
    g = scenes.upstream_grad(0, a.cameras)[0]
    assert g.shape == (3, 256, 256) and g.dtype == np.float32
    assert abs(g.mean()) < 0.01 and abs(g.std() - 1) < 0.01
    np.testing.assert_array_equal(g, scenes.upstream_grad(0, a.cameras)[0])
