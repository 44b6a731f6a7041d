"""Pins of the FP64 oracle against facts fixed outside it: hand-derived closed
forms, library routines (scipy densities, rotations, spherical harmonics),
invariants of Eq. 1, brute force and finite differences.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2604_02120_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _splat_set(mean2d, conic, opac, rgb, radius, depth):
    return dict(mean2d=np.asarray(mean2d, float), conic=np.asarray(conic, float),
                opac=np.asarray(opac, float), rgb=np.asarray(rgb, float),
                radius=np.asarray(radius, np.int32), depth=np.asarray(depth, np.float32))


def _blend_set(s, W, H, bg=(0, 0, 0)):
    bs = oracle.bin_sort(s["mean2d"], s["radius"], s["depth"], W, H)
    return oracle.blend(W, H, bs["tile_ranges"], bs["ids"], s["mean2d"], s["conic"], s["opac"], s["rgb"], bg=bg)


# ---------------------------------------------------------------- Eq. 6 ----

def test_eq6_dot_product_equals_quadratic():
    """Sec. 3.2, Eq. 6: v_g . v_p reproduces the quadratic exponent of Eq. 3."""
    rng = np.random.default_rng(1)
    n = 4000
    L = rng.standard_normal((n, 2, 2))
    cov = L @ np.transpose(L, (0, 2, 1)) + 0.1 * np.eye(2)
    inv = np.linalg.inv(cov)
    abc = np.stack([inv[:, 0, 0], inv[:, 0, 1], inv[:, 1, 1]], 1)
    hat = rng.uniform(-40, 40, (n, 2))
    bar = rng.integers(-7, 8, (n, 2)) + 0.5
    dot, direct = oracle.power_eq6(abc, hat, bar)
    # independent evaluation: -1/2 d^T Sigma^-1 d with d = hat + bar
    d = hat + bar
    ref = -0.5 * np.einsum("ni,nij,nj->n", d, inv, d)
    scale = np.abs(abc).max(1) * (np.abs(hat).max(1) + 8) ** 2
    assert np.max(np.abs(dot - ref) / scale) < 1e-13
    assert np.max(np.abs(direct - ref) / scale) < 1e-13


# ---------------------------------------------------------------- blend ----

def test_single_splat_matches_gaussian_density():
    """Eq. 2: alpha = o * exp(-1/2 x^T Sigma^-1 x) is the normalised 2D Gaussian
    density (scipy) scaled by the opacity, clamped at 0.99 and skipped below 1/255."""
    from scipy.stats import multivariate_normal
    W, H = 48, 40
    th = 0.7
    Rm = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    cov = Rm @ np.diag([25.0, 4.0]) @ Rm.T
    inv = np.linalg.inv(cov)
    m = np.array([20.3, 17.8])
    for o in (0.8, 1.0):
        s = _splat_set([m], [[inv[0, 0], inv[0, 1], inv[1, 1]]], [o], [[1.0, 0.5, 0.25]], [100], [1.0])
        r = _blend_set(s, W, H)
        mvn = multivariate_normal(mean=m, cov=cov)
        ys, xs = np.mgrid[0:H, 0:W]
        pts = np.stack([xs + 0.5, ys + 0.5], -1).reshape(-1, 2)
        ratio = (mvn.pdf(pts) / mvn.pdf(m)).reshape(H, W)
        alpha = np.minimum(0.99, o * ratio)
        alpha = np.where(alpha < 1 / 255, 0.0, alpha)
        for ch, c in enumerate((1.0, 0.5, 0.25)):
            np.testing.assert_allclose(r["image"][ch], c * alpha, rtol=0, atol=1e-12)
        np.testing.assert_allclose(r["T_final"], 1 - alpha, rtol=0, atol=1e-12)
        np.testing.assert_array_equal(r["n_contrib"], (alpha > 0).astype(np.int32))


def test_two_splat_composite_golden():
    """Eq. 1 on a hand-derived two-splat case (tests/golden/two_splat_composite.json)."""
    with open(os.path.join(GOLDEN, "two_splat_composite.json")) as f:
        gold = json.load(f)
    sp = gold["splats"]
    s = _splat_set([x["mean2d"] for x in sp], [x["conic"] for x in sp], [x["opacity"] for x in sp],
                   [x["rgb"] for x in sp], [3, 3], [x["depth"] for x in sp])
    px, py = gold["pixel"]
    for case in gold["cases"]:
        r = _blend_set(s, gold["width"], gold["height"], bg=case["bg"])
        np.testing.assert_allclose(r["image"][:, py, px], case["C"], rtol=0, atol=1e-15)
        assert r["T_final"][py, px] == pytest.approx(case["T"], abs=1e-15)
        assert r["n_contrib"][py, px] == case["n_contrib"]


def _stack_at_pixel(opacs, W=16, H=16, px=3, py=5):
    n = len(opacs)
    return _splat_set([[px + 0.5, py + 0.5]] * n, [[0.5, 0.0, 0.5]] * n, opacs,
                      [[1.0, 1.0, 1.0]] * n, [2] * n, np.arange(1, n + 1))


def test_alpha_skip_clamp_and_termination():
    """Alg. 1 rules: skip alpha < 1/255, clamp at 0.99, stop once T would drop below 1e-4."""
    px, py = 3, 5
    # skip: opacity just under 1/255 contributes nothing, n_contrib counts the later splat
    r = _blend_set(_stack_at_pixel([0.99 / 255, 0.5]), 16, 16)
    assert r["T_final"][py, px] == pytest.approx(0.5, abs=1e-15)
    assert r["n_contrib"][py, px] == 2
    # clamp: opacity 1 at the centre gives alpha 0.99
    r = _blend_set(_stack_at_pixel([1.0]), 16, 16)
    assert r["T_final"][py, px] == pytest.approx(0.01, abs=1e-15)
    # termination: T = 0.01 * 0.01 = 1e-4 is kept (not below), the third would reach 1e-6: stop
    r = _blend_set(_stack_at_pixel([1.0, 1.0, 1.0, 0.5]), 16, 16)
    assert r["n_contrib"][py, px] == 2
    assert r["T_final"][py, px] == pytest.approx(1e-4, rel=1e-12)
    assert r["image"][0, py, px] == pytest.approx(0.99 + 0.99 * 0.01, abs=1e-14)
    # boundaries are strict: alpha == 1/255 exactly is kept (skip only below it)
    r = _blend_set(_stack_at_pixel([1.0 / 255.0]), 16, 16)
    assert r["n_contrib"][py, px] == 1
    assert r["T_final"][py, px] == 1.0 - 1.0 / 255.0
    # ... and a test transmittance exactly equal to 1e-4 is kept (stop only below it):
    # 13 splats of alpha 1/2 leave T = 2^-13; alpha = 1 - 1e-4 * 2^13 (exact in FP64)
    # then gives T * (1 - alpha) == 1e-4 to the last bit.
    v = 1e-4 * 8192.0
    last = 1.0 - v
    assert 1.0 - last == v and (2.0 ** -13) * (1.0 - last) == 1e-4
    r = _blend_set(_stack_at_pixel([0.5] * 13 + [last, 0.5]), 16, 16)
    assert r["n_contrib"][py, px] == 14
    assert r["T_final"][py, px] == 1e-4


def test_partition_of_unity_and_monotone_transmittance():
    """Eq. 1 telescopes: with white splats and a black background, C + T_final = 1;
    and truncating every list can only raise T (T is non-increasing)."""
    sc = scenes.tiny_scene(3, n=64, width=64, height=48)
    cam = sc.cameras[0]
    pr = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, 0, cam)
    bs = oracle.bin_sort(pr["mean2d"], pr["radius"], pr["depth"].astype(np.float32), cam.width, cam.height)
    white = np.ones_like(pr["rgb"])
    r = oracle.blend(cam.width, cam.height, bs["tile_ranges"], bs["ids"], pr["mean2d"], pr["conic"],
                     sc.opacities.astype(float), white)
    assert np.max(np.abs(r["image"][0] + r["T_final"] - 1)) < 1e-12
    assert (r["n_contrib"] > 0).mean() > 0.3
    ranges = bs["tile_ranges"].astype(np.int64)
    ranges[1::2] = np.maximum(ranges[0::2], ranges[1::2] - 1)
    ranges = ranges.astype(np.uint32)
    r2 = oracle.blend(cam.width, cam.height, ranges, bs["ids"], pr["mean2d"], pr["conic"],
                      sc.opacities.astype(float), white)
    assert np.all(r2["T_final"] >= r["T_final"] - 1e-15)


@pytest.mark.parametrize("seed,W,H", [(0, 48, 40), (1, 33, 17), (2, 64, 64), (5, 16, 16)])
def test_tiled_blend_equals_per_pixel_brute_force(seed, W, H):
    """Duplication + sort + per-tile blending equals compositing, per pixel, all
    splats whose rectangle covers the pixel's tile in depth order."""
    sc = scenes.tiny_scene(seed, n=48, width=W, height=H)
    cam = sc.cameras[0]
    pr = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, 0, cam)
    d32 = pr["depth"].astype(np.float32)
    bs = oracle.bin_sort(pr["mean2d"], pr["radius"], d32, W, H)
    bg = (0.1, 0.2, 0.3)
    tiled = oracle.blend(W, H, bs["tile_ranges"], bs["ids"], pr["mean2d"], pr["conic"],
                         sc.opacities.astype(float), pr["rgb"], bg=bg)
    brute = oracle.brute_force(pr["mean2d"], pr["conic"], sc.opacities.astype(float), pr["rgb"],
                               pr["radius"], d32, W, H, bg=bg, use_rect=True)
    np.testing.assert_array_equal(tiled["image"], brute["image"])
    np.testing.assert_array_equal(tiled["T_final"], brute["T_final"])
    np.testing.assert_array_equal(tiled["n_contrib"], brute["n_contrib"])


def test_permutation_invariance():
    """With distinct depths the render does not depend on the input order."""
    sc = scenes.tiny_scene(7, n=40, width=48, height=48, sh_degree=1)
    base = oracle.render(sc)
    assert len(np.unique(base["project"]["depth"].astype(np.float32))) == sc.n
    perm = np.random.default_rng(0).permutation(sc.n)
    sc2 = scenes.Scene(sc.means[perm], sc.scales[perm], sc.quats[perm], sc.opacities[perm], sc.sh[perm],
                       sc.sh_degree, sc.cameras)
    other = oracle.render(sc2)
    np.testing.assert_array_equal(base["blend"]["image"], other["blend"]["image"])
    np.testing.assert_array_equal(base["blend"]["n_contrib"], other["blend"]["n_contrib"])


# ------------------------------------------------------------- bin/sort ----

def test_bin_sort_membership_and_order():
    """Sec. 2.1 stages 2-3: tile t's list holds exactly the splats whose closed
    3-sigma square meets the tile's half-open pixel box, ordered by (float
    depth, index), with key (t << 32) | depth bits."""
    sc = scenes.tiny_scene(11, n=80, width=70, height=45)
    cam = sc.cameras[0]
    pr = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, 0, cam)
    d32 = pr["depth"].astype(np.float32)
    bs = oracle.bin_sort(pr["mean2d"], pr["radius"], d32, cam.width, cam.height)
    tx, ty = cam.tiles_x, cam.tiles_y
    m, r = pr["mean2d"], pr["radius"].astype(float)
    total = 0
    for t in range(tx * ty):
        a, b = bs["tile_ranges"][2 * t], bs["tile_ranges"][2 * t + 1]
        got = list(bs["ids"][a:b])
        x0, y0 = 16 * (t % tx), 16 * (t // tx)
        meet = ((pr["radius"] > 0) & (m[:, 0] - r < x0 + 16) & (m[:, 0] + r >= x0)
                & (m[:, 1] - r < y0 + 16) & (m[:, 1] + r >= y0))
        want = sorted(np.nonzero(meet)[0], key=lambda g: (d32[g], g))
        assert got == want
        dbits = d32.view(np.uint32)
        for i, g in zip(range(a, b), got):
            assert int(bs["keys"][i]) == (t << 32) | int(dbits[g])
        total += len(got)
    assert total == bs["n_instances"] > 0


def _power_min(opac):
    """ln(1/(255 o)) - 2e-3 in float32, +inf where o is below the blend's
    float32 threshold 1/255 (the library computes the same with
    gs_alpha_power_min and hands it to both sides)."""
    o = np.asarray(opac, np.float64)
    keep = np.asarray(opac, np.float32) >= np.float32(1.0) / np.float32(255.0)
    return np.where(keep, -np.log(255 * o) - 2e-3, np.inf).astype(np.float32)


def _tight_case(seed, W, H, n=120):
    sc = scenes.tiny_scene(seed, n=n, width=W, height=H, sh_degree=0, scale_lo=-3.2, scale_hi=-1.2,
                           opac_lo=0.02, opac_hi=0.99)
    cam = sc.cameras[0]
    pr = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, 0, cam)
    # the kernels' float32 inputs
    m32, c32 = pr["mean2d"].astype(np.float32), pr["conic"].astype(np.float32)
    d32 = pr["depth"].astype(np.float32)
    pmin = _power_min(sc.opacities)
    full = oracle.bin_sort(m32.astype(np.float64), pr["radius"], d32, W, H)
    tight = oracle.bin_sort(m32.astype(np.float64), pr["radius"], d32, W, H, conic=c32, power_min=pmin)
    return sc, cam, m32, c32, d32, pmin, full, tight


@pytest.mark.parametrize("seed,W,H", [(3, 70, 45), (4, 64, 64), (9, 33, 50)])
def test_tight_lists_render_like_full_lists(seed, W, H):
    """Opacity-aware lists drop only splats that fail alpha >= 1/255 at every
    pixel of the tile: each tile's list is a sub-sequence of the full one, the
    composite (Eq. 1 with the skip rule) is bit for bit the same, and fewer
    instances remain."""
    sc, cam, m32, c32, d32, pmin, full, tight = _tight_case(seed, W, H)
    assert 0 < tight["n_instances"] < full["n_instances"]
    for t in range(cam.num_tiles):
        a = list(full["ids"][full["tile_ranges"][2 * t]:full["tile_ranges"][2 * t + 1]])
        b = list(tight["ids"][tight["tile_ranges"][2 * t]:tight["tile_ranges"][2 * t + 1]])
        it = iter(a)
        assert all(g in it for g in b), f"tile {t}: not a sub-sequence"
    args = (m32.astype(np.float64), c32.astype(np.float64), sc.opacities.astype(np.float64),
            np.full((sc.n, 3), 0.5))
    bg = (0.2, 0.1, 0.0)
    rf = oracle.blend(W, H, full["tile_ranges"], full["ids"], *args, bg=bg)
    rt = oracle.blend(W, H, tight["tile_ranges"], tight["ids"], *args, bg=bg)
    np.testing.assert_array_equal(rt["image"], rf["image"])
    np.testing.assert_array_equal(rt["T_final"], rf["T_final"])
    assert (rt["n_contrib"] <= rf["n_contrib"]).all()


def test_tight_lists_keep_every_pair_that_reaches_the_threshold():
    """Brute force: a splat whose alpha = o exp(power) reaches 1/255 at any pixel
    centre of a tile (FP64) is in that tile's opacity-aware list."""
    sc, cam, m32, c32, d32, pmin, full, tight = _tight_case(21, 80, 64, n=200)
    W, H = cam.width, cam.height
    o = sc.opacities.astype(np.float64)
    ys, xs = np.mgrid[0:H, 0:W] + 0.5
    checked = 0
    for t in range(cam.num_tiles):
        x0, y0 = 16 * (t % cam.tiles_x), 16 * (t // cam.tiles_x)
        px, py = xs[y0:y0 + 16, x0:x0 + 16], ys[y0:y0 + 16, x0:x0 + 16]
        kept = set(tight["ids"][tight["tile_ranges"][2 * t]:tight["tile_ranges"][2 * t + 1]])
        for g in full["ids"][full["tile_ranges"][2 * t]:full["tile_ranges"][2 * t + 1]]:
            A, B, C = c32[g].astype(np.float64)
            dx, dy = m32[g, 0] - px, m32[g, 1] - py
            power = -0.5 * (A * dx * dx + 2 * B * dx * dy + C * dy * dy)
            if (o[g] * np.exp(np.minimum(power, 0.0))).max() >= 1 / 255:
                assert g in kept, f"tile {t} lost splat {g}"
                checked += 1
    assert checked > 100


def test_tight_test_is_the_box_maximum():
    """The opacity-aware rule keeps a splat on a tile exactly when the largest
    exponent -q/2 over the tile's box of pixel-centre offsets reaches
    power_min (the box meets the ellipse q <= -2 power_min): the box minimum
    of q comes from a library box-constrained minimiser (L-BFGS-B, q convex)
    in FP64, and every decision whose exponent is clear of the threshold by
    more than rounding must agree.  The pairs the oracle reports as
    ambiguous are exactly those near the threshold."""
    from scipy.optimize import minimize

    sc, cam, m32, c32, d32, pmin, full, tight = _tight_case(5, 96, 64, n=160)
    amb = {(int(t), int(g)) for t, g, _ in tight["ambiguous"]}
    decided = dropped = 0
    for t in range(cam.num_tiles):
        tx, ty = t % cam.tiles_x, t // cam.tiles_x
        kept = set(tight["ids"][tight["tile_ranges"][2 * t]:tight["tile_ranges"][2 * t + 1]])
        for g in set(full["ids"][full["tile_ranges"][2 * t]:full["tile_ranges"][2 * t + 1]]):
            A, B, C = c32[g].astype(np.float64)
            mx, my = m32[g].astype(np.float64)
            box = [(mx - 16 * tx - 15.5, mx - 16 * tx - 0.5), (my - 16 * ty - 15.5, my - 16 * ty - 0.5)]

            def q(d):
                return A * d[0] ** 2 + 2 * B * d[0] * d[1] + C * d[1] ** 2

            def dq(d):
                return np.array([2 * (A * d[0] + B * d[1]), 2 * (B * d[0] + C * d[1])])

            start = np.array([sum(box[0]) / 2, sum(box[1]) / 2])
            res = minimize(q, start, jac=dq, method="L-BFGS-B", bounds=box, options={"ftol": 1e-15, "gtol": 1e-12})
            power = -0.5 * max(res.fun, 0.0)
            if abs(power - float(pmin[g])) <= 1e-4 + 1e-5 * abs(res.fun):
                continue
            assert (t, int(g)) not in amb, f"tile {t} splat {g}: clear of the threshold but reported ambiguous"
            assert (g in kept) == (power >= pmin[g]), f"tile {t} splat {g}: box max {power} vs {pmin[g]}"
            decided += 1
            dropped += g not in kept
    assert decided > 300 and dropped > 50


def _dense_box_min(A, B, C, box, n=1601):
    """min of q over the box sampled on its four edges and an interior grid
    (an upper bound of the true minimum, within |grad q| * h / 2)."""
    (x0, x1), (y0, y1) = box
    xs, ys = np.linspace(x0, x1, n), np.linspace(y0, y1, n)
    pts = [(xs, np.full(n, y0)), (xs, np.full(n, y1)), (np.full(n, x0), ys), (np.full(n, x1), ys)]
    gx, gy = np.meshgrid(np.linspace(x0, x1, 81), np.linspace(y0, y1, 81))
    pts.append((gx.ravel(), gy.ravel()))
    return min(float((A * x * x + 2 * B * x * y + C * y * y).min()) for x, y in pts)


def test_tight_rule_on_needles_and_indefinite_conics():
    """Nearly singular and indefinite conics (the projected 2D covariance of
    a Gaussian with one huge scale gives A C - B^2 ~ 0, and rounded to float32
    it can come out <= 0): the box minimum is still that of q over the box,
    which a dense sampling of the box bounds from above; every pair the
    sampling puts clearly below or above the threshold is decided that way,
    and an indefinite form keeps the tiles near its zero lines only."""
    rng = np.random.default_rng(3)
    W, H = 160, 128
    n = 24
    mean2d = np.column_stack([rng.uniform(-40, W + 40, n), rng.uniform(-40, H + 40, n)]).astype(np.float32)
    theta = rng.uniform(0, np.pi, n)
    a2 = 10.0 ** rng.uniform(-2, 0, n)           # curvature across the needle
    b2 = a2 * 10.0 ** rng.uniform(-9, -5, n)     # along it: A C - B^2 = a2 b2 ~ 0
    b2[n // 2:] = -b2[n // 2:]                   # half of them indefinite
    c, s_ = np.cos(theta), np.sin(theta)
    conic = np.column_stack([a2 * c * c + b2 * s_ * s_, (a2 - b2) * c * s_, a2 * s_ * s_ + b2 * c * c])
    conic = conic.astype(np.float32)
    assert (conic[:, 0] > 0).all() and (conic[:, 2] > 0).all()
    opac = rng.uniform(0.05, 0.9, n)
    pmin = _power_min(opac)
    radius = np.full(n, 400, np.int32)
    depth = np.arange(1, n + 1, dtype=np.float32)
    full = oracle.bin_sort(mean2d.astype(np.float64), radius, depth, W, H)
    tight = oracle.bin_sort(mean2d.astype(np.float64), radius, depth, W, H, conic=conic, power_min=pmin)
    assert full["n_instances"] == n * ((W // 16) * (H // 16))
    amb = {(int(t), int(g)) for t, g, _ in tight["ambiguous"]}
    tx_n = (W + 15) // 16
    clear = kept_n = 0
    for t in range(tx_n * ((H + 15) // 16)):
        tx, ty = t % tx_n, t // tx_n
        kept = set(tight["ids"][tight["tile_ranges"][2 * t]:tight["tile_ranges"][2 * t + 1]].tolist())
        for g in range(n):
            A, B, C = conic[g].astype(np.float64)
            mx, my = mean2d[g].astype(np.float64)
            tau2 = -2.0 * float(pmin[g])
            box = [(mx - 16 * tx - 15.5, mx - 16 * tx - 0.5), (my - 16 * ty - 15.5, my - 16 * ty - 0.5)]
            qs = _dense_box_min(A, B, C, box)
            # the sampled minimum is within |grad q| * h of the true one (h = 15/1600)
            slack = 2 * (abs(A) * 200 + abs(B) * 200 + abs(C) * 200) * (15.0 / 1600) + 1e-9
            if qs - slack > tau2 * (1 + 1e-5):
                assert g not in kept, f"tile {t} needle {g}: kept, sampled box min {qs} > tau2 {tau2}"
            elif qs <= tau2 * (1 - 1e-5):
                assert g in kept, f"tile {t} needle {g}: dropped, sampled box min {qs} <= tau2 {tau2}"
                kept_n += 1
            else:
                continue
            assert (t, g) not in amb
            clear += 1
    assert clear > 0.9 * n * tx_n * ((H + 15) // 16) and 0 < kept_n < tight["n_instances"] + 1
    assert tight["n_instances"] < 0.5 * full["n_instances"]


def test_tight_rule_exact_threshold_is_kept_and_ambiguous():
    """A box whose minimum of q equals tau2 exactly (isotropic conic A = C = 1,
    B = 0, tau2 = 4, the box's near edge 2 px from the mean and the mean's
    row inside the box) is kept (max power = power_min reaches it) and is
    reported ambiguous; moved 1e-6 px further it is dropped and still
    ambiguous; moved 0.01 px further it is dropped and clear."""
    W, H = 64, 32
    shifts = [0.0, 1e-6, 0.01]
    # splat k sits right of tile (0, 0): the tile's offsets run x in [mx - 15.5, mx - 0.5]
    mean2d = np.array([[15.5 + 2.0 + s, 8.0] for s in shifts], np.float64)
    mean2d = mean2d.astype(np.float32).astype(np.float64)
    conic = np.tile(np.array([1.0, 0.0, 1.0], np.float32), (len(shifts), 1))
    pmin = np.full(len(shifts), -2.0, np.float32)
    radius = np.full(len(shifts), 6, np.int32)
    depth = np.arange(1, len(shifts) + 1, dtype=np.float32)
    tight = oracle.bin_sort(mean2d, radius, depth, W, H, conic=conic, power_min=pmin)
    kept0 = set(tight["ids"][tight["tile_ranges"][0]:tight["tile_ranges"][1]].tolist())
    amb = {(int(t), int(g)): int(k) for t, g, k in tight["ambiguous"]}
    x0 = mean2d[:, 0] - 15.5
    assert x0[0] == 2.0 and x0[1] > 2.0
    assert 0 in kept0 and amb.get((0, 0)) == 1
    assert 1 not in kept0 and amb.get((0, 1)) == 0
    assert 2 not in kept0 and (0, 2) not in amb


def test_rounding_model_bounds_float32_exponent_of_needles():
    """The oracle's rounding model for ambiguity (sum margin): a float32
    evaluation of Eq. 3's exponent errs by at most a few unit roundoffs times
    the magnitude sum S of its three terms, which for a nearly singular conic
    far from its centre is thousands of times the exponent itself.  An
    independent float32 evaluation (numpy, one rounding per operation) stays
    within 4 u S of the FP64 value on random needles, while a flat 2e-6
    margin does not cover it; and a pixel whose alpha lies within 4 u S of
    1/255, but not within 2e-6, is ambiguous only under the sum margin."""
    f32, u = np.float32, 2.0 ** -24
    rng = np.random.default_rng(9)
    n = 20000
    theta = rng.uniform(0, np.pi, n)
    a2 = 10.0 ** rng.uniform(-3, 0, n)
    b2 = a2 * 10.0 ** rng.uniform(-6, -2, n)
    c, s_ = np.cos(theta), np.sin(theta)
    A = (a2 * c * c + b2 * s_ * s_).astype(f32)
    B = ((a2 - b2) * c * s_).astype(f32)
    C = (a2 * s_ * s_ + b2 * c * c).astype(f32)
    # offsets along the needle's null direction, where the terms cancel
    t = rng.uniform(50, 2000, n)
    dx = (t * -s_ + rng.normal(0, 2, n)).astype(f32)
    dy = (t * c + rng.normal(0, 2, n)).astype(f32)
    pw32 = (-f32(0.5) * (A * dx * dx + C * dy * dy) - B * dx * dy).astype(np.float64)
    A64, B64, C64, dx64, dy64 = (x.astype(np.float64) for x in (A, B, C, dx, dy))
    pw64 = -0.5 * A64 * dx64 ** 2 - B64 * dx64 * dy64 - 0.5 * C64 * dy64 ** 2
    S = 0.5 * np.abs(A64) * dx64 ** 2 + np.abs(B64 * dx64 * dy64) + 0.5 * np.abs(C64) * dy64 ** 2
    err = np.abs(pw32 - pw64)
    assert (err <= 4 * u * S).all()
    assert (err > 2e-6).mean() > 0.5
    # one needle, one pixel: alpha just above 1/255 by more than 2e-6 but less than 4 u S
    k = int(np.argmax(S * ((pw64 > -5.4) & (pw64 < -0.2))))
    o = float(np.exp(np.log(1 / 255) - pw64[k]) * (1 + 0.5 * 4 * u * S[k]))
    assert 2e-6 < 0.5 * 4 * u * S[k] and o < 1
    mean2d = np.array([[0.5 + float(dx64[k]), 0.5 + float(dy64[k])]])
    conic = np.array([[A64[k], B64[k], C64[k]]])
    ranges, ids = np.array([0, 1], np.uint32), np.array([0], np.uint32)
    W = H = 1
    base = dict(alpha_margin=2e-6, t_margin=1e-5)
    flat = oracle.blend(W, H, ranges, ids, mean2d, conic, np.array([o]), np.ones((1, 3)), **base)
    model = oracle.blend(W, H, ranges, ids, mean2d, conic, np.array([o]), np.ones((1, 3)), sum_margin=4 * u,
                         sum_slack=0.0, **base)
    assert flat["n_contrib"][0, 0] == 1 and not flat["ambiguous"][0, 0]
    assert model["ambiguous"][0, 0]
    np.testing.assert_array_equal(model["image"], flat["image"])
    # without margins there is no bound; with them the bound covers alpha's relative error
    assert flat["err_bound"][0, 0] > 0 and model["err_bound"][0, 0] > flat["err_bound"][0, 0]
    none = oracle.blend(W, H, ranges, ids, mean2d, conic, np.array([o]), np.ones((1, 3)))
    assert none["err_bound"][0, 0] == 0 and not none["ambiguous"][0, 0]


def test_bin_sort_capacity_overflow_reports():
    sc = scenes.tiny_scene(11, n=20, width=48, height=48)
    cam = sc.cameras[0]
    pr = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, 0, cam)
    bs = oracle.bin_sort(pr["mean2d"], pr["radius"], pr["depth"].astype(np.float32), 48, 48, capacity=1)
    assert bs["n_instances"] == -1


# ------------------------------------------------------------ projection ----

def _cam(W=64, H=48, f=50.0):
    return scenes.Camera(W, H, f, f, W / 2, H / 2, np.eye(3), np.array([0.0, 0.0, 3.0]))


def _one(mean, scale, quat=(1.0, 0.0, 0.0, 0.0), sh=None, deg=0):
    sh = np.zeros((1, (deg + 1) ** 2, 3), np.float32) if sh is None else np.asarray(sh, np.float32)
    return (np.asarray([mean], np.float32), np.asarray([scale], np.float32),
            np.asarray([quat], np.float32), sh, deg)


def test_project_isotropic_closed_form():
    """An isotropic splat on the optical axis at depth z projects to a circle of
    variance (f s / z)^2 + lowpass centred on the principal point."""
    cam = _cam()
    s = np.float32(0.05)
    pr = oracle.project(*_one((0, 0, 0), (s, s, s)), cam)
    var = (50.0 * float(s) / 3.0) ** 2 + 0.3
    np.testing.assert_allclose(pr["cov2d"][0], [var, 0, var], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(pr["conic"][0], [1 / var, 0, 1 / var], rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(pr["mean2d"][0], [32.0, 24.0], rtol=0, atol=1e-13)
    assert pr["depth"][0] == pytest.approx(3.0)
    assert pr["radius"][0] == math.ceil(3 * math.sqrt(var))


def test_project_offaxis_closed_form():
    """Hand-derived EWA for an axis-aligned splat at world (x, 0, 0): with J =
    [[f/z, 0, -f x/z^2], [0, f/z, 0]], Sigma2 = diag((f/z)^2 sx^2 + (f x/z^2)^2 sz^2,
    (f/z)^2 sy^2) + lowpass I; quaternion (cos 45, 0, 0, sin 45) swaps sx and sy."""
    cam = _cam()
    x = np.float32(0.4)
    sx, sy, sz = (np.float32(v) for v in (0.03, 0.07, 0.11))
    f, z = 50.0, 3.0
    pr = oracle.project(*_one((x, 0, 0), (sx, sy, sz)), cam)
    a = (f / z) ** 2 * float(sx) ** 2 + (f * float(x) / z ** 2) ** 2 * float(sz) ** 2 + 0.3
    c = (f / z) ** 2 * float(sy) ** 2 + 0.3
    np.testing.assert_allclose(pr["cov2d"][0], [a, 0, c], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(pr["mean2d"][0], [f * float(x) / z + 32, 24], rtol=1e-14)
    h = math.sqrt(0.5)
    pr2 = oracle.project(*_one((0, 0, 0), (sx, sy, sz), (h, 0, 0, h)), cam)
    c2 = (f / z) ** 2 * float(sx) ** 2 + 0.3
    a2 = (f / z) ** 2 * float(sy) ** 2 + 0.3
    np.testing.assert_allclose(pr2["cov2d"][0], [a2, 0, c2], rtol=1e-6, atol=1e-6)


def test_project_matches_numerical_jacobian():
    """EWA splatting: Sigma2 = J Sigma3 J^T + lowpass I, where J is the Jacobian of
    the pixel projection of the mean (central differences of the oracle's own
    mean2d) and Sigma3 = R S^2 R^T from scipy's quaternion rotation."""
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(4)
    R0 = Rotation.from_euler("xyz", [0.2, -0.3, 0.1]).as_matrix()
    cam = scenes.Camera(96, 80, 70.0, 65.0, 47.0, 41.0, R0, np.array([0.1, -0.2, 3.5]))
    for _ in range(6):
        mean = rng.uniform(-0.6, 0.6, 3).astype(np.float32)
        scale = np.exp(rng.uniform(-4, -2, 3)).astype(np.float32)
        q = rng.standard_normal(4)
        q = (q / np.linalg.norm(q)).astype(np.float32)
        pr = oracle.project(*_one(mean, scale, q), cam)
        h = 1e-4
        J = np.zeros((2, 3))
        for j in range(3):
            mp = mean.astype(np.float64).copy()
            mm = mp.copy()
            mp[j] += h
            mm[j] -= h
            # the oracle takes float32 means, so evaluate the projection in double here
            def proj(p):
                pc = cam.R @ p + cam.t
                return np.array([cam.fx * pc[0] / pc[2] + cam.cx, cam.fy * pc[1] / pc[2] + cam.cy])
            J[:, j] = (proj(mp) - proj(mm)) / (2 * h)
        qd = q.astype(np.float64)
        Rq = Rotation.from_quat([qd[1], qd[2], qd[3], qd[0]]).as_matrix()
        S3 = Rq @ np.diag(scale.astype(np.float64) ** 2) @ Rq.T
        S2 = J @ S3 @ J.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(pr["cov2d"][0], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(pr["mean2d"][0], proj(mean.astype(np.float64)), rtol=1e-12)
        inv = np.linalg.inv(np.array([[pr["cov2d"][0][0], pr["cov2d"][0][1]],
                                      [pr["cov2d"][0][1], pr["cov2d"][0][2]]]))
        np.testing.assert_allclose(pr["conic"][0], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-10)


def test_project_camera_rotation_invariance():
    """Rotating the world by Q = R0^T Rk and viewing it from camera 0 equals
    viewing the original world from ring camera k (SH degree 0 colours)."""
    from scipy.spatial.transform import Rotation
    sc = scenes.tiny_scene(9, n=30, width=64, height=64)
    ring = scenes.ring_cameras(8, 3.0, [(64, 64)] * 8)
    c0 = ring[0]
    for k in (1, 3, 6):
        ck = ring[k]
        Q = c0.R.T @ ck.R
        means2 = (sc.means.astype(np.float64) @ Q.T).astype(np.float32)
        qs = sc.quats.astype(np.float64)
        rot = Rotation.from_matrix(Q) * Rotation.from_quat(qs[:, [1, 2, 3, 0]])
        q2 = rot.as_quat()[:, [3, 0, 1, 2]].astype(np.float32)
        a = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, 0, ck)
        b = oracle.project(means2, sc.scales, q2, sc.sh, 0, c0)
        for key in ("mean2d", "cov2d", "depth", "rgb"):
            np.testing.assert_allclose(a[key], b[key], rtol=2e-5, atol=2e-5)


def test_project_culling():
    cam = _cam()
    # behind the camera, and in front of it but nearer than znear
    pr = oracle.project(*_one((0, 0, -3.5), (0.05, 0.05, 0.05)), cam)
    assert pr["radius"][0] == 0 and pr["tiles_touched"][0] == 0
    pr = oracle.project(*_one((0, 0, -2.9), (0.05, 0.05, 0.05)), cam)
    assert pr["radius"][0] == 0
    # far outside the image: rectangle empty
    pr = oracle.project(*_one((30.0, 0, 0), (0.01, 0.01, 0.01)), cam)
    assert pr["tiles_touched"][0] == 0
    # degenerate covariance without the low-pass: det = 0, culled
    c2 = _cam()
    c2.lowpass = 0.0
    pr = oracle.project(*_one((0, 0, 0), (0.0, 0.05, 0.05)), c2)
    assert pr["radius"][0] == 0


def test_sh_basis_matches_scipy():
    """Real SH to degree 3: sqrt(2) Re/Im of scipy's complex harmonics (with the
    Condon-Shortley phase), order m = -l..l."""
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(2)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    got = oracle.sh_basis(d)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            Y = sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                ref = math.sqrt(2) * Y.real
            elif m < 0:
                ref = math.sqrt(2) * Y.imag
            else:
                ref = Y.real
            np.testing.assert_allclose(got[:, k], ref, rtol=0, atol=1e-12, err_msg=f"l={l} m={m}")
            k += 1


def test_sh_degree0_colour():
    cam = _cam()
    sh = np.array([[[0.3, -0.2, -2.5]]], np.float32)
    pr = oracle.project(*_one((0, 0, 0), (0.05, 0.05, 0.05), sh=sh), cam)
    y00 = 0.28209479177387814  # 1 / (2 sqrt(pi))
    want = np.maximum(0, y00 * sh[0, 0].astype(np.float64) + 0.5)
    np.testing.assert_allclose(pr["rgb"][0], want, rtol=1e-15)


# ------------------------------------------------------------- gradients ----

def test_blend_grad_matches_central_differences():
    """The analytic blend gradient equals FP64 central differences of the loss
    L = sum(w * image) for every parameter whose perturbation changes no
    skip / stop decision (two step sizes must agree)."""
    sc = scenes.tiny_scene(21, n=24, width=40, height=36, sh_degree=1)
    cam = sc.cameras[0]
    W, H = cam.width, cam.height
    pr = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, 1, cam)
    bs = oracle.bin_sort(pr["mean2d"], pr["radius"], pr["depth"].astype(np.float32), W, H)
    rng = np.random.default_rng(5)
    w = rng.standard_normal((3, H, W))
    bg = (0.2, 0.1, 0.05)
    params = dict(mean2d=pr["mean2d"].copy(), conic=pr["conic"].copy(),
                  opacity=sc.opacities.astype(float).copy(), rgb=pr["rgb"].copy())

    def loss(p):
        r = oracle.blend(W, H, bs["tile_ranges"], bs["ids"], p["mean2d"], p["conic"], p["opacity"],
                         p["rgb"], bg=bg)
        return float(np.sum(w * r["image"]))

    g = oracle.blend_grad(W, H, bs["tile_ranges"], bs["ids"], params["mean2d"], params["conic"],
                          params["opacity"], params["rgb"], w, bg=bg)
    live = np.nonzero(pr["radius"] > 0)[0]
    checked = 0
    for name in ("mean2d", "conic", "opacity", "rgb"):
        fd_all, an_all = [], []
        arr = params[name]
        for gidx in live:
            for j in range(arr.shape[1] if arr.ndim == 2 else 1):
                idx = (gidx, j) if arr.ndim == 2 else (gidx,)
                base = arr[idx]
                ests = []
                for h in (1e-6 * max(1.0, abs(base)), 2.5e-7 * max(1.0, abs(base))):
                    arr[idx] = base + h
                    lp = loss(params)
                    arr[idx] = base - h
                    lm = loss(params)
                    arr[idx] = base
                    ests.append((lp - lm) / (2 * h))
                if abs(ests[0] - ests[1]) > 1e-6 * (abs(ests[0]) + 1e-6):
                    continue  # a decision flipped inside the step
                fd_all.append(ests[0])
                an_all.append(g[name][idx])
        fd_all, an_all = np.array(fd_all), np.array(an_all)
        assert len(fd_all) > 0.8 * len(live) * (arr.shape[1] if arr.ndim == 2 else 1)
        denom = max(np.linalg.norm(fd_all), 1e-12)
        assert np.linalg.norm(an_all - fd_all) / denom < 1e-6, name
        checked += len(fd_all)
    assert checked > 100


@pytest.mark.parametrize("deg,lowpass", [(3, 0.3), (0, 0.3), (1, 0.3), (2, 0.0)])
def test_project_backward_matches_central_differences(deg, lowpass):
    """The analytic projection gradient (means, scales, unnormalised
    quaternions, SH of every degree) equals central differences of the
    oracle's own forward projection for L = sum(wm * mean2d) + sum(wc * conic)
    + sum(wr * rgb), seen from an off-axis camera, with and without the 2D
    low-pass; a Gaussian whose colour channel is clamped at 0 passes no
    gradient through it."""
    n = 14
    sc = scenes.tiny_scene(12, n=n, width=80, height=64, sh_degree=deg, scale_lo=-2.5, scale_hi=-1.2)
    cam = scenes.look_at_camera((1.1, -0.6, -2.7), (0.05, 0.1, 0.0), 80, 64, lowpass=lowpass)
    rng = np.random.default_rng(5)
    means = sc.means.astype(np.float32).copy()
    scales = sc.scales.astype(np.float32).copy()
    quats = (sc.quats * rng.uniform(0.5, 2.0, (n, 1))).astype(np.float32)  # not unit length
    sh = sc.sh.astype(np.float32).copy()
    sh[0, 0, 1] = -4.0  # Gaussian 0's green channel is clamped
    base = oracle.project(means, scales, quats, sh, deg, cam)
    live = base["radius"] > 0
    assert live.sum() >= 10 and base["rgb"][0, 1] == 0.0
    wm, wc, wr = rng.standard_normal((n, 2)), rng.standard_normal((n, 3)), rng.standard_normal((n, 3))
    g = oracle.project_backward(means, scales, quats, sh, deg, cam, base["radius"], wm, wc, wr)

    def loss(args):
        o = oracle.project(*args, deg, cam)
        assert ((o["radius"] > 0) == live).all()
        return float((wm * o["mean2d"]).sum() + (wc * o["conic"]).sum() + (wr * o["rgb"]).sum())

    params = [means, scales, quats, sh]
    for k, (name, key) in enumerate((("means", "dmeans"), ("scales", "dscales"), ("quats", "dquats"),
                                     ("sh", "dsh"))):
        arr = params[k]
        fd, an = [], []
        for idx in np.ndindex(arr.shape):
            x = float(arr[idx])
            h = 1e-3 * max(abs(x), 0.05)
            xp, xm = np.float32(x + h), np.float32(x - h)
            arr[idx] = xp
            lp = loss(params)
            arr[idx] = xm
            lm = loss(params)
            arr[idx] = x
            fd.append((lp - lm) / (float(xp) - float(xm)))
            an.append(g[key][idx])
        fd, an = np.array(fd), np.array(an)
        scale = np.abs(an).max()
        assert scale > 0
        np.testing.assert_allclose(an, fd, rtol=2e-5, atol=2e-5 * scale, err_msg=name)
    assert not g["dmeans"][~live].any() and not g["dsh"][~live].any()
    assert (g["dsh"][0, :, 1] == 0).all() and np.abs(g["dsh"][0, :, 0]).max() > 0
    # the projection depends on q only through q / |q|: its gradient is orthogonal to q
    assert np.abs((g["dquats"] * quats).sum(1)).max() < 1e-9 * np.abs(g["dquats"]).max()


@pytest.mark.parametrize("seed,W,H,n,scales", [(0, 48, 40, 64, (-3.0, -1.5)), (3, 77, 45, 64, (-3.0, -1.5)),
                                                (7, 160, 128, 600, (-2.2, -0.6))])
def test_three_sigma_rectangle_bounds_what_it_drops(seed, W, H, n, scales):
    """Tile membership by the 3-sigma square (reading 9): at every pixel
    centre outside the tiles a splat is listed on, its alpha is at most
    o e^-4.5, because the square reaches ceil(3 sqrt(lambda_max)) pixels and
    the Mahalanobis distance beyond it is at least 3 (FP64, every splat and
    pixel).  The truncation this causes is reported: the brute-force image
    with and without the rectangle."""
    from gpu_common import report

    sc = scenes.tiny_scene(seed, n=n, width=W, height=H, scale_lo=scales[0], scale_hi=scales[1], opac_lo=0.3,
                           opac_hi=0.99)
    cam = sc.cameras[0]
    pr = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, 0, cam)
    d32 = pr["depth"].astype(np.float32)
    bs = oracle.bin_sort(pr["mean2d"], pr["radius"], d32, W, H)
    o = sc.opacities.astype(np.float64)
    ys, xs = np.mgrid[0:H, 0:W] + 0.5
    tile_of = (ys.astype(int) // 16) * cam.tiles_x + xs.astype(int) // 16
    listed = [set() for _ in range(sc.n)]
    for t in range(cam.num_tiles):
        for g in bs["ids"][bs["tile_ranges"][2 * t]:bs["tile_ranges"][2 * t + 1]]:
            listed[g].add(t)
    worst, worst_alpha, outside = 0.0, 0.0, 0
    for g in range(sc.n):
        if pr["radius"][g] <= 0:
            continue
        mask = ~np.isin(tile_of, list(listed[g]))
        A, B, C = pr["conic"][g]
        dx, dy = pr["mean2d"][g, 0] - xs[mask], pr["mean2d"][g, 1] - ys[mask]
        power = -0.5 * (A * dx * dx + 2 * B * dx * dy + C * dy * dy)
        if power.size:
            worst = max(worst, float((np.exp(power)).max()))
            worst_alpha = max(worst_alpha, float(o[g] * np.exp(power.max())))
            outside += int(power.size)
            assert power.max() <= -4.5 + 1e-9, (g, power.max())
    assert outside > 1000
    bg = (0.1, 0.2, 0.3)
    args = (pr["mean2d"], pr["conic"], o, pr["rgb"], pr["radius"], d32, W, H)
    rect = oracle.brute_force(*args, bg=bg, use_rect=True)
    full = oracle.brute_force(*args, bg=bg, use_rect=False)
    diff = np.abs(rect["image"] - full["image"])
    report(f"three_sigma_truncation_{W}x{H}", {"max_abs_image": float(diff.max()),
                                             "pixels_changed": float((diff.max(0) > 0).mean()),
                                             "max_exp_power_outside": worst, "max_alpha_outside": worst_alpha})
    if worst_alpha < 1 / 255:  # every dropped pair would be skipped: the rectangle changes nothing
        assert diff.max() == 0 and np.array_equal(rect["n_contrib"] > 0, full["n_contrib"] > 0)


def test_blend_grad_central_differences_at_1080p_clustered():
    """The analytic blend gradient at full scale (1920x1080, 1M clustered
    Gaussians, 11.4M instances): for 16 seeded visible Gaussians (non-zero
    analytic gradient, listed on at most 4 tiles), each of the 9 blend
    parameters is perturbed by h = 1e-4 max(1, |theta|) (1e-4 px for the
    mean, a position) and only the tiles the
    splat is listed on are re-rendered (the loss changes nowhere else).  A
    parameter is discarded when a decision flips inside the step (the two step
    sizes disagree, or n_contrib changes); the relative L2 error per group
    must stay below 1e-3 and is reported."""
    from gpu_common import report

    sc = scenes.make_config(2, seed=0)
    cam = sc.cameras[0]
    W, H = cam.width, cam.height
    pr = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, sc.sh_degree, cam)
    bs = oracle.bin_sort(pr["mean2d"], pr["radius"], pr["depth"].astype(np.float32), W, H)
    rng = np.random.default_rng(17)
    w = rng.standard_normal((3, H, W))
    bg = (0.1, 0.2, 0.3)
    p = dict(mean2d=np.ascontiguousarray(pr["mean2d"], np.float64), conic=np.ascontiguousarray(pr["conic"], np.float64),
             opacity=sc.opacities.astype(np.float64), rgb=np.ascontiguousarray(pr["rgb"], np.float64))
    ranges = bs["tile_ranges"]
    lens = ranges[1::2].astype(np.int64) - ranges[0::2]
    inst_tile = np.repeat(np.arange(cam.num_tiles), lens)
    g_an = oracle.blend_grad(W, H, ranges, bs["ids"], p["mean2d"], p["conic"], p["opacity"], p["rgb"], w, bg=bg,
                             n_threads=os.cpu_count() or 1)
    listed = np.bincount(bs["ids"], minlength=sc.n)
    visible = np.nonzero((g_an["opacity"] != 0) & (listed > 0) & (listed <= 4))[0]
    sample = rng.choice(visible, 16, replace=False)  # visible, and cheap to re-render
    chosen = np.zeros(sc.n, bool)
    chosen[sample] = True
    sel = chosen[bs["ids"]]
    tiles_of = {int(g): np.unique(inst_tile[sel & (bs["ids"] == g)]).astype(np.int32) for g in sample}

    def loss(tiles):
        r = oracle.blend(W, H, ranges, bs["ids"], p["mean2d"], p["conic"], p["opacity"], p["rgb"], bg=bg,
                         tile_subset=tiles)
        tx = tiles % cam.tiles_x
        ty = tiles // cam.tiles_x
        total, ncs = 0.0, []
        for x0, y0 in zip(16 * tx, 16 * ty):
            total += float(np.sum(w[:, y0:y0 + 16, x0:x0 + 16] * r["image"][:, y0:y0 + 16, x0:x0 + 16]))
            ncs.append(r["n_contrib"][y0:y0 + 16, x0:x0 + 16].copy())
        return total, ncs

    rel, discarded, nonzero = {}, 0, 0
    for name, arr in p.items():
        fd_all, an_all = [], []
        for g in sample:
            for j in range(arr.shape[1] if arr.ndim == 2 else 1):
                idx = (g, j) if arr.ndim == 2 else (g,)
                base = arr[idx]
                ests, flipped = [], False
                scale = 1.0 if name == "mean2d" else max(1.0, abs(base))  # a position: steps in pixels
                for h in (1e-4 * scale, 2.5e-5 * scale):
                    arr[idx] = base + h
                    lp, ncp = loss(tiles_of[int(g)])
                    arr[idx] = base - h
                    lm, ncm = loss(tiles_of[int(g)])
                    arr[idx] = base
                    ests.append((lp - lm) / (2 * h))
                    flipped |= any(not np.array_equal(a, b) for a, b in zip(ncp, ncm))
                if flipped or abs(ests[0] - ests[1]) > 1e-4 * (abs(ests[0]) + 1e-9):
                    discarded += 1
                    continue
                fd_all.append(ests[0])
                an_all.append(g_an[name][idx])
                nonzero += an_all[-1] != 0
        fd_all, an_all = np.array(fd_all), np.array(an_all)
        rel[name] = float(np.linalg.norm(an_all - fd_all) / max(np.linalg.norm(fd_all), 1e-30))
    report("blend_grad_fd_1080p_clustered", {"rel_l2": rel, "discarded": discarded, "checked_nonzero": int(nonzero)})
    assert discarded <= 0.2 * 16 * 9 and nonzero >= 100
    for name, e in rel.items():
        assert e < 1e-3, (name, e)


def test_bin_sort_tile_mask_gives_the_marked_tiles_lists():
    """oracle.bin_sort with a tile mask (used to sample large images): the
    marked tiles' lists equal the full call's, every other tile is empty."""
    sc = scenes.tiny_scene(3, n=300, width=96, height=80, sh_degree=0)
    cam = sc.cameras[0]
    pr = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, 0, cam)
    d32 = pr["depth"].astype(np.float32)
    for kw in ({}, {"conic": pr["conic"].astype(np.float32), "power_min": _power_min(sc.opacities)}):
        full = oracle.bin_sort(pr["mean2d"], pr["radius"], d32, 96, 80, **kw)
        mask = np.zeros(cam.num_tiles, bool)
        mask[[3, 7, 12, 29]] = True
        sub = oracle.bin_sort(pr["mean2d"], pr["radius"], d32, 96, 80, tile_mask=mask, **kw)
        assert 0 < sub["n_instances"] < full["n_instances"]
        for t in range(cam.num_tiles):
            a = full["ids"][full["tile_ranges"][2 * t]:full["tile_ranges"][2 * t + 1]]
            b = sub["ids"][sub["tile_ranges"][2 * t]:sub["tile_ranges"][2 * t + 1]]
            assert (list(a) == list(b)) if mask[t] else len(b) == 0
