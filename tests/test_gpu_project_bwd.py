"""Parity of gs_project_backward (the projection's gradient: EWA, quaternion
and scale, SH colour) with the FP64 oracle, through the C ABI.

Bars: relative L2 error of every gradient array below 1e-4 against the
oracle evaluated on the same float32 inputs and the same culling (the GPU's
radius); culled Gaussians get exact zeros; the sum over several views equals
the per-view oracle gradients summed; and the whole chain blend backward ->
projection backward matches the oracle chain within the FP32 blend's 1e-3.
Colour channels whose FP64 value lies within rounding of the clamp at 0 are
left out (the two sides may legitimately decide the clamp differently)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_02120_gb300 import gs, scenes

from gpu_common import CORES, report, to_np

pytestmark = pytest.mark.gpu

NAMES = (("dmeans", "means"), ("dscales", "scales"), ("dquats", "quats"), ("dsh", "sh"))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gs.load()


def _scene(kind):
    if kind == "256x256_10k":
        return scenes.make_config(0)
    if kind == "1280x720_200k":
        return scenes.make_config(1)
    if kind == "1920x1080_clustered_100k":
        return scenes.make_config(2, n=100_000)
    if kind == "tiny_ragged":
        return scenes.tiny_scene(3, n=96, width=77, height=45, sh_degree=2)
    if kind == "tiny_dense":
        return scenes.tiny_scene(8, n=600, width=64, height=48, sh_degree=3, scale_lo=-2.5, scale_hi=-1.2)
    raise KeyError(kind)


def _upstream(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((n, 2)).astype(np.float32), rng.standard_normal((n, 3)).astype(np.float32),
            rng.standard_normal((n, 3)).astype(np.float32))


def _clamp_ambiguous(sc, cam, rgb_gpu):
    """Gaussians with a colour channel within rounding of the clamp at 0."""
    ref = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, sc.sh_degree, cam)["rgb"]
    return (((ref > 0) & (ref < 1e-4)) | ((ref == 0) != (rgb_gpu == 0))).any(1)


def _rel_errors(g, ref, keep):
    out = {}
    for key, _ in NAMES:
        a = g[key].astype(np.float64)[keep].ravel()
        b = ref[key][keep].ravel()
        out[key] = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
    return out


@pytest.mark.parametrize("kind", ["256x256_10k", "tiny_ragged", "tiny_dense", "1920x1080_clustered_100k",
                                  "1280x720_200k"])
def test_project_backward_matches_oracle(kind):
    sc = _scene(kind)
    cam = sc.cameras[0]
    dev = gs.scene_to_device(sc)
    proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
    dm, dc, dr = _upstream(sc.n, 3)
    g = to_np(gs.project_backward(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam,
                                  proj["radius"], torch.from_numpy(dm).cuda(), torch.from_numpy(dc).cuda(),
                                  torch.from_numpy(dr).cuda()))
    assert gs.gs_sync_status() == gs.GS_OK
    pn = to_np(proj)
    ref = oracle.project_backward(sc.means, sc.scales, sc.quats, sc.sh, sc.sh_degree, cam, pn["radius"], dm, dc,
                                  dr)
    culled = pn["radius"] <= 0
    for key, _ in NAMES:
        assert not g[key][culled].any(), f"{key}: culled Gaussians got a gradient"
    amb = _clamp_ambiguous(sc, cam, pn["rgb"])
    keep = ~culled & ~amb
    assert keep.sum() > 0.3 * sc.n and amb.sum() <= max(3, 1e-3 * sc.n)
    rel = _rel_errors(g, ref, keep)
    report(f"project_bwd_rel_{kind}", rel)
    for key, e in rel.items():
        assert e < 1e-4, f"{key}: relative error {e:.2e}"


def test_project_backward_sums_over_views():
    """Three cameras in one call: the gradient is the sum of the per-view
    gradients (each view's upstream gradient and culling its own)."""
    sc = scenes.tiny_scene(8, n=600, width=64, height=48, sh_degree=3, scale_lo=-2.5, scale_hi=-1.2)
    cams = [scenes.look_at_camera(p, (0.0, 0.0, 0.0), w, h) for p, w, h in
            (((0, 0, -3), 64, 48), ((2.2, -0.4, -2.0), 80, 45), ((-1.5, 0.8, -2.6), 33, 50))]
    V, n = len(cams), sc.n
    dev = gs.scene_to_device(sc)
    f32 = dict(device="cuda", dtype=torch.float32)
    out = dict(mean2d=torch.empty(V, n, 2, **f32), conic=torch.empty(V, n, 3, **f32),
               depth=torch.empty(V, n, **f32), radius=torch.empty(V, n, device="cuda", dtype=torch.int32),
               rgb=torch.empty(V, n, 3, **f32), touched=torch.empty(V, n, device="cuda", dtype=torch.int32))
    gs.gs_project_views(n, dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cams,
                        out["mean2d"], out["conic"], out["depth"], out["radius"], out["rgb"], out["touched"])
    dm, dc, dr = _upstream(V * n, 4)
    g = to_np(gs.project_backward(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cams,
                                  out["radius"], torch.from_numpy(dm).cuda(), torch.from_numpy(dc).cuda(),
                                  torch.from_numpy(dr).cuda()))
    assert gs.gs_sync_status() == gs.GS_OK
    radius = out["radius"].cpu().numpy()
    rgb = out["rgb"].cpu().numpy()
    ref = {key: 0.0 for key, _ in NAMES}
    amb = np.zeros(n, bool)
    for v, cam in enumerate(cams):
        sl = slice(v * n, (v + 1) * n)
        r = oracle.project_backward(sc.means, sc.scales, sc.quats, sc.sh, sc.sh_degree, cam, radius[v], dm[sl],
                                    dc[sl], dr[sl])
        for key, _ in NAMES:
            ref[key] = ref[key] + r[key]
        amb |= _clamp_ambiguous(sc, cam, rgb[v])
    live = (radius > 0).any(0)
    assert ((radius > 0).sum(0) >= 2).sum() > 100  # many Gaussians seen by more than one view
    rel = _rel_errors(g, ref, live & ~amb)
    report("project_bwd_rel_three_views", rel)
    for key, e in rel.items():
        assert e < 1e-4, f"{key}: relative error {e:.2e}"


@pytest.mark.parametrize("variant", ["fp32", "fp16_split"])
def test_training_gradient_chain(variant):
    """dL/d(means, scales, quats, sh) of L = sum(w * image) through the whole
    path on the GPU (project, bin/sort, blend forward, blend backward,
    projection backward) against the oracle chain (FP64 blend gradient on
    the GPU's lists and FP32 splat parameters, then the FP64 projection
    gradient)."""
    sc = _scene("tiny_dense")
    cam = sc.cameras[0]
    dev = gs.scene_to_device(sc)
    proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
    bs = gs.BinSorter("cuda", 1 << 20).run(proj["mean2d"], proj["radius"], proj["depth"], cam.width, cam.height)
    bg = (0.2, 0.1, 0.05)
    opts = gs.make_opts(variant, bg=bg)
    fwd = gs.blend_forward(cam.width, cam.height, bs, proj, dev["opacities"], opts)
    w = np.random.default_rng(6).standard_normal((3, cam.height, cam.width)).astype(np.float32)
    gb = gs.blend_backward(cam.width, cam.height, bs, proj, dev["opacities"], opts, fwd, torch.from_numpy(w).cuda())
    g = to_np(gs.project_backward(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam,
                                  proj["radius"], gb["mean2d"], gb["conic"], gb["rgb"]))
    assert gs.gs_sync_status() == gs.GS_OK
    pn, bn = to_np(proj), to_np(bs)
    rb = oracle.blend_grad(cam.width, cam.height, bn["tile_ranges"].view(np.uint32), bn["ids"].view(np.uint32),
                           pn["mean2d"].astype(np.float64), pn["conic"].astype(np.float64),
                           sc.opacities.astype(np.float64), pn["rgb"].astype(np.float64), w.astype(np.float64),
                           bg=bg, n_threads=CORES)
    ref = oracle.project_backward(sc.means, sc.scales, sc.quats, sc.sh, sc.sh_degree, cam, pn["radius"],
                                  rb["mean2d"], rb["conic"], rb["rgb"])
    keep = (pn["radius"] > 0) & ~_clamp_ambiguous(sc, cam, pn["rgb"])
    rel = _rel_errors(g, ref, keep)
    report(f"training_grad_rel_{variant}", rel)
    for key, e in rel.items():
        assert e < 1e-3, f"{key}: relative error {e:.2e}"


def test_project_backward_rejects_unaligned_dmean2d():
    sc = _scene("tiny_ragged")
    dev = gs.scene_to_device(sc)
    cam = sc.cameras[0]
    proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
    buf = torch.zeros(2 * sc.n + 1, device="cuda")
    dc = torch.zeros(sc.n, 3, device="cuda")
    with pytest.raises(gs.GsError):
        gs.project_backward(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam,
                            proj["radius"], buf[1:], dc, dc)


def test_project_backward_sh1_without_lowpass():
    """SH degree 1 and a camera without the 2D low-pass, with splats small
    enough that some 2D covariances have an FP32 determinant below 1e-6 (the
    forward's and the backward's FP64 branch)."""
    sc = scenes.tiny_scene(14, n=400, width=70, height=52, sh_degree=1, scale_lo=-8.0, scale_hi=-3.0)
    cam = scenes.look_at_camera((0.4, -0.3, -2.8), (0.0, 0.0, 0.0), 70, 52, lowpass=0.0)
    dev = gs.scene_to_device(sc)
    proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
    pn = to_np(proj)
    ref_cov = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, sc.sh_degree, cam)["cov2d"]
    det = ref_cov[:, 0] * ref_cov[:, 2] - ref_cov[:, 1] ** 2
    fp64 = (det < 1e-6) & (pn["radius"] > 0)
    assert fp64.sum() > 0  # the FP64 branch runs
    # its forward outputs: the conic (inverse of the float32 2D covariance, taken
    # in FP64) within the float32 covariance's rounding times the inversion's
    # condition (|ac| + b^2) / det, the radius exact up to integer boundaries
    ref_fwd = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, sc.sh_degree, cam)
    a, b, c = ref_cov[fp64, 0], ref_cov[fp64, 1], ref_cov[fp64, 2]
    cond = (np.abs(a * c) + b * b) / np.abs(det[fp64])
    scale = np.abs(ref_fwd["conic"][fp64]).max(1)
    err = np.abs(pn["conic"][fp64] - ref_fwd["conic"][fp64]).max(1) / scale
    assert (err <= 8 * 2.0 ** -24 * cond + 1e-6).all(), f"FP64-branch conic error {err.max():.2e}"
    np.testing.assert_allclose(pn["mean2d"][fp64], ref_fwd["mean2d"][fp64], rtol=1e-5, atol=2e-4)
    r_ok = (pn["radius"][fp64] == ref_fwd["radius"][fp64]).mean()
    assert r_ok > 0.95, f"FP64-branch radius agreement {r_ok:.3f}"
    report("project_fp64_branch_forward", {"splats": int(fp64.sum()), "conic_rel_err_max": float(err.max()),
                                           "radius_equal": float(r_ok)})
    dm, dc, dr = _upstream(sc.n, 5)
    g = to_np(gs.project_backward(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam,
                                  proj["radius"], torch.from_numpy(dm).cuda(), torch.from_numpy(dc).cuda(),
                                  torch.from_numpy(dr).cuda()))
    assert gs.gs_sync_status() == gs.GS_OK
    ref = oracle.project_backward(sc.means, sc.scales, sc.quats, sc.sh, sc.sh_degree, cam, pn["radius"], dm, dc,
                                  dr)
    keep = (pn["radius"] > 0) & ~_clamp_ambiguous(sc, cam, pn["rgb"])
    rel = _rel_errors(g, ref, keep)
    report("project_bwd_rel_sh1_no_lowpass", rel)
    for key, e in rel.items():
        assert e < 1e-4, f"{key}: relative error {e:.2e}"
