"""Parity of gs_project_bin_small (projection + per-tile lists in one
cooperative launch, for small scenes) with gs_project + gs_bin_sort and with
the FP64 oracle's bin/sort, and of gs_render_small (the same launch with the
tensor-core blend of every tile) with gs_blend_forward and the FP64 oracle's
blend, through the C ABI.

Bars: projection outputs bit-identical to gs_project's; every tile's list
bit-identical to gs_bin_sort's (full rectangles and opacity-aware) and to the
oracle's; images blended from the fused lists bit-identical; the fused
render's image, T_final and n_contrib bit-identical to gs_blend_forward's
(fp16 split) on those lists and within the split variant's bar of the
oracle's (1e-3 plus its rounding bound; n_contrib exact off ambiguous
pixels); the backward takes its outputs as they are; a tile over
max_per_tile reports GS_ERR_CAPACITY."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_02120_gb300 import gs, scenes

from gpu_common import MAX_AMB_SPLIT, check_tight_lists, compare_to_oracle, oracle_blend_on_gpu_params, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gs.load()


def _scene(kind):
    if kind == "256x256_10k":
        return scenes.make_config(0)
    if kind == "1280x720_10k_sh3":
        return scenes.make_config(1, n=10_000)
    if kind == "tiny_ragged":
        return scenes.tiny_scene(3, n=96, width=77, height=45, sh_degree=2)
    if kind == "tiny_dense":
        return scenes.tiny_scene(8, n=600, width=64, height=48, sh_degree=3, scale_lo=-2.5, scale_hi=-1.2)
    raise KeyError(kind)


def _tile_lists(ranges, ids):
    r = ranges.view(np.uint32).reshape(-1, 2)
    return [ids[a:b].view(np.uint32).tolist() for a, b in r]


@pytest.mark.parametrize("tight", [False, True])
@pytest.mark.parametrize("kind", ["256x256_10k", "1280x720_10k_sh3", "tiny_ragged", "tiny_dense"])
def test_fused_lists_equal_bin_sort(kind, tight):
    sc = _scene(kind)
    cam = sc.cameras[0]
    dev = gs.scene_to_device(sc)
    pmin = gs.alpha_power_min(dev["opacities"]) if tight else None
    fproj, fbs = gs.project_bin_small(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam,
                                      max_per_tile=2048, power_min=pmin)
    assert gs.gs_sync_status() == gs.GS_OK
    proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
    for k in ("mean2d", "conic", "depth", "radius", "rgb", "tiles_touched"):
        assert torch.equal(fproj[k], proj[k]), k
    n = sc.n
    if tight:
        cap = 1 << 22
        ws = torch.empty(gs.gs_bin_sort_workspace_size(n, cap, cam.width, cam.height) + 256, device="cuda",
                         dtype=torch.uint8)
        keys = torch.empty(cap, device="cuda", dtype=torch.int64)
        ids = torch.empty(cap, device="cuda", dtype=torch.int32)
        ranges = torch.empty(2 * cam.num_tiles, device="cuda", dtype=torch.int32)
        _, count = gs.gs_bin_sort_views(1, n, proj["mean2d"], proj["radius"], proj["depth"], [cam.width],
                                        [cam.height], cap, ws, keys, ids, ranges, conic=proj["conic"],
                                        power_min=pmin)
        bs = dict(tile_ranges=ranges, ids=ids[:count])
    else:
        bs = gs.BinSorter("cuda", 1 << 20).run(proj["mean2d"], proj["radius"], proj["depth"], cam.width, cam.height)
    assert gs.gs_sync_status() == gs.GS_OK
    got = _tile_lists(fbs["tile_ranges"].cpu().numpy(), fbs["ids"].cpu().numpy())
    want = _tile_lists(bs["tile_ranges"].cpu().numpy(), bs["ids"].cpu().numpy())
    assert got == want
    pn = to_np(proj)
    full = oracle.bin_sort(pn["mean2d"].astype(np.float64), pn["radius"], pn["depth"], cam.width, cam.height)
    if tight:  # the FP64 definition, up to pairs within rounding of the threshold
        ref = oracle.bin_sort(pn["mean2d"].astype(np.float64), pn["radius"], pn["depth"], cam.width, cam.height,
                              conic=pn["conic"], power_min=pmin.cpu().numpy())
        check_tight_lists(to_np(bs), ref, full)
    else:
        assert got == _tile_lists(full["tile_ranges"], full["ids"])
    assert sum(len(x) for x in got) > 0
    # the blend takes the fused lists as they are
    opts = gs.make_opts("fp16_split", bg=(0.1, 0.2, 0.3))
    a = gs.blend_forward(cam.width, cam.height, bs, proj, dev["opacities"], opts)
    b = gs.blend_forward(cam.width, cam.height, fbs, fproj, dev["opacities"], opts)
    assert gs.gs_sync_status() == gs.GS_OK
    for k in ("image", "T_final", "n_contrib"):
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("tight", [False, True])
@pytest.mark.parametrize("kind", ["256x256_10k", "1280x720_10k_sh3", "tiny_ragged", "tiny_dense"])
def test_fused_render_equals_blend_forward_and_oracle(kind, tight):
    sc = _scene(kind)
    cam = sc.cameras[0]
    dev = gs.scene_to_device(sc)
    pmin = gs.alpha_power_min(dev["opacities"]) if tight else None
    bg = (0.1, 0.2, 0.3)
    rproj, rbs, rfwd = gs.render_small(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"],
                                       dev["opacities"], cam, bg=bg, max_per_tile=2048, power_min=pmin)
    assert gs.gs_sync_status() == gs.GS_OK
    # projection and lists as gs_project_bin_small's
    fproj, fbs = gs.project_bin_small(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam,
                                      max_per_tile=2048, power_min=pmin)
    assert gs.gs_sync_status() == gs.GS_OK
    for k in fproj:
        assert torch.equal(rproj[k], fproj[k]), k
    assert _tile_lists(rbs["tile_ranges"].cpu().numpy(), rbs["ids"].cpu().numpy()) == \
        _tile_lists(fbs["tile_ranges"].cpu().numpy(), fbs["ids"].cpu().numpy())
    # the blend of the same lists by the persistent tensor-core kernel, every built shape
    for chunk, stages in ((32, 2), (16, 4), (0, 0)):
        opts = gs.make_opts("fp16_split", bg=bg, chunk=chunk, stages=stages)
        ref = gs.blend_forward(cam.width, cam.height, fbs, fproj, dev["opacities"], opts)
        assert gs.gs_sync_status() == gs.GS_OK
        for k in ("image", "T_final", "n_contrib"):
            assert torch.equal(rfwd[k], ref[k]), (k, chunk, stages)
    # the FP64 oracle's blend over the same lists and float32 splat parameters
    pn, bn = to_np(rproj), to_np(rbs)
    want = oracle_blend_on_gpu_params(cam, pn, bn, sc.opacities, bg=bg, variant="fp16_split")
    compare_to_oracle(to_np(rfwd), want, 1e-3, nc_exact=True, max_amb=MAX_AMB_SPLIT)
    assert (rfwd["n_contrib"] > 0).float().mean() > 0.05
    # the backward takes the fused outputs as they are
    dL = torch.from_numpy(scenes.upstream_grad(1, [cam])[0]).cuda()
    opts = gs.make_opts("fp16_split", bg=bg)
    g1 = gs.blend_backward(cam.width, cam.height, rbs, rproj, dev["opacities"], opts, rfwd, dL)
    fwd2 = gs.blend_forward(cam.width, cam.height, fbs, fproj, dev["opacities"], opts)
    g2 = gs.blend_backward(cam.width, cam.height, fbs, fproj, dev["opacities"], opts, fwd2, dL)
    assert gs.gs_sync_status() == gs.GS_OK
    for k in g1:  # atomics add in any order: equal up to the order of the sums
        rel = ((g1[k] - g2[k]).norm() / g2[k].norm().clamp_min(1e-30)).item()
        assert rel < 1e-5, (k, rel)


def test_fused_render_capacity_and_arguments():
    sc = _scene("tiny_dense")
    cam = sc.cameras[0]
    dev = gs.scene_to_device(sc)
    assert gs.gs_sync_status() == gs.GS_OK
    gs.render_small(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], dev["opacities"], cam,
                    max_per_tile=4)
    assert gs.gs_sync_status() == gs.GS_ERR_CAPACITY
    assert gs.gs_sync_status() == gs.GS_OK
    for mpt in (0, gs.SMALL_MAX_PER_TILE + 1):
        with pytest.raises(gs.GsError):
            gs.render_small(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], dev["opacities"],
                            cam, max_per_tile=mpt)


def test_fused_capacity_overflow_reports():
    sc = _scene("tiny_dense")
    cam = sc.cameras[0]
    dev = gs.scene_to_device(sc)
    assert gs.gs_sync_status() == gs.GS_OK
    gs.project_bin_small(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam,
                         max_per_tile=4)
    assert gs.gs_sync_status() == gs.GS_ERR_CAPACITY
    assert gs.gs_sync_status() == gs.GS_OK


def test_fused_rejects_bad_arguments():
    sc = _scene("tiny_ragged")
    cam = sc.cameras[0]
    dev = gs.scene_to_device(sc)
    for mpt in (0, gs.SMALL_MAX_PER_TILE + 1):
        with pytest.raises(gs.GsError):
            gs.project_bin_small(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam,
                                 max_per_tile=mpt)
