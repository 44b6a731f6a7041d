"""Batched rendering of several views (cameras) in one pass: projection of all
views in one launch, one bin/sort over all views' tiles (also without host
synchronisation, for CUDA-graph capture), one persistent tensor-core blend
over the tiles of all views, the batched backward, a captured CUDA graph and
the autotuner.  Results must equal the single-view calls and the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_02120_gb300 import gs, scenes

from gpu_common import CORES, MAX_AMB_FP32, MAX_AMB_SPLIT, check_tight_lists, margins, to_np

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gs.load()


def _ring_scene(n=500, sizes=((80, 48), (61, 37), (96, 96), (33, 70)), seed=12):
    sc = scenes.tiny_scene(seed, n=n, width=64, height=64, sh_degree=1, scale_lo=-2.6, scale_hi=-1.4)
    sc.cameras = scenes.ring_cameras(len(sizes), 3.0, list(sizes))
    return sc


def _single(dev, cam, variant):
    proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
    bs = gs.BinSorter("cuda", 1 << 16).run(proj["mean2d"], proj["radius"], proj["depth"], cam.width, cam.height)
    out = gs.blend_forward(cam.width, cam.height, bs, proj, dev["opacities"], gs.make_opts(variant))
    return proj, bs, out


@pytest.mark.parametrize("variant", ["fp32", "fp16_split", "bf16"])
def test_batched_views_equal_single_view_calls(variant):
    sc = _ring_scene()
    dev = gs.scene_to_device(sc)
    br = gs.BatchRenderer(dev, sc.cameras, gs.make_opts(variant), capacity=1 << 17)
    br.forward()
    assert gs.gs_sync_status() == gs.GS_OK
    n = sc.n
    ranges_b = br.ranges.cpu().numpy().view(np.uint32)
    ids_b = br.ids.cpu().numpy().view(np.uint32)
    tile0 = 0
    for v, cam in enumerate(sc.cameras):
        proj, bs, out = _single(dev, cam, variant)
        for key in ("mean2d", "conic", "depth", "radius", "rgb"):
            torch.testing.assert_close(getattr(br, key)[v * n:(v + 1) * n], proj[key], rtol=0, atol=0)
        # per tile: the batched list is the single-view list with item ids offset by v * n
        r1 = bs["tile_ranges"].cpu().numpy().view(np.uint32)
        i1 = bs["ids"].cpu().numpy().view(np.uint32)
        for t in range(cam.num_tiles):
            a = ids_b[ranges_b[2 * (tile0 + t)]:ranges_b[2 * (tile0 + t) + 1]]
            b = i1[r1[2 * t]:r1[2 * t + 1]] + v * n
            np.testing.assert_array_equal(a, b)
        img, T, nc = br.view_image(v)
        torch.testing.assert_close(img, out["image"], rtol=0, atol=0)
        torch.testing.assert_close(T, out["T_final"], rtol=0, atol=0)
        torch.testing.assert_close(nc, out["n_contrib"], rtol=0, atol=0)
        tile0 += cam.num_tiles


def test_graph_mode_bin_sort_matches_synchronising_mode_and_reports_overflow():
    sc = _ring_scene()
    dev = gs.scene_to_device(sc)
    br = gs.BatchRenderer(dev, sc.cameras, gs.make_opts("fp32"), capacity=1 << 17)
    br.forward()
    count = int(br.count.item())
    keys = torch.empty(1 << 17, device="cuda", dtype=torch.int64)
    ids = torch.empty(1 << 17, device="cuda", dtype=torch.int32)
    ranges = torch.empty_like(br.ranges)
    st, c2 = gs.gs_bin_sort_views(br.V, br.n, br.mean2d, br.radius, br.depth, br.widths, br.heights, 1 << 17,
                                  br.workspace, keys, ids, ranges)
    assert st == gs.GS_OK and c2 == count > 0
    torch.testing.assert_close(ids[:count], br.ids[:count], rtol=0, atol=0)
    torch.testing.assert_close(ranges, br.ranges, rtol=0, atol=0)
    # graph mode with too small a capacity: count reported, error word set
    small = count // 2
    ws = torch.empty(gs.gs_bin_sort_workspace_size(br.V * br.n, small, 64, 64) + 256, device="cuda",
                     dtype=torch.uint8)
    cdev = torch.zeros(1, device="cuda", dtype=torch.int64)
    gs.gs_bin_sort_views(br.V, br.n, br.mean2d, br.radius, br.depth, br.widths, br.heights, small, ws, keys, ids,
                         ranges, count_dev=cdev)
    assert gs.gs_sync_status() == gs.GS_ERR_CAPACITY
    assert int(cdev.item()) == count
    assert gs.gs_sync_status() == gs.GS_OK


def test_graph_mode_capacity_over_2_28_gives_the_same_lists():
    """In graph mode the pair sort's grids and status words are sized by the
    capacity: with a capacity above 2^28 (and most pair-sort tiles empty) the
    lists equal those of a tight capacity, also on a reused workspace."""
    sc = _ring_scene()
    dev = gs.scene_to_device(sc)
    br = gs.BatchRenderer(dev, sc.cameras, gs.make_opts("fp32"), capacity=1 << 17)
    br.forward()
    count = int(br.count.item())
    big = (1 << 28) + 4096
    ws = torch.empty(gs.gs_bin_sort_workspace_size(br.V * br.n, big, 64, 64) + 256, device="cuda", dtype=torch.uint8)
    ids = torch.empty(big, device="cuda", dtype=torch.int32)
    ranges = torch.empty_like(br.ranges)
    cdev = torch.zeros(1, device="cuda", dtype=torch.int64)
    for _ in range(2):  # the second call finds the first one's status words in the workspace
        ranges.fill_(-1)
        gs.gs_bin_sort_views(br.V, br.n, br.mean2d, br.radius, br.depth, br.widths, br.heights, big, ws, None, ids,
                             ranges, count_dev=cdev)
        assert gs.gs_sync_status() == gs.GS_OK
        assert int(cdev.item()) == count > 0
        torch.testing.assert_close(ranges, br.ranges, rtol=0, atol=0)
        torch.testing.assert_close(ids[:count], br.ids[:count], rtol=0, atol=0)


@pytest.mark.parametrize("variant", ["fp32", "fp16_split"])
def test_batched_backward_equals_sum_over_views(variant):
    sc = _ring_scene(n=300)
    dev = gs.scene_to_device(sc)
    opts = gs.make_opts(variant, bg=(0.1, 0.2, 0.3))
    br = gs.BatchRenderer(dev, sc.cameras, opts, capacity=1 << 17)
    rng = np.random.default_rng(3)
    br.dL.copy_(torch.from_numpy(rng.standard_normal(3 * br.pixels).astype(np.float32)))
    br.step()
    assert gs.gs_sync_status() == gs.GS_OK
    n = sc.n
    g_opac = torch.zeros(n, device="cuda")
    off = 0
    for v, cam in enumerate(sc.cameras):
        proj, bs, out = _single(dev, cam, variant)
        P = cam.width * cam.height
        dL = br.dL[3 * off:3 * (off + P)].view(3, cam.height, cam.width)
        g = gs.blend_backward(cam.width, cam.height, bs, proj, dev["opacities"], opts, out, dL)
        torch.testing.assert_close(br.g_mean2d[v * n:(v + 1) * n], g["mean2d"], rtol=1e-4, atol=1e-5)
        torch.testing.assert_close(br.g_conic[v * n:(v + 1) * n], g["conic"], rtol=1e-4, atol=1e-5)
        torch.testing.assert_close(br.g_rgb[v * n:(v + 1) * n], g["rgb"], rtol=1e-4, atol=1e-5)
        g_opac += g["opacity"]
        off += P
    torch.testing.assert_close(br.g_opac, g_opac, rtol=1e-4, atol=1e-5)


def test_cuda_graph_replay_matches_eager_step():
    sc = _ring_scene()
    dev = gs.scene_to_device(sc)
    br = gs.BatchRenderer(dev, sc.cameras, gs.make_opts("fp16_split"), capacity=1 << 17)
    br.dL.normal_()
    br.step()
    torch.cuda.synchronize()
    want = [t.clone() for t in (br.image, br.T, br.nc, br.g_mean2d, br.g_opac)]
    graph = br.capture()
    for t in (br.image, br.T, br.g_mean2d):
        t.fill_(-1.0)
    graph.replay()
    torch.cuda.synchronize()
    assert gs.gs_sync_status() == gs.GS_OK
    got = (br.image, br.T, br.nc, br.g_mean2d, br.g_opac)
    for a, b in zip(got[:3], want[:3]):
        torch.testing.assert_close(a, b, rtol=0, atol=0)
    for a, b in zip(got[3:], want[3:]):  # atomics: summation order may differ
        torch.testing.assert_close(a, b, rtol=1e-5, atol=1e-6)


def test_autotune_picks_a_built_shape():
    sc = _ring_scene()
    dev = gs.scene_to_device(sc)
    br = gs.BatchRenderer(dev, sc.cameras, gs.make_opts("fp16_split"), capacity=1 << 17)
    br.forward()
    opts = gs.make_opts("fp16_split")
    ms = gs.gs_blend_autotune(br.widths, br.heights, br.n, br.ranges, br.ids, br.mean2d, br.conic,
                              dev["opacities"], br.rgb, opts, br.image, br.T, br.nc, reps=3)
    assert ms > 0
    assert (opts.chunk, opts.stages) in [(32, 2), (32, 4), (16, 4), (16, 6)]


@pytest.mark.parametrize("variant", ["fp16_split", "bf16_split", "fp8_split"])
def test_batched_views_tma_records_equal_loads(variant):
    """The batched forward over a mixed-resolution ring with the splat
    records packed after projection and staged by TMA gathers equals the
    per-thread-load producer bit for bit (items of several views, opacity
    indexed per Gaussian), as does the backward that follows."""
    sc = _ring_scene(n=800, sizes=((160, 120), (128, 72), (200, 112), (240, 135)))
    dev = gs.scene_to_device(sc)
    out = []
    for tma in (False, True):
        br = gs.BatchRenderer(dev, sc.cameras, gs.make_opts(variant, bg=(0.1, 0.2, 0.1)), capacity=1 << 19,
                              tma_records=tma)
        br.dL.copy_(torch.linspace(-1, 1, br.dL.numel(), device="cuda"))
        br.step()
        assert gs.gs_sync_status() == gs.GS_OK
        out.append((br.image.clone(), br.T.clone(), br.nc.clone()))
    for a, b in zip(*out):
        assert torch.equal(a, b)


@pytest.mark.parametrize("variant", ["fp32", "fp16_split"])
def test_batched_views_match_oracle(variant):
    """Mixed-resolution ring of views (a small stand-in for the 16-camera
    batch): every view against the FP64 oracle."""
    sc = _ring_scene(n=800, sizes=((160, 120), (128, 72), (200, 112), (240, 135)))
    dev = gs.scene_to_device(sc)
    br = gs.BatchRenderer(dev, sc.cameras, gs.make_opts(variant, bg=(0.1, 0.1, 0.1)), capacity=1 << 19)
    br.forward()
    assert gs.gs_sync_status() == gs.GS_OK
    n = sc.n
    ranges = br.ranges.cpu().numpy().view(np.uint32)
    ids = br.ids.cpu().numpy().view(np.uint32)
    m2 = br.mean2d.cpu().numpy().astype(np.float64)
    co = br.conic.cpu().numpy().astype(np.float64)
    rgb = br.rgb.cpu().numpy().astype(np.float64)
    tile0 = 0
    tol = 1e-4 if variant == "fp32" else 1e-3
    for v, cam in enumerate(sc.cameras):
        T = cam.num_tiles
        r = ranges[2 * tile0:2 * (tile0 + T)].astype(np.int64)
        # the oracle blends view v with its own local tile ranges; ids index all items
        ref = oracle.blend(cam.width, cam.height, r.astype(np.uint32), ids, m2, co,
                           np.tile(sc.opacities.astype(np.float64), len(sc.cameras)), rgb, bg=(0.1, 0.1, 0.1),
                           n_threads=CORES, **margins(variant))
        img, Tf, nc = (x.cpu().numpy() for x in br.view_image(v))
        ok = ~ref["ambiguous"]
        assert ref["ambiguous"].mean() <= (MAX_AMB_FP32 if variant == "fp32" else MAX_AMB_SPLIT)
        assert (np.abs(img - ref["image"])[:, ok] <= tol + ref["err_bound"][ok]).all()
        np.testing.assert_array_equal(nc[ok], ref["n_contrib"][ok])
        tile0 += T


def test_sixteen_camera_batch_full_size():
    """The 16-camera, 1.5M-Gaussian batch: the batched bin/sort (24M items,
    beyond the two-launch scan) equals the 16 single-view sorts, and the
    batched tensor-core blend equals the single-view blends, bit for bit."""
    sc = scenes.make_config(3)
    dev = gs.scene_to_device(sc)
    n = sc.n
    # capacity from the single views
    counts, singles = [], []
    for cam in sc.cameras:
        proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
        bs = gs.BinSorter("cuda", 1 << 23).run(proj["mean2d"], proj["radius"], proj["depth"], cam.width, cam.height)
        counts.append(bs["n_instances"])
        singles.append((bs["tile_ranges"].cpu().numpy().view(np.uint32), bs["ids"].cpu().numpy().view(np.uint32)))
        del proj, bs
    br = gs.BatchRenderer(dev, sc.cameras, gs.make_opts("fp16_split"), capacity=sum(counts) + 1024)
    br.forward()
    assert gs.gs_sync_status() == gs.GS_OK
    assert int(br.count.item()) == sum(counts)
    ranges = br.ranges.cpu().numpy().view(np.uint32)
    ids = br.ids.cpu().numpy().view(np.uint32)
    tile0 = 0
    for v, cam in enumerate(sc.cameras):
        r1, i1 = singles[v]
        T = cam.num_tiles
        rb = ranges[2 * tile0:2 * (tile0 + T)].astype(np.int64)
        shift = int(sum(counts[:v]))
        nonempty = rb[1::2] > rb[0::2]
        np.testing.assert_array_equal(nonempty, r1[1::2] > r1[0::2])
        np.testing.assert_array_equal(rb[0::2][nonempty] - shift, r1[0::2][nonempty].astype(np.int64))
        np.testing.assert_array_equal(rb[1::2][nonempty] - shift, r1[1::2][nonempty].astype(np.int64))
        np.testing.assert_array_equal(ids[shift:shift + counts[v]], i1 + v * n)
        tile0 += T
    # blend: view 5 through the single-view path, bit for bit
    v = 5
    cam = sc.cameras[v]
    proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
    bs = gs.BinSorter("cuda", 1 << 23).run(proj["mean2d"], proj["radius"], proj["depth"], cam.width, cam.height)
    out = gs.blend_forward(cam.width, cam.height, bs, proj, dev["opacities"], gs.make_opts("fp16_split"))
    img, Tf, nc = br.view_image(v)
    torch.testing.assert_close(img, out["image"], rtol=0, atol=0)
    torch.testing.assert_close(nc, out["n_contrib"], rtol=0, atol=0)


@pytest.mark.parametrize("tight", [False, True])
def test_bin_sort_views_three_tile_digit_passes_match_oracle_per_view(tight):
    """12 views of 4000 x 4000 pixels hold 750,000 tiles, so the tile-id sort
    takes three 8-bit passes; 250 tiles per row put rectangle rows across
    multiples of 256 tile ids, and rectangles of hundreds of tiles take the
    warp-cooperative paths.  Every view's lists (full, or opacity-aware) must
    equal the oracle's single-view bin/sort, shifted to the view's global tile
    and item range."""
    sizes = [(4000, 4000)] * 12
    sc = scenes.tiny_scene(21, n=300, width=64, height=64, sh_degree=0, scale_lo=-3.5, scale_hi=-2.5)
    sc.cameras = scenes.ring_cameras(len(sizes), 3.0, sizes)
    dev = gs.scene_to_device(sc)
    V, n = len(sizes), sc.n
    f32 = dict(device="cuda", dtype=torch.float32)
    out = dict(mean2d=torch.empty(V * n, 2, **f32), conic=torch.empty(V * n, 3, **f32),
               depth=torch.empty(V * n, **f32), radius=torch.empty(V * n, device="cuda", dtype=torch.int32),
               rgb=torch.empty(V * n, 3, **f32), touched=torch.empty(V * n, device="cuda", dtype=torch.int32))
    gs.gs_project_views(n, dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], sc.cameras,
                        out["mean2d"], out["conic"], out["depth"], out["radius"], out["rgb"], out["touched"])
    total_tiles = sum(gs.num_tiles(w, h) for w, h in sizes)
    assert total_tiles > 1 << 16
    capacity = int(out["touched"].sum().item()) + 1000
    ws = torch.empty(gs.gs_bin_sort_workspace_size(V * n, capacity, 64, 64) + 256, device="cuda", dtype=torch.uint8)
    keys = torch.empty(capacity, device="cuda", dtype=torch.int64)
    ids = torch.empty(capacity, device="cuda", dtype=torch.int32)
    ranges = torch.empty(2 * total_tiles, device="cuda", dtype=torch.int32)
    pmin = gs.alpha_power_min(dev["opacities"]) if tight else None
    _, count = gs.gs_bin_sort_views(V, n, out["mean2d"], out["radius"], out["depth"], [w for w, _ in sizes],
                                    [h for _, h in sizes], capacity, ws, keys, ids, ranges,
                                    conic=out["conic"] if tight else None, power_min=pmin)
    assert gs.gs_sync_status() == gs.GS_OK
    keys_np = keys[:count].cpu().numpy().view(np.uint64)
    ids_np = ids[:count].cpu().numpy().view(np.uint32)
    ranges_np = ranges.cpu().numpy().view(np.uint32)
    m2 = out["mean2d"].cpu().numpy()
    rad = out["radius"].cpu().numpy()
    dep = out["depth"].cpu().numpy()
    tile0, total = 0, 0
    for v, (w, h) in enumerate(sizes):
        sl = slice(v * n, (v + 1) * n)
        nt = gs.num_tiles(w, h)
        got_r = ranges_np[2 * tile0:2 * (tile0 + nt)].astype(np.int64).reshape(-1, 2)
        busy = got_r[:, 1] > got_r[:, 0]
        assert busy.any()
        lo, hi = int(got_r[busy, 0].min()), int(got_r[busy, 1].max())
        assert (got_r[~busy] == 0).all()
        # this view's lists, taken back to the view's own tile ids and Gaussian indices
        view = dict(tile_ranges=np.where(busy[:, None], got_r - lo, 0).astype(np.uint32).reshape(-1),
                    ids=(ids_np[lo:hi] - np.uint32(v * n)).astype(np.uint32),
                    keys=keys_np[lo:hi] - (np.uint64(tile0) << np.uint64(32)))
        full = oracle.bin_sort(m2[sl].astype(np.float64), rad[sl], dep[sl], w, h)
        if tight:  # the FP64 definition, up to pairs within rounding of the threshold
            ref = oracle.bin_sort(m2[sl].astype(np.float64), rad[sl], dep[sl], w, h,
                                  conic=out["conic"].cpu().numpy()[sl], power_min=pmin.cpu().numpy())
            check_tight_lists(view, ref, full)
        else:
            assert hi - lo == full["n_instances"]
            np.testing.assert_array_equal(view["ids"], full["ids"])
            np.testing.assert_array_equal(view["keys"], full["keys"])
            np.testing.assert_array_equal(view["tile_ranges"], full["tile_ranges"])
        tile0 += nt
        total += hi - lo
    assert total == count
