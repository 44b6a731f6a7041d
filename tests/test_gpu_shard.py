"""Tile sharding (the multi-GPU partition) on one GPU: the shards of a blend
call, run one after the other, together give exactly the unsharded call —
every pixel from exactly one shard, and gradients that sum to the full
gradient (the sum the multi-GPU all-reduce forms)."""
import numpy as np
import pytest
import torch

from paper_2604_02120_gb300 import dist as gsdist
from paper_2604_02120_gb300 import gs, scenes

from gpu_common import gpu_pipeline, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gs.load()


@pytest.mark.parametrize("variant", ["fp32", "fp16_split"])
@pytest.mark.parametrize("world", [2, 3])
def test_sharded_blend_equals_full(variant, world):
    sc = scenes.tiny_scene(31, n=800, width=77, height=61, sh_degree=1, scale_lo=-3.0, scale_hi=-1.6)
    dev, cam, proj, bs = gpu_pipeline(sc)
    bg = (0.1, 0.2, 0.3)
    dL = torch.randn(3, cam.height, cam.width, device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    full_opts = gs.make_opts(variant, bg=bg)
    full = gs.blend_forward(cam.width, cam.height, bs, proj, dev["opacities"], full_opts)
    gfull = gs.blend_backward(cam.width, cam.height, bs, proj, dev["opacities"], full_opts, full, dL)
    tx = (cam.width + 15) // 16
    owner = np.zeros((cam.height, cam.width), np.int64) - 1
    gsum = {k: torch.zeros_like(v) for k, v in gfull.items()}
    img = np.zeros((3, cam.height, cam.width), np.float32)
    for r in range(world):
        fwd, g = gsdist.blend_step_sharded(cam.width, cam.height, bs, proj, dev["opacities"], variant, dL, r, world,
                                           bg=bg, reduce=False)
        f = to_np(fwd)
        for t in gsdist.shard_tiles(cam.num_tiles, r, world):
            y0, x0 = (t // tx) * 16, (t % tx) * 16
            sl = (slice(y0, y0 + 16), slice(x0, x0 + 16))
            assert (owner[sl] == -1).all()
            owner[sl] = r
            img[(slice(None),) + sl] = f["image"][(slice(None),) + sl]
            np.testing.assert_array_equal(f["T_final"][sl], to_np(full)["T_final"][sl])
            np.testing.assert_array_equal(f["n_contrib"][sl], to_np(full)["n_contrib"][sl])
        for k in gsum:
            gsum[k] += g[k]
    assert (owner >= 0).all()
    np.testing.assert_array_equal(img, to_np(full)["image"])
    for k in gsum:
        torch.testing.assert_close(gsum[k], gfull[k], rtol=1e-5, atol=1e-6)


def test_shard_option_is_validated():
    sc = scenes.tiny_scene(32, n=50, width=32, height=32)
    dev, cam, proj, bs = gpu_pipeline(sc)
    out = {k: torch.empty(s, device="cuda", dtype=d) for k, s, d in
           [("image", (3, 32, 32), torch.float32), ("T", (32, 32), torch.float32), ("nc", (32, 32), torch.int32)]}
    st = gs.load().gs_blend_forward(32, 32, gs._ptr(bs["tile_ranges"]), gs._ptr(bs["ids"]), gs._ptr(proj["mean2d"]),
                                    gs._ptr(proj["conic"]), gs._ptr(dev["opacities"]), gs._ptr(proj["rgb"]),
                                    gs.ctypes.byref(gs.make_opts("fp32", shard_count=2, shard_index=2)),
                                    gs._ptr(out["image"]), gs._ptr(out["T"]), gs._ptr(out["nc"]), None)
    assert st == gs.GS_ERR_INVALID_ARG
