"""gs_tile_order (longest tile list first) and gs_blend_opts.tile_order.

The order is a permutation of the tile ids whose length buckets never
increase; blending in that order gives bit for bit the same image, T_final
and n_contrib as in id order (each tile is one block's work), and the same
gradients up to the order of the atomic additions; with sharding the shards
still cover every pixel once."""
import numpy as np
import pytest
import torch

from paper_2604_02120_gb300 import gs, scenes

from gpu_common import gpu_pipeline, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gs.load()


def _bucket(lens):
    lens = np.asarray(lens, np.int64)
    out = lens.copy()
    big = lens >= 4
    lg = np.floor(np.log2(np.maximum(lens, 1))).astype(np.int64)
    out[big] = 4 * lg[big] + ((lens[big] >> (lg[big] - 2)) & 3) - 4
    return out


@pytest.mark.parametrize("kind", ["256x256_10k", "1280x720_20k"])
def test_tile_order_is_longest_first_permutation(kind):
    sc = scenes.make_config(0) if kind == "256x256_10k" else scenes.make_config(1, n=20_000)
    dev, cam, proj, bs = gpu_pipeline(sc)
    order = gs.tile_order(bs["tile_ranges"], [cam.width], [cam.height]).cpu().numpy()
    assert gs.gs_sync_status() == gs.GS_OK
    r = bs["tile_ranges"].cpu().numpy().view(np.uint32).reshape(-1, 2).astype(np.int64)
    lens = r[:, 1] - r[:, 0]
    assert sorted(order.tolist()) == list(range(cam.num_tiles))
    b = _bucket(lens[order])
    assert (np.diff(b) <= 0).all()
    assert b[0] == _bucket([lens.max()])[0]  # the first tile is in the longest lists' bucket


@pytest.mark.parametrize("variant", ["fp32", "fp16_split"])
def test_ordered_blend_equals_id_order(variant):
    sc = scenes.make_config(1, n=20_000)
    dev, cam, proj, bs = gpu_pipeline(sc)
    order = gs.tile_order(bs["tile_ranges"], [cam.width], [cam.height])
    bg = (0.2, 0.1, 0.05)
    plain = gs.make_opts(variant, bg=bg)
    ordered = gs.make_opts(variant, bg=bg, tile_order=order)
    a = gs.blend_forward(cam.width, cam.height, bs, proj, dev["opacities"], plain)
    b = gs.blend_forward(cam.width, cam.height, bs, proj, dev["opacities"], ordered)
    for k in ("image", "T_final", "n_contrib"):
        assert torch.equal(a[k], b[k]), k
    dL = torch.randn(3, cam.height, cam.width, device="cuda", generator=torch.Generator("cuda").manual_seed(2))
    ga = to_np(gs.blend_backward(cam.width, cam.height, bs, proj, dev["opacities"], plain, a, dL))
    gb = to_np(gs.blend_backward(cam.width, cam.height, bs, proj, dev["opacities"], ordered, b, dL))
    assert gs.gs_sync_status() == gs.GS_OK
    for k in ga:
        np.testing.assert_allclose(gb[k], ga[k], rtol=1e-4, atol=1e-6 * np.abs(ga[k]).max())


def test_ordered_shards_cover_every_pixel_once():
    sc = scenes.make_config(0)
    dev, cam, proj, bs = gpu_pipeline(sc)
    order = gs.tile_order(bs["tile_ranges"], [cam.width], [cam.height])
    full = gs.blend_forward(cam.width, cam.height, bs, proj, dev["opacities"], gs.make_opts("fp16_split"))
    seen = torch.zeros(cam.height, cam.width, device="cuda", dtype=torch.int32)
    img = torch.zeros_like(full["image"])
    for k in range(3):
        o = gs.make_opts("fp16_split", shard_count=3, shard_index=k, tile_order=order)
        out = gs.blend_forward(cam.width, cam.height, bs, proj, dev["opacities"], o)
        touched = torch.zeros_like(seen)
        ordn = order.cpu().numpy()
        for p in range(k, cam.num_tiles, 3):
            t = int(ordn[p])
            ty, tx = divmod(t, cam.tiles_x)
            touched[16 * ty:16 * ty + 16, 16 * tx:16 * tx + 16] = 1
        seen += touched
        img += out["image"] * touched
    assert gs.gs_sync_status() == gs.GS_OK
    assert (seen == 1).all()
    assert torch.equal(img, full["image"])


def _opaque_wall(n=50):
    """One 16x16 tile covered by n large, nearly opaque splats: every pixel
    stops within three of them."""
    f = np.float32
    means = np.zeros((n, 3), f)
    means[:, 2] = np.linspace(-1.0, 0.5, n, dtype=f)  # distinct depths in front of nothing else
    scales = np.full((n, 3), 5.0, f)
    quats = np.tile(np.array([1, 0, 0, 0], f), (n, 1))
    opac = np.full(n, 0.99, f)
    sh = np.zeros((n, 1, 3), f)
    return scenes.Scene(means, scales, quats, opac, sh, 0, [scenes.look_at_camera((0, 0, -3), (0, 0, 0), 16, 16)])


def test_issued_pairs_counter():
    """gs_blend_opts.issued_pairs: the tensor-core forward's issued pairs lie
    between the evaluated pairs (sum of n_contrib) and 256 x the instances
    (three scenes, one where every pixel stops within three splats), and
    equal 256 x the instances when no pixel can stop early (opacities scaled
    down)."""
    dense = scenes.tiny_scene(8, n=600, width=64, height=48, sh_degree=3, scale_lo=-2.5, scale_hi=-1.2)
    for sc, scale in ((dense, 0.02), (scenes.make_config(0), 1.0), (_opaque_wall(), 1.0)):
        dev, cam, proj, bs = gpu_pipeline(sc)
        n_inst = int(bs["n_instances"])
        issued = torch.zeros(1, device="cuda", dtype=torch.int64)
        o = gs.make_opts("fp16_split", chunk=32, issued_pairs=issued)
        out = gs.blend_forward(cam.width, cam.height, bs, proj, (dev["opacities"] * scale).contiguous(), o)
        assert gs.gs_sync_status() == gs.GS_OK
        got = int(issued.item())
        evaluated = int(out["n_contrib"].sum().item())
        assert evaluated <= got <= 256 * n_inst
        if scale < 1.0:
            assert got == 256 * n_inst
        if sc.n == 50:  # the producer may issue the second chunk before the first reports every pixel stopped
            assert n_inst == 50 and (out["n_contrib"] <= 3).all()
