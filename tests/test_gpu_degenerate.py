"""Degenerate inputs of the newer entry points: every Gaussian culled, empty
tile lists, zero Gaussians.  Results are the defined ones (zero gradients,
background images, empty lists, a permutation as tile order) and no call
reports an error."""
import numpy as np
import pytest
import torch

from paper_2604_02120_gb300 import gs, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gs.load()


def _behind_camera(n=64):
    """A scene whose Gaussians all lie behind the camera (every one culled)."""
    sc = scenes.tiny_scene(2, n=n, width=40, height=24, sh_degree=1)
    sc.means[:, 2] = -5.0  # the camera sits at z = -3 looking towards +z
    return sc


def test_project_backward_all_culled_and_empty():
    sc = _behind_camera()
    cam = sc.cameras[0]
    dev = gs.scene_to_device(sc)
    proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
    assert int(proj["radius"].abs().sum()) == 0
    ones2, ones3 = torch.ones(sc.n, 2, device="cuda"), torch.ones(sc.n, 3, device="cuda")
    g = gs.project_backward(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam,
                            proj["radius"], ones2, ones3, ones3)
    assert gs.gs_sync_status() == gs.GS_OK
    for k, v in g.items():
        assert not v.any(), k
    # zero Gaussians: nothing to do, no error
    e = torch.empty(0, device="cuda")
    gs.gs_project_backward(0, e, e, e, e, 1, [cam], e, e, e, e, e, e, e, e)
    assert gs.gs_sync_status() == gs.GS_OK


def test_empty_lists_blend_to_the_background():
    """All tiles empty: the tile order is a permutation, the forward writes the
    background with T = 1 and n_contrib = 0 and issues no pair, and the
    backward gives zero gradients."""
    sc = _behind_camera()
    cam = sc.cameras[0]
    dev = gs.scene_to_device(sc)
    proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
    bs = gs.BinSorter("cuda", 1024).run(proj["mean2d"], proj["radius"], proj["depth"], cam.width, cam.height)
    assert bs["n_instances"] == 0
    order = gs.tile_order(bs["tile_ranges"], [cam.width], [cam.height])
    assert sorted(order.cpu().tolist()) == list(range(cam.num_tiles))
    bg = (0.25, 0.5, 0.75)
    for variant in ("fp32", "fp16_split"):
        issued = torch.zeros(1, device="cuda", dtype=torch.int64)
        o = gs.make_opts(variant, bg=bg, tile_order=order, issued_pairs=issued if variant != "fp32" else None)
        out = gs.blend_forward(cam.width, cam.height, bs, proj, dev["opacities"], o)
        assert gs.gs_sync_status() == gs.GS_OK
        for ch in range(3):
            assert torch.all(out["image"][ch] == bg[ch]), variant
        assert torch.all(out["T_final"] == 1.0) and not out["n_contrib"].any()
        assert int(issued.item()) == 0
        dL = torch.ones(3, cam.height, cam.width, device="cuda")
        g = gs.blend_backward(cam.width, cam.height, bs, proj, dev["opacities"], o, out, dL)
        assert gs.gs_sync_status() == gs.GS_OK
        for k, v in g.items():
            assert not v.any(), (variant, k)


def test_fused_small_all_culled():
    sc = _behind_camera()
    cam = sc.cameras[0]
    dev = gs.scene_to_device(sc)
    proj, bs = gs.project_bin_small(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam,
                                    max_per_tile=64)
    assert gs.gs_sync_status() == gs.GS_OK
    r = bs["tile_ranges"].cpu().numpy().view(np.uint32).reshape(-1, 2)
    assert (r[:, 1] == r[:, 0]).all()
    assert int(proj["radius"].abs().sum()) == 0
