"""PipelinedRenderer: frames whose uploads, compute and downloads overlap
give the results of rendering each frame on its own (image, T and counts bit
for bit; gradients up to the order of atomic additions)."""
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


def _host(sc):
    return {k: torch.from_numpy(np_).pin_memory() for k, np_ in
            (("means", sc.means), ("scales", sc.scales), ("quats", sc.quats), ("opacities", sc.opacities),
             ("sh", sc.sh))}


@pytest.mark.parametrize("graphs", [False, True])
def test_pipelined_frames_equal_separate_renders(graphs):
    a, b = scenes.make_config(0, seed=0), scenes.make_config(0, seed=1)
    cam = a.cameras[0]
    dL = torch.from_numpy(scenes.upstream_grad(0, [cam])[0]).cuda()
    opts = gs.make_opts("fp16_split", bg=(0.1, 0.2, 0.3))
    ha, hb = _host(a), _host(b)
    n = a.n
    pr = gs.PipelinedRenderer(ha, a.sh_degree, [cam], opts, 1 << 20, dL, graphs=graphs)

    def outs():
        return {"image": torch.empty(3, cam.height, cam.width).pin_memory(), "mean2d": torch.empty(n, 2).pin_memory(),
                "conic": torch.empty(n, 3).pin_memory(), "opacity": torch.empty(n).pin_memory(),
                "rgb": torch.empty(n, 3).pin_memory()}

    frames = [ha, hb, ha, hb, hb]
    res = [outs() for _ in frames]
    for k, h in enumerate(frames):
        pr.submit(k, h, res[k])
    for k in range(len(frames)):
        pr.wait(k)
    assert gs.gs_sync_status() == gs.GS_OK
    for sc, h in ((a, ha), (b, hb)):
        dev = gs.scene_to_device(sc)
        br = gs.BatchRenderer(dev, [cam], opts, 1 << 20)
        br.dL.copy_(dL.reshape(-1))
        br.step()
        torch.cuda.synchronize()
        want = {"image": br.image.view(3, cam.height, cam.width).cpu(), "mean2d": br.g_mean2d.cpu(),
                "conic": br.g_conic.cpu(), "opacity": br.g_opac.cpu(), "rgb": br.g_rgb.cpu()}
        for k, hk in enumerate(frames):
            if hk is not h:
                continue
            assert torch.equal(res[k]["image"], want["image"]), k
            for key in ("mean2d", "conic", "opacity", "rgb"):
                w = want[key].numpy()
                np.testing.assert_allclose(res[k][key].numpy(), w, rtol=1e-4, atol=1e-6 * np.abs(w).max())
