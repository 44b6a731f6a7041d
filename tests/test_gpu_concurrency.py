"""Host threads using the library at the same time, each on its own stream.

Each persistent-blend launch takes its own tile-queue slot and the launch
shapes are computed once under a lock, so forwards launched from several
threads at once give images bit-identical to a single-threaded forward."""
import threading

import pytest
import torch

from paper_2604_02120_gb300 import gs, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gs.load()


@pytest.mark.parametrize("variant", ["fp16_split", "fp32"])
def test_concurrent_forwards_on_streams(variant):
    sc = scenes.make_config(0)  # 256x256, 10k Gaussians
    cam = sc.cameras[0]
    dev = gs.scene_to_device(sc)
    proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
    bs = gs.BinSorter("cuda", 1 << 20).run(proj["mean2d"], proj["radius"], proj["depth"], cam.width, cam.height)
    opts = gs.make_opts(variant, bg=(0.1, 0.2, 0.3))
    ref = gs.blend_forward(cam.width, cam.height, bs, proj, dev["opacities"], opts)
    threads, rounds = 4, 6
    streams = [torch.cuda.Stream() for _ in range(threads)]
    outs = [[{k: torch.empty_like(v) for k, v in ref.items()} for _ in range(rounds)] for _ in range(threads)]
    torch.cuda.synchronize()
    errors = []

    def work(t):
        try:
            for o in outs[t]:
                gs.gs_blend_forward(cam.width, cam.height, bs["tile_ranges"], bs["ids"], proj["mean2d"],
                                    proj["conic"], dev["opacities"], proj["rgb"], opts, o["image"], o["T_final"],
                                    o["n_contrib"], streams[t])
        except Exception as e:  # reported below, after every thread has joined
            errors.append(e)

    pool = [threading.Thread(target=work, args=(t,)) for t in range(threads)]
    for th in pool:
        th.start()
    for th in pool:
        th.join()
    torch.cuda.synchronize()
    assert not errors, errors
    assert gs.gs_sync_status() == gs.GS_OK
    for t in range(threads):
        for o in outs[t]:
            for k in ("image", "T_final", "n_contrib"):
                assert torch.equal(o[k], ref[k]), (t, k)
