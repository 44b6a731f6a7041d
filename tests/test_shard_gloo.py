"""The multi-GPU backward's host logic on CPU ranks (gloo, world size 2):
each rank computes the gradient of its tile shard (the partition the
kernels use) with the FP64 oracle, the ranks all-reduce, and the result must
equal the single-process gradient over all tiles."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2604_02120_gb300 import dist as gsdist
from paper_2604_02120_gb300 import scenes


def _scene_inputs():
    sc = scenes.tiny_scene(41, n=400, width=70, height=50, sh_degree=1, scale_lo=-3.0, scale_hi=-1.8)
    cam = sc.cameras[0]
    pr = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, sc.sh_degree, cam)
    bs = oracle.bin_sort(pr["mean2d"], pr["radius"], pr["depth"].astype(np.float32), cam.width, cam.height)
    dL = np.random.default_rng(3).standard_normal((3, cam.height, cam.width))
    return sc, cam, pr, bs, dL


def _grad(cam, pr, bs, sc, dL, tiles=None):
    return oracle.blend_grad(cam.width, cam.height, bs["tile_ranges"], bs["ids"], pr["mean2d"], pr["conic"],
                             sc.opacities.astype(np.float64), pr["rgb"], dL, bg=(0.1, 0.2, 0.3), n_threads=2,
                             tile_subset=tiles)


def _rank(rank, world, port, out_path):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc, cam, pr, bs, dL = _scene_inputs()
        tiles = np.asarray(gsdist.shard_tiles(cam.num_tiles, rank, world), np.int32)
        g = {k: torch.from_numpy(np.ascontiguousarray(v)) for k, v in _grad(cam, pr, bs, sc, dL, tiles).items()}
        gsdist.allreduce_gradients(g)
        if rank == 0:
            np.savez(out_path, **{k: v.numpy() for k, v in g.items()})
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_gradient_allreduce_equals_full_gradient(tmp_path):
    out = str(tmp_path / "g.npz")
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    sc, cam, pr, bs, dL = _scene_inputs()
    want = _grad(cam, pr, bs, sc, dL)
    for k in ("mean2d", "conic", "opacity", "rgb"):
        assert np.abs(want[k]).max() > 0
        np.testing.assert_allclose(got[k], want[k], rtol=1e-12, atol=1e-12 * np.abs(want[k]).max())


def test_shard_tiles_partition():
    for world in (1, 2, 3, 5):
        seen = sorted(t for r in range(world) for t in gsdist.shard_tiles(23, r, world))
        assert seen == list(range(23))
    with pytest.raises(ValueError):
        gsdist.shard_tiles(10, 2, 2)
