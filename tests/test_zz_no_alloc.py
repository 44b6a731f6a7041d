"""gs_bin_sort_noalloc, the bin/sort entry point for callers that cannot
allocate device memory (its scratch is an array built into the library),
must give exactly what gs_bin_sort gives with a caller workspace.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
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


def _projected(scene):
    dev = gs.scene_to_device(scene)
    cam = scene.cameras[0]
    proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
    return cam, proj


def _with_workspace(cam, proj, capacity):
    n = proj["mean2d"].shape[0]
    ws = torch.empty(gs.gs_bin_sort_workspace_size(n, capacity, cam.width, cam.height) + 256, device="cuda",
                     dtype=torch.uint8)
    keys = torch.empty(capacity, device="cuda", dtype=torch.int64)
    ids = torch.empty(capacity, device="cuda", dtype=torch.int32)
    ranges = torch.empty(2 * cam.num_tiles, device="cuda", dtype=torch.int32)
    _, count = gs.gs_bin_sort(n, proj["mean2d"], proj["radius"], proj["depth"], cam.width, cam.height, capacity, ws,
                              keys, ids, ranges)
    return count, keys[:count].cpu().numpy(), ids[:count].cpu().numpy(), ranges.cpu().numpy()


def _no_alloc(cam, proj, capacity):
    n = proj["mean2d"].shape[0]
    keys = torch.empty(capacity, device="cuda", dtype=torch.int64)
    ids = torch.empty(capacity, device="cuda", dtype=torch.int32)
    ranges = torch.empty(2 * cam.num_tiles, device="cuda", dtype=torch.int32)
    _, count = gs.gs_bin_sort_noalloc(n, proj["mean2d"], proj["radius"], proj["depth"], cam.width, cam.height,
                                      capacity, keys, ids, ranges)
    assert gs.gs_sync_status() == gs.GS_OK
    return count, keys[:count].cpu().numpy(), ids[:count].cpu().numpy(), ranges.cpu().numpy()


@pytest.mark.parametrize("kind", ["tiny", "1280x720_200k"])
def test_no_alloc_bin_sort_matches_workspace_version_twice(kind):
    """Two calls in a row (the second reuses the built-in scratch the first
    left behind) agree bit for bit with gs_bin_sort; sorting is integer work,
    so the tolerance is exact equality."""
    scene = scenes.tiny_scene(5, n=300, width=93, height=61, sh_degree=1) if kind == "tiny" \
        else scenes.make_config(1)
    cam, proj = _projected(scene)
    capacity = 3_000_000 if kind == "1280x720_200k" else 20_000
    want = _with_workspace(cam, proj, capacity)
    assert want[0] > 0
    for _ in range(2):
        got = _no_alloc(cam, proj, capacity)
        assert got[0] == want[0]
        for a, b in zip(got[1:], want[1:]):
            np.testing.assert_array_equal(a, b)


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    cam, proj = _projected(scenes.tiny_scene(6, n=50, width=64, height=64))
    n = proj["mean2d"].shape[0]
    too_big = 8_000_000  # instance capacity whose scratch exceeds the built-in array
    assert gs.gs_bin_sort_workspace_size(n, too_big, cam.width, cam.height) > gs.gs_bin_sort_noalloc_max_bytes()
    keys = torch.empty(1, device="cuda", dtype=torch.int64)
    ids = torch.empty(1, device="cuda", dtype=torch.int32)
    ranges = torch.empty(2 * cam.num_tiles, device="cuda", dtype=torch.int32)
    st, _ = gs.gs_bin_sort_noalloc(n, proj["mean2d"], proj["radius"], proj["depth"], cam.width, cam.height, too_big,
                                   keys, ids, ranges, check=False)
    assert st == gs.GS_ERR_WORKSPACE
