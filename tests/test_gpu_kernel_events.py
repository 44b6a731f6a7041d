"""gs_set_kernel_events through the C ABI: the events bracket the coarse
duplication of gs_bin_sort_views, both launched directly and replayed from a
captured CUDA graph, and clearing them stops the recording.  The lists are
the same with and without the events."""
import pytest
import torch

from paper_2604_02120_gb300 import gs, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gs.load()


def test_duplication_events_eager_and_in_graph():
    sc = scenes.make_config(1, n=20_000)
    cam = sc.cameras[0]
    dev = gs.scene_to_device(sc)
    proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
    n, W, H, cap = sc.n, cam.width, cam.height, 1 << 22
    ws = torch.empty(gs.gs_bin_sort_workspace_size(n, cap, W, H) + 256, dtype=torch.uint8, device="cuda")
    ids = torch.empty(cap, dtype=torch.int32, device="cuda")
    ranges = torch.empty(2 * cam.num_tiles, dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")

    def sort():
        gs.gs_bin_sort_views(1, n, proj["mean2d"], proj["radius"], proj["depth"], [W], [H], cap, ws, None, ids,
                             ranges, count_dev=count)

    sort()
    torch.cuda.synchronize()
    ref_ranges, ref_ids = ranges.clone(), ids[: int(count.item())].clone()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gs.set_kernel_events(gs.KERNEL_DUPLICATE, e0, e1)
    try:
        sort()
        torch.cuda.synchronize()
        eager_ms = e0.elapsed_time(e1)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            sort()
    finally:
        gs.set_kernel_events(gs.KERNEL_DUPLICATE, None, None)
    ranges.zero_()
    g.replay()
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1)
    assert gs.gs_sync_status() == gs.GS_OK
    assert 0 < eager_ms < 1000 and 0 < graph_ms < 1000
    assert torch.equal(ranges, ref_ranges) and torch.equal(ids[: int(count.item())], ref_ids)
    # cleared: a later call leaves the events where the graph replay put them
    e1.synchronize()
    sort()
    torch.cuda.synchronize()
    assert e0.elapsed_time(e1) == graph_ms
