"""Host-side argument checks of the C ABI, on a machine without a GPU: every
malformed call below returns its status before any CUDA call, and
gs_last_error names the entry point.

The calls pass made-up device addresses (never dereferenced by the host), so
this module runs only where no GPU is visible: there a call that wrongly
passed its checks could only fail in the CUDA runtime, never reach a kernel."""
import ctypes

import pytest
import torch

from paper_2604_02120_gb300 import build, gs

pytestmark = pytest.mark.skipif(torch.cuda.is_available(), reason="made-up device addresses: CPU-only machine")

INVALID, WORKSPACE = gs.GS_ERR_INVALID_ARG, 6
P = ctypes.c_void_p(1 << 20)      # an aligned made-up device address
ODD = ctypes.c_void_p((1 << 20) + 4)  # 4-byte aligned only
I32P = ctypes.POINTER(ctypes.c_int32)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return gs.load()


def _cam(w=64, h=48):
    c = gs.gs_camera()
    c.width, c.height, c.fx, c.fy, c.cx, c.cy, c.znear = w, h, 50.0, 50.0, w / 2, h / 2, 0.2
    for i in range(3):
        c.world_to_cam[4 * i + i] = 1.0
    return c


def _sizes(*vals):
    return (ctypes.c_int32 * len(vals))(*vals)


def _expect(lib, st, want, name):
    assert st == want, (name, st, lib.gs_last_error())
    assert name.encode() in lib.gs_last_error(), lib.gs_last_error()


def test_project_checks(lib):
    cam = _cam()
    out = [P] * 6
    _expect(lib, lib.gs_project(-1, P, P, P, P, 0, ctypes.byref(cam), *out, None), INVALID, "gs_project")
    _expect(lib, lib.gs_project(10, P, P, P, P, 4, ctypes.byref(cam), *out, None), INVALID, "gs_project")
    _expect(lib, lib.gs_project(10, P, P, P, P, 0, None, *out, None), INVALID, "gs_project")
    _expect(lib, lib.gs_project(10, None, P, P, P, 0, ctypes.byref(cam), *out, None), INVALID, "gs_project")
    _expect(lib, lib.gs_project(10, P, P, P, P, 0, ctypes.byref(_cam(0, 48)), *out, None), INVALID, "gs_project")
    _expect(lib, lib.gs_project_views(10, P, P, P, P, 0, ctypes.byref(cam), 0, *out, None), INVALID, "gs_project")
    _expect(lib, lib.gs_project_views(10, P, P, P, P, 0, ctypes.byref(cam), 33, *out, None), INVALID, "gs_project")


def test_project_backward_checks(lib):
    cam = _cam()
    args = [P] * 4 + [0, ctypes.byref(cam), 1]
    grads = [P] * 4
    _expect(lib, lib.gs_project_backward(-1, P, P, P, P, 0, ctypes.byref(cam), 1, P, P, P, P, *grads, None),
            INVALID, "gs_project_backward")
    _expect(lib, lib.gs_project_backward(10, *args, P, ODD, P, P, *grads, None), INVALID, "gs_project_backward")
    _expect(lib, lib.gs_project_backward(10, *args, P, P, P, None, *grads, None), INVALID, "gs_project_backward")


def test_project_bin_small_checks(lib):
    cam = _cam()
    out = [P] * 8
    for n, mpt in ((10, 0), (10, gs.SMALL_MAX_PER_TILE + 1), (0, 16)):
        _expect(lib, lib.gs_project_bin_small(n, P, P, P, P, 0, ctypes.byref(cam), None, mpt, *out, None), INVALID,
                "gs_project_bin_small")
    _expect(lib, lib.gs_project_bin_small(10, P, P, P, P, 0, ctypes.byref(cam), None, 16, ODD, *out[1:], None),
            INVALID, "gs_project_bin_small")


def test_render_small_checks(lib):
    cam = _cam()
    bg = (ctypes.c_float * 3)(0.0, 0.0, 0.0)
    proj = [P] * 8  # mean2d .. tile_ranges
    img = [P] * 3   # image, T_final, n_contrib
    for n, mpt in ((10, 0), (10, gs.SMALL_MAX_PER_TILE + 1), (0, 16)):
        _expect(lib, lib.gs_render_small(n, P, P, P, P, 0, ctypes.byref(cam), None, mpt, P, bg, *proj, *img, None),
                INVALID, "gs_render_small")
    _expect(lib, lib.gs_render_small(10, P, P, P, P, 0, ctypes.byref(cam), None, 16, P, bg, ODD, *proj[1:], *img,
                                     None), INVALID, "gs_render_small")
    _expect(lib, lib.gs_render_small(10, P, P, P, P, 0, ctypes.byref(cam), None, 16, None, bg, *proj, *img, None),
            INVALID, "gs_render_small")
    _expect(lib, lib.gs_render_small(10, P, P, P, P, 0, ctypes.byref(cam), None, 16, P, bg, *proj, P, P, None, None),
            INVALID, "gs_render_small")


def test_set_kernel_events_checks(lib):
    _expect(lib, lib.gs_set_kernel_events(0, None, None), INVALID, "gs_set_kernel_events")
    _expect(lib, lib.gs_set_kernel_events(gs.KERNEL_DUPLICATE, P, None), INVALID, "gs_set_kernel_events")
    assert lib.gs_set_kernel_events(gs.KERNEL_DUPLICATE, None, None) == gs.GS_OK


def test_bin_sort_checks(lib):
    w, h = _sizes(64), _sizes(48)
    cnt = ctypes.c_int64(0)
    need = ctypes.c_size_t(0)
    assert lib.gs_bin_sort_workspace_size(100, 1000, 64, 48, ctypes.byref(need)) == gs.GS_OK

    def views(n_views=1, n=100, conic=None, pmin=None, cap=1000, ws=P, ws_bytes=None, ninst=ctypes.byref(cnt),
              ids=P):
        return lib.gs_bin_sort_views(n_views, n, P, P, P, conic, pmin, w, h, cap, ws,
                                     need.value if ws_bytes is None else ws_bytes, None, ids, P, ninst, None, None)

    _expect(lib, views(n_views=0), INVALID, "gs_bin_sort")
    _expect(lib, views(n=-1), INVALID, "gs_bin_sort")
    _expect(lib, views(cap=1 << 32), INVALID, "gs_bin_sort")
    _expect(lib, views(conic=P), INVALID, "gs_bin_sort")  # conic without power_min
    _expect(lib, views(ninst=None), INVALID, "gs_bin_sort")  # neither a host nor a device count
    _expect(lib, views(ids=None), INVALID, "gs_bin_sort")
    _expect(lib, views(ws=ctypes.c_void_p((1 << 20) + 64)), INVALID, "gs_bin_sort")  # workspace alignment
    _expect(lib, views(ws_bytes=need.value - 1), WORKSPACE, "gs_bin_sort")
    _expect(lib, lib.gs_bin_sort(100, P, P, P, 64, 48, 1000, P, need.value, None, P, P, None, None), INVALID,
            "gs_bin_sort")


def test_blend_checks(lib):
    w, h = _sizes(64), _sizes(48)
    opts = gs.make_opts("fp16_split")
    fwd_out = [P] * 3

    def fwd(n_views=1, ranges=P, o=opts):
        return lib.gs_blend_forward_views(n_views, w, h, 0, ranges, P, P, P, P, P, ctypes.byref(o), *fwd_out, None)

    _expect(lib, fwd(n_views=0), INVALID, "gs_blend_forward")
    _expect(lib, fwd(ranges=None), INVALID, "null input pointer")
    bad_shard = gs.make_opts("fp16_split", shard_count=2, shard_index=2)
    _expect(lib, fwd(o=bad_shard), INVALID, "gs_blend_forward")
    bad_size = _sizes(1 << 21)
    _expect(lib, lib.gs_blend_forward_views(1, bad_size, h, 0, P, P, P, P, P, P, ctypes.byref(opts), *fwd_out, None),
            INVALID, "gs_blend_forward")
    unknown = gs.make_opts("fp32")
    unknown.variant = 99
    _expect(lib, lib.gs_blend_backward_views(1, w, h, 0, P, P, P, P, P, P, ctypes.byref(unknown), P, P, P, P, P, P, P,
                                             None), INVALID, "gs_blend_backward")
    _expect(lib, lib.gs_blend_backward_views(1, w, h, 0, P, P, P, P, P, P, ctypes.byref(opts), P, P, None, P, P, P,
                                             P, None), INVALID, "gs_blend_backward")
    best = ctypes.c_float(0)
    for o, reps in ((gs.make_opts("fp32"), 3), (gs.make_opts("fp16_split"), 0)):
        _expect(lib, lib.gs_blend_autotune(1, w, h, 0, P, P, P, P, P, P, ctypes.byref(o), P, P, P, reps,
                                           ctypes.byref(best), None), INVALID, "gs_blend_autotune")


def test_small_entry_point_checks(lib):
    _expect(lib, lib.gs_tile_order(0, _sizes(64), _sizes(48), P, P, None), INVALID, "gs_tile_order")
    _expect(lib, lib.gs_tile_order(1, _sizes(64), _sizes(48), None, P, None), INVALID, "gs_tile_order")
    _expect(lib, lib.gs_alpha_power_min(-1, P, P, None), INVALID, "gs_alpha_power_min")
    _expect(lib, lib.gs_alpha_power_min(10, None, P, None), INVALID, "gs_alpha_power_min")
    _expect(lib, lib.gs_selftest_bounded_wait(-1, None), INVALID, "gs_selftest_bounded_wait")


def test_bin_sort_noalloc_checks(lib):
    """The allocation-free bin/sort rejects what gs_bin_sort rejects, before
    any CUDA call: sizes beyond 2^20 per side, images of 2^31 tiles or more
    (where tiles_x * tiles_y would overflow an int), null pointers, and
    sizes whose scratch exceeds the built-in array."""
    cnt = ctypes.c_int64(0)

    def call(n=100, w=64, h=48, cap=1000, m=P, ids=P, ranges=P, ninst=ctypes.byref(cnt)):
        return lib.gs_bin_sort_noalloc(n, m, P, P, w, h, cap, None, ids, ranges, ninst, None)

    _expect(lib, call(n=-1), INVALID, "gs_bin_sort_noalloc")
    _expect(lib, call(w=0), INVALID, "gs_bin_sort_noalloc")
    _expect(lib, call(h=(1 << 20) + 1), INVALID, "gs_bin_sort_noalloc")
    _expect(lib, call(w=1 << 20, h=1 << 19), INVALID, "gs_bin_sort_noalloc")  # 2^31 tiles
    _expect(lib, call(w=1 << 20, h=1 << 20), INVALID, "gs_bin_sort_noalloc")  # 2^32 tiles
    _expect(lib, call(cap=1 << 32), INVALID, "gs_bin_sort_noalloc")
    _expect(lib, call(m=None), INVALID, "gs_bin_sort_noalloc")
    _expect(lib, call(ids=None), INVALID, "gs_bin_sort_noalloc")
    _expect(lib, call(ranges=None), INVALID, "gs_bin_sort_noalloc")
    _expect(lib, call(ninst=None), INVALID, "gs_bin_sort_noalloc")
    _expect(lib, call(n=1 << 24, cap=1 << 28), WORKSPACE, "gs_bin_sort_noalloc")
    # a successful check leaves no earlier message behind: the size query succeeds and clears it
    need = ctypes.c_size_t(0)
    assert lib.gs_bin_sort_workspace_size(100, 1000, 64, 48, ctypes.byref(need)) == gs.GS_OK
    assert lib.gs_last_error() == b""
    assert lib.gs_bin_sort_workspace_size(100, 1000, 1 << 20, 1 << 20, ctypes.byref(need)) == INVALID


def test_pack_splats_and_record_option_checks(lib):
    """gs_pack_splats rejects bad sizes and misaligned buffers; a blend call
    whose splat_records option is misaligned or has no row count is refused
    before any CUDA call."""
    _expect(lib, lib.gs_pack_splats(-1, 1, P, P, P, P, P, None), INVALID, "gs_pack_splats")
    _expect(lib, lib.gs_pack_splats(10, 3, P, P, P, P, P, None), INVALID, "gs_pack_splats")  # not a multiple
    _expect(lib, lib.gs_pack_splats(10, 10, P, P, None, P, P, None), INVALID, "gs_pack_splats")
    _expect(lib, lib.gs_pack_splats(10, 10, P, P, P, P, ODD, None), INVALID, "gs_pack_splats")
    w, h = _sizes(64), _sizes(48)
    for ptr, count in ((ODD, 10), (P, 0), (P, 1 << 31)):
        o = gs.make_opts("fp16_split")
        o.splat_records, o.splat_record_count = ptr.value, count
        _expect(lib, lib.gs_blend_forward_views(1, w, h, 0, P, P, P, P, P, P, ctypes.byref(o), P, P, P, None),
                INVALID, "gs_blend_forward")
    assert ctypes.sizeof(gs.gs_blend_opts) == 80
