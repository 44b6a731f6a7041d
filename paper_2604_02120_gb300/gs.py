"""Python binding of the C ABI in include/gs.h (ctypes; argument marshalling only).

Every function named gs_* here calls the C entry point of the same name with
raw device pointers taken from torch tensors; all computation runs in the
CUDA library ``libgs.so`` built in-tree by ``paper_2604_02120_gb300/build.py``.
There is no fallback: if the library is missing or fails to load, the calls
raise.  PyTorch provides device memory and the current CUDA stream only.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgs.so")

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CUDA, GS_ERR_CAPACITY, GS_ERR_TIMEOUT, GS_ERR_UNSUPPORTED, GS_ERR_WORKSPACE = range(7)
(GS_BLEND_FP32, GS_BLEND_TC_FP16, GS_BLEND_TC_BF16, GS_BLEND_TC_FP16_SPLIT, GS_BLEND_TC_BF16_SPLIT,
 GS_BLEND_TC_FP8_SPLIT, GS_BLEND_PERSISTENT_FP32) = range(7)
VARIANTS = {
    "fp32": GS_BLEND_FP32, "fp16": GS_BLEND_TC_FP16, "bf16": GS_BLEND_TC_BF16,
    "fp16_split": GS_BLEND_TC_FP16_SPLIT, "bf16_split": GS_BLEND_TC_BF16_SPLIT, "fp8_split": GS_BLEND_TC_FP8_SPLIT,
    # the tensor-core kernel with the exponent contraction on CUDA cores (forward only)
    "fp32_persistent": GS_BLEND_PERSISTENT_FP32,
}

# Entry points declared in include/gs.h
ABI_FUNCTIONS = (
    "gs_version", "gs_status_string", "gs_last_error", "gs_project", "gs_bin_sort_workspace_size",
    "gs_bin_sort", "gs_blend_forward", "gs_blend_backward", "gs_tile_power", "gs_sync_status",
    "gs_selftest_bounded_wait", "gs_launch_count", "gs_bin_sort_noalloc", "gs_bin_sort_noalloc_max_bytes",
    "gs_project_views", "gs_bin_sort_views", "gs_blend_forward_views", "gs_blend_backward_views",
    "gs_blend_autotune", "gs_measure_peaks", "gs_alpha_power_min", "gs_project_backward",
    "gs_project_bin_small", "gs_tile_order", "gs_pack_splats", "gs_blend_autotune_backward", "gs_render_small",
    "gs_set_kernel_events",
)


class gs_peaks(ctypes.Structure):
    _fields_ = [("ex2_per_s", ctypes.c_double), ("rcp_per_s", ctypes.c_double), ("fma_per_s", ctypes.c_double),
                ("sm_mhz", ctypes.c_double), ("sms", ctypes.c_int32)]


class GsError(RuntimeError):
    def __init__(self, status: int, where: str, text: str):
        super().__init__(f"{where}: status {status} ({text})")
        self.status = status


class gs_camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("world_to_cam", ctypes.c_float * 12), ("znear", ctypes.c_float), ("lowpass", ctypes.c_float)]


class gs_blend_opts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("chunk", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("ref_origin", ctypes.c_int32), ("bg", ctypes.c_float * 3), ("bwd_stages", ctypes.c_int32),
                ("timeout_ns", ctypes.c_int64), ("shard_count", ctypes.c_int32), ("shard_index", ctypes.c_int32),
                ("tile_order", ctypes.c_void_p), ("issued_pairs", ctypes.c_void_p),
                ("splat_records", ctypes.c_void_p), ("splat_record_count", ctypes.c_int64)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libgs.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    lib.gs_version.restype = i32
    lib.gs_launch_count.restype = i64
    lib.gs_bin_sort_noalloc_max_bytes.restype = sz
    lib.gs_bin_sort_noalloc.argtypes = [i32, vp, vp, vp, i32, i32, i64, vp, vp, vp, ctypes.POINTER(i64), vp]
    lib.gs_status_string.restype = ctypes.c_char_p
    lib.gs_status_string.argtypes = [ctypes.c_int]
    lib.gs_last_error.restype = ctypes.c_char_p
    lib.gs_project.argtypes = [i32, vp, vp, vp, vp, i32, ctypes.POINTER(gs_camera), vp, vp, vp, vp, vp, vp, vp]
    lib.gs_bin_sort_workspace_size.argtypes = [i32, i64, i32, i32, ctypes.POINTER(sz)]
    lib.gs_bin_sort.argtypes = [i32, vp, vp, vp, i32, i32, i64, vp, sz, vp, vp, vp, ctypes.POINTER(i64), vp]
    lib.gs_blend_forward.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, ctypes.POINTER(gs_blend_opts), vp, vp, vp, vp]
    lib.gs_blend_backward.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, ctypes.POINTER(gs_blend_opts), vp, vp, vp,
                                      vp, vp, vp, vp, vp]
    lib.gs_tile_power.argtypes = [i32, i32, vp, vp, vp, vp, vp, ctypes.POINTER(gs_blend_opts), vp, i32, i32, vp, vp]
    i32p, i64p = ctypes.POINTER(i32), ctypes.POINTER(i64)
    lib.gs_project_views.argtypes = [i32, vp, vp, vp, vp, i32, ctypes.POINTER(gs_camera), i32, vp, vp, vp, vp, vp,
                                     vp, vp]
    lib.gs_bin_sort_views.argtypes = [i32, i32, vp, vp, vp, vp, vp, i32p, i32p, i64, vp, sz, vp, vp, vp, i64p, vp, vp]
    lib.gs_alpha_power_min.argtypes = [i32, vp, vp, vp]
    lib.gs_pack_splats.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp]
    lib.gs_tile_order.argtypes = [i32, i32p, i32p, vp, vp, vp]
    lib.gs_project_bin_small.argtypes = [i32, vp, vp, vp, vp, i32, ctypes.POINTER(gs_camera), vp, i32, vp, vp, vp,
                                         vp, vp, vp, vp, vp, vp]
    lib.gs_set_kernel_events.argtypes = [i32, vp, vp]
    lib.gs_render_small.argtypes = [i32, vp, vp, vp, vp, i32, ctypes.POINTER(gs_camera), vp, i32, vp,
                                    ctypes.POINTER(ctypes.c_float), vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.gs_project_backward.argtypes = [i32, vp, vp, vp, vp, i32, ctypes.POINTER(gs_camera), i32, vp, vp, vp, vp,
                                        vp, vp, vp, vp, vp]
    lib.gs_blend_forward_views.argtypes = [i32, i32p, i32p, i32, vp, vp, vp, vp, vp, vp,
                                           ctypes.POINTER(gs_blend_opts), vp, vp, vp, vp]
    lib.gs_blend_backward_views.argtypes = [i32, i32p, i32p, i32, vp, vp, vp, vp, vp, vp,
                                            ctypes.POINTER(gs_blend_opts), vp, vp, vp, vp, vp, vp, vp, vp]
    lib.gs_blend_autotune.argtypes = [i32, i32p, i32p, i32, vp, vp, vp, vp, vp, vp, ctypes.POINTER(gs_blend_opts),
                                      vp, vp, vp, i32, ctypes.POINTER(ctypes.c_float), vp]
    lib.gs_blend_autotune_backward.argtypes = [i32, i32p, i32p, i32, vp, vp, vp, vp, vp, vp,
                                               ctypes.POINTER(gs_blend_opts), vp, vp, vp, vp, vp, vp, vp, i32,
                                               ctypes.POINTER(ctypes.c_float), vp]
    lib.gs_sync_status.argtypes = [vp]
    lib.gs_selftest_bounded_wait.argtypes = [i64, vp]
    lib.gs_measure_peaks.argtypes = [ctypes.POINTER(gs_peaks), vp]
    for name in ABI_FUNCTIONS:
        if name not in ("gs_version", "gs_status_string", "gs_last_error", "gs_launch_count",
                        "gs_bin_sort_noalloc_max_bytes"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != GS_OK:
        lib = load()
        raise GsError(st, where, f"{lib.gs_status_string(st).decode()}; {lib.gs_last_error().decode()}")


def _ptr(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def make_camera(cam) -> gs_camera:
    """gs_camera from any object with width, height, fx, fy, cx, cy, R, t, znear, lowpass."""
    c = gs_camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    for i in range(3):
        for j in range(3):
            c.world_to_cam[4 * i + j] = float(cam.R[i][j])
        c.world_to_cam[4 * i + 3] = float(cam.t[i])
    c.znear, c.lowpass = float(cam.znear), float(cam.lowpass)
    return c


def make_opts(variant="fp32", chunk=0, stages=0, ref_origin=0, bg=(0.0, 0.0, 0.0), timeout_ns=0, shard_count=0,
              shard_index=0, tile_order=None, issued_pairs=None, splat_records=None, bwd_stages=0) -> gs_blend_opts:
    """Blend options; tile_order (a device tensor from tile_order(), kept
    alive by the caller while the options are used) makes the kernels take
    the longest tile lists first; splat_records (from pack_splats, kept alive
    likewise) makes the tensor-core kernels stage splats by TMA gathers."""
    o = gs_blend_opts()
    o.variant = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    o.chunk, o.stages, o.ref_origin, o.bwd_stages = int(chunk), int(stages), int(ref_origin), int(bwd_stages)
    for i in range(3):
        o.bg[i] = float(bg[i])
    o.timeout_ns = int(timeout_ns)
    o.shard_count, o.shard_index = int(shard_count), int(shard_index)
    o.tile_order = None if tile_order is None else tile_order.data_ptr()
    o.issued_pairs = None if issued_pairs is None else issued_pairs.data_ptr()
    set_records(o, splat_records)
    return o


def set_records(opts, records):
    """Point the options at a packed record table (None: the load-based path)."""
    opts.splat_records = None if records is None else records.data_ptr()
    opts.splat_record_count = 0 if records is None else int(records.shape[0])
    return opts


# ------------------------------------------------------------- raw entry points

def gs_version() -> int:
    return int(load().gs_version())


def gs_launch_count() -> int:
    return int(load().gs_launch_count())


def gs_project(n, means, scales, quats, sh, sh_degree, cam, mean2d, conic, depth, radius, rgb, tiles_touched,
               stream=None):
    camera = cam if isinstance(cam, gs_camera) else make_camera(cam)
    _check(load().gs_project(n, _ptr(means), _ptr(scales), _ptr(quats), _ptr(sh), sh_degree, ctypes.byref(camera),
                             _ptr(mean2d), _ptr(conic), _ptr(depth), _ptr(radius), _ptr(rgb), _ptr(tiles_touched),
                             _stream(stream)), "gs_project")


def gs_bin_sort_workspace_size(n, capacity, width, height) -> int:
    out = ctypes.c_size_t(0)
    _check(load().gs_bin_sort_workspace_size(n, capacity, width, height, ctypes.byref(out)),
           "gs_bin_sort_workspace_size")
    return int(out.value)


def gs_bin_sort(n, mean2d, radius, depth, width, height, capacity, workspace, keys_sorted, ids_sorted, tile_ranges,
                stream=None, check=True):
    """Returns (status, n_instances)."""
    count = ctypes.c_int64(0)
    st = load().gs_bin_sort(n, _ptr(mean2d), _ptr(radius), _ptr(depth), width, height, capacity, _ptr(workspace),
                            workspace.numel() * workspace.element_size() if workspace is not None else 0,
                            _ptr(keys_sorted), _ptr(ids_sorted), _ptr(tile_ranges), ctypes.byref(count),
                            _stream(stream))
    if check:
        _check(st, "gs_bin_sort")
    return st, int(count.value)


def gs_bin_sort_noalloc_max_bytes() -> int:
    return int(load().gs_bin_sort_noalloc_max_bytes())


def gs_bin_sort_noalloc(n, mean2d, radius, depth, width, height, capacity, keys_sorted, ids_sorted, tile_ranges,
                        stream=None, check=True):
    """gs_bin_sort without a workspace argument (scratch built into the
    library).  Returns (status, n_instances)."""
    count = ctypes.c_int64(0)
    st = load().gs_bin_sort_noalloc(n, _ptr(mean2d), _ptr(radius), _ptr(depth), width, height, capacity,
                                    _ptr(keys_sorted), _ptr(ids_sorted), _ptr(tile_ranges), ctypes.byref(count),
                                    _stream(stream))
    if check:
        _check(st, "gs_bin_sort_noalloc")
    return st, int(count.value)


def gs_blend_forward(width, height, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, opts, image, T_final,
                     n_contrib, stream=None):
    _check(load().gs_blend_forward(width, height, _ptr(tile_ranges), _ptr(ids_sorted), _ptr(mean2d), _ptr(conic),
                                   _ptr(opacity), _ptr(rgb), ctypes.byref(opts), _ptr(image), _ptr(T_final),
                                   _ptr(n_contrib), _stream(stream)), "gs_blend_forward")


def gs_blend_backward(width, height, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, opts, T_final, n_contrib,
                      dL_dimage, dmean2d, dconic, dopacity, drgb, stream=None):
    _check(load().gs_blend_backward(width, height, _ptr(tile_ranges), _ptr(ids_sorted), _ptr(mean2d), _ptr(conic),
                                    _ptr(opacity), _ptr(rgb), ctypes.byref(opts), _ptr(T_final), _ptr(n_contrib),
                                    _ptr(dL_dimage), _ptr(dmean2d), _ptr(dconic), _ptr(dopacity), _ptr(drgb),
                                    _stream(stream)), "gs_blend_backward")


def gs_tile_power(width, height, tile_ranges, ids_sorted, mean2d, conic, opacity, opts, tiles, max_len, out,
                  stream=None):
    _check(load().gs_tile_power(width, height, _ptr(tile_ranges), _ptr(ids_sorted), _ptr(mean2d), _ptr(conic),
                                _ptr(opacity), ctypes.byref(opts), _ptr(tiles), int(tiles.numel()), int(max_len),
                                _ptr(out), _stream(stream)), "gs_tile_power")


def _i32arr(vals):
    arr = (ctypes.c_int32 * len(vals))(*[int(v) for v in vals])
    return arr


def gs_project_views(n, means, scales, quats, sh, sh_degree, cams, mean2d, conic, depth, radius, rgb,
                     tiles_touched, stream=None):
    arr = (gs_camera * len(cams))(*[c if isinstance(c, gs_camera) else make_camera(c) for c in cams])
    _check(load().gs_project_views(n, _ptr(means), _ptr(scales), _ptr(quats), _ptr(sh), sh_degree, arr, len(cams),
                                   _ptr(mean2d), _ptr(conic), _ptr(depth), _ptr(radius), _ptr(rgb),
                                   _ptr(tiles_touched), _stream(stream)), "gs_project_views")


def gs_project_bin_small(n, means, scales, quats, sh, sh_degree, cam, power_min, max_per_tile, mean2d, conic, depth,
                         radius, rgb, tiles_touched, ids, tile_ranges, stream=None):
    camera = cam if isinstance(cam, gs_camera) else make_camera(cam)
    _check(load().gs_project_bin_small(n, _ptr(means), _ptr(scales), _ptr(quats), _ptr(sh), sh_degree,
                                       ctypes.byref(camera), _ptr(power_min), int(max_per_tile), _ptr(mean2d),
                                       _ptr(conic), _ptr(depth), _ptr(radius), _ptr(rgb), _ptr(tiles_touched),
                                       _ptr(ids), _ptr(tile_ranges), _stream(stream)), "gs_project_bin_small")


def gs_render_small(n, means, scales, quats, sh, sh_degree, cam, power_min, max_per_tile, opacity, bg, mean2d, conic,
                    depth, radius, rgb, tiles_touched, ids, tile_ranges, image, T_final, n_contrib, stream=None):
    camera = cam if isinstance(cam, gs_camera) else make_camera(cam)
    bgv = (ctypes.c_float * 3)(*[float(x) for x in bg])
    _check(load().gs_render_small(n, _ptr(means), _ptr(scales), _ptr(quats), _ptr(sh), sh_degree,
                                  ctypes.byref(camera), _ptr(power_min), int(max_per_tile), _ptr(opacity), bgv,
                                  _ptr(mean2d), _ptr(conic), _ptr(depth), _ptr(radius), _ptr(rgb),
                                  _ptr(tiles_touched), _ptr(ids), _ptr(tile_ranges), _ptr(image), _ptr(T_final),
                                  _ptr(n_contrib), _stream(stream)), "gs_render_small")


SMALL_MAX_PER_TILE = 16384
KERNEL_DUPLICATE = 1


def set_kernel_events(kernel, start=None, end=None):
    """gs_set_kernel_events: record the torch.cuda.Events start and end around
    every launch of `kernel` (KERNEL_DUPLICATE) until cleared with None."""
    def handle(e):
        if e is None:
            return None
        if not e.cuda_event:  # torch creates the CUDA event on its first record
            e.record()
            e.synchronize()
        return ctypes.c_void_p(e.cuda_event)
    _check(load().gs_set_kernel_events(int(kernel), handle(start), handle(end)), "gs_set_kernel_events")


def gs_tile_order(widths, heights, tile_ranges, order, stream=None):
    _check(load().gs_tile_order(len(widths), _i32arr(widths), _i32arr(heights), _ptr(tile_ranges), _ptr(order),
                                _stream(stream)), "gs_tile_order")


def tile_order(tile_ranges, widths, heights, out=None, stream=None):
    """Global tile ids, longest list first (gs_tile_order), for make_opts(tile_order=...)."""
    out = torch.empty(tile_ranges.numel() // 2, device=tile_ranges.device, dtype=torch.int32) if out is None else out
    gs_tile_order(list(widths), list(heights), tile_ranges, out, stream)
    return out


def project_bin_small(means, scales, quats, sh, sh_degree, cam, max_per_tile=1024, power_min=None,
                      stream=None):
    """gs_project + per-tile lists in one cooperative launch (small scenes).
    Returns (proj, bs): the gs_project outputs and a bin/sort dict
    (tile_ranges, ids) that the blend calls take as gs_bin_sort's."""
    n = means.shape[0]
    dev = means.device
    f32 = dict(device=dev, dtype=torch.float32)
    proj = dict(mean2d=torch.empty(n, 2, **f32), conic=torch.empty(n, 3, **f32), depth=torch.empty(n, **f32),
                radius=torch.empty(n, device=dev, dtype=torch.int32), rgb=torch.empty(n, 3, **f32),
                tiles_touched=torch.empty(n, device=dev, dtype=torch.int32))
    nt = num_tiles(cam.width, cam.height)
    ids = torch.empty(nt * max_per_tile, device=dev, dtype=torch.int32)
    ranges = torch.empty(2 * nt, device=dev, dtype=torch.int32)
    gs_project_bin_small(n, means, scales, quats, sh, sh_degree, cam, power_min, max_per_tile, proj["mean2d"],
                         proj["conic"], proj["depth"], proj["radius"], proj["rgb"], proj["tiles_touched"], ids, ranges,
                         stream)
    return proj, dict(tile_ranges=ranges, ids=ids)


def render_small(means, scales, quats, sh, sh_degree, opacities, cam, bg=(0.0, 0.0, 0.0), max_per_tile=1024,
                 power_min=None, stream=None):
    """gs_render_small: projection, per-tile lists and the tensor-core blend
    forward in one cooperative launch (small scenes).  Returns (proj, bs, fwd)
    as project(), a bin/sort dict and blend_forward() would."""
    n = means.shape[0]
    dev = means.device
    f32 = dict(device=dev, dtype=torch.float32)
    proj = dict(mean2d=torch.empty(n, 2, **f32), conic=torch.empty(n, 3, **f32), depth=torch.empty(n, **f32),
                radius=torch.empty(n, device=dev, dtype=torch.int32), rgb=torch.empty(n, 3, **f32),
                tiles_touched=torch.empty(n, device=dev, dtype=torch.int32))
    nt = num_tiles(cam.width, cam.height)
    ids = torch.empty(nt * max_per_tile, device=dev, dtype=torch.int32)
    ranges = torch.empty(2 * nt, device=dev, dtype=torch.int32)
    W, H = cam.width, cam.height
    fwd = dict(image=torch.zeros(3, H, W, **f32), T_final=torch.zeros(H, W, **f32),
               n_contrib=torch.zeros(H, W, device=dev, dtype=torch.int32))
    gs_render_small(n, means, scales, quats, sh, sh_degree, cam, power_min, max_per_tile, opacities, bg,
                    proj["mean2d"], proj["conic"], proj["depth"], proj["radius"], proj["rgb"], proj["tiles_touched"],
                    ids, ranges, fwd["image"], fwd["T_final"], fwd["n_contrib"], stream)
    return proj, dict(tile_ranges=ranges, ids=ids), fwd


def gs_project_backward(n, means, scales, quats, sh, sh_degree, cams, radius, dmean2d, dconic, drgb, dmeans, dscales,
                        dquats, dsh, stream=None):
    arr = (gs_camera * len(cams))(*[c if isinstance(c, gs_camera) else make_camera(c) for c in cams])
    _check(load().gs_project_backward(n, _ptr(means), _ptr(scales), _ptr(quats), _ptr(sh), sh_degree, arr, len(cams),
                                      _ptr(radius), _ptr(dmean2d), _ptr(dconic), _ptr(drgb), _ptr(dmeans),
                                      _ptr(dscales), _ptr(dquats), _ptr(dsh), _stream(stream)), "gs_project_backward")


def gs_bin_sort_views(n_views, n_per_view, mean2d, radius, depth, widths, heights, capacity, workspace, keys_sorted,
                      ids_sorted, tile_ranges, count_dev=None, stream=None, check=True, conic=None, power_min=None):
    """Synchronising mode if count_dev is None (returns (status, count)),
    otherwise graph mode: the count goes to the int64 device tensor count_dev.
    conic and power_min (both or neither) select opacity-aware tile lists."""
    count = ctypes.c_int64(0)
    st = load().gs_bin_sort_views(n_views, n_per_view, _ptr(mean2d), _ptr(radius), _ptr(depth), _ptr(conic),
                                  _ptr(power_min), _i32arr(widths),
                                  _i32arr(heights), capacity, _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), _ptr(keys_sorted), _ptr(ids_sorted),
                                  _ptr(tile_ranges), None if count_dev is not None else ctypes.byref(count),
                                  _ptr(count_dev), _stream(stream))
    if check:
        _check(st, "gs_bin_sort_views")
    return st, int(count.value)


def gs_blend_forward_views(widths, heights, n_per_view, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, opts,
                           image, T_final, n_contrib, stream=None):
    _check(load().gs_blend_forward_views(len(widths), _i32arr(widths), _i32arr(heights), n_per_view,
                                         _ptr(tile_ranges), _ptr(ids_sorted), _ptr(mean2d), _ptr(conic),
                                         _ptr(opacity), _ptr(rgb), ctypes.byref(opts), _ptr(image), _ptr(T_final),
                                         _ptr(n_contrib), _stream(stream)), "gs_blend_forward_views")


def gs_blend_backward_views(widths, heights, n_per_view, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, opts,
                            T_final, n_contrib, dL_dimage, dmean2d, dconic, dopacity, drgb, stream=None):
    _check(load().gs_blend_backward_views(len(widths), _i32arr(widths), _i32arr(heights), n_per_view,
                                          _ptr(tile_ranges), _ptr(ids_sorted), _ptr(mean2d), _ptr(conic),
                                          _ptr(opacity), _ptr(rgb), ctypes.byref(opts), _ptr(T_final),
                                          _ptr(n_contrib), _ptr(dL_dimage), _ptr(dmean2d), _ptr(dconic),
                                          _ptr(dopacity), _ptr(drgb), _stream(stream)), "gs_blend_backward_views")


def gs_blend_autotune(widths, heights, n_per_view, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb, opts,
                      image, T_final, n_contrib, reps=5, stream=None) -> float:
    """Sets opts.chunk / opts.stages to the fastest built pair; returns its ms."""
    best = ctypes.c_float(0.0)
    _check(load().gs_blend_autotune(len(widths), _i32arr(widths), _i32arr(heights), n_per_view, _ptr(tile_ranges),
                                    _ptr(ids_sorted), _ptr(mean2d), _ptr(conic), _ptr(opacity), _ptr(rgb),
                                    ctypes.byref(opts), _ptr(image), _ptr(T_final), _ptr(n_contrib), int(reps),
                                    ctypes.byref(best), _stream(stream)), "gs_blend_autotune")
    return float(best.value)


def gs_blend_autotune_backward(widths, heights, n_per_view, tile_ranges, ids_sorted, mean2d, conic, opacity, rgb,
                               opts, T_final, n_contrib, dL_dimage, grads, reps=5, stream=None) -> float:
    """Sets opts.bwd_stages to the fastest built ring depth of the tensor-core
    backward; `grads` (mean2d, conic, opacity, rgb buffers) are overwritten
    with unspecified values.  Returns the best ms."""
    best = ctypes.c_float(0.0)
    _check(load().gs_blend_autotune_backward(len(widths), _i32arr(widths), _i32arr(heights), n_per_view,
                                             _ptr(tile_ranges), _ptr(ids_sorted), _ptr(mean2d), _ptr(conic),
                                             _ptr(opacity), _ptr(rgb), ctypes.byref(opts), _ptr(T_final),
                                             _ptr(n_contrib), _ptr(dL_dimage), _ptr(grads["mean2d"]),
                                             _ptr(grads["conic"]), _ptr(grads["opacity"]), _ptr(grads["rgb"]),
                                             int(reps), ctypes.byref(best), _stream(stream)),
           "gs_blend_autotune_backward")
    return float(best.value)


def gs_alpha_power_min(n, opacity, power_min, stream=None):
    _check(load().gs_alpha_power_min(n, _ptr(opacity), _ptr(power_min), _stream(stream)), "gs_alpha_power_min")


def gs_pack_splats(n_items, n_per_view, mean2d, conic, opacity, rgb, records, stream=None):
    _check(load().gs_pack_splats(n_items, n_per_view, _ptr(mean2d), _ptr(conic), _ptr(opacity), _ptr(rgb),
                                 _ptr(records), _stream(stream)), "gs_pack_splats")


def pack_splats(proj, opacity, out=None, stream=None):
    """Packed splat records (n_items x 16 floats) of a projection's outputs
    (one view, or view-major items of several views over the same opacity)."""
    n_items = proj["mean2d"].shape[0]
    rec = out if out is not None else torch.empty(n_items, 16, device=opacity.device, dtype=torch.float32)
    gs_pack_splats(n_items, opacity.shape[0], proj["mean2d"], proj["conic"], opacity, proj["rgb"], rec, stream)
    return rec


def alpha_power_min(opacity, stream=None):
    out = torch.empty_like(opacity)
    gs_alpha_power_min(opacity.shape[0], opacity, out, stream)
    return out


def gs_sync_status(stream=None) -> int:
    return int(load().gs_sync_status(_stream(stream)))


def gs_selftest_bounded_wait(timeout_ns, stream=None):
    _check(load().gs_selftest_bounded_wait(int(timeout_ns), _stream(stream)), "gs_selftest_bounded_wait")


def gs_measure_peaks(stream=None) -> dict:
    """Measured MUFU ex2 / rcp and FP32 FMA rates of the current GPU (whole
    GPU, per second) and the SM clock during the measurement."""
    p = gs_peaks()
    _check(load().gs_measure_peaks(ctypes.byref(p), _stream(stream)), "gs_measure_peaks")
    return {"ex2_per_s": p.ex2_per_s, "rcp_per_s": p.rcp_per_s, "fma_per_s": p.fma_per_s, "sm_mhz": p.sm_mhz,
            "sms": p.sms}


# ------------------------------------------------------------ tensor helpers

def num_tiles(width, height):
    return ((width + 15) // 16) * ((height + 15) // 16)


def project(means, scales, quats, sh, sh_degree, cam, stream=None) -> dict:
    n = means.shape[0]
    dev = means.device
    f32 = dict(device=dev, dtype=torch.float32)
    out = dict(mean2d=torch.empty(n, 2, **f32), conic=torch.empty(n, 3, **f32), depth=torch.empty(n, **f32),
               radius=torch.empty(n, device=dev, dtype=torch.int32), rgb=torch.empty(n, 3, **f32),
               tiles_touched=torch.empty(n, device=dev, dtype=torch.int32))
    gs_project(n, means, scales, quats, sh, sh_degree, cam, out["mean2d"], out["conic"], out["depth"],
               out["radius"], out["rgb"], out["tiles_touched"], stream)
    return out


def project_backward(means, scales, quats, sh, sh_degree, cams, radius, dmean2d, dconic, drgb, stream=None) -> dict:
    """dL/d(means, scales, quats, sh) from dL/d(mean2d, conic, rgb) of
    gs_project / gs_project_views outputs (view-major for several cameras),
    summed over the views."""
    cams = cams if isinstance(cams, (list, tuple)) else [cams]
    n = means.shape[0]
    f32 = dict(device=means.device, dtype=torch.float32)
    out = dict(dmeans=torch.empty(n, 3, **f32), dscales=torch.empty(n, 3, **f32), dquats=torch.empty(n, 4, **f32),
               dsh=torch.empty(sh.shape, **f32))
    gs_project_backward(n, means, scales, quats, sh, sh_degree, cams, radius, dmean2d.contiguous(),
                        dconic.contiguous(), drgb.contiguous(), out["dmeans"], out["dscales"], out["dquats"],
                        out["dsh"], stream)
    return out


class BinSorter:
    """Holds the workspace and output buffers of gs_bin_sort for a capacity,
    growing them when an instance count exceeds it."""

    def __init__(self, device, capacity=1 << 20):
        self.device = device
        self.capacity = 0
        self.n = -1
        self.width = self.height = 0
        self._alloc(capacity)

    def _alloc(self, capacity):
        self.capacity = int(capacity)
        self.keys = torch.empty(max(self.capacity, 1), device=self.device, dtype=torch.int64)
        self.ids = torch.empty(max(self.capacity, 1), device=self.device, dtype=torch.int32)
        self.workspace = None

    def _ensure_ws(self, n, width, height):
        need = gs_bin_sort_workspace_size(n, self.capacity, width, height)
        if self.workspace is None or self.workspace.numel() < need:
            self.workspace = torch.empty(need + 256, device=self.device, dtype=torch.uint8)

    def run(self, mean2d, radius, depth, width, height, stream=None):
        n = mean2d.shape[0]
        ranges = torch.empty(2 * num_tiles(width, height), device=self.device, dtype=torch.int32)
        for _ in range(2):
            self._ensure_ws(n, width, height)
            st, count = gs_bin_sort(n, mean2d, radius, depth, width, height, self.capacity, self.workspace,
                                    self.keys, self.ids, ranges, stream, check=False)
            if st == GS_ERR_CAPACITY:
                self._alloc(int(count * 1.25) + 1024)
                continue
            _check(st, "gs_bin_sort")
            return dict(keys=self.keys[:count], ids=self.ids[:count], tile_ranges=ranges, n_instances=count)
        raise GsError(GS_ERR_CAPACITY, "gs_bin_sort", "capacity growth failed")


def _list_ids(bs):
    """The sorted ids, or a one-element placeholder when there are no
    instances (every tile range is then empty and nothing is read; the C ABI
    takes no null pointer)."""
    ids = bs["ids"]
    return ids if ids.numel() > 0 else torch.zeros(1, device=ids.device, dtype=ids.dtype)


def blend_forward(width, height, bs, proj, opacity, opts, stream=None) -> dict:
    dev = opacity.device
    # a sharded call writes only its tiles' pixels: the others are zero
    new = torch.zeros if opts.shard_count > 1 else torch.empty
    image = new(3, height, width, device=dev, dtype=torch.float32)
    T = new(height, width, device=dev, dtype=torch.float32)
    nc = new(height, width, device=dev, dtype=torch.int32)
    gs_blend_forward(width, height, bs["tile_ranges"], _list_ids(bs), proj["mean2d"], proj["conic"], opacity,
                     proj["rgb"], opts, image, T, nc, stream)
    return dict(image=image, T_final=T, n_contrib=nc)


def blend_backward(width, height, bs, proj, opacity, opts, fwd, dL_dimage, stream=None) -> dict:
    n = opacity.shape[0]
    # the four outputs accumulate by atomics: views of one buffer, zeroed by one fill
    buf = torch.zeros(9 * n, device=opacity.device)
    g = dict(mean2d=buf[:2 * n].view(n, 2), conic=buf[2 * n:5 * n].view(n, 3), opacity=buf[5 * n:6 * n],
             rgb=buf[6 * n:].view(n, 3))
    gs_blend_backward(width, height, bs["tile_ranges"], _list_ids(bs), proj["mean2d"], proj["conic"], opacity,
                      proj["rgb"], opts, fwd["T_final"], fwd["n_contrib"], dL_dimage.contiguous(), g["mean2d"],
                      g["conic"], g["opacity"], g["rgb"], stream)
    return g


class BlendFunction(torch.autograd.Function):
    """Differentiable blend: (mean2d, conic, opacity, rgb) -> image, with the
    tile lists fixed by a preceding gs_bin_sort."""

    @staticmethod
    def forward(ctx, mean2d, conic, opacity, rgb, tile_ranges, ids, width, height, opts):
        proj = dict(mean2d=mean2d.contiguous(), conic=conic.contiguous(), rgb=rgb.contiguous())
        bs = dict(tile_ranges=tile_ranges, ids=ids)
        out = blend_forward(width, height, bs, proj, opacity.contiguous(), opts)
        ctx.save_for_backward(proj["mean2d"], proj["conic"], opacity.contiguous(), proj["rgb"], tile_ranges, ids,
                              out["T_final"], out["n_contrib"])
        ctx.meta = (width, height, opts)
        ctx.mark_non_differentiable(out["T_final"], out["n_contrib"])
        return out["image"], out["T_final"], out["n_contrib"]

    @staticmethod
    def backward(ctx, dimage, _dT, _dn):
        mean2d, conic, opacity, rgb, ranges, ids, T, nc = ctx.saved_tensors
        width, height, opts = ctx.meta
        g = blend_backward(width, height, dict(tile_ranges=ranges, ids=ids),
                           dict(mean2d=mean2d, conic=conic, rgb=rgb), opacity, opts,
                           dict(T_final=T, n_contrib=nc), dimage)
        return g["mean2d"], g["conic"], g["opacity"], g["rgb"], None, None, None, None, None


def scene_to_device(scene, device="cuda") -> dict:
    t = lambda a: torch.from_numpy(a).to(device).contiguous()  # noqa: E731
    return dict(means=t(scene.means), scales=t(scene.scales), quats=t(scene.quats), opacities=t(scene.opacities),
                sh=t(scene.sh), sh_degree=scene.sh_degree)


def render(dev_scene, cam, opts, sorter: BinSorter | None = None, stream=None) -> dict:
    """project -> bin_sort -> blend_forward for one camera."""
    proj = project(dev_scene["means"], dev_scene["scales"], dev_scene["quats"], dev_scene["sh"],
                   dev_scene["sh_degree"], cam, stream)
    sorter = sorter or BinSorter(dev_scene["means"].device)
    bs = sorter.run(proj["mean2d"], proj["radius"], proj["depth"], cam.width, cam.height, stream)
    out = blend_forward(cam.width, cam.height, bs, proj, dev_scene["opacities"], opts, stream)
    return dict(project=proj, bin_sort=bs, blend=out)


class PipelinedRenderer:
    """Forward + backward of a stream of frames whose inputs live in (pinned)
    host memory, with the copies overlapped: frame k's host-to-device copy
    runs on an upload stream while frame k-1 computes, and its results go
    back on a download stream while frame k+1 computes, so a frame costs
    about max(compute, copies) instead of their sum.  Two BatchRenderers
    alternate (double-buffered device inputs and outputs); compute runs on
    the current stream.  The frames must be independent (rendering many
    scenes or camera sets): a training loop, whose next inputs depend on this
    step's gradients, gains nothing from it.  graphs=True replays each
    renderer's step as a CUDA graph.

    submit(k, host_in, host_out) enqueues frame k: host_in maps
    means/scales/quats/opacities/sh to pinned tensors shaped like the scene,
    host_out maps image/mean2d/conic/opacity/rgb to pinned tensors shaped
    like the renderer's outputs; wait(k) blocks until frame k's results are
    in host_out."""

    KEYS = ("means", "scales", "quats", "opacities", "sh")

    def __init__(self, template_scene, sh_degree, cams, opts, capacity, dL, device="cuda", graphs=False,
                 opacity_aware=False):
        # graphs: each renderer's step is recorded once in a CUDA graph (after
        # one run on the template scene's values) and replayed per frame, one
        # host call instead of one per kernel
        self.r = []
        for _ in range(2):
            dev = {k: torch.empty_like(template_scene[k], device=device) for k in self.KEYS}
            dev["sh_degree"] = sh_degree
            r = BatchRenderer(dev, cams, opts, capacity, device, opacity_aware=opacity_aware)
            r.dL.copy_(dL.reshape(-1))
            if graphs:
                for k in self.KEYS:
                    dev[k].copy_(template_scene[k])
                r.capture()
            self.r.append(r)
        self.up, self.down = torch.cuda.Stream(device), torch.cuda.Stream(device)
        E = torch.cuda.Event
        self.in_ready = [E(), E()]
        self.done = [E(), E()]
        self.out_done = [E(), E()]
        self.used = [False, False]
        self.frame_slot = {}

    def submit(self, k, host_in, host_out):
        i = k % 2
        r = self.r[i]
        cur = torch.cuda.current_stream()
        with torch.cuda.stream(self.up):
            if self.used[i]:
                self.up.wait_event(self.done[i])  # the last frame on these buffers has read its inputs
            for key in self.KEYS:
                r.scene[key].copy_(host_in[key], non_blocking=True)
            self.in_ready[i].record(self.up)
        cur.wait_event(self.in_ready[i])
        if self.used[i]:
            cur.wait_event(self.out_done[i])  # its results have left the output buffers
        if r.graph is not None:
            r.graph.replay()
        else:
            r.step()
        self.done[i].record(cur)
        with torch.cuda.stream(self.down):
            self.down.wait_event(self.done[i])
            H, W = r.heights[0], r.widths[0]
            host_out["image"].copy_(r.image.view(3, H, W), non_blocking=True)
            host_out["mean2d"].copy_(r.g_mean2d, non_blocking=True)
            host_out["conic"].copy_(r.g_conic, non_blocking=True)
            host_out["opacity"].copy_(r.g_opac, non_blocking=True)
            host_out["rgb"].copy_(r.g_rgb, non_blocking=True)
            self.out_done[i].record(self.down)
        self.used[i] = True
        self.frame_slot[k] = i

    def wait(self, k):
        self.out_done[self.frame_slot[k]].synchronize()


class BatchRenderer:
    """Batched forward + backward of one scene seen by several cameras:
    gs_project_views -> gs_bin_sort_views (no host synchronisation) ->
    gs_blend_forward_views (one persistent launch over the tiles of all views)
    -> gs_blend_backward_views.  All buffers are allocated once for a fixed
    instance capacity, so `step` can be captured in a CUDA graph (`capture`);
    an instance count above the capacity is reported by gs_sync_status() as
    GS_ERR_CAPACITY.  With longest_first the blends take the tiles in the
    order of gs_tile_order (longest list first), computed after every sort.
    With opacity_aware the lists are the opacity-aware ones (gs_alpha_power_min
    and the conics passed to gs_bin_sort_views): same images, fewer instances.
    With tma_records the splats are packed after projection (gs_pack_splats)
    and the tensor-core forward stages them by TMA gathers."""

    def __init__(self, dev_scene, cams, opts, capacity, device="cuda", longest_first=True, opacity_aware=False,
                 tma_records=False):
        self.scene = dev_scene
        self.cams = [make_camera(c) for c in cams]
        self.opts = gs_blend_opts.from_buffer_copy(opts)
        self.widths = [c.width for c in self.cams]
        self.heights = [c.height for c in self.cams]
        V, n = len(self.cams), int(dev_scene["means"].shape[0])
        self.n, self.V, self.capacity = n, V, int(capacity)
        f32 = dict(device=device, dtype=torch.float32)
        i32 = dict(device=device, dtype=torch.int32)
        self.mean2d = torch.empty(V * n, 2, **f32)
        self.conic = torch.empty(V * n, 3, **f32)
        self.depth = torch.empty(V * n, **f32)
        self.radius = torch.empty(V * n, **i32)
        self.rgb = torch.empty(V * n, 3, **f32)
        self.touched = torch.empty(V * n, **i32)
        self.total_tiles = sum(num_tiles(w, h) for w, h in zip(self.widths, self.heights))
        self.pixels = sum(w * h for w, h in zip(self.widths, self.heights))
        self.ids = torch.empty(max(self.capacity, 1), **i32)
        self.ranges = torch.empty(2 * self.total_tiles, **i32)
        self.order = torch.empty(self.total_tiles, **i32) if longest_first else None
        self.opts.tile_order = self.order.data_ptr() if longest_first else opts.tile_order
        self.count = torch.zeros(1, device=device, dtype=torch.int64)
        self.pmin = torch.empty(n, **f32) if opacity_aware else None
        self.rec = torch.empty(V * n, 16, **f32) if tma_records and V * n > 0 else None
        set_records(self.opts, self.rec)
        ws = gs_bin_sort_workspace_size(V * n, self.capacity, self.widths[0], self.heights[0])
        self.workspace = torch.empty(ws + 256, device=device, dtype=torch.uint8)
        self.image = torch.empty(3 * self.pixels, **f32)
        self.T = torch.empty(self.pixels, **f32)
        self.nc = torch.empty(self.pixels, **i32)
        self.dL = torch.zeros(3 * self.pixels, **f32)
        # the gradients accumulate by atomics: views of one buffer, zeroed by one fill per step
        self.g_buf = torch.zeros(8 * V * n + n, **f32)
        self.g_mean2d = self.g_buf[:2 * V * n].view(V * n, 2)
        self.g_conic = self.g_buf[2 * V * n:5 * V * n].view(V * n, 3)
        self.g_rgb = self.g_buf[5 * V * n:8 * V * n].view(V * n, 3)
        self.g_opac = self.g_buf[8 * V * n:]
        self.graph = None

    def forward(self, stream=None):
        sc = self.scene
        gs_project_views(self.n, sc["means"], sc["scales"], sc["quats"], sc["sh"], sc["sh_degree"], self.cams,
                         self.mean2d, self.conic, self.depth, self.radius, self.rgb, self.touched, stream)
        if self.rec is not None:
            gs_pack_splats(self.V * self.n, self.n, self.mean2d, self.conic, sc["opacities"], self.rgb, self.rec,
                           stream)
        if self.pmin is not None:
            gs_alpha_power_min(self.n, sc["opacities"], self.pmin, stream)
        gs_bin_sort_views(self.V, self.n, self.mean2d, self.radius, self.depth, self.widths, self.heights,
                          self.capacity, self.workspace, None, self.ids, self.ranges, count_dev=self.count,
                          stream=stream, conic=self.conic if self.pmin is not None else None, power_min=self.pmin)
        if self.order is not None:
            gs_tile_order(self.widths, self.heights, self.ranges, self.order, stream)
        gs_blend_forward_views(self.widths, self.heights, self.n, self.ranges, self.ids, self.mean2d, self.conic,
                               sc["opacities"], self.rgb, self.opts, self.image, self.T, self.nc, stream)

    def backward(self, stream=None):
        self.g_buf.zero_()
        gs_blend_backward_views(self.widths, self.heights, self.n, self.ranges, self.ids, self.mean2d, self.conic,
                                self.scene["opacities"], self.rgb, self.opts, self.T, self.nc, self.dL,
                                self.g_mean2d, self.g_conic, self.g_opac, self.g_rgb, stream)

    def step(self, stream=None):
        self.forward(stream)
        self.backward(stream)

    def capture(self):
        """Record step() into a CUDA graph (run step() once uncaptured first)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step()
        return self.graph

    def view_image(self, v):
        off = sum(self.widths[u] * self.heights[u] for u in range(v))
        W, H = self.widths[v], self.heights[v]
        return (self.image[3 * off:3 * (off + W * H)].view(3, H, W), self.T[off:off + W * H].view(H, W),
                self.nc[off:off + W * H].view(H, W))
