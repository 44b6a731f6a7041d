"""FP64 CPU oracle for the Gaussian-splatting hot path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library never
imports, links or calls anything here, and nothing here imports the CUDA
package.  The arithmetic lives in ``gs_oracle.cpp`` (plain FP64 C++); this
module only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

ORACLE_CFLAGS = ["-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-ffp-contract=off"]


def build(force: bool = False) -> str:
    """Compile gs_oracle.cpp into liboracle.so next to it (g++, no GPU)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", *ORACLE_CFLAGS, _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB_PATH)
        _lib.oracle_bin_sort.restype = ctypes.c_int64
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def camera_array(cam) -> np.ndarray:
    """Pack a scenes.Camera into the oracle's 22-double layout."""
    c = np.zeros(22, dtype=np.float64)
    c[0], c[1] = cam.width, cam.height
    c[2:6] = cam.fx, cam.fy, cam.cx, cam.cy
    c[6:15] = np.asarray(cam.R, dtype=np.float64).reshape(-1)
    c[15:18] = np.asarray(cam.t, dtype=np.float64)
    c[18], c[19] = cam.znear, cam.lowpass
    return c


def num_tiles(width: int, height: int) -> int:
    return ((width + 15) // 16) * ((height + 15) // 16)


def project(means, scales, quats, sh, sh_degree, cam) -> dict:
    n = int(means.shape[0])
    means, scales, quats, sh = (_c(a, np.float32) for a in (means, scales, quats, sh))
    out = dict(
        mean2d=np.zeros((n, 2)), cov2d=np.zeros((n, 3)), conic=np.zeros((n, 3)),
        depth=np.zeros(n), radius=np.zeros(n, np.int32), rgb=np.zeros((n, 3)),
        rect=np.zeros((n, 4), np.int32), tiles_touched=np.zeros(n, np.int64))
    lib().oracle_project(
        ctypes.c_int(n), _p(means), _p(scales), _p(quats), _p(sh), ctypes.c_int(sh_degree),
        _p(camera_array(cam)), _p(out["mean2d"]), _p(out["cov2d"]), _p(out["conic"]),
        _p(out["depth"]), _p(out["radius"]), _p(out["rgb"]), _p(out["rect"]),
        _p(out["tiles_touched"]))
    return out


def project_backward(means, scales, quats, sh, sh_degree, cam, radius, dmean2d, dconic, drgb) -> dict:
    """Gradient of ``project`` for one camera: dL/d(means, scales, quats, sh)
    from dL/d(mean2d, conic, rgb); Gaussians with radius 0 get zeros."""
    n = int(means.shape[0])
    K = (sh_degree + 1) ** 2
    means, scales, quats, sh = (_c(a, np.float32) for a in (means, scales, quats, sh))
    radius = _c(radius, np.int32)
    dmean2d, dconic, drgb = (_c(a, np.float64) for a in (dmean2d, dconic, drgb))
    out = dict(dmeans=np.zeros((n, 3)), dscales=np.zeros((n, 3)), dquats=np.zeros((n, 4)),
               dsh=np.zeros((n, K, 3)))
    lib().oracle_project_backward(
        ctypes.c_int(n), _p(means), _p(scales), _p(quats), _p(sh), ctypes.c_int(sh_degree),
        _p(camera_array(cam)), _p(radius), _p(dmean2d), _p(dconic), _p(drgb), _p(out["dmeans"]),
        _p(out["dscales"]), _p(out["dquats"]), _p(out["dsh"]))
    return out


def sh_basis(dirs) -> np.ndarray:
    dirs = _c(dirs, np.float64)
    out = np.zeros((dirs.shape[0], 16))
    lib().oracle_sh_basis(ctypes.c_int(dirs.shape[0]), _p(dirs), _p(out))
    return out


def bin_sort(mean2d, radius, depth, width, height, capacity=None, conic=None, power_min=None,
             tile_mask=None) -> dict:
    """Duplicate + stable sort; mean2d may be the CUDA path's float32 values
    (converted exactly to double), depth is used through its float32 bits.
    With conic and power_min (float32, per Gaussian) a tile is kept only if
    the largest exponent over the tile's box of pixel-centre offsets reaches
    power_min (opacity-aware lists, decided in FP64); then ``ambiguous`` holds
    one row (tile, Gaussian, decision) per rectangle pair whose decision lies
    within rounding of the threshold.  tile_mask (bool per tile): lists for
    the marked tiles only, the others empty."""
    n = int(mean2d.shape[0])
    mean2d = _c(mean2d, np.float64)
    radius = _c(radius, np.int32)
    depth = _c(depth, np.float32)
    # instance count upper bound from the rectangles is computed by the oracle
    # itself; size buffers generously first, then trim.
    cap = capacity if capacity is not None else None
    if cap is None:
        cap = _count_instances(mean2d, radius, width, height, tile_mask)
    keys = np.zeros(max(cap, 1), np.uint64)
    ids = np.zeros(max(cap, 1), np.uint32)
    ranges = np.zeros(2 * num_tiles(width, height), np.uint32)
    tight = conic is not None and power_min is not None
    c32 = _c(conic, np.float32) if tight else None
    p32 = _c(power_min, np.float32) if tight else None
    amb_cap = 1 << 16
    while True:
        amb = np.zeros((amb_cap, 3), np.int64)
        n_amb = ctypes.c_int64(0)
        I = lib().oracle_bin_sort(ctypes.c_int(n), _p(mean2d), _p(radius), _p(depth), ctypes.c_int(width),
                                  ctypes.c_int(height), ctypes.c_int64(cap), _p(keys), _p(ids), _p(ranges),
                                  _p(c32), _p(p32), _p(amb), ctypes.c_int64(amb_cap), ctypes.byref(n_amb),
                                  _p(None if tile_mask is None else _c(tile_mask, np.uint8)))
        if n_amb.value <= amb_cap:
            break
        amb_cap = int(n_amb.value)
    amb = amb[:n_amb.value]
    if I < 0:
        return dict(n_instances=-1, keys=None, ids=None, tile_ranges=ranges, ambiguous=amb)
    return dict(n_instances=int(I), keys=keys[:I], ids=ids[:I], tile_ranges=ranges, ambiguous=amb)


def _count_instances(mean2d, radius, width, height, tile_mask=None) -> int:
    # only used to size the output buffers; the oracle recomputes rectangles
    tx, ty = (width + 15) // 16, (height + 15) // 16
    if tile_mask is not None:  # at most every marked tile's share of the rectangles that meet it
        m = np.asarray(tile_mask, bool).reshape(ty, tx)
        cols, rows = m.any(0), m.any(1)
        cnt = 0
        r = radius.astype(np.float64)
        x0 = np.clip(np.floor((mean2d[:, 0] - r) / 16), 0, tx - 1).astype(np.int64)
        x1 = np.clip(np.floor((mean2d[:, 0] + r) / 16), 0, tx - 1).astype(np.int64)
        y0 = np.clip(np.floor((mean2d[:, 1] - r) / 16), 0, ty - 1).astype(np.int64)
        y1 = np.clip(np.floor((mean2d[:, 1] + r) / 16), 0, ty - 1).astype(np.int64)
        ccol = np.concatenate([[0], np.cumsum(cols)])
        crow = np.concatenate([[0], np.cumsum(rows)])
        live = radius > 0
        cnt = ((ccol[x1 + 1] - ccol[x0]) * (crow[y1 + 1] - crow[y0]))[live].sum()
        return int(min(cnt, int(m.sum()) * int(live.sum())))
    r = radius.astype(np.float64)
    x0 = np.clip(np.floor((mean2d[:, 0] - r) / 16), 0, None)
    x1 = np.clip(np.floor((mean2d[:, 0] + r) / 16), None, tx - 1)
    y0 = np.clip(np.floor((mean2d[:, 1] - r) / 16), 0, None)
    y1 = np.clip(np.floor((mean2d[:, 1] + r) / 16), None, ty - 1)
    cnt = np.where((radius > 0) & (x1 >= x0) & (y1 >= y0), (x1 - x0 + 1) * (y1 - y0 + 1), 0)
    return int(cnt.sum())


def blend(width, height, tile_ranges, ids, mean2d, conic, opac, rgb, bg=(0.0, 0.0, 0.0),
          alpha_margin=0.0, t_margin=0.0, n_threads=1, tile_subset=None, sum_margin=0.0, sum_slack=0.0) -> dict:
    """Blend over the sorted lists (Eq. 1, Alg. 1's rules) in FP64.  The
    margins describe a lower-precision path's rounding (the oracle's decisions
    do not depend on them): a pixel is ``ambiguous`` when one of its decisions
    lies within that rounding of its threshold, and ``err_bound`` is the
    first-order bound the same rounding puts on its colour.  alpha_margin:
    relative error of alpha; t_margin: relative error of the transmittance
    product; sum_margin: exponent error per unit of the magnitude sum of
    Eq. 3's terms, with offsets enlarged by sum_slack pixels."""
    image = np.zeros((3, height, width))
    T = np.zeros((height, width))
    nc = np.zeros((height, width), np.int32)
    amb = np.zeros((height, width), np.uint8)
    eb = np.zeros((height, width))
    subset = None if tile_subset is None else _c(tile_subset, np.int32)
    margins = np.array([alpha_margin, t_margin, sum_margin, sum_slack], np.float64)
    lib().oracle_blend(
        ctypes.c_int(width), ctypes.c_int(height), _p(_c(tile_ranges, np.uint32)), _p(_c(ids, np.uint32)),
        _p(_c(mean2d, np.float64)), _p(_c(conic, np.float64)), _p(_c(opac, np.float64)),
        _p(_c(rgb, np.float64)), _p(_c(bg, np.float64)), _p(margins), ctypes.c_int(n_threads), _p(subset),
        ctypes.c_int(0 if subset is None else len(subset)),
        _p(image), _p(T), _p(nc), _p(amb), _p(eb))
    return dict(image=image, T_final=T, n_contrib=nc, ambiguous=amb.astype(bool), err_bound=eb)


def brute_force(mean2d, conic, opac, rgb, radius, depth, width, height, bg=(0.0, 0.0, 0.0),
                use_rect=True) -> dict:
    n = int(mean2d.shape[0])
    image = np.zeros((3, height, width))
    T = np.zeros((height, width))
    nc = np.zeros((height, width), np.int32)
    lib().oracle_brute_force(
        ctypes.c_int(n), _p(_c(mean2d, np.float64)), _p(_c(conic, np.float64)), _p(_c(opac, np.float64)),
        _p(_c(rgb, np.float64)), _p(_c(radius, np.int32)), _p(_c(depth, np.float32)), ctypes.c_int(width),
        ctypes.c_int(height), _p(_c(bg, np.float64)), ctypes.c_int(1 if use_rect else 0),
        _p(image), _p(T), _p(nc))
    return dict(image=image, T_final=T, n_contrib=nc)


def blend_grad(width, height, tile_ranges, ids, mean2d, conic, opac, rgb, dL_dimage,
               bg=(0.0, 0.0, 0.0), n_threads=1, tile_subset=None) -> dict:
    n = int(np.asarray(mean2d).shape[0])
    out = dict(mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)))
    subset = None if tile_subset is None else _c(tile_subset, np.int32)
    lib().oracle_blend_grad(
        ctypes.c_int(width), ctypes.c_int(height), _p(_c(tile_ranges, np.uint32)), _p(_c(ids, np.uint32)),
        _p(_c(mean2d, np.float64)), _p(_c(conic, np.float64)), _p(_c(opac, np.float64)),
        _p(_c(rgb, np.float64)), _p(_c(bg, np.float64)), _p(_c(dL_dimage, np.float64)), ctypes.c_int(n),
        ctypes.c_int(n_threads), _p(subset), ctypes.c_int(0 if subset is None else len(subset)),
        _p(out["mean2d"]), _p(out["conic"]), _p(out["opacity"]), _p(out["rgb"]))
    return out


def power_eq6(abc, hat, bar):
    abc, hat, bar = _c(abc, np.float64), _c(hat, np.float64), _c(bar, np.float64)
    n = abc.shape[0]
    dot = np.zeros(n)
    direct = np.zeros(n)
    lib().oracle_power_eq6(ctypes.c_int(n), _p(abc), _p(hat), _p(bar), _p(dot), _p(direct))
    return dot, direct


def tile_power(width, tile, tile_ranges, ids, mean2d, conic) -> np.ndarray:
    tile_ranges = _c(tile_ranges, np.uint32)
    L = int(tile_ranges[2 * tile + 1]) - int(tile_ranges[2 * tile])
    out = np.zeros((max(L, 0), 256))
    lib().oracle_tile_power(ctypes.c_int(width), ctypes.c_int(tile), _p(tile_ranges), _p(_c(ids, np.uint32)),
                            _p(_c(mean2d, np.float64)), _p(_c(conic, np.float64)), _p(out))
    return out


def render(scene, cam_index=0, bg=(0.0, 0.0, 0.0), n_threads=1) -> dict:
    """Whole forward pass in FP64: project -> bin/sort -> blend."""
    cam = scene.cameras[cam_index]
    pr = project(scene.means, scene.scales, scene.quats, scene.sh, scene.sh_degree, cam)
    bs = bin_sort(pr["mean2d"], pr["radius"], pr["depth"].astype(np.float32), cam.width, cam.height)
    bl = blend(cam.width, cam.height, bs["tile_ranges"], bs["ids"], pr["mean2d"], pr["conic"],
               scene.opacities.astype(np.float64), pr["rgb"], bg=bg, n_threads=n_threads)
    return dict(project=pr, bin_sort=bs, blend=bl)
