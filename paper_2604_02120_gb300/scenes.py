"""Seeded synthetic scenes and cameras: the one module that feeds both the
CUDA path and the FP64 oracle.

It draws random numbers and builds pinhole cameras; it holds none of the
method's arithmetic (no projection, sorting or blending).  Every array is
float32 in the layout the C ABI takes (``include/gs.h``):

* ``means``     N x 3   world-space centres
* ``scales``    N x 3   linear per-axis standard deviations (exp of log-scales)
* ``quats``     N x 4   unit quaternions (w, x, y, z)
* ``opacities`` N       in (0, 1)
* ``sh``        N x K x 3, K = (degree + 1)^2 real SH coefficients per channel

The scene recipes follow the workload descriptions used for the benchmark
configurations (3D Gaussian scenes of the sizes the paper evaluates in its
Table 1, which are trained real captures; these synthetic scenes stand in for
them).  Draw order inside a recipe is fixed so a seed reproduces a scene
bit for bit: means, log-scales, quaternions, opacities, SH.
"""
from __future__ import annotations

import dataclasses
import hashlib
import math

import numpy as np

__all__ = [
    "Camera", "Scene", "look_at_camera", "ring_cameras", "make_config",
    "tiny_scene", "scene_digest", "CONFIG_NAMES",
]

CONFIG_NAMES = {
    0: "fp32 fwd 256x256, 10k gaussians, SH0",
    1: "fwd 1280x720, 200k gaussians, SH3",
    2: "fwd+bwd 1920x1080, 1M clustered gaussians",
    3: "batched fwd+bwd, 16 cameras of mixed resolution, 1.5M clustered gaussians",
    4: "4K stress 3840x2160, 3M heavy-tailed gaussians, SH3",
}


@dataclasses.dataclass
class Camera:
    """Pinhole camera, OpenCV axes (x right, y down, z forward).

    ``R``/``t`` map world points into camera space: p_cam = R @ p + t.
    Pixel (px, py) covers [px, px+1) x [py, py+1); its centre is at +0.5.
    """
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray          # 3 x 3 float64
    t: np.ndarray          # 3 float64
    znear: float = 0.2
    lowpass: float = 0.3

    @property
    def tiles_x(self) -> int:
        return (self.width + 15) // 16

    @property
    def tiles_y(self) -> int:
        return (self.height + 15) // 16

    @property
    def num_tiles(self) -> int:
        return self.tiles_x * self.tiles_y

    def world_to_cam_3x4(self) -> np.ndarray:
        m = np.zeros((3, 4), dtype=np.float64)
        m[:, :3] = self.R
        m[:, 3] = self.t
        return m

    def position(self) -> np.ndarray:
        return -self.R.T @ self.t


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    scales: np.ndarray
    quats: np.ndarray
    opacities: np.ndarray
    sh: np.ndarray
    sh_degree: int
    cameras: list
    target: list = dataclasses.field(default_factory=list)  # per camera 3 x H x W

    @property
    def n(self) -> int:
        return int(self.means.shape[0])


def look_at_camera(pos, target, width, height, fov_y_deg=60.0, znear=0.2, lowpass=0.3) -> Camera:
    """Camera at ``pos`` looking at ``target``; world +y maps to image down.

    Intrinsics: fy = fx = (H/2)/tan(fov_y/2), principal point at (W/2, H/2).
    """
    pos = np.asarray(pos, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    z = target - pos
    z /= np.linalg.norm(z)
    down = np.array([0.0, 1.0, 0.0])
    x = np.cross(down, z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z], axis=0)
    t = -R @ pos
    f = (height / 2.0) / math.tan(math.radians(fov_y_deg) / 2.0)
    return Camera(width, height, f, f, width / 2.0, height / 2.0, R, t, znear, lowpass)


def ring_cameras(k: int, radius: float, resolutions) -> list:
    """``k`` cameras on the y = 0 ring of ``radius`` at angles 2*pi*i/k, all
    looking at the origin; camera 0 sits at (0, 0, -radius)."""
    cams = []
    for i in range(k):
        a = 2.0 * math.pi * i / k
        pos = (radius * math.sin(a), 0.0, -radius * math.cos(a))
        w, h = resolutions[i]
        cams.append(look_at_camera(pos, (0.0, 0.0, 0.0), w, h))
    return cams


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sh(rng, n, degree, dc_std, rest_std):
    k = (degree + 1) ** 2
    sh = np.zeros((n, k, 3), dtype=np.float64)
    sh[:, 0, :] = rng.normal(0.0, dc_std, (n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, rest_std, (n, k - 1, 3))
    return sh


def _f32(a):
    # heavy-tailed log-scales can exceed the float32 range; those scales become
    # inf (the projection culls such Gaussians)
    with np.errstate(over="ignore"):
        return np.ascontiguousarray(a, dtype=np.float32)


def _uniform_gaussians(rng, n, degree):
    means = rng.uniform(-1.0, 1.0, (n, 3))
    log_scales = rng.normal(-4.0, 0.5, (n, 3))
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.standard_normal(n))
    sh = _sh(rng, n, degree, 0.3, 0.05)
    return means, np.exp(log_scales), quats, opac, sh


def _clustered_means(rng, n, clusters=64):
    centres = rng.uniform(-2.0, 2.0, (clusters, 3))
    member = rng.integers(0, clusters, n)
    return centres[member] + rng.normal(0.0, 0.2, (n, 3))


def _shrunk_log_scales(rng, n, mean, std):
    # "one axis shrunk by 2.0": log-scale minus 2.0 on one uniformly chosen axis
    ls = rng.normal(mean, std, (n, 3))
    axis = rng.integers(0, 3, n)
    ls[np.arange(n), axis] -= 2.0
    return ls


def _clustered_gaussians(rng, n, degree):
    means = _clustered_means(rng, n)
    log_scales = _shrunk_log_scales(rng, n, -4.5, 0.8)
    quats = _unit_quats(rng, n)
    opac = _sigmoid(rng.standard_normal(n))
    sh = _sh(rng, n, degree, 0.3, 0.05)
    return means, np.exp(log_scales), quats, opac, sh


def _heavy_tailed_gaussians(rng, n, degree):
    means = _clustered_means(rng, n)
    log_scales = -4.5 + 0.7 * rng.standard_t(3.0, (n, 3))
    quats = _unit_quats(rng, n)
    opac = rng.beta(0.5, 0.5, n)
    # keep opacity strictly inside (0, 1) as float32
    opac = np.clip(opac, 1e-7, 1.0 - 1e-7)
    sh = _sh(rng, n, degree, 0.3, 0.05)
    return means, np.exp(log_scales), quats, opac, sh


def _pack(parts, degree, cams, rng, with_target):
    means, scales, quats, opac, sh = parts
    sc = Scene(_f32(means), _f32(scales), _f32(quats), _f32(opac), _f32(sh), degree, cams)
    if with_target:
        sc.target = [_f32(rng.uniform(0.0, 1.0, (3, c.height, c.width))) for c in cams]
    return sc


def make_config(k: int, seed: int = 0, n: int | None = None, with_target: bool = False) -> Scene:
    """Synthetic scene ``k`` of the five workloads:
    0: 256x256, 10k uniform Gaussians, SH degree 0;
    1: 1280x720, 200k uniform Gaussians, SH degree 3;
    2: 1920x1080, 1M Gaussians in 64 anisotropic clusters, SH degree 0;
    3: 16 ring cameras of mixed resolution, 1.5M clustered Gaussians;
    4: 3840x2160, 3M Gaussians, heavy-tailed scales, Beta(0.5, 0.5) opacity, SH 3.

    ``n`` overrides the Gaussian count (same recipe, fewer draws) for tests.
    """
    rng = np.random.default_rng(seed)
    if k == 0:
        n = 10_000 if n is None else n
        parts = _uniform_gaussians(rng, n, 0)
        cams = [look_at_camera((0, 0, -3), (0, 0, 0), 256, 256)]
        return _pack(parts, 0, cams, rng, with_target)
    if k == 1:
        n = 200_000 if n is None else n
        parts = _uniform_gaussians(rng, n, 3)
        cams = [look_at_camera((0, 0, -3), (0, 0, 0), 1280, 720)]
        return _pack(parts, 3, cams, rng, with_target)
    if k == 2:
        n = 1_000_000 if n is None else n
        parts = _clustered_gaussians(rng, n, 0)
        cams = [look_at_camera((0, 0, -3), (0, 0, 0), 1920, 1080)]
        return _pack(parts, 0, cams, rng, with_target)
    if k == 3:
        n = 1_500_000 if n is None else n
        parts = _clustered_gaussians(rng, n, 0)
        choices = [(640, 480), (1280, 720), (1600, 900), (1920, 1080)]
        res = [choices[i] for i in rng.integers(0, 4, 16)]
        cams = ring_cameras(16, 3.0, res)
        return _pack(parts, 0, cams, rng, with_target)
    if k == 4:
        n = 3_000_000 if n is None else n
        parts = _heavy_tailed_gaussians(rng, n, 3)
        cams = [look_at_camera((0, 0, -3), (0, 0, 0), 3840, 2160)]
        return _pack(parts, 3, cams, rng, with_target)
    raise ValueError(f"unknown configuration {k}")


def tiny_scene(seed: int, n: int = 32, width: int = 48, height: int = 40, sh_degree: int = 0,
               scale_lo: float = -3.0, scale_hi: float = -1.5, opac_lo: float = 0.05,
               opac_hi: float = 0.99) -> Scene:
    """Small scene whose splats are a few pixels to a few tiles wide, for
    brute-force checks and ragged-edge tests (width/height need not be
    multiples of 16)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-0.8, 0.8, (n, 3))
    log_scales = rng.uniform(scale_lo, scale_hi, (n, 3))
    quats = _unit_quats(rng, n)
    opac = rng.uniform(opac_lo, opac_hi, n)
    sh = _sh(rng, n, sh_degree, 0.4, 0.1)
    cams = [look_at_camera((0, 0, -3), (0, 0, 0), width, height)]
    return _pack((means, np.exp(log_scales), quats, opac, sh), sh_degree, cams, rng, False)


def upstream_grad(seed: int, cams) -> list:
    """Seeded synthetic dL/d(image) for each camera (3 x H x W, N(0, 1))."""
    rng = np.random.default_rng(seed + 7919)
    return [_f32(rng.standard_normal((3, c.height, c.width))) for c in cams]


def scene_digest(sc: Scene) -> str:
    h = hashlib.sha256()
    for a in (sc.means, sc.scales, sc.quats, sc.opacities, sc.sh):
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()
