"""Seeded synthetic inputs shaped like the paper's indoor SLAM workloads.

This module is the one piece both the CUDA path and the FP64 oracle consume.  It
draws numbers and nothing else: no projection, blending, merging or optimiser
arithmetic lives here.  Every array is a fresh ``numpy`` array in the storage
layout of the library (structure of arrays, float32 attributes, uint64 birth
stamps), so the two sides read bit-identical inputs.

The paper evaluates on Replica (1200x680) and TUM RGB-D (640x480) sequences
(Sec. III-A).  Those datasets are not available, so these generators stand in
for them:

* ``box_scene``   - means uniform in a 2x2x2 m box centred 3 m in front of a
  pinhole camera at the origin (the small 10k-Gaussian / 320x240 workload).
* ``room_scene``  - a 4x3x3 m room: means drawn on its six walls with 1 cm
  normal jitter, plus a tail of near-duplicates (2 mm mean jitter, 5 % scale
  jitter) appended with later birth stamps, standing in for the densified
  clones the voxel merge of Sec. II-D is meant to remove.
* ``room_poses``  - keyframe poses inside the room looking at a wall point.

Parameter conventions (shared with the library header):
  means f32[N,3] world frame; log_scales f32[N,3] (scale = exp); quats f32[N,4]
  as (w, x, y, z), not necessarily unit; opacity_logit f32[N] (opacity =
  sigmoid); sh f32[N,K,3] with K = (degree+1)^2; birth u64[N] (smaller = older).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Constant of the degree-0 real spherical harmonic, 1/(2*sqrt(pi)).  Used only to
# turn a drawn colour into the DC coefficient that reproduces it (input recipe).
_DC_OF_COLOUR = 2.0 * math.sqrt(math.pi)


@dataclasses.dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logit: np.ndarray
    sh: np.ndarray
    birth: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(),
                     self.quats[idx].copy(), self.opacity_logit[idx].copy(),
                     self.sh[idx].copy(), self.birth[idx].copy(), self.sh_degree)

    def copy(self) -> "Scene":
        return self.subset(np.arange(self.n))


@dataclasses.dataclass
class Camera:
    """World-to-camera rotation R (row-major 3x3), translation t, pinhole intrinsics.

    Camera frame: x right, y down, z forward.  Pixel (u, v) is the point (u, v).
    """
    R: np.ndarray
    t: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.2


def intrinsics(width: int, height: int):
    """Pinhole intrinsics used for each resolution of the workloads."""
    table = {
        (320, 240): (300.0, 300.0, 160.0, 120.0),
        (640, 480): (525.0, 525.0, 319.5, 239.5),
        (1200, 680): (600.0, 600.0, 599.5, 339.5),
        (1920, 1080): (960.0, 960.0, 959.5, 539.5),
    }
    if (width, height) in table:
        return table[(width, height)]
    f = 0.5 * width
    return (f, f, 0.5 * (width - 1), 0.5 * (height - 1))


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def _uniform_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly distributed unit quaternions (Shoemake's subgroup algorithm), (w,x,y,z)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a, b = np.sqrt(1.0 - u1), np.sqrt(u1)
    x = a * np.sin(2 * np.pi * u2)
    y = a * np.cos(2 * np.pi * u2)
    z = b * np.sin(2 * np.pi * u3)
    w = b * np.cos(2 * np.pi * u3)
    return np.stack([w, x, y, z], axis=1)


def _logit(p):
    return np.log(p) - np.log1p(-p)


def _attributes(rng, n, sh_degree, sh_mode):
    log_scales = rng.uniform(math.log(0.01), math.log(0.1), size=(n, 3))
    quats = _uniform_quats(rng, n)
    opacity = rng.uniform(0.1, 0.9, size=n)
    k = (sh_degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    if sh_mode == "colour":
        sh[:, 0, :] = (rng.random((n, 3)) - 0.5) * _DC_OF_COLOUR
    else:  # "normal": every coefficient (DC included) ~ N(0, 0.1)
        sh[:] = rng.normal(0.0, 0.1, size=(n, k, 3))
    return log_scales, quats, _logit(opacity), sh


def _pack(means, log_scales, quats, opacity_logit, sh, birth, deg) -> Scene:
    f = np.float32
    return Scene(np.ascontiguousarray(means, f), np.ascontiguousarray(log_scales, f),
                 np.ascontiguousarray(quats, f), np.ascontiguousarray(opacity_logit, f),
                 np.ascontiguousarray(sh, f), np.ascontiguousarray(birth, np.uint64), deg)


def box_scene(n: int = 10_000, seed: int = 0, sh_degree: int = 0) -> Scene:
    """Means uniform in the 2x2x2 m box centred at (0, 0, 3); colours uniform in [0,1]."""
    rng = _rng(seed, 0)
    means = rng.uniform(-1.0, 1.0, size=(n, 3)) + np.array([0.0, 0.0, 3.0])
    ls, q, ol, sh = _attributes(rng, n, sh_degree, "colour")
    return _pack(means, ls, q, ol, sh, np.arange(n, dtype=np.uint64), sh_degree)


def box_camera(width: int = 320, height: int = 240) -> Camera:
    fx, fy, cx, cy = intrinsics(width, height)
    return Camera(np.eye(3, dtype=np.float32), np.zeros(3, np.float32), fx, fy, cx, cy,
                  width, height)


ROOM = np.array([4.0, 3.0, 3.0])


def _room_wall_points(rng, n, jitter):
    """Area-weighted uniform points on the 6 walls of [0,4]x[0,3]x[0,3], with normal jitter."""
    L = ROOM
    areas = np.array([L[1] * L[2], L[1] * L[2], L[0] * L[2], L[0] * L[2], L[0] * L[1], L[0] * L[1]])
    face = rng.choice(6, size=n, p=areas / areas.sum())
    pts = rng.random((n, 3)) * L
    axis = face // 2
    side = face % 2
    rows = np.arange(n)
    pts[rows, axis] = side * L[axis] + rng.normal(0.0, jitter, size=n)
    return pts


def room_scene(n: int, seed: int, sh_degree: int = 0, dup_fraction: float = 0.2) -> Scene:
    """Surface-like room scene with a fraction of near-duplicates appended (later births)."""
    rng = _rng(seed, 1)
    n_dup = int(round(dup_fraction * n))
    n_base = n - n_dup
    means = _room_wall_points(rng, n_base, 0.01)
    ls, q, ol, sh = _attributes(rng, n_base, sh_degree, "colour" if sh_degree == 0 else "normal")
    src = rng.choice(n_base, size=n_dup, replace=False)
    d_means = means[src] + rng.normal(0.0, 0.002, size=(n_dup, 3))
    d_ls = ls[src] + rng.normal(0.0, 0.05, size=(n_dup, 3))
    means = np.concatenate([means, d_means])
    ls = np.concatenate([ls, d_ls])
    q = np.concatenate([q, q[src]])
    ol = np.concatenate([ol, ol[src]])
    sh = np.concatenate([sh, sh[src]])
    return _pack(means, ls, q, ol, sh, np.arange(n, dtype=np.uint64), sh_degree)


def look_at(centre, target, width, height) -> Camera:
    """Camera at ``centre`` looking at ``target`` with world +z up (falls back to +y)."""
    c = np.asarray(centre, np.float64)
    f = np.asarray(target, np.float64) - c
    f /= np.linalg.norm(f)
    up = np.array([0.0, 0.0, 1.0])
    if np.linalg.norm(np.cross(f, up)) < 1e-3:
        up = np.array([0.0, 1.0, 0.0])
    x = np.cross(f, up)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])            # rows: camera axes in world coordinates
    t = -R @ c
    fx, fy, cx, cy = intrinsics(width, height)
    return Camera(R.astype(np.float32), t.astype(np.float32), fx, fy, cx, cy, width, height)


def room_poses(n_views: int, seed: int, width: int, height: int):
    """Keyframe poses: centre uniform in the room shrunk by 0.5 m, looking at a wall point."""
    rng = _rng(seed, 2)
    lo = np.full(3, 0.5)
    hi = ROOM - 0.5
    cams = []
    for _ in range(n_views):
        c = lo + rng.random(3) * (hi - lo)
        tgt = _room_wall_points(rng, 1, 0.0)[0]
        while np.linalg.norm(tgt - c) < 0.5:
            tgt = _room_wall_points(rng, 1, 0.0)[0]
        cams.append(look_at(c, tgt, width, height))
    return cams


def image_cotangents(n_views: int, width: int, height: int, seed: int):
    """dL/d(rgb, depth, alpha) ~ U[-1, 1] per element: rgb [V,3,H,W], depth/alpha [V,H,W]."""
    rng = _rng(seed, 3)
    f = np.float32
    g_rgb = rng.uniform(-1.0, 1.0, size=(n_views, 3, height, width)).astype(f)
    g_depth = rng.uniform(-1.0, 1.0, size=(n_views, height, width)).astype(f)
    g_alpha = rng.uniform(-1.0, 1.0, size=(n_views, height, width)).astype(f)
    return g_rgb, g_depth, g_alpha


def workload(name: str):
    """The seeded workloads: returns (scene, cameras).

    ``box10k``      10k Gaussians, 320x240, SH0, one camera (seed 0).
    ``room300k``    300k Gaussians, 640x480 (fx=fy=525), SH0, one pose (seed 1).
    ``room1m_sh3``  1M Gaussians, SH3 coefficients N(0, 0.1), 8 poses at 1200x680 (seed 2).
    """
    if name == "box10k":
        return box_scene(10_000, 0, 0), [box_camera(320, 240)]
    if name == "room300k":
        return room_scene(300_000, 1, 0), room_poses(1, 1, 640, 480)
    if name == "room1m_sh3":
        return room_scene(1_000_000, 2, 3), room_poses(8, 2, 1200, 680)
    raise KeyError(name)
