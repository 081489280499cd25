"""Seeded camera poses: a single fixed view and a Catmull-Rom flight path.

A camera is an eye position in world coordinates (FP64), a forward and an up
direction, a vertical field of view, near/far clip distances along the
forward axis, an image size and the cascade settings of the view.
"""

from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

from .fbm import FBm
from .quadtree import Quadtree


@dataclass
class Camera:
    eye: tuple            # world metres (FP64)
    forward: tuple
    up: tuple
    vfov: float           # radians
    znear: float
    zfar: float
    width: int
    height: int
    n_cascades: int
    cascade_size: int
    split_lambda: float = 1.0
    overlap_frac: float = 0.05
    texel_ladder: int = 0         # 0: stable fit; n > 0: lattice fit, n texel sizes per octave
    lod_pixels: float = 0.0       # 0: exact surface; > 0: coarse-level stop at this many pixels
    traversal: int = 0            # 0: max-mip walk one level up per step; 1: climb to the coarsest node entered

    def with_(self, **kw) -> "Camera":
        return replace(self, **kw)


def _dir(yaw: float, pitch: float):
    cp = np.cos(pitch)
    return (float(cp * np.cos(yaw)), float(cp * np.sin(yaw)), float(np.sin(pitch)))


def fixed_camera(tree: Quadtree, fbm: FBm, local_xy, agl: float, yaw_deg: float,
                 pitch_deg: float, vfov_deg: float, width: int, height: int,
                 n_cascades: int, cascade_size: int, split_lambda=1.0,
                 overlap_frac=0.05, znear=1.0, zfar=1.0e5) -> Camera:
    """Eye ``agl`` metres above the terrain at domain-local ``local_xy``."""
    gx, gy = float(local_xy[0]), float(local_xy[1])
    ground = float(fbm(gx, gy))
    eye = (tree.origin_x + gx, tree.origin_y + gy, ground + agl)
    return Camera(eye, _dir(np.radians(yaw_deg), np.radians(pitch_deg)),
                  (0.0, 0.0, 1.0), float(np.radians(vfov_deg)), znear, zfar,
                  width, height, n_cascades, cascade_size, split_lambda, overlap_frac)


def _catmull_rom(p: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Uniform Catmull-Rom through the rows of ``p`` at parameters t in [0, len-1]."""
    n = p.shape[0]
    seg = np.minimum(np.floor(t).astype(int), n - 2)
    u = (t - seg)[:, None]
    i0 = np.clip(seg - 1, 0, n - 1)
    i1, i2 = seg, seg + 1
    i3 = np.clip(seg + 2, 0, n - 1)
    p0, p1, p2, p3 = p[i0], p[i1], p[i2], p[i3]
    return 0.5 * ((2 * p1) + (-p0 + p2) * u + (2 * p0 - 5 * p1 + 4 * p2 - p3) * u ** 2
                  + (-p0 + 3 * p1 - 3 * p2 + p3) * u ** 3)


def flight_path(tree: Quadtree, fbm: FBm, seed: int, n_frames: int, width: int,
                height: int, n_cascades: int, cascade_size: int,
                split_lambda: float, overlap_frac=0.05, n_waypoints=8,
                agl_range=(200.0, 1500.0), pitch_range_deg=(-45.0, -15.0),
                vfov_deg=60.0, znear=1.0, zfar=1.0e5) -> list:
    """Seeded Catmull-Rom flight through ``n_waypoints`` waypoints over the
    inner 80 % of the domain; altitude above ground and pitch are
    interpolated too, and the heading follows the path tangent."""
    rng = np.random.default_rng(seed)
    w, h = tree.width, tree.height
    xy = np.stack([rng.uniform(0.1 * w, 0.9 * w, n_waypoints),
                   rng.uniform(0.1 * h, 0.9 * h, n_waypoints)], axis=1)
    agl = rng.uniform(*agl_range, n_waypoints)
    pitch = rng.uniform(*pitch_range_deg, n_waypoints)
    ctrl = np.column_stack([xy, agl, pitch])
    t = np.linspace(0.0, n_waypoints - 1.0, n_frames)
    pts = _catmull_rom(ctrl, t)
    eps = 1e-3
    ahead = _catmull_rom(ctrl, np.minimum(t + eps, n_waypoints - 1.0))
    behind = _catmull_rom(ctrl, np.maximum(t - eps, 0.0))
    tang = ahead[:, :2] - behind[:, :2]
    cams = []
    for k in range(n_frames):
        x, y = float(np.clip(pts[k, 0], 0.0, w)), float(np.clip(pts[k, 1], 0.0, h))
        a = float(np.clip(pts[k, 2], *agl_range))
        p = float(np.clip(pts[k, 3], *pitch_range_deg))
        yaw = float(np.degrees(np.arctan2(tang[k, 1], tang[k, 0])))
        cams.append(fixed_camera(tree, fbm, (x, y), a, yaw, p, vfov_deg, width, height,
                                 n_cascades, cascade_size, split_lambda, overlap_frac,
                                 znear, zfar))
    return cams
