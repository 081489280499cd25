"""The benchmark workloads as seeded generators.

* ``tiny_config``: 64 x 64 root cells of 10 m, 25 % of them split and 25 % of
  those children split again (10 / 5 / 2.5 m cells); fBm amplitude 500 m; one
  256^2 cascade, a 320 x 240 image, one camera 300 m above the ground,
  pitched down 30 deg, 60 deg vertical field of view.
* ``dem_config``: 4096^2 finest-equivalent cells of 10 m (256^2 root cells of
  160 m, 5 levels) refined by terrain curvature to about 4.5 M leaves (the
  Florence scenario's cell count, Table 1); fBm amplitude 2000 m; four
  2048^2 cascades split with lambda = 0.5; a 1920 x 1080 image along a
  120-frame flight path 200-1500 m above the ground.
* ``precision_config``: ``tiny_config`` with the domain moved to a world
  origin of (5e6, 5e6) m, which FP32 cannot hold to centimetres.
* ``batch_config``: independent tiles of uneven finest size with 1-4
  cascades each and a 960 x 540 view per tile.
* ``serve_config``: a 16384^2-equivalent quadtree (6 levels, 10-320 m cells,
  fBm amplitude 3000 m, a mosaic of curvature-refined blocks) kept resident,
  and a Poisson stream of view requests (rate 200/s) of 1280 x 720,
  1920 x 1080 or 3840 x 2160 with 2-6 cascades of 2048^2.
* ``flood_config`` / ``tiny_flood_config``: the DEM (or tiny) scene plus
  relative water depths at the same cells, a "bathtub" flood: every cell
  below a water level L gets depth L - v (the paper's scenarios carry a flood
  simulation's depths; a level flood is the simplest such field), with L
  chosen so that a given fraction of the domain's area is under water.

All use a Gaussian RBF with sigma = 1.5 cell sizes truncated at 3 cell sizes.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .cameras import Camera, fixed_camera, flight_path
from .fbm import FBm
from .quadtree import Quadtree, curvature_quadtree, random_split_quadtree, tiled_curvature_quadtree

RBF_SIGMA = 1.5
RBF_RADIUS = 3.0


@dataclass
class Scene:
    name: str
    tree: Quadtree
    fbm: FBm
    sigma: float
    radius: float
    cameras: list = field(default_factory=list)
    depth: np.ndarray | None = None   # water depths per leaf (flood scenes)


def flood_depths(tree: Quadtree, wet_area: float) -> tuple:
    """(depths, level): depth = max(L - v, 0) per leaf, L the value below which
    ``wet_area`` of the domain's area lies."""
    area = tree.cell_sizes() ** 2
    order = np.argsort(tree.value, kind="stable")
    cum = np.cumsum(area[order]) / area.sum()
    L = float(tree.value[order][min(int(np.searchsorted(cum, wet_area)), order.size - 1)])
    return np.maximum(np.float32(L) - tree.value, np.float32(0)).astype(np.float32), L


def tiny_config(seed: int = 1, origin=(0.0, 0.0), shuffle=True) -> Scene:
    fbm = FBm(seed, amplitude=500.0, wavelength=640.0)
    tree = random_split_quadtree(64, 10.0, (0.25, 0.25), fbm, seed, origin=origin,
                                 shuffle=shuffle)
    cam = fixed_camera(tree, fbm, (320.0, 80.0), 300.0, 90.0, -30.0, 60.0, 320, 240,
                       n_cascades=1, cascade_size=256, znear=1.0, zfar=1.0e4)
    return Scene("tiny", tree, fbm, RBF_SIGMA, RBF_RADIUS, [cam])


def precision_config(seed: int = 1) -> Scene:
    s = tiny_config(seed, origin=(5.0e6, 5.0e6))
    s.name = "precision"
    return s


def dem_config(seed: int = 2, n_frames: int = 120, target_leaves: int = 4_500_000,
               root_n: int = 256, cascade_size: int = 2048, width: int = 1920,
               height: int = 1080) -> Scene:
    fbm = FBm(seed, amplitude=2000.0, wavelength=10240.0 * root_n / 256)
    tree = curvature_quadtree(root_n, root_n, 160.0, 4, fbm, target_leaves, seed)
    cams = flight_path(tree, fbm, seed, n_frames, width, height, n_cascades=4,
                       cascade_size=cascade_size, split_lambda=0.5)
    return Scene("dem", tree, fbm, RBF_SIGMA, RBF_RADIUS, cams)


def tiny_flood_config(seed: int = 1, wet_area: float = 0.3) -> Scene:
    s = tiny_config(seed)
    s.name = "tiny_flood"
    s.depth, _ = flood_depths(s.tree, wet_area)
    return s


def flood_config(seed: int = 2, n_frames: int = 120, wet_area: float = 0.2, **kw) -> Scene:
    s = dem_config(seed, n_frames, **kw)
    s.name = "flood"
    s.depth, _ = flood_depths(s.tree, wet_area)
    return s


def _batch_tile(args) -> Scene:
    seed, t, side, amp, n_c, n_tex, width, height, leaf_frac = args
    levels = 4 if side >= 256 else 2
    root_n = max(side >> levels, 1)
    fbm = FBm(seed * 100 + t, amplitude=amp, wavelength=side * 10.0 / 4)
    tree = curvature_quadtree(root_n, root_n, 10.0 * (1 << levels), levels, fbm,
                              max(int(leaf_frac * side * side), root_n * root_n),
                              seed * 100 + t)
    cam = flight_path(tree, fbm, seed * 100 + t, 2, width, height, n_c, n_tex,
                      split_lambda=0.5)[0]
    return Scene(f"tile{t}", tree, fbm, RBF_SIGMA, RBF_RADIUS, [cam])


def parallel_map(fn, items, workers: int | None = None) -> list:
    """map(fn, items) over worker processes started with 'spawn' (safe after
    CUDA has been initialised in the caller); in order, same results as a
    plain map.  workers = 1 runs in this process."""
    import os
    items = list(items)
    if workers is None:
        workers = min(len(items), len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                      else (os.cpu_count() or 1))
    if workers <= 1 or len(items) <= 1:
        return [fn(x) for x in items]
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(fn, items))


def batch_config(seed: int = 4, n_tiles: int = 64, min_side: int = 256,
                 max_side: int = 4096, width: int = 960, height: int = 540,
                 leaf_frac: float = 0.3, workers: int | None = None) -> list:
    """Independent tiles: finest side log-uniform in [min_side, max_side],
    10 m finest cells, curvature refinement to ``leaf_frac`` of the finest
    count, 1-4 cascades of 512^2-2048^2 and one camera each.  Tiles are
    generated in parallel processes (the result does not depend on
    ``workers``)."""
    rng = np.random.default_rng(seed)
    jobs = []
    for t in range(n_tiles):
        side = int(2 ** np.round(rng.uniform(np.log2(min_side), np.log2(max_side))))
        amp = float(rng.uniform(300, 2000))
        n_c = int(rng.integers(1, 5))
        n_tex = int(2 ** rng.integers(9, 12))
        jobs.append((seed, t, side, amp, n_c, n_tex, width, height, leaf_frac))
    # largest tiles first so that the pool ends together
    order = sorted(range(n_tiles), key=lambda t: -jobs[t][2])
    done = parallel_map(_batch_tile, [jobs[t] for t in order], workers)
    scenes = [None] * n_tiles
    for t, sc in zip(order, done):
        scenes[t] = sc
    return scenes


@dataclass
class Request:
    rid: int
    arrival: float        # seconds from the start of the stream
    camera: Camera


def serve_config(seed: int = 5, blocks: int = 4, leaves_per_block: int = 2_500_000,
                 block_root: int = 128, rate: float = 200.0, duration: float = 2.0,
                 cascade_size: int = 2048, workers: int | None = None) -> tuple:
    """(Scene, requests): the resident quadtree and the request stream (the
    blocks of the mosaic are refined in parallel processes)."""
    span = blocks * block_root * 320.0
    fbm = FBm(seed, amplitude=3000.0, wavelength=span / 8)
    tree = tiled_curvature_quadtree(blocks, block_root, 320.0, 5, fbm, leaves_per_block, seed,
                                    pmap=lambda f, xs: parallel_map(f, xs, workers))
    rng = np.random.default_rng(seed)
    n = int(rng.poisson(rate * duration))
    arrivals = np.sort(rng.uniform(0.0, duration, n))
    resolutions = [(1280, 720), (1920, 1080), (3840, 2160)]
    path = flight_path(tree, fbm, seed, max(n, 2), 16, 16, 2, cascade_size, split_lambda=0.5,
                       n_waypoints=12)
    reqs = []
    for k in range(n):
        w, h = resolutions[int(rng.integers(0, 3))]
        cam = path[int(rng.integers(0, len(path)))].with_(width=w, height=h,
                                                          n_cascades=int(rng.integers(2, 7)))
        reqs.append(Request(k, float(arrivals[k]), cam))
    return Scene("serve", tree, fbm, RBF_SIGMA, RBF_RADIUS, []), reqs
