"""Seeded quadtree (adaptive grid) layouts with fBm values at the cell centres.

A quadtree heightfield here is a ``root_nx x root_ny`` grid of square root
cells of edge ``root_cell``; a cell at level ``L`` has edge
``root_cell / 2**L`` and integer indices ``(ix, iy)`` on that level's grid.
The leaves tile the domain ``[0, root_nx*root_cell] x [0, root_ny*root_cell]``
(domain-local metres) exactly; the domain's world position is
``(origin_x, origin_y)``.  Every leaf carries one FP32 value, the terrain
height at its centre (Section 2: data are given at the cell centres).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .fbm import FBm


@dataclass
class Quadtree:
    origin_x: float
    origin_y: float
    root_cell: float
    root_nx: int
    root_ny: int
    max_level: int
    level: np.ndarray  # int32 [n]
    ix: np.ndarray     # int32 [n]
    iy: np.ndarray     # int32 [n]
    value: np.ndarray  # float32 [n]

    @property
    def n_leaves(self) -> int:
        return int(self.level.size)

    @property
    def finest_cell(self) -> float:
        return self.root_cell / (1 << self.max_level)

    @property
    def width(self) -> float:
        return self.root_nx * self.root_cell

    @property
    def height(self) -> float:
        return self.root_ny * self.root_cell

    def cell_sizes(self) -> np.ndarray:
        return self.root_cell / np.exp2(self.level.astype(np.float64))

    def level_histogram(self) -> dict:
        lv, cnt = np.unique(self.level, return_counts=True)
        return {int(a): int(b) for a, b in zip(lv, cnt)}


def _values_at_centres(fbm: FBm, level, ix, iy, root_cell) -> np.ndarray:
    c = root_cell / np.exp2(level.astype(np.float64))
    return fbm((ix + 0.5) * c, (iy + 0.5) * c).astype(np.float32)


def _finish(origin, root_cell, nx, ny, max_level, level, ix, iy, value, seed,
            shuffle) -> Quadtree:
    level = np.asarray(level, np.int32)
    ix = np.asarray(ix, np.int32)
    iy = np.asarray(iy, np.int32)
    value = np.asarray(value, np.float32)
    if shuffle:
        perm = np.random.default_rng(seed + 77).permutation(level.size)
        level, ix, iy, value = level[perm], ix[perm], iy[perm], value[perm]
    return Quadtree(float(origin[0]), float(origin[1]), float(root_cell), int(nx),
                    int(ny), int(max_level), level, ix, iy, value)


def random_split_quadtree(root_n: int, root_cell: float, split_fracs, fbm: FBm,
                          seed: int, origin=(0.0, 0.0), shuffle=True) -> Quadtree:
    """Root grid ``root_n x root_n``; at each level a seeded fraction of the
    current leaves is split (e.g. 25 % of the root cells, then 25 % of their
    children)."""
    rng = np.random.default_rng(seed)
    max_level = len(split_fracs)
    lv_out, ix_out, iy_out = [], [], []
    iy, ix = np.meshgrid(np.arange(root_n), np.arange(root_n), indexing="ij")
    ix, iy = ix.ravel(), iy.ravel()
    for L in range(max_level + 1):
        if L < max_level:
            split = rng.random(ix.size) < split_fracs[L]
        else:
            split = np.zeros(ix.size, bool)
        keep = ~split
        lv_out.append(np.full(int(keep.sum()), L))
        ix_out.append(ix[keep])
        iy_out.append(iy[keep])
        sx, sy = ix[split], iy[split]
        ix = np.concatenate([2 * sx, 2 * sx + 1, 2 * sx, 2 * sx + 1])
        iy = np.concatenate([2 * sy, 2 * sy, 2 * sy + 1, 2 * sy + 1])
    level = np.concatenate(lv_out)
    ixa = np.concatenate(ix_out)
    iya = np.concatenate(iy_out)
    value = _values_at_centres(fbm, level, ixa, iya, root_cell)
    return _finish(origin, root_cell, root_n, root_n, max_level, level, ixa, iya,
                   value, seed, shuffle)


def _block_max(a: np.ndarray, b: int) -> np.ndarray:
    ny, nx = a.shape
    return a.reshape(ny // b, b, nx // b, b).max(axis=(1, 3))


def curvature_quadtree(root_nx: int, root_ny: int, root_cell: float, max_level: int,
                       fbm: FBm, target_leaves: int, seed: int,
                       origin=(0.0, 0.0), shuffle=False, fbm_offset=(0.0, 0.0)) -> Quadtree:
    """Refine a node wherever the largest |Laplacian| of the terrain over its
    footprint exceeds one threshold; the threshold is bisected so that the
    leaf count is close to ``target_leaves``.  The terrain is sampled at
    ``fbm_offset`` + domain-local coordinates."""
    fine = 1 << max_level
    fnx, fny = root_nx * fine, root_ny * fine
    cf = root_cell / fine
    xs = fbm_offset[0] + (np.arange(fnx) + 0.5) * cf
    ys = fbm_offset[1] + (np.arange(fny) + 0.5) * cf
    h = fbm.grid(xs, ys)
    hp = np.pad(h, 1, mode="edge")
    lap = np.abs(hp[1:-1, 2:] + hp[1:-1, :-2] + hp[2:, 1:-1] + hp[:-2, 1:-1]
                 - 4.0 * h) / (cf * cf)
    bmax = [_block_max(lap, 1 << (max_level - L)) for L in range(max_level)]

    def layout(tau):
        exists = np.ones((root_ny, root_nx), bool)
        leaves = []
        for L in range(max_level):
            split = exists & (bmax[L] > tau)
            leaves.append(exists & ~split)
            exists = np.repeat(np.repeat(split, 2, axis=0), 2, axis=1)
        leaves.append(exists)
        return leaves

    lo, hi = np.log(max(lap.min(), 1e-30)), np.log(lap.max() + 1e-30)
    best = None
    for _ in range(48):
        mid = 0.5 * (lo + hi)
        leaves = layout(np.exp(mid))
        n = sum(int(m.sum()) for m in leaves)
        if best is None or abs(n - target_leaves) < abs(best[0] - target_leaves):
            best = (n, leaves)
        if abs(n - target_leaves) <= 0.002 * target_leaves:
            break
        if n > target_leaves:
            lo = mid
        else:
            hi = mid
    leaves = best[1]
    lv_out, ix_out, iy_out, val_out = [], [], [], []
    for L, m in enumerate(leaves):
        iy, ix = np.nonzero(m)
        lv_out.append(np.full(ix.size, L))
        ix_out.append(ix)
        iy_out.append(iy)
        if L == max_level:
            val_out.append(h[iy, ix].astype(np.float32))
        else:
            c = root_cell / (1 << L)
            val_out.append(fbm(fbm_offset[0] + (ix + 0.5) * c,
                               fbm_offset[1] + (iy + 0.5) * c).astype(np.float32))
    return _finish(origin, root_cell, root_nx, root_ny, max_level,
                   np.concatenate(lv_out), np.concatenate(ix_out),
                   np.concatenate(iy_out), np.concatenate(val_out), seed, shuffle)


def _mosaic_block(args):
    block_root, root_cell, max_level, fbm, leaves_per_block, seed, blocks, bx, by = args
    span = block_root * root_cell
    t = curvature_quadtree(block_root, block_root, root_cell, max_level, fbm,
                           leaves_per_block, seed + by * blocks + bx,
                           fbm_offset=(bx * span, by * span))
    shift = (block_root << t.level.astype(np.int64))
    return t.level, t.ix + bx * shift, t.iy + by * shift, t.value


def tiled_curvature_quadtree(blocks: int, block_root: int, root_cell: float, max_level: int,
                             fbm: FBm, leaves_per_block: int, seed: int, pmap=None) -> Quadtree:
    """A blocks x blocks mosaic of curvature-refined blocks of one continuous
    terrain (each block refined with its own threshold), for domains too
    large to sample at the finest level at once.  ``pmap(fn, items)`` maps
    the blocks (e.g. over processes); default: in this process."""
    jobs = [(block_root, root_cell, max_level, fbm, leaves_per_block, seed, blocks, bx, by)
            for by in range(blocks) for bx in range(blocks)]
    parts = (pmap or (lambda f, xs: [f(x) for x in xs]))(_mosaic_block, jobs)
    level = np.concatenate([p[0] for p in parts])
    ix = np.concatenate([p[1] for p in parts])
    iy = np.concatenate([p[2] for p in parts])
    value = np.concatenate([p[3] for p in parts])
    return _finish((0.0, 0.0), root_cell, blocks * block_root, blocks * block_root, max_level,
                   level, ix, iy, value, seed, False)
