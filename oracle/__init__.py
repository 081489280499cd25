"""Python access to the CPU FP64 oracle (test infrastructure only).

The oracle is a plain C restatement of the paper's method (see
``hf_oracle.c``).  Only ``tests/``, the smoke check and the benchmark's CPU
baseline may import this package; the product library never does.
"""

from __future__ import annotations

import copy
import ctypes as ct
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, "hf_oracle.c")]

MAX_CASCADES = 8
MAX_POLY = 64


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (OpenMP, -O2, no fast-math)."""
    newest = max(os.path.getmtime(p) for p in _SRC + [os.path.join(_HERE, "hf_oracle.h")])
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp] + _SRC + ["-lm"])
        os.replace(tmp, _SO)
    return _SO


class Domain(ct.Structure):
    _fields_ = [("width", ct.c_double), ("height", ct.c_double), ("zmin", ct.c_double),
                ("zmax", ct.c_double), ("c_min", ct.c_double), ("c_max", ct.c_double)]


class CameraC(ct.Structure):
    _fields_ = [("eye", ct.c_double * 3), ("forward", ct.c_double * 3), ("up", ct.c_double * 3),
                ("vfov", ct.c_double), ("znear", ct.c_double), ("zfar", ct.c_double),
                ("width", ct.c_int), ("height", ct.c_int), ("n_cascades", ct.c_int),
                ("cascade_size", ct.c_int), ("split_lambda", ct.c_double),
                ("overlap_frac", ct.c_double), ("texel_ladder", ct.c_int)]


class CascadeC(ct.Structure):
    _fields_ = [("near", ct.c_double), ("far", ct.c_double), ("far_ext", ct.c_double),
                ("n_poly", ct.c_int), ("poly", (ct.c_double * 2) * MAX_POLY),
                ("aabb", ct.c_double * 4), ("snap_x", ct.c_longlong),
                ("snap_y", ct.c_longlong), ("snap_k", ct.c_longlong), ("ox", ct.c_double),
                ("oy", ct.c_double), ("E", ct.c_double), ("h", ct.c_double), ("N", ct.c_int)]

    def polygon(self) -> np.ndarray:
        return np.array([[self.poly[i][0], self.poly[i][1]] for i in range(self.n_poly)])


class ViewC(ct.Structure):
    _fields_ = [("dir2", ct.c_double * 2), ("n", ct.c_double), ("f", ct.c_double),
                ("split", ct.c_double * (MAX_CASCADES + 1)), ("n_hull", ct.c_int),
                ("hull", (ct.c_double * 2) * MAX_POLY), ("n_cascades", ct.c_int),
                ("cas", CascadeC * MAX_CASCADES)]

    def hull_points(self) -> np.ndarray:
        return np.array([[self.hull[i][0], self.hull[i][1]] for i in range(self.n_hull)])


class RCascade(ct.Structure):
    _fields_ = [("ox", ct.c_double), ("oy", ct.c_double), ("h", ct.c_double),
                ("near", ct.c_double), ("far_ext", ct.c_double), ("N", ct.c_int),
                ("stop_level", ct.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ct.CDLL(build())
        d, i, f, L = ct.c_double, ct.c_int, ct.c_float, ct.c_long
        P = ct.POINTER
        _lib.orc_rbf_weight.restype = d
        _lib.orc_rbf_weight.argtypes = [d, d, d, d, i]
        _lib.orc_ray_patch.restype = i
        _lib.orc_ray_patch.argtypes = [d] * 11 + [P(d)]
        _lib.orc_fit.restype = i
        _lib.orc_fit.argtypes = [P(CameraC), P(Domain), P(ViewC)]
        _lib.orc_stop_level.restype = i
        _lib.orc_stop_level.argtypes = [d, d, i, d, d, i]
        _lib.orc_fit_follow.restype = i
        _lib.orc_fit_follow.argtypes = [P(CameraC), P(Domain), P(ct.c_longlong), P(ViewC)]
        _lib.orc_ladder_fit.restype = None
        _lib.orc_ladder_fit.argtypes = [d, d, d, d, d, i, i, P(ct.c_longlong), P(ct.c_longlong),
                                        P(ct.c_longlong), P(d)]
        _lib.orc_frustum_box_vertices.restype = i
        _lib.orc_frustum_box_vertices.argtypes = [P(CameraC), P(Domain), P(d), i]
        _lib.orc_maxmip_size.restype = L
        _lib.orc_maxmip_size.argtypes = [i]
        _lib.orc_threads.restype = i
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ct.POINTER(t))


class Cells:
    """Cell centres, sizes and values of a quadtree's leaves (FP64)."""

    def __init__(self, tree):
        n = tree.n_leaves
        self.n = n
        self.cx = np.empty(n)
        self.cy = np.empty(n)
        self.cs = np.empty(n)
        self.cv = np.empty(n)
        lv = np.ascontiguousarray(tree.level, np.int32)
        ix = np.ascontiguousarray(tree.ix, np.int32)
        iy = np.ascontiguousarray(tree.iy, np.int32)
        val = np.ascontiguousarray(tree.value, np.float32)
        lib().orc_cells_from_leaves(ct.c_double(tree.root_cell), _p(lv, ct.c_int), _p(ix, ct.c_int),
                                    _p(iy, ct.c_int), _p(val, ct.c_float), ct.c_long(n),
                                    _p(self.cx, ct.c_double), _p(self.cy, ct.c_double),
                                    _p(self.cs, ct.c_double), _p(self.cv, ct.c_double))
        self.domain = Domain(tree.width, tree.height, float(self.cv.min()), float(self.cv.max()),
                             float(self.cs.min()), float(self.cs.max()))


GAUSSIAN, WENDLAND_C2 = 0, 1   # weight functions (kernel argument)


def rbf_weight(dist, c, sigma, radius, kernel=GAUSSIAN) -> float:
    return lib().orc_rbf_weight(float(dist), float(c), float(sigma), float(radius), int(kernel))


def rbf_points(cells: Cells, sigma, radius, px, py, mode=1, with_counts=False, kernel=GAUSSIAN):
    px = np.ascontiguousarray(px, np.float64).ravel()
    py = np.ascontiguousarray(py, np.float64).ravel()
    m = px.size
    out = np.empty(m)
    cnt = np.empty(m, np.int32)
    lib().orc_rbf_points(_p(cells.cx, ct.c_double), _p(cells.cy, ct.c_double),
                         _p(cells.cs, ct.c_double), _p(cells.cv, ct.c_double), ct.c_long(cells.n),
                         ct.c_double(sigma), ct.c_double(radius), ct.c_int(kernel),
                         ct.c_double(cells.domain.width), ct.c_double(cells.domain.height),
                         _p(px, ct.c_double), _p(py, ct.c_double), ct.c_long(m), ct.c_int(mode),
                         _p(out, ct.c_double), _p(cnt, ct.c_int))
    return (out, cnt) if with_counts else out


def camera_struct(cam, tree) -> CameraC:
    """Camera in the domain-local frame (the eye's world offset removed in FP64)."""
    eye = (cam.eye[0] - tree.origin_x, cam.eye[1] - tree.origin_y, cam.eye[2])
    return CameraC((ct.c_double * 3)(*eye), (ct.c_double * 3)(*cam.forward),
                   (ct.c_double * 3)(*cam.up), cam.vfov, cam.znear, cam.zfar, cam.width,
                   cam.height, cam.n_cascades, cam.cascade_size, cam.split_lambda,
                   cam.overlap_frac, int(getattr(cam, "texel_ladder", 0)))


def fit(cam, tree, cells: Cells, follow=None) -> ViewC:
    """Section 3 fit; `follow` (ladder steps of an earlier frame's cascades)
    applies the lattice fit's hysteresis."""
    v = ViewC()
    c = camera_struct(cam, tree)
    if follow is not None:
        steps = (ct.c_longlong * MAX_CASCADES)(*([int(x) for x in follow] + [0] * (MAX_CASCADES - len(follow))))
        rc = lib().orc_fit_follow(ct.byref(c), ct.byref(cells.domain), steps, ct.byref(v))
    else:
        rc = lib().orc_fit(ct.byref(c), ct.byref(cells.domain), ct.byref(v))
    if rc != 0:
        raise ValueError("orc_fit rejected the camera")
    return v


def ladder_fit(x0: float, y0: float, x1: float, y1: float, c_min: float, N: int, n: int):
    """Lattice fit of one box: (m, i0, j0, h) with h = c_min 2^(m/n)."""
    m, i0, j0, h = ct.c_longlong(), ct.c_longlong(), ct.c_longlong(), ct.c_double()
    lib().orc_ladder_fit(x0, y0, x1, y1, c_min, N, n, ct.byref(m), ct.byref(i0), ct.byref(j0), ct.byref(h))
    return m.value, i0.value, j0.value, h.value


def frustum_box_vertices(cam, tree, cells: Cells) -> np.ndarray:
    buf = np.empty(3 * 220)
    c = camera_struct(cam, tree)
    n = lib().orc_frustum_box_vertices(ct.byref(c), ct.byref(cells.domain), _p(buf, ct.c_double), 220)
    return buf[: 3 * n].reshape(n, 3)


def _ij(N, ii=None, jj=None):
    if ii is None:
        jj, ii = np.meshgrid(np.arange(N, dtype=np.int32), np.arange(N, dtype=np.int32), indexing="ij")
    return np.ascontiguousarray(ii, np.int32).ravel(), np.ascontiguousarray(jj, np.int32).ravel()


def mask(cas: CascadeC, cells: Cells, ii=None, jj=None):
    ii, jj = _ij(cas.N, ii, jj)
    vis = np.empty(ii.size, np.uint8)
    mg = np.empty(ii.size)
    lib().orc_mask(ct.byref(cas), ct.byref(cells.domain), _p(ii, ct.c_int), _p(jj, ct.c_int),
                   ct.c_long(ii.size), _p(vis, ct.c_uint8), _p(mg, ct.c_double))
    return vis, mg


def texel_heights(cas: CascadeC, cells: Cells, sigma, radius, ii=None, jj=None, kernel=GAUSSIAN) -> np.ndarray:
    ii, jj = _ij(cas.N, ii, jj)
    out = np.empty(ii.size)
    lib().orc_texel_heights(ct.byref(cas), ct.byref(cells.domain), _p(cells.cx, ct.c_double),
                            _p(cells.cy, ct.c_double), _p(cells.cs, ct.c_double),
                            _p(cells.cv, ct.c_double), ct.c_long(cells.n), ct.c_double(sigma),
                            ct.c_double(radius), ct.c_int(kernel), _p(ii, ct.c_int), _p(jj, ct.c_int),
                            ct.c_long(ii.size), _p(out, ct.c_double))
    return out


def depth_cells(cells: Cells, depths) -> Cells:
    """The same cells carrying the water depths (leaf order) as their values."""
    c = copy.copy(cells)
    c.cv = np.ascontiguousarray(np.asarray(depths, np.float32), np.float64)
    return c


def water_heights(cas: CascadeC, cells: Cells, depths, sigma, radius, ii=None, jj=None):
    """Terrain height v, discretized depth d and water surface at texels.

    Section 2: terrain values and relative water depths live on the same
    cells, and both are approximated by Eq. 2 (so with the same weights).
    Reading: the texel's water surface is v + d where d > 0 (some
    influencing cell is wet), else -inf (dry); invisible texels are -inf."""
    v = texel_heights(cas, cells, sigma, radius, ii, jj)
    d = texel_heights(cas, depth_cells(cells, depths), sigma, radius, ii, jj)
    with np.errstate(invalid="ignore"):
        w = np.where(np.isfinite(v) & (d > 0), v + d, -np.inf)
    return v, d, w


def maxmip(tex: np.ndarray) -> np.ndarray:
    tex = np.ascontiguousarray(tex, np.float32)
    N = tex.shape[-1]
    out = np.empty(lib().orc_maxmip_size(N), np.float32)
    lib().orc_maxmip(_p(tex, ct.c_float), ct.c_int(N), _p(out, ct.c_float))
    return out


def mip_levels(mip: np.ndarray, N: int) -> list:
    """Split a flat max mipmap into its levels (level k is (P>>k) x (P>>k))."""
    P = 1
    while P < N - 1:
        P <<= 1
    out, off = [], 0
    while P >= 1:
        out.append(mip[off: off + P * P].reshape(P, P))
        off += P * P
        P >>= 1
    return out


def ray_patch(h00, h10, h01, h11, a0, b0, z0, da, db, dz, dt):
    tau = ct.c_double()
    hit = lib().orc_ray_patch(h00, h10, h01, h11, a0, b0, z0, da, db, dz, dt, ct.byref(tau))
    return (tau.value if hit else None)


def rcascades(cascades) -> "ct.Array":
    """Ray-casting descriptors from objects with ox, oy, h, near, far_ext, N
    and optionally stop_level (coarse-level stop; 0 = the bilinear surface)."""
    arr = (RCascade * len(cascades))()
    for k, c in enumerate(cascades):
        arr[k] = RCascade(c.ox, c.oy, c.h, c.near, c.far_ext, c.N, int(getattr(c, "stop_level", 0)))
    return arr


def stop_level(lod_pixels: float, vfov: float, height: int, near: float, h: float, N: int) -> int:
    """Coarse-level stop level of a cascade (orc_stop_level)."""
    return lib().orc_stop_level(lod_pixels, vfov, height, near, h, N)


def raycast(cam, tree, cascades, textures, mips=None, pixels=None, mode=0, water_textures=None):
    """Cast rays for ``pixels`` (arrays px, py) or the whole image.

    Returns t (world distance), hit (0 miss, 1 + first cascade hit, + 0x80
    when that hit is on the water surface), seg (length of the first-hit
    cascade's ray segment), visits.  mode 0: per-patch DDA; 1: max-mip
    traversal climbing one level per step; 2: climbing at once to the
    coarsest node entered.  ``water_textures`` (one per cascade)
    adds the water surface: inside each cascade the first surface met wins."""
    C = len(cascades)
    rc = rcascades(cascades)
    texs = [np.ascontiguousarray(t, np.float32) for t in textures]
    if mips is None and any(rc[k].stop_level > 0 for k in range(C)):
        if water_textures is not None:
            raise ValueError("the coarse-level stop is defined for the terrain alone")
        mips = [maxmip(t) for t in texs]  # the box field of a coarse-level stop
    tp = (ct.POINTER(ct.c_float) * C)(*[_p(t, ct.c_float) for t in texs])
    if water_textures is not None:
        if mode != 0:
            raise ValueError("the water surface is traced by the DDA (mode 0)")
        wts = [np.ascontiguousarray(t, np.float32) for t in water_textures]
        wp = (ct.POINTER(ct.c_float) * C)(*[_p(t, ct.c_float) for t in wts])
    else:
        wp = None
    if mips is not None:
        ms = [np.ascontiguousarray(m, np.float32) for m in mips]
        mp = (ct.POINTER(ct.c_float) * C)(*[_p(m, ct.c_float) for m in ms])
    else:
        if mode in (1, 2):
            raise ValueError("mip traversal needs the max mipmaps")
        mp = None
    if pixels is None:
        py, px = np.meshgrid(np.arange(cam.height, dtype=np.int32),
                             np.arange(cam.width, dtype=np.int32), indexing="ij")
    else:
        px, py = pixels
    px = np.ascontiguousarray(px, np.int32).ravel()
    py = np.ascontiguousarray(py, np.int32).ravel()
    m = px.size
    t = np.empty(m)
    hit = np.empty(m, np.int32)
    seg = np.empty(m)
    visits = np.empty(m, np.int64)
    c = camera_struct(cam, tree)
    lib().orc_raycast(ct.byref(c), rc, ct.c_int(C), tp, wp, mp, _p(px, ct.c_int), _p(py, ct.c_int),
                      ct.c_long(m), ct.c_int(mode), _p(t, ct.c_double), _p(hit, ct.c_int),
                      _p(seg, ct.c_double), _p(visits, ct.c_longlong))
    return t, hit, seg, visits


def raycast_water(cam, tree, cascades, terrain_textures, water_textures, pixels=None):
    """Terrain and water surface together (t, hit, seg): see ``raycast``."""
    t, hit, seg, _ = raycast(cam, tree, cascades, terrain_textures, pixels=pixels,
                             water_textures=water_textures)
    return t, hit, seg


def maxmip_pair(tex: np.ndarray, wtex: np.ndarray) -> np.ndarray:
    """Max mipmap bounding both surfaces: the entrywise larger of the two
    surfaces' max mipmaps (max commutes with the 2x2 reductions)."""
    return np.maximum(maxmip(tex), maxmip(wtex))


def threads() -> int:
    return lib().orc_threads()
