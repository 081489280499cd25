"""Helpers shared by the GPU parity tests: conversion of the library's
cascade descriptors into oracle inputs, and the comparison rules.

Tolerances (FP32 path):
  heights   |v_gpu - v_ref| <= 1e-5 * max(|v_ref|, A), A = largest |cell value|
  ray t     |t_gpu - t_ref| <= 1e-4 * (length of the ray segment inside the
            first-hit cascade), or 4 FP32 ulps of t where that is larger: t is
            an FP32 number, which cannot come closer than half an ulp to the
            exact hit, so a segment shorter than 2.4e-3 t would ask for more
            than its precision
  hit/miss  at most 0.1 % of pixels differ, and only at silhouettes: pixels
            whose 3x3 reference neighbourhood mixes hit and miss, or whose
            reference t jumps by more than 5 % inside it
  water     the water surface texture: the wet/dry decision (discretized
            depth > 0) may differ only where the oracle's depth is below 1e-6
            of the largest depth (a cell at the truncation radius has a
            weight of order the FP32 exp error there); wet on both sides:
            the height rule above.  Water flag of a hit: see
            check_water_flags.
  grazing   a pixel outside the two rules above is still correct if the
            oracle, run on the same surface raised and lowered by
            delta = 2e-6 * (t + A), brackets it (backward error): a ray that
            skims the surface changes its first hit under any FP32 rounding
            of its direction.  delta covers a lateral ray displacement of
            ~2e-7 t (FP32 direction and exit times) plus ~2e-4 texels (FP32
            texel coordinates) on slopes up to 2, and ~1e-7 (z + t) of ray
            height.  The rule may pass at most EXCUSE_REL of a frame's
            pixels (at least EXCUSE_MIN), so that a regression which turns
            many rays ill-conditioned cannot hide behind it; a hit/miss
            difference off a silhouette passes only through this rule.  With
            the coarse-level stop the surface is a field of flat box tops,
            and a ray that meets a flat top at a shallow angle moves its hit
            by dz / sin(angle) under a rounding dz of its height: such rays
            are far more common than on bilinear patches, and the cap is
            BOX_EXCUSE_REL there.
  mask      identical, except texels whose centre lies within 1e-7 texels of
            a decision boundary (both sides decide in FP64, by different
            formulas); a texel is finite on both sides or on neither, with
            the same exception
  max mip   identical (max is exact)
"""

from __future__ import annotations

from typing import NamedTuple

import numpy as np

HEIGHT_REL = 1e-5
RAY_REL = 1e-4
T_ULPS = 4 * 2.0 ** -24   # four FP32 ulps of t, relative
HIT_MISMATCH = 1e-3
GRAZE_REL = 2e-6
EXCUSE_REL = 1e-5    # share of a frame's pixels the backward-error rule may pass
EXCUSE_MIN = 2       # ... but at least this many pixels in a small frame
BOX_EXCUSE_REL = 1e-4  # the same for the box-field surface of the coarse-level stop
MASK_MARGIN = 1e-7   # texels this close (in texels) to a mask boundary may differ


def ocas(orc, info):
    c = orc.CascadeC()
    c.ox, c.oy, c.h, c.N, c.n_poly = info.ox, info.oy, info.texel, info.N, info.n_poly
    c.E = info.extent
    for k in range(info.n_poly):
        c.poly[k][0], c.poly[k][1] = info.poly[k][0], info.poly[k][1]
    return c


class RC:
    def __init__(self, info):
        self.ox, self.oy, self.h = info.ox, info.oy, info.texel
        self.near, self.far_ext, self.N = info.near, info.far_ext, info.N
        self.stop_level = getattr(info, "stop_level", 0)


def mask_from_spans(spans: np.ndarray, N: int) -> np.ndarray:
    i = np.arange(N)[None, :]
    return (i >= spans[:, 0:1]) & (i <= spans[:, 1:2])


def mask_margin(orc, info, cells):
    """The oracle's visibility mask of a cascade and, per texel, the distance
    (in texels) of its centre from the nearest decision boundary."""
    vis_ref, margin = orc.mask(ocas(orc, info), cells)
    return vis_ref.reshape(info.N, info.N).astype(bool), margin.reshape(info.N, info.N)


def check_mask(orc, info, cells, spans):
    """(texels whose visibility differs from the oracle's away from a
    boundary, the oracle's mask, the texels within MASK_MARGIN of a
    boundary)."""
    vis_ref, margin = mask_margin(orc, info, cells)
    got = mask_from_spans(spans, info.N)
    near = margin <= MASK_MARGIN
    bad = (got != vis_ref) & ~near
    return int(bad.sum()), vis_ref, near


def height_error(tex, ref, amp, exempt=None):
    """Largest |tex - ref| / max(|ref|, amp) over the texels finite on both
    sides.  The finite texels must coincide, except where `exempt` (texels
    within MASK_MARGIN of a mask boundary) is set: a texel defined on one
    side only is an error, not a texel to skip."""
    vis = np.isfinite(ref)
    differ = np.isfinite(tex) != vis
    if exempt is not None:
        differ &= ~exempt
    assert not differ.any(), f"{int(differ.sum())} texels finite on one side only"
    both = vis & np.isfinite(tex)
    rel = np.abs(tex[both].astype(np.float64) - ref[both]) / np.maximum(np.abs(ref[both]), amp)
    return float(rel.max()) if rel.size else 0.0


def silhouettes(hit_ref: np.ndarray, t_ref: np.ndarray) -> np.ndarray:
    H, W = hit_ref.shape
    h = np.pad(hit_ref > 0, 1, mode="edge")
    t = np.pad(np.where(hit_ref > 0, t_ref, np.nan), 1, mode="edge")
    mixed = np.zeros((H, W), bool)
    jump = np.zeros((H, W), bool)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            hn = h[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
            tn = t[1 + dy:1 + dy + H, 1 + dx:1 + dx + W]
            mixed |= hn != (hit_ref > 0)
            with np.errstate(invalid="ignore"):
                jump |= np.abs(tn - t_ref) > 0.05 * t_ref
    return mixed | jump


def surface_bracket(orc, cam, tree, rcs, texs, px, py, delta, water_texs=None):
    """Oracle rays at pixels (px, py) on the surface (both surfaces with the
    water layer) raised and lowered by delta: (t_up, hit_up, t_down, hit_down)."""
    d = np.float32(delta)

    def shift(ts, s):
        return [np.where(np.isfinite(t), t + s * d, t).astype(np.float32) for t in ts]
    out = []
    for sgn in (1, -1):
        if water_texs is None:
            t, h, _, _ = orc.raycast(cam, tree, rcs, shift(texs, sgn), pixels=(px, py))
        else:
            t, h, _ = orc.raycast_water(cam, tree, rcs, shift(texs, sgn), shift(water_texs, sgn), pixels=(px, py))
        out += [t, h]
    return tuple(out)


def ray_scale(seg, t):
    """The length the ray tolerance is relative to: the first-hit cascade's
    segment, at least T_ULPS * t / RAY_REL (see the module docstring)."""
    return np.maximum(np.nan_to_num(seg, nan=0.0), T_ULPS / RAY_REL * np.abs(np.nan_to_num(t, nan=0.0)))


def bracketed(gt, gh, seg, tu, hu, td, hd):
    """True where the result lies between the raised and the lowered
    surface's answers (within the ray tolerance)."""
    tol = RAY_REL * ray_scale(seg, gt)
    hit_ok = (gh > 0) & (hu > 0) & (gt >= tu - tol) & ((hd == 0) | (gt <= td + tol))
    miss_ok = (gh == 0) & (hd == 0)
    return hit_ok | miss_ok


def frame_bracket(orc, cam, tree, rcs, texs, gt, gh, ot, seg, amp, water_texs=None):
    """Callable for check_rays: flat pixel indices -> explained by a surface
    perturbation of size GRAZE_REL * (t + A)."""
    def f(idx):
        px, py = (idx % cam.width).astype(np.int32), (idx // cam.width).astype(np.int32)
        tmax = np.nanmax(np.concatenate([np.where(gh[idx] > 0, gt[idx], np.nan),
                                         np.where(np.isfinite(ot[idx]), ot[idx], np.nan), [0.0]]))
        delta = GRAZE_REL * (tmax + amp)
        tu, hu, td, hd = surface_bracket(orc, cam, tree, rcs, texs, px, py, delta, water_texs)
        return bracketed(gt[idx], gh[idx], seg[idx], tu, hu, td, hd)
    return f


def check_water_flags(orc, cam, tree, rcs, texs, water_texs, gh, oh, seg):
    """Where both sides hit, the water flag (0x80) must agree, except where
    the oracle's terrain and water hits are closer than the ray tolerance
    (a water layer thinner than the comparison can resolve, e.g. at a
    shore where the discretized depth tends to 0).  Returns (mismatches,
    unexplained mismatches)."""
    gh, oh, seg = np.asarray(gh).ravel(), np.asarray(oh).ravel(), np.asarray(seg).ravel()
    both = (gh > 0) & (oh > 0)
    mis = np.nonzero(both & ((gh & 0x80) != (oh & 0x80)))[0]
    if mis.size == 0:
        return 0, 0
    px, py = (mis % cam.width).astype(np.int32), (mis // cam.width).astype(np.int32)
    tt, ht, _, _ = orc.raycast(cam, tree, rcs, texs, pixels=(px, py))
    tw, hw, _, _ = orc.raycast(cam, tree, rcs, water_texs, pixels=(px, py))
    thin = (ht > 0) & (hw > 0) & (np.abs(tw - tt) <= RAY_REL * seg[mis])
    return int(mis.size), int((~thin).sum())


class RayCheck(NamedTuple):
    frac: float       # share of pixels whose hit/miss differs
    off: int          # hit/miss differences explained neither by a silhouette nor by backward error
    terr: float       # worst |dt| / tolerance scale among the pixels not passed by backward error
    errs: np.ndarray  # |dt| / scale of every pixel hit on both sides
    excused: int      # pixels passed by the backward-error rule
    n: int            # pixels compared


def excuse_cap(n: int, rel: float = EXCUSE_REL) -> int:
    """Pixels of an n-pixel frame that the backward-error rule may pass."""
    return max(EXCUSE_MIN, int(rel * n))


def assert_rays(res: RayCheck, what: str = "", excuse_rel: float = EXCUSE_REL) -> None:
    """The ray rules of the module docstring: hit/miss differences at most
    HIT_MISMATCH of the pixels and only at silhouettes (or passed by the
    backward-error rule), t within RAY_REL of its scale, and no more pixels
    passed by the backward-error rule than excuse_cap allows."""
    print(f"rays {what}: {res.n} pixels, hit/miss differ {res.frac:.2e}, off-silhouette {res.off}, "
          f"worst t error {res.terr:.2e}, passed by backward error {res.excused} "
          f"(cap {excuse_cap(res.n, excuse_rel)})")
    assert res.frac <= HIT_MISMATCH and res.off == 0, (what, res.frac, res.off)
    assert res.terr <= RAY_REL, (what, res.terr)
    assert res.excused <= excuse_cap(res.n, excuse_rel), (what, res.excused, excuse_cap(res.n, excuse_rel))


def check_rays(gt, gh, ot, oh, seg, shape=None, silhouette=None, bracket=None) -> RayCheck:
    """Compare a frame's rays with the oracle's (see RayCheck for the fields).
    ``bracket(idx)`` says which of the flat pixel indices idx are explained
    by a perturbation of the surface (grazing rays)."""
    gt, gh, ot, oh, seg = (np.asarray(a).ravel() for a in (gt, gh, ot, oh, seg))
    mism = (gh > 0) != (oh > 0)
    if silhouette is None and shape is not None:
        silhouette = silhouettes(oh.reshape(shape), ot.reshape(shape)).ravel()
    both = (gh > 0) & (oh > 0)
    err = np.zeros(gt.size)
    err[both] = np.abs(gt[both] - ot[both]) / ray_scale(seg[both], ot[both])
    explained = np.zeros(gt.size, bool)
    if bracket is not None:
        idx = np.nonzero(mism | (both & (err > RAY_REL)))[0]
        if idx.size:
            explained[idx] = bracket(idx)
    off = int((mism & ~silhouette & ~explained).sum()) if silhouette is not None else 0
    rest = both & ~explained
    # pixels that pass only through the backward-error rule: t outside its
    # tolerance, or a hit/miss difference that no silhouette explains
    sil = silhouette if silhouette is not None else np.zeros(gt.size, bool)
    excused = explained & ((both & (err > RAY_REL)) | (mism & ~sil))
    return RayCheck(float(mism.mean()), off, (float(err[rest].max()) if rest.any() else 0.0), err[both],
                    int(excused.sum()), int(gt.size))
