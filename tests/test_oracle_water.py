"""Pins of the oracle's water layer (Section 2: terrain values and relative
water depths at the cells of one adaptive grid, both approximated by Eq. 2).

Reading pinned here: the discretized depth uses the terrain's RBF weights, the
water surface is terrain + depth where that depth is positive (else dry), and
inside each cascade a ray stops at whichever surface it meets first (flag
0x80 for water).  Pins: zero depth is dry everywhere; a constant depth D lifts
the surface by exactly D (partition of unity); a "bathtub" flood (depth =
max(L - v, 0)) is never below L and equals L where a texel's whole stencil is
wet; flat terrain and flat water give the closed-form plane hits; a half-wet
flat field keeps the water hit on the wet side and the terrain hit on the dry
side; on rough terrain with a flood level the first hit is the first crossing
of the upper envelope of both surfaces found by dense marching.
"""

import numpy as np
import pytest

from test_oracle_render import _look_at_rays, _one_cascade_scene, _scene_camera


def _tiny_cascade(orc, tiny):
    cells = orc.Cells(tiny.tree)
    view = orc.fit(tiny.cameras[0], tiny.tree, cells)
    return cells, view.cas[0]


def test_zero_depth_is_dry(orc, tiny):
    cells, cas = _tiny_cascade(orc, tiny)
    v, d, w = orc.water_heights(cas, cells, np.zeros(cells.n), tiny.sigma, tiny.radius)
    vis = np.isfinite(v)
    assert vis.sum() > 1000
    assert np.all(d[vis] == 0.0)
    assert np.all(w == -np.inf)


@pytest.mark.parametrize("D", [0.25, 3.0, 40.0])
def test_constant_depth_lifts_the_surface_exactly(orc, tiny, D):
    cells, cas = _tiny_cascade(orc, tiny)
    v, d, w = orc.water_heights(cas, cells, np.full(cells.n, D), tiny.sigma, tiny.radius)
    vis = np.isfinite(v)
    assert np.max(np.abs(d[vis] - D)) <= 1e-12 * D * 10
    assert np.max(np.abs(w[vis] - (v[vis] + D))) <= 1e-9 * np.abs(v[vis]).max()
    assert np.all(w[~vis] == -np.inf)


def test_bathtub_flood_level(orc, tiny):
    cells, cas = _tiny_cascade(orc, tiny)
    L = float(np.quantile(cells.cv, 0.3))
    depth = np.maximum(L - cells.cv, 0.0).astype(np.float32)
    v, d, w = orc.water_heights(cas, cells, depth, tiny.sigma, tiny.radius)
    wet = np.isfinite(w)
    assert 0.05 < wet.mean() < 0.95
    # depths are FP32 inputs, so v_i + d_i = L only up to their rounding
    tol = 2.0 ** -23 * (abs(L) + float(depth.max()))
    # v + d averages max(v_i, L) with the RBF weights: never below L
    assert np.all(w[wet] >= L - tol)
    flat = wet & (np.abs(w - L) <= tol)
    assert flat.sum() > 100                     # lake interiors sit at the level
    assert np.all(v[flat] < L)
    # dry texels: no wet cell reaches them, so their terrain is not below the
    # level anywhere in the stencil -- in particular v >= L there
    dry = np.isfinite(v) & ~wet
    assert dry.sum() > 100 and np.all(v[dry] >= L - tol)


def _plane_t(cam, tiny, z):
    py, px = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    eye, d = _look_at_rays(cam, tiny.tree, px.ravel().astype(float), py.ravel().astype(float))
    t = (eye[2] - z) / (-d[:, 2])
    return t, eye[None, :] + t[:, None] * d, d


def test_flat_water_plane_hit(orc, tiny):
    N = 33
    terrain, cas = _one_cascade_scene(N, 0, flat=12.5)
    water = np.full_like(terrain, 12.5 + 1.75)
    cam = _scene_camera(tiny, (32.0, -20.0, 60.0), (0.0, 1.0, -0.9))
    t, hit, _ = orc.raycast_water(cam, tiny.tree, [cas], [terrain], [water])
    tp, P, d = _plane_t(cam, tiny, 14.25)
    ext = (N - 1) * cas.h
    inside = (d[:, 2] < 0) & (P[:, 0] > 1e-6) & (P[:, 0] < ext - 1e-6) & (P[:, 1] > 1e-6) & (P[:, 1] < ext - 1e-6)
    assert inside.sum() > 500
    assert np.all(hit[inside] & 0x80)
    assert np.max(np.abs(t[inside] - tp[inside])) < 1e-9 * tp[inside].max()
    # without water the same rays reach the terrain plane, unflagged
    t0, h0, _ = orc.raycast_water(cam, tiny.tree, [cas], [terrain], [np.full_like(terrain, -np.inf)])
    tq, Q, _ = _plane_t(cam, tiny, 12.5)
    ins0 = (d[:, 2] < 0) & (Q[:, 0] > 1e-6) & (Q[:, 0] < ext - 1e-6) & (Q[:, 1] > 1e-6) & (Q[:, 1] < ext - 1e-6)
    assert np.all((h0[ins0] > 0) & (h0[ins0] & 0x80 == 0))
    assert np.max(np.abs(t0[ins0] - tq[ins0])) < 1e-9 * tq[ins0].max()


def test_half_wet_field_keeps_the_nearer_surface(orc, tiny):
    N = 33
    terrain, cas = _one_cascade_scene(N, 0, flat=12.5)
    water = np.full_like(terrain, 14.25)
    x0 = 16                                      # texel columns < x0 wet
    water[:, x0:] = -np.inf
    cam = _scene_camera(tiny, (32.0, -20.0, 60.0), (0.0, 1.0, -0.9))
    t, hit, _ = orc.raycast_water(cam, tiny.tree, [cas], [terrain], [water])
    tw, Pw, d = _plane_t(cam, tiny, 14.25)
    tt, Pt, _ = _plane_t(cam, tiny, 12.5)
    ext = (N - 1) * cas.h
    in_w = (d[:, 2] < 0) & (Pw[:, 0] > 1e-6) & (Pw[:, 0] < (x0 - 1) * cas.h - 1e-6) & (Pw[:, 1] > 1e-6) & (Pw[:, 1] < ext - 1e-6)
    # dry side: the ray's water-plane point and its terrain point both lie in dry columns
    in_t = (d[:, 2] < 0) & (Pw[:, 0] > (x0 - 1) * cas.h + 1e-6) & (Pt[:, 0] < ext - 1e-6) & (Pt[:, 1] > 1e-6) & (Pt[:, 1] < ext - 1e-6) & (Pw[:, 1] > 1e-6)
    assert in_w.sum() > 100 and in_t.sum() > 100
    assert np.all(hit[in_w] & 0x80)
    assert np.max(np.abs(t[in_w] - tw[in_w])) < 1e-9 * tw.max()
    assert np.all((hit[in_t] > 0) & (hit[in_t] & 0x80 == 0))
    assert np.max(np.abs(t[in_t] - tt[in_t])) < 1e-9 * tt.max()


def _water_bilinear(wtex, cas, x, y):
    """Water surface height, -inf where the containing patch has a dry corner."""
    u, v = (x - cas.ox) / cas.h, (y - cas.oy) / cas.h
    N = wtex.shape[0]
    ok = (u >= 0) & (u <= N - 1) & (v >= 0) & (v <= N - 1)
    i = np.clip(np.floor(u).astype(int), 0, N - 2)
    j = np.clip(np.floor(v).astype(int), 0, N - 2)
    c = np.stack([wtex[j, i], wtex[j, i + 1], wtex[j + 1, i], wtex[j + 1, i + 1]])
    ok &= np.all(np.isfinite(c), axis=0)
    a, b = u - i, v - j
    cz = np.where(np.isfinite(c), c, 0.0)
    h = cz[0] * (1 - a) * (1 - b) + cz[1] * a * (1 - b) + cz[2] * (1 - a) * b + cz[3] * a * b
    return np.where(ok, h, -np.inf)


@pytest.mark.parametrize("seed", [0, 1])
def test_union_matches_dense_marching(orc, tiny, seed):
    """Terrain plus a flat water level over the texels below it: the first
    hit equals the first crossing of the upper envelope of both surfaces
    found by dense marching and bisection, and the flag says which surface
    forms the envelope there."""
    from test_oracle_render import _bilinear
    N = 33
    tex, cas = _one_cascade_scene(N, seed)
    level = float(np.quantile(tex, 0.55))
    wtex = np.where(tex < level, np.float32(level), np.float32(-np.inf)).astype(np.float32)
    eyes = [(32.0, -25.0, 70.0), (-10.0, 30.0, 45.0)]
    fwds = [(0.1, 1.0, -0.6), (1.0, 0.2, -0.35)]
    cam = _scene_camera(tiny, eyes[seed], fwds[seed])
    t, hit, _ = orc.raycast_water(cam, tiny.tree, [cas], [tex], [wtex])
    py, px = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    eye, d = _look_at_rays(cam, tiny.tree, px.ravel().astype(float), py.ravel().astype(float))
    fd = d @ (np.array(cam.forward) / np.linalg.norm(cam.forward))
    ts = np.linspace(0.0, 400.0, 40001)

    def env(x, y):
        return np.maximum(_bilinear(tex, cas, x, y), _water_bilinear(wtex, cas, x, y))
    agree, skipped, wet = 0, 0, 0
    for q in range(d.shape[0]):
        tt = ts[ts >= cam.znear / fd[q]]
        P = eye + tt[:, None] * d[q]
        f = env(P[:, 0], P[:, 1]) - P[:, 2]
        pos = np.nonzero(f >= 0)[0]
        fin = np.isfinite(f)
        if pos.size == 0:
            if fin.any() and f[fin].max() > -1e-3:
                skipped += 1
                continue
            assert hit[q] == 0
            agree += 1
            continue
        k = pos[0]
        if k == 0 or not np.isfinite(f[k - 1]):
            skipped += 1
            continue
        lo, hi = tt[k - 1], tt[k]
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            Pm = eye + mid * d[q]
            fm = env(np.array([Pm[0]]), np.array([Pm[1]]))[0] - Pm[2]
            lo, hi = (mid, hi) if fm < 0 else (lo, mid)
        th = 0.5 * (lo + hi)
        Ph = eye + hi * d[q]
        on_water = _water_bilinear(wtex, cas, np.array([Ph[0]]), np.array([Ph[1]]))[0] >= \
            _bilinear(tex, cas, np.array([Ph[0]]), np.array([Ph[1]]))[0]
        assert hit[q] & 0x7F == 1
        assert bool(hit[q] & 0x80) == bool(on_water), q
        assert t[q] == pytest.approx(th, abs=1e-7 * hi + 1e-9)
        agree += 1
        wet += bool(on_water)
    assert agree > 0.95 * d.shape[0] and skipped < 0.05 * d.shape[0]
    assert wet > 0.05 * agree
