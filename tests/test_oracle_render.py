"""Pins of the oracle's maximum mipmap and ray caster (Section 5).

The max mipmap is checked against numpy reductions of the same definition;
the ray/bilinear-patch root against closed forms (hyperbolic paraboloid,
plane) and bisection; the whole ray caster against dense ray marching with
rays built from an independently written look-at / perspective unprojection,
and the DDA against the max-mip traversal.
"""

import math

import numpy as np
import pytest


def _patch_max(tex):
    N = tex.shape[0]
    c = np.stack([tex[:-1, :-1], tex[:-1, 1:], tex[1:, :-1], tex[1:, 1:]])
    m = c.max(0)
    m[~np.all(np.isfinite(c), axis=0)] = -np.inf
    P = 1
    while P < N - 1:
        P *= 2
    out = np.full((P, P), -np.inf, np.float32)
    out[: N - 1, : N - 1] = m
    return out


@pytest.mark.parametrize("N", [2, 3, 16, 17, 33, 100])
def test_maxmip_matches_block_maxima(orc, N):
    rng = np.random.default_rng(N)
    tex = rng.normal(100, 30, (N, N)).astype(np.float32)
    tex[rng.random((N, N)) < 0.1] = -np.inf
    mip = orc.maxmip(tex)
    levels = orc.mip_levels(mip, N)
    l0 = _patch_max(tex)
    assert np.array_equal(levels[0], l0)
    P = l0.shape[0]
    for k, lv in enumerate(levels):
        b = 1 << k
        ref = l0.reshape(P // b, b, P // b, b).max(axis=(1, 3))
        assert np.array_equal(lv, ref)
        if k:
            prev = levels[k - 1]
            for dy in (0, 1):
                for dx in (0, 1):
                    assert np.all(lv >= prev[dy::2, dx::2])
    fin = l0[np.isfinite(l0)]
    assert levels[-1][0, 0] == (fin.max() if fin.size else -np.inf)


def test_ray_patch_hyperbolic_paraboloid(orc):
    """h = a x y on the unit patch (corners 0, 0, 0, a); a vertical ray at
    (x, y) from height z0 hits at depth z0 - a x y."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        a = rng.uniform(-5, 5)
        x, y = rng.uniform(0, 1, 2)
        z0 = max(a, 0) + rng.uniform(0.1, 3)
        tau = orc.ray_patch(0.0, 0.0, 0.0, a, x, y, z0, 0.0, 0.0, -1.0, 10.0)
        assert tau == pytest.approx(z0 - a * x * y, abs=1e-12)


def test_ray_patch_plane_and_start_under_surface(orc):
    # tilted plane h = 1 + 2a + 3b; ray from (0,0,10) along (0.5, 0.25, -1)
    h00, h10, h01, h11 = 1.0, 3.0, 4.0, 6.0
    tau = orc.ray_patch(h00, h10, h01, h11, 0.0, 0.0, 10.0, 0.5, 0.25, -1.0, 5.0)
    # 10 - t = 1 + 2 (0.5 t) + 3 (0.25 t)  ->  t = 9 / 2.75
    assert tau == pytest.approx(9.0 / 2.75, rel=1e-14)
    assert orc.ray_patch(h00, h10, h01, h11, 0.2, 0.2, 0.5, 0.1, 0.1, 1.0, 1.0) == 0.0
    # ray above and rising: no hit
    assert orc.ray_patch(h00, h10, h01, h11, 0.0, 0.0, 10.0, 0.1, 0.1, 0.5, 1.0) is None
    # hit beyond the segment end: no hit in this patch
    assert orc.ray_patch(h00, h10, h01, h11, 0.0, 0.0, 10.0, 0.5, 0.25, -1.0, 3.0) is None


def test_ray_patch_matches_bisection(orc):
    rng = np.random.default_rng(8)
    checked = 0
    for _ in range(2000):
        h = rng.uniform(0, 10, 4)
        a0, b0 = rng.uniform(0, 1, 2)
        da, db = rng.uniform(-1, 1, 2)
        dz = rng.uniform(-8, 2)
        z0 = rng.uniform(0, 12)
        dt = 1.0
        ts = np.linspace(0, dt, 20001)
        a, b = a0 + ts * da, b0 + ts * db
        H = h[0] * (1 - a) * (1 - b) + h[1] * a * (1 - b) + h[2] * (1 - a) * b + h[3] * a * b
        f = H - (z0 + ts * dz)
        tau = orc.ray_patch(*h, a0, b0, z0, da, db, dz, dt)
        pos = np.nonzero(f >= 0)[0]
        if f[0] >= 0:
            assert tau == 0.0
            continue
        if pos.size == 0:
            if f.max() < -1e-6:
                assert tau is None
            continue
        k = pos[0]
        if f[max(k - 1, 0)] > -1e-9 or (k + 1 < f.size and f[k + 1] < 0 and f[k] < 1e-9):
            continue  # grazing: skip
        lo, hi = ts[k - 1], ts[k]
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            am, bm = a0 + mid * da, b0 + mid * db
            fm = (h[0] * (1 - am) * (1 - bm) + h[1] * am * (1 - bm) + h[2] * (1 - am) * bm
                  + h[3] * am * bm) - (z0 + mid * dz)
            lo, hi = (mid, hi) if fm < 0 else (lo, mid)
        assert tau is not None and tau == pytest.approx(0.5 * (lo + hi), abs=1e-9)
        checked += 1
    assert checked > 400


# --- camera-level checks --------------------------------------------------

def _look_at_rays(cam, tree, px, py):
    """Pixel-centre rays from a look-at view matrix and a perspective
    projection, unprojected with a matrix inverse."""
    eye = np.array([cam.eye[0] - tree.origin_x, cam.eye[1] - tree.origin_y, cam.eye[2]])
    f = np.array(cam.forward, float)
    f /= np.linalg.norm(f)
    s = np.cross(f, np.array(cam.up, float))
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    V = np.eye(4)
    V[0, :3], V[1, :3], V[2, :3] = s, u, -f
    V[:3, 3] = -V[:3, :3] @ eye
    aspect = cam.width / cam.height
    g = 1.0 / math.tan(cam.vfov / 2)
    n, fa = cam.znear, cam.zfar
    Pm = np.array([[g / aspect, 0, 0, 0], [0, g, 0, 0],
                   [0, 0, (fa + n) / (n - fa), 2 * fa * n / (n - fa)], [0, 0, -1, 0]])
    inv = np.linalg.inv(Pm @ V)
    x_ndc = 2 * (px + 0.5) / cam.width - 1
    y_ndc = 1 - 2 * (py + 0.5) / cam.height
    pts = []
    for z in (-1.0, 1.0):
        c = np.stack([x_ndc, y_ndc, np.full_like(x_ndc, z), np.ones_like(x_ndc)])
        w = inv @ c
        pts.append((w[:3] / w[3]).T)
    d = pts[1] - pts[0]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return eye, d


def _bilinear(tex, cas, x, y):
    u = (x - cas.ox) / cas.h
    v = (y - cas.oy) / cas.h
    N = tex.shape[0]
    ok = (u >= 0) & (u <= N - 1) & (v >= 0) & (v <= N - 1)
    i = np.clip(np.floor(u).astype(int), 0, N - 2)
    j = np.clip(np.floor(v).astype(int), 0, N - 2)
    a, b = u - i, v - j
    h = (tex[j, i] * (1 - a) * (1 - b) + tex[j, i + 1] * a * (1 - b) + tex[j + 1, i] * (1 - a) * b
         + tex[j + 1, i + 1] * a * b)
    return np.where(ok, h, -np.inf)


class _Cas:
    def __init__(self, ox, oy, h, near, far_ext, N):
        self.ox, self.oy, self.h, self.near, self.far_ext, self.N = ox, oy, h, near, far_ext, N


def _one_cascade_scene(N, seed, flat=None):
    rng = np.random.default_rng(seed)
    h = 2.0
    if flat is not None:
        tex = np.full((N, N), flat, np.float32)
    else:
        x = np.arange(N) * h
        tex = (20 + 8 * np.sin(x[None, :] / 7.0) * np.cos(x[:, None] / 5.0)
               + rng.normal(0, 1.5, (N, N))).astype(np.float32)
    cas = _Cas(0.0, 0.0, h, -1e9, 1e9, N)
    return tex, cas


def _scene_camera(tiny, eye, fwd, w=48, h=36):
    cam = tiny.cameras[0].with_(eye=(tiny.tree.origin_x + eye[0], tiny.tree.origin_y + eye[1], eye[2]),
                                forward=fwd, width=w, height=h, n_cascades=1)
    return cam


def test_flat_field_plane_hit(orc, tiny):
    """Flat heightfield h0: t = (o_z - h0) / (-d_z) for every downward ray
    that meets the plane inside the texture."""
    N = 33
    tex, cas = _one_cascade_scene(N, 0, flat=12.5)
    cam = _scene_camera(tiny, (32.0, -20.0, 60.0), (0.0, 1.0, -0.9))
    t, hit, _, _ = orc.raycast(cam, tiny.tree, [cas], [tex])
    py, px = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    eye, d = _look_at_rays(cam, tiny.tree, px.ravel().astype(float), py.ravel().astype(float))
    tp = (eye[2] - 12.5) / (-d[:, 2])
    P = eye + tp[:, None] * d
    inside = (d[:, 2] < 0) & (P[:, 0] >= 0) & (P[:, 0] <= (N - 1) * 2.0) & (P[:, 1] >= 0) & (P[:, 1] <= (N - 1) * 2.0)
    margin = (P[:, 0] > 1e-6) & (P[:, 0] < 64 - 1e-6) & (P[:, 1] > 1e-6) & (P[:, 1] < 64 - 1e-6)
    assert inside.sum() > 500
    assert np.array_equal(hit[margin] > 0, inside[margin])
    assert np.max(np.abs(t[inside & margin] - tp[inside & margin])) < 1e-9 * tp.max()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_raycast_matches_dense_marching(orc, tiny, seed):
    """First hit from the DDA = first sign change of bilinear(x(t)) - z(t)
    found by dense marching plus bisection, rays unprojected independently."""
    N = 33
    tex, cas = _one_cascade_scene(N, seed)
    eyes = [(32.0, -25.0, 70.0), (-10.0, 30.0, 45.0), (30.0, 30.0, 90.0)]
    fwds = [(0.1, 1.0, -0.6), (1.0, 0.2, -0.35), (0.2, 0.3, -1.0)]
    cam = _scene_camera(tiny, eyes[seed], fwds[seed])
    t, hit, _, _ = orc.raycast(cam, tiny.tree, [cas], [tex])
    py, px = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    eye, d = _look_at_rays(cam, tiny.tree, px.ravel().astype(float), py.ravel().astype(float))
    fd = d @ (np.array(cam.forward) / np.linalg.norm(cam.forward))
    ts = np.linspace(0.0, 400.0, 40001)
    agree, skipped = 0, 0
    for q in range(d.shape[0]):
        tt = ts[ts >= cam.znear / fd[q]]
        P = eye + tt[:, None] * d[q]
        f = _bilinear(tex, cas, P[:, 0], P[:, 1]) - P[:, 2]
        pos = np.nonzero(f >= 0)[0]
        fin = np.isfinite(f)
        if pos.size == 0:
            if fin.any() and f[fin].max() > -1e-3:
                skipped += 1          # grazing
                continue
            assert hit[q] == 0
            agree += 1
            continue
        k = pos[0]
        if k == 0 or not np.isfinite(f[k - 1]):
            skipped += 1              # starts under the surface / enters it from the side
            continue
        lo, hi = tt[k - 1], tt[k]
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            Pm = eye + mid * d[q]
            fm = _bilinear(tex, cas, np.array([Pm[0]]), np.array([Pm[1]]))[0] - Pm[2]
            lo, hi = (mid, hi) if fm < 0 else (lo, mid)
        assert hit[q] == 1
        assert t[q] == pytest.approx(0.5 * (lo + hi), abs=1e-7 * hi + 1e-9)
        agree += 1
    assert agree > 0.97 * d.shape[0] and skipped < 0.03 * d.shape[0]


def test_dda_equals_mip_traversal_tiny_scene(orc, tiny):
    """Empty-space skipping must not change the first hit (Section 5): the
    max-mip traversal and the per-patch DDA agree on the tiny workload, and
    the traversal tests far fewer nodes."""
    cells = orc.Cells(tiny.tree)
    cam = tiny.cameras[0].with_(n_cascades=3, cascade_size=128)
    v = orc.fit(cam, tiny.tree, cells)
    casl, texs, mips = [], [], []
    for k in range(v.n_cascades):
        c = v.cas[k]
        tex = orc.texel_heights(c, cells, tiny.sigma, tiny.radius).reshape(c.N, c.N).astype(np.float32)
        casl.append(c)
        texs.append(tex)
        mips.append(orc.maxmip(tex))
    t0, h0, s0, v0 = orc.raycast(cam, tiny.tree, casl, texs, mode=0)
    t1, h1, s1, v1 = orc.raycast(cam, tiny.tree, casl, texs, mips, mode=1)
    assert np.array_equal(h0, h1)
    both = h0 > 0
    assert both.mean() > 0.3
    assert np.max(np.abs(t0[both] - t1[both]) / s0[both]) < 1e-9
    assert v1.sum() < v0.sum()


def test_blend_is_continuous_across_overlap(orc, tiny):
    """Reading of the overlap blend: t varies continuously down each image
    column, also where the first-hit cascade changes."""
    cells = orc.Cells(tiny.tree)
    cam = tiny.cameras[0].with_(n_cascades=3, cascade_size=256, overlap_frac=0.1)
    v = orc.fit(cam, tiny.tree, cells)
    casl, texs = [], []
    for k in range(v.n_cascades):
        c = v.cas[k]
        casl.append(c)
        texs.append(orc.texel_heights(c, cells, tiny.sigma, tiny.radius).reshape(c.N, c.N).astype(np.float32))
    t, hit, _, _ = orc.raycast(cam, tiny.tree, casl, texs)
    T = t.reshape(cam.height, cam.width)
    Hh = hit.reshape(cam.height, cam.width)
    both = (Hh[1:] > 0) & (Hh[:-1] > 0)
    rel = np.abs(T[1:] - T[:-1]) / np.minimum(T[1:], T[:-1])
    change = both & (Hh[1:] != Hh[:-1])
    same = both & (Hh[1:] == Hh[:-1])
    assert change.sum() > 50
    assert np.percentile(rel[change], 99) < 4 * np.percentile(rel[same], 99)


def test_blend_closed_form(orc, tiny):
    """Two cascades over the same square holding flat planes at z1 > z2,
    bands [1, 200] and [150, inf): a ray whose first hit (plane z1, cascade
    0) projects to depth s in the overlap [150, 200] returns
    (1 - a) t1 + a t2 with a = (s - 150) / 50, t1, t2 the closed-form plane
    hits (the blend weight grows linearly with the projected depth across the
    overlap band, from 0 where the next cascade starts to 1 at the end of the
    band); before the overlap t1, cascade 0 reported."""
    N = 33
    z1, z2 = 12.5, 11.0
    tex1, _ = _one_cascade_scene(N, 0, flat=z1)
    tex2, _ = _one_cascade_scene(N, 0, flat=z2)
    near0, far0, near1 = 1.0, 200.0, 150.0
    c0 = _Cas(0.0, 0.0, 12.0, near0, far0, N)
    c1 = _Cas(0.0, 0.0, 12.0, near1, 1e9, N)
    cam = _scene_camera(tiny, (192.0, -60.0, 120.0), (0.0, 1.0, -0.55), w=64, h=48)
    t, hit, _, _ = orc.raycast(cam, tiny.tree, [c0, c1], [tex1, tex2])
    py, px = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    eye, d = _look_at_rays(cam, tiny.tree, px.ravel().astype(float), py.ravel().astype(float))
    f = np.array(cam.forward, float)
    dir2 = f[:2] / np.linalg.norm(f[:2])
    ks = d[:, :2] @ dir2
    t1 = (eye[2] - z1) / (-d[:, 2])
    t2 = (eye[2] - z2) / (-d[:, 2])
    P1 = eye + t1[:, None] * d
    P2 = eye + t2[:, None] * d
    ext = (N - 1) * 12.0
    inside = lambda P: (P[:, 0] > 1e-6) & (P[:, 0] < ext - 1e-6) & (P[:, 1] > 1e-6) & (P[:, 1] < ext - 1e-6)
    s1 = t1 * ks
    a = np.clip((s1 - near1) / (far0 - near1), 0.0, 1.0)
    band = (d[:, 2] < 0) & inside(P1) & inside(P2) & (s1 > near1 + 1e-6) & (s1 < far0 - 1e-6)
    early = (d[:, 2] < 0) & inside(P1) & (s1 > near0 + 1e-6) & (s1 < near1 - 1e-6)
    assert band.sum() > 100 and early.sum() > 100
    assert np.all(hit[band] == 1) and np.all(hit[early] == 1)
    expect = (1 - a) * t1 + a * t2
    assert np.max(np.abs(t[band] - expect[band])) < 1e-9 * t2.max()
    assert np.max(np.abs(t[early] - t1[early])) < 1e-9 * t1.max()
    assert np.ptp(a[band]) > 0.5                  # the band is crossed, not touched


# ---- coarse-level stop (extension: the level-L box field of the max mipmap) ----

def test_stop_level_worked_example(orc):
    """60 deg vertical field of view over 1080 rows: a pixel spans
    2 tan(30 deg) / 1080 = 1.0692e-3 of the distance, so 2 pixels at 1 km are
    2.138 m.  Nodes of 0.5 m texels: 2^2 * 0.5 = 2 m fits, 4 m does not -> 2;
    3 m texels: even level 0 is too wide -> 0.  No stop without a positive
    distance or pixel count; capped at the top level (N = 33: P = 32, K = 5)."""
    v = math.radians(60.0)
    assert orc.stop_level(2.0, v, 1080, 1000.0, 0.5, 2048) == 2
    assert orc.stop_level(2.0, v, 1080, 1000.0, 3.0, 2048) == 0
    assert orc.stop_level(0.0, v, 1080, 1000.0, 0.5, 2048) == 0
    assert orc.stop_level(2.0, v, 1080, -5.0, 0.5, 2048) == 0
    assert orc.stop_level(1e6, v, 1080, 1000.0, 0.5, 33) == 5


def _box_height(mip, N, L, u, v):
    """Height of the level-L box field at texel coordinates (u, v)."""
    P = 1
    while P < N - 1:
        P <<= 1
    off = sum((P >> k) ** 2 for k in range(L))
    PL = P >> L
    ni = np.clip(np.floor(u / (1 << L)).astype(int), 0, PL - 1)
    nj = np.clip(np.floor(v / (1 << L)).astype(int), 0, PL - 1)
    ok = (u >= 0) & (u <= N - 1) & (v >= 0) & (v <= N - 1)
    return np.where(ok, mip[off + nj * PL + ni].astype(np.float64), -np.inf)


@pytest.mark.parametrize("seed,L", [(0, 1), (1, 2), (2, 3)])
def test_coarse_stop_matches_box_field_marching(orc, tiny, seed, L):
    """With stop level L the first hit is the first point where the ray comes
    down to the level-L box field (the max mipmap's level-L entries as flat box
    tops), found here by dense marching plus bisection; and it never lies
    beyond the bilinear surface's first hit (the boxes bound the surface)."""
    N = 33
    tex, cas = _one_cascade_scene(N, seed)
    cas.stop_level = L
    mip = orc.maxmip(tex)
    eyes = [(32.0, -25.0, 70.0), (-10.0, 30.0, 45.0), (30.0, 30.0, 90.0)]
    fwds = [(0.1, 1.0, -0.6), (1.0, 0.2, -0.35), (0.2, 0.3, -1.0)]
    cam = _scene_camera(tiny, eyes[seed], fwds[seed])
    t, hit, _, _ = orc.raycast(cam, tiny.tree, [cas], [tex])
    cas.stop_level = 0
    t0, hit0, _, _ = orc.raycast(cam, tiny.tree, [cas], [tex])
    py, px = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    eye, d = _look_at_rays(cam, tiny.tree, px.ravel().astype(float), py.ravel().astype(float))
    fd = d @ (np.array(cam.forward) / np.linalg.norm(cam.forward))
    ts = np.linspace(0.0, 400.0, 40001)
    agree = skipped = 0
    for q in range(d.shape[0]):
        tt = ts[ts >= cam.znear / fd[q]]
        P = eye + tt[:, None] * d[q]
        f = _box_height(mip, N, L, P[:, 0] / cas.h, P[:, 1] / cas.h) - P[:, 2]
        pos = np.nonzero(f >= 0)[0]
        if pos.size == 0:
            fin = np.isfinite(f)
            if fin.any() and f[fin].max() > -1e-3:
                skipped += 1
                continue
            assert hit[q] == 0
            agree += 1
            continue
        k = pos[0]
        if k == 0 or not np.isfinite(f[k - 1]):
            skipped += 1              # starts under the boxes / enters the texture under them
            continue
        lo, hi = tt[k - 1], tt[k]
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            Pm = eye + mid * d[q]
            fm = _box_height(mip, N, L, np.array([Pm[0] / cas.h]), np.array([Pm[1] / cas.h]))[0] - Pm[2]
            lo, hi = (mid, hi) if fm < 0 else (lo, mid)
        assert hit[q] == 1, q
        assert t[q] == pytest.approx(0.5 * (lo + hi), abs=1e-7 * hi + 1e-9), q
        agree += 1
    assert agree > 0.97 * d.shape[0] and skipped < 0.03 * d.shape[0]
    both = (hit > 0) & (hit0 > 0)
    assert both.sum() > 100 and np.all(hit[hit0 > 0] > 0)
    assert np.all(t[both] <= t0[both] + 1e-9 * t0[both])
    assert np.mean(t[both] < t0[both] * (1 - 1e-6)) > 0.3     # the coarse surface is really coarser


@pytest.mark.parametrize("N,C", [(128, 3), (97, 2), (256, 1)])
def test_jump_ascent_traversal_equals_dda(orc, tiny, N, C):
    """The max-mip walk that climbs at once to the coarsest node it entered
    (the improved traversal after Dick et al.) finds the DDA's first hit on
    every pixel, as the one-level-per-step walk does, and visits no more
    nodes than the DDA walks patches."""
    cells = orc.Cells(tiny.tree)
    cam = tiny.cameras[0].with_(n_cascades=C, cascade_size=N)
    v = orc.fit(cam, tiny.tree, cells)
    casl, texs, mips = [], [], []
    for k in range(v.n_cascades):
        c = v.cas[k]
        tex = orc.texel_heights(c, cells, tiny.sigma, tiny.radius).reshape(c.N, c.N).astype(np.float32)
        casl.append(c)
        texs.append(tex)
        mips.append(orc.maxmip(tex))
    t0, h0, s0, v0 = orc.raycast(cam, tiny.tree, casl, texs, mode=0)
    t1, h1, s1, v1 = orc.raycast(cam, tiny.tree, casl, texs, mips, mode=1)
    t2, h2, s2, v2 = orc.raycast(cam, tiny.tree, casl, texs, mips, mode=2)
    assert np.array_equal(h0, h2) and np.array_equal(h1, h2)
    both = h0 > 0
    assert both.mean() > 0.3
    assert np.max(np.abs(t0[both] - t2[both]) / s0[both]) < 1e-9
    assert np.array_equal(t1[both], t2[both])
    assert v2.sum() < v0.sum()
    print(f"N={N} C={C}: visits per ray DDA {v0.mean():.1f}, one level per step {v1.mean():.1f}, "
          f"climb to the node entered {v2.mean():.1f}")
