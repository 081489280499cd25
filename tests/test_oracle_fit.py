"""Pins of the oracle's cascade fitting (Section 3) and visible-texel mask.

Checked against an independent convex-hull routine (scipy), a camera-space
containment test, Monte-Carlo coverage of the potentially visible area, the
paper's logarithmic split formula, and the stable-fit rules.
"""

import ctypes as ct
import math

import numpy as np
import pytest

scipy_spatial = pytest.importorskip("scipy.spatial")


def _basis(cam):
    F = np.array(cam.forward, float)
    F /= np.linalg.norm(F)
    up = np.array(cam.up, float)
    U = up - up.dot(F) * F
    U /= np.linalg.norm(U)
    return F, U, np.cross(F, U)


def _in_frustum(cam, eye, p, tol=1e-7):
    F, U, R = _basis(cam)
    q = p - eye
    zc, xc, yc = q @ F, q @ R, q @ U
    tv = math.tan(cam.vfov / 2)
    th = tv * cam.width / cam.height
    return ((zc >= cam.znear - tol) & (zc <= cam.zfar + tol) & (np.abs(xc) <= th * zc + tol)
            & (np.abs(yc) <= tv * zc + tol))


def _in_convex(poly, pts, tol=1e-7):
    poly = np.asarray(poly)
    inside = np.ones(len(pts), bool)
    for k in range(len(poly)):
        a, b = poly[k], poly[(k + 1) % len(poly)]
        cr = (b[0] - a[0]) * (pts[:, 1] - a[1]) - (b[1] - a[1]) * (pts[:, 0] - a[0])
        inside &= cr >= -tol * np.linalg.norm(b - a)
    return inside


def _cam_local_eye(cam, tree):
    return np.array([cam.eye[0] - tree.origin_x, cam.eye[1] - tree.origin_y, cam.eye[2]])


def _cams(tiny):
    base = tiny.cameras[0]
    out = [base, base.with_(n_cascades=3, split_lambda=1.0),
           base.with_(n_cascades=4, split_lambda=0.5, forward=(0.3, 0.9, -0.2)),
           base.with_(n_cascades=2, forward=(0.0, 0.2, -1.0)),        # steep: hull behind the eye
           base.with_(n_cascades=3, forward=(-0.8, 0.1, -0.6), vfov=math.radians(40))]
    return out


def test_frustum_box_vertices_are_in_both_volumes(orc, tiny):
    cells = orc.Cells(tiny.tree)
    d = cells.domain
    for cam in _cams(tiny):
        v = orc.frustum_box_vertices(cam, tiny.tree, cells)
        assert len(v) >= 4
        eye = _cam_local_eye(cam, tiny.tree)
        assert np.all(_in_frustum(cam, eye, v, tol=1e-6))
        assert np.all((v[:, 0] > -1e-6) & (v[:, 0] < d.width + 1e-6))
        assert np.all((v[:, 2] > d.zmin - 1e-6) & (v[:, 2] < d.zmax + 1e-6))


def test_hull_matches_scipy_and_covers_visible_volume(orc, tiny):
    cells = orc.Cells(tiny.tree)
    d = cells.domain
    rng = np.random.default_rng(3)
    for cam in _cams(tiny):
        view = orc.fit(cam, tiny.tree, cells)
        v = orc.frustum_box_vertices(cam, tiny.tree, cells)
        ref = scipy_spatial.ConvexHull(v[:, :2])
        ref_pts = v[ref.vertices, :2]
        hull = view.hull_points()
        assert len(hull) == len(ref_pts)
        for p in ref_pts:
            assert np.min(np.linalg.norm(hull - p, axis=1)) < 1e-7
        area = 0.5 * np.sum(hull[:, 0] * np.roll(hull[:, 1], -1) - np.roll(hull[:, 0], -1) * hull[:, 1])
        assert area == pytest.approx(ref.volume, rel=1e-9) and area > 0  # CCW
        # Monte Carlo: points of (frustum AND box) project into the hull
        p = np.column_stack([rng.uniform(0, d.width, 200000), rng.uniform(0, d.height, 200000),
                             rng.uniform(d.zmin, d.zmax, 200000)])
        eye = _cam_local_eye(cam, tiny.tree)
        inside = p[_in_frustum(cam, eye, p, tol=0.0)]
        assert len(inside) > 100
        assert np.all(_in_convex(hull, inside[:, :2], tol=1e-6))


def test_log_splits_follow_the_paper(orc, tiny):
    """lambda = 1, three cascades: splits at n (f/n)^(1/3) and n (f/n)^(2/3)
    (Section 3); lambda = 0: uniform splits."""
    cells = orc.Cells(tiny.tree)
    cam = tiny.cameras[0].with_(n_cascades=3, split_lambda=1.0)
    v = orc.fit(cam, tiny.tree, cells)
    n, f = v.n, v.f
    assert n > max(cam.znear, cells.domain.c_min)
    assert v.split[1] == pytest.approx(n * (f / n) ** (1 / 3), rel=1e-12)
    assert v.split[2] == pytest.approx(n * (f / n) ** (2 / 3), rel=1e-12)
    assert v.split[0] == n and v.split[3] == f
    v0 = orc.fit(cam.with_(split_lambda=0.0), tiny.tree, cells)
    assert v0.split[1] == pytest.approx(n + (f - n) / 3, rel=1e-12)
    assert v0.split[2] == pytest.approx(n + 2 * (f - n) / 3, rel=1e-12)


def test_depth_range_is_hull_extent_along_view(orc, tiny):
    cells = orc.Cells(tiny.tree)
    for cam in _cams(tiny):
        v = orc.fit(cam, tiny.tree, cells)
        eye = _cam_local_eye(cam, tiny.tree)
        d2 = np.array(_basis(cam)[0][:2])
        d2 /= np.linalg.norm(d2)
        s = (v.hull_points() - eye[:2]) @ d2
        assert v.n == pytest.approx(s.min(), abs=1e-9) and v.f == pytest.approx(s.max(), abs=1e-9)


def test_cascades_cover_hull_and_overlap(orc, tiny):
    """Every potentially visible point lies in at least one cascade polygon;
    points in the overlap band of cascades k and k+1 lie in both."""
    cells = orc.Cells(tiny.tree)
    rng = np.random.default_rng(4)
    for cam in _cams(tiny):
        v = orc.fit(cam, tiny.tree, cells)
        hull = v.hull_points()
        lo, hi = hull.min(0), hull.max(0)
        pts = np.column_stack([rng.uniform(lo[0], hi[0], 50000), rng.uniform(lo[1], hi[1], 50000)])
        pts = pts[_in_convex(hull, pts, tol=0.0)]
        eye = _cam_local_eye(cam, tiny.tree)
        s = (pts - eye[:2]) @ np.array(v.dir2)
        covered = np.zeros(len(pts), bool)
        for k in range(v.n_cascades):
            c = v.cas[k]
            if c.n_poly == 0:
                continue
            inc = _in_convex(c.polygon(), pts, tol=1e-6)
            band = (s >= c.near - 1e-9) & (s <= c.far_ext + 1e-9)
            assert np.array_equal(inc[~np.isclose(s, c.near) & ~np.isclose(s, c.far_ext)],
                                  band[~np.isclose(s, c.near) & ~np.isclose(s, c.far_ext)])
            covered |= inc
            if k + 1 < v.n_cascades:
                ov = (s > v.cas[k + 1].near + 1e-6) & (s < c.far_ext - 1e-6)
                nxt = _in_convex(v.cas[k + 1].polygon(), pts[ov], tol=1e-6)
                assert np.all(nxt) and np.all(inc[ov])
                assert c.far_ext > c.far
        assert np.all(covered)


def test_stable_fit_rules(orc, tiny):
    cells = orc.Cells(tiny.tree)
    cmin = cells.domain.c_min
    for cam in _cams(tiny):
        v = orc.fit(cam, tiny.tree, cells)
        for k in range(v.n_cascades):
            c = v.cas[k]
            assert c.E == 2 * c.snap_k * cmin                     # even multiple of c_min
            assert c.ox == c.snap_x * cmin and c.oy == c.snap_y * cmin
            assert c.ox + (c.N - 1) * c.h == pytest.approx(c.ox + c.E, rel=1e-14)  # corners on texels
            if c.n_poly:
                x0, y0, x1, y1 = c.aabb
                assert c.ox <= x0 + 1e-9 and c.oy <= y0 + 1e-9
                assert c.ox + c.E >= x1 - 1e-9 and c.oy + c.E >= y1 - 1e-9
                assert c.ox > x0 - cmin - 1e-9 and c.oy > y0 - cmin - 1e-9
                # minimal: one step smaller would not cover the box from this origin
                smaller = c.E - 2 * cmin
                assert (smaller < max(x1 - x0, y1 - y0) - 1e-9 or c.ox + smaller < x1 - 1e-9
                        or c.oy + smaller < y1 - 1e-9)


def test_fit_is_stable_under_cell_multiple_translation(orc):
    """Moving the camera by a whole number of minimum cells moves the texel
    grid by the same whole number and keeps its extent (no texel swimming,
    Section 3)."""
    lib = orc.lib()
    dom = orc.Domain(1.0e5, 1.0e5, 0.0, 80.0, 2.5, 40.0)
    for yaw in [0.3, 1.2, 2.9]:
        for shift in [(7, 0), (0, -3), (11, 5)]:
            def cam_at(dx, dy):
                fwd = (math.cos(yaw) * 0.8, math.sin(yaw) * 0.8, -0.6)
                return orc.CameraC((ct.c_double * 3)(50000.0 + dx, 50000.0 + dy, 600.0),
                                   (ct.c_double * 3)(*fwd), (ct.c_double * 3)(0, 0, 1),
                                   math.radians(60), 1.0, 4000.0, 640, 480, 3, 512, 0.5, 0.05)
            va, vb = orc.ViewC(), orc.ViewC()
            assert lib.orc_fit(ct.byref(cam_at(0, 0)), ct.byref(dom), ct.byref(va)) == 0
            assert lib.orc_fit(ct.byref(cam_at(shift[0] * 2.5, shift[1] * 2.5)), ct.byref(dom),
                               ct.byref(vb)) == 0
            for k in range(3):
                assert vb.cas[k].snap_k == va.cas[k].snap_k
                assert vb.cas[k].snap_x == va.cas[k].snap_x + shift[0]
                assert vb.cas[k].snap_y == va.cas[k].snap_y + shift[1]


def test_empty_view(orc, tiny):
    """A camera looking away from the domain sees nothing: empty cascades."""
    cells = orc.Cells(tiny.tree)
    cam = tiny.cameras[0].with_(forward=(0.0, -1.0, 0.2))
    cam = cam.with_(eye=(cam.eye[0], tiny.tree.origin_y - 100.0, cam.eye[2]))
    v = orc.fit(cam, tiny.tree, cells)
    assert v.n_hull == 0
    assert all(v.cas[k].n_poly == 0 for k in range(v.n_cascades))
    vis, _ = orc.mask(v.cas[0], cells)
    assert vis.sum() == 0


def _square_cascade(orc, x0, x1, ox, oy, h, N):
    c = orc.CascadeC()
    pts = [(x0, x0), (x1, x0), (x1, x1), (x0, x1)]
    c.n_poly = 4
    for k, p in enumerate(pts):
        c.poly[k][0], c.poly[k][1] = p
    c.ox, c.oy, c.h, c.N = ox, oy, h, N
    c.E = h * (N - 1)
    return c


def test_mask_of_axis_aligned_square(orc):
    """For an axis-aligned square the grown polygon is the square grown by
    sqrt(2) h on each side, cut to the domain."""
    dom = orc.Domain(100.0, 100.0, 0, 1, 1, 1)
    for (x0, x1, ox, h, N) in [(10.3, 40.7, 0.0, 1.5, 64), (-5.0, 30.0, -10.0, 0.75, 80),
                               (90.0, 130.0, 85.0, 1.0, 33)]:
        cas = _square_cascade(orc, x0, x1, ox, ox, h, N)
        vis, mg = orc.mask(cas, type("C", (), {"domain": dom})())
        vis = vis.reshape(N, N)
        p = ox + np.arange(N) * h
        d = math.sqrt(2) * h
        ax = (p >= x0 - d) & (p <= x1 + d) & (p >= -1e-6 * h) & (p <= 100.0 + 1e-6 * h)
        assert np.array_equal(vis, (ax[:, None] & ax[None, :]).astype(np.uint8))


def test_mask_covers_polygon_with_valid_patches(orc, tiny):
    """Every point of a cascade polygon lies in a bilinear patch whose four
    corner texels are all visible (away from the domain border, where a
    patch reaching outside the domain is not drawn)."""
    cells = orc.Cells(tiny.tree)
    rng = np.random.default_rng(5)
    for cam in _cams(tiny)[1:3]:
        v = orc.fit(cam.with_(cascade_size=96), tiny.tree, cells)
        for k in range(v.n_cascades):
            c = v.cas[k]
            if c.n_poly == 0:
                continue
            vis, _ = orc.mask(c, cells)
            vis = vis.reshape(c.N, c.N)
            poly = c.polygon()
            lo, hi = poly.min(0), poly.max(0)
            pts = np.column_stack([rng.uniform(lo[0], hi[0], 20000), rng.uniform(lo[1], hi[1], 20000)])
            pts = pts[_in_convex(poly, pts, tol=0.0)]
            W, H = tiny.tree.width, tiny.tree.height
            away = ((pts[:, 0] > c.h) & (pts[:, 0] < W - c.h) & (pts[:, 1] > c.h)
                    & (pts[:, 1] < H - c.h))
            pts = pts[away]
            assert len(pts) > 1000
            pi = np.clip(np.floor((pts[:, 0] - c.ox) / c.h).astype(int), 0, c.N - 2)
            pj = np.clip(np.floor((pts[:, 1] - c.oy) / c.h).astype(int), 0, c.N - 2)
            ok = vis[pj, pi] & vis[pj, pi + 1] & vis[pj + 1, pi] & vis[pj + 1, pi + 1]
            assert np.all(ok)


# ---- lattice fit (texel reuse across frames; not part of the paper) ----

def test_ladder_fit_worked_examples(orc):
    """Hand-derived cases.  Box 1000 x 500 m at (3.3, 7.9), N = 1026, c_min
    = 10: a spacing must reach 1000 / 1024 = 0.9765625 m.  With 4 steps per
    octave 10 * 2^(-13/4) = 1.05112 >= 0.97656 > 10 * 2^(-14/4) = 0.88388,
    so m = -13, and the origin is (floor(3.3 / 1.05112), floor(7.9 /
    1.05112)) = (3, 7).  With 1 step per octave 10 * 2^-3 = 1.25 >= 0.97656 >
    0.625: m = -3, origin (floor(2.64), floor(6.32)) = (2, 6)."""
    m, i0, j0, h = orc.ladder_fit(3.3, 7.9, 1003.3, 507.9, 10.0, 1026, 4)
    assert (m, i0, j0) == (-13, 3, 7)
    assert h == pytest.approx(10.0 * 2.0 ** -3.25, rel=1e-15)
    assert orc.ladder_fit(3.3, 7.9, 1003.3, 507.9, 10.0, 1026, 1)[:3] == (-3, 2, 6)


def test_ladder_fit_boundaries(orc):
    """A side of exactly (N - 2) h_m keeps m (the 1e-9 slack), a side larger
    by 1e-6 takes the next step; an origin exactly on a lattice point stays on
    it; a tiny box takes the finest allowed spacing c_min 2^-8."""
    cmin, N, n = 2.5, 130, 2
    h3 = cmin * 2.0 ** 1.5
    side = 128 * h3
    assert orc.ladder_fit(0.0, 0.0, side, 1.0, cmin, N, n)[0] == 3
    assert orc.ladder_fit(0.0, 0.0, side * (1 + 1e-6), 1.0, cmin, N, n)[0] == 4
    m, i0, j0, h = orc.ladder_fit(5 * h3, 7 * h3, 5 * h3 + side, 7 * h3 + 1.0, cmin, N, n)
    assert (m, i0, j0) == (3, 5, 7)
    m, _, _, h = orc.ladder_fit(1.0, 1.0, 1.0 + 1e-6, 1.0, cmin, N, n)
    assert m == -16 and h == pytest.approx(cmin / 256.0, rel=1e-15)


@pytest.mark.parametrize("n", [1, 2, 4])
def test_ladder_fit_rules(orc, tiny, n):
    """For every camera: h on the ladder, the smallest step whose N - 2
    spacings reach the box's larger side, the origin on the lattice of h at
    most one spacing below the box corner, and the N x N texels covering the
    box."""
    cells = orc.Cells(tiny.tree)
    cmin = cells.domain.c_min
    seen = 0
    for cam in _cams(tiny):
        v = orc.fit(cam.with_(texel_ladder=n), tiny.tree, cells)
        for k in range(v.n_cascades):
            c = v.cas[k]
            if not c.n_poly:
                continue
            seen += 1
            x0, y0, x1, y1 = c.aabb
            side = max(x1 - x0, y1 - y0)
            assert c.h == pytest.approx(cmin * 2.0 ** (c.snap_k / n), rel=1e-14)
            assert (c.N - 2) * c.h >= side * (1 - 1e-9)
            assert (c.N - 2) * cmin * 2.0 ** ((c.snap_k - 1) / n) < side * (1 - 1e-9)
            assert c.ox == c.snap_x * c.h and c.oy == c.snap_y * c.h
            assert c.E == (c.N - 1) * c.h
            assert x0 - c.h < c.ox <= x0 + 1e-9 * c.h and y0 - c.h < c.oy <= y0 + 1e-9 * c.h
            assert c.ox + c.E >= x1 - 1e-9 * side and c.oy + c.E >= y1 - 1e-9 * side
    assert seen >= 10


def test_ladder_fit_keeps_spacing_under_translation(orc):
    """Moving the camera by any distance (far from the domain's edges) keeps
    the box size, hence the ladder step, and moves the origin along the
    lattice: texels of the two frames coincide wherever they overlap."""
    lib = orc.lib()
    dom = orc.Domain(1.0e5, 1.0e5, 0.0, 80.0, 2.5, 40.0)
    for yaw in [0.3, 1.2, 2.9]:
        for shift in [(7.3, 0.0), (0.0, -3.9), (11.1, 5.7), (123.45, -67.8)]:
            def cam_at(dx, dy):
                fwd = (math.cos(yaw) * 0.8, math.sin(yaw) * 0.8, -0.6)
                return orc.CameraC((ct.c_double * 3)(50000.0 + dx, 50000.0 + dy, 600.0),
                                   (ct.c_double * 3)(*fwd), (ct.c_double * 3)(0, 0, 1),
                                   math.radians(60), 1.0, 4000.0, 640, 480, 3, 512, 0.5, 0.05, 4)
            va, vb = orc.ViewC(), orc.ViewC()
            assert lib.orc_fit(ct.byref(cam_at(0, 0)), ct.byref(dom), ct.byref(va)) == 0
            assert lib.orc_fit(ct.byref(cam_at(*shift)), ct.byref(dom), ct.byref(vb)) == 0
            for k in range(3):
                a, b = va.cas[k], vb.cas[k]
                assert b.snap_k == a.snap_k and b.h == a.h
                for ax, d in ((0, shift[0]), (1, shift[1])):
                    da = (b.snap_x - a.snap_x) if ax == 0 else (b.snap_y - a.snap_y)
                    assert abs(da * a.h - d) <= a.h * (1 + 1e-9)


def test_ladder_fit_follow_rule(orc, tiny):
    """Hysteresis of the lattice fit: a cascade keeps an earlier frame's
    ladder step only when it is exactly one step coarser than the smallest
    that fits; the box stays covered and the origin on the lattice."""
    cells = orc.Cells(tiny.tree)
    cmin = cells.domain.c_min
    seen = 0
    for cam in _cams(tiny):
        cam = cam.with_(texel_ladder=4)
        v0 = orc.fit(cam, tiny.tree, cells)
        m = [v0.cas[k].snap_k for k in range(v0.n_cascades)]
        for delta, expect in ((1, 1), (2, 0), (-1, 0), (0, 0)):
            v = orc.fit(cam, tiny.tree, cells, follow=[x + delta for x in m])
            for k in range(v.n_cascades):
                c = v.cas[k]
                if not c.n_poly:
                    continue
                seen += 1
                assert c.snap_k == m[k] + expect, (delta, k)
                x0, y0, x1, y1 = c.aabb
                assert c.h == pytest.approx(cmin * 2.0 ** (c.snap_k / 4), rel=1e-14)
                assert c.ox == c.snap_x * c.h and x0 - c.h < c.ox <= x0 + 1e-9 * c.h
                assert c.oy == c.snap_y * c.h and y0 - c.h < c.oy <= y0 + 1e-9 * c.h
                assert c.ox + c.E >= x1 - 1e-9 * c.E and c.oy + c.E >= y1 - 1e-9 * c.E
    assert seen >= 40
