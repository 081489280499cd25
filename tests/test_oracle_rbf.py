"""Pins of the oracle's Eq. 1 / Eq. 2 against closed forms and invariants.

Each test would fail for a plausible slip in the oracle: a dropped division
by the cell size, a wrong sign or value of the truncation constant, a
missing clamp of negative weights, a missing normalisation, a wrong
neighbour search.
"""

import math

import numpy as np
import pytest


class _CellsArr:
    """Arbitrary cells for the brute-force path."""

    def __init__(self, cx, cy, cs, cv, w=1000.0, h=1000.0):
        import oracle
        self.cx = np.ascontiguousarray(cx, float)
        self.cy = np.ascontiguousarray(cy, float)
        self.cs = np.ascontiguousarray(cs, float)
        self.cv = np.ascontiguousarray(cv, float)
        self.n = self.cx.size
        self.domain = oracle.Domain(w, h, float(self.cv.min()), float(self.cv.max()),
                                    float(self.cs.min()), float(self.cs.max()))


def _uniform(n, c=1.0, values=None):
    iy, ix = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    cx = (ix.ravel() + 0.5) * c
    cy = (iy.ravel() + 0.5) * c
    cv = np.zeros(n * n) if values is None else values(cx, cy)
    return _CellsArr(cx, cy, np.full(n * n, c), cv, n * c, n * c)


def test_weight_special_values(orc):
    """Eq. 1: 1 - K at the centre, 1/2 - K at the half-maximum distance
    sigma*c*sqrt(2 ln 2), 0 at the truncation radius R*c and beyond."""
    for sigma, R, c in [(1.0, 3.5, 3.0), (1.5, 3.0, 10.0), (0.7, 2.0, 0.75)]:
        K = math.exp(-R * R / (2 * sigma * sigma))
        assert orc.rbf_weight(0.0, c, sigma, R) == pytest.approx(1.0 - K, abs=1e-15)
        dh = sigma * c * math.sqrt(2 * math.log(2))
        assert orc.rbf_weight(dh, c, sigma, R) == pytest.approx(0.5 - K, abs=1e-14)
        assert orc.rbf_weight(R * c, c, sigma, R) == 0.0
        assert orc.rbf_weight(R * c * 1.0001, c, sigma, R) == 0.0
        assert orc.rbf_weight(R * c * 0.999, c, sigma, R) > 0.0


def test_paper_truncation_constant(orc):
    """With sigma = 1 and R = 3.5 the subtracted constant is exp(-3.5^2/2)
    (Eq. 1): the weight at the centre is 1 - 0.0021874911..."""
    assert orc.rbf_weight(0.0, 1.0, 1.0, 3.5) == pytest.approx(1.0 - 0.0021874911181828851, abs=1e-15)


def test_weight_scale_invariance(orc):
    """w depends on d only through d / c_i."""
    for d in [0.0, 0.3, 1.1, 2.9]:
        a = orc.rbf_weight(d, 1.0, 1.5, 3.0)
        b = orc.rbf_weight(8.0 * d, 8.0, 1.5, 3.0)
        assert a == pytest.approx(b, rel=1e-14, abs=1e-16)


def test_two_cells_hand_example(orc):
    """Two cells of different size placed so that their Gaussian factors are
    exactly 1/2 and 1/4, plus a third cell just beyond its truncation radius
    carrying a huge value: v = ((1/2-K) 10 + (1/4-K) 30) / (3/4 - 2K)."""
    sigma, R = 1.0, 3.5
    K = math.exp(-R * R / 2)
    dA = 1.0 * sigma * math.sqrt(2 * math.log(2))      # cA = 1 -> factor 1/2
    dB = 2.0 * sigma * math.sqrt(2 * math.log(4))      # cB = 2 -> factor 1/4
    dC = 4.0 * R * 1.001                                # cC = 4 -> outside
    cells = _CellsArr([dA, 0.0, -dC], [0.0, dB, 0.0], [1.0, 2.0, 4.0], [10.0, 30.0, 1e6])
    expect = ((0.5 - K) * 10 + (0.25 - K) * 30) / (0.75 - 2 * K)
    for mode in (0,):
        v, cnt = orc.rbf_points(cells, sigma, R, [0.0], [0.0], mode=mode, with_counts=True)
        assert cnt[0] == 2
        assert v[0] == pytest.approx(expect, rel=1e-13)


def test_constant_field_is_reproduced(orc, tiny):
    """Eq. 2 is a normalised sum: a constant field is reproduced exactly on
    any adaptive grid."""
    cells = orc.Cells(tiny.tree)
    cells.cv[:] = 123.25
    rng = np.random.default_rng(0)
    px = rng.uniform(0, tiny.tree.width, 2000)
    py = rng.uniform(0, tiny.tree.height, 2000)
    v = orc.rbf_points(cells, tiny.sigma, tiny.radius, px, py)
    assert np.all(np.abs(v - 123.25) < 1e-11)


def test_isolated_bump_closed_form(orc):
    """Unit lattice, one cell of value H, all others 0.  At the bump centre
    v = H (1-K) / sum_{m^2+n^2 < R^2} (exp(-(m^2+n^2)/(2 sigma^2)) - K),
    the sum running over integer offsets (m, n)."""
    H = 50.0
    for sigma, R in [(1.0, 3.5), (1.5, 3.0)]:
        K = math.exp(-R * R / (2 * sigma * sigma))
        den = 0.0
        r = int(math.ceil(R))
        for m in range(-r, r + 1):
            for n in range(-r, r + 1):
                if m * m + n * n < R * R:
                    den += math.exp(-(m * m + n * n) / (2 * sigma * sigma)) - K
        cells = _uniform(21)
        centre = 10 * 21 + 10
        cells.cv[centre] = H
        x0, y0 = cells.cx[centre], cells.cy[centre]
        for mode in (0, 1):
            v = orc.rbf_points(cells, sigma, R, [x0], [y0], mode=mode)
            assert v[0] == pytest.approx(H * (1 - K) / den, rel=1e-13)


def test_linear_field_at_symmetric_points(orc):
    """On a uniform lattice the weights are point-symmetric about cell
    centres, cell corners and edge midpoints, so a linear field is
    reproduced exactly there (away from the border)."""
    a, b, c0 = 0.37, -1.25, 40.0
    cells = _uniform(24, c=2.0, values=lambda x, y: a * x + b * y + c0)
    pts = []
    for i in range(8, 16):
        for j in range(8, 16):
            for ox, oy in [(0.5, 0.5), (0.0, 0.0), (0.5, 0.0), (0.0, 0.5)]:
                pts.append(((i + ox) * 2.0, (j + oy) * 2.0))
    px, py = np.array(pts).T
    for sigma, R in [(1.0, 3.5), (1.5, 3.0)]:
        v = orc.rbf_points(cells, sigma, R, px, py, mode=1)
        assert np.max(np.abs(v - (a * px + b * py + c0))) < 1e-10


def test_brute_force_equals_binned_search(orc, tiny):
    """The binned enumeration finds exactly the influencing set."""
    cells = orc.Cells(tiny.tree)
    rng = np.random.default_rng(1)
    W, H = tiny.tree.width, tiny.tree.height
    px = np.concatenate([rng.uniform(0, W, 1500), [0.0, W, 0.0, W, -1e-7], rng.uniform(-5, 5, 50)])
    py = np.concatenate([rng.uniform(0, H, 1500), [0.0, 0.0, H, H, 3.0], rng.uniform(0, H, 50)])
    vb, nb = orc.rbf_points(cells, tiny.sigma, tiny.radius, px, py, mode=0, with_counts=True)
    vn, nn = orc.rbf_points(cells, tiny.sigma, tiny.radius, px, py, mode=1, with_counts=True)
    assert np.array_equal(nb, nn)
    assert np.max(np.abs(vb - vn)) < 1e-9


def test_convexity_and_influencer_counts(orc, tiny):
    """v is a convex combination of its influencers' values, and the number
    of influencers at a point of a uniform region is the number of lattice
    points strictly inside the truncation disc (25 for R = 3 lattice units,
    in units of the local cell size, when the point is a cell centre)."""
    cells = orc.Cells(tiny.tree)
    rng = np.random.default_rng(2)
    px = rng.uniform(0, tiny.tree.width, 500)
    py = rng.uniform(0, tiny.tree.height, 500)
    v = orc.rbf_points(cells, tiny.sigma, tiny.radius, px, py)
    assert np.all(v >= cells.cv.min() - 1e-9) and np.all(v <= cells.cv.max() + 1e-9)
    uni = _uniform(15)
    _, cnt = orc.rbf_points(uni, 1.5, 3.0, [7.5], [7.5], mode=0, with_counts=True)
    lattice = sum(1 for m in range(-3, 4) for n in range(-3, 4) if m * m + n * n < 9)
    assert cnt[0] == lattice == 25


# ---- Wendland's psi_{3,1}: another interpolant in the discretization slot ----

def test_wendland_values_support_and_smoothness(orc):
    """psi_{3,1}(r) = (1 - r)_+^4 (4 r + 1) (Wendland, 1995) of r = d / (R c):
    psi(0) = 1, psi(1/2) = 3/16, zero from the support radius R c on; the
    function is C2 at the support edge (value, slope and curvature vanish
    there) and flat at the centre; only d / c matters."""
    W = orc.WENDLAND_C2
    for R, c in [(3.0, 10.0), (3.5, 2.0), (1.0, 0.75)]:
        def w(r):
            return orc.rbf_weight(r * R * c, c, 1.5, R, W)
        assert w(0.0) == 1.0
        assert w(0.5) == pytest.approx(3.0 / 16.0, rel=1e-14)
        assert w(1.0) == 0.0 and w(1.2) == 0.0 and w(0.999) > 0.0
        h = 1e-3
        assert abs((w(1.0) - w(1.0 - h)) / h) < 1e-7                         # slope -> 0
        assert abs((w(1.0) - 2 * w(1.0 - h) + w(1.0 - 2 * h)) / h ** 2) < 2e-4  # curvature -> 0
        assert abs((w(h) - w(0.0)) / h) < 1e-2                                # flat peak
        assert w(0.3) > w(0.6) > w(0.9) > 0.0                                 # decreasing
    for d in [0.0, 0.3, 1.1, 2.9]:
        assert orc.rbf_weight(d, 1.0, 1.5, 3.0, W) == pytest.approx(orc.rbf_weight(8 * d, 8.0, 1.5, 3.0, W),
                                                                 rel=1e-14, abs=1e-16)


def test_wendland_constant_linear_and_binned(orc, tiny):
    """With the Wendland weights Eq. 2 still reproduces a constant field on
    the adaptive grid, a linear field at lattice-symmetric points of a
    uniform grid, and the binned search still finds exactly the influencers
    (the supports equal the Gaussian's truncation radius)."""
    W = orc.WENDLAND_C2
    cells = orc.Cells(tiny.tree)
    cells.cv[:] = -7.5
    rng = np.random.default_rng(3)
    px = rng.uniform(0, tiny.tree.width, 1500)
    py = rng.uniform(0, tiny.tree.height, 1500)
    assert np.all(np.abs(orc.rbf_points(cells, tiny.sigma, tiny.radius, px, py, kernel=W) + 7.5) < 1e-11)
    a, b, c0 = 0.37, -1.25, 40.0
    uni = _uniform(24, c=2.0, values=lambda x, y: a * x + b * y + c0)
    pts = [((i + ox) * 2.0, (j + oy) * 2.0) for i in range(8, 16) for j in range(8, 16)
           for ox, oy in [(0.5, 0.5), (0.0, 0.0), (0.5, 0.0), (0.0, 0.5)]]
    qx, qy = np.array(pts).T
    v = orc.rbf_points(uni, 1.5, 3.0, qx, qy, mode=1, kernel=W)
    assert np.max(np.abs(v - (a * qx + b * qy + c0))) < 1e-10
    cells = orc.Cells(tiny.tree)
    vb, nb = orc.rbf_points(cells, tiny.sigma, tiny.radius, px, py, mode=0, with_counts=True, kernel=W)
    vn, nn = orc.rbf_points(cells, tiny.sigma, tiny.radius, px, py, mode=1, with_counts=True, kernel=W)
    assert np.array_equal(nb, nn) and np.max(np.abs(vb - vn)) < 1e-9
    # same support as the truncated Gaussian: the same influencing sets
    _, ng = orc.rbf_points(cells, tiny.sigma, tiny.radius, px, py, mode=1, with_counts=True)
    assert np.array_equal(nn, ng)
