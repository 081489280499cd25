"""The synthetic workloads stand in for the paper's scenarios (Table 1,
tests/golden/table1_scenarios.txt): the DEM stand-in has Florence's cell count,
and both large workloads lie within the paper's ranges of extents, cell
counts and cell-size octaves."""

import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_scenarios.txt")


def _table1():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            name, ex, ey, cmin, cmax, cells = line.split()[:6]
            rows.append((name, float(ex), float(ey), float(cmin), float(cmax), float(cells) * 1e6))
    return rows


def test_table1_fixture():
    rows = _table1()
    assert [r[0] for r in rows] == ["Marchfeld", "Petzenkirchen", "Wachau", "Florence"]
    assert all(r[4] == 96 for r in rows)


def test_paper_context_quotes_table1():
    """The bench line's paper context is Table 1's timings, frame = sum."""
    import bench
    ctx = bench.paper_context()
    assert "GTX 1080" in ctx["hardware"]
    f = ctx["scenarios"]["Florence"]
    assert (f["approximation_ms"], f["ray_casting_ms"]) == (1.5, 2.8)
    assert f["frame_ms"] == 4.3
    assert ctx["scenarios"]["Petzenkirchen"]["frame_ms"] == 25.1


def test_dem_stand_in_has_the_papers_shape():
    import workloads
    rows = _table1()
    florence = [r for r in rows if r[0] == "Florence"][0]
    s = workloads.dem_config(n_frames=2)
    t = s.tree
    assert abs(t.n_leaves - florence[5]) < 0.02 * florence[5]          # 4.5 M cells, as Florence
    sizes = np.unique(t.root_cell / (2.0 ** np.asarray(t.level)))
    octaves = math.log2(sizes.max() / sizes.min())
    paper_octaves = [math.log2(r[4] / r[3]) for r in rows]               # 5 to 7 octaves of cell size
    assert min(paper_octaves) - 1 <= octaves <= max(paper_octaves)
    ext_km = t.width / 1000.0
    assert min(min(r[1], r[2]) for r in rows) <= ext_km <= max(max(r[1], r[2]) for r in rows)
