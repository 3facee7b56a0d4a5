"""Pins against the paper's printed test-problem table (Table 1, section 4.1),
stored in tests/golden/table1_test_problem.txt.

* The sphere generator reproduces the paper's meshes at the sizes recursive
  subdivision reaches (Ns = 1280, 5120, 20480): minimum and average edge
  length to the table's three decimals.  The maximum is a little smaller:
  recursive midpoint subdivision is more uniform than a one-shot geodesic
  frequency.
* Reading of eq. (Mt): with a root cube of side 2a = 1, cells of side
  1 / 2^lmax and c dt = 0.005, Mt^(lmax) = floor(ds / (c dt)) gives every
  entry of the table's last column, while the printed ceiling does not
  (12.5 -> 13 for cases 4 and 5).  The library takes the floor.
* GPU: the library's octree over those meshes (N_leaf = 100, dt = 0.005;
  case 1's triangles span up to 17 c dt, a triangle pair up to 37 lags) has
  the table's lmax; its finest interval holds no more steps than the table's,
  since its boxes are enlarged by the triangles' extent (the paper ignores
  it), and at least floor((ds - 2 r_max) / (c dt)) with ds the finest cell of
  the vertices' bounding cube and r_max the largest triangle radius.
"""
import math
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SUBDIV = {1280: 3, 5120: 4, 20480: 5}


def _table():
    rows = []
    for ln in open(os.path.join(HERE, "golden", "table1_test_problem.txt")):
        if ln.strip() and not ln.startswith("#"):
            c, ns, dmin, dave, dmax, lmax, mt = ln.split()
            rows.append(dict(case=int(c), ns=int(ns), dmin=float(dmin), dave=float(dave), dmax=float(dmax),
                             lmax=int(lmax), mt=int(mt)))
    return rows


def _mesh(ns):
    from workloads.meshes import icosphere

    return icosphere(0.5, SUBDIV[ns])


def _edge_lengths(v, t):
    e = {(min(a, b), max(a, b)) for tri in t for a, b in ((tri[0], tri[1]), (tri[1], tri[2]), (tri[2], tri[0]))}
    e = np.array(sorted(e))
    return np.linalg.norm(v[e[:, 0]] - v[e[:, 1]], axis=1)


def test_table_is_complete():
    rows = _table()
    assert [r["case"] for r in rows] == list(range(1, 8))
    # Ns = 20 f^2 (geodesic frequency f = 8, 12, 16, 24, 32, 48, 64)
    assert [r["ns"] for r in rows] == [20 * f * f for f in (8, 12, 16, 24, 32, 48, 64)]


@pytest.mark.parametrize("ns", sorted(SUBDIV))
def test_sphere_meshes_match_table(ns):
    row = next(r for r in _table() if r["ns"] == ns)
    v, t = _mesh(ns)
    assert len(t) == ns
    L = _edge_lengths(v, t)
    assert abs(L.min() - row["dmin"]) <= 5e-4, (L.min(), row)
    assert abs(L.mean() - row["dave"]) <= 5e-4, (L.mean(), row)
    assert row["dmax"] - 4e-3 <= L.max() <= row["dmax"] + 5e-4, (L.max(), row)


def test_mt_column_is_the_floor_reading():
    a = 0.005  # c dt
    for r in _table():
        ds = 1.0 / 2 ** r["lmax"]  # root cube side 2 x radius 0.5
        assert math.floor(ds / a + 1e-12) == r["mt"], r
    assert any(math.ceil(1.0 / 2 ** r["lmax"] / a - 1e-12) != r["mt"] for r in _table())


@pytest.mark.gpu
@pytest.mark.parametrize("ns", sorted(SUBDIV))
def test_library_octree_matches_table(ns):
    from paper_2303_05006_gb300 import Solver

    row = next(r for r in _table() if r["ns"] == ns)
    v, t = _mesh(ns)
    s = Solver(v, t, 0.005, 64, mode=1, n_leaf=100)
    inf = s.info()
    s.close()
    assert inf.lmax == row["lmax"], (inf.lmax, row)
    ds = (v.max(0) - v.min(0)).max() / 2 ** row["lmax"]  # the root is the vertices' bounding cube
    rmax = max(np.linalg.norm(v[t[:, k]] - v[t].mean(1), axis=1).max() for k in range(3))
    assert math.floor((ds - 2 * rmax) / 0.005) <= inf.mt_leaf <= row["mt"], (inf.mt_leaf, row)


@pytest.mark.parametrize("case", range(1, 8))
def test_geodesic_meshes_match_table_edges(case):
    """Every case of Table 1 is the equal-arc icosahedral geodesic sphere of
    frequency f (Ns = 20 f^2): its edge lengths' minimum, mean and maximum
    equal the table's to the printed three decimals.  The one exception is
    case 7's mean, 0.00945 against a printed 0.010: the mean scales as 1/f
    (case 1's 0.075 x 8/64 = 0.0094), so the printed value is read as a
    rounding slip, and case 7 is held to its minimum and maximum."""
    from workloads.meshes import geodesic_sphere

    row = [r for r in _table() if r["case"] == case][0]
    f = int(round((row["ns"] / 20) ** 0.5))
    v, t = geodesic_sphere(0.5, f)
    assert len(t) == row["ns"]
    d = _edge_lengths(v, t)
    assert 3 * len(t) == 2 * len(d)  # closed 2-manifold
    assert round(d.min(), 3) == pytest.approx(row["dmin"], abs=1e-9)
    if case != 7:
        assert round(d.mean(), 3) == pytest.approx(row["dave"], abs=1e-9)
    assert round(d.max(), 3) == pytest.approx(row["dmax"], abs=1e-9)
