"""Pins of the oracle's space-time hierarchy and far-field window
(oracle/far_window.py), on the CPU.

* Appendix A: the far field sums J-hat against the truncated-power kernel
  over a window of source steps, the oldest interval's J-hat truncated at the
  window start.  For every pair of points in the boxes of an interaction pair
  that window sum must equal the plain B-spline sum over the whole history,
      sum_{beta} J^beta N(alpha - beta - r/(c dt)),
  exactly (N from the oracle's B-spline, itself pinned to the textbook
  pieces).  The point pairs include the boxes' nearest points and opposite
  far corners, so a window one interval short at either end, a wrong window
  start or a missing truncation breaks it.
* Table 1 (section 4.1): the hierarchy has the paper's lmax for N_leaf = 100,
  dt = 0.005 on the geodesic spheres of radius 0.5, and its finest interval
  holds no more steps than the table's (its boxes are enlarged by the
  triangles' extent, which the paper ignores).
* The classification partitions every triangle pair: near at the first level
  where the cells are neighbours and one is a leaf, far (levels >= 2) where
  they are not, with cell offsets of Chebyshev norm 2 or 3.
"""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _tree(subdiv=3, n_leaf=16, dt_frac=0.25):
    from oracle.far_window import Hierarchy
    from workloads.meshes import icosphere, mean_edge_length

    v, t = icosphere(1.0, subdiv)
    dt = dt_frac * mean_edge_length(v, t)
    return Hierarchy(v, t, dt, n_leaf=n_leaf), v, t, dt


def test_partition_and_offsets():
    h, v, t, dt = _tree()
    assert h.lmax >= 3, "two far levels are needed to exercise M2M and L2L"
    rng = np.random.default_rng(7)
    levels = set()
    for tt in rng.choice(h.nt, 40, replace=False):
        kind, lev, off = h.classify(tt, np.arange(h.nt))
        assert np.all((kind == 0) | (kind == 1))
        far = kind == 1
        cheb = np.max(np.abs(off[far]), axis=1)
        assert np.all((cheb == 2) | (cheb == 3)), np.unique(cheb)
        assert np.all(lev[far] >= 2)
        levels |= set(lev[far].tolist())
        # the triangle itself and its edge neighbours are near
        assert kind[tt] == 0
    assert len(levels) >= 2, levels


def test_window_sum_equals_bspline_sum():
    """Appendix A: windowed, truncated J-hat against (alpha - gamma - r/a)_+^2
    equals sum_beta J^beta N(alpha - beta - r/a), for every alpha."""
    from oracle.far_window import jhat_window
    from oracle.oracle import bspline

    h, v, t, dt = _tree()
    rng = np.random.default_rng(11)
    a = h.a
    cases = []
    for tt in rng.choice(h.nt, 12, replace=False):
        kind, lev, off = h.classify(tt, np.arange(h.nt))
        for s in rng.choice(np.nonzero(kind == 1)[0], 3, replace=False):
            cases.append((tt, s, lev[s], off[s]))
    n_steps = 8 * h.M(2) + 7
    J = rng.standard_normal(n_steps)
    checked = 0
    for tt, s, l, o in cases:
        q_lo, q_hi = h.lag_range(l, o)
        ct = h.root + (h.coords(np.array([tt]), l)[0] + 0.5) * h.ds(l)
        cs = ct + o * h.ds(l)
        # random points, and the two extreme pairs: the boxes' nearest points
        # (r = r_min) and their opposite far corners (r = r_max)
        sg = np.where(o > 0, 1.0, np.where(o < 0, -1.0, 0.0))
        pts = [(ct + (rng.random(3) * 2 - 1) * h.H(l), cs + (rng.random(3) * 2 - 1) * h.H(l)) for _ in range(2)]
        near_x = ct + sg * h.H(l)
        near_y = np.where(sg != 0, cs - sg * h.H(l), near_x)
        pts.append((near_x, near_y))
        far_sg = np.where(sg != 0, sg, 1.0)
        pts.append((ct - far_sg * h.H(l), cs + far_sg * h.H(l)))
        for x, y in pts:
            r = float(np.linalg.norm(x - y))
            for alpha in range(1, n_steps + 1):
                G, g0, g1 = h.window(l, q_lo, q_hi, alpha)
                lhs = 0.0
                if g1 >= g0:
                    Jh = jhat_window(J[: alpha - 1], G, g0, g1)
                    u = (alpha - np.arange(g0, g1 + 1)) - r / a
                    lhs = float(np.sum(Jh * np.where(u > 0, u * u, 0.0)))
                rhs = sum(J[b] * bspline(alpha - b - r / a) for b in range(0, alpha - 1))
                assert abs(lhs - rhs) <= 1e-11 * (1 + np.sum(np.abs(J))), (l, o, alpha, lhs, rhs)
                checked += 1
    assert checked > 1000


def _table1():
    rows = []
    for ln in open(os.path.join(HERE, "golden", "table1_test_problem.txt")):
        if ln.strip() and not ln.startswith("#"):
            c, ns, _, _, _, lmax, mt = ln.split()
            rows.append((int(ns), int(lmax), int(mt)))
    return rows


@pytest.mark.parametrize("ns,subdiv", [(1280, 3), (5120, 4), (20480, 5)])
def test_hierarchy_matches_table1(ns, subdiv):
    from oracle.far_window import Hierarchy
    from workloads.meshes import icosphere

    row = [r for r in _table1() if r[0] == ns][0]
    v, t = icosphere(0.5, subdiv)
    h = Hierarchy(v, t, 0.005, n_leaf=100)
    assert h.lmax == row[1]
    assert 3 <= h.M(h.lmax) <= row[2]


@pytest.mark.parametrize("tdeg", [3, 2])
def test_planted_window_faults_exceed_the_gpu_bar(tdeg):
    """The GPU exactness check (tests/test_gpu_far_exact.py) compares the
    library's far field with far_field_poly at a bar of TOL of the largest
    value.  On its own mesh, history and rows, each planted bookkeeping fault
    moves the reference by at least 50 TOL: the newest interval dropped
    (q_lo + 1) at every step, and, once the windows reach back past the first
    step, the oldest interval dropped (q_hi - 1) or the window start left
    untruncated.  Both check kernels: T3 in time, and T2 (the one the CHI
    interpolant reproduces).  With T2 the oldest interval is invisible: the
    third difference J-hat summed against a quadratic in time telescopes to
    terms at the window's ends, and the truncation at the start removes those
    there, so the sum depends on the newest end alone (the T3 check covers
    q_hi)."""
    import oracle.far_window as fw
    from oracle.far_window import Hierarchy, far_field_poly
    from oracle.oracle import Oracle
    from tests.test_gpu_far_exact import TOL, _smooth_history
    from workloads.meshes import icosphere, mean_edge_length

    v, t = icosphere(1.0, 3)
    dt = 0.25 * mean_edge_length(v, t)
    h = Hierarchy(v, t, dt, n_leaf=16)
    ed = Oracle(v, t, dt).edges()
    ne = len(ed[0])
    J = _smooth_history(ne, 200, seed=5)
    rows = np.sort(np.random.default_rng(9).choice(ne, 12, replace=False))
    orig_lr, orig_jh = fw.Hierarchy.lag_range, fw.jhat_window
    faults = {
        "q_lo + 1": lambda: setattr(fw.Hierarchy, "lag_range", lambda s, l, o: (orig_lr(s, l, o)[0] + 1,
                                                                                    orig_lr(s, l, o)[1])),
        "q_hi - 1": lambda: setattr(fw.Hierarchy, "lag_range", lambda s, l, o: (orig_lr(s, l, o)[0],
                                                                                    orig_lr(s, l, o)[1] - 1)),
        "untruncated": lambda: setattr(fw, "jhat_window", lambda J_, G, g0, g1: orig_jh(J_, G - 8, g0, g1)),
    }
    try:
        late = list(faults) if tdeg == 3 else ["q_lo + 1", "untruncated"]
        for alpha, names in ((12, ["q_lo + 1"]), (150, late)):
            ref = far_field_poly(h, ed, rows, J[: alpha - 1], alpha, tdeg=tdeg)
            scale = np.abs(ref).max()
            for name in names:
                faults[name]()
                planted = far_field_poly(h, ed, rows, J[: alpha - 1], alpha, tdeg=tdeg)
                fw.Hierarchy.lag_range, fw.jhat_window = orig_lr, orig_jh
                assert np.abs(planted - ref).max() >= 50 * TOL * scale, (alpha, name)
    finally:
        fw.Hierarchy.lag_range, fw.jhat_window = orig_lr, orig_jh
