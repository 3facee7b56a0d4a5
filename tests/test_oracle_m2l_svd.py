"""Low-rank compression of the M2L operators (section 3.6.1), evaluated on
the CPU with oracle/m2l_svd.py: the operators of the 16 canonical far offsets
of a cell of side 1 (time intervals of one cell length, c dt = 1/4, p_s = p_t
points), over the lag window of Appendix A for each offset
(q_lo = max(1, floor(r_min / (M c dt))), q_hi = ceil((1 + r_max/(c dt)) / M),
M = 4, r_min and r_max the nearest and farthest point pairs of the cells).

A truncated SVD at 1e-7 of the largest singular value (the operator accuracy
the split-precision forms keep) replaces P^2 multiply-adds per moment column
by 2 P r.  Per operator the cheaper of the two forms is taken.
"""
import itertools
import math

import numpy as np
import pytest

from oracle.m2l_svd import factor, factored_cost, numerical_rank, operator

TOL = 1e-7
A = 0.25
M = 4


def _offsets():
    return sorted({tuple(sorted(map(abs, o), reverse=True)) for o in itertools.product(range(-3, 4), repeat=3)
                   if max(map(abs, o)) in (2, 3)})


def _window(off):
    rmin = math.sqrt(sum(max(0, o - 1) ** 2 for o in off))
    rmax = math.sqrt(sum((o + 1) ** 2 for o in off))
    return max(1, math.floor(rmin / (M * A))), math.ceil((1 + rmax / A) / M)


def test_sixteen_canonical_offsets():
    offs = _offsets()
    assert len(offs) == 16 and offs[0] == (2, 0, 0) and offs[-1] == (3, 3, 3)


@pytest.mark.parametrize("off, lag", [((2, 0, 0), 1), ((2, 2, 1), 3), ((3, 1, 0), 5)])
def test_factored_product_within_the_truncation_bound(off, lag):
    """||T x - U_r S_r V_r^T x|| <= sigma_(r+1) ||x|| <= TOL sigma_1 ||x||."""
    T = operator(off, lag, 4, 4, a=A)
    US, Vt = factor(T, TOL)
    s1 = np.linalg.norm(T, 2)
    rng = np.random.default_rng(1)
    for _ in range(5):
        x = rng.standard_normal(T.shape[1])
        assert np.linalg.norm(T @ x - US @ (Vt @ x)) <= TOL * s1 * np.linalg.norm(x) * (1 + 1e-6)


def test_rank_structure_follows_the_light_cone():
    """Outside the light cone the operator vanishes; well inside it the kernel
    is smooth and the rank small; where the cone crosses the cells it is high."""
    P = 4 ** 3 * 4
    assert not operator((3, 3, 3), 1, 4, 4, a=A).any()
    assert numerical_rank(operator((2, 0, 0), 6, 4, 4, a=A), TOL) < 0.3 * P
    assert numerical_rank(operator((2, 2, 1), 3, 4, 4, a=A), TOL) > 0.5 * P


def test_window_average_cost_at_p4():
    """Over the 78 non-zero operators of the windows at p = 4 the cheaper form
    costs about 0.65 of the dense products (a third saved at best), with
    ranks from 0.4% to 95% of P (median 32%)."""
    costs, ranks, P = [], [], 4 ** 3 * 4
    for off in _offsets():
        lo, hi = _window(off)
        for lag in range(lo, hi + 1):
            T = operator(off, lag, 4, 4, a=A)
            if not T.any():
                continue
            r = numerical_rank(T, TOL)
            ranks.append(r / P)
            costs.append(min(1.0, factored_cost(P, r)))
    print(f"\np = 4: {len(costs)} operators, mean cost of the cheaper form {np.mean(costs):.3f}, "
          f"rank/P median {np.median(ranks):.3f}, max {max(ranks):.3f}")
    assert len(costs) == 78
    assert 0.55 < np.mean(costs) < 0.75
