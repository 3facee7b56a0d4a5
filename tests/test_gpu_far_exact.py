"""Exactness of the fast path's far-field machinery (the exact-kernel
check), on the GPU.

With far_kernel = 1 the library's M2L operators hold the polynomial kernel
K = (1 + |x - y|^2) ((t - s)/dt)^3 and its time derivative instead of the
truncated powers.  The kernel has degree 2 in each coordinate and 3 in t and
s, so the interpolation of every stage (P2M, M2M, M2L through the 48 cube
symmetries, L2L, L2P with its time derivatives) reproduces it exactly; what
is left is the bookkeeping -- the octree and interaction lists, the per-level
intervals and their time gating, the lag range of each offset, the J-hat
window truncated at its start, the full and truncated moment sets through
M2M -- and FP32 rounding.  far_kernel = 2 zeroes the far field, so the
difference of the two history evaluations is the library's far field alone.
It must equal the oracle's plain windowed sum (oracle/far_window.py, pinned to
Appendix A's identity and to Table 1 on the CPU) row by row.  The same holds
with the paper's CHI interpolant (section 3.2) in space, and in time for the
check kernel with the Chebyshev quadratic T2 (CHI reproduces degree 2), and
for each placement of the vector potential's two time derivatives (section
4.3.2): every stage then reproduces the kernel.

Bar: the far field runs in FP32 (moments, operators, local coefficients) with
FP64 accumulation into the right-hand side.  In the J-hat form the windowed
sum is a strongly cancelling one (the terms' absolute sum is 1e4 to 1e5 times
the result here, as for the method's own kernel), so FP32 rounding leaves
about 1e-5 of the result; the bar is 1e-3 of the largest far value among the
sampled rows.  tests/test_far_window.py shows on the CPU that a window one
interval short at either end, or an untruncated window start, moves the
reference by at least 50 times that bar.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-3  # of the largest far-field value among the sampled rows


@pytest.fixture(scope="module")
def setup():
    from oracle.far_window import Hierarchy
    from oracle.oracle import Oracle
    from workloads.meshes import icosphere, mean_edge_length

    v, t = icosphere(1.0, 3)
    dt = 0.25 * mean_edge_length(v, t)
    h = Hierarchy(v, t, dt, n_leaf=16)
    edges = Oracle(v, t, dt).edges()
    return v, t, dt, h, edges


def _smooth_history(ne, n, seed):
    """J^b_j = sin(2 pi b / P_j + phi_j), periods of 40 to 80 steps."""
    rng = np.random.default_rng(seed)
    P = rng.uniform(40, 80, ne)
    ph = rng.uniform(0, 2 * np.pi, ne)
    return np.sin(2 * np.pi * np.arange(n)[:, None] / P[None, :] + ph[None, :])


# (M2L precision, check kernel, s_interp, t_interp, a_deriv): FP32 CUDA cores,
# TF32x3 tensor cores, and FP16x3 with the operator resident in shared memory
# (k_m2l_res); the T3 kernel under Lagrange interpolation, with
# CHI in space, and with the two other placements of the vector potential's
# time derivatives; the T2 kernel (degree 2 in time, which CHI reproduces)
# under CHI in space and time, with every placement.
CASES = [(0, 1, 0, 0, 0), (4, 1, 0, 0, 0), (5, 1, 0, 0, 0), (4, 1, 1, 0, 0), (4, 1, 0, 0, 1), (4, 1, 0, 0, 2),
         (4, 3, 1, 1, 0), (4, 3, 1, 1, 1), (4, 3, 1, 1, 2)]


@pytest.mark.parametrize("prec,kern,s_interp,t_interp,a_deriv", CASES)
def test_far_field_equals_windowed_sum(setup, prec, kern, s_interp, t_interp, a_deriv):
    from oracle.far_window import far_field_poly
    from paper_2303_05006_gb300 import Solver

    v, t, dt, h, edges = setup
    Nt = 200
    kw = dict(mode=1, p_s=4, p_t=4, n_leaf=16, m2l_prec=prec, s_interp=s_interp, t_interp=t_interp,
              a_deriv=a_deriv)
    s1 = Solver(v, t, dt, Nt, far_kernel=kern, **kw)
    s2 = Solver(v, t, dt, Nt, far_kernel=2, **kw)
    inf = s1.info()
    # the library's hierarchy is the oracle's
    assert inf.lmax == h.lmax == 3
    assert inf.mt_leaf == h.M(h.lmax)
    ne = s1.ne
    J = _smooth_history(ne, Nt, seed=5)
    rows = np.sort(np.random.default_rng(9).choice(ne, 12, replace=False))
    M2 = h.M(2)
    # early steps (windows still reaching before the first step), interval
    # boundaries of both levels, and the steady state
    for alpha in (M2 + 1, 2 * M2, 3 * M2 + 2, 61, 150, Nt - 1):
        Jh = J[: alpha - 1]
        far = s2.history_eval(alpha, Jh) - s1.history_eval(alpha, Jh)
        ref = far_field_poly(h, edges, rows, Jh, alpha, tdeg=3 if kern == 1 else 2)
        scale = np.max(np.abs(ref))
        assert scale > 0
        err = np.max(np.abs(far[rows] - ref))
        assert err <= TOL * scale, (alpha, err / scale)
    s1.close()
    s2.close()


def test_zero_far_kernel_leaves_the_near_field(setup):
    """far_kernel = 2 with the method's near field: on a mesh small enough to
    be all near field (no interaction list) every far_kernel gives the same
    history sum."""
    from paper_2303_05006_gb300 import Solver
    from workloads import workload

    w = workload("sphere80")
    J = _smooth_history(120, 40, seed=2)
    R = [Solver(w.verts, w.tris, w.dt, w.Nt, mode=1, far_kernel=k).history_eval(30, J[:29]) for k in (0, 1, 2)]
    assert np.array_equal(R[0], R[1]) and np.array_equal(R[0], R[2])


@pytest.mark.parametrize("prec", [4, 5])
def test_batched_far_field_equals_windowed_sum(setup, prec):
    """The batched form (three right-hand sides, each with its own history):
    the far field of every right-hand side equals the oracle's windowed sum,
    through the batched P2M, M2M, M2L columns (pair, right-hand side,
    component), L2L and L2P."""
    from oracle.far_window import far_field_poly
    from paper_2303_05006_gb300 import Solver

    v, t, dt, h, edges = setup
    Nt, R = 200, 3
    kw = dict(mode=1, p_s=4, p_t=4, n_leaf=16, m2l_prec=prec, n_rhs=R)
    s1 = Solver(v, t, dt, Nt, far_kernel=1, **kw)
    s2 = Solver(v, t, dt, Nt, far_kernel=2, **kw)
    alpha = 150
    H = np.stack([_smooth_history(s1.ne, alpha - 1, seed=20 + r) for r in range(R)], axis=1)  # (a-1, R, ne)
    far = s2.history_eval(alpha, H) - s1.history_eval(alpha, H)
    rows = np.sort(np.random.default_rng(13).choice(s1.ne, 8, replace=False))
    for r in range(R):
        ref = far_field_poly(h, edges, rows, H[:, r], alpha)
        scale = np.max(np.abs(ref))
        err = np.max(np.abs(far[r][rows] - ref))
        assert err <= TOL * scale, (prec, r, err / scale)
    s1.close()
    s2.close()
