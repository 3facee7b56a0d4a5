"""Low-rank compression of the M2L operators (test infrastructure only: only
tests/ may import this module).

Section 3.6.1: the M2L step multiplies each source cell's multipole moments
by the kernel evaluated at every (target node, source node) pair of the
space-time interpolation points,

    T[(a, c), (b, d)] = K(|x_a - y_b|, t_c - s_d),

x_a, y_b the p_s^3 Chebyshev points of the target and source cells (side
`side`, source offset `offset` cells), t_c, s_d the p_t points of the target
interval and of the source interval `lag` intervals earlier (interval length
`T`).  One such P x P matrix (P = p_s^3 p_t) serves every cell pair with that
offset and lag.  The paper mentions a 4-D FFT for uniform points; the other
standard compression is a truncated SVD per operator, T ~ U_r S_r V_r^T,
which replaces P^2 multiply-adds per moment column by 2 P r.  This module
builds the operators from that definition and reports their numerical ranks
and the cost of the factored product, so that the choice made for the GPU
path (dense products on the tensor cores) can be checked.
"""
from __future__ import annotations

import numpy as np

from .interp import cheb_nodes, k_A, k_phi


def operator(offset, lag: int, p_s: int, p_t: int, side: float = 1.0, T: float = 1.0, a: float = 0.25,
             kernel=k_phi) -> np.ndarray:
    """The P x P M2L operator of one (offset, lag, kernel)."""
    ax = [cheb_nodes(p_s, 0.0, side) for _ in range(3)]
    ay = [cheb_nodes(p_s, o * side, (o + 1) * side) for o in offset]
    X = np.stack(np.meshgrid(*ax, indexing="ij"), -1).reshape(-1, 3)
    Y = np.stack(np.meshgrid(*ay, indexing="ij"), -1).reshape(-1, 3)
    tn = cheb_nodes(p_t, 0.0, T)
    sn = cheb_nodes(p_t, -lag * T, -lag * T + T)
    r = np.linalg.norm(X[:, None, :] - Y[None, :, :], axis=-1)  # [ns^3, ns^3]
    tau = tn[:, None] - sn[None, :]  # [p_t, p_t]
    K = kernel(r[:, None, :, None], tau[None, :, None, :], a)  # [(a, c), (b, d)]
    P = len(X) * p_t
    return K.reshape(P, P)


def numerical_rank(Tm: np.ndarray, tol: float) -> int:
    """Number of singular values above tol times the largest (0 for a zero operator)."""
    s = np.linalg.svd(Tm, compute_uv=False)
    if s[0] == 0.0:
        return 0
    return int(np.sum(s > tol * s[0]))


def factor(Tm: np.ndarray, tol: float):
    """U_r S_r and V_r^T of the truncated SVD at relative tolerance tol."""
    U, s, Vt = np.linalg.svd(Tm)
    r = int(np.sum(s > tol * s[0])) if s[0] > 0 else 0
    return U[:, :r] * s[:r], Vt[:r]


def factored_cost(P: int, r: int) -> float:
    """Multiply-adds per moment column of the factored product over the dense one."""
    return 2.0 * P * r / (P * P)


KERNELS = {"phi": k_phi, "A": k_A}
