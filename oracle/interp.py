"""Space-time Lagrange interpolation of the far-field kernel of one pair of
cells (test infrastructure only: only tests/ may import this module).

Section 3.2 (eq. U_expand): between a target cell X (times t in an interval
I_t) and a well-separated source cell Y (times s in I_s), the kernel of eq. U
is replaced by its tensor-product interpolant on p_s Chebyshev points per
direction of each cell and p_t per interval,

    U(x, y, t - s) ~ sum_{a, b, c, d} L_a(x) L_b(y) l_c(t) l_d(s) U(x_a, y_b, t_c - s_d),

L the 3-D tensor products of the 1-D Lagrange polynomials.  This module
builds that interpolant from its definition (nodes, 1-D basis polynomials,
kernel values at the node tuples) and evaluates it at given points, so that
tests can compare it with the kernel itself (brute force) and show how its
error falls with p_s and p_t.  Kernels (eq. U, d = 2, a = c dt):

    K_phi(r, tau) = (c tau - r)_+^2 / (r a^2),   K_A = dK_phi/dt = 2 c (c tau - r)_+ / (r a^2).
"""
from __future__ import annotations

import numpy as np


def cheb_nodes(p: int, lo: float, hi: float) -> np.ndarray:
    """p Chebyshev points of the first kind on [lo, hi]."""
    k = np.arange(p)
    return 0.5 * (lo + hi) + 0.5 * (hi - lo) * np.cos((2 * k + 1) * np.pi / (2 * p))


def lagrange_basis(nodes: np.ndarray, x: np.ndarray) -> np.ndarray:
    """L[i, j] = l_j(x_i), the Lagrange basis polynomials of `nodes` at the points x."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    p = len(nodes)
    L = np.ones((len(x), p))
    for j in range(p):
        for m in range(p):
            if m != j:
                L[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return L


def k_phi(r, tau, a: float, c: float = 1.0):
    return np.maximum(c * tau - r, 0.0) ** 2 / (r * a * a)


def k_A(r, tau, a: float, c: float = 1.0):
    return 2.0 * c * np.maximum(c * tau - r, 0.0) / (r * a * a)


class PairInterpolant:
    """The interpolant of `kernel` for target cell [xlo, xhi]^3 x I_t and
    source cell [ylo, yhi]^3 x I_s (each cell given by its lower corner and
    side), p_s points per direction, p_t per interval."""

    def __init__(self, kernel, xc, yc, side: float, It, Is, p_s: int, p_t: int, a: float):
        self.ax = [cheb_nodes(p_s, xc[k], xc[k] + side) for k in range(3)]
        self.ay = [cheb_nodes(p_s, yc[k], yc[k] + side) for k in range(3)]
        self.nt = cheb_nodes(p_t, *It)
        self.ns = cheb_nodes(p_t, *Is)
        X = np.stack(np.meshgrid(*self.ax, indexing="ij"), -1).reshape(-1, 3)
        Y = np.stack(np.meshgrid(*self.ay, indexing="ij"), -1).reshape(-1, 3)
        r = np.linalg.norm(X[:, None, :] - Y[None, :, :], axis=-1)  # [nx, ny]
        tau = self.nt[:, None] - self.ns[None, :]  # [p_t, p_t]
        # kernel at every node tuple: [nx, ny, p_t, p_t]
        self.K = kernel(r[:, :, None, None], tau[None, None, :, :], a)
        self.p_s = p_s

    def _space(self, axes, pts):
        """3-D tensor basis at pts [n, 3]: [n, p_s^3]."""
        Ls = [lagrange_basis(axes[k], pts[:, k]) for k in range(3)]
        return np.einsum("ni,nj,nk->nijk", *Ls).reshape(len(pts), -1)

    def __call__(self, x, y, t, s):
        """The interpolant at the sample points x, y [n, 3], t, s [n]."""
        Lx = self._space(self.ax, np.asarray(x, dtype=np.float64))
        Ly = self._space(self.ay, np.asarray(y, dtype=np.float64))
        Lt = lagrange_basis(self.nt, t)
        Ls = lagrange_basis(self.ns, s)
        return np.einsum("na,nb,nc,nd,abcd->n", Lx, Ly, Lt, Ls, self.K, optimize=True)
