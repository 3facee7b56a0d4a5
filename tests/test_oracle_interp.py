"""Interpolation error of the space-time FMM against brute force (CPU only).

oracle/interp.py builds the tensor-product Lagrange interpolant of the kernel
of eq. U between a target cell and a source cell two cells away (offset
(2, 0, 0), the nearest far offset of Program 4), from its definition on
Chebyshev points (section 3.2, eq. U_expand).  Here it is compared with the
kernel itself at random points of the two cells and time intervals:

* inside the light cone (c tau > r for every point pair) the kernels are
  smooth: the error falls geometrically with p_s, and in time the
  interpolant reproduces K_phi (quadratic in tau) from p_t = 3 and K_A
  (linear) from p_t = 2, down to the spatial error;
* across the light cone (c tau = r inside the cells) the truncated power
  breaks the smoothness and the error falls only slowly with p_t: the
  mechanism behind the fast path's accuracy floor.

The interpolant itself is pinned first: it reproduces a polynomial of degree
p - 1 in each variable to rounding.
"""
import numpy as np
import pytest

from oracle.interp import PairInterpolant, k_A, k_phi

A = 0.25  # c dt
SIDE = 1.0
XC, YC = np.zeros(3), np.array([2.0, 0.0, 0.0])
INSIDE = ((9.0, 10.0), (4.0, 5.0))  # c tau in [4, 6] > r in [1, 3.32]
CROSS = ((4.0, 5.0), (1.5, 2.5))  # c tau in [1.5, 3.5]: the cone crosses the cells


def _samples(n=300, seed=3, It=INSIDE[0], Is=INSIDE[1]):
    rng = np.random.default_rng(seed)
    x = XC + rng.random((n, 3)) * SIDE
    y = YC + rng.random((n, 3)) * SIDE
    t = It[0] + rng.random(n) * (It[1] - It[0])
    s = Is[0] + rng.random(n) * (Is[1] - Is[0])
    return x, y, t, s


def _err(kern, p_s, p_t, It, Is):
    x, y, t, s = _samples(It=It, Is=Is)
    P = PairInterpolant(kern, XC, YC, SIDE, It, Is, p_s, p_t, A)
    exact = kern(np.linalg.norm(x - y, axis=1), t - s, A)
    return np.abs(P(x, y, t, s) - exact).max() / np.abs(exact).max()


def test_interpolant_reproduces_polynomials():
    """A kernel polynomial of degree p_s - 1 in each coordinate and p_t - 1 in
    t and s is reproduced to rounding (pins the nodes and the basis)."""
    p_s, p_t = 3, 4
    It, Is = INSIDE

    class Poly(PairInterpolant):
        def __init__(self):
            super().__init__(k_phi, XC, YC, SIDE, It, Is, p_s, p_t, A)
            X = np.stack(np.meshgrid(*self.ax, indexing="ij"), -1).reshape(-1, 3)
            Y = np.stack(np.meshgrid(*self.ay, indexing="ij"), -1).reshape(-1, 3)
            self.K = _f(X[:, None, None, None, :], Y[None, :, None, None, :], self.nt[None, None, :, None],
                        self.ns[None, None, None, :])

    def _f(x, y, t, s):
        return ((1 + x[..., 0] ** 2 - 0.5 * x[..., 1] * x[..., 2]) * (y[..., 0] - 2 * y[..., 1] ** 2 + y[..., 2])
                * (t ** 3 - 0.7 * t) * (1.0 + s - 0.2 * s * s))

    x, y, t, s = _samples()
    got = Poly()(x, y, t, s)
    ref = _f(x, y, t, s)
    assert np.abs(got - ref).max() <= 1e-11 * np.abs(ref).max()


@pytest.mark.parametrize("kern", [k_phi, k_A])
def test_space_error_falls_with_p_s_inside_the_cone(kern):
    e = [_err(kern, p, 4, *INSIDE) for p in (2, 3, 4, 5, 6)]
    print(f"\n{kern.__name__} inside the cone, p_s = 2..6:", " ".join(f"{v:.1e}" for v in e))
    assert all(b < a for a, b in zip(e, e[1:])), e
    assert e[-1] < e[0] / 500


def test_time_interpolation_reproduces_the_tau_polynomials_inside_the_cone():
    """K_phi is quadratic and K_A linear in tau where c tau > r: from p_t = 3
    (K_phi) and p_t = 2 (K_A) only the spatial error is left."""
    floor_phi = _err(k_phi, 6, 6, *INSIDE)
    floor_A = _err(k_A, 6, 6, *INSIDE)
    assert _err(k_phi, 6, 2, *INSIDE) > 30 * floor_phi
    assert _err(k_phi, 6, 3, *INSIDE) < 1.5 * floor_phi
    assert _err(k_A, 6, 1, *INSIDE) > 30 * floor_A
    assert _err(k_A, 6, 2, *INSIDE) < 1.5 * floor_A


@pytest.mark.parametrize("kern, factor", [(k_phi, 3.0), (k_A, 30.0)])
def test_light_cone_crossing_slows_time_convergence(kern, factor):
    """Across the light cone the error falls with p_t at first and then levels
    off above the smooth case's floor (p_s = 6, p_t = 6): at p_t = 8 about 5
    times that floor for K_phi, whose second derivative jumps on the cone, and
    about 130 times for K_A, which has a kink there."""
    e = [_err(kern, 6, p, *CROSS) for p in (2, 3, 4, 6, 8)]
    print(f"\n{kern.__name__} across the cone, p_t = 2, 3, 4, 6, 8:", " ".join(f"{v:.1e}" for v in e))
    assert e[-1] < 0.5 * e[0] and min(e) >= 0.99 * e[-1], e
    assert e[-1] > factor * _err(kern, 6, 6, *INSIDE)
