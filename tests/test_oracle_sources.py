"""Pins of the oracle's inner integrals against closed-form retarded potentials
of a point source and of a straight-segment source (CPU only).

The inner integrals of eq. (layer_disc_tmp) (paper section 2.3) over a source
triangle T, seen from a point x, are

    phi[m] = int_T N(tau)/r dS,   A0[m] = int_T Nddot(tau)/r dS,   tau = m - r/(c dt),

with N the cardinal quadratic B-spline (section 2.2), plus the vector and MFIE
parts A1 and P1.  Two limits have closed forms that share nothing with the
oracle's adaptive polar quadrature:

* a point source: a triangle of size s far from x gives A f(centroid) up to
  O(s^2) (the centroid rule is exact for linear integrands), for phi, A0,
  A1 = int Nddot/r (y - x) dS and P1 = int g'(r)/r (y - x) dS;
* a line source: the thin isosceles triangle with its apex at z1 and a base of
  width 2w at z2, on the z axis, carries 2w (z - z1)/L of area per unit length,
  so phi and A0 reduce to integrals of (z - z1) P(R)/R dz along the segment,
  with P the B-spline's piece written as a polynomial in R = |x - (0, 0, z)|.
  Those integrals are elementary (asinh, powers of R); the width direction
  adds O(w^2) only, the triangle being symmetric about the segment.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle


def _pieces():
    """The quadratic B-spline's pieces on [k, k+1] as (alpha, beta, gamma) of
    alpha tau^2 + beta tau + gamma (de Boor's recurrence, textbook values)."""
    return {0: (0.5, 0.0, 0.0), 1: (-1.0, 3.0, -1.5), 2: (0.5, -3.0, 4.5)}


def _N(t, q=0):
    """q-th derivative (q = 0, 1, 2) of the cardinal quadratic B-spline."""
    if t <= 0 or t >= 3:
        return 0.0
    al, be, ga = _pieces()[int(math.floor(t))]
    return [al * t * t + be * t + ga, 2 * al * t + be, 2 * al][q]


def _tet(face):
    """A closed mesh (tetrahedron) whose face 0 is `face`, the fourth vertex far behind it."""
    face = np.asarray(face, dtype=np.float64)
    c = face.mean(0)
    n = np.cross(face[1] - face[0], face[2] - face[0])
    n /= np.linalg.norm(n)
    v = np.vstack([face, c - 5.0 * n])
    t = np.array([[0, 1, 2], [0, 3, 1], [1, 3, 2], [2, 3, 0]], dtype=np.int32)
    return v, t


@pytest.mark.parametrize("R", [1.234, 2.05])
def test_point_source_limit(R):
    a = 0.3  # c dt, c = 1
    s = 1e-4
    c0 = np.array([0.2, -0.1, 0.3])
    face = c0 + s * np.array([[1.0, 0.0, 0.0], [-0.5, 0.8, 0.1], [-0.5, -0.8, -0.1]])
    v, t = _tet(face)
    o = Oracle(v, t, dt=a)  # theta = zeta = chi = 1
    A = 0.5 * np.linalg.norm(np.cross(face[1] - face[0], face[2] - face[0]))
    cen = face.mean(0)
    d = np.array([0.6, -0.7, 0.38])
    x = cen + R * d / np.linalg.norm(d)
    nm = int(math.ceil(R / a + 3))
    phi, A0, A1, P1 = o.inner(x, 0, 1, nm)
    dt, chi, zeta = a, 1.0, 1.0
    e = cen - x
    for i in range(nm):
        tau = (1 + i) - R / a
        assert min(abs(tau - k) for k in range(4)) > 0.05  # no knot circle crosses the small triangle
        f_phi = A * _N(tau) / R
        f_A0 = A * _N(tau, 2) / R
        G = chi * _N(tau, 1) / dt + zeta * _N(tau)
        Gp = chi * _N(tau, 2) / dt + zeta * _N(tau, 1)
        gp = -Gp / (a * R) - G / R ** 2  # d/dr [G(tau(r))/r], dtau/dr = -1/a
        sc_phi = max(A / R, 1e-300)
        assert abs(phi[i] - f_phi) <= 1e-6 * sc_phi, (i, phi[i], f_phi)
        assert abs(A0[i] - f_A0) <= 1e-6 * 2 * sc_phi, (i, A0[i], f_A0)
        np.testing.assert_allclose(A1[i], f_A0 * e, atol=1e-6 * 2 * sc_phi * R)
        np.testing.assert_allclose(P1[i], A * gp / R * e, atol=1e-6 * A * (1 / (a * a * dt) + 1 / R ** 2) * 4)


def _segment_closed_form(x, z1, z2, a, m, q):
    """int_{z1}^{z2} (z - z1) N^(q)(m - R/a)/R dz, R = |x - (0, 0, z)|, by pieces
    (q = 0: N, q = 2: Nddot), with the elementary antiderivatives
      int u R^(j-1) du = R^(j+1)/(j+1),
      int R^-1 du = asinh(u/rho), int 1 du = u, int R du = (u R + rho^2 asinh(u/rho))/2,
    u = z - x_z, rho the distance of x from the z axis."""
    rho = math.hypot(x[0], x[1])
    z0 = x[2]
    u1, u2 = z1 - z0, z2 - z0
    u0 = z0 - z1  # z - z1 = u + u0
    cuts = {u1, u2}
    if u1 < 0 < u2:
        cuts.add(0.0)
    for k in range(4):  # knot circles R = a (m - k)
        Rk = a * (m - k)
        if Rk > rho:
            for sgn in (-1, 1):
                u = sgn * math.sqrt(Rk * Rk - rho * rho)
                if u1 < u < u2:
                    cuts.add(u)
    cuts = sorted(cuts)
    R = lambda u: math.hypot(rho, u)
    ash = lambda u: math.asinh(u / rho)
    K = [ash, lambda u: u, lambda u: 0.5 * (u * R(u) + rho * rho * ash(u))]  # int R^(j-1) du
    total = 0.0
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        tau_mid = m - R(0.5 * (lo + hi)) / a
        if tau_mid <= 0 or tau_mid >= 3:
            continue
        al, be, ga = _pieces()[int(math.floor(tau_mid))]
        if q == 2:
            al, be, ga = 0.0, 0.0, 2 * al
        # alpha tau^2 + beta tau + gamma with tau = m - R/a, as d0 + d1 R + d2 R^2
        dj = [al * m * m + be * m + ga, -(2 * al * m + be) / a, al / (a * a)]
        for j in range(3):
            if dj[j] == 0.0:
                continue
            F = lambda u: R(u) ** (j + 1) / (j + 1) + u0 * K[j](u)
            total += dj[j] * (F(hi) - F(lo))
    return total


@pytest.mark.parametrize("x", [(0.25, 0.3, 0.1), (0.9, -0.2, 1.4), (0.05, 0.31, -0.45)])
def test_segment_source_limit(x):
    a, w = 0.3, 1e-4
    z1, z2 = -0.5, 0.7
    L = z2 - z1
    face = np.array([[0.0, 0.0, z1], [w, 0.0, z2], [-w, 0.0, z2]])
    v, t = _tet(face)
    o = Oracle(v, t, dt=a)
    x = np.asarray(x, dtype=np.float64)
    rmax = max(np.linalg.norm(x - p) for p in face)
    nm = int(math.ceil(rmax / a + 3))
    phi, A0, _, _ = o.inner(x, 0, 1, nm)
    ref_phi = np.array([2 * w / L * _segment_closed_form(x, z1, z2, a, 1 + i, 0) for i in range(nm)])
    ref_A0 = np.array([2 * w / L * _segment_closed_form(x, z1, z2, a, 1 + i, 2) for i in range(nm)])
    assert np.abs(ref_phi).max() > 0 and np.abs(ref_A0).max() > 0
    assert np.abs(phi - ref_phi).max() <= 1e-6 * np.abs(ref_phi).max()
    assert np.abs(A0 - ref_A0).max() <= 1e-6 * np.abs(ref_A0).max()


def test_segment_closed_form_against_quadrature():
    """The closed form itself against scipy's adaptive quadrature of its own
    definition (the integrand written directly from N, R and the weight)."""
    from scipy.integrate import quad

    x, a, z1, z2 = np.array([0.25, 0.3, 0.1]), 0.3, -0.5, 0.7
    rho = math.hypot(x[0], x[1])
    for m in range(1, 8):
        for q in (0, 2):
            f = lambda z: (z - z1) * _N(m - math.hypot(rho, z - x[2]) / a, q) / math.hypot(rho, z - x[2])
            knots = [x[2] + sg * math.sqrt((a * (m - k)) ** 2 - rho * rho) for k in range(4) for sg in (-1, 1)
                     if a * (m - k) > rho]
            ref, _ = quad(f, z1, z2, points=[p for p in knots if z1 < p < z2] or None, limit=200, epsabs=1e-14,
                          epsrel=1e-12)
            got = _segment_closed_form(x, z1, z2, a, m, q)
            assert abs(got - ref) <= 1e-10 * max(1.0, abs(ref)), (m, q, got, ref)


def test_planted_wrong_retardation_fails_the_point_pin():
    """The point pin detects a retardation with the wrong speed: the closed
    form with tau = m - r/(2a) disagrees with the oracle by far more than the
    bar."""
    a, s, R = 0.3, 1e-4, 1.234
    c0 = np.array([0.2, -0.1, 0.3])
    face = c0 + s * np.array([[1.0, 0.0, 0.0], [-0.5, 0.8, 0.1], [-0.5, -0.8, -0.1]])
    v, t = _tet(face)
    o = Oracle(v, t, dt=a)
    A = 0.5 * np.linalg.norm(np.cross(face[1] - face[0], face[2] - face[0]))
    x = face.mean(0) + R * np.array([0.6, -0.7, 0.38]) / np.linalg.norm([0.6, -0.7, 0.38])
    nm = int(math.ceil(R / a + 3))
    phi = o.inner(x, 0, 1, nm)[0]
    wrong = np.array([A * _N((1 + i) - R / (2 * a)) / R for i in range(nm)])
    assert np.abs(phi - wrong).max() > 1e-2 * A / R
