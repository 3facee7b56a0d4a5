"""Pins of the oracle's inner integrals against the closed-form triangle
integrals of 1/R and R (CPU only).

For an observation point x, let p be its projection on the plane of the
source triangle T and h its height.  T splits into the three sub-triangles
(p, v_a, v_b) over its edges, signed by the in-plane distance d from p to the
edge line (positive on the inner side).  In polar coordinates about p, with
s the coordinate along the edge (s_a < s_b at its ends), R0^2 = d^2 + h^2 and
R(s) = sqrt(R0^2 + s^2), the radial integrals are elementary and the angular
ones follow by s = |d| tan(theta):

  int 1/R dS over (p, v_a, v_b) = sign(d) [ |d| asinh(s/R0)
        + |h| atan(|h| s / (|d| R)) - |h| atan(s/|d|) ]_{s_a}^{s_b},
  int R dS over (p, v_a, v_b)   = sign(d)/3 [ |d| s R/2 + |d| (R0^2/2 + h^2) asinh(s/R0)
        + |h|^3 atan(|h| s / (|d| R)) - |h|^3 atan(s/|d|) ]_{s_a}^{s_b}.

(derived here from the definitions, and checked below against scipy's
adaptive quadrature).  When every point of T lies within one piece
[k, k+1] of the quadratic B-spline in tau = m - r/(c dt), the piece is a
polynomial d0 + d1 r + d2 r^2 and

  phi[m] = int_T N(tau)/r dS = d0 int 1/R + d1 area + d2 int R,
  A0[m]  = int_T Nddot(tau)/r dS = 2 alpha_k int 1/R,

with alpha_k the leading coefficient of the piece: closed forms for the
oracle's inner integrals at any observation point, not only above the disk.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle

TRI = np.array([[0.0, 0.0, 0.0], [0.6, 0.05, 0.0], [0.2, 0.55, 0.1]])


def _edge_terms(x, v):
    n = np.cross(v[1] - v[0], v[2] - v[0])
    n /= np.linalg.norm(n)
    h = float(np.dot(x - v[0], n))
    p = x - h * n
    out = []
    for k in range(3):
        va, vb = v[k], v[(k + 1) % 3]
        t = (vb - va) / np.linalg.norm(vb - va)
        u = np.cross(t, n)  # in-plane, outward for a counter-clockwise triangle about n
        d = float(np.dot(va - p, u))
        out.append((d, float(np.dot(va - p, t)), float(np.dot(vb - p, t))))
    return h, out


def int_inv_r(x, v):
    h, edges = _edge_terms(x, v)
    ah = abs(h)
    total = 0.0
    for d, sa, sb in edges:
        if abs(d) < 1e-14:
            continue
        ad, R0 = abs(d), math.hypot(d, h)

        def F(s):
            R = math.hypot(R0, s)
            return ad * math.asinh(s / R0) + ah * math.atan(ah * s / (ad * R)) - ah * math.atan(s / ad)

        total += math.copysign(1.0, d) * (F(sb) - F(sa))
    return total


def int_r(x, v):
    h, edges = _edge_terms(x, v)
    ah = abs(h)
    total = 0.0
    for d, sa, sb in edges:
        if abs(d) < 1e-14:
            continue
        ad, R0 = abs(d), math.hypot(d, h)

        def F(s):
            R = math.hypot(R0, s)
            return (ad * s * R / 2 + ad * (R0 * R0 / 2 + h * h) * math.asinh(s / R0)
                    + ah ** 3 * math.atan(ah * s / (ad * R)) - ah ** 3 * math.atan(s / ad))

        total += math.copysign(1.0, d) * (F(sb) - F(sa)) / 3
    return total


POINTS = {
    "above_inside": TRI.mean(0) + np.array([0.05, -0.03, 0.37]),
    "below_outside": np.array([0.9, -0.4, -0.55]),
    "far": np.array([1.1, 0.9, 1.3]),
    "coplanar_outside": TRI[0] + 1.4 * (TRI[1] - TRI[0]) + 0.3 * (TRI[2] - TRI[1]),
}


@pytest.mark.parametrize("name", list(POINTS))
def test_closed_forms_against_quadrature(name):
    """The two closed forms against scipy's adaptive quadrature over the
    triangle (barycentric parametrisation, its own Jacobian)."""
    from scipy.integrate import dblquad

    x = POINTS[name]
    v = TRI
    e1, e2 = v[1] - v[0], v[2] - v[0]
    jac = np.linalg.norm(np.cross(e1, e2))

    def integrand(b, a, f):
        y = v[0] + a * e1 + b * e2
        return f(np.linalg.norm(y - x)) * jac

    for f, closed in ((lambda r: 1.0 / r, int_inv_r), (lambda r: r, int_r)):
        ref, _ = dblquad(integrand, 0.0, 1.0, 0.0, lambda a: 1.0 - a, args=(f,), epsabs=1e-13, epsrel=1e-12)
        got = closed(x, v)
        assert abs(got - ref) <= 1e-9 * abs(ref), (name, got, ref)


def _tet(face):
    c = face.mean(0)
    n = np.cross(face[1] - face[0], face[2] - face[0])
    n /= np.linalg.norm(n)
    v = np.vstack([face, c - 5.0 * n])
    t = np.array([[0, 1, 2], [0, 3, 1], [1, 3, 2], [2, 3, 0]], dtype=np.int32)
    return v, t


PIECES = {0: (0.5, 0.0, 0.0), 1: (-1.0, 3.0, -1.5), 2: (0.5, -3.0, 4.5)}  # alpha tau^2 + beta tau + gamma


@pytest.mark.parametrize("name", ["below_outside", "far"])
def test_oracle_inner_integrals_equal_the_closed_forms(name):
    """c dt is set so that the light-cone band of lag m covers the whole
    triangle inside piece m - 2 of the B-spline (centred on tau = m - 1.5):
    lags 2, 3 and 4 then exercise the three pieces, and the oracle's phi and
    A0 there equal the closed forms."""
    x = POINTS[name]
    rmax = np.linalg.norm(TRI - x, axis=1).max()
    rmin = _min_distance(x, TRI)
    a = (rmax + rmin) / 3.0
    v, t = _tet(TRI)
    o = Oracle(v, t, dt=a)
    nm = int(math.ceil(rmax / a + 3))
    phi, A0, _, _ = o.inner(x, 0, 1, nm)
    I1, Ir = int_inv_r(x, TRI), int_r(x, TRI)
    area = 0.5 * np.linalg.norm(np.cross(TRI[1] - TRI[0], TRI[2] - TRI[0]))
    for m in (2, 3, 4):
        k = m - 2
        lo, hi = m - rmax / a, m - rmin / a  # tau over the triangle
        assert k < lo and hi < k + 1  # the band lies inside the piece
        al, be, ga = PIECES[k]
        d0, d1, d2 = al * m * m + be * m + ga, -(2 * al * m + be) / a, al / (a * a)
        ref_phi = d0 * I1 + d1 * area + d2 * Ir
        assert abs(phi[m - 1] - ref_phi) <= 1e-11 * max(abs(ref_phi), area / rmax), (m, phi[m - 1], ref_phi)
        assert abs(A0[m - 1] - 2 * al * I1) <= 1e-11 * abs(2 * al * I1), (m, A0[m - 1])


def _min_distance(x, v):
    """A lower bound of the distance from x to the triangle: the closest of a
    401 x 401 barycentric sample, less 1e-3 (more than the sample spacing's
    error), so the band checked above is never narrower than the true one."""
    g = np.linspace(0.0, 1.0, 401)
    A, B = np.meshgrid(g, g)
    msk = A + B <= 1.0
    Y = v[0] + A[msk, None] * (v[1] - v[0]) + B[msk, None] * (v[2] - v[0])
    best = np.linalg.norm(Y - x, axis=1).min()
    return best - 1e-3  # the sampling step bounds the error; a margin keeps the band inside the piece
