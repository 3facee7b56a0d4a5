"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: textbook
B-spline pieces, numpy's Gauss-Legendre rule, closed forms of the inner
integrals when the light-cone support is a full disk inside the triangle, an
independent 2D polar quadrature of the inner integrals written from their
definition (paper section 2.3, eq. layer_disc_tmp), invariance of the
discretised operator under rigid motions, its dimensional scaling law, and the
late-time decay of the marched current.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle, bspline, bspline_weights, gauss_legendre


# --------------------------------------------------------------------------
# B-spline (paper section 2.2: N^{beta,d} as d+2 truncated powers)
def N_textbook(t):
    """Cardinal quadratic B-spline on [0, 3], piecewise (de Boor's recurrence)."""
    if t <= 0 or t >= 3:
        return 0.0
    if t < 1:
        return t * t / 2
    if t < 2:
        return (-2 * t * t + 6 * t - 3) / 2
    return (3 - t) ** 2 / 2


def test_bspline_weights_match_formula_values():
    # w^{k,d} = (d+1)/prod_{i != k}(i - k): d=2 -> 1/2, -3/2, 3/2, -1/2; d=1 -> 1, -2, 1 (hat)
    np.testing.assert_allclose(bspline_weights(2), [0.5, -1.5, 1.5, -0.5], rtol=0, atol=1e-15)
    np.testing.assert_allclose(bspline_weights(1), [1.0, -2.0, 1.0], rtol=0, atol=1e-15)


def test_bspline_equals_textbook_pieces_and_partition_of_unity():
    rng = np.random.default_rng(0)
    for t in rng.uniform(-1, 4, 200):
        assert abs(bspline(t) - N_textbook(t)) < 1e-14
    assert abs(bspline(1.0) - 0.5) < 1e-15 and abs(bspline(2.0) - 0.5) < 1e-15
    for t in rng.uniform(0, 1, 50):
        assert abs(sum(bspline(t + k) for k in range(-1, 4)) - 1.0) < 1e-14


def test_bspline_derivatives_and_running_integral():
    rng = np.random.default_rng(1)
    h = 1e-6
    for t in rng.uniform(0.05, 2.95, 60):
        if min(abs(t - k) for k in range(4)) < 1e-3:
            continue
        fd1 = (N_textbook(t + h) - N_textbook(t - h)) / (2 * h)
        assert abs(bspline(t, 1) - fd1) < 1e-7
        assert bspline(t, 2) == {0: 1.0, 1: -2.0, 2: 1.0}[int(t)]
        xs, ws = np.polynomial.legendre.leggauss(20)
        acc = 0.0
        for lo in range(0, int(t) + 1):
            hi = min(t, lo + 1)
            acc += sum(w * N_textbook(lo + (hi - lo) * (x + 1) / 2) * (hi - lo) / 2 for x, w in zip(xs, ws))
        assert abs(bspline(t, -1) - acc) < 1e-13
    assert bspline(3.5, -1) == 1.0 and bspline(3.5, 0) == 0.0


def test_vanishing_property_pointwise():
    # sum_k w^k (tau - k)_+^2 == 0 for tau >= d+1 (paper eq. vanish): the third
    # difference of a quadratic polynomial
    w = bspline_weights(2)
    for tau in [3.0, 3.3, 7.9, 55.2]:
        s = sum(w[k] * max(tau - k, 0.0) ** 2 for k in range(4))
        assert abs(s) < 1e-10 * tau * tau


def test_gauss_legendre_rule():
    x, w = gauss_legendre()
    xr, wr = np.polynomial.legendre.leggauss(len(x))
    np.testing.assert_allclose(np.sort(x), np.sort(xr), atol=1e-15)
    np.testing.assert_allclose(w[np.argsort(x)], wr[np.argsort(xr)], atol=1e-15)


# --------------------------------------------------------------------------
# Inner integrals
def _big_triangle_oracle(a=1.0):
    side = 30.0
    v = np.array([[0, 0, 0], [side, 0, 0], [side / 2, side * math.sqrt(3) / 2, 0],
                  [side / 2, side * math.sqrt(3) / 6, -5.0]], dtype=np.float64)
    t = np.array([[0, 1, 2], [0, 3, 1], [1, 3, 2], [2, 3, 0]], dtype=np.int32)
    return Oracle(v, t, dt=a), v


@pytest.mark.parametrize("h", [0.0, 0.37, -0.9, 2.4])
def test_inner_disk_closed_forms(h):
    """Light-cone support is a full disk around p inside the triangle: then
    int N/r dS = 2 pi a C(m - |h|/a), int Nddot/r dS = 2 pi a Ndot(m - |h|/a),
    the in-plane vector parts vanish and int g'(r)/r (y-x) dS = 2 pi h g(|h|) n."""
    a = 1.0
    o, v = _big_triangle_oracle(a)
    c = v[:3].mean(0)
    n = np.array([0.0, 0.0, 1.0])
    x = c + h * n
    m0, nm = 1, 7  # support r < 7a, inradius 8.66a
    phi, A0, A1, P1 = o.inner(x, 0, m0, nm)
    zeta, dt = 1.0, a
    for i in range(nm):
        m = m0 + i
        tau = m - abs(h) / a
        assert abs(phi[i] - 2 * math.pi * a * bspline(tau, -1)) < 1e-12
        assert abs(A0[i] - 2 * math.pi * a * bspline(tau, 1)) < 1e-12
        np.testing.assert_allclose(A1[i], -h * n * A0[i], atol=1e-11)
        if h != 0.0:
            g = (bspline(tau, 1) / dt + zeta * bspline(tau, 0)) / abs(h)
            np.testing.assert_allclose(P1[i], 2 * math.pi * h * g * n, atol=1e-11)
        else:
            assert np.all(P1[i] == 0.0)


def _polar_bruteforce(o, x, tri, m0, nm, a, dt, zeta):
    """2D integrals over triangle ``tri`` written from their definition, in polar
    coordinates about the projection p of x, with scipy's adaptive quad_vec in
    rho (split at the light-cone radii) and in theta (split at the vertices)."""
    from scipy.integrate import quad_vec

    v = o.verts[o.tris[tri]]
    n = np.cross(v[1] - v[0], v[2] - v[0])
    n /= np.linalg.norm(n)
    h = (x - v[0]) @ n
    p = x - h * n
    e1 = (v[1] - v[0]) / np.linalg.norm(v[1] - v[0])
    e2 = np.cross(n, e1)
    P2 = np.array([[(vv - p) @ e1, (vv - p) @ e2] for vv in v])
    # inward normals of the 2D triangle (counter-clockwise)
    inw = []
    for k in range(3):
        d = P2[(k + 1) % 3] - P2[k]
        inw.append((np.array([-d[1], d[0]]), P2[k]))

    def ray_range(th):
        u = np.array([math.cos(th), math.sin(th)])
        lo, hi = 0.0, np.inf
        for nu, q in inw:
            # inside: (t u - q) . nu >= 0
            den = u @ nu
            num = q @ nu
            if abs(den) < 1e-300:
                if num > 0:
                    return 1.0, 0.0
                continue
            t = num / den
            if den > 0:
                lo = max(lo, t)
            else:
                hi = min(hi, t)
        return lo, hi

    def Nq(tau, q):
        # textbook pieces of the quadratic B-spline and its first two derivatives
        if tau <= 0 or tau >= 3:
            return 0.0
        k = int(tau)
        if q == 0:
            return N_textbook(tau)
        if q == 1:
            return (tau, -2 * tau + 3, tau - 3)[k]
        return (1.0, -2.0, 1.0)[k]

    knots_r = [j * a for j in range(1, 200)]

    def integrand_rho(rho, th):
        u = math.cos(th) * e1 + math.sin(th) * e2
        r = math.sqrt(h * h + rho * rho)
        ymx = rho * u - h * n
        out = []
        for i in range(nm):
            tau = m0 + i - r / a
            F_phi = Nq(tau, 0) / r
            F_A = Nq(tau, 2) / r
            g = (Nq(tau, 1) / dt + zeta * Nq(tau, 0)) / r
            if abs(h) > 1e-12:
                gp = ((-Nq(tau, 2) / a / dt - zeta * Nq(tau, 1) / a) * r - (Nq(tau, 1) / dt + zeta * Nq(tau, 0))) / (r * r)
            else:  # in-plane observation point: the P-term is not compared (it is tested as zero)
                gp = 0.0
            out += [F_phi * rho, F_A * rho, *(F_A * ymx * rho), *(gp / r * ymx * rho)]
        return np.array(out)

    def inner_theta(th):
        lo, hi = ray_range(th)
        if not hi > lo:
            return np.zeros(8 * nm)
        pts = [math.sqrt(R * R - h * h) for R in knots_r if R * R - h * h > 0]
        pts = [q for q in pts if lo < q < hi]
        return quad_vec(lambda rr: integrand_rho(rr, th), lo, hi, points=pts or None, epsabs=1e-14,
                        epsrel=1e-12, limit=400)[0]

    angs = sorted(math.atan2(q[1], q[0]) % (2 * math.pi) for q in P2)
    bounds = [0.0] + angs + [2 * math.pi]
    tot = np.zeros(8 * nm)
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        if hi - lo > 1e-15:
            tot += quad_vec(inner_theta, lo, hi, epsabs=1e-13, epsrel=1e-11, limit=400)[0]
    tot = tot.reshape(nm, 8)
    return tot[:, 0], tot[:, 1], tot[:, 2:5], tot[:, 5:8], h


@pytest.mark.parametrize("case", ["above_inside", "coplanar_outside", "offplane_outside", "far", "self_point"])
def test_inner_matches_polar_bruteforce(case):
    a = 0.3
    v = np.array([[0.0, 0.0, 0.0], [0.6, 0.05, 0.0], [0.2, 0.55, 0.1], [0.3, 0.2, -0.6]])
    t = np.array([[0, 1, 2], [0, 3, 1], [1, 3, 2], [2, 3, 0]], dtype=np.int32)
    o = Oracle(v, t, dt=a)
    c = v[:3].mean(0)
    nrm = np.cross(v[1] - v[0], v[2] - v[0])
    nrm /= np.linalg.norm(nrm)
    x = {
        "above_inside": c + 0.13 * nrm + 0.05 * (v[1] - v[0]),
        "coplanar_outside": v[0] + 1.3 * (v[1] - v[0]) + 0.4 * (v[2] - v[1]),
        "offplane_outside": v[0] + 1.1 * (v[1] - v[0]) + 0.3 * (v[2] - v[1]) + 0.08 * nrm,
        "far": c + 2.1 * nrm + 1.3 * (v[1] - v[0]),
        "self_point": 0.2 * v[0] + 0.5 * v[1] + 0.3 * v[2],
    }[case]
    dmax = np.linalg.norm(v[:3] - x, axis=1).max()
    m0, nm = 1, int(math.ceil(dmax / a + 3))
    phi, A0, A1, P1 = o.inner(x, 0, m0, nm)
    bphi, bA0, bA1, bP1, h = _polar_bruteforce(o, x, 0, m0, nm, a, a, 1.0)
    sc = lambda u: max(1e-300, np.abs(u).max())
    assert np.abs(phi - bphi).max() < 1e-9 * sc(bphi)
    assert np.abs(A0 - bA0).max() < 1e-9 * sc(bA0)
    assert np.abs(A1 - bA1).max() < 1e-9 * sc(bA1)
    if abs(h) > 1e-12:
        assert np.abs(P1 - bP1).max() < 1e-8 * sc(bP1)


# --------------------------------------------------------------------------
# Assembled operator
def _all_lags(o):
    m_lo, Zw = o.assemble()
    W = Zw.shape[2]
    mmax = int(m_lo.max()) + W
    out = np.zeros((mmax + 1, o.ne, o.ne))
    for w in range(W):
        r, j = np.nonzero(np.ones_like(m_lo, bool))
        out[m_lo[r, j] + w, r, j] = Zw[r, j, w]
    return out


def test_operator_invariant_under_rigid_motion():
    from workloads import icosphere, mean_edge_length

    v, t = icosphere(1.0, 1)
    dt = 0.5 * mean_edge_length(v, t)
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    R = R @ np.array([[1, 0, 0], [0, math.cos(0.3), -math.sin(0.3)], [0, math.sin(0.3), math.cos(0.3)]])
    Z = _all_lags(Oracle(v, t, dt))
    Zr = _all_lags(Oracle(v @ R.T + np.array([3.0, -1.0, 2.5]), t, dt))
    np.testing.assert_allclose(Zr, Z, atol=1e-11 * np.abs(Z).max(), rtol=0)


def test_operator_dimensional_scaling():
    """Scaling lengths and dt by s (and zeta by 1/s) scales every Zt^(m) by s:
    each term is (area)^2 / length times 1/dt^2, 1/length^2 or 1/(length dt)."""
    from workloads import icosphere, mean_edge_length

    v, t = icosphere(1.0, 1)
    dt = 0.5 * mean_edge_length(v, t)
    s = 2.5
    Z = _all_lags(Oracle(v, t, dt, zeta=1.0))
    Zs = _all_lags(Oracle(s * v, t, s * dt, zeta=1.0 / s))
    np.testing.assert_allclose(Zs, s * Z, atol=1e-11 * np.abs(s * Z).max(), rtol=0)


def test_instantaneous_matrix_is_local_and_well_conditioned(sphere320_oracle):
    """Zt^(1) couples only edges whose supports come within c dt (tau = 1 - r/(c dt) > 0)."""
    w, o = sphere320_oracle
    Z1 = o.z_lag(1)
    ev, et, eo = o.edges()
    V = o.verts
    # supports of two edges further apart than c dt cannot couple at lag 1
    supp = [set(o.tris[et[i, 0]]) | set(o.tris[et[i, 1]]) for i in range(o.ne)]
    rng = np.random.default_rng(0)
    for i in rng.choice(o.ne, 20, replace=False):
        for j in np.nonzero(Z1[i])[0]:
            dmin = min(np.linalg.norm(V[p] - V[q]) for p in supp[i] for q in supp[j])
            assert dmin < 2.5 * w.dt + 1e-12
    assert np.linalg.cond(Z1) < 10


def test_march_late_time_decay(sphere320_oracle, sphere320_march):
    J = sphere320_march
    peak = np.abs(J).max()
    assert peak > 0.1
    assert np.abs(J[-10:]).max() < 1e-3 * peak


@pytest.fixture(scope="module")
def sphere80_oracle():
    from workloads import workload

    w = workload("sphere80")
    o = Oracle(w.verts, w.tris, w.dt)
    o.assemble()
    return w, o


def test_march_is_shift_invariant_in_time(sphere80_oracle):
    """Delaying the incident pulse by k whole steps delays the marched currents
    by exactly k steps (the incident field is sampled at t = alpha dt and the
    history sum only involves lags): a one-step error in the time argument of
    the right-hand side, in the history indices or in the lag convention
    breaks it.  The pulse is centred late enough (t0 = 12 sigma) that its
    value before step 0 is below 1e-30 of its peak."""
    import dataclasses

    w, o = sphere80_oracle
    p0 = dataclasses.replace(w.pulses[0], t0=12.0 * w.pulses[0].sigma)
    k = 3
    p1 = dataclasses.replace(p0, t0=p0.t0 + k * w.dt)
    Nt = 64
    J0 = o.march(p0, Nt)
    J1 = o.march(p1, Nt)
    scale = np.abs(J0).max()
    assert scale > 0
    assert np.abs(J1[:k]).max() <= 1e-12 * scale
    assert np.abs(J1[k:] - J0[: Nt - 1 - k]).max() <= 1e-11 * scale


def test_march_superposes_right_hand_sides(sphere80_oracle):
    """The march of the sum of two incident waves' right-hand sides is the
    sum of their marches (the batched form relies on this linearity)."""
    import dataclasses

    w, o = sphere80_oracle
    pa = w.pulses[0]
    pb = dataclasses.replace(pa, k=(1.0, 0.0, 0.0), pol=(0.0, 0.0, 1.0),
                             z_min=float(np.min(np.asarray(w.verts)[:, 0])))
    Nt = 40
    Va = np.array([o.rhs(pa, a) for a in range(1, Nt)])
    Vb = np.array([o.rhs(pb, a) for a in range(1, Nt)])
    Ja = o.march(None, Nt, V_all=Va)
    Jb = o.march(None, Nt, V_all=Vb)
    Jab = o.march(None, Nt, V_all=Va + 2.5 * Vb)
    assert np.abs(Jab - (Ja + 2.5 * Jb)).max() <= 1e-12 * np.abs(Jab).max()
    # and a caller-supplied table equal to the plane wave's gives its march
    assert np.abs(Ja - o.march(pa, Nt)).max() <= 1e-13 * np.abs(Ja).max()
