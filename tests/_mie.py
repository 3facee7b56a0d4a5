"""Mie series of a perfectly conducting sphere (test infrastructure).

Time-harmonic fields with the exp(-i omega t) convention, incident plane wave
E_i = x_hat exp(i k z), H_i = y_hat exp(i k z) / eta, expanded in vector
spherical harmonics with the azimuthal order 1 only.  The expansion follows the
standard textbook treatment of scattering by a sphere (vector harmonics
M_{e/o,1,n}, N_{e/o,1,n} built from z_n(k r) P_n^1(cos theta)); the perfect
conductor is the limit of infinite refractive index, which leaves the
coefficients

    a_n = psi_n'(ka) / xi_n'(ka),    b_n = psi_n(ka) / xi_n(ka),

psi_n(x) = x j_n(x), xi_n(x) = x h_n^(1)(x).  Nothing here is trusted by
recollection alone: ``check_expansion`` verifies the incident expansion against
the plane wave, the scattered electric field against the boundary condition
(zero tangential total E on the sphere) and the scattered magnetic field
against a finite-difference curl of the scattered electric field, so a wrong
sign or index anywhere in the harmonics fails it.

The physical surface current is J = n_out x (H_i + H_s) on r = a.
"""
from __future__ import annotations

import numpy as np
from scipy.special import spherical_jn, spherical_yn


def _pi_tau(nmax: int, mu: np.ndarray):
    """pi_n = P_n^1 / sin(theta) and tau_n = d P_n^1 / d theta, n = 1..nmax, by
    the upward recurrences of the associated Legendre functions of order 1."""
    pi = np.zeros((nmax + 1,) + mu.shape)
    tau = np.zeros_like(pi)
    pi[1] = 1.0
    for n in range(2, nmax + 1):
        pi[n] = ((2 * n - 1) * mu * pi[n - 1] - n * pi[n - 2]) / (n - 1)
    for n in range(1, nmax + 1):
        tau[n] = n * mu * pi[n] - (n + 1) * pi[n - 1]
    return pi[1:], tau[1:]


def _radial(n: np.ndarray, rho: np.ndarray, kind: int):
    """z_n(rho) and [rho z_n(rho)]'/rho for z = j_n (kind 1) or h_n^(1) (kind 3)."""
    j = spherical_jn(n, rho)
    jd = spherical_jn(n, rho, derivative=True)
    if kind == 1:
        z, zd = j, jd
    else:
        z = j + 1j * spherical_yn(n, rho)
        zd = jd + 1j * spherical_yn(n, rho, derivative=True)
    return z, (z + rho * zd) / rho


def _harmonics(n, r, th, ph, k, kind):
    """M_o1n, M_e1n, N_o1n, N_e1n at (r, theta, phi) in spherical components
    (r, theta, phi); arrays of shape (nmax, npts, 3)."""
    mu = np.cos(th)
    st = np.sin(th)
    pi, tau = _pi_tau(len(n), mu)
    rho = k * r
    z, dz = _radial(n[:, None], rho[None, :], kind)
    cp, sp = np.cos(ph)[None, :], np.sin(ph)[None, :]
    nn = (n * (n + 1))[:, None]
    zero = np.zeros_like(z)
    Mo = np.stack([zero, cp * pi * z, -sp * tau * z], axis=-1)
    Me = np.stack([zero, -sp * pi * z, -cp * tau * z], axis=-1)
    No = np.stack([sp * nn * st * pi * z / rho, sp * tau * dz, cp * pi * dz], axis=-1)
    Ne = np.stack([cp * nn * st * pi * z / rho, cp * tau * dz, -sp * pi * dz], axis=-1)
    return Mo, Me, No, Ne


def _sph_to_cart(v, th, ph):
    st, ct, sp, cp = np.sin(th), np.cos(th), np.sin(ph), np.cos(ph)
    er = np.stack([st * cp, st * sp, ct], axis=-1)
    et = np.stack([ct * cp, ct * sp, -st], axis=-1)
    ep = np.stack([-sp, cp, np.zeros_like(ph)], axis=-1)
    return v[..., 0:1] * er + v[..., 1:2] * et + v[..., 2:3] * ep


class PECSphere:
    """Fields of a unit-amplitude x-polarised plane wave along +z on a PEC
    sphere of radius ``a`` at wavenumber ``k`` (eps = mu = 1, eta = 1)."""

    def __init__(self, a: float, k: float, nmax: int | None = None):
        self.a, self.k = float(a), float(k)
        x = self.k * self.a
        self.nmax = nmax or int(x + 4.05 * x ** (1 / 3) + 10)
        n = np.arange(1, self.nmax + 1)
        self.n = n
        self.En = (1j ** n) * (2 * n + 1) / (n * (n + 1))
        j = spherical_jn(n, x)
        jd = spherical_jn(n, x, derivative=True)
        h = j + 1j * spherical_yn(n, x)
        hd = jd + 1j * spherical_yn(n, x, derivative=True)
        psi, dpsi = x * j, j + x * jd
        xi, dxi = x * h, h + x * hd
        self.an = dpsi / dxi
        self.bn = psi / xi

    @staticmethod
    def _sph(p):
        p = np.atleast_2d(np.asarray(p, dtype=np.float64))
        r = np.linalg.norm(p, axis=1)
        th = np.arccos(np.clip(p[:, 2] / r, -1.0, 1.0))
        ph = np.arctan2(p[:, 1], p[:, 0])
        return r, th, ph

    def fields(self, p, which: str):
        """Cartesian E or H ('Ei', 'Hi', 'Es', 'Hs') at points p (N x 3)."""
        r, th, ph = self._sph(p)
        k, n, En = self.k, self.n, self.En[:, None, None]
        if which in ("Ei", "Hi"):
            Mo, Me, No, Ne = _harmonics(n, r, th, ph, k, 1)
            v = (En * (Mo - 1j * Ne)).sum(0) if which == "Ei" else (-En * (Me + 1j * No)).sum(0)
        else:
            Mo, Me, No, Ne = _harmonics(n, r, th, ph, k, 3)
            a, b = self.an[:, None, None], self.bn[:, None, None]
            v = (En * (1j * a * Ne - b * Mo)).sum(0) if which == "Es" else (En * (1j * b * No + a * Me)).sum(0)
        return _sph_to_cart(v, th, ph)

    def surface_current(self, p):
        """Physical current n_out x H_total at points p projected onto r = a."""
        p = np.atleast_2d(np.asarray(p, dtype=np.float64))
        q = self.a * p / np.linalg.norm(p, axis=1, keepdims=True)
        H = self.fields(q, "Hi") + self.fields(q, "Hs")
        n = q / self.a
        return np.cross(n, H)

    def check_expansion(self, seed: int = 0) -> dict:
        """Largest relative residuals of the four self-checks (see module doc)."""
        rng = np.random.default_rng(seed)
        k, a = self.k, self.a
        # interior points: the incident expansion must equal the plane wave
        d = rng.standard_normal((20, 3))
        p_in = d / np.linalg.norm(d, axis=1, keepdims=True) * rng.uniform(0.1, 0.95, (20, 1)) * a
        ph = np.exp(1j * k * p_in[:, 2])[:, None]
        e_inc = np.abs(self.fields(p_in, "Ei") - ph * np.array([1.0, 0, 0])).max()
        h_inc = np.abs(self.fields(p_in, "Hi") - ph * np.array([0, 1.0, 0])).max()
        # on the sphere: tangential total E vanishes
        p_s = d / np.linalg.norm(d, axis=1, keepdims=True) * a
        nrm = p_s / a
        Et = self.fields(p_s, "Ei") + self.fields(p_s, "Es")
        e_bc = np.abs(np.cross(nrm, Et)).max()
        # outside: curl E_s = i omega mu H_s (omega = k when c = mu = 1)
        p_o = d / np.linalg.norm(d, axis=1, keepdims=True) * a * 1.7
        hstep = 1e-5
        curl = np.zeros((len(p_o), 3), complex)
        J = np.zeros((len(p_o), 3, 3), complex)  # J[:, i, j] = d E_i / d x_j
        for jx in range(3):
            e = np.zeros(3)
            e[jx] = hstep
            J[:, :, jx] = (self.fields(p_o + e, "Es") - self.fields(p_o - e, "Es")) / (2 * hstep)
        curl[:, 0] = J[:, 2, 1] - J[:, 1, 2]
        curl[:, 1] = J[:, 0, 2] - J[:, 2, 0]
        curl[:, 2] = J[:, 1, 0] - J[:, 0, 1]
        Hs = self.fields(p_o, "Hs")
        h_curl = np.abs(curl / (1j * k) - Hs).max() / np.abs(Hs).max()
        return {"incident_E": e_inc, "incident_H": h_inc, "boundary_E": e_bc, "curl_H": h_curl}


def transient_current(a: float, points, times, g, delay: float, along_minus_z: bool, dt: float,
                      f_cut: float, npad: int = 2):
    """Physical surface current n_out x H of the PEC sphere at `points` (N x 3)
    and `times` (multiples of dt) for an x-polarised plane wave along +z or -z
    whose field at the origin is g(t - delay).  The transfer function is the
    Mie series (exp(-i omega t) convention, conjugated for the exp(+i omega t)
    transform of the real signal), applied to the pulse's discrete Fourier
    transform on a grid of step dt, zero-padded to npad times the span, with
    frequencies above f_cut dropped.  Incidence along -z is the +z series
    rotated by 180 degrees about the x axis.  Returns [len(times)][N][3]."""
    times = np.asarray(times, dtype=np.float64)
    n_t = int(np.ceil(times.max() / dt)) + 1
    N = 1 << int(np.ceil(np.log2(npad * n_t)))
    t = np.arange(N) * dt
    G = np.fft.rfft(g(t - delay))
    f = np.fft.rfftfreq(N, dt)
    P = np.atleast_2d(np.asarray(points, dtype=np.float64))
    if along_minus_z:
        P = P * np.array([1.0, -1.0, -1.0])
    out = np.zeros((len(f), len(P), 3), complex)
    for kk in range(len(f)):
        if f[kk] > f_cut:
            break
        om = max(2 * np.pi * f[kk], 1e-4)  # the static limit is finite
        out[kk] = np.conj(PECSphere(a, om).surface_current(P)) * G[kk]
    J = np.fft.irfft(out, n=N, axis=0)
    idx = np.rint(times / dt).astype(int)
    J = J[idx]
    if along_minus_z:
        J = J * np.array([1.0, -1.0, -1.0])
    return J
