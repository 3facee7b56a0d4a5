"""Physics pin of the oracle: the marched surface current of a perfectly
conducting sphere against the Mie series (CPU only).

The oracle marches the 320-triangle unit sphere under a low-frequency
modulated Gaussian plane wave (x-polarised, along +z).  The Fourier transform
of the marched current, J(x, omega) = sum_beta J^beta f(x) * dt e^{-i omega
beta dt} Nhat(omega dt) with Nhat the transform of the cardinal quadratic
B-spline (the time basis of section 2.2), divided by the incident field's
transform at the origin, is compared at every triangle centroid with the
Mie-series current of the same sphere.  The paper's unknown is J := n x H with
n pointing into the conductor (section 2.1), i.e. minus the physical current
n_out x H, and its time-harmonic fields use exp(+i omega t), so the expected
value is -conj(J_mie) for the exp(-i omega t) series.

What the pin catches: the error is the discretisation error of a 320-triangle
RWG mesh (a few percent, growing with ka); a dropped or mis-signed MFIE
identity term (the reading of eq. cfie), a wrong sign or factor of any of the
three potential terms, a wrong incident right-hand side or a wrong time basis
gives an error of order one (the dropped identity term is planted below), and
the opposite overall sign gives about 2.
"""
import numpy as np
import pytest

from _mie import PECSphere

F0, SIGMA = 0.25, 1.2          # low-frequency pulse: ka = 1.57 at f0, 13 edges per wavelength
NT = 220                        # 33 time units: the current has decayed to 5e-6 of its peak
FREQS = (0.15, 0.25, 0.35)      # ka = 0.94, 1.57, 2.20 (below the first interior resonance, 2.74)
# measured errors 0.035, 0.065, 0.092; bars 1.5x
BARS = (0.053, 0.098, 0.14)


def _pulse(w):
    from workloads.configs import Pulse

    return Pulse((0.0, 0.0, 1.0), (1.0, 0.0, 0.0), F0, SIGMA, 6 * SIGMA, float(w.verts[:, 2].min()))


def _centroid_spectra(o, w, J, freqs):
    """J(x_c, omega) / E_inc(origin, omega) at every triangle centroid."""
    ev, et, eo = o.edges()
    V, T = w.verts, w.tris
    cen = V[T].mean(1)
    area = 0.5 * np.linalg.norm(np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]]), axis=1)
    ell = np.linalg.norm(V[ev[:, 0]] - V[ev[:, 1]], axis=1)
    beta = np.arange(J.shape[0])
    dt, zmin = w.dt, float(w.verts[:, 2].min())
    out = []
    for f in freqs:
        om = 2 * np.pi * f
        Om = om * dt
        nhat = ((1 - np.exp(-1j * Om)) / (1j * Om)) ** 3
        Jw = dt * nhat * (np.exp(-1j * om * beta * dt) @ J)
        w0 = 2 * np.pi * F0
        # transform of g(u) = cos(w0 (u - t0)) exp(-(u - t0)^2 / (2 sigma^2)), delayed to the origin
        G = np.exp(-1j * om * 6 * SIGMA) * SIGMA * np.sqrt(2 * np.pi) / 2 * (
            np.exp(-SIGMA ** 2 * (om - w0) ** 2 / 2) + np.exp(-SIGMA ** 2 * (om + w0) ** 2 / 2))
        E0 = G * np.exp(-1j * om * (-zmin))
        Jc = np.zeros((len(T), 3), complex)
        for s, sg in ((0, 1.0), (1, -1.0)):  # RWG: +-l/(2A) (x - o) on T+ / T-
            t_ = et[:, s]
            fj = sg * (ell / (2 * area[t_]))[:, None] * (cen[t_] - V[eo[:, s]])
            np.add.at(Jc, t_, Jw[:, None] * fj)
        out.append((om, cen, Jc / E0))
    return out


def _errors(o, w):
    J = o.march(_pulse(w), NT)
    errs, flips = [], []
    for om, cen, Jc in _centroid_spectra(o, w, J, FREQS):
        ref = -np.conj(PECSphere(1.0, om).surface_current(cen))
        errs.append(np.linalg.norm(Jc - ref) / np.linalg.norm(ref))
        flips.append(np.linalg.norm(Jc + ref) / np.linalg.norm(ref))
    return J, errs, flips


def test_mie_reference_satisfies_its_own_definition():
    for k in (0.5, 1.5, 3.0):
        chk = PECSphere(1.0, k).check_expansion()
        assert chk["incident_E"] < 1e-12 and chk["incident_H"] < 1e-12, chk
        assert chk["boundary_E"] < 1e-12, chk
        assert chk["curl_H"] < 1e-7, chk


def test_marched_current_matches_mie_series(sphere320_oracle):
    w, o = sphere320_oracle
    J, errs, flips = _errors(o, w)
    late = np.abs(J[-10:]).max() / np.abs(J).max()
    assert late < 1e-4, late  # the transform sees the whole transient
    for f, e, bar, fl in zip(FREQS, errs, BARS, flips):
        assert e < bar, (f, e)
        assert fl > 1.9, (f, fl)
    # discretisation error: grows with the electrical size
    assert errs[0] < errs[1] < errs[2], errs


def test_cfie2_also_matches_mie_series(sphere320_oracle):
    """The paper's CFIE2 (time-differentiated EFIE and MFIE, no MFIE term:
    zeta = 0, section 4.3) is another discretisation of the same physics: the
    same bars hold.  (CFIE3, chi = 0, is left out here: its discrete current
    decays too slowly for a transform over a bounded march, still 1.8% of its
    peak after 800 steps.)"""
    from oracle.oracle import Oracle

    w, _ = sphere320_oracle
    o = Oracle(w.verts, w.tris, w.dt, zeta=0.0)
    o.assemble()
    J, errs, flips = _errors(o, w)
    assert np.abs(J[-10:]).max() / np.abs(J).max() < 1e-4
    for f, e, bar, fl in zip(FREQS, errs, BARS, flips):
        assert e < bar, (f, e)
        assert fl > 1.9, (f, fl)


def test_mie_pin_catches_a_dropped_mfie_identity_term(sphere320_oracle):
    """Plant a mistake in the oracle (no MFIE identity term, s_J = 0): the
    same comparison must fail by a wide margin."""
    from oracle.oracle import Oracle

    w, _ = sphere320_oracle
    o = Oracle(w.verts, w.tris, w.dt, sJ=0.0)
    o.assemble()
    _, errs, _ = _errors(o, w)
    assert min(errs) > 1.0, errs


def _centroid_transient(o, w, J):
    """J(S_i, t_alpha) at every centroid for alpha = 2 .. : the time basis puts
    N(1) = N(2) = 1/2 on J^{alpha-1} and J^{alpha-2} (eq. J)."""
    ev, et, eo = o.edges()
    V, T = w.verts, w.tris
    cen = V[T].mean(1)
    area = 0.5 * np.linalg.norm(np.cross(V[T[:, 1]] - V[T[:, 0]], V[T[:, 2]] - V[T[:, 0]]), axis=1)
    ell = np.linalg.norm(V[ev[:, 0]] - V[ev[:, 1]], axis=1)
    Jh = 0.5 * (J[1:] + J[:-1])  # row alpha - 2 holds J(., t_alpha)
    out = np.zeros((len(Jh), len(T), 3))
    for s, sg in ((0, 1.0), (1, -1.0)):
        t_ = et[:, s]
        fj = sg * (ell / (2 * area[t_]))[:, None] * (cen[t_] - V[eo[:, s]])
        for b in range(len(Jh)):
            np.add.at(out[b], t_, Jh[b][:, None] * fj)
    return cen, out


def test_transient_current_matches_mie_series_in_time(sphere320_oracle):
    """The same pin in the time domain, with the paper's error measure (eq.
    error: squared differences at triangle centres over all steps, over the
    squared TDBEM current) and incidence along -z as in section 4.1: the
    reference is the Mie transfer function applied to the pulse's discrete
    transform (tests/_mie.py).  Measured 4.7e-3 (6.9% in norm); the opposite
    sign gives about 4."""
    from _mie import transient_current
    from workloads.configs import Pulse

    w, o = sphere320_oracle
    zmin = float(np.min(w.verts @ np.array([0.0, 0.0, -1.0])))
    pu = Pulse((0.0, 0.0, -1.0), (1.0, 0.0, 0.0), F0, SIGMA, 6 * SIGMA, zmin)
    J = o.march(pu, NT)
    cen, Jt = _centroid_transient(o, w, J)
    times = np.arange(2, NT) * w.dt

    def g(u):
        return np.cos(2 * np.pi * F0 * (u - 6 * SIGMA)) * np.exp(-(u - 6 * SIGMA) ** 2 / (2 * SIGMA ** 2))

    Jr = -transient_current(1.0, cen, times, g, -zmin, True, w.dt, 1.5)
    den = np.sum(Jt ** 2)
    err = np.sum((Jt - Jr) ** 2) / den
    assert err < 7.1e-3, err
    assert np.sum((Jt + Jr) ** 2) / den > 3.5
