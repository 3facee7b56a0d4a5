"""The paper's test problem on the GPU (section 4.1, case 3 of Table 1): a PEC
sphere of radius 0.5 meshed with 5120 triangles, dt = 0.005, the Sin^2 pulse
along -x3 (Lambda = A = 0.5), theta = zeta = 1, N_leaf = 100.

The error measure is the paper's eq. (error): squared differences of the
current at the triangle centres over all steps, divided by the squared TDBEM
current.  The reference is the Mie series of the sphere applied to the
pulse's spectrum (tests/_mie.py, pinned against the oracle in the time domain
in tests/test_oracle_mie.py), evaluated at a seeded sample of 1024 centres
and cut at 8 in frequency (the cut changes the measure by 2e-4).  The paper's
own values (tests/golden/paper_case3_errors.txt) come from an inverse-Laplace
reference; the measured values here are printed with -s.

Bars: the direct FP64 march (the paper's CONV) and the fast march at p = 4
no worse than the paper's CONV and FAST4; the fast march at p_s = 6, p_t = 4
no worse than the paper's FAST6.  At p_s = p_t = 6 the fast march grows late
in time in this regime with theta = zeta = 1 (dt = h/7.6, 18 steps per leaf
interval): it is measured and printed, not held to the paper's FAST6; with
theta = zeta = 3 it is stable and held to it.  With the paper's own
interpolant, CHI in space and time (section 3.2), the march at p = 6 and
theta = zeta = 1 is stable and both CHI marches are held to the paper's FAST4
and FAST6 (measured on a GB300: 1.93e-2 and 5.06e-3, against Lagrange's
2.32e-2 and 1.33e-1).
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
NT = 1000  # 5 time units: the current has decayed to 0.4% of its peak
DT = 0.005


def _paper():
    out = {}
    for ln in open(os.path.join(HERE, "golden", "paper_case3_errors.txt")):
        if ln.strip() and not ln.startswith("#"):
            k, v = ln.split()
            out[k] = float(v)
    return out


def test_paper_case3_errors():
    from _mie import transient_current
    from paper_2303_05006_gb300 import Solver
    from workloads.configs import sin2_pulse
    from workloads.meshes import icosphere

    v, t = icosphere(0.5, 4)
    pulse = sin2_pulse(v)
    rng = np.random.default_rng(31)
    sample = np.sort(rng.choice(len(t), 1024, replace=False))

    def centre_currents(s, J):
        """J(S_i, t_alpha) at the sampled centres, alpha = 1 .. NT-1: the time
        basis puts N(1) = N(2) = 1/2 on J^{alpha-1} and J^{alpha-2} (eq. J)."""
        import scipy.sparse as sp

        ev, et = s.edges()
        cen = v[t].mean(1)
        area = 0.5 * np.linalg.norm(np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]]), axis=1)
        ell = np.linalg.norm(v[ev[:, 0]] - v[ev[:, 1]], axis=1)
        Jh = np.concatenate([0.5 * J[:1], 0.5 * (J[1:] + J[:-1])])
        out = np.zeros((len(Jh), len(sample), 3))
        for s_, sg in ((0, 1.0), (1, -1.0)):
            tri = et[:, s_]
            tv = t[tri]
            opp = np.where((tv != ev[:, :1]) & (tv != ev[:, 1:]), tv, -1).max(1)
            fj = sg * (ell / (2 * area[tri]))[:, None] * (cen[tri] - v[opp])  # RWG at the centre
            for k in range(3):
                B = sp.csr_matrix((fj[:, k], (tri, np.arange(len(ev)))), shape=(len(t), len(ev)))[sample]
                out[:, :, k] += (B @ Jh.T).T
        return out

    def march(**kw):
        s = Solver(v, t, DT, NT, **kw)
        s.set_incident_plane(pulse)
        J = s.march(NT - 1)
        Jc = centre_currents(s, J)
        s.close()
        return Jc

    runs = {"CONV": march(mode=0), "FAST4": march(mode=1, p_s=4, p_t=4, n_leaf=100, m2l_prec=4),
            "FAST6x4": march(mode=1, p_s=6, p_t=4, n_leaf=100, m2l_prec=4),
            "FAST6": march(mode=1, p_s=6, p_t=6, n_leaf=100, m2l_prec=4),
            "FAST6_theta3": march(mode=1, p_s=6, p_t=6, n_leaf=100, m2l_prec=4, theta=3.0, zeta=3.0),
            # the paper's own interpolant, CHI in space and time (section 3.2)
            "FAST4_chi": march(mode=1, p_s=4, p_t=4, n_leaf=100, m2l_prec=4, s_interp=1, t_interp=1),
            "FAST6_chi": march(mode=1, p_s=6, p_t=6, n_leaf=100, m2l_prec=4, s_interp=1, t_interp=1)}
    zmax = float(v[:, 2].max())
    Lam, A = 0.5, 0.5

    def g(u):
        return np.where((u >= 0) & (u <= Lam), A * np.sin(2 * np.pi * u / Lam) ** 2, 0.0)

    cen = v[t].mean(1)[sample]
    Jref = -transient_current(0.5, cen, np.arange(1, NT) * DT, g, zmax, True, DT, 8.0)
    paper = _paper()
    err = {k: float(np.sum((J - Jref) ** 2) / np.sum(J ** 2)) for k, J in runs.items()}
    print("\ncase 3, eq. (error):", {k: f"{e:.3e}" for k, e in err.items()}, "paper:", paper)
    assert err["CONV"] <= paper["CONV"], err
    assert err["FAST4"] <= paper["FAST4"], err
    assert err["FAST6x4"] <= paper["FAST6"], err
    assert np.isfinite(err["FAST6"]), err
    # the same discretisation of the same physics with a heavier MFIE share
    # (theta = zeta = 3): stable at p = 6, and the Mie reference still applies
    assert err["FAST6_theta3"] <= paper["FAST6"], err
    # the paper's interpolant at the paper's coupling
    assert err["FAST4_chi"] <= paper["FAST4"], err
    assert err["FAST6_chi"] <= paper["FAST6"], err
