"""The paper's test problem on the GPU, cases 1 and 2 of Table 1 (section 4.1):
the PEC sphere of radius 0.5 meshed as the equal-arc icosahedral geodesics of
frequency 8 and 12 (Ns = 1280 and 2880; the meshes reproduce the table's edge
lengths, tests/test_golden_table1.py), dt = 0.005, the Sin^2 pulse along -x3
(Lambda = A = 0.5), theta = zeta = 1, N_leaf = 100.

The error is the paper's eq. (error) against the Mie series of the sphere
applied to the pulse's spectrum at a seeded sample of centres, as for case 3
(tests/test_gpu_paper_case3.py).  The paper prints errors for case 3 only; for
cases 1 and 2 its accuracy figure shows the conventional method converging
with Ns.  Checked here: the conventional march (CONV) is more accurate on
case 2 than on case 1, both stay below the paper's case-3 CONV value, and the
fast march at p = 4 is finite.  The march times of both paths are printed
(the paper finds FAST faster than CONV for cases 1 to 3).
"""
import os
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
NT = 1000
DT = 0.005


def _paper_conv3():
    for ln in open(os.path.join(HERE, "golden", "paper_case3_errors.txt")):
        if ln.startswith("CONV"):
            return float(ln.split()[1])


def _case_errors(freq, sample_n=768, seed=37):
    from _mie import transient_current
    from paper_2303_05006_gb300 import Solver
    from workloads.configs import sin2_pulse
    from workloads.meshes import geodesic_sphere

    v, t = geodesic_sphere(0.5, freq)
    pulse = sin2_pulse(v)
    sample = np.sort(np.random.default_rng(seed).choice(len(t), min(sample_n, len(t)), replace=False))
    cen_all = v[t].mean(1)
    area = 0.5 * np.linalg.norm(np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]]), axis=1)

    def centre_currents(s, J):
        # J(S_i, t_alpha): N(1) = N(2) = 1/2 on J^{alpha-1} and J^{alpha-2} (eq. J)
        import scipy.sparse as sp

        ev, et = s.edges()
        ell = np.linalg.norm(v[ev[:, 0]] - v[ev[:, 1]], axis=1)
        Jh = np.concatenate([0.5 * J[:1], 0.5 * (J[1:] + J[:-1])])
        out = np.zeros((len(Jh), len(sample), 3))
        for s_, sg in ((0, 1.0), (1, -1.0)):
            tri = et[:, s_]
            tv = t[tri]
            opp = np.where((tv != ev[:, :1]) & (tv != ev[:, 1:]), tv, -1).max(1)
            fj = sg * (ell / (2 * area[tri]))[:, None] * (cen_all[tri] - v[opp])
            for k in range(3):
                B = sp.csr_matrix((fj[:, k], (tri, np.arange(len(ev)))), shape=(len(t), len(ev)))[sample]
                out[:, :, k] += (B @ Jh.T).T
        return out

    runs, secs = {}, {}
    for name, kw in (("CONV", dict(mode=0)), ("FAST4", dict(mode=1, p_s=4, p_t=4, n_leaf=100, m2l_prec=4))):
        s = Solver(v, t, DT, NT, **kw)
        s.set_incident_plane(pulse)
        t0 = time.perf_counter()
        J = s.march(NT - 1)
        secs[name] = time.perf_counter() - t0
        runs[name] = centre_currents(s, J)
        s.close()
    zmax = float(v[:, 2].max())

    def g(u):
        return np.where((u >= 0) & (u <= 0.5), 0.5 * np.sin(2 * np.pi * u / 0.5) ** 2, 0.0)

    Jref = -transient_current(0.5, cen_all[sample], np.arange(1, NT) * DT, g, zmax, True, DT, 8.0)
    err = {k: float(np.sum((J - Jref) ** 2) / np.sum(J ** 2)) for k, J in runs.items()}
    return err, secs


def test_paper_cases_1_and_2():
    e1, t1 = _case_errors(8)
    e2, t2 = _case_errors(12)
    print("\ncase 1, eq. (error):", {k: f"{v:.3e}" for k, v in e1.items()}, "march s:", t1)
    print("case 2, eq. (error):", {k: f"{v:.3e}" for k, v in e2.items()}, "march s:", t2)
    conv3 = _paper_conv3()
    assert e2["CONV"] < e1["CONV"], (e1, e2)
    assert e1["CONV"] <= conv3 and e2["CONV"] <= conv3, (e1, e2, conv3)
    assert np.isfinite(e1["FAST4"]) and np.isfinite(e2["FAST4"])
