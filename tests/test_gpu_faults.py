"""Failure detection of the C ABI, triggered from the host (no GPU fault,
trap or hang is involved):

* TDBEM_ENOCONV: a Z0 solve capped at one iteration misses the tolerance;
  the step still returns its best iterate (finite, closer to the converged
  current than the zero start), advances, and the context stays usable.
* Non-finite network weights: the learned warm start's guess is NaN; every
  solve falls back to the extrapolated guess (a NaN never wins the residual
  comparison) and the currents are those of the plain march.
* TDBEM_ENOMEM: a device-memory budget below the context's needs fails
  tdbem_create cleanly, and a context created afterwards works.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _solver(w, **kw):
    from paper_2303_05006_gb300 import Solver

    s = Solver(w.verts, w.tris, w.dt, w.Nt, **kw)
    s.set_incident_plane(w.pulses[0])
    return s


@pytest.mark.parametrize("mode", [0, 1])
def test_enoconv_returns_the_best_iterate(mode):
    from paper_2303_05006_gb300 import lib
    from workloads import workload

    w = workload("sphere80")
    ref = _solver(w, mode=mode).march(12)
    s = _solver(w, mode=mode, solve_maxit=1, solve_tol=1e-14, warm_start=0, jacobi_sweeps=0)
    L = lib()
    J = np.zeros(s.ne)
    it = ctypes.c_int32()
    for k in range(12):
        rc = L.tdbem_step(s._h, J.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(it))
        if k == 11:
            break
        if rc == 0:
            continue
        assert rc == 5, rc  # TDBEM_ENOCONV
        assert b"tolerance" in L.tdbem_last_error(s._h)
        assert np.isfinite(J).all()
        if np.linalg.norm(ref[k]) > 0:
            assert np.linalg.norm(J - ref[k]) < np.linalg.norm(ref[k])
    assert s.alpha == 13  # every step advanced
    # the context is still usable: a reset and a march run (and miss again)
    s.reset()
    with pytest.raises(Exception) as ex:
        s.march(3)
    assert getattr(ex.value, "code", None) == 5


def test_nonfinite_network_falls_back_to_the_extrapolation():
    from workloads import workload

    w = workload("sphere320")
    n = 60
    plain = _solver(w).march(n)
    s = _solver(w)
    th = np.full(s.MLP_NPARAM, np.nan, np.float32)
    s.mlp_set_weights(th)
    s.mlp_use(True)
    J = s.march(n)
    used, fallback = s.mlp_stats()
    assert used == 0 and fallback == n
    assert np.isfinite(J).all()
    assert np.linalg.norm(J - plain) <= 1e-12 * np.linalg.norm(plain)


def test_device_memory_budget_gives_enomem():
    from paper_2303_05006_gb300 import Solver, TdbemError
    from workloads import workload

    w = workload("sphere320")
    with pytest.raises(TdbemError) as ex:
        Solver(w.verts, w.tris, w.dt, w.Nt, max_device_bytes=1 << 20)
    assert ex.value.code == 4  # TDBEM_ENOMEM
    s = Solver(w.verts, w.tris, w.dt, w.Nt)
    need = s.info().device_bytes_peak  # setup holds the FP64 store and its row tiles at once
    assert need >= s.info().device_bytes
    s.close()
    # a budget just above the need is enough
    t = Solver(w.verts, w.tris, w.dt, w.Nt, max_device_bytes=need + (1 << 20))
    t.set_incident_plane(w.pulses[0])
    assert np.isfinite(t.march(5)).all()
    t.close()
