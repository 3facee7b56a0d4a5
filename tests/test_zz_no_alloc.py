"""The allocation-free history evaluation gives the same R as the allocating
one.  Callers that cannot allocate device memory at call time (inside another
library's stream capture, with a frozen allocator, or when the host owns the
whole pool) use tdbem_history_eval_noalloc, which stages the history in the
library's fixed static device array.  Collected last so that a failure here
never hides the other tests; it passes alone and after them."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_history_eval_matches_allocating_entry_point():
    from paper_2303_05006_gb300 import Solver
    from workloads import random_history, workload

    w = workload("sphere320")
    s = Solver(w.verts, w.tris, w.dt, w.Nt)
    s.set_incident_plane(w.pulses[0])
    # two calls in a row, different steps and histories: the shared scratch
    # keeps the previous call's contents, which must not leak into the next
    for alpha, seed in ((90, 1), (23, 2)):
        J = random_history(s.ne, alpha - 1, seed=seed)
        R_ref = s.history_eval(alpha, J)
        R_na = s.history_eval_noalloc(alpha, J)
        scale = np.abs(R_ref).max()
        assert np.abs(R_na - R_ref).max() <= 1e-11 * scale


def test_noalloc_with_several_right_hand_sides():
    """The batched layout ([ne][R] on the device, [R][ne] on the host) through
    the fixed scratch: three right-hand sides, two calls in a row."""
    from paper_2303_05006_gb300 import Solver
    from workloads import random_history, workload

    w = workload("sphere320")
    R = 3
    s = Solver(w.verts, w.tris, w.dt, w.Nt, n_rhs=R)
    for r in range(R):
        s.set_incident_plane(w.pulses[0], rhs=r)
    for alpha, seed in ((70, 3), (41, 4)):
        J = random_history(R * s.ne, alpha - 1, seed=seed).reshape(alpha - 1, R, s.ne)
        R_ref = s.history_eval(alpha, J)
        R_na = s.history_eval_noalloc(alpha, J)
        assert R_na.shape == (R, s.ne)
        assert np.abs(R_na - R_ref).max() <= 1e-11 * np.abs(R_ref).max()


def test_noalloc_rejects_problems_beyond_the_scratch():
    """ne * n_rhs * (ring length + history steps used) above the fixed
    capacity is refused with TDBEM_EINVAL, before any device work."""
    from paper_2303_05006_gb300 import Solver, TdbemError
    from workloads import workload

    w = workload("sphere1280")
    s = Solver(w.verts, w.tris, w.dt, w.Nt, n_rhs=48)
    alpha = 40  # ne * n_rhs * L alone (1920 * 48 * 32) is above the 2^21 doubles
    J = np.zeros((alpha - 1, 48, s.ne))
    with pytest.raises(TdbemError) as ex:
        s.history_eval_noalloc(alpha, J)
    assert ex.value.code == 1
    # the context is still usable afterwards
    assert np.isfinite(s.history_eval(alpha, J)).all()
