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
