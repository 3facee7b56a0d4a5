"""Edge cases of the C ABI on the GPU: degenerate meshes, the smallest march,
empty histories, out-of-range arguments and unsupported combinations.  Every
error comes back as a status code; the context stays usable after EINVAL."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _code(fn):
    from paper_2303_05006_gb300 import TdbemError

    with pytest.raises(TdbemError) as e:
        fn()
    return e.value.code


def test_degenerate_triangle_is_rejected():
    from paper_2303_05006_gb300 import Solver
    from workloads.meshes import icosphere

    v, t = icosphere(1.0, 1)
    v = v.copy()
    v[t[0, 1]] = v[t[0, 0]]  # two corners of one triangle coincide
    assert _code(lambda: Solver(v, t, 0.1, 10)) == 2  # EMESH


@pytest.mark.parametrize("bad", [dict(solve_grid=3), dict(far_overlap=2), dict(n_rhs=65), dict(n_rhs=0),
                                 dict(m2l_tile_rows=64), dict(p_s=9), dict(precond=2)])
def test_invalid_parameters_are_rejected(bad):
    from paper_2303_05006_gb300 import Solver
    from workloads import workload

    w = workload("sphere80")
    assert _code(lambda: Solver(w.verts, w.tris, w.dt, w.Nt, mode=1, **bad)) == 1  # EINVAL


@pytest.mark.parametrize("mode", [0, 1])
def test_smallest_march_and_empty_history(mode):
    """Nt = 2 is a single step; an empty history gives R = V; a zero-step march
    returns nothing and leaves the state alone; out-of-range steps are EINVAL
    and the context keeps working."""
    from paper_2303_05006_gb300 import Solver
    from workloads import workload

    w = workload("sphere80")
    s = Solver(w.verts, w.tris, w.dt, 2, mode=mode)
    s.set_incident_plane(w.pulses[0])
    R1 = s.history_eval(1, np.zeros((0, s.ne)))
    assert np.isfinite(R1).all()
    assert s.march(0).shape == (0, s.ne)
    J = s.march(1)
    assert J.shape == (1, s.ne) and np.isfinite(J).all()
    assert _code(lambda: s.history_eval(0, np.zeros((0, s.ne)))) == 1
    assert _code(lambda: s.history_eval(2, np.zeros((0, s.ne)))) == 1
    assert _code(lambda: s.step()) == 7  # ESTATE: all Nt - 1 steps taken
    s.reset()
    J2 = s.march(1)
    assert np.array_equal(J, J2) or np.linalg.norm(J2 - J) <= 1e-12 * np.linalg.norm(J)


def test_noalloc_entry_point_rejects_fast_mode():
    from paper_2303_05006_gb300 import Solver
    from workloads import workload

    w = workload("sphere80")
    s = Solver(w.verts, w.tris, w.dt, w.Nt, mode=1)
    s.set_incident_plane(w.pulses[0])
    assert _code(lambda: s.history_eval_noalloc(5, np.zeros((4, s.ne)))) == 1
    # still usable afterwards
    assert np.isfinite(s.march(3)).all()


def test_single_rhs_options_agree_on_a_tiny_mesh():
    """Every schedule of the single-RHS march (pipelined or serial; cluster or
    grid-wide solve) gives the same currents on a mesh smaller than one block
    of the solver per SM."""
    from paper_2303_05006_gb300 import Solver
    from workloads import workload

    w = workload("sphere80")
    ref = None
    for kw in (dict(far_overlap=0, solve_grid=1), dict(far_overlap=1, solve_grid=1),
               dict(far_overlap=1, solve_grid=2), dict(far_overlap=0, solve_grid=2)):
        s = Solver(w.verts, w.tris, w.dt, w.Nt, mode=1, **kw)
        s.set_incident_plane(w.pulses[0])
        J = s.march(w.Nt - 1)
        s.close()
        if ref is None:
            ref = J
        assert np.linalg.norm(J - ref) <= 1e-6 * np.linalg.norm(ref), kw
