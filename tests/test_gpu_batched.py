"""Batched form: R right-hand sides (incident plane waves) on one scatterer
marched together through shared operators.

Every operator is linear in the current history and the R marches are
independent, so a batched march must reproduce R separate single-RHS marches:
in direct mode to the rounding level of the FP64 path (the Z0 solves of both
stop at a 1e-13 relative residual), in fast mode to the level at which FP32
atomics in a different order differ.  The batched direct march is also pinned
to the FP64 oracle on every right-hand side.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _pulses(w, n, seed):
    from workloads.configs import pulse_star, random_plane_waves

    return [pulse_star(w.verts, k=k, pol=pol) for k, pol in random_plane_waves(n, seed)]


def _batched(w, pulses, **kw):
    from paper_2303_05006_gb300 import Solver

    s = Solver(w.verts, w.tris, w.dt, w.Nt, n_rhs=len(pulses), **kw)
    for r, pu in enumerate(pulses):
        s.set_incident_plane(pu, rhs=r)
    return s


def _single(w, pulse, **kw):
    from paper_2303_05006_gb300 import Solver

    s = Solver(w.verts, w.tris, w.dt, w.Nt, **kw)
    s.set_incident_plane(pulse)
    return s


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_batched_direct_matches_oracle(sphere320_oracle):
    """480-RWG sphere, 127 steps, 3 plane waves: every column of the batched
    FP64 march against the oracle's march of that wave (bar 1e-10)."""
    w, o = sphere320_oracle
    pulses = _pulses(w, 3, seed=41)
    J = _batched(w, pulses).march(w.Nt - 1)
    assert J.shape == (w.Nt - 1, 3, o.ne)
    for r, pu in enumerate(pulses):
        Jo = o.march(pu, w.Nt)
        assert _rel(J[:, r], Jo) < 1e-10, r


@pytest.mark.parametrize("R", [2, 5, 33])
def test_batched_direct_matches_single(R):
    """Ragged batch sizes (lanes per RHS group 2, 8, 32 with a second pass;
    solver clusters with unequal RHS slices) on the 120-RWG sphere."""
    from workloads import workload

    w = workload("sphere80")
    pulses = _pulses(w, R, seed=R)
    Jb = _batched(w, pulses).march(w.Nt - 1)
    for r in sorted({0, R // 2, R - 1}):
        Js = _single(w, pulses[r]).march(w.Nt - 1)
        assert _rel(Jb[:, r], Js) < 1e-11, r


def test_batched_fast_matches_single():
    """Fast mode (p = 4, TF32x3 M2L), 1920-RWG sphere, 299 steps, 4 waves.
    The far field is summed with FP32 atomics whose order differs between a
    batched and a single launch, and the march carries that rounding along
    (measured 2.0e-5 with FP32 near-field row sums; TF32x3 itself is within
    1e-4 of the FP32 M2L).  An indexing mistake in any batched kernel gives
    an O(1) error."""
    from workloads import workload

    w = workload("sphere1280")
    pulses = _pulses(w, 4, seed=7)
    Jb = _batched(w, pulses, mode=1, m2l_prec=4).march(w.Nt - 1)
    for r in (0, 3):
        Js = _single(w, pulses[r], mode=1, m2l_prec=4).march(w.Nt - 1)
        assert _rel(Jb[:, r], Js) < 1e-4, r


@pytest.mark.parametrize("mode", [0, 1])
def test_batched_history_eval(mode):
    """history_eval of a batch on per-RHS random histories equals the
    single-RHS evaluations (fast mode replays the far field of the batch)."""
    from workloads import random_history, workload

    w = workload("sphere320" if mode == 0 else "sphere1280")
    pulses = _pulses(w, 3, seed=5)
    sb = _batched(w, pulses, mode=mode)
    a = 60
    H = np.stack([random_history(sb.ne, a - 1, seed=100 + r) for r in range(3)], axis=1)  # (a-1, R, ne)
    Rb = sb.history_eval(a, H)
    assert Rb.shape == (3, sb.ne)
    for r in range(3):
        Rs = _single(w, pulses[r], mode=mode).history_eval(a, H[:, r])
        tol = 1e-12 if mode == 0 else 1e-4
        assert np.linalg.norm(Rb[r] - Rs) <= tol * np.linalg.norm(Rs), r


def test_batched_step_v_and_set_rhs():
    """Caller-supplied right-hand sides: step_v with (R, ne) arrays and
    set_rhs per column give the plane-wave march."""
    from paper_2303_05006_gb300 import Solver
    from workloads import workload

    w = workload("sphere80")
    pulses = _pulses(w, 2, seed=3)
    ref = _batched(w, pulses)
    # V^{alpha-1} of each wave: the history evaluation of an empty history
    singles = [_single(w, pu) for pu in pulses]
    V = np.array([[s1.history_eval(a + 1, np.zeros((0, s1.ne))) for s1 in singles] for a in range(w.Nt - 1)])
    Jref = ref.march(20)
    s = Solver(w.verts, w.tris, w.dt, w.Nt, n_rhs=2)
    J = np.zeros((2, s.ne))
    out = []
    for a in range(20):
        s.step_v(V[a], J)
        out.append(J.copy())
    assert _rel(np.array(out), Jref) < 1e-12
    s2 = Solver(w.verts, w.tris, w.dt, w.Nt, n_rhs=2)
    for r in range(2):
        s2.set_rhs(V[:, r], rhs=r)
    assert _rel(s2.march(20), Jref) < 1e-12


def test_batched_argument_errors():
    from paper_2303_05006_gb300 import Solver, TdbemError
    from workloads import workload

    w = workload("sphere80")
    for bad in (0, 65):
        with pytest.raises(TdbemError):
            Solver(w.verts, w.tris, w.dt, w.Nt, n_rhs=bad)
    s = Solver(w.verts, w.tris, w.dt, w.Nt, n_rhs=2)
    with pytest.raises(TdbemError):
        s.set_incident_plane(w.pulses[0], rhs=2)


def test_march_many_matches_separate_marches():
    """Several scatterers marched together (steps issued in rounds, one stream
    per context) give the currents of their separate marches: two direct
    FP64 contexts exactly to rounding, one fast context to the order of its
    FP32 atomics."""
    import torch

    from paper_2303_05006_gb300 import Solver, march_many
    from workloads import workload

    specs = [("sphere80", dict(mode=0), 1e-12), ("sphere320", dict(mode=0), 1e-12),
             ("sphere1280", dict(mode=1, m2l_prec=4), 1e-4)]
    ws = [workload(n) for n, _, _ in specs]
    steps = [min(w.Nt - 1, 120) for w in ws]
    ref = []
    for w, (_, kw, _), n in zip(ws, specs, steps):
        s = Solver(w.verts, w.tris, w.dt, w.Nt, **kw)
        s.set_incident_plane(w.pulses[0])
        ref.append(s.march(n))
        s.close()
    solvers = []
    for w, (_, kw, _) in zip(ws, specs):
        s = Solver(w.verts, w.tris, w.dt, w.Nt, **kw)
        s.set_incident_plane(w.pulses[0])
        solvers.append(s)
    outs = [torch.zeros((n, s.ne), dtype=torch.float64, device="cuda") for n, s in zip(steps, solvers)]
    march_many(solvers, steps, [o.data_ptr() for o in outs])
    torch.cuda.synchronize()
    for o, r, (name, _, tol) in zip(outs, ref, specs):
        assert _rel(o.cpu().numpy(), r) < tol, name
    with pytest.raises(Exception):
        march_many([solvers[0], solvers[0]], [1, 1])
