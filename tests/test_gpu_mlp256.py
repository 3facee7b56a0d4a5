"""The learned warm start at width 256, whose dense layers and weight
gradients run on the tcgen05 tensor cores (BF16 operands, FP32 accumulation;
FP32 parameters and Adam).

* Forward outputs, loss and every gradient block against the FP64 reference
  network (oracle/mlp.py, pinned by finite differences on the CPU), on a
  ragged batch of 1000 samples.  BF16 keeps 8 significand bits, so the
  operands carry a relative rounding of 2^-9.  Measured on a GB300: forward
  4.4e-3 of the largest output, loss 3e-4, gradient blocks 3.1e-3 to
  3.6e-3 (relative l2).  The bars (1.5e-2) sit a few times above that and
  far below what a wrong transpose, stride or tile index gives (order 1).
* Training lowers the loss, and on a held-out wave the network's guess is
  kept by the residual fallback in most solves while the currents stay those
  of the plain solve.
"""
import numpy as np
import pytest

from oracle import mlp as ref

pytestmark = pytest.mark.gpu

F, H = 25, 256


def _theta(rng, scale=1.0, zero_out=False):
    W1 = rng.standard_normal((H, F)) * scale / np.sqrt(F)
    W2 = rng.standard_normal((H, H)) * scale / np.sqrt(H)
    w3 = np.zeros(H) if zero_out else rng.standard_normal(H) * scale / np.sqrt(H)
    return np.concatenate([W1.ravel(), W2.ravel(), w3]).astype(np.float32)


def _solver(w, **kw):
    from paper_2303_05006_gb300 import Solver

    s = Solver(w.verts, w.tris, w.dt, w.Nt, **kw)
    s.mlp_set_width(H)
    return s


def _pulses(w, n, seed):
    from workloads.configs import pulse_star, random_plane_waves

    return [pulse_star(w.verts, k=k, pol=pol) for k, pol in random_plane_waves(n, seed)]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_width256_forward_and_gradient_match_reference():
    from workloads import workload

    w = workload("sphere80")
    s = _solver(w)
    assert s.MLP_NPARAM == H * F + H * H + H
    rng = np.random.default_rng(11)
    th = _theta(rng)
    s.mlp_set_weights(th)
    assert np.array_equal(s.mlp_get_weights(), th)
    n = 1000
    X = rng.standard_normal((n, F)).astype(np.float32)
    T = rng.standard_normal(n).astype(np.float32)
    th64 = th.astype(np.float64)
    y_ref = ref.forward(th64, X.astype(np.float64), F, H)
    y = s.mlp_forward(X)
    ey = float(np.abs(y - y_ref).max() / np.abs(y_ref).max())
    Wt = rng.uniform(0.1, 3.0, n).astype(np.float32)
    errs = []
    for W in (None, Wt):
        loss, g = s.mlp_grad(X, T, W)
        loss_ref, g_ref = ref.loss_and_grad(th64, X.astype(np.float64), T.astype(np.float64), F, H,
                                            None if W is None else W.astype(np.float64))
        el = abs(loss - loss_ref) / loss_ref
        eb = [_rel(g[a:b], g_ref[a:b]) for a, b in ((0, H * F), (H * F, H * F + H * H),
                                                     (H * F + H * H, H * F + H * H + H))]
        errs.append((el, eb))
    print(f"\nwidth 256 vs FP64 reference: forward {ey:.2e}; loss, gradient blocks (W1, W2, w3):", errs)
    assert ey <= 1.5e-2, ey
    for el, eb in errs:
        assert el <= 1.5e-2, errs
        assert max(eb) <= 1.5e-2, errs


def test_width256_training_and_fallback():
    """1920-RWG sphere, direct FP64 path: record 3 seeded waves, train at width
    256 on the GPU, then march a held-out wave with and without the network."""
    from workloads import workload

    w = workload("sphere1280")
    train_p = _pulses(w, 3, seed=21)
    test_p = _pulses(w, 1, seed=99)[0]
    s = _solver(w)
    s.mlp_set_weights(_theta(np.random.default_rng(5), zero_out=True))
    nsteps = w.Nt - 1
    s.mlp_record(len(train_p) * nsteps * s.ne)
    for pu in train_p:
        s.set_incident_plane(pu)
        s.reset()
        s.march(nsteps)
    X, T, Wt = s.mlp_samples(0, s.mlp_count())
    base = float(np.mean(Wt * T.astype(np.float64) ** 2))
    loss = s.mlp_train(epochs=6, batch=4096, lr=3e-4, seed=3)
    s.mlp_record(0)

    def run(use):
        s.set_incident_plane(test_p)
        s.reset()
        s.mlp_use(use)
        J = s.march(nsteps)
        return J, s.info().total_solver_iters, s.mlp_stats()

    J0, it0, _ = run(False)
    J1, it1, (used, fb) = run(True)
    print(f"\nwidth 256: loss {base:.3e} -> {list(np.round(loss, 4))}; Krylov iterations {it0} -> {it1}; "
          f"network used {used}, fallback {fb}")
    assert loss[-1] < loss[0] and loss[-1] < 0.9 * base, (base, loss)
    assert np.linalg.norm(J1 - J0) <= 1e-11 * np.linalg.norm(J0)
    assert used > fb, (used, fb)
