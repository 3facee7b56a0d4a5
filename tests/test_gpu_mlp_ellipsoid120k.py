"""The learned warm start at its stated configuration: a width-256 network
(tensor-core inference and training) trained on 200 seeded-pulse
trajectories of the 5120-triangle ellipsoid (2, 0.5, 0.25) and used on the
8:2:1 ellipsoid with 80000 triangles (120000 RWG), the Z0 solve run to a
residual of 1e-10, fast path p_s = p_t = 4, FP16x3 M2L, theta = zeta = 3.

The training trajectories march 400 steps each (dt = h/2 of the training
mesh) from seeded plane waves with directions uniform on the sphere; every
20th step is recorded (30.7 M samples).  The network is then used on a
held-out wave at 120000 RWG for 400 steps and compared with the plain cubic
extrapolation: Krylov iterations of the Z0 solve, march time, and how often
the residual fallback kept the network's guess.

Measured on a GB300: the training loss falls from 1 (the extrapolation) to
0.66, but at 120000 RWG the network's guess wins the residual comparison in
only 3 of 400 solves and the Krylov iterations are unchanged (4419 ->
4418).  The finer mesh's step is four times shorter, so the cubic
extrapolation is far better there than on the training mesh, and the
network's corrections (learned where it was worse) overshoot.  Training
with the finer mesh's step instead was unstable (the per-step loss weights
blow up where the extrapolation is nearly exact).  What is held: training
lowers the loss, the currents agree with the plain run (the solve to 1e-10
decides them), and the fallback keeps the solver's work within 2% of the
plain run's.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_warm_start_trained_on_ellipsoid5k_used_at_120000_rwg():
    from paper_2303_05006_gb300 import Solver
    from workloads import workload
    from workloads.configs import pulse_star, random_plane_waves

    kw = dict(mode=1, p_s=4, p_t=4, m2l_prec=5, solve_tol=1e-10)
    H = 256
    w5 = workload("ellipsoid5k")
    s = Solver(w5.verts, w5.tris, w5.dt, w5.Nt, theta=w5.theta, zeta=w5.zeta, **kw)
    s.mlp_set_width(H)
    rng = np.random.default_rng(17)
    F = s.MLP_FEATURES
    th0 = np.concatenate([rng.standard_normal(H * F) / np.sqrt(F), rng.standard_normal(H * H) / np.sqrt(H),
                          np.zeros(H)]).astype(np.float32)
    s.mlp_set_weights(th0)
    nsteps, every, ntraj = 400, 20, 200
    s.mlp_record_every(every)
    s.mlp_record(ntraj * (nsteps // every) * s.ne)
    t0 = time.perf_counter()
    for k, pol in random_plane_waves(ntraj, seed=41):
        s.set_incident_plane(pulse_star(w5.verts, k=k, pol=pol))
        s.reset()
        s.march(nsteps)
    t_rec = time.perf_counter() - t0
    n = s.mlp_count()
    _, T, Wt = s.mlp_samples(0, n)
    base = float(np.mean(Wt * T.astype(np.float64) ** 2))
    t0 = time.perf_counter()
    loss = s.mlp_train(epochs=4, batch=8192, lr=1e-3, seed=5)
    t_train = time.perf_counter() - t0
    theta = s.mlp_get_weights()
    s.close()

    w = workload("ellipsoid80k")
    big = Solver(w.verts, w.tris, w.dt, w.Nt, theta=w.theta, zeta=w.zeta, **kw)
    (k, pol), = random_plane_waves(1, seed=977)
    big.set_incident_plane(pulse_star(w.verts, k=k, pol=pol))
    m = 400

    def run(use):
        big.reset()
        if use:
            big.mlp_set_width(H)
            big.mlp_set_weights(theta)
        big.mlp_use(use)
        it_before = big.info().total_solver_iters
        t = time.perf_counter()
        J = big.march(m)
        dt = time.perf_counter() - t
        return J, big.info().total_solver_iters - it_before, dt, big.mlp_stats() if use else (0, 0)

    J0, it0, t0_, _ = run(False)
    J1, it1, t1_, (used, fb) = run(True)
    rel = float(np.linalg.norm(J1 - J0) / np.linalg.norm(J0))
    print(f"\nwarm start at 120000 RWG: {n} samples from {ntraj} trajectories ({t_rec:.0f} s), "
          f"loss {base:.3e} -> {[round(float(x), 4) for x in loss]} ({t_train:.0f} s); "
          f"Krylov iterations over {m} steps {it0} -> {it1}; march {t0_:.2f} s -> {t1_:.2f} s; "
          f"network kept {used}, fallback {fb}; currents rel l2 {rel:.2e}")
    assert loss[-1] < loss[0]
    assert rel < 1e-4, rel
    assert used + fb == m
    assert it1 <= 1.02 * it0, (it0, it1)
