"""Fast mode (space-time interpolation FMM, paper section 3) on the GPU.

The fast path evaluates the same discretisation as the direct path (near
pairs with the identical coefficients, stored in FP32) and replaces the far
pairs by interpolation of the kernel in space and time.  Its bookkeeping --
hierarchy, time gating, lag ranges, window truncation, the M2L symmetries,
M2M and L2L -- is checked exact by tests/test_gpu_far_exact.py (a kernel the
interpolation reproduces, against the oracle's plain windowed sum).  What is
left here is the interpolation error of the method's own kernels:

* it must fall with the interpolation orders (a property, not a tuned bar);
* the absolute bounds below are regression guards at about twice the values
  measured on a GB300 (stated per test), not accuracy claims;
* the metric's 1e-4 on the 7680-RWG sphere is not reached, and the test that
  asks for it is an expected failure (strict): the collocated second time
  derivative of the quadratic B-spline makes the discrete vector-potential
  response step with r at the scale c dt, which no polynomial interpolant of
  the kernel follows (measured floor about 3e-4 at p = 8).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _solver(w, **kw):
    from paper_2303_05006_gb300 import Solver

    s = Solver(w.verts, w.tris, w.dt, w.Nt, **kw)
    s.set_incident_plane(w.pulses[0])
    return s


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def sphere1280_direct():
    from workloads import workload

    w = workload("sphere1280")
    s = _solver(w, mode=0)
    J = s.march(w.Nt - 1)
    s.close()
    return w, J


def test_plan_structure_sphere7680():
    from workloads import workload

    w = workload("sphere7680")
    s = _solver(w, mode=1)
    inf = s.info()
    assert inf.lmax == 3 and inf.mt_leaf >= 3
    assert inf.n_far_pairs > 10000
    assert inf.n_near_pairs < 0.1 * s.ne * s.ne


def test_fast_converges_with_interpolation_order(sphere1280_direct):
    """1920-RWG sphere, 299 steps: rel l2 (fast vs direct) measured 1.3e-2 at
    p = 4 and 9.1e-4 at p = 6."""
    w, Jd = sphere1280_direct
    e4 = _rel(_solver(w, mode=1, p_s=4, p_t=4).march(w.Nt - 1), Jd)
    e6 = _rel(_solver(w, mode=1, p_s=6, p_t=6).march(w.Nt - 1), Jd)
    assert e4 < 3e-2, e4
    assert e6 < 2e-3, e6
    assert e6 < e4 / 5


def test_fast_history_eval_is_the_march_operator(sphere1280_direct):
    """history_eval in fast mode (far field replayed from step 1 on the given
    history) against the direct operator on the same physical history; the
    relative error of the history part falls with p."""
    w, Jd = sphere1280_direct
    sd = _solver(w, mode=0)
    errs = {}
    for p in (4, 6):
        sf = _solver(w, mode=1, p_s=p, p_t=p)
        e = []
        for a in (40, 80, 120):
            V = sd.history_eval(a, np.zeros((0, sd.ne)))
            Rd = sd.history_eval(a, Jd[: a - 1])
            Rf = sf.history_eval(a, Jd[: a - 1])
            e.append(np.linalg.norm(Rf - Rd) / np.linalg.norm(V - Rd))
        errs[p] = max(e)
    # measured: 2.0e-2 (p = 4) and 3.9e-3 (p = 6)
    assert errs[4] < 4e-2, errs
    assert errs[6] < errs[4] / 3, errs


def test_fast_step_equals_march():
    from workloads import workload

    w = workload("sphere1280")
    s = _solver(w, mode=1)
    J1 = np.stack([s.step()[0] for _ in range(40)])
    s.reset()
    J2 = s.march(40)
    # far-field contributions are summed with FP32 atomics in any order
    assert _rel(J1, J2) < 1e-6


def test_fast_history_eval_vs_oracle_rows(sphere1280_direct):
    """Sampled rows of the fast history evaluation against the FP64 oracle
    (rows assembled one by one) on the physical history of the march."""
    from oracle.oracle import Oracle

    w, Jd = sphere1280_direct
    o = Oracle(w.verts, w.tris, w.dt)
    rows = np.sort(np.random.default_rng(3).choice(o.ne, 24, replace=False))
    mats = o.assemble(rows)
    sf = _solver(w, mode=1, p_s=6, p_t=6)
    for a in (60, 110):
        Rf = sf.history_eval(a, Jd[: a - 1])[rows]
        V = o.rhs(w.pulses[0], a, rows)
        Hr = o.history(a, Jd[: a - 1], rows, mats=mats)
        assert np.linalg.norm(Rf - (V - Hr)) <= 5e-3 * np.linalg.norm(Hr)


def test_fast_full_size_sphere7680():
    """The benchmark workload: 7680 RWG, 999 steps, p = 4; measured rel l2
    7.3e-3 against the direct FP64 path (itself pinned to the oracle)."""
    from workloads import workload

    w = workload("sphere7680")
    Jd = _solver(w, mode=0).march(w.Nt - 1)
    Jf = _solver(w, mode=1).march(w.Nt - 1)
    e = _rel(Jf, Jd)
    assert e < 1.5e-2, e
    assert np.abs(Jf[-50:]).max() < 1e-2 * np.abs(Jd).max()


@pytest.mark.xfail(strict=True, reason="interpolation floor of the vector-potential term: 6.0e-3 at p = 4, "
                   "2.8e-4 at p = 8 (the collocated B-spline second derivative steps with r at the scale c dt)")
def test_fast_meets_the_metric_bar_sphere7680():
    """The metric's accuracy bar: fast currents within 1e-4 relative l2 of the
    FP64 direct march (itself the oracle's to 1e-10) over all 999 steps of the
    7680-RWG sphere at p_s = p_t = 4."""
    from workloads import workload

    w = workload("sphere7680")
    Jd = _solver(w, mode=0).march(w.Nt - 1)
    Jf = _solver(w, mode=1).march(w.Nt - 1)
    assert _rel(Jf, Jd) <= 1e-4


def test_tensor_core_m2l_precisions(sphere1280_direct):
    """M2L on tcgen05 tensor cores against the FP32 CUDA-core M2L (1920-RWG
    sphere, 299 steps).  The truncated-power kernel grows quadratically with
    the lag and the far field of old sources is a telescoping cancellation
    across lags, so operand rounding is amplified: the split forms (about 16
    and 22 operand bits) track FP32, the single-pass TF32 and BF16 forms do
    not (measured: BF16x3 6.8e-4, TF32 4.1e-2, BF16 3.6e-1).  The FP16 split
    (operators and moment columns scaled by powers of two into FP16's range)
    carries as many bits as the TF32 split and is held to the same bar."""
    w, Jd = sphere1280_direct
    J = {prec: _solver(w, mode=1, m2l_prec=prec).march(w.Nt - 1) for prec in (0, 1, 2, 3, 4, 5)}
    e = {prec: _rel(J[prec], J[0]) for prec in (1, 2, 3, 4, 5)}
    print("\nM2L forms, rel l2 against the FP32 M2L:", {k: f"{v:.2e}" for k, v in e.items()})
    assert e[4] < 1e-4, e     # TF32 x 3
    assert e[5] < 1e-4, e     # FP16 x 3
    assert e[3] < 3e-3, e     # BF16 x 3
    assert e[1] > 10 * e[4] and e[2] > 10 * e[3], e
    # the accurate tensor-core forms keep the fast path's error at the FP32 level
    assert abs(_rel(J[4], Jd) - _rel(J[0], Jd)) < 1e-4
    assert abs(_rel(J[5], Jd) - _rel(J[0], Jd)) < 1e-4


def test_m2l_tile_shapes_and_autotuner(sphere1280_direct):
    """Both tensor-core M2L shapes (one or two 128-row operator tiles per CTA)
    give the same march up to the order of FP32 atomic additions, and the
    setup autotuner reports the shape it measured faster on every far level."""
    w, Jd = sphere1280_direct
    J = {rows: _solver(w, mode=1, m2l_prec=4, m2l_tile_rows=rows).march(w.Nt - 1) for rows in (128, 256)}
    # measured 2.4e-5: the far field's FP32 atomics add in a different order
    # (an indexing fault in either shape gives an O(1) difference)
    assert _rel(J[256], J[128]) < 1e-4
    assert abs(_rel(J[256], Jd) - _rel(J[128], Jd)) < 1e-4
    s = _solver(w, mode=1, m2l_prec=4)
    inf = s.info()
    chosen = [inf.m2l_tile_rows[l] for l in range(2, inf.lmax + 1)]
    assert chosen and all(r in (128, 256) for r in chosen), chosen


def test_fp16_resident_operator_kernel(sphere1280_direct):
    """The FP16 form's two kernels -- the tiled one and the one that keeps the
    operator's 128-row tiles resident in shared memory (m2l_tile_rows = 1
    forces it) -- give the same march up to the order of the FP32 atomic
    additions, and the autotuner reports which one each level runs."""
    w, Jd = sphere1280_direct
    Jt = _solver(w, mode=1, m2l_prec=5, m2l_tile_rows=128).march(w.Nt - 1)
    sr = _solver(w, mode=1, m2l_prec=5, m2l_tile_rows=1)
    inf = sr.info()
    assert inf.m2l_resident == sum(1 << l for l in range(2, inf.lmax + 1)), inf.m2l_resident
    Jr = sr.march(w.Nt - 1)
    assert _rel(Jr, Jt) < 1e-4
    assert abs(_rel(Jr, Jd) - _rel(Jt, Jd)) < 1e-4
    sa = _solver(w, mode=1, m2l_prec=5)
    ia = sa.info()
    print("\nautotuned: resident levels mask", ia.m2l_resident, "tile rows", list(ia.m2l_tile_rows))
    assert ia.m2l_resident & ~sum(1 << l for l in range(2, ia.lmax + 1)) == 0


def test_far_overlap_matches_program_order():
    """The M2L products of lag q >= 2, whose local coefficients are first read
    one interval after the event that fires them, run on the context's second
    stream while the next steps proceed (far_overlap = 1).  The currents must
    equal those of Program 1's serial order (far_overlap = 0) up to the order
    of the FP32 atomic additions into the local coefficients, which already
    makes two serial marches differ (measured 4.2e-5 relative l2 over 260
    steps of the 7680-RWG sphere, against 7.3e-3 for the interpolation error):
    with two far levels (the level-2 L2L meets the deferred level-3 products),
    the tensor-core and the CUDA-core M2L, through march, step by step (calls
    that return without waiting for the second stream), after a reset and in
    history evaluation."""
    from workloads import workload

    w = workload("sphere7680")
    n = 260  # past the pulse's arrival (step ~140)
    ref = {}
    for prec in (4, 0):
        Ja = _solver(w, mode=1, m2l_prec=prec, far_overlap=1).march(n)
        Jb = _solver(w, mode=1, m2l_prec=prec, far_overlap=0).march(n)
        Jc = _solver(w, mode=1, m2l_prec=prec, far_overlap=0).march(n)
        floor = _rel(Jc, Jb)
        assert np.abs(Jb).max() > 0
        assert floor < 2e-4, floor
        assert _rel(Ja, Jb) < max(4 * floor, 1e-6), (prec, _rel(Ja, Jb), floor)
        ref[prec] = (Jb, floor)
    Jb, floor = ref[4]
    s = _solver(w, mode=1, m2l_prec=4, far_overlap=1)
    Js = np.stack([s.step()[0] for _ in range(n)])
    assert _rel(Js, Jb) < max(4 * floor, 1e-6)
    # reset and history evaluation wait for the deferred products
    s.reset()
    Jr = s.march(n)
    assert _rel(Jr, Jb) < max(4 * floor, 1e-6)
    # caller-supplied right-hand sides (step_v) use the same sums launched ahead
    m = 180
    V = [s.history_eval(a, np.zeros((0, s.ne))) for a in range(1, m + 1)]
    s.reset()
    Jv = np.zeros((m, s.ne))
    for a in range(m):
        s.step_v(V[a], Jv[a])
    assert _rel(Jv, Jb[:m]) < max(4 * floor, 1e-6)
    alpha = 200
    Rm = s.history_eval(alpha, Jb[: alpha - 1])
    R0 = _solver(w, mode=1, m2l_prec=4, far_overlap=0).history_eval(alpha, Jb[: alpha - 1])
    assert _rel(Rm, R0) < 1e-6
