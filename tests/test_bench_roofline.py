"""Host logic of bench.py's roofline key (CPU only): the dominant kernel class
is the one with the most device time, and `achieved` is its algorithmic work
per launch over its mean launch time, against the peak of its own unit."""
import types

import numpy as np
import pytest


def _setup():
    import bench

    hbm, bf16, _ = bench._peaks()
    info = types.SimpleNamespace(m2l_flops_per_step=2.0e10, m2l_tile_rows=[0, 0, 256, 256, 0, 0, 0, 0],
                                 near_coef_bytes=4.0e9, n_near_pairs=5.0e7, z0_nnz=2.0e5,
                                 total_solver_iters=400, ne=7680, history_bytes=0)
    args = types.SimpleNamespace(prec="tf32x3", p=4, rhs=1, workload="sphere7680", far_overlap=1,
                                 mode="fast", precond=1)
    return bench, hbm, bf16, info, args


def _times(bench, dominant, ms_dom, launches_dom):
    n = len(bench.KERNELS)
    launches = np.ones(n, dtype=np.int64)
    ms = np.full(n, 1e-3)
    k = bench.KERNELS.index(dominant)
    launches[k], ms[k] = launches_dom, ms_dom
    return launches, ms


def test_profile_classes_match_the_header():
    import os

    import bench

    hdr = open(os.path.join(bench.ROOT, "include", "tdbem.h")).read()
    assert len(bench.KERNELS) == 11 and bench.KERNELS[9] == "history_split" and bench.KERNELS[10] == "history_reduce"
    assert "9 history split" in hdr and "1 history/near field" in hdr and "10 history reduction" in hdr


def test_m2l_tensor_roofline():
    bench, hbm, bf16, info, args = _setup()
    K = 100
    launches, ms = _times(bench, "m2l", 40.0, 300)
    r = bench.roofline(args, info, launches, ms, K, 3)
    tflops = info.m2l_flops_per_step * K / 0.040 / 1e12
    assert r["kernel"] == "m2l" and r["bound"] == "tensor"
    assert r["achieved"] == pytest.approx(tflops)
    assert r["peak"] == pytest.approx(bf16 * 1.1 / 2.25)  # TF32 from the BF16 peak by the nominal ratio
    assert r["frac"] == pytest.approx(tflops / r["peak"])
    assert r["flops_per_launch"] == pytest.approx(info.m2l_flops_per_step * K / 300)
    assert r["traffic"] == pytest.approx(bench.M2L_TRAFFIC_TF32X3)
    # the committed DRAM traffic belongs to one configuration only
    args.p = 5
    assert bench.roofline(args, info, launches, ms, K, 3)["traffic"] is None
    args.p, args.prec = 4, "bf16x3"
    r = bench.roofline(args, info, launches, ms, K, 3)
    assert r["peak"] == pytest.approx(bf16) and r["traffic"] is None


def test_direct_history_hbm_roofline():
    bench, hbm, _, info, args = _setup()
    args.mode = "direct"
    launches, ms = _times(bench, "near_history", 180.0, 100)
    r = bench.roofline(args, info, launches, ms, 100, 5)
    nbytes = info.near_coef_bytes + info.n_near_pairs * 3  # coefficients + lag window (m_lo, nlag) per pair
    gbs = nbytes / 1.8e-3 / 1e9
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["bytes_per_launch"] == pytest.approx(nbytes)
    assert r["achieved"] == pytest.approx(gbs) and r["frac"] == pytest.approx(gbs / hbm)


@pytest.mark.parametrize("mode", ["direct", "direct32"])
def test_row_tile_history_counts_its_store(mode):
    """The row-tile history sum streams its store once per launch: the bytes
    the library reports (values, first-lag bytes, group offsets); the solve
    beside it does not take the roofline even where it runs longer."""
    bench, hbm, _, info, args = _setup()
    args.mode = mode
    info.history_bytes = 2.3e9
    launches, ms = _times(bench, "near_history", 50.0, 100)
    k = bench.KERNELS.index("z0_solve")
    ms[k] = 60.0
    r = bench.roofline(args, info, launches, ms, 100, 5)
    assert r["kernel"] == "near_history" and r["bytes_per_launch"] == pytest.approx(2.3e9)
    assert r["achieved"] == pytest.approx(2.3e9 / 0.5e-3 / 1e9)


def test_fast_near_field_counts_flattened_entries():
    bench, hbm, _, info, args = _setup()
    launches, ms = _times(bench, "near_history", 20.0, 100)
    r = bench.roofline(args, info, launches, ms, 100, 5)
    assert r["bytes_per_launch"] == pytest.approx(2 * info.near_coef_bytes)  # 8 B entry per 4 B coefficient


def test_other_dominant_classes_are_latency_bound():
    bench, _, _, info, args = _setup()
    launches, ms = _times(bench, "l2p", 50.0, 100)
    r = bench.roofline(args, info, launches, ms, 100, 5)
    assert r["kernel"] == "l2p" and r["bound"] == "latency" and r["frac"] is None


def test_clock_sampler_parses_samples_and_reasons(tmp_path):
    """The clocks key: median SM clock over the samples under load (utilisation
    >= 50 %), the maximum, and every throttle reason seen active in any sample
    (nvidia-smi csv, no header)."""
    import bench

    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    s = bench.ClockSampler.__new__(bench.ClockSampler)
    s.path = str(tmp_path / "clocks.csv")
    s.p = _Done()
    rows = ["0, 2070, 2070, 900.1, 98, Not Active, Not Active, Not Active, Not Active",
            "0, 2055, 2070, 1390.0, 100, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1200.5, 99, Not Active, Not Active, Not Active, Not Active",
            "0, 1200, 2070, 150.0, 0, Not Active, Not Active, Not Active, Not Active",
            "0, [N/A], 2070, 0, 0, Not Active, Not Active, Not Active, Not Active"]
    open(s.path, "w").write("\n".join(rows) + "\n")
    c = s.stop()
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 4,
                 "samples_under_load": 3}
    # with no sample under load the median covers every sample
    c = bench.ClockSampler.parse(rows[3:])
    assert c["sm_mhz"] == 1200.0 and c["samples_under_load"] == 0


def test_z0_solve_counts_operand_bytes_per_solve():
    bench, hbm, _, info, args = _setup()
    K, W = 100, 4
    launches, ms = _times(bench, "z0_solve", 25.0, K + W)
    r = bench.roofline(args, info, launches, ms, K, W)
    its = info.total_solver_iters / (K + W)
    # per inner iteration two FP32 ELL SpMVs and 21 + 2 x 12 vector passes (triangle-block
    # preconditioner); two FP64 residuals per solve
    nbytes = its * (16 * info.z0_nnz + 4 * 45 * info.ne) + 2 * (12 * info.z0_nnz + 24 * info.ne)
    assert r["bound"] == "hbm" and r["bytes_per_launch"] == pytest.approx(nbytes)
    assert r["achieved"] == pytest.approx(nbytes / (25.0e-3 / (K + W)) / 1e9)


def test_headline_is_the_fastest_path_meeting_the_bar():
    import bench

    rates = {"direct": 1180.0, "direct32": 2170.0, "direct24": 2140.0, "fast": 2700.0}
    assert bench.headline_path(rates, {"direct32": True, "direct24": True, "fast": False}) == "direct32"
    # the 24-bit store is never the headline, even when faster
    rates24 = {**rates, "direct24": 2300.0}
    assert bench.headline_path(rates24, {"direct32": True, "direct24": True, "fast": False}) == "direct32"
    assert bench.headline_path(rates, {"direct32": True, "direct24": True, "fast": True}) == "fast"
    assert bench.headline_path(rates, {}) == "direct"  # the reference always qualifies
    assert bench.headline_path({"direct": 1.0, "fast": 2.0}, {"fast": False}) == "direct"


def test_per_step_history_error_uses_the_reference_history():
    """Each evaluation gets J^0 .. J^{alpha-2} of the reference march; steps
    beyond it are skipped."""
    import bench

    rng = np.random.default_rng(0)
    J = rng.standard_normal((50, 7))
    seen = []

    def ref(a, h):
        seen.append((a, h.shape[0]))
        return h.sum(axis=0) + 1.0

    def path(a, h):
        return (h.sum(axis=0) + 1.0) * (1 + 1e-3)

    out = bench.per_step_history_error(ref, path, J, (10, 40, 60))
    assert set(out) == {"10", "40"} and seen == [(10, 9), (40, 39)]
    assert all(abs(v - 1e-3) < 1e-12 for v in out.values())
