"""Checkpoint and resume (tdbem_save / tdbem_load) on the GPU.

A march saved at step k and continued in a fresh context from the file must
give the currents of the uninterrupted march: bit for bit in direct mode
(the assembly and every reduction there run in a fixed order), and in fast mode within the
noise of the far field's FP32 atomic accumulation, measured here as the
difference between two uninterrupted marches.  Loading a file into a context
that does not match it is refused with EINVAL and leaves the state alone.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _solver(w, **kw):
    from paper_2303_05006_gb300 import Solver

    s = Solver(w.verts, w.tris, w.dt, w.Nt, theta=w.theta, zeta=w.zeta, **kw)
    s.set_incident_plane(w.pulses[0])
    return s


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_direct_march_is_reproducible():
    """Two contexts of the same problem march bit for bit alike: the coefficient
    assembly adds each edge pair's four triangle-pair contributions in a fixed
    order, and every later reduction runs in a fixed order too."""
    from workloads import workload

    w = workload("sphere320")
    assert np.array_equal(_solver(w).march(w.Nt - 1), _solver(w).march(w.Nt - 1))


def test_direct_resume_is_bit_identical(tmp_path):
    from workloads import workload

    w = workload("sphere320")
    n, k = w.Nt - 1, 53
    Jref = _solver(w).march(n)
    a = _solver(w)
    J1 = a.march(k)
    path = str(tmp_path / "direct.ck")
    a.save(path)
    a.close()
    b = _solver(w)
    b.load(path)
    J2 = b.march(n - k)
    assert np.array_equal(np.concatenate([J1, J2]), Jref)


def test_fast_resume_matches_uninterrupted(tmp_path):
    """Two far levels with gating events in flight at the save (step 83 is in
    the middle of intervals of both levels), deferred M2L products and
    near-field sums launched ahead (far_overlap = 1)."""
    from workloads import workload

    w = workload("sphere1280")
    n, k = 200, 83
    Ja = _solver(w, mode=1).march(n)
    Jb = _solver(w, mode=1).march(n)
    floor = _rel(Ja, Jb)
    a = _solver(w, mode=1)
    assert a.info().lmax >= 2
    J1 = a.march(k)
    path = str(tmp_path / "fast.ck")
    a.save(path)
    J1b = a.march(n - k)  # the saving context marches on unchanged
    a.close()
    b = _solver(w, mode=1)
    b.load(path)
    J2 = b.march(n - k)
    e = _rel(np.concatenate([J1, J2]), Ja)
    assert e <= max(4 * floor, 1e-6), (e, floor)
    assert _rel(np.concatenate([J1, J1b]), Ja) <= max(4 * floor, 1e-6)
    # a resume that lost the far field in flight would be far off
    c = _solver(w, mode=1)
    c.load(path)
    c.reset()
    assert _rel(c.march(n - k), Ja[k:]) > 1e-2


def test_load_refuses_a_foreign_checkpoint(tmp_path):
    from paper_2303_05006_gb300 import TdbemError
    from workloads import workload

    w = workload("sphere320")
    a = _solver(w)
    a.march(10)
    path = str(tmp_path / "a.ck")
    a.save(path)
    # another mesh
    w2 = workload("sphere80")
    ref = _solver(w2).march(10)
    b = _solver(w2)
    b.march(5)
    with pytest.raises(TdbemError) as ex:
        b.load(path)
    assert ex.value.code == 1  # TDBEM_EINVAL
    # the refused load left b's march where it was
    assert np.array_equal(b.march(5), ref[5:])
    # another mode on the same mesh
    c = _solver(w, mode=1)
    with pytest.raises(TdbemError):
        c.load(path)
    # a truncated file
    data = open(path, "rb").read()
    bad = str(tmp_path / "cut.ck")
    open(bad, "wb").write(data[: len(data) // 2])
    d = _solver(w)
    with pytest.raises(TdbemError):
        d.load(bad)
    with pytest.raises(TdbemError):
        d.load(str(tmp_path / "missing.ck"))
    # the intact file still loads
    d.load(path)
    assert os.path.getsize(path) > 8 * w.n_edge
