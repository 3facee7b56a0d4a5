"""Mirror symmetries of the oracle's marched currents on the sphere (CPU only).

The 80-triangle icosphere maps onto itself under the reflections y -> -y and
x -> -x (every coordinate sign of the icosahedron's vertices appears, and the
midpoint subdivision and its normalisation commute with a sign change).  The
incident plane wave of the reference pulse travels along +z, polarised along
x: E = x g(t - z).  A reflection R maps a polar vector field V to
R V(R r), so the incident field is even under y -> -y and odd under x -> -x
(its x component is the normal one).  The PEC problem is linear and the
scatterer symmetric, so the surface current obeys

    J(R r) = sigma R J(r),   sigma = +1 for y -> -y,  -1 for x -> -x,

at every step.  The current density is rebuilt at each triangle's centroid
from the RWG coefficients (section 2.2: on T+ it is l/(2A+) (r - v+), on T-
l/(2A-) (v- - r), v+- the vertices opposite the edge) and compared with the
reflected one of the mirror triangle.  A mistake in the oracle that breaks the
symmetry (a wrong vertex, edge orientation or quadrature point in the
assembly, an index transposed) fails here.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def sphere80_march():
    from oracle.oracle import Oracle
    from workloads import workload

    w = workload("sphere80")
    o = Oracle(w.verts, w.tris, w.dt)
    J = o.march(w.pulses[0], 41)  # J^0 .. J^39
    return w, o, J


def _centroid_currents(v, t, o, J):
    ev, et, eo = o.edges()
    cen = v[t].mean(axis=1)
    area = 0.5 * np.linalg.norm(np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]]), axis=1)
    Jc = np.zeros((J.shape[0], len(t), 3))
    for e in range(len(ev)):
        le = np.linalg.norm(v[ev[e, 1]] - v[ev[e, 0]])
        tp, tm = et[e]
        fp = le / (2 * area[tp]) * (cen[tp] - v[eo[e, 0]])
        fm = le / (2 * area[tm]) * (v[eo[e, 1]] - cen[tm])
        Jc[:, tp, :] += J[:, e, None] * fp[None, :]
        Jc[:, tm, :] += J[:, e, None] * fm[None, :]
    return Jc


def _mirror_triangles(v, t, axis):
    R = np.ones(3)
    R[axis] = -1.0
    index = {tuple(p): i for i, p in enumerate(v)}
    vmap = np.array([index[tuple(p * R)] for p in v])  # exact: a sign change is exact
    tri_index = {frozenset(tr): k for k, tr in enumerate(t)}
    return np.array([tri_index[frozenset(vmap[tr])] for tr in t]), R


@pytest.mark.parametrize("axis, sigma", [(1, 1.0), (0, -1.0)])
def test_currents_mirror_symmetric(sphere80_march, axis, sigma):
    w, o, J = sphere80_march
    v, t = np.asarray(w.verts), np.asarray(w.tris)
    Jc = _centroid_currents(v, t, o, J)
    tmap, R = _mirror_triangles(v, t, axis)
    scale = np.abs(Jc).max()
    assert scale > 0
    err = np.abs(Jc[:, tmap, :] - sigma * Jc * R[None, None, :]).max()
    assert err <= 1e-12 * scale, err / scale  # measured 1.5e-15
    # the other parity is far off: the check is not trivially satisfied
    assert np.abs(Jc[:, tmap, :] + sigma * Jc * R[None, None, :]).max() > 0.1 * scale


def test_mirror_maps_are_involutions(sphere80_march):
    w, _, _ = sphere80_march
    v, t = np.asarray(w.verts), np.asarray(w.tris)
    for axis in (0, 1):
        tmap, _ = _mirror_triangles(v, t, axis)
        assert np.array_equal(tmap[tmap], np.arange(len(t)))
        assert not np.array_equal(tmap, np.arange(len(t)))


def test_planted_asymmetric_incidence_breaks_the_mirror(sphere80_march):
    """Polarisation rotated by 0.17 rad towards y: the y -> -y mirror no
    longer holds, by far more than the bar above."""
    from workloads.configs import pulse_star

    w, o, _ = sphere80_march
    v, t = np.asarray(w.verts), np.asarray(w.tris)
    J = o.march(pulse_star(w.verts, pol=(np.cos(0.17), np.sin(0.17), 0.0)), 41)
    Jc = _centroid_currents(v, t, o, J)
    tmap, R = _mirror_triangles(v, t, 1)
    assert np.abs(Jc[:, tmap, :] - Jc * R[None, None, :]).max() > 0.1 * np.abs(Jc).max()
