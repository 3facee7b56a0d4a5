"""Closed triangle meshes for the synthetic workloads.

Every generator returns ``(verts, tris)``: ``verts`` is a float64 array of shape
``(nv, 3)`` and ``tris`` an int32 array of shape ``(nf, 3)`` whose rows are wound
counter-clockwise when seen from outside the body (outward winding).  The meshes
are closed 2-manifolds: every edge is shared by exactly two triangles.
"""
from __future__ import annotations

import numpy as np


def _orient_outward(verts: np.ndarray, tris: np.ndarray, centre: np.ndarray) -> np.ndarray:
    """Flip any triangle whose winding normal points towards ``centre``.

    Valid for bodies that are star-shaped about ``centre`` (all bodies here).
    """
    v0, v1, v2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = np.cross(v1 - v0, v2 - v0)
    cen = (v0 + v1 + v2) / 3.0 - centre
    flip = np.einsum("ij,ij->i", nrm, cen) < 0
    out = tris.copy()
    out[flip] = out[flip][:, [0, 2, 1]]
    return out


def icosphere(radius: float = 1.0, subdivisions: int = 2):
    """Icosahedron refined by recursive midpoint subdivision, projected to a sphere.

    ``subdivisions`` = 2 gives 320 triangles, 3 gives 1280, 4 gives 5120.
    """
    g = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, g, 0), (1, g, 0), (-1, -g, 0), (1, -g, 0),
         (0, -1, g), (0, 1, g), (0, -1, -g), (0, 1, -g),
         (g, 0, -1), (g, 0, 1), (-g, 0, -1), (-g, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(subdivisions):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    V = np.array(verts) * radius
    T = np.array(faces, dtype=np.int32)
    return V, _orient_outward(V, T, np.zeros(3))


def geodesic_sphere(radius: float = 1.0, freq: int = 8):
    """Icosahedral geodesic sphere of frequency ``freq`` with equal-arc
    spacing (20 freq^2 triangles): on every face (A, B, C) of the icosahedron
    inscribed in the unit sphere, the grid point with weights (n - i - j, i, j)
    lies on the great circle between the points at arc fraction (i + j)/n from
    A towards B and towards C, at fraction j/(i + j) of the arc between them.
    These are the meshes of the paper's test problem (section 4.1, Table 1):
    their edge lengths match the table's minimum, mean and maximum."""
    g = (1.0 + 5.0 ** 0.5) / 2.0
    base = np.array([(-1, g, 0), (1, g, 0), (-1, -g, 0), (1, -g, 0),
                     (0, -1, g), (0, 1, g), (0, -1, -g), (0, 1, -g),
                     (g, 0, -1), (g, 0, 1), (-g, 0, -1), (-g, 0, 1)], dtype=np.float64)
    base /= np.linalg.norm(base, axis=1)[:, None]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    n = freq

    def slerp(p, q, t):
        w = np.arccos(np.clip(p @ q, -1.0, 1.0))
        if w < 1e-14:
            return p
        return (np.sin((1 - t) * w) * p + np.sin(t * w) * q) / np.sin(w)

    index: dict[tuple, int] = {}
    verts = []

    def vid(a, b, c, i, j):
        # points shared by two faces get one index through their integer weights
        w = {a: n - i - j, b: i, c: j}
        key = tuple(sorted((k, v) for k, v in w.items() if v))
        if key not in index:
            r = i + j
            p = base[a] if r == 0 else slerp(slerp(base[a], base[b], r / n), slerp(base[a], base[c], r / n), j / r)
            verts.append(p / np.linalg.norm(p))
            index[key] = len(verts) - 1
        return index[key]

    tris = []
    for a, b, c in faces:
        for i in range(n):
            for j in range(n - i):
                tris.append((vid(a, b, c, i, j), vid(a, b, c, i + 1, j), vid(a, b, c, i, j + 1)))
                if i + j < n - 1:
                    tris.append((vid(a, b, c, i + 1, j), vid(a, b, c, i + 1, j + 1), vid(a, b, c, i, j + 1)))
    V = np.array(verts) * radius
    T = np.array(tris, dtype=np.int32)
    return V, _orient_outward(V, T, np.zeros(3))


def cube_jittered(side: float = 2.0, n: int = 16, jitter: float = 0.02, seed: int = 3,
                  centre=(0.0, 0.0, 0.0)):
    """Cube surface: each face is an ``n``x``n`` grid of squares, each square split
    into 4 triangles by a centre vertex (``6*n*n*4`` triangles).  Every vertex
    coordinate is then perturbed by U(-jitter*h, +jitter*h), h = side/n, seeded.
    """
    h = side / n
    key_to_idx: dict[tuple[int, int, int], int] = {}
    verts: list[tuple[float, float, float]] = []

    def vid(ix: int, iy: int, iz: int) -> int:
        # integer lattice of half-squares: coordinates in units of h/2
        k = (ix, iy, iz)
        if k not in key_to_idx:
            key_to_idx[k] = len(verts)
            verts.append((ix * h / 2 - side / 2, iy * h / 2 - side / 2, iz * h / 2 - side / 2))
        return key_to_idx[k]

    tris = []
    N2 = 2 * n
    for axis in range(3):
        for lo_hi in (0, N2):
            for a in range(n):
                for b in range(n):
                    def P(u: int, w: int) -> int:
                        c = [0, 0, 0]
                        c[axis] = lo_hi
                        c[(axis + 1) % 3] = u
                        c[(axis + 2) % 3] = w
                        return vid(*c)
                    p00, p10 = P(2 * a, 2 * b), P(2 * a + 2, 2 * b)
                    p11, p01 = P(2 * a + 2, 2 * b + 2), P(2 * a, 2 * b + 2)
                    pc = P(2 * a + 1, 2 * b + 1)
                    tris += [(p00, p10, pc), (p10, p11, pc), (p11, p01, pc), (p01, p00, pc)]
    V = np.array(verts, dtype=np.float64)
    rng = np.random.default_rng(seed)
    V = V + rng.uniform(-jitter * h, jitter * h, size=V.shape)
    V = V + np.asarray(centre, dtype=np.float64)
    T = np.array(tris, dtype=np.int32)
    return V, _orient_outward(V, T, np.asarray(centre, dtype=np.float64))


def cylinder_cone(diameter: float = 1.0, length: float = 2.0, n_around: int = 64,
                  n_body: int = 25, cone_height: float = 0.5, n_cone: int = 4):
    """Cylinder along z capped by a cone at each end.

    ``n_body`` quad bands on the body and ``n_cone`` rings per cone (the last one a
    fan to the apex): ``2*n_around*n_body + 2*(n_around + 2*n_around*(n_cone-1))``
    triangles (4096 for the defaults).
    """
    R = diameter / 2
    th = 2 * np.pi * np.arange(n_around) / n_around
    rings = []
    for k in range(n_body + 1):
        z = -length / 2 + length * k / n_body
        rings.append(np.stack([R * np.cos(th), R * np.sin(th), np.full_like(th, z)], 1))
    verts = list(np.concatenate(rings))
    ring_idx = [np.arange(n_around) + k * n_around for k in range(n_body + 1)]
    tris = []

    def band(r0, r1):
        for i in range(n_around):
            j = (i + 1) % n_around
            tris.append((r0[i], r0[j], r1[j]))
            tris.append((r0[i], r1[j], r1[i]))

    for k in range(n_body):
        band(ring_idx[k], ring_idx[k + 1])
    for end, sgn in ((0, -1.0), (n_body, 1.0)):
        prev = ring_idx[end]
        z0 = sgn * length / 2
        for c in range(1, n_cone):
            frac = c / n_cone
            r = R * (1 - frac)
            z = z0 + sgn * cone_height * frac
            base = len(verts)
            verts += list(np.stack([r * np.cos(th), r * np.sin(th), np.full_like(th, z)], 1))
            cur = np.arange(n_around) + base
            band(prev, cur)
            prev = cur
        apex = len(verts)
        verts.append(np.array([0.0, 0.0, z0 + sgn * cone_height]))
        for i in range(n_around):
            tris.append((prev[i], prev[(i + 1) % n_around], apex))
    V = np.array(verts, dtype=np.float64)
    T = np.array(tris, dtype=np.int32)
    return V, _orient_outward(V, T, np.zeros(3))


def ellipsoid_uv(axes=(2.0, 0.5, 0.25), n_lon: int = 80, n_lat: int = 65):
    """UV ellipsoid: ``n_lat`` latitude bands (polar fans at both ends) by ``n_lon``
    longitudes; ``2*n_lon*(n_lat-1)`` triangles (10240 for the defaults)."""
    a, b, c = axes
    verts = [np.array([0.0, 0.0, c])]
    for i in range(1, n_lat):
        phi = np.pi * i / n_lat
        for j in range(n_lon):
            lam = 2 * np.pi * j / n_lon
            verts.append(np.array([a * np.sin(phi) * np.cos(lam), b * np.sin(phi) * np.sin(lam), c * np.cos(phi)]))
    verts.append(np.array([0.0, 0.0, -c]))
    south = len(verts) - 1

    def idx(i: int, j: int) -> int:
        return 1 + (i - 1) * n_lon + (j % n_lon)

    tris = []
    for j in range(n_lon):
        tris.append((0, idx(1, j), idx(1, j + 1)))
    for i in range(1, n_lat - 1):
        for j in range(n_lon):
            tris.append((idx(i, j), idx(i + 1, j), idx(i + 1, j + 1)))
            tris.append((idx(i, j), idx(i + 1, j + 1), idx(i, j + 1)))
    for j in range(n_lon):
        tris.append((idx(n_lat - 1, j), south, idx(n_lat - 1, j + 1)))
    V = np.array(verts, dtype=np.float64)
    T = np.array(tris, dtype=np.int32)
    return V, _orient_outward(V, T, np.zeros(3))


def octa_ellipsoid(axes=(2.0, 0.5, 0.25), freq: int = 100):
    """Octahedral geodesic sphere of frequency ``freq`` (8*freq^2 triangles) scaled
    to an ellipsoid with the given semi-axes."""
    corners = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], dtype=np.float64)
    faces = [(0, 1, 4), (1, 2, 4), (2, 3, 4), (3, 0, 4), (1, 0, 5), (2, 1, 5), (3, 2, 5), (0, 3, 5)]
    key_to_idx: dict[tuple[int, int, int], int] = {}
    verts: list[np.ndarray] = []

    def vid(p: np.ndarray) -> int:
        k = tuple(np.round(p * freq).astype(np.int64))
        if k not in key_to_idx:
            key_to_idx[k] = len(verts)
            verts.append(p)
        return key_to_idx[k]

    tris = []
    for fa, fb, fc in faces:
        A, B, C = corners[fa], corners[fb], corners[fc]

        def P(i: int, j: int) -> int:  # i + j <= freq
            return vid((A * (freq - i - j) + B * i + C * j) / freq)

        for i in range(freq):
            for j in range(freq - i):
                tris.append((P(i, j), P(i + 1, j), P(i, j + 1)))
                if i + j < freq - 1:
                    tris.append((P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)))
    V = np.array(verts)
    V = V / np.linalg.norm(V, axis=1, keepdims=True) * np.asarray(axes, dtype=np.float64)
    T = np.array(tris, dtype=np.int32)
    return V, _orient_outward(V, T, np.zeros(3))


def mean_edge_length(verts: np.ndarray, tris: np.ndarray) -> float:
    """Mean length over the distinct edges of the mesh."""
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    e = np.unique(np.sort(e, axis=1), axis=0)
    return float(np.linalg.norm(verts[e[:, 0]] - verts[e[:, 1]], axis=1).mean())
