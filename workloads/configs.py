"""Workload definitions: meshes, time stepping and incident-pulse parameters.

Units are normalised (c = eps = mu = eta = 1): lengths in metres, time in m/c.
The incident pulse is a modulated Gaussian plane wave

    E(x, t) = pol * g(t - (k . x - z_min)/c),  H = k x E / eta,
    g(u) = cos(2 pi f0 (u - t0)) * exp(-(u - t0)^2 / (2 sigma^2)),

whose band edge f_max = c / (10 h_ref) puts at least ten mean edges of the
5120-triangle sphere (h_ref) in the shortest wavelength; f0 = f_max/2 and sigma
is chosen so that the spectrum has fallen to 1e-3 of its peak at f_max; t0 = 6
sigma.  Only the parameters live here; evaluating the field is each solver's job.
"""
from __future__ import annotations

import dataclasses
import functools
import math

import numpy as np

from .meshes import cube_jittered, cylinder_cone, ellipsoid_uv, icosphere, mean_edge_length, octa_ellipsoid


@dataclasses.dataclass(frozen=True)
class Pulse:
    k: tuple[float, float, float]      # unit propagation direction
    pol: tuple[float, float, float]    # unit polarisation, orthogonal to k
    f0: float
    sigma: float
    t0: float
    z_min: float                       # min over the mesh of k . x (time origin)

    def as_array(self) -> np.ndarray:
        return np.array([*self.k, *self.pol, self.f0, self.sigma, self.t0, self.z_min], dtype=np.float64)


@functools.lru_cache(maxsize=1)
def _h_ref() -> float:
    v, t = icosphere(1.0, 4)
    return mean_edge_length(v, t)


def pulse_star(verts: np.ndarray, k=(0.0, 0.0, 1.0), pol=(1.0, 0.0, 0.0), f_scale: float = 1.0,
               sigma_scale: float = 1.0) -> Pulse:
    """The reference pulse (x-polarised, travelling along +z by default)."""
    f_max = 1.0 / (10.0 * _h_ref())
    f0 = 0.5 * f_max * f_scale
    sigma = math.sqrt(math.log(1e3) / 2.0) / (math.pi * (f_max - 0.5 * f_max)) * sigma_scale
    kk = np.asarray(k, dtype=np.float64)
    kk = kk / np.linalg.norm(kk)
    z_min = float(np.min(verts @ kk))
    return Pulse(tuple(float(x) for x in kk), tuple(float(x) for x in np.asarray(pol, dtype=np.float64)),
                 float(f0), float(sigma), float(6.0 * sigma), z_min)


def sin2_pulse(verts: np.ndarray, k=(0.0, 0.0, -1.0), pol=(1.0, 0.0, 0.0), length: float = 0.5,
               amplitude: float = 0.5) -> Pulse:
    """The Sin^2 pulse of the paper's test problem (section 4.1): E = pol A
    Sin^2(2 pi (c t - (k.x - z_min)) / Lambda), one period of sin^2 long; stored
    in the pulse record as f0 = Lambda and sigma = -A (a negative sigma selects
    this shape).  Defaults: along -x3, x-polarised, Lambda = A = 0.5."""
    kk = np.asarray(k, dtype=np.float64)
    kk = kk / np.linalg.norm(kk)
    z_min = float(np.min(verts @ kk))
    return Pulse(tuple(float(x) for x in kk), tuple(float(x) for x in np.asarray(pol, dtype=np.float64)),
                 float(length), -float(amplitude), 0.0, z_min)


def random_plane_waves(n: int, seed: int):
    """``n`` seeded (direction, polarisation) pairs: directions uniform on the
    sphere (normalised Gaussian 3-vectors), polarisation at a uniform angle in the
    plane orthogonal to the direction."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        k = rng.standard_normal(3)
        k /= np.linalg.norm(k)
        a = np.cross(k, [1.0, 0.0, 0.0])
        if np.linalg.norm(a) < 0.3:
            a = np.cross(k, [0.0, 1.0, 0.0])
        a /= np.linalg.norm(a)
        b = np.cross(k, a)
        phi = rng.uniform(0, 2 * np.pi)
        out.append((k, np.cos(phi) * a + np.sin(phi) * b))
    return out


@dataclasses.dataclass
class Workload:
    name: str
    verts: np.ndarray
    tris: np.ndarray
    dt: float
    Nt: int
    pulses: list
    p_s: int = 4
    p_t: int = 4
    n_leaf: int = 64
    # CFIE coupling of eq. cfie; the paper's theta = zeta = 1 on the spheres.
    # The other shapes use 3: there the fast march at 1 grows without bound
    # after the pulse has passed, and a heavier MFIE share keeps it stable
    theta: float = 1.0
    zeta: float = 1.0

    @property
    def n_tri(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_edge(self) -> int:
        return int(self.tris.shape[0] * 3 // 2)


def _sphere(sub: int, Nt: int, name: str) -> Workload:
    v, t = icosphere(1.0, sub)
    return Workload(name, v, t, 0.5 * mean_edge_length(v, t), Nt, [pulse_star(v)])


def workload(name: str) -> Workload:
    """Build a named workload.

    * ``sphere320``   : icosphere r=1, 320 triangles (480 RWG), Nt=128
    * ``sphere1280``  : icosphere r=1, 1280 triangles (1920 RWG), Nt=300
    * ``sphere7680``  : icosphere r=1, 5120 triangles (7680 RWG), Nt=1000
    * ``sphere_cube`` : the 5120-triangle sphere plus a jittered cube of side 2
                        (6144 triangles) centred at (3.5, 0, 0), Nt=1000
    * ``cylinder``    : cone-capped cylinder, 4096 triangles, Nt=1500
    * ``ellipsoid10k``: UV ellipsoid (2, 0.5, 0.25), 10240 triangles, Nt=1500
    * ``ellipsoid5k`` : the 5120-triangle icosphere scaled to the ellipsoid (2, 0.5, 0.25), Nt=1000
                        (the learned warm start's training shape)
    * ``ellipsoid80k``: octahedral geodesic ellipsoid, 80000 triangles, Nt=4000
    * ``*_small``     : the same shapes with fewer steps, for quick tests
    """
    if name == "sphere320":
        return _sphere(2, 128, name)
    if name == "sphere1280":
        return _sphere(3, 300, name)
    if name == "sphere7680":
        return _sphere(4, 1000, name)
    if name == "sphere80":
        return _sphere(1, 64, name)
    if name == "sphere_cube":
        vs, ts = icosphere(1.0, 4)
        vc, tc = cube_jittered(2.0, 16, 0.02, 3, centre=(3.5, 0.0, 0.0))
        v = np.concatenate([vs, vc])
        t = np.concatenate([ts, tc + len(vs)]).astype(np.int32)
        return Workload(name, v, t, 0.5 * mean_edge_length(vs, ts), 1000, [pulse_star(v)], theta=3.0, zeta=3.0)
    if name == "cylinder":
        v, t = cylinder_cone()
        return Workload(name, v, t, 0.5 * mean_edge_length(v, t), 1500, [pulse_star(v)], theta=3.0, zeta=3.0)
    if name == "ellipsoid10k":
        v, t = ellipsoid_uv()
        return Workload(name, v, t, 0.5 * mean_edge_length(v, t), 1500, [pulse_star(v)], theta=3.0, zeta=3.0)
    if name == "ellipsoid5k":
        v, t = icosphere(1.0, 4)
        v = v * np.array([2.0, 0.5, 0.25])
        return Workload(name, v, t, 0.5 * mean_edge_length(v, t), 1000, [pulse_star(v)], theta=3.0, zeta=3.0)
    if name == "ellipsoid80k":
        v, t = octa_ellipsoid(freq=100)
        return Workload(name, v, t, 0.5 * mean_edge_length(v, t), 4000, [pulse_star(v)], theta=3.0, zeta=3.0)
    raise KeyError(name)


WORKLOADS = ("sphere80", "sphere320", "sphere1280", "sphere7680", "sphere_cube", "cylinder",
             "ellipsoid10k", "ellipsoid5k", "ellipsoid80k")


def random_history(n_edge: int, n_steps: int, seed: int) -> np.ndarray:
    """Seeded standard-normal current history, shape (n_steps, n_edge), float64."""
    return np.random.default_rng(seed).standard_normal((n_steps, n_edge))
