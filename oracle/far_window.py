"""The space-time hierarchy and the windowed far field of the fast method
(test infrastructure only: only tests/ may import this module).

This is a plain restatement of what the interpolation-based FMM of section 3
sums, so that the CUDA FMM's bookkeeping can be checked with a kernel that the
interpolation reproduces exactly.  Nothing here interpolates: the far field of
a triangle pair is summed directly over its window of source steps.

Hierarchy (section 3.4.1, with the readings listed in the design notes):
  * the root is the bounding cube of the vertices (side D = largest extent,
    enlarged by one part in 1e9 so that every centroid lies strictly inside),
    anchored at the smallest coordinates;
  * a triangle belongs to the cell that holds its centroid; a cell is split
    while it holds more than n_leaf edges (1.5 per triangle) and while its
    children's time intervals still hold d + 1 = 3 steps; empty cells are
    dropped;
  * eq. (Mt), floor reading: M at the deepest level l_max is
    floor((ds - 2 delta) / (c dt)), doubling towards the root, where delta is
    the largest distance from a centroid to its 7 outer-rule points (the
    interpolation boxes have half-width H = ds/2 + delta);
  * a triangle pair is near at the first level where the two cells are
    neighbours (27-neighbourhood) and one of them is a leaf; it is far at the
    first level (>= 2) where the cells are not neighbours: the interaction
    list of Program 4.

Window (Appendix A: the J-hat rewriting with the window-start truncation).
For a far pair at level l with cell offset o (canonically |o| sorted), the
boxes give r_min = |max(0, |o_k| ds - 2H)| and r_max = |(|o_k| ds + 2H)|, and
    q_lo = max(1, floor(r_min / (M c dt))),  q_hi = ceil((1 + r_max/(c dt)) / M).
The far field of target step alpha (the right-hand side R^{alpha-1}, target
time t_alpha, in interval k' = floor((alpha-1)/M)) sums the source steps gamma
of intervals k' - q_hi .. k' - q_lo against J-hat truncated at the window
start G = (k' - q_hi) M:
    Jhat_G^gamma = sum_{kappa = 0}^{min(3, gamma - G)} w^kappa J^{gamma - kappa},
    w = (1/2, -3/2, 3/2, -1/2)  (eq. hat_J, d = 2).
With the truncated-power kernel of eq. U this window sum equals the plain
B-spline sum over the whole history exactly; tests/test_far_window.py checks
that identity, which pins q_lo, q_hi, G and the truncation.
"""
from __future__ import annotations

import numpy as np

W_HAT = np.array([0.5, -1.5, 1.5, -0.5])  # w^{kappa,2} of eq. hat_J


def outer_rule():
    """The 7-point degree-5 rule on a triangle (Radon; Stroud T2:5-1):
    barycentric points [7, 3] and weights summing to 1."""
    s = np.sqrt(15.0)
    a1, a2 = (6 - s) / 21, (6 + s) / 21
    w1, w2 = (155 - s) / 1200, (155 + s) / 1200
    pts = [(1 / 3, 1 / 3, 1 / 3)]
    wts = [9 / 40]
    for a, w in ((a1, w1), (a2, w2)):
        pts += [(a, a, 1 - 2 * a), (a, 1 - 2 * a, a), (1 - 2 * a, a, a)]
        wts += [w, w, w]
    return np.array(pts), np.array(wts)


class Hierarchy:
    """Octree, per-level intervals and near/far classification of triangle pairs."""

    def __init__(self, verts, tris, dt, n_leaf=64, c=1.0):
        V = np.asarray(verts, dtype=np.float64)
        T = np.asarray(tris, dtype=np.int64)
        self.V, self.T, self.dt, self.c = V, T, float(dt), float(c)
        self.a = self.c * self.dt
        self.nt = len(T)
        P = V[T]  # [nt, 3, 3]
        self.cen = P.mean(axis=1)
        qb, _ = outer_rule()
        X = np.einsum("qk,tkd->tqd", qb, P)
        self.delta = float(np.max(np.linalg.norm(X - self.cen[:, None, :], axis=2)))
        lo, hi = V.min(axis=0), V.max(axis=0)
        self.root = lo
        self.D = float(np.max(hi - lo)) * (1 + 1e-9)
        # deepest level whose intervals still hold d + 1 = 3 steps
        self.lcap = max([l for l in range(30) if np.floor((self.ds(l) - 2 * self.delta) / self.a) >= 3] or [0])
        self.leaf = {}       # (level, ix, iy, iz) -> True (leaf) / False (split)
        self.leaf_level = np.zeros(self.nt, dtype=np.int64)
        self._split(0, (0, 0, 0), np.arange(self.nt), n_leaf)
        self.lmax = int(self.leaf_level.max())
        self.far = self.lmax >= 2
        self.M_deep = int(np.floor((self.ds(self.lmax) - 2 * self.delta) / self.a)) if self.far else 0

    def ds(self, l):
        return self.D / (1 << l)

    def H(self, l):
        return self.ds(l) / 2 + self.delta

    def M(self, l):
        """Steps per time interval at level l (eq. Mt, floor reading, doubling upwards)."""
        return self.M_deep << (self.lmax - l)

    def coords(self, t, l):
        """Integer cell coordinates at level l of the cell holding triangle(s) t."""
        return np.floor((self.cen[t] - self.root) / self.ds(l)).astype(np.int64)

    def _split(self, l, ijk, tris, n_leaf):
        split = 1.5 * len(tris) > n_leaf and l < self.lcap
        self.leaf[(l, *ijk)] = not split
        if not split:
            self.leaf_level[tris] = l
            return
        cc = self.coords(tris, l + 1)
        for child in {tuple(x) for x in cc}:
            sel = tris[np.all(cc == np.array(child), axis=1)]
            self._split(l + 1, child, sel, n_leaf)

    def is_leaf(self, l, ijk):
        return self.leaf[(l, *ijk)]

    def classify(self, t, S):
        """For triangle t against triangles S: kind (0 near, 1 far), level and
        cell offset (source cell minus target cell) at that level."""
        S = np.asarray(S, dtype=np.int64)
        kind = np.full(len(S), -1)
        lev = np.zeros(len(S), dtype=np.int64)
        off = np.zeros((len(S), 3), dtype=np.int64)
        todo = np.ones(len(S), dtype=bool)
        for l in range(0, self.lmax + 1):
            if not todo.any():
                break
            ct = self.coords(np.array([t]), l)[0]
            cs = self.coords(S, l)
            d = cs - ct
            adj = np.max(np.abs(d), axis=1) <= 1
            tleaf = self.leaf_level[t] == l
            sleaf = self.leaf_level[S] == l
            near = todo & adj & (tleaf | sleaf)
            far = todo & ~adj
            kind[near] = 0
            lev[near] = l
            kind[far] = 1
            lev[far] = l
            off[far] = d[far]
            todo &= ~(near | far)
        assert not todo.any(), "classification did not terminate"
        assert not np.any((kind == 1) & (lev < 2)), "far pair above level 2"
        return kind, lev, off

    def lag_range(self, l, offset):
        """(q_lo, q_hi) of the source intervals that reach a target interval (Appendix A reading)."""
        cv = np.sort(np.abs(np.asarray(offset, dtype=np.float64)))
        ds, H, M = self.ds(l), self.H(l), self.M(l)
        rmin = np.sqrt(np.sum(np.maximum(0.0, cv * ds - 2 * H) ** 2))
        rmax = np.sqrt(np.sum((cv * ds + 2 * H) ** 2))
        q_lo = max(1, int(np.floor(rmin / (M * self.a))))
        q_hi = int(np.ceil((1.0 + rmax / self.a) / M))
        return q_lo, q_hi

    def window(self, l, q_lo, q_hi, alpha):
        """(G, first source step, last source step) of target step alpha."""
        M = self.M(l)
        k = (alpha - 1) // M
        G = (k - q_hi) * M
        return G, max(G, 0), (k - q_lo + 1) * M - 1


def jhat_window(J, G, g0, g1):
    """Jhat_G^gamma for gamma = g0 .. g1 (rows of J: J[b] = J^b, J^{b<0} = 0);
    returns [g1 - g0 + 1, ...]."""
    out = []
    for g in range(g0, g1 + 1):
        acc = 0.0
        for kap in range(0, min(3, g - G) + 1):
            b = g - kap
            if 0 <= b < len(J):
                acc = acc + W_HAT[kap] * J[b]
        out.append(acc)
    return np.array(out)


def far_field_poly(h: Hierarchy, edges, rows, J, alpha, theta=1.0, zeta=1.0, chi=1.0, eps=1.0, mu=1.0,
                   absolute=False, tdeg=3):
    """sum over far triangle pairs of the tested coefficients times J, for the
    polynomial kernel K(x, y, t, s) = (1 + |x - y|^2) T3((t - s)/ts - 1), with
    T3(x) = 4x^3 - 3x (the Chebyshev cubic; with tdeg=2 the quadratic
    T2(x) = 2x^2 - 1 instead) and ts = 64 dt, on rows
    `rows` at target step alpha (the part of R^{alpha-1} = V - near - far that
    the far field contributes with a minus sign).  J[b] = J^b ([n_hist][ne]).

    The tested coefficient of a triangle pair follows eq. z_ij with the
    retarded integrals written through the kernel (section 3.3): with x on the
    test triangle (7-point rule), y on the source triangle (the same rule,
    exact for the cubic integrands here) and tau = t_alpha - s_gamma,
      mu/(4 pi) f_i . f_j d^2K/dt^2 + 1/(4 pi eps) div f_i div f_j K
      + theta eta/(4 pi) (f_i x n) . (f_j x grad_y (chi dK/dt + zeta K)),
    n the unit normal of the test triangle pointing into the conductor, summed
    against Jhat over the window of the pair.  The kernel is separable, so the
    time sums sum_gamma Jhat_G^gamma T3^(p)(x_gamma), x_gamma = (alpha -
    gamma) dt/ts - 1 (p = 0, 1, 2 derivatives), are formed once per edge and
    window.

    absolute=True returns instead a bound on the sum of the absolute values of
    all the terms (every factor taken in absolute value): the size against
    which rounding in a finite precision is measured."""
    ev, et, eo = edges
    V, T, dt = h.V, h.T, h.dt
    eta = np.sqrt(mu / eps)
    qb, qw = outer_rule()
    P = V[T]
    cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    area = 0.5 * np.linalg.norm(cr, axis=1)
    nout = cr / np.linalg.norm(cr, axis=1)[:, None]
    X = np.einsum("qk,tkd->tqd", qb, P)  # rule points of every triangle [nt, 7, 3]
    elen = np.linalg.norm(V[ev[:, 1]] - V[ev[:, 0]], axis=1)
    # sides of every triangle: edge, sign of its RWG function there, opposite vertex
    side_e = np.zeros((h.nt, 3), dtype=np.int64)
    side_s = np.zeros((h.nt, 3))
    side_o = np.zeros((h.nt, 3), dtype=np.int64)
    cnt = np.zeros(h.nt, dtype=np.int64)
    for j in range(len(ev)):
        for r, sg in ((0, 1.0), (1, -1.0)):
            t = et[j, r]
            side_e[t, cnt[t]], side_s[t, cnt[t]], side_o[t, cnt[t]] = j, sg, eo[j, r]
            cnt[t] += 1
    assert np.all(cnt == 3)
    J = np.asarray(J, dtype=np.float64).reshape(-1, len(ev))
    ts = 64.0 * dt
    tsum = {}  # (G, g0, g1) -> [3, ne]: sum over the window of Jhat T3(x), T3'(x), T3''(x)

    def time_sums(G, g0, g1):
        if (G, g0, g1) not in tsum:
            Jh = jhat_window(J, G, g0, g1)                               # [n, ne]
            x = (alpha - np.arange(g0, g1 + 1)) * dt / ts - 1.0
            if tdeg == 3:
                T = [4 * x ** 3 - 3 * x, 12 * x ** 2 - 3, 24 * x]        # T3 and its x-derivatives
            else:
                T = [2 * x ** 2 - 1, 4 * x, 4 + 0 * x]                   # T2 and its x-derivatives
            if absolute:
                Jh, T = np.abs(Jh), [np.abs(v) for v in T]
            tsum[(G, g0, g1)] = np.stack([v @ Jh for v in T])
        return tsum[(G, g0, g1)]

    out = np.zeros(len(rows))
    for ir, i in enumerate(rows):
        for r, sgi in ((0, 1.0), (1, -1.0)):
            t = et[i, r]
            fi = sgi * elen[i] / (2 * area[t]) * (X[t] - V[eo[i, r]])   # [7, 3]
            divi = sgi * elen[i] / area[t]
            fixn = np.cross(fi, -nout[t])                                  # f_i x n (n inward)
            wx = qw * area[t]
            kind, lev, off = h.classify(t, np.arange(h.nt))
            groups = {}
            for s in np.nonzero(kind == 1)[0]:
                q_lo, q_hi = h.lag_range(lev[s], off[s])
                G, g0, g1 = h.window(lev[s], q_lo, q_hi, alpha)
                if g1 >= g0:
                    groups.setdefault((G, g0, g1), []).append(s)
            for key, S in groups.items():
                S = np.array(S)
                Hs = time_sums(*key)                                       # [3, ne]
                Y = X[S]                                                   # [nS, 7, 3]
                dxy = Y[:, None, :, :] - X[t][None, :, None, :]           # y - x [nS, 7q, 7y, 3]
                g = 1.0 + np.sum(dxy * dxy, axis=3)
                ww = wx[None, :, None] * (qw[None, :] * area[S][:, None])[:, None, :]
                for k in range(3):
                    j = side_e[S, k]
                    cj = side_s[S, k] * elen[j] / (2 * area[S])
                    fj = cj[:, None, None] * (Y - V[side_o[S, k]][:, None, :])   # [nS, 7y, 3]
                    divj = 2 * cj
                    ab = np.abs if absolute else (lambda v: v)
                    sA = np.sum(ab(ww * np.einsum("qd,syd->sqy", fi, fj) * g), axis=(1, 2))
                    sF = ab(divi * divj) * np.sum(ww * g, axis=(1, 2))
                    sP = np.sum(ab(ww * np.einsum("qd,sqyd->sqy", fixn, np.cross(fj[:, None, :, :], 2 * dxy))),
                                axis=(1, 2))
                    K0, K1, K2 = Hs[0, j], Hs[1, j] / ts, Hs[2, j] / ts ** 2   # K, dK/dt, d2K/dt2 (g aside)
                    out[ir] += np.sum(mu / (4 * np.pi) * sA * K2
                                      + 1 / (4 * np.pi * eps) * sF * K0
                                      + theta * eta / (4 * np.pi) * sP * (chi * K1 + zeta * K0))
    return out
