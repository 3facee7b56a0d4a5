"""Python front end of the FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It loads ``liboracle.so`` (built from
``oracle.c`` by :func:`build`) through ctypes and adds the two steps the C file
leaves to library routines: the LU factorisation of the instantaneous matrix
Zt^(1) (paper eq. solve: w^{0,d} Z^(1) J^{alpha-1} = R^{alpha-1}) and the
marching loop of the paper's Program 1 specialised to the conventional method
(section 3.6.3), i.e. for alpha = 1 .. Nt-1:

    R^{alpha-1} = V^{alpha-1} - sum_{m >= 2} Zt^(m) J^{alpha-m}     (eq. R)
    J^{alpha-1} = Zt^(1)^{-1} R^{alpha-1}                          (eq. solve)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

c_double_p = ctypes.POINTER(ctypes.c_double)
c_int32_p = ctypes.POINTER(ctypes.c_int32)
c_int64_p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc and OpenMP (FP64, no fast-math)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _SO, _SRC, "-lm"])
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        L.orc_create.argtypes = [c_double_p, ctypes.c_int64, c_int32_p, ctypes.c_int64, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
        L.orc_create.restype = ctypes.c_int
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_num_edges.argtypes = [ctypes.c_void_p]
        L.orc_num_edges.restype = ctypes.c_int64
        L.orc_edges.argtypes = [ctypes.c_void_p, c_int32_p, c_int32_p, c_int32_p]
        L.orc_window.argtypes = [ctypes.c_void_p]
        L.orc_window.restype = ctypes.c_int
        L.orc_window_rows.argtypes = [ctypes.c_void_p, c_int64_p, ctypes.c_int64]
        L.orc_window_rows.restype = ctypes.c_int
        L.orc_inner.argtypes = [ctypes.c_void_p, c_double_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                c_double_p, c_double_p, c_double_p, c_double_p]
        L.orc_inner.restype = ctypes.c_int
        L.orc_assemble.argtypes = [ctypes.c_void_p, c_int64_p, ctypes.c_int64, ctypes.c_int, c_int32_p, c_double_p]
        L.orc_assemble.restype = ctypes.c_int
        L.orc_history.argtypes = [ctypes.c_void_p, c_int32_p, c_double_p, ctypes.c_int, ctypes.c_int64,
                                  c_double_p, ctypes.c_int64, ctypes.c_int64, c_double_p]
        L.orc_rhs.argtypes = [ctypes.c_void_p, c_double_p, ctypes.c_int64, c_int64_p, ctypes.c_int64, c_double_p]
        L.orc_threads.restype = ctypes.c_int
        L.orc_bspline.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int]
        L.orc_bspline.restype = ctypes.c_double
        L.orc_bspline_weights.argtypes = [ctypes.c_int, c_double_p]
        L.orc_gl.argtypes = [c_double_p, c_double_p]
        L.orc_gl.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def threads() -> int:
    return int(lib().orc_threads())


def bspline(tau: float, q: int = 0, d: int = 2) -> float:
    """q-th derivative of the order-d B-spline N (q = -1: its running integral)."""
    return float(lib().orc_bspline(d, float(tau), q))


def bspline_weights(d: int = 2) -> np.ndarray:
    w = np.zeros(d + 2)
    lib().orc_bspline_weights(d, _p(w, c_double_p))
    return w


def gauss_legendre():
    x = np.zeros(64); w = np.zeros(64)
    n = lib().orc_gl(_p(x, c_double_p), _p(w, c_double_p))
    return x[:n].copy(), w[:n].copy()


class Oracle:
    """Conventional FP64 MOT TDBEM on one closed triangle mesh."""

    def __init__(self, verts, tris, dt, theta=1.0, zeta=1.0, eps=1.0, mu=1.0, sJ=1.0, d=2, chi=1.0):
        L = lib()
        self.verts = np.ascontiguousarray(verts, dtype=np.float64)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32)
        self.dt = float(dt)
        self.params = dict(theta=theta, zeta=zeta, eps=eps, mu=mu, sJ=sJ, d=d, chi=chi)
        h = ctypes.c_void_p()
        rc = L.orc_create(_p(self.verts, c_double_p), len(self.verts), _p(self.tris, c_int32_p), len(self.tris),
                          self.dt, eps, mu, theta, zeta, sJ, chi, d, ctypes.byref(h))
        if rc != 0:
            raise ValueError(f"oracle: invalid mesh or parameters (code {rc})")
        self._h = h
        self.ne = int(L.orc_num_edges(h))
        self._W = None
        self._full = None
        self._lu = None

    def __del__(self):
        try:
            if self._h:
                lib().orc_destroy(self._h)
        except Exception:
            pass

    # -- mesh tables ------------------------------------------------------
    def edges(self):
        ev = np.zeros((self.ne, 2), np.int32)
        et = np.zeros((self.ne, 2), np.int32)
        eo = np.zeros((self.ne, 2), np.int32)
        lib().orc_edges(self._h, _p(ev, c_int32_p), _p(et, c_int32_p), _p(eo, c_int32_p))
        return ev, et, eo

    def window(self) -> int:
        if self._W is None:
            self._W = int(lib().orc_window(self._h))
        return self._W

    # -- inner integrals (for the pins) ------------------------------------
    def inner(self, x, tri: int, m0: int, nm: int):
        x = np.ascontiguousarray(x, dtype=np.float64)
        phi = np.zeros(nm); A0 = np.zeros(nm); A1 = np.zeros((nm, 3)); P1 = np.zeros((nm, 3))
        rc = lib().orc_inner(self._h, _p(x, c_double_p), tri, m0, nm, _p(phi, c_double_p), _p(A0, c_double_p),
                             _p(A1, c_double_p), _p(P1, c_double_p))
        if rc != 0:
            raise ValueError("oracle: inner integral arguments out of range")
        return phi, A0, A1, P1

    # -- matrices -----------------------------------------------------------
    def assemble(self, rows=None):
        """Rows of every Zt^(m): returns (m_lo [nrows, ne] int32, Zw [nrows, ne, W])
        with Zw[r, j, w] = Zt^(m_lo[r, j] + w)_{rows[r], j}."""
        full = rows is None
        if full and self._full is not None:
            return self._full
        rows = np.arange(self.ne, dtype=np.int64) if full else np.ascontiguousarray(rows, dtype=np.int64)
        # the storage window: over all pairs once for a full assembly, over the
        # requested rows' pairs otherwise
        W = self.window() if full else int(lib().orc_window_rows(self._h, _p(rows, c_int64_p), len(rows)))
        m_lo = np.zeros((len(rows), self.ne), np.int32)
        Zw = np.zeros((len(rows), self.ne, W), np.float64)
        rc = lib().orc_assemble(self._h, _p(rows, c_int64_p), len(rows), W, _p(m_lo, c_int32_p), _p(Zw, c_double_p))
        if rc != 0:
            raise RuntimeError("oracle: assembly window overflow")
        if full:
            self._full = (m_lo, Zw)
        return m_lo, Zw

    def z_lag(self, m: int, rows=None) -> np.ndarray:
        """Dense Zt^(m) restricted to ``rows`` (all rows by default)."""
        m_lo, Zw = self.assemble(rows)
        w = m - m_lo
        ok = (w >= 0) & (w < Zw.shape[2])
        out = np.zeros(m_lo.shape)
        r, j = np.nonzero(ok)
        out[r, j] = Zw[r, j, w[r, j]]
        return out

    # -- right-hand sides -----------------------------------------------------
    def rhs(self, pulse, alpha: int, rows=None) -> np.ndarray:
        """V^{alpha-1} (incident field tested at t_alpha), eq. v_i."""
        rows = np.arange(self.ne, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
        P = np.ascontiguousarray(pulse.as_array() if hasattr(pulse, "as_array") else pulse, dtype=np.float64)
        V = np.zeros(len(rows))
        lib().orc_rhs(self._h, _p(P, c_double_p), alpha, _p(rows, c_int64_p), len(rows), _p(V, c_double_p))
        return V

    def history(self, alpha: int, J_hist: np.ndarray, rows=None, mats=None) -> np.ndarray:
        """sum_{m >= 2} Zt^(m) J^{alpha-m} for the given rows; J_hist[b] = J^b."""
        m_lo, Zw = mats if mats is not None else self.assemble(rows)
        J = np.ascontiguousarray(J_hist, dtype=np.float64)
        out = np.zeros(m_lo.shape[0])
        lib().orc_history(self._h, _p(m_lo, c_int32_p), _p(Zw, c_double_p), Zw.shape[2], m_lo.shape[0],
                          _p(J, c_double_p), J.shape[0], alpha, _p(out, c_double_p))
        return out

    def history_eval(self, alpha: int, J_hist: np.ndarray, V=None, rows=None) -> np.ndarray:
        """R^{alpha-1} = V^{alpha-1} - sum_{m>=2} Zt^(m) J^{alpha-m} (eq. R)."""
        h = self.history(alpha, J_hist, rows)
        return (0.0 if V is None else V) - h

    # -- marching ------------------------------------------------------------
    def _factor(self):
        if self._lu is None:
            import scipy.linalg
            import scipy.sparse
            import scipy.sparse.linalg
            Z0 = self.z_lag(1)
            if self.ne <= 3000:
                self._lu = ("dense", scipy.linalg.lu_factor(Z0))
            else:
                self._lu = ("sparse", scipy.sparse.linalg.splu(scipy.sparse.csc_matrix(Z0)))
        return self._lu

    def solve0(self, R: np.ndarray) -> np.ndarray:
        """Zt^(1)^{-1} R by the LU factors (computed once)."""
        kind, f = self._factor()
        if kind == "dense":
            import scipy.linalg
            return scipy.linalg.lu_solve(f, R)
        return f.solve(R)

    def march(self, pulse, Nt: int, V_all=None) -> np.ndarray:
        """J^0 .. J^{Nt-2} (shape [Nt-1, ne]) for the incident ``pulse`` or the
        supplied right-hand sides ``V_all[alpha-1]``."""
        self.assemble()
        self._factor()
        J = np.zeros((Nt - 1, self.ne))
        for alpha in range(1, Nt):
            V = V_all[alpha - 1] if V_all is not None else self.rhs(pulse, alpha)
            R = V - self.history(alpha, J[: alpha - 1])
            J[alpha - 1] = self.solve0(R)
        return J
