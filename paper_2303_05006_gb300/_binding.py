"""ctypes binding of ``include/tdbem.h`` (argument marshalling only).

Function names follow the C ABI one to one (``lib().tdbem_step`` ...); the
:class:`Solver` class wraps a context with numpy arrays for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "libtdbem.so")

TDBEM_DIRECT, TDBEM_FAST = 0, 1
TDBEM_P_FP32, TDBEM_P_TF32, TDBEM_P_BF16, TDBEM_P_BF16X3, TDBEM_P_TF32X3 = 0, 1, 2, 3, 4
TDBEM_P_F16X3, TDBEM_P_FP64, TDBEM_P_FP24 = 5, 6, 7
_STATUS = {0: "OK", 1: "EINVAL", 2: "EMESH", 3: "EBREAKDOWN", 4: "ENOMEM", 5: "ENOCONV", 6: "ETIMEOUT",
           7: "ESTATE", 8: "ECUDA"}

_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_fp = ctypes.POINTER(ctypes.c_float)


class Params(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("p_s", ctypes.c_int32), ("p_t", ctypes.c_int32), ("n_leaf", ctypes.c_int32),
                ("theta", ctypes.c_double), ("zeta", ctypes.c_double), ("eps", ctypes.c_double),
                ("mu", ctypes.c_double), ("s_jump", ctypes.c_double), ("mode", ctypes.c_int32),
                ("m2l_prec", ctypes.c_int32), ("solve_tol", ctypes.c_double), ("solve_maxit", ctypes.c_int32),
                ("warm_start", ctypes.c_int32), ("n_rhs", ctypes.c_int32), ("jacobi_sweeps", ctypes.c_int32),
                ("m2l_tile_rows", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("far_overlap", ctypes.c_int32), ("solve_grid", ctypes.c_int32), ("chi", ctypes.c_double),
                ("far_kernel", ctypes.c_int32), ("s_interp", ctypes.c_int32), ("t_interp", ctypes.c_int32),
                ("a_deriv", ctypes.c_int32), ("solve_cluster", ctypes.c_int32),
                ("max_device_bytes", ctypes.c_int64), ("p2p_prec", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("ne", ctypes.c_int64), ("n_tri", ctypes.c_int64), ("lmax", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("mt_leaf", ctypes.c_int32), ("n_near_pairs", ctypes.c_int64),
                ("near_coef_bytes", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("setup_seconds", ctypes.c_double), ("total_solver_iters", ctypes.c_int64),
                ("solver_cluster", ctypes.c_int32), ("n_far_pairs", ctypes.c_int64),
                ("m2l_flops_per_step", ctypes.c_double), ("total_jacobi_sweeps", ctypes.c_int64),
                ("m2l_tile_rows", ctypes.c_int32 * 8), ("z0_nnz", ctypes.c_int64), ("max_lag", ctypes.c_int32),
                ("m2l_resident", ctypes.c_int32), ("device_bytes_peak", ctypes.c_int64),
                ("history_bytes", ctypes.c_int64)]


class TdbemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"tdbem {_STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _LIB


def lib():
    """Load ``libtdbem.so``; raises if it is missing (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            raise ImportError(f"{_LIB} is not built; run __graft_entry__.build() "
                              "(the CUDA library is the only implementation)")
        L = ctypes.CDLL(_LIB)
        vp = ctypes.c_void_p
        L.tdbem_default_params.argtypes = [ctypes.POINTER(Params)]
        L.tdbem_default_params.restype = None
        L.tdbem_create.argtypes = [_dp, ctypes.c_int64, _i32p, ctypes.c_int64, ctypes.c_double, ctypes.c_int32,
                                   ctypes.POINTER(Params), ctypes.POINTER(vp)]
        L.tdbem_num_edges.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
        L.tdbem_edges.argtypes = [vp, _i32p, _i32p]
        L.tdbem_set_stream.argtypes = [vp, vp]
        L.tdbem_set_incident_plane.argtypes = [vp, ctypes.c_int32, _dp]
        L.tdbem_set_rhs.argtypes = [vp, ctypes.c_int32, _dp]
        L.tdbem_history_eval.argtypes = [vp, ctypes.c_int32, _dp, ctypes.c_int32, _dp]
        L.tdbem_history_eval_noalloc.argtypes = [vp, ctypes.c_int32, _dp, ctypes.c_int32, _dp]
        L.tdbem_step.argtypes = [vp, _dp, _i32p]
        L.tdbem_march.argtypes = [vp, ctypes.c_int32, _dp]
        L.tdbem_march_dev.argtypes = [vp, ctypes.c_int32, vp]
        L.tdbem_step_v.argtypes = [vp, _dp, _dp, _i32p]
        L.tdbem_step_v_async.argtypes = [vp, _dp, _dp]
        L.tdbem_step_wait.argtypes = [vp, _i32p]
        L.tdbem_profile_enable.argtypes = [vp, ctypes.c_int32]
        L.tdbem_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), _dp, _i32p]
        L.tdbem_reset.argtypes = [vp]
        L.tdbem_alpha.argtypes = [vp, _i32p]
        L.tdbem_get_info.argtypes = [vp, ctypes.POINTER(Info)]
        L.tdbem_last_error.argtypes = [vp]
        L.tdbem_last_error.restype = ctypes.c_char_p
        L.tdbem_destroy.argtypes = [vp]
        L.tdbem_destroy.restype = None
        i64, i64p = ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)
        L.tdbem_mlp_set_width.argtypes = [vp, ctypes.c_int32]
        L.tdbem_mlp_set_weights.argtypes = [vp, _fp]
        L.tdbem_mlp_get_weights.argtypes = [vp, _fp]
        L.tdbem_mlp_record.argtypes = [vp, i64]
        L.tdbem_mlp_record_every.argtypes = [vp, ctypes.c_int32]
        L.tdbem_mlp_samples.argtypes = [vp, i64, i64, _fp, _fp, _fp, i64p]
        L.tdbem_mlp_train.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_uint64, _fp]
        L.tdbem_mlp_grad.argtypes = [vp, _fp, _fp, _fp, i64, ctypes.POINTER(ctypes.c_float), _fp]
        L.tdbem_mlp_forward.argtypes = [vp, _fp, i64, _fp]
        L.tdbem_mlp_use.argtypes = [vp, ctypes.c_int32]
        L.tdbem_mlp_stats.argtypes = [vp, i64p, i64p]
        L.tdbem_march_many.argtypes = [ctypes.POINTER(vp), ctypes.c_int32, _i32p, ctypes.POINTER(vp), _i32p]
        L.tdbem_save.argtypes = [vp, ctypes.c_char_p]
        L.tdbem_load.argtypes = [vp, ctypes.c_char_p]
        for name in ("tdbem_create", "tdbem_num_edges", "tdbem_edges", "tdbem_set_stream", "tdbem_set_incident_plane",
                     "tdbem_set_rhs", "tdbem_history_eval", "tdbem_step", "tdbem_march", "tdbem_march_dev",
                     "tdbem_reset", "tdbem_alpha", "tdbem_get_info", "tdbem_step_v", "tdbem_step_v_async", "tdbem_step_wait",
                     "tdbem_profile_enable",
                     "tdbem_profile_read", "tdbem_history_eval_noalloc", "tdbem_mlp_set_width", "tdbem_mlp_set_weights",
                     "tdbem_mlp_get_weights", "tdbem_mlp_record", "tdbem_mlp_record_every", "tdbem_mlp_samples", "tdbem_mlp_train",
                     "tdbem_mlp_grad", "tdbem_mlp_forward", "tdbem_mlp_use", "tdbem_mlp_stats", "tdbem_march_many",
                     "tdbem_save", "tdbem_load"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


class Solver:
    """One marching context (a thin owner of a ``tdbem_ctx*``).

    With ``n_rhs = R > 1`` every per-step array carries the right-hand side
    index before the edge index: J and R are (R, ne), histories (n, R, ne) and
    march results (n_steps, R, ne).  With R = 1 they keep the plain (ne,) and
    (n, ne) shapes.
    """

    def __init__(self, verts, tris, dt: float, Nt: int, **params):
        L = lib()
        p = Params()
        L.tdbem_default_params(ctypes.byref(p))
        for k, v in params.items():
            if not hasattr(p, k):
                raise TypeError(f"unknown parameter {k}")
            setattr(p, k, v)
        self.params = p
        self.verts = np.ascontiguousarray(verts, dtype=np.float64)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32)
        self.Nt = int(Nt)
        h = ctypes.c_void_p()
        rc = L.tdbem_create(_ptr(self.verts), len(self.verts), _ptr(self.tris, _i32p), len(self.tris), float(dt),
                            self.Nt, ctypes.byref(p), ctypes.byref(h))
        if rc != 0:
            raise TdbemError(rc, "tdbem_create failed")
        self._h = h
        ne = ctypes.c_int64()
        L.tdbem_num_edges(h, ctypes.byref(ne))
        self.ne = int(ne.value)
        self.R = int(p.n_rhs)

    def _vshape(self, *lead):
        return (*lead, self.ne) if self.R == 1 else (*lead, self.R, self.ne)

    def _check(self, rc):
        if rc != 0:
            raise TdbemError(rc, lib().tdbem_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().tdbem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def edges(self):
        ev = np.zeros((self.ne, 2), np.int32)
        et = np.zeros((self.ne, 2), np.int32)
        self._check(lib().tdbem_edges(self._h, _ptr(ev, _i32p), _ptr(et, _i32p)))
        return ev, et

    def set_stream(self, stream_handle: int | None):
        self._check(lib().tdbem_set_stream(self._h, ctypes.c_void_p(stream_handle or 0)))

    def set_incident_plane(self, pulse, rhs: int = 0):
        a = np.ascontiguousarray(pulse.as_array() if hasattr(pulse, "as_array") else pulse, dtype=np.float64)
        self._check(lib().tdbem_set_incident_plane(self._h, rhs, _ptr(a)))

    def set_rhs(self, V, rhs: int = 0):
        V = np.ascontiguousarray(V, dtype=np.float64)
        if V.shape != (self.Nt - 1, self.ne):
            raise ValueError("V must have shape (Nt-1, ne)")
        self._check(lib().tdbem_set_rhs(self._h, rhs, _ptr(V)))

    def history_eval(self, alpha: int, J_hist) -> np.ndarray:
        J = np.ascontiguousarray(J_hist, dtype=np.float64).reshape(-1, self.R * self.ne)
        out = np.zeros(self._vshape())
        self._check(lib().tdbem_history_eval(self._h, int(alpha), _ptr(J) if J.size else None, J.shape[0], _ptr(out)))
        return out

    def history_eval_noalloc(self, alpha: int, J_hist) -> np.ndarray:
        """As history_eval, staging the history in the library's fixed device
        scratch array instead of allocating device memory."""
        J = np.ascontiguousarray(J_hist, dtype=np.float64).reshape(-1, self.R * self.ne)
        out = np.zeros(self._vshape())
        self._check(lib().tdbem_history_eval_noalloc(self._h, int(alpha), _ptr(J) if J.size else None, J.shape[0],
                                                     _ptr(out)))
        return out

    def step(self):
        J = np.zeros(self._vshape())
        it = ctypes.c_int32()
        self._check(lib().tdbem_step(self._h, _ptr(J), ctypes.byref(it)))
        return J, int(it.value)

    def step_v(self, V, J_out=None):
        V = np.ascontiguousarray(V, dtype=np.float64)
        if V.size != self.R * self.ne:
            raise ValueError("V must hold n_rhs * ne values")
        it = ctypes.c_int32()
        self._check(lib().tdbem_step_v(self._h, _ptr(V), _ptr(J_out), ctypes.byref(it)))
        return int(it.value)

    def step_v_async(self, V, J_out=None):
        """Enqueue one step with right-hand side V (tdbem_step_v_async).  V
        and J_out should be pinned host arrays that stay alive until the step
        is waited for; J_out is written then."""
        if V.size != self.R * self.ne or V.dtype != np.float64 or not V.flags.c_contiguous:
            raise ValueError("V must be a contiguous float64 array of n_rhs * ne values")
        self._check(lib().tdbem_step_v_async(self._h, _ptr(V), _ptr(J_out)))

    def step_wait(self) -> int:
        """Wait for the oldest outstanding asynchronous step; its solver iterations."""
        it = ctypes.c_int32()
        self._check(lib().tdbem_step_wait(self._h, ctypes.byref(it)))
        return int(it.value)

    def profile(self, on: bool = True):
        self._check(lib().tdbem_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        n = ctypes.c_int32()
        launches = (ctypes.c_int64 * 16)()
        ms = np.zeros(16)
        self._check(lib().tdbem_profile_read(self._h, launches, _ptr(ms), ctypes.byref(n)))
        k = int(n.value)
        return np.array(launches[:k]), ms[:k]

    def march(self, n_steps: int, out=None) -> np.ndarray:
        if out is None:
            out = np.zeros(self._vshape(n_steps))
        self._check(lib().tdbem_march(self._h, int(n_steps), _ptr(out)))
        return out

    def march_dev(self, n_steps: int, dev_ptr: int | None = None):
        self._check(lib().tdbem_march_dev(self._h, int(n_steps), ctypes.c_void_p(dev_ptr or 0)))

    def reset(self):
        self._check(lib().tdbem_reset(self._h))

    @property
    def alpha(self) -> int:
        a = ctypes.c_int32()
        self._check(lib().tdbem_alpha(self._h, ctypes.byref(a)))
        return int(a.value)

    # ---- learned warm start (see include/tdbem.h)
    MLP_FEATURES, MLP_WIDTH = 25, 64

    @property
    def MLP_NPARAM(self) -> int:
        H = self.MLP_WIDTH
        return H * self.MLP_FEATURES + H * H + H

    def mlp_set_width(self, width: int):
        self._check(lib().tdbem_mlp_set_width(self._h, int(width)))
        self.MLP_WIDTH = int(width)

    def mlp_set_weights(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        if t.size != self.MLP_NPARAM:
            raise ValueError(f"theta must hold {self.MLP_NPARAM} values")
        self._check(lib().tdbem_mlp_set_weights(self._h, t.ctypes.data_as(_fp)))

    def mlp_get_weights(self) -> np.ndarray:
        t = np.zeros(self.MLP_NPARAM, np.float32)
        self._check(lib().tdbem_mlp_get_weights(self._h, t.ctypes.data_as(_fp)))
        return t

    def mlp_record(self, capacity: int):
        self._check(lib().tdbem_mlp_record(self._h, ctypes.c_int64(int(capacity))))

    def mlp_record_every(self, every: int):
        self._check(lib().tdbem_mlp_record_every(self._h, int(every)))

    def mlp_count(self) -> int:
        n = ctypes.c_int64()
        self._check(lib().tdbem_mlp_samples(self._h, ctypes.c_int64(0), ctypes.c_int64(0), None, None, None,
                                            ctypes.byref(n)))
        return int(n.value)

    def mlp_samples(self, first: int, n: int):
        X = np.zeros((n, self.MLP_FEATURES), np.float32)
        T = np.zeros(n, np.float32)
        W = np.zeros(n, np.float32)
        self._check(lib().tdbem_mlp_samples(self._h, ctypes.c_int64(first), ctypes.c_int64(n),
                                            X.ctypes.data_as(_fp), T.ctypes.data_as(_fp), W.ctypes.data_as(_fp),
                                            None))
        return X, T, W

    def mlp_train(self, epochs: int, batch: int, lr: float, seed: int = 0) -> np.ndarray:
        loss = np.zeros(max(epochs, 1), np.float32)
        self._check(lib().tdbem_mlp_train(self._h, int(epochs), int(batch), ctypes.c_float(lr),
                                          ctypes.c_uint64(seed), loss.ctypes.data_as(_fp)))
        return loss[:epochs]

    def mlp_grad(self, X, T, W=None):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        Wp = None if W is None else np.ascontiguousarray(W, dtype=np.float32)
        g = np.zeros(self.MLP_NPARAM, np.float32)
        loss = ctypes.c_float()
        self._check(lib().tdbem_mlp_grad(self._h, X.ctypes.data_as(_fp), T.ctypes.data_as(_fp),
                                         None if Wp is None else Wp.ctypes.data_as(_fp), ctypes.c_int64(len(T)),
                                         ctypes.byref(loss), g.ctypes.data_as(_fp)))
        return float(loss.value), g

    def mlp_forward(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float32)
        Y = np.zeros(X.shape[0], np.float32)
        self._check(lib().tdbem_mlp_forward(self._h, X.ctypes.data_as(_fp), ctypes.c_int64(X.shape[0]),
                                            Y.ctypes.data_as(_fp)))
        return Y

    def mlp_use(self, on: bool = True):
        self._check(lib().tdbem_mlp_use(self._h, 1 if on else 0))

    def mlp_stats(self):
        u, f = ctypes.c_int64(), ctypes.c_int64()
        self._check(lib().tdbem_mlp_stats(self._h, ctypes.byref(u), ctypes.byref(f)))
        return int(u.value), int(f.value)

    def save(self, path: str) -> None:
        """Write the march state to `path` (tdbem_save)."""
        self._check(lib().tdbem_save(self._h, os.fsencode(path)))

    def load(self, path: str) -> None:
        """Continue from the march state in `path` (tdbem_load)."""
        self._check(lib().tdbem_load(self._h, os.fsencode(path)))

    def info(self) -> Info:
        inf = Info()
        self._check(lib().tdbem_get_info(self._h, ctypes.byref(inf)))
        return inf


def march_many(solvers, n_steps, dev_ptrs=None) -> None:
    """March several Solver contexts together (tdbem_march_many): steps are
    issued in rounds, each context on its own stream.  n_steps: one count per
    solver; dev_ptrs: optional device pointers (ints) receiving each
    context's currents, [n_steps][n_rhs][ne] float64."""
    n = len(solvers)
    hs = (ctypes.c_void_p * n)(*[s._h.value if hasattr(s._h, "value") else s._h for s in solvers])
    ns = np.ascontiguousarray(n_steps, dtype=np.int32)
    dp = None if dev_ptrs is None else (ctypes.c_void_p * n)(*[p or 0 for p in dev_ptrs])
    failed = ctypes.c_int32(-1)
    rc = lib().tdbem_march_many(hs, n, ns.ctypes.data_as(_i32p), dp, ctypes.byref(failed))
    if rc != 0:
        who = solvers[failed.value] if 0 <= failed.value < n else None
        raise TdbemError(rc, lib().tdbem_last_error(who._h).decode() if who else "tdbem_march_many failed")
