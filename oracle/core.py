"""ctypes binding of the C oracle (TEST INFRASTRUCTURE ONLY)."""
import ctypes
import os
import threading

import numpy as np

from . import build as _build

KIND_IDS = {"linear": 0, "vdp": 1, "mlp_tanh": 2, "mlp_silu": 3, "mds": 4, "chaboche": 5,
            "neuron": 6}

_lock = threading.Lock()
_lib = None


class _CModel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("h1", ctypes.c_int),
                ("h2", ctypes.c_int), ("per_series", ctypes.c_int)]


class Model:
    """Model description: kind in KIND_IDS, state size n, MLP hidden widths."""

    def __init__(self, kind, n, hidden=(0, 0), per_series=False):
        if kind not in KIND_IDS:
            raise ValueError(f"unknown model kind {kind!r}")
        self.kind, self.n = kind, int(n)
        self.hidden = (int(hidden[0]), int(hidden[1])) if hidden else (0, 0)
        self.per_series = bool(per_series)

    @classmethod
    def from_spec(cls, spec):
        return cls(spec["kind"], spec["n"], tuple(spec.get("hidden", (0, 0))),
                   spec.get("per_series", False))

    def c(self):
        return _CModel(KIND_IDS[self.kind], self.n, self.hidden[0], self.hidden[1],
                       int(self.per_series))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            lib = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            mp = ctypes.POINTER(_CModel)
            lib.tvo_param_count.argtypes = [mp]
            lib.tvo_param_count.restype = ctypes.c_int
            for name in ("tvo_rhs", "tvo_jac"):
                getattr(lib, name).argtypes = [mp, dp, dp, ctypes.c_double, dp]
                getattr(lib, name).restype = None
            lib.tvo_vjp_p.argtypes = [mp, dp, dp, ctypes.c_double, dp, ctypes.c_double, dp]
            lib.tvo_vjp_p.restype = None
            lib.tvo_forward.argtypes = [mp, ctypes.c_int, ctypes.c_int, dp, dp, ip, dp,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_int, dp, ip, ip]
            lib.tvo_forward.restype = ctypes.c_int
            lib.tvo_step_solves.argtypes = [mp, ctypes.c_int, ctypes.c_int, dp, ip, dp, dp,
                                            ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_int, dp, ip]
            lib.tvo_step_solves.restype = ctypes.c_int
            lib.tvo_adjoint.argtypes = [mp, ctypes.c_int, ctypes.c_int, dp, ip, dp, dp, dp,
                                        ctypes.c_int, dp, dp]
            lib.tvo_adjoint.restype = ctypes.c_int
            lib.tvo_forward_euler.argtypes = [mp, ctypes.c_int, ctypes.c_int, dp, dp, ip, dp,
                                              ctypes.c_int, dp, ip]
            lib.tvo_forward_euler.restype = ctypes.c_int
            lib.tvo_adjoint_euler.argtypes = [mp, ctypes.c_int, ctypes.c_int, dp, ip, dp, dp, dp,
                                              ctypes.c_int, dp, dp]
            lib.tvo_adjoint_euler.restype = ctypes.c_int
            lib.tvo_step_matrices.argtypes = [mp, ctypes.c_int, ctypes.c_int, dp, ip, dp, dp, dp]
            lib.tvo_step_matrices.restype = ctypes.c_int
            lib.tvo_max_threads.argtypes = []
            lib.tvo_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _dptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def max_threads():
    return _load().tvo_max_threads()


def param_count(model):
    return _load().tvo_param_count(ctypes.byref(model.c()))


def rhs(model, p, y, t=0.0):
    p, y = _f64(p), _f64(y)
    out = np.empty(model.n)
    _load().tvo_rhs(ctypes.byref(model.c()), _dptr(p), _dptr(y), float(t), _dptr(out))
    return out


def jac(model, p, y, t=0.0):
    p, y = _f64(p), _f64(y)
    out = np.empty((model.n, model.n))
    _load().tvo_jac(ctypes.byref(model.c()), _dptr(p), _dptr(y), float(t), _dptr(out))
    return out


def vjp_p(model, p, y, a, t=0.0, scale=1.0):
    p, y, a = _f64(p), _f64(y), _f64(a)
    out = np.zeros(param_count(model))
    _load().tvo_vjp_p(ctypes.byref(model.c()), _dptr(p), _dptr(y), float(t), _dptr(a),
                      float(scale), _dptr(out))
    return out


def forward(model, y0, times, params, lengths=None, tol_abs=1e-10, tol_rel=0.0, max_iter=50,
            nthreads=0):
    """Step-by-step backward-Euler Newton.  Returns (y [B][N+1][n], iters [B][N], status [B])."""
    y0, times, params = _f64(y0), _f64(times), _f64(params)
    B, n = y0.shape
    N = times.shape[1] - 1
    lens = None if lengths is None else np.ascontiguousarray(lengths, dtype=np.int32)
    y = np.empty((B, N + 1, n))
    iters = np.zeros((B, N), dtype=np.int32)
    status = np.zeros(B, dtype=np.int32)
    rc = _load().tvo_forward(ctypes.byref(model.c()), B, N, _dptr(y0), _dptr(times),
                             _iptr(lens), _dptr(params), float(tol_abs), float(tol_rel),
                             int(max_iter), int(nthreads), _dptr(y), _iptr(iters),
                             _iptr(status))
    if rc < 0:
        raise ValueError("tvo_forward rejected its arguments")
    return y, iters, status


def step_solves(model, times, params, y_prev, lengths=None, tol_abs=1e-13, tol_rel=0.0,
                max_iter=100, nthreads=0):
    """Every backward-Euler step solved on its own from the given previous states:
    out[b][k] solves step k from y_prev[b][k-1] (Sec. 2.2, the Newton of forward()).
    Returns (out [B][N+1][n], status [B])."""
    times, params, y_prev = _f64(times), _f64(params), _f64(y_prev)
    B, Np1, n = y_prev.shape
    lens = None if lengths is None else np.ascontiguousarray(lengths, dtype=np.int32)
    out = np.empty_like(y_prev)
    status = np.zeros(B, dtype=np.int32)
    rc = _load().tvo_step_solves(ctypes.byref(model.c()), B, Np1 - 1, _dptr(times), _iptr(lens),
                                 _dptr(params), _dptr(y_prev), float(tol_abs), float(tol_rel),
                                 int(max_iter), int(nthreads), _dptr(out), _iptr(status))
    if rc < 0:
        raise ValueError("tvo_step_solves rejected its arguments")
    return out, status


def adjoint(model, times, params, y, grad_out, lengths=None, nthreads=0):
    """Discrete adjoint.  Returns (dparams (shape of params), dy0 [B][n])."""
    times, params, y, grad_out = _f64(times), _f64(params), _f64(y), _f64(grad_out)
    B, Np1, n = y.shape
    lens = None if lengths is None else np.ascontiguousarray(lengths, dtype=np.int32)
    dparams = np.zeros_like(params)
    dy0 = np.zeros((B, n))
    rc = _load().tvo_adjoint(ctypes.byref(model.c()), B, Np1 - 1, _dptr(times), _iptr(lens),
                             _dptr(params), _dptr(y), _dptr(grad_out), int(nthreads),
                             _dptr(dparams), _dptr(dy0))
    if rc < 0:
        raise ValueError("tvo_adjoint rejected its arguments")
    return dparams, dy0


def forward_euler(model, y0, times, params, lengths=None, nthreads=0):
    """Forward Euler, step by step (Sec. 2.2, explicit methods).  Returns
    (y [B][N+1][n], status [B])."""
    y0, times, params = _f64(y0), _f64(times), _f64(params)
    B, n = y0.shape
    N = times.shape[1] - 1
    lens = None if lengths is None else np.ascontiguousarray(lengths, dtype=np.int32)
    y = np.empty((B, N + 1, n))
    status = np.zeros(B, dtype=np.int32)
    rc = _load().tvo_forward_euler(ctypes.byref(model.c()), B, N, _dptr(y0), _dptr(times),
                                   _iptr(lens), _dptr(params), int(nthreads), _dptr(y),
                                   _iptr(status))
    if rc < 0:
        raise ValueError("tvo_forward_euler rejected its arguments")
    return y, status


def adjoint_euler(model, times, params, y, grad_out, lengths=None, nthreads=0):
    """Discrete adjoint of the forward-Euler recursion.  Returns (dparams, dy0)."""
    times, params, y, grad_out = _f64(times), _f64(params), _f64(y), _f64(grad_out)
    B, Np1, n = y.shape
    lens = None if lengths is None else np.ascontiguousarray(lengths, dtype=np.int32)
    dparams = np.zeros_like(params)
    dy0 = np.zeros((B, n))
    rc = _load().tvo_adjoint_euler(ctypes.byref(model.c()), B, Np1 - 1, _dptr(times),
                                   _iptr(lens), _dptr(params), _dptr(y), _dptr(grad_out),
                                   int(nthreads), _dptr(dparams), _dptr(dy0))
    if rc < 0:
        raise ValueError("tvo_adjoint_euler rejected its arguments")
    return dparams, dy0


def step_matrices(model, times, params, y, lengths=None):
    """A_k = I - dt_k j(y_k) for every series and step: [B][N][n][n]."""
    times, params, y = _f64(times), _f64(params), _f64(y)
    B, Np1, n = y.shape
    lens = None if lengths is None else np.ascontiguousarray(lengths, dtype=np.int32)
    A = np.empty((B, Np1 - 1, n, n))
    rc = _load().tvo_step_matrices(ctypes.byref(model.c()), B, Np1 - 1, _dptr(times), _iptr(lens),
                                   _dptr(params), _dptr(y), _dptr(A))
    if rc < 0:
        raise ValueError("tvo_step_matrices rejected its arguments")
    return A


def forward_error_estimate(model, times, params, y, tol, lengths=None, trials=4, seed=0):
    """Relative forward error (per series) that Newton stopping at residual tol
    leaves in a backward-Euler trajectory: random per-step residuals r_k, uniform
    in [-tol, tol]^n, propagated through the linearised recursion
    d_k = A_k^-1 (d_{k-1} + r_k); the largest max_k |d_k| / max_k |y_k| over trials."""
    A = step_matrices(model, times, params, y, lengths)
    B, N, n, _ = A.shape
    g = np.random.default_rng(seed)
    scale = np.maximum(np.abs(y).max(axis=(1, 2)), 1e-300)
    est = np.zeros(B)
    for _ in range(trials):
        d = np.zeros((B, n))
        dmax = np.zeros(B)
        r = g.uniform(-tol, tol, (B, N, n))
        for k in range(N):
            d = np.linalg.solve(A[:, k], (d + r[:, k])[..., None])[..., 0]
            dmax = np.maximum(dmax, np.abs(d).max(axis=1))
        est = np.maximum(est, dmax / scale)
    return est
