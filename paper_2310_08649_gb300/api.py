"""Python API over the C ABI: integrate / adjoint on torch CUDA tensors, and an
autograd Function whose backward is the adjoint pass.

PyTorch supplies device memory and the stream; the computation is the CUDA
library's.  Inputs must already be CUDA float64 (int32 for lengths) tensors:
the binding checks and never moves data to the host.
"""
import ctypes
from dataclasses import dataclass, field

import torch

from . import _lib


@dataclass(frozen=True)
class Model:
    """kind: 'linear' | 'vdp' | 'mlp_tanh' | 'mlp_silu' | 'user'; n: state size;
    hidden: MLP hidden widths; per_series: one parameter vector per series;
    user: the UserModel of kind 'user' (UserModel.model() builds this)."""
    kind: str
    n: int
    hidden: tuple = (0, 0)
    per_series: bool = False
    user: object = None

    @classmethod
    def from_spec(cls, spec):
        return cls(spec["kind"], int(spec["n"]), tuple(spec.get("hidden", (0, 0))),
                   bool(spec.get("per_series", False)))

    def c(self):
        if self.kind not in _lib.MODEL_KINDS:
            raise ValueError(f"unknown model kind {self.kind!r}")
        h = tuple(self.hidden) if self.hidden else (0, 0)
        handle = self.user.handle if self.user is not None else None
        return _lib.TviModel(_lib.MODEL_KINDS[self.kind], self.n, h[0], h[1],
                             int(self.per_series), handle)

    def param_count(self):
        return _lib.load().tvi_param_count(ctypes.byref(self.c()))


class UserModel:
    """A small-state model given as CUDA C++ device source (tvi_user_model_create):
    `source` defines tvi_rhs(y, p, h), tvi_jac(y, p, J) and tvi_vjp_p(y, p, a, g)
    over FP64 pointers, with TVI_N = n and TVI_P = P defined.  The source is
    compile-checked here (no GPU needed); the solver kernels compile on first
    use, or all at once with prepare(precision)."""

    def __init__(self, n, P, source):
        lib = _lib.load()
        h = ctypes.c_void_p()
        rc = lib.tvi_user_model_create(int(n), int(P), source.encode(), ctypes.byref(h))
        if rc != 0:
            raise _lib.TviError(rc, _lib.last_error())
        self.n, self.P, self.handle = int(n), int(P), h.value
        self._lib = lib

    def prepare(self, precision="fp64"):
        if precision not in _lib.PRECISIONS:
            raise ValueError(f"unknown precision {precision!r}")
        rc = self._lib.tvi_user_model_prepare(self.handle, _lib.PRECISIONS[precision])
        if rc != 0:
            raise _lib.TviError(rc, _lib.last_error())
        return self

    def model(self, per_series=True):
        return Model("user", self.n, per_series=per_series, user=self)

    def close(self):
        """Unload the kernels; call after the work that uses them has completed."""
        if self.handle:
            self._lib.tvi_user_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Options:
    """Solver options (tvi_options).  precision: 'fp64' | 'fp32' | 'bf16';
    scheme: 'backward' | 'forward' Euler."""
    chunk: int = 1
    tol_abs: float = 1e-8
    tol_rel: float = 0.0
    max_iter: int = 50
    precision: str = "fp64"
    retry_halving: bool = True
    adjoint_refine: int = 2
    rows_per_thread: int = 0
    sync_status: bool = True
    predictor: object = None      # packed predictor: CUDA float32 tensor, or None
    predictor_chunk: int = 0
    predictor_hidden: int = 0
    scheme: str = "backward"      # 'backward' | 'forward' (Euler)

    def c(self):
        if self.precision not in _lib.PRECISIONS:
            raise ValueError(f"unknown precision {self.precision!r}")
        if self.scheme not in _lib.SCHEMES:
            raise ValueError(f"unknown scheme {self.scheme!r}")
        pred = None
        if self.predictor is not None:
            _check(self.predictor, "predictor", torch.float32, tuple(self.predictor.shape))
            pred = self.predictor.data_ptr()
        return _lib.TviOptions(int(self.chunk), float(self.tol_abs), float(self.tol_rel),
                               int(self.max_iter), _lib.PRECISIONS[self.precision],
                               int(bool(self.retry_halving)), int(self.adjoint_refine),
                               int(self.rows_per_thread), int(bool(self.sync_status)), pred,
                               int(self.predictor_chunk), int(self.predictor_hidden),
                               _lib.SCHEMES[self.scheme])


def _check(t, name, dtype, shape, allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (no host fallback exists)")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _param_shape(model, B):
    P = model.param_count()
    if P < 0:
        raise ValueError(f"bad model {model}")
    return (B, P) if model.per_series else (P,)


def workspace_bytes(model, opts, B, N):
    return _lib.load().tvi_workspace_bytes(ctypes.byref(model.c()), ctypes.byref(opts.c()), B, N)


def effective_chunk(model, opts, N):
    """Steps one chunk attempt holds (tvi_effective_chunk): the requested chunk,
    at most N, and at most 1024 on the small-state engine."""
    return _lib.load().tvi_effective_chunk(ctypes.byref(model.c()), ctypes.byref(opts.c()), N)


def make_workspace(model, opts, B, N, device):
    return torch.empty(max(workspace_bytes(model, opts, B, N), 256), dtype=torch.uint8,
                       device=device)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def integrate(model, opts, y0, times, params, lengths=None, y_out=None, stats=None,
              series_status=None, workspace=None, stream=None, raise_on_status=True):
    """Chunked backward-Euler integration (tvi_integrate).

    Returns (y [B][N+1][n], stats [B][6] int32, series_status [B] int32, rc).  With
    raise_on_status=False the per-series failure codes (TVI_ENOTCONV, TVI_ENONFINITE,
    TVI_ETIMEOUT) are returned in rc instead of raised."""
    lib = _lib.load()
    B, n = y0.shape
    N = times.shape[1] - 1
    dev = y0.device
    _check(y0, "y0", torch.float64, (B, model.n))
    _check(times, "times", torch.float64, (B, N + 1))
    _check(params, "params", torch.float64, _param_shape(model, B))
    _check(lengths, "lengths", torch.int32, (B,), allow_none=True)
    if y_out is None:
        y_out = torch.empty((B, N + 1, n), dtype=torch.float64, device=dev)
    _check(y_out, "y_out", torch.float64, (B, N + 1, n))
    if stats is None:
        stats = torch.empty((B, _lib.STATS), dtype=torch.int32, device=dev)
    if series_status is None:
        series_status = torch.empty((B,), dtype=torch.int32, device=dev)
    if workspace is None:
        workspace = make_workspace(model, opts, B, N, dev)
    rc = lib.tvi_integrate(ctypes.byref(model.c()), ctypes.byref(opts.c()), B, N, _ptr(y0),
                           _ptr(times), _ptr(lengths), _ptr(params), _ptr(y_out), _ptr(stats),
                           _ptr(series_status), _ptr(workspace), workspace.numel(),
                           _stream(stream))
    status_codes = (_lib.TVI_ENOTCONV, _lib.TVI_ENONFINITE, _lib.TVI_ETIMEOUT)
    if rc != 0 and (raise_on_status or rc not in status_codes):
        raise _lib.TviError(rc, _lib.last_error())
    return y_out, stats, series_status, rc


def adjoint(model, opts, times, params, y, grad_out, lengths=None, dparams=None, dy0=None,
            workspace=None, stream=None):
    """Discrete adjoint (tvi_adjoint).  Returns (dparams, dy0)."""
    lib = _lib.load()
    B, Np1, n = y.shape
    N = Np1 - 1
    dev = y.device
    _check(times, "times", torch.float64, (B, N + 1))
    _check(params, "params", torch.float64, _param_shape(model, B))
    _check(y, "y", torch.float64, (B, N + 1, model.n))
    _check(grad_out, "grad_out", torch.float64, (B, N + 1, model.n))
    _check(lengths, "lengths", torch.int32, (B,), allow_none=True)
    if dparams is None:
        dparams = torch.empty(_param_shape(model, B), dtype=torch.float64, device=dev)
    if dy0 is None:
        dy0 = torch.empty((B, n), dtype=torch.float64, device=dev)
    if workspace is None:
        workspace = make_workspace(model, opts, B, N, dev)
    rc = lib.tvi_adjoint(ctypes.byref(model.c()), ctypes.byref(opts.c()), B, N, _ptr(times),
                         _ptr(lengths), _ptr(params), _ptr(y), _ptr(grad_out), _ptr(dparams),
                         _ptr(dy0), _ptr(workspace), workspace.numel(), _stream(stream))
    if rc != 0:
        raise _lib.TviError(rc, _lib.last_error())
    return dparams, dy0


def adjoint_noalloc(model, opts, times, params, y, grad_out, lengths=None, dparams=None,
                    dy0=None, stream=None):
    """tvi_adjoint_noalloc: the adjoint without a workspace, for callers that cannot
    allocate device memory (its scratch is a fixed array inside the library).
    Pass dparams and dy0 to keep the call itself free of allocations.
    Returns (dparams, dy0)."""
    lib = _lib.load()
    B, Np1, n = y.shape
    N = Np1 - 1
    dev = y.device
    _check(times, "times", torch.float64, (B, N + 1))
    _check(params, "params", torch.float64, _param_shape(model, B))
    _check(y, "y", torch.float64, (B, N + 1, model.n))
    _check(grad_out, "grad_out", torch.float64, (B, N + 1, model.n))
    _check(lengths, "lengths", torch.int32, (B,), allow_none=True)
    if dparams is None:
        dparams = torch.empty(_param_shape(model, B), dtype=torch.float64, device=dev)
    if dy0 is None:
        dy0 = torch.empty((B, n), dtype=torch.float64, device=dev)
    rc = lib.tvi_adjoint_noalloc(ctypes.byref(model.c()), ctypes.byref(opts.c()), B, N,
                                 _ptr(times), _ptr(lengths), _ptr(params), _ptr(y),
                                 _ptr(grad_out), _ptr(dparams), _ptr(dy0), _stream(stream))
    if rc != 0:
        raise _lib.TviError(rc, _lib.last_error())
    return dparams, dy0


class Integrate(torch.autograd.Function):
    """y = Integrate.apply(y0, params, times, model, opts, lengths): forward is
    tvi_integrate, backward is tvi_adjoint (gradients w.r.t. y0 and params)."""

    @staticmethod
    def forward(ctx, y0, params, times, model, opts, lengths=None):
        times, params = times.contiguous(), params.contiguous()
        y, _, _, _ = integrate(model, opts, y0.contiguous(), times, params, lengths)
        ctx.model, ctx.opts = model, opts
        ctx.save_for_backward(times, params, y, lengths if lengths is not None else torch.empty(0))
        ctx.has_lengths = lengths is not None
        return y

    @staticmethod
    def backward(ctx, grad_y):
        times, params, y, lengths = ctx.saved_tensors
        dparams, dy0 = adjoint(ctx.model, ctx.opts, times, params, y, grad_y.contiguous(),
                               lengths if ctx.has_lengths else None)
        return dy0, dparams, None, None, None, None


def odeint(model, opts, y0, params, times, lengths=None):
    """Differentiable integration: returns y [B][N+1][n] with adjoint gradients."""
    return Integrate.apply(y0, params, times, model, opts, lengths)
