"""tvi_adjoint_noalloc: the adjoint for callers that cannot allocate device memory.

Its scratch (per-series partial gradients of shared parameters) is a fixed
array inside the library instead of a caller workspace.  The GPU test calls it
through the C ABI twice in a row and compares both results with tvi_adjoint on
the same inputs; the second call also shows that what the first left in the
shared array does not leak into the next result.  This file is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import workloads


def _buf(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.mark.gpu
def test_noalloc_adjoint_matches_workspace_adjoint_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08649_gb300 import Model, Options, _lib, adjoint, build
    build.build()
    lib = _lib.load()
    # shared parameters (one A for all series) so the fixed scratch is used
    w = workloads.linear_stiff(B=16, N=1000)
    m = Model.from_spec(w["spec"])
    g1 = workloads.random_grad_out(501, 16, 1000, 4)
    g2 = workloads.random_grad_out(502, 16, 1000, 4)
    times, params = _buf(w["times"], torch.float64), _buf(w["params"], torch.float64)
    # any fixed trajectory works: the adjoint is linear in grad_out given y
    y = _buf(np.cumsum(workloads.random_grad_out(503, 16, 1000, 4), axis=1) * 1e-2,
             torch.float64)
    for precision, tol in (("fp64", 1e-12), ("fp32", 1e-9)):
        o = Options(chunk=50, precision=precision, adjoint_refine=2)
        for g in (g1, g2):  # two calls in a row
            gd = _buf(g, torch.float64)
            ref_dp, ref_dy0 = adjoint(m, o, times, params, y, gd)
            dp = torch.empty_like(ref_dp)
            dy0 = torch.empty_like(ref_dy0)
            rc = lib.tvi_adjoint_noalloc(ctypes.byref(m.c()), ctypes.byref(o.c()), 16, 1000,
                                         ctypes.c_void_p(times.data_ptr()), None,
                                         ctypes.c_void_p(params.data_ptr()),
                                         ctypes.c_void_p(y.data_ptr()),
                                         ctypes.c_void_p(gd.data_ptr()),
                                         ctypes.c_void_p(dp.data_ptr()),
                                         ctypes.c_void_p(dy0.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert rc == 0, _lib.last_error()
            torch.cuda.synchronize()
            a, b = dp.cpu().numpy(), ref_dp.cpu().numpy()
            assert np.abs(a - b).max() <= tol * np.abs(b).max(), precision
            a, b = dy0.cpu().numpy(), ref_dy0.cpu().numpy()
            assert np.abs(a - b).max() <= tol * np.abs(b).max(), precision


@pytest.mark.gpu
def test_noalloc_user_model_shared_parameters_twice():
    """A run-time compiled user model (linear h = A y, n = 3, one A shared by all
    series) takes the same scratch path: its adjoint kernel writes the per-series
    partial gradients into the fixed array and the series-ordered sum reads them.
    Two calls in a row, each against tvi_adjoint on the same inputs."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_08649_gb300 import Options, UserModel, _lib, adjoint, build
    from paper_2310_08649_gb300.user_sources import LINEAR
    build.build()
    lib = _lib.load()
    B, N, n = 12, 600, 3
    user = UserModel(n, n * n, LINEAR)
    m = user.model(per_series=False)
    g = np.random.default_rng(504)
    A = -np.eye(n) * 20.0 + g.standard_normal((n, n))
    times = _buf(workloads.uniform_times(B, N, 1.0), torch.float64)
    params = _buf(A.reshape(-1), torch.float64)
    y = _buf(g.standard_normal((B, N + 1, n)), torch.float64)
    for precision, tol in (("fp64", 1e-12), ("fp32", 1e-9)):
        o = Options(chunk=64, precision=precision, adjoint_refine=2)
        for seed in (505, 506):  # two calls in a row
            gd = _buf(workloads.random_grad_out(seed, B, N, n), torch.float64)
            ref_dp, ref_dy0 = adjoint(m, o, times, params, y, gd)
            dp = torch.empty_like(ref_dp)
            dy0 = torch.empty_like(ref_dy0)
            rc = lib.tvi_adjoint_noalloc(ctypes.byref(m.c()), ctypes.byref(o.c()), B, N,
                                         ctypes.c_void_p(times.data_ptr()), None,
                                         ctypes.c_void_p(params.data_ptr()),
                                         ctypes.c_void_p(y.data_ptr()),
                                         ctypes.c_void_p(gd.data_ptr()),
                                         ctypes.c_void_p(dp.data_ptr()),
                                         ctypes.c_void_p(dy0.data_ptr()),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert rc == 0, _lib.last_error()
            torch.cuda.synchronize()
            a, b = dp.cpu().numpy(), ref_dp.cpu().numpy()
            assert np.abs(a - b).max() <= tol * np.abs(b).max(), precision
            a, b = dy0.cpu().numpy(), ref_dy0.cpu().numpy()
            assert np.abs(a - b).max() <= tol * np.abs(b).max(), precision
    user.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    """B * P above the fixed 524,288-double scratch is refused before any GPU work."""
    from paper_2310_08649_gb300 import Model, Options, _lib, build
    build.build()
    lib = _lib.load()
    m = Model("linear", 4)  # P = 16, shared
    vp = ctypes.c_void_p(16)  # never dereferenced: the call fails its size check first
    rc = lib.tvi_adjoint_noalloc(ctypes.byref(m.c()), ctypes.byref(Options(chunk=8).c()),
                                 524288 // 16 + 1, 10, vp, None, vp, vp, vp, vp, None, None)
    assert rc == -1
    assert "scratch" in lib.tvi_last_error().decode()
