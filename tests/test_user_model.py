"""User models compiled at run time (tvi_user_model_create / _prepare /
_destroy), on the host: NVRTC compiles the user's functions together with the
fused solver kernels for sm_103a without a GPU, so the interface checks, the
compiler-log reporting and the full kernel compile are tested here."""
import ctypes

import pytest

from paper_2310_08649_gb300.user_sources import LINEAR, MDS, VDP, VDP_FP64_JAC, \
    mds_param_count, mlp_param_count, mlp_tanh

tvi = pytest.importorskip("paper_2310_08649_gb300")
from paper_2310_08649_gb300 import _lib  # noqa: E402

EINVAL, EUNSUPPORTED = -1, -7


@pytest.fixture(scope="module")
def lib():
    from paper_2310_08649_gb300 import build
    build.build()
    lib = _lib.load()
    h = ctypes.c_void_p()
    rc = lib.tvi_user_model_create(2, 1, VDP.encode(), ctypes.byref(h))
    if rc == EUNSUPPORTED and "could not be loaded" in _lib.last_error():
        pytest.skip("NVRTC is not available: " + _lib.last_error())
    assert rc == 0, _lib.last_error()
    lib.tvi_user_model_destroy(h)
    return lib


def create(lib, n, P, src):
    h = ctypes.c_void_p()
    rc = lib.tvi_user_model_create(n, P, src.encode() if src is not None else None,
                                   ctypes.byref(h))
    return rc, h


def test_create_and_param_count(lib):
    u = tvi.UserModel(2, 1, VDP)
    assert u.model().param_count() == 1
    m = _lib.TviModel(4, 3, 0, 0, 1, u.handle)  # n differs from the user model's
    assert lib.tvi_param_count(ctypes.byref(m)) == -1
    m = _lib.TviModel(4, 2, 0, 0, 1, None)      # no user model
    assert lib.tvi_param_count(ctypes.byref(m)) == -1
    u.close()
    assert u.handle is None


def test_compile_error_reports_the_users_line(lib):
    bad = VDP.replace("h[0] = y[1];", "h[0] = undefined_name;")  # line 4 of the source
    rc, _ = create(lib, 2, 1, bad)
    assert rc == EINVAL
    msg = _lib.last_error()
    assert "does not compile" in msg and "user_model.cu(4)" in msg, msg
    assert "undefined_name" in msg


def test_missing_function_is_rejected(lib):
    no_vjp = VDP[:VDP.index("__device__ void tvi_vjp_p")]
    rc, _ = create(lib, 2, 1, no_vjp)
    assert rc == EINVAL and "tvi_vjp_p" in _lib.last_error()


@pytest.mark.parametrize("n,P", [(0, 1), (41, 1), (2, 0), (2, 33), (5, 161), (-1, -1)])
def test_bad_sizes(lib, n, P):
    rc, h = create(lib, n, P, VDP)
    assert rc == EINVAL and h.value is None


def test_null_arguments(lib):
    rc, _ = create(lib, 2, 1, None)
    assert rc == EINVAL
    assert lib.tvi_user_model_create(2, 1, VDP.encode(), None) == EINVAL
    assert lib.tvi_user_model_prepare(None, 0) == EINVAL
    lib.tvi_user_model_destroy(None)  # ignored


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_prepare_compiles_every_tiling(lib, precision):
    """Every steps-per-thread tiling of the forward and adjoint kernels compiles
    for a nonlinear model with shared MLP parameters (n = 3, P = 23) and for a
    linear model of the largest state size (n = 4, P = 16)."""
    u = tvi.UserModel(3, mlp_param_count(3, 2, 2), mlp_tanh(2, 2))
    u.prepare(precision)
    u.close()
    v = tvi.UserModel(4, 16, LINEAR)
    v.prepare(precision)
    v.close()


@pytest.mark.parametrize("src", [VDP, VDP_FP64_JAC], ids=["template_jac", "fp64_jac"])
def test_prepare_both_jacobian_forms(lib, src):
    """tvi_jac as a template over the block type, or as a plain FP64 function."""
    u = tvi.UserModel(2, 1, src)
    u.prepare("fp32")
    u.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_prepare_large_state_route(lib, precision):
    """n > 4 compiles the large-state kernels: a time-dependent model with a
    template Jacobian (mass-damper-spring, n = 20) and one with an FP64 Jacobian
    and a padded width (linear, n = 5)."""
    u = tvi.UserModel(20, mds_param_count(10), MDS)
    u.prepare(precision)
    u.close()
    v = tvi.UserModel(5, 25, LINEAR)
    v.prepare(precision)
    v.close()


def test_large_route_takes_64_parameters(lib):
    """Above n = 4 up to 64 parameters (read from memory past 32): four coupled
    neurons, 61 parameters."""
    from paper_2310_08649_gb300.user_sources import NEURON, neuron_param_count
    u = tvi.UserModel(16, neuron_param_count(4), NEURON)
    assert u.model().param_count() == 61
    u.prepare("fp32")
    u.close()


def test_prepare_rejects_bf16(lib):
    u = tvi.UserModel(1, 1, LINEAR)
    with pytest.raises(_lib.TviError) as e:
        u.prepare("bf16")
    assert e.value.code == EUNSUPPORTED
    u.close()


def test_large_route_host_checks(lib):
    """Without a GPU: the workspace of a large-state user model grows with the
    chunk; BF16 blocks and the allocation-free adjoint are rejected on that route
    before anything is launched, and forward Euler passes the scheme check."""
    u = tvi.UserModel(20, mds_param_count(10), MDS)
    m = u.model(per_series=True).c()
    o = _lib.TviOptions()
    lib.tvi_default_options(ctypes.byref(o))
    o.precision = 1
    o.chunk = 100
    w100 = lib.tvi_workspace_bytes(ctypes.byref(m), ctypes.byref(o), 8, 1000)
    o.chunk = 1000
    w1000 = lib.tvi_workspace_bytes(ctypes.byref(m), ctypes.byref(o), 8, 1000)
    assert 0 < w100 < w1000
    # 8 series x 1000 steps x 20 x 20 FP32 blocks at least
    assert w1000 >= 8 * 1000 * 20 * 20 * 4
    o.scheme = 1  # forward Euler: accepted, then the NULL arrays are the error
    rc = lib.tvi_integrate(ctypes.byref(m), ctypes.byref(o), 8, 1000, None, None, None, None,
                           None, None, None, None, 0, None)
    assert rc == EINVAL and "must not be NULL" in _lib.last_error()
    o.scheme = 0
    o.precision = 2  # BF16
    rc = lib.tvi_integrate(ctypes.byref(m), ctypes.byref(o), 8, 1000, None, None, None, None,
                           None, None, None, None, 0, None)
    assert rc == EUNSUPPORTED
    o.precision = 1
    rc = lib.tvi_adjoint_noalloc(ctypes.byref(m), ctypes.byref(o), 8, 1000, None, None, None,
                                 None, None, None, None, None)
    assert rc == EUNSUPPORTED and "noalloc" in _lib.last_error()
    u.close()
