"""GPU parity of the forward-Euler scheme (chunked, Newton on the explicit chunk
system) with the step-by-step forward-Euler oracle, through the C ABI.

The explicit recursion has one solution per series; Newton on the chunk system
is stopped at a tight tolerance (1e-12), so the GPU trajectory is that solution
up to residuals of that size, which the recursion may amplify (van der Pol's
growing phase).  Gates per series: max(1e-10 relative with FP64 blocks, 1e-5 with
FP32 blocks, 10 x the propagated forward-error estimate); and every step against
the explicit step from the GPU's own previous state at 1e-10 (parity_helpers), a
check no conditioning enters.  Both adjoints run on the oracle's trajectory and
are compared directly.
"""
import numpy as np
import pytest

import workloads
from oracle import Model as OModel
from parity_helpers import STEP_GATE, fe_step_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module")
def tvi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2310_08649_gb300 as tvi
    from paper_2310_08649_gb300 import build
    build.build()
    return tvi


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def relerr_series(a, b):
    return np.abs(a - b).max(axis=(1, 2)) / np.maximum(np.abs(b).max(axis=(1, 2)), 1e-300)


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def forward(tvi, w, chunk, precision, lengths=None):
    m = tvi.Model.from_spec(w["spec"])
    o = tvi.Options(chunk=chunk, tol_abs=1e-12, precision=precision, scheme="forward",
                    max_iter=60)
    lens = None if lengths is None else dev(lengths, torch.int32)
    y, stats, st, rc = tvi.integrate(m, o, dev(w["y0"]), dev(w["times"]), dev(w["params"]), lens,
                                     raise_on_status=False)
    torch.cuda.synchronize()
    return y.cpu().numpy(), st.cpu().numpy(), rc


def adjoint(tvi, w, chunk, precision, y, g, lengths=None):
    m = tvi.Model.from_spec(w["spec"])
    o = tvi.Options(chunk=chunk, precision=precision, scheme="forward", adjoint_refine=2)
    lens = None if lengths is None else dev(lengths, torch.int32)
    dp, dy0 = tvi.adjoint(m, o, dev(w["times"]), dev(w["params"]), dev(y), dev(g), lens)
    torch.cuda.synchronize()
    return dp.cpu().numpy(), dy0.cpu().numpy()


def fe_error_estimate(oracle_lib, m, w, y, tol, trials=4, seed=0):
    """Per-series forward error that per-step residuals of size tol leave after
    propagation through the linearised forward-Euler recursion
    delta_k = (I + dt_k j(y_{k-1})) delta_{k-1} + r_k, r_k uniform in [-tol, tol]^n,
    relative to max_k |y_k| (the conditioning of the explicit recursion)."""
    B, Np1, n = y.shape
    shifted = np.concatenate([y[:, :1], y[:, :-1]], axis=1)  # row k holds y_{k-1}
    A = oracle_lib.step_matrices(m, w["times"], w["params"], shifted)  # I - dt_k j(y_{k-1})
    Bk = 2.0 * np.eye(n)[None, None] - A
    g = np.random.default_rng(seed)
    d = np.zeros((B, trials, n))
    worst = np.zeros(B)
    for k in range(Np1 - 1):
        d = np.einsum("bij,btj->bti", Bk[:, k], d) + g.uniform(-tol, tol, d.shape)
        worst = np.maximum(worst, np.abs(d).max(axis=(1, 2)))
    return worst / np.abs(y).max(axis=(1, 2))


def workloads_fe():
    # linear: eigenvalues up to 100 at dt = 1/500 (1 - dt lam in (0, 1));
    # van der Pol: mu in [10, 100] with spans short enough that mu dt <= 0.2;
    # neural ODEs on the MLP engine: tanh n = 4 and n = 16 (the n = 16 blocks and
    # the FP32 backward passes of the mixed-precision adjoint), SiLU n = 8
    return {"linear": workloads.linear_stiff(B=8, N=500, lam_decades=(0.0, 2.0)),
            "vdp": workloads.vdp(B=16, N=2000, seed=51, mu_dt_max=0.2, mu_decades=(1.0, 2.0)),
            "mlp4": workloads.mlp_ode(B=4, N=300, n=4, hidden=(8, 12), t_end=3.0, seed=54),
            "mlp16": workloads.mlp_ode(B=4, N=400, n=16, hidden=(64, 64), t_end=4.0, seed=55),
            "silu8": workloads.mlp_ode(B=3, N=300, n=8, hidden=(16, 8), act="silu", t_end=3.0,
                                       seed=56)}


@pytest.mark.parametrize("which", ["linear", "vdp", "mlp4", "mlp16", "silu8"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("chunk", [1, 7, 64, 500])
def test_forward_euler_forward_and_adjoint(tvi, oracle_lib, which, precision, chunk):
    w = workloads_fe()[which]
    m = OModel.from_spec(w["spec"])
    ref, st = oracle_lib.forward_euler(m, w["y0"], w["times"], w["params"])
    assert not st.any()
    y, status, rc = forward(tvi, w, chunk, precision)
    assert rc == 0 and not status.any()
    est = fe_error_estimate(oracle_lib, m, w, ref, 1e-12)
    err = relerr_series(y, ref)
    bad = np.nonzero(err > np.maximum(GATE[precision], 10.0 * est))[0]
    assert bad.size == 0, (bad, err[bad], est[bad])
    assert fe_step_errors(oracle_lib, m, w, y).max() <= STEP_GATE
    B, Np1, n = ref.shape
    g = workloads.random_grad_out(81, B, Np1 - 1, n)
    dp_ref, dy0_ref = oracle_lib.adjoint_euler(m, w["times"], w["params"], ref, g)
    dp, dy0 = adjoint(tvi, w, chunk, precision, ref, g)
    assert relerr(dp, dp_ref) <= GATE[precision]
    assert relerr(dy0, dy0_ref) <= GATE[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_forward_euler_padded_lengths(tvi, oracle_lib, precision):
    w = workloads.vdp(B=4, N=600, seed=52, mu_dt_max=0.2, mu_decades=(1.0, 2.0))
    m = OModel.from_spec(w["spec"])
    lens = np.array([600, 1, 0, 333], dtype=np.int32)
    ref, st = oracle_lib.forward_euler(m, w["y0"], w["times"], w["params"], lengths=lens)
    y, status, rc = forward(tvi, w, 64, precision, lengths=lens)
    assert rc == 0 and not status.any()
    for b, L in enumerate(lens):
        assert np.all(y[b, L + 1:] == y[b, L])
    est = fe_error_estimate(oracle_lib, m, dict(w, times=_padded_times(w["times"], lens)), ref,
                            1e-12)
    assert np.all(relerr_series(y, ref) <= np.maximum(GATE[precision], 10.0 * est))
    assert fe_step_errors(oracle_lib, m, w, y, lengths=lens).max() <= STEP_GATE
    g = workloads.random_grad_out(82, 4, 600, 2)
    for b, L in enumerate(lens):
        g[b, L + 1:] = 0.0
    dp_ref, dy0_ref = oracle_lib.adjoint_euler(m, w["times"], w["params"], ref, g, lengths=lens)
    dp, dy0 = adjoint(tvi, w, 64, precision, ref, g, lengths=lens)
    assert relerr(dp, dp_ref) <= GATE[precision]
    assert relerr(dy0, dy0_ref) <= GATE[precision]


def _padded_times(times, lens):
    """Times whose steps past each length have dt = 0 (padding)."""
    t = times.copy()
    for b, L in enumerate(lens):
        t[b, L + 1:] = t[b, L]
    return t


def test_forward_euler_rejections(tvi):
    """Forward Euler runs without tensor-core (BF16) blocks."""
    import paper_2310_08649_gb300._lib as L
    w = workloads.mlp_ode(B=2, N=20, n=16, hidden=(64, 64), seed=53)
    m = tvi.Model.from_spec(w["spec"])
    with pytest.raises(L.TviError) as e:
        tvi.integrate(m, tvi.Options(chunk=5, scheme="forward", precision="bf16"), dev(w["y0"]),
                      dev(w["times"]), dev(w["params"]))
    assert e.value.code == -7


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_forward_euler_mlp_padded_lengths(tvi, oracle_lib, precision):
    """Forward Euler on the MLP engine with per-series lengths padded into one launch
    (dt = 0 past each length): padded steps keep the state, and trajectory and
    gradients match the oracle's explicit recursion and its adjoint."""
    w = workloads.mlp_ode(B=4, N=240, n=8, hidden=(16, 16), t_end=2.5, seed=57,
                          lengths_range=(1, 240))
    lens = w["lengths"]
    lens[1] = 0
    m = OModel.from_spec(w["spec"])
    ref, st = oracle_lib.forward_euler(m, w["y0"], w["times"], w["params"], lengths=lens)
    assert not st.any()
    y, status, rc = forward(tvi, w, 50, precision, lengths=lens)
    assert rc == 0 and not status.any()
    for b, L in enumerate(lens):
        assert np.all(y[b, L + 1:] == y[b, L])
    est = fe_error_estimate(oracle_lib, m, dict(w, times=_padded_times(w["times"], lens)), ref,
                            1e-12)
    assert np.all(relerr_series(y, ref) <= np.maximum(GATE[precision], 10.0 * est))
    assert fe_step_errors(oracle_lib, m, w, y, lengths=lens).max() <= STEP_GATE
    g = workloads.random_grad_out(83, 4, 240, 8)
    for b, L in enumerate(lens):
        g[b, L + 1:] = 0.0
    dp_ref, dy0_ref = oracle_lib.adjoint_euler(m, w["times"], w["params"], ref, g, lengths=lens)
    dp, dy0 = adjoint(tvi, w, 50, precision, ref, g, lengths=lens)
    assert relerr(dp, dp_ref) <= GATE[precision]
    assert relerr(dy0, dy0_ref) <= GATE[precision]
