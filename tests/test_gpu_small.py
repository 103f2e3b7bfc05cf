"""GPU parity of the fused small-state path (linear n=4, van der Pol n=2) with the
CPU FP64 oracle, through the C ABI.

Error metric (per series): max_k |y_gpu - y_ref|_inf / max_k |y_ref|_inf.
Gates: 1e-10 relative with FP64 blocks, 1e-5 relative with FP32 blocks.

Van der Pol trajectories pass through steep relaxation jumps, so two correct
solvers that each stop Newton at residual tol can differ by much more than
tol: the forward error is the problem's conditioning times the backward error.
For each series the test estimates that forward error from the oracle's
trajectory (random residuals of size tol propagated through the linearised
backward-Euler recursion, oracle.forward_error_estimate) and accepts
max(gate, 10 x estimate).  It also checks every step of every series on its
own, conditioning-free: the oracle's one-step Newton solve from the GPU's own
y_{k-1} must match the GPU's y_k within 1e-10 relative (parity_helpers).
"""
import numpy as np
import pytest

import workloads
from oracle import Model as OModel
from parity_helpers import STEP_GATE, be_step_errors

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


def run_gpu(tvi, w, chunk, precision, tol, lengths=None, **kw):
    m = tvi.Model.from_spec(w["spec"])
    o = tvi.Options(chunk=chunk, tol_abs=tol, precision=precision, **kw)
    lens = None if lengths is None else dev(lengths, torch.int32)
    y, stats, st, rc = tvi.integrate(m, o, dev(w["y0"]), dev(w["times"]), dev(w["params"]), lens,
                                     raise_on_status=False)
    torch.cuda.synchronize()
    return y.cpu().numpy(), stats.cpu().numpy(), st.cpu().numpy(), rc


# ---------------------------------------------------------------------------
# Linear stiff system (well conditioned: kappa(I - dt A) <= 11): strict gates.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("chunk", [50, 1, 7, 64, 1000, 1500])
def test_linear_forward_parity(tvi, oracle_lib, precision, chunk):
    w = workloads.linear_stiff()
    m = OModel.from_spec(w["spec"])
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-13)
    assert not st.any()
    y, stats, status, rc = run_gpu(tvi, w, chunk, precision, 1e-13)
    assert rc == 0 and not status.any()
    assert np.array_equal(y[:, 0], w["y0"])
    assert relerr_series(y, ref).max() <= GATE[precision]


def test_linear_whole_range_chunks(tvi, oracle_lib):
    """chunk >= N (a single chunk, and the 1024-step on-chip limit) on a system
    whose chunked equations are linear, so Newton converges from any guess."""
    w = workloads.linear_stiff(B=3, N=3000)
    m = OModel.from_spec(w["spec"])
    ref, _, _ = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-13)
    for chunk in [3000, 4096, 1024, 1023]:
        y, stats, status, rc = run_gpu(tvi, w, chunk, "fp64", 1e-13)
        assert rc == 0 and relerr_series(y, ref).max() <= 1e-10, chunk


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("chunk", [50, 1, 333])
def test_linear_adjoint_parity(tvi, oracle_lib, precision, chunk):
    w = workloads.linear_stiff(B=16, N=1000)
    m = OModel.from_spec(w["spec"])
    ref, _, _ = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-13)
    g = workloads.random_grad_out(77, 16, 1000, 4)
    dA, dy0 = oracle_lib.adjoint(m, w["times"], w["params"], ref, g)
    tm = tvi.Model.from_spec(w["spec"])
    o = tvi.Options(chunk=chunk, precision=precision, adjoint_refine=2)
    dAg, dy0g = tvi.adjoint(tm, o, dev(w["times"]), dev(w["params"]), dev(ref), dev(g))
    dAg, dy0g = dAg.cpu().numpy(), dy0g.cpu().numpy()
    assert np.abs(dAg - dA).max() / np.abs(dA).max() <= GATE[precision]
    assert np.abs(dy0g - dy0).max() / np.abs(dy0).max() <= GATE[precision]


# ---------------------------------------------------------------------------
# Van der Pol, the full paper-shaped workload (128 series x 10,000 log steps).
# ---------------------------------------------------------------------------
_VDP_REF = {}


def vdp_reference(oracle_lib, tol):
    """Oracle trajectory of the full workload at Newton tolerance tol, and the
    per-series forward error that stopping at tol can leave (propagated estimate)."""
    if tol not in _VDP_REF:
        w = workloads.vdp()
        m = OModel.from_spec(w["spec"])
        ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=tol,
                                        max_iter=100)
        assert not st.any()
        est = oracle_lib.forward_error_estimate(m, w["times"], w["params"], ref, tol)
        _VDP_REF[tol] = (w, ref, est)
    return _VDP_REF[tol]


@pytest.mark.parametrize("tol", [1e-12, 1e-10])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("chunk", [1000, 100, 10, 1])
def test_vdp_forward_parity_full_size(tvi, oracle_lib, precision, chunk, tol):
    """Gate per series: max(parity gate, 10 x the forward error that residuals of
    size tol leave after propagation through the linearised recursion); and, for
    all 128 series and every one of the 10,000 steps, the GPU's y_k against the
    oracle's solve of step k from the GPU's y_{k-1} at 1e-10 relative."""
    w, ref, est = vdp_reference(oracle_lib, tol)
    y, stats, status, rc = run_gpu(tvi, w, chunk, precision, tol)
    assert rc == 0 and not status.any(), (rc, np.nonzero(status))
    err = relerr_series(y, ref)
    bound = np.maximum(GATE[precision], 10.0 * est)
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, (bad, err[bad], est[bad])
    step = be_step_errors(oracle_lib, OModel.from_spec(w["spec"]), w, y)
    assert step.max() <= STEP_GATE, (step.argmax(), step.max())


@pytest.mark.parametrize("refine", [2, 1])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("chunk", [1000, 37, 1])
def test_vdp_adjoint_parity_full_size(tvi, oracle_lib, precision, chunk, refine):
    """Both adjoints run on the oracle's trajectory, so they solve the same
    linear system; the gradient is compared directly.  One refinement sweep is
    the benchmark's setting."""
    w, ref, _ = vdp_reference(oracle_lib, 1e-10)
    m = OModel.from_spec(w["spec"])
    g = workloads.random_grad_out(78, 128, 10000, 2)
    dmu, dy0 = oracle_lib.adjoint(m, w["times"], w["params"], ref, g)
    tm = tvi.Model.from_spec(w["spec"])
    o = tvi.Options(chunk=chunk, precision=precision, adjoint_refine=refine)
    dmug, dy0g = tvi.adjoint(tm, o, dev(w["times"]), dev(w["params"]), dev(ref), dev(g))
    dmug, dy0g = dmug.cpu().numpy(), dy0g.cpu().numpy()
    e_mu = np.abs(dmug - dmu)[:, 0] / np.maximum(np.abs(dmu)[:, 0], 1e-300)
    e_y0 = np.abs(dy0g - dy0).max(1) / np.maximum(np.abs(dy0).max(1), 1e-300)
    assert e_mu.max() <= GATE[precision], (e_mu.argmax(), e_mu.max())
    assert e_y0.max() <= GATE[precision], (e_y0.argmax(), e_y0.max())


# ---------------------------------------------------------------------------
# Edge cases and failure reporting.
# ---------------------------------------------------------------------------
def test_ragged_tail_lengths_and_tiny_sizes(tvi, oracle_lib):
    """Ragged lengths (a full series, one step, none, and two in between) padded
    into one launch: padded steps keep the state bit-exactly, the trajectory meets
    the per-series gate max(1e-10, 10 x the propagated forward-error estimate) and
    every real step meets 1e-10 against the oracle's solve from the GPU's y_{k-1}."""
    w = workloads.vdp(B=5, N=1003, seed=41)
    m = OModel.from_spec(w["spec"])
    lengths = np.array([1003, 1, 0, 500, 777], dtype=np.int32)
    ref, _, _ = oracle_lib.forward(m, w["y0"], w["times"], w["params"], lengths=lengths,
                                   tol_abs=1e-12)
    est = oracle_lib.forward_error_estimate(m, w["times"], w["params"], ref, 1e-12,
                                            lengths=lengths)
    for chunk in [100, 37, 1]:
        y, _, status, rc = run_gpu(tvi, w, chunk, "fp64", 1e-12, lengths=lengths)
        assert rc == 0
        for b, L in enumerate(lengths):
            assert np.all(y[b, L + 1:] == y[b, L])  # padded steps keep the state exactly
        assert np.all(relerr_series(y, ref) <= np.maximum(GATE["fp64"], 10.0 * est))
        assert be_step_errors(oracle_lib, m, w, y, lengths=lengths).max() <= STEP_GATE
    # B = 1, N = 1 and N = 0
    w1 = workloads.vdp(B=1, N=1, seed=42)
    ref1, _, _ = oracle_lib.forward(m, w1["y0"], w1["times"], w1["params"], tol_abs=1e-13)
    y1, _, _, rc = run_gpu(tvi, w1, 16, "fp32", 1e-13)
    assert rc == 0 and relerr_series(y1, ref1).max() <= 1e-10
    w0 = dict(w1, times=w1["times"][:, :1])
    y0o, _, _, rc = run_gpu(tvi, w0, 16, "fp64", 1e-13)
    assert rc == 0 and y0o.shape == (1, 1, 2) and np.array_equal(y0o[:, 0], w1["y0"])


def test_status_reporting(tvi):
    import paper_2310_08649_gb300._lib as L
    w = workloads.vdp(B=4, N=300, seed=43)
    p = w["params"].copy()
    p[2, 0] = np.nan
    y, _, status, rc = run_gpu(tvi, dict(w, params=p), 50, "fp32", 1e-10)
    assert rc == L.TVI_ENONFINITE and status.tolist() == [0, 0, 2, 0]
    y, _, status, rc = run_gpu(tvi, w, 50, "fp64", 1e-30, max_iter=1)
    assert rc == L.TVI_ENOTCONV and np.all(status == 1)
    with pytest.raises(L.TviError):
        tvi.integrate(tvi.Model.from_spec(w["spec"]),
                      tvi.Options(chunk=50, tol_abs=1e-30, max_iter=1),
                      dev(w["y0"]), dev(w["times"]), dev(w["params"]))


def test_series_independence_bitwise(tvi):
    w = workloads.vdp(B=32, N=2000, seed=44)
    y, _, _, _ = run_gpu(tvi, w, 100, "fp32", 1e-10)
    sub = [3, 17, 30]
    ws = dict(w, y0=w["y0"][sub], times=w["times"][sub], params=w["params"][sub])
    ys, _, _, _ = run_gpu(tvi, ws, 100, "fp32", 1e-10)
    assert np.array_equal(y[sub], ys)


def test_autograd_function_matches_oracle_gradient(tvi, oracle_lib):
    w = workloads.vdp(B=6, N=800, seed=45)
    m = OModel.from_spec(w["spec"])
    tm = tvi.Model.from_spec(w["spec"])
    o = tvi.Options(chunk=50, tol_abs=1e-12, precision="fp64")
    y0 = dev(w["y0"]).requires_grad_(True)
    mu = dev(w["params"]).requires_grad_(True)
    y = tvi.odeint(tm, o, y0, mu, dev(w["times"]))
    loss = (y ** 2).sum()
    loss.backward()
    ref, _, _ = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-12)
    dmu, dy0 = oracle_lib.adjoint(m, w["times"], w["params"], ref, 2.0 * ref)
    assert np.abs(mu.grad.cpu().numpy() - dmu).max() / np.abs(dmu).max() <= 1e-8
    assert np.abs(y0.grad.cpu().numpy() - dy0).max() / np.abs(dy0).max() <= 1e-8


def test_kernel_launch_counter(tvi):
    """One fused launch per forward pass and one per adjoint (per-series parameters:
    no shared-parameter sum)."""
    from paper_2310_08649_gb300 import _lib
    lib = _lib.load()
    w = workloads.vdp(B=4, N=300, seed=46)
    c0 = lib.tvi_kernel_launches()
    y, _, _, rc = run_gpu(tvi, w, 100, "fp32", 1e-10)
    assert rc == 0 and lib.tvi_kernel_launches() - c0 == 1
    tm = tvi.Model.from_spec(w["spec"])
    c1 = lib.tvi_kernel_launches()
    tvi.adjoint(tm, tvi.Options(chunk=100, precision="fp32"), dev(w["times"]), dev(w["params"]),
                dev(y), dev(np.ones_like(y)))
    torch.cuda.synchronize()
    assert lib.tvi_kernel_launches() - c1 == 1
