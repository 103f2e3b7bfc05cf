"""GPU parity of the neural-ODE (MLP right-hand side) path with the CPU FP64
oracle, through the C ABI.

Gates: 1e-10 relative with FP64 blocks, 1e-5 with FP32 blocks and with BF16
block products (the Newton residual and the adjoint refinement residuals are
FP64 in every mode, so the block precision changes iteration counts, not the
converged result), per series on the trajectory (max_k |y - y_ref|_inf / max_k |y_ref|_inf) and per
tensor on the gradients.  The tanh/SiLU networks here are smooth and bounded,
so the problems are well conditioned and the gates apply directly; the
trajectories are compared at a tight Newton tolerance (1e-12) so that both
sides solve the same discrete equations to well below the gate.
"""
import numpy as np
import pytest

import workloads
from oracle import Model as OModel
from parity_helpers import STEP_GATE, be_step_bound, be_step_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = {"fp64": 1e-10, "fp32": 1e-5, "bf16": 1e-5}


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


def gpu_forward(tvi, w, chunk, precision, tol, lengths=None):
    m = tvi.Model.from_spec(w["spec"])
    o = tvi.Options(chunk=chunk, tol_abs=tol, precision=precision, max_iter=60)
    lens = None if lengths is None else dev(lengths, torch.int32)
    y, stats, st, rc = tvi.integrate(m, o, dev(w["y0"]), dev(w["times"]), dev(w["params"]), lens,
                                     raise_on_status=False)
    torch.cuda.synchronize()
    return y.cpu().numpy(), stats.cpu().numpy(), st.cpu().numpy(), rc


def gpu_adjoint(tvi, w, chunk, precision, y, g, lengths=None, refine=2):
    m = tvi.Model.from_spec(w["spec"])
    o = tvi.Options(chunk=chunk, precision=precision, adjoint_refine=refine)
    lens = None if lengths is None else dev(lengths, torch.int32)
    dp, dy0 = tvi.adjoint(m, o, dev(w["times"]), dev(w["params"]), dev(y), dev(g), lens)
    torch.cuda.synchronize()
    return dp.cpu().numpy(), dy0.cpu().numpy()


@pytest.mark.parametrize("act", ["tanh", "silu"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("chunk", [1, 7, 40, 120, 500])
def test_small_mlp_forward_and_adjoint(tvi, oracle_lib, act, precision, chunk):
    w = workloads.mlp_ode(B=3, N=120, n=4, hidden=(8, 12), act=act, t_end=3.0, seed=61)
    m = OModel.from_spec(w["spec"])
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-12)
    assert not st.any()
    y, stats, status, rc = gpu_forward(tvi, w, chunk, precision, 1e-12)
    assert rc == 0 and not status.any()
    assert relerr_series(y, ref).max() <= GATE[precision]
    g = workloads.random_grad_out(62, 3, 120, 4)
    dp_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g)
    dp, dy0 = gpu_adjoint(tvi, w, chunk, precision, ref, g)
    assert relerr(dp, dp_ref) <= GATE[precision]
    assert relerr(dy0, dy0_ref) <= GATE[precision]


@pytest.fixture(scope="module")
def node16(oracle_lib):
    """The n = 16 neural-ODE workload: MLP 16-64-64-16 tanh, 64 series x 2000 steps."""
    w = workloads.mlp_ode()
    m = OModel.from_spec(w["spec"])
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-12)
    assert not st.any()
    g = workloads.random_grad_out(63, 64, 2000, 16)
    dp_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g)
    # forward error that stopping Newton at residual 1e-12 can leave over 2000 steps
    est = oracle_lib.forward_error_estimate(m, w["times"], w["params"], ref, 1e-12)
    return w, ref, g, dp_ref, dy0_ref, est


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_node16_full_size(tvi, oracle_lib, node16, precision):
    w, ref, g, dp_ref, dy0_ref, est = node16
    y, stats, status, rc = gpu_forward(tvi, w, 200, precision, 1e-12)
    assert rc == 0 and not status.any()
    err = relerr_series(y, ref)
    assert np.all(err <= np.maximum(GATE[precision], 10.0 * est)), (err.max(), est.max())
    assert be_step_errors(oracle_lib, OModel.from_spec(w["spec"]), w, y).max() <= STEP_GATE
    dp, dy0 = gpu_adjoint(tvi, w, 200, precision, ref, g)
    assert relerr(dp, dp_ref) <= GATE[precision]
    assert relerr(dy0, dy0_ref) <= GATE[precision]


def test_node32_silu_padded_lengths(tvi, oracle_lib):
    """n = 32 SiLU network (MLP 32-128-128-32), per-series lengths padded into one
    launch (dt = 0 past each length), reduced batch so the oracle stays quick."""
    w = workloads.mlp_large(B=4, N=1200, lengths_range=(200, 1200))
    m = OModel.from_spec(w["spec"])
    lens = w["lengths"]
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], lengths=lens,
                                    tol_abs=1e-12)
    assert not st.any()
    g = workloads.random_grad_out(64, 4, 1200, 32)
    for b, L in enumerate(lens):
        g[b, L + 1:] = 0.0  # masked loss past each length
    dp_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g, lengths=lens)
    for precision in ("fp32", "fp64"):
        y, _, status, rc = gpu_forward(tvi, w, 500, precision, 1e-12, lengths=lens)
        assert rc == 0 and not status.any()
        for b, L in enumerate(lens):
            assert np.all(y[b, L + 1:] == y[b, L])
        assert relerr_series(y, ref).max() <= GATE[precision]
        dp, dy0 = gpu_adjoint(tvi, w, 500, precision, ref, g, lengths=lens)
        assert relerr(dp, dp_ref) <= GATE[precision]
        assert relerr(dy0, dy0_ref) <= GATE[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_with_lengths_skips_padded_chunks_exactly(tvi, oracle_lib, precision):
    """With per-series lengths, an adjoint chunk wholly past a series' length with zero
    dL/dy there is skipped for that series (identity blocks, no parameter terms: its
    carry passes through).  Short chunks and lengths from 30 to 200 make most chunks of
    most series skippable.  Both the masked loss (skips taken) and a loss with nonzero
    dL/dy past the lengths (no skip allowed) must match the oracle's adjoint."""
    w = workloads.mlp_ode(B=6, N=200, n=4, hidden=(8, 12), t_end=4.0, seed=91,
                          lengths_range=(30, 200))
    lens = w["lengths"]
    m = OModel.from_spec(w["spec"])
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], lengths=lens,
                                    tol_abs=1e-12)
    assert not st.any()
    g_full = workloads.random_grad_out(92, 6, 200, 4)
    g_masked = g_full.copy()
    for b, L in enumerate(lens):
        g_masked[b, L + 1:] = 0.0
    for g in (g_masked, g_full):
        dp_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g, lengths=lens)
        dp, dy0 = gpu_adjoint(tvi, w, 20, precision, ref, g, lengths=lens)
        assert relerr(dp, dp_ref) <= GATE[precision]
        assert relerr(dy0, dy0_ref) <= GATE[precision]
    # forward Euler's adjoint couples a_k to step k + 1: the same skips
    ref_fe, st = oracle_lib.forward_euler(m, w["y0"], w["times"], w["params"], lengths=lens)
    assert not st.any()
    tm = tvi.Model.from_spec(w["spec"])
    o = tvi.Options(chunk=20, precision=precision, adjoint_refine=2, scheme="forward")
    for g in (g_masked, g_full):
        dp_ref, dy0_ref = oracle_lib.adjoint_euler(m, w["times"], w["params"], ref_fe, g,
                                                   lengths=lens)
        dp, dy0 = tvi.adjoint(tm, o, dev(w["times"]), dev(w["params"]), dev(ref_fe), dev(g),
                              dev(lens, torch.int32))
        torch.cuda.synchronize()
        assert relerr(dp.cpu().numpy(), dp_ref) <= GATE[precision]
        assert relerr(dy0.cpu().numpy(), dy0_ref) <= GATE[precision]


def test_mlp_status_and_rejections(tvi):
    import paper_2310_08649_gb300._lib as L
    w = workloads.mlp_ode(B=3, N=50, n=4, hidden=(8, 8), seed=65)
    p = w["params"].copy()
    p[5] = np.nan
    _, _, status, rc = gpu_forward(tvi, dict(w, params=p), 10, "fp32", 1e-10)
    assert rc == L.TVI_ENONFINITE and np.all(status == 2)
    bad = workloads.mlp_ode(B=2, N=10, n=4, hidden=(6, 8), seed=66)
    with pytest.raises(L.TviError):  # hidden width not a multiple of 4
        tvi.integrate(tvi.Model.from_spec(bad["spec"]), tvi.Options(chunk=5), dev(bad["y0"]),
                      dev(bad["times"]), dev(bad["params"]))


def test_mlp_chunk_halving(tvi, oracle_lib):
    """A stiff network (weights x3, 240 steps on [0, 5]) whose 240-step chunk Newton
    cannot solve within 12 updates: without halving the series report the
    iteration limit; with it the failed series re-solve the chunk by halves until
    Newton converges, and the trajectory is the oracle's (same equations, same
    tolerance), every step checked on its own."""
    import paper_2310_08649_gb300._lib as L
    w = workloads.mlp_ode(B=3, N=240, n=4, hidden=(8, 12), t_end=5.0, seed=61)
    w["params"] = w["params"] * 3.0
    m = OModel.from_spec(w["spec"])
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-12,
                                    max_iter=60)
    assert not st.any()
    tm = tvi.Model.from_spec(w["spec"])
    args = (dev(w["y0"]), dev(w["times"]), dev(w["params"]))
    o = tvi.Options(chunk=240, tol_abs=1e-12, precision="fp64", max_iter=12, retry_halving=False)
    _, _, status, rc = tvi.integrate(tm, o, *args, raise_on_status=False)
    assert rc == L.TVI_ENOTCONV and status.cpu().numpy().all()
    o = tvi.Options(chunk=240, tol_abs=1e-12, precision="fp64", max_iter=12)
    y, stats, status, rc = tvi.integrate(tm, o, *args, raise_on_status=False)
    torch.cuda.synchronize()
    y, stats = y.cpu().numpy(), stats.cpu().numpy()
    assert rc == 0 and not status.cpu().numpy().any()
    assert stats[:, 2].min() >= 1  # every series halved at least once
    est = oracle_lib.forward_error_estimate(m, w["times"], w["params"], ref, 1e-12)
    assert np.all(relerr_series(y, ref) <= np.maximum(GATE["fp64"], 10.0 * est))
    assert be_step_errors(oracle_lib, m, w, y).max() <= STEP_GATE


FIRST_PASS_CASES = [
    # (n, hidden, act, precision, scheme, chunk)
    (4, (8, 12), "tanh", "fp64", "backward", 240),   # halves (stiff weights below)
    (16, (64, 64), "tanh", "bf16", "backward", 37),
    (16, (64, 64), "silu", "fp32", "forward", 50),
    (32, (128, 128), "silu", "bf16", "backward", 64),
    (32, (128, 128), "silu", "fp64", "forward", 64),
]


@pytest.mark.parametrize("case", FIRST_PASS_CASES)
def test_first_pass_once_per_series_is_bit_identical(tvi, monkeypatch, case):
    """Every chunk attempt starts from dy = 0, so its first residual evaluates the
    network at the chunk start for every step; the forward pass evaluates it once per
    series.  With the test hook TVI_TEST_PER_PAIR_FIRST_PASS=1 every step evaluates it
    itself.  Trajectory, statistics and status must agree bit for bit (non-uniform
    steps, padded lengths, ragged chunks; the first case also halves its chunks)."""
    n, hidden, act, precision, scheme, chunk = case
    B, N = 5, 240
    w = workloads.mlp_ode(B=B, N=N, n=n, hidden=hidden, act=act, t_end=5.0 if n == 4 else 2.0,
                          seed=71, lengths_range=(150, N))
    if n == 4:
        w["params"] = w["params"] * 3.0
    rng = np.random.default_rng(72)
    dt = rng.uniform(0.5, 1.5, (B, N)) * w["times"][:, 1:2]
    w["times"] = np.concatenate([np.zeros((B, 1)), np.cumsum(dt, axis=1)], axis=1)
    m = tvi.Model.from_spec(w["spec"])
    o = tvi.Options(chunk=chunk, tol_abs=1e-11, precision=precision, max_iter=12 if n == 4 else 60,
                    scheme=scheme)
    args = (dev(w["y0"]), dev(w["times"]), dev(w["params"]), dev(w["lengths"], torch.int32))
    runs = []
    for hook in ("0", "1"):
        monkeypatch.setenv("TVI_TEST_PER_PAIR_FIRST_PASS", hook)
        y, stats, st, rc = tvi.integrate(m, o, *args, raise_on_status=False)
        torch.cuda.synchronize()
        runs.append((y.cpu().numpy(), stats.cpu().numpy(), st.cpu().numpy(), rc))
    monkeypatch.delenv("TVI_TEST_PER_PAIR_FIRST_PASS")
    (y0, s0, st0, rc0), (y1, s1, st1, rc1) = runs
    assert rc0 == rc1 == 0 and not st0.any() and np.array_equal(st0, st1)
    assert np.array_equal(s0, s1)
    assert np.array_equal(y0.view(np.uint64), y1.view(np.uint64))
    if n == 4:
        assert s0[:, 2].max() >= 1  # chunks were halved


def test_tc_wait_timeout_reports_status(tvi, monkeypatch):
    """The tensor-core block kernel bounds every mbarrier wait.  With the test hook
    TVI_TEST_TC_FIRST_WAIT_POLLS = 0 the first data wait of every block gives up at
    once (the bulk copy it waits for is still in flight, and is drained before the
    block frees its tensor memory and exits): the forward pass returns TVI_ETIMEOUT
    with status 3 for every series, the adjoint NaN gradients, and the context
    stays usable -- the same calls without the hook succeed afterwards."""
    import paper_2310_08649_gb300._lib as L
    w = workloads.mlp_ode(B=4, N=60, n=16, hidden=(64, 64), seed=67)
    g = workloads.random_grad_out(68, 4, 60, 16)
    monkeypatch.setenv("TVI_TEST_TC_FIRST_WAIT_POLLS", "0")
    y, _, status, rc = gpu_forward(tvi, w, 20, "bf16", 1e-10)
    assert rc == L.TVI_ETIMEOUT == -6 and np.all(status == 3), (rc, status)
    dp, dy0 = gpu_adjoint(tvi, w, 20, "bf16", np.zeros((4, 61, 16)), g)
    assert np.all(np.isnan(dp)) and np.all(np.isnan(dy0))
    monkeypatch.delenv("TVI_TEST_TC_FIRST_WAIT_POLLS")
    y, _, status, rc = gpu_forward(tvi, w, 20, "bf16", 1e-10)
    assert rc == 0 and not status.any()
    dp, dy0 = gpu_adjoint(tvi, w, 20, "bf16", y, g)
    assert np.all(np.isfinite(dp)) and np.all(np.isfinite(dy0))


# ---------------------------------------------------------------------------
# BF16 block products on the tensor cores (n >= 16)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("act", ["tanh", "silu"])
@pytest.mark.parametrize("chunk", [1, 7, 40, 120])
def test_bf16_blocks_small(tvi, oracle_lib, act, chunk):
    """Ragged tiles (chunk 7 and the 120-step tail of 40-step chunks are not
    multiples of the 8 steps of a 128-row tile) and one-step chunks."""
    w = workloads.mlp_ode(B=3, N=120, n=16, hidden=(64, 64), act=act, t_end=3.0, seed=67)
    m = OModel.from_spec(w["spec"])
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-12)
    assert not st.any()
    y, stats, status, rc = gpu_forward(tvi, w, chunk, "bf16", 1e-12)
    assert rc == 0 and not status.any()
    assert relerr_series(y, ref).max() <= GATE["bf16"]
    g = workloads.random_grad_out(68, 3, 120, 16)
    dp_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g)
    dp, dy0 = gpu_adjoint(tvi, w, chunk, "bf16", ref, g)
    assert relerr(dp, dp_ref) <= GATE["bf16"]
    assert relerr(dy0, dy0_ref) <= GATE["bf16"]


def test_bf16_blocks_are_the_jacobian(tvi, node16):
    """Without refinement the adjoint is exactly the chain of the blocks, so its
    error measures the blocks themselves.  BF16 rounding (2^-9 relative) of the
    products making dt J, |dt J| ~ 0.05, perturbs each step by ~1e-4, which over
    2000 steps accumulates to a few 1e-3 at most; a wrong operand layout, a
    transposed block or a dropped scaling perturbs each step by O(|dt J|) and the
    gradient by O(1).  FP32 blocks give the floor of the same measurement."""
    w, ref, g, dp_ref, dy0_ref, _ = node16
    dp32, _ = gpu_adjoint(tvi, w, 200, "fp32", ref, g, refine=0)
    dp16, dy016 = gpu_adjoint(tvi, w, 200, "bf16", ref, g, refine=0)
    e32, e16 = relerr(dp32, dp_ref), relerr(dp16, dp_ref)
    assert e32 <= 1e-4, (e32, e16)
    assert e16 <= 5e-3, (e32, e16)
    assert relerr(dy016, dy0_ref) <= 5e-3


def test_bf16_node16_full_size(tvi, oracle_lib, node16):
    w, ref, g, dp_ref, dy0_ref, est = node16
    y32, s32, _, rc32 = gpu_forward(tvi, w, 200, "fp32", 1e-12)
    y, stats, status, rc = gpu_forward(tvi, w, 200, "bf16", 1e-12)
    assert rc == 0 and rc32 == 0 and not status.any()
    err = relerr_series(y, ref)
    assert np.all(err <= np.maximum(GATE["bf16"], 10.0 * est)), (err.max(), est.max())
    assert be_step_errors(oracle_lib, OModel.from_spec(w["spec"]), w, y).max() <= STEP_GATE
    # inexact-Newton blocks cost few extra updates; a wrong Jacobian costs many
    assert stats[:, 0].sum() <= 1.3 * s32[:, 0].sum(), (stats[:, 0].sum(), s32[:, 0].sum())
    dp, dy0 = gpu_adjoint(tvi, w, 200, "bf16", ref, g)
    assert relerr(dp, dp_ref) <= GATE["bf16"]
    assert relerr(dy0, dy0_ref) <= GATE["bf16"]


def test_bf16_node32_silu_padded_lengths(tvi, oracle_lib):
    w = workloads.mlp_large(B=4, N=1200, lengths_range=(200, 1200))
    m = OModel.from_spec(w["spec"])
    lens = w["lengths"]
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], lengths=lens,
                                    tol_abs=1e-12)
    assert not st.any()
    g = workloads.random_grad_out(64, 4, 1200, 32)
    for b, L in enumerate(lens):
        g[b, L + 1:] = 0.0
    dp_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g, lengths=lens)
    y, _, status, rc = gpu_forward(tvi, w, 500, "bf16", 1e-12, lengths=lens)
    assert rc == 0 and not status.any()
    for b, L in enumerate(lens):
        assert np.all(y[b, L + 1:] == y[b, L])
    assert relerr_series(y, ref).max() <= GATE["bf16"]
    dp, dy0 = gpu_adjoint(tvi, w, 500, "bf16", ref, g, lengths=lens)
    assert relerr(dp, dp_ref) <= GATE["bf16"]
    assert relerr(dy0, dy0_ref) <= GATE["bf16"]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_mlp_degenerate_sizes(tvi, oracle_lib, precision):
    """Series of length 0 and 1 among a full one, N = 1 and N = 0 (the trajectory
    is y0 alone, the gradient is the loss gradient at y0), on every block path."""
    w = workloads.mlp_ode(B=3, N=50, n=16, hidden=(64, 64), act="silu", t_end=1.0, seed=69)
    m = OModel.from_spec(w["spec"])
    lens = np.array([50, 0, 1], dtype=np.int32)
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], lengths=lens,
                                    tol_abs=1e-12)
    assert not st.any()
    y, _, status, rc = gpu_forward(tvi, w, 16, precision, 1e-12, lengths=lens)
    assert rc == 0 and not status.any()
    for b, L in enumerate(lens):
        assert np.all(y[b, L + 1:] == y[b, L])
    assert relerr_series(y, ref).max() <= GATE[precision]
    g = workloads.random_grad_out(70, 3, 50, 16)
    for b, L in enumerate(lens):
        g[b, L + 1:] = 0.0
    dp_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g, lengths=lens)
    dp, dy0 = gpu_adjoint(tvi, w, 16, precision, ref, g, lengths=lens)
    assert relerr(dp, dp_ref) <= GATE[precision]
    assert relerr(dy0, dy0_ref) <= GATE[precision]
    # N = 1 and N = 0
    w1 = dict(w, times=w["times"][:, :2], lengths=None)
    ref1, _, _ = oracle_lib.forward(m, w1["y0"], w1["times"], w1["params"], tol_abs=1e-12)
    y1, _, _, rc = gpu_forward(tvi, w1, 16, precision, 1e-12)
    assert rc == 0 and relerr_series(y1, ref1).max() <= GATE[precision]
    w0 = dict(w, times=w["times"][:, :1], lengths=None)
    y0o, _, _, rc = gpu_forward(tvi, w0, 16, precision, 1e-12)
    assert rc == 0 and y0o.shape == (3, 1, 16) and np.array_equal(y0o[:, 0], w["y0"])
    g0 = workloads.random_grad_out(71, 3, 0, 16)
    dp0, dy00 = gpu_adjoint(tvi, w0, 16, precision, y0o, g0)
    assert not dp0.any() and np.array_equal(dy00, g0[:, 0])


def test_node32_full_size_sampled(tvi, oracle_lib):
    """The benchmark's n = 32 configuration at full size (512 series x 20,000 padded
    steps, chunk 1000, BF16 blocks, tol 1e-8) against the oracle on sampled series:
    series are independent, so three of them are integrated by the oracle alone; and
    the adjoint is linear in dL/dy, so a loss gradient that is nonzero only on the
    sampled series makes the shared-parameter gradient a sum over those three."""
    w = workloads.mlp_large()
    B = w["y0"].shape[0]
    sample = np.array([0, 257, B - 1])
    m = OModel.from_spec(w["spec"])
    lens = w["lengths"]
    sub = dict(w, y0=w["y0"][sample], times=w["times"][sample], lengths=lens[sample])
    tol = 1e-8
    ref, _, st = oracle_lib.forward(m, sub["y0"], sub["times"], w["params"], lengths=sub["lengths"],
                                    tol_abs=tol, max_iter=60)
    assert not st.any()
    est = oracle_lib.forward_error_estimate(m, sub["times"], w["params"], ref, tol,
                                            lengths=sub["lengths"])
    y, stats, status, rc = gpu_forward(tvi, w, 1000, "bf16", tol, lengths=lens)
    assert rc == 0 and not status.any()
    err = relerr_series(y[sample], ref)
    assert np.all(err <= np.maximum(GATE["bf16"], 10.0 * est)), (err, est)
    # every real step of the sampled series against the oracle's solve of that step
    # from the GPU's own previous state: residuals of tol 1e-8 leave at most
    # be_step_bound there (one step's conditioning)
    step = be_step_errors(oracle_lib, m, sub, y[sample], lengths=sub["lengths"])
    assert np.all(step <= be_step_bound(oracle_lib, m, sub, y[sample], tol,
                                        lengths=sub["lengths"])), step
    g = np.zeros_like(y)
    g[sample] = workloads.random_grad_out(72, len(sample), y.shape[1] - 1, 32)
    for b_, L in zip(sample, lens[sample]):
        g[b_, L + 1:] = 0.0
    dp_ref, dy0_ref = oracle_lib.adjoint(m, sub["times"], w["params"], ref, g[sample],
                                         lengths=sub["lengths"])
    # both adjoints on the oracle's trajectory for the sampled series (the others
    # carry zero loss gradient, so their trajectories do not enter dL/dp)
    y_mix = y.copy()
    y_mix[sample] = ref
    dp, dy0 = gpu_adjoint(tvi, w, 1000, "bf16", y_mix, g, lengths=lens)
    assert relerr(dp, dp_ref) <= GATE["bf16"]
    assert relerr(dy0[sample], dy0_ref) <= GATE["bf16"]
    assert not dy0[np.setdiff1d(np.arange(B), sample)].any()
