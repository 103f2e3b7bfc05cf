"""GPU parity of user models (device source compiled at run time: n <= 4 into
the fused small-state kernels, larger n into the large-state kernels) with the
CPU FP64 oracle, through the C ABI.

Each user source restates one of the oracle's models (van der Pol, linear of
any size, a tanh MLP, the mass-damper-spring chain, Chaboche viscoplasticity,
coupled neurons), so forward trajectories and adjoint gradients are compared
with the oracle exactly as for the built-in models: 1e-10 relative with FP64
blocks, 1e-5 with FP32 blocks, and for nonlinear models max(gate, 10 x the
propagated forward-error estimate) per series, together with the
conditioning-free check of every step against the oracle's solve of that step
from the GPU's own previous state at 1e-10 (parity_helpers).  Sizes run from
n = 1 to 20, most of them ones the built-in engines do not have.
"""
import ctypes

import numpy as np
import pytest

import workloads
from oracle import Model as OModel
from parity_helpers import STEP_GATE, be_step_errors, fe_step_errors
from test_gpu_euler import fe_error_estimate
from paper_2310_08649_gb300.user_sources import CHABOCHE, LINEAR, MDS, NEURON, VDP, \
    VDP_FP64_JAC, chaboche_param_count, mds_param_count, mlp_param_count, mlp_tanh, \
    neuron_param_count

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


@pytest.fixture(scope="module")
def users(tvi):
    made = {"vdp": tvi.UserModel(2, 1, VDP), "vdp64": tvi.UserModel(2, 1, VDP_FP64_JAC),
            "lin1": tvi.UserModel(1, 1, LINEAR),
            "lin3": tvi.UserModel(3, 9, LINEAR),
            "mlp3": tvi.UserModel(3, mlp_param_count(3, 2, 2), mlp_tanh(2, 2)),
            "mds1": tvi.UserModel(2, mds_param_count(1), MDS),
            "mds2": tvi.UserModel(4, mds_param_count(2), MDS),
            # n > 4: the large-state route
            "mds3": tvi.UserModel(6, mds_param_count(3), MDS),
            "mds5": tvi.UserModel(10, mds_param_count(5), MDS),
            "mds10": tvi.UserModel(20, mds_param_count(10), MDS),
            "lin5": tvi.UserModel(5, 25, LINEAR),
            **{f"chab{u}": tvi.UserModel(2 + u, chaboche_param_count(u), CHABOCHE)
               for u in (1, 2, 3, 5)},
            **{f"neuron{u}": tvi.UserModel(4 * u, neuron_param_count(u), NEURON)
               for u in (1, 2, 4, 6, 7, 8, 9, 10)},
            "mlp5": tvi.UserModel(5, mlp_param_count(5, 2, 1), mlp_tanh(2, 1))}
    yield made
    torch.cuda.synchronize()
    for u in made.values():
        u.close()


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def relerr_series(a, b):
    return np.abs(a - b).max(axis=(1, 2)) / np.maximum(np.abs(b).max(axis=(1, 2)), 1e-300)


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def forward(tvi, model, w, o, lengths=None):
    lens = None if lengths is None else dev(lengths, torch.int32)
    y, stats, st, rc = tvi.integrate(model, o, dev(w["y0"]), dev(w["times"]), dev(w["params"]),
                                     lens, raise_on_status=False)
    torch.cuda.synchronize()
    return y.cpu().numpy(), stats.cpu().numpy(), st.cpu().numpy(), rc


def adjoint(tvi, model, w, o, y, g, lengths=None):
    lens = None if lengths is None else dev(lengths, torch.int32)
    dp, dy0 = tvi.adjoint(model, o, dev(w["times"]), dev(w["params"]), dev(y), dev(g), lens)
    torch.cuda.synchronize()
    return dp.cpu().numpy(), dy0.cpu().numpy()


@pytest.mark.parametrize("jac", ["vdp", "vdp64"])  # Jacobian in the block type / in FP64
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("chunk", [1000, 64, 1])
def test_user_vdp_matches_oracle(tvi, users, oracle_lib, precision, chunk, jac):
    w = workloads.vdp(B=32, N=3000, seed=61)
    m = OModel.from_spec(w["spec"])
    tol = 1e-10
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=tol,
                                    max_iter=100)
    assert not st.any()
    est = oracle_lib.forward_error_estimate(m, w["times"], w["params"], ref, tol)
    model = users[jac].model(per_series=True)
    o = tvi.Options(chunk=chunk, tol_abs=tol, precision=precision, adjoint_refine=2)
    y, stats, status, rc = forward(tvi, model, w, o)
    assert rc == 0 and not status.any()
    err = relerr_series(y, ref)
    bad = np.nonzero(err > np.maximum(GATE[precision], 10.0 * est))[0]
    assert bad.size == 0, (bad, err[bad], est[bad])
    assert be_step_errors(oracle_lib, m, w, y).max() <= STEP_GATE
    g = workloads.random_grad_out(91, 32, 3000, 2)
    dp_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g)
    dp, dy0 = adjoint(tvi, model, w, o, ref, g)
    e_mu = np.abs(dp - dp_ref)[:, 0] / np.maximum(np.abs(dp_ref)[:, 0], 1e-300)
    assert e_mu.max() <= GATE[precision]
    assert relerr_series(dy0[:, None], dy0_ref[:, None]).max() <= GATE[precision]


def test_user_vdp_agrees_with_builtin(tvi, users):
    """Same equations, same solver: the user and built-in van der Pol runs agree
    to the Newton tolerance and take the same Newton path (update counts)."""
    w = workloads.vdp(B=16, N=2000, seed=62)
    o = tvi.Options(chunk=100, tol_abs=1e-12, precision="fp64")
    yb, sb, _, rc1 = forward(tvi, tvi.Model.from_spec(w["spec"]), w, o)
    yu, su, _, rc2 = forward(tvi, users["vdp"].model(per_series=True), w, o)
    assert rc1 == 0 and rc2 == 0
    assert relerr_series(yu, yb).max() <= 1e-9
    assert np.abs(su[:, 0] - sb[:, 0]).max() <= 0.05 * sb[:, 0].max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,chunk", [(1, 7), (3, 64), (3, 500)])
def test_user_linear_shared_params(tvi, users, oracle_lib, precision, n, chunk):
    """Shared parameters: the adjoint sums the per-series partials."""
    w = workloads.linear_stiff(B=8, N=500, n=n, lam_decades=(0.0, 3.0))
    m = OModel.from_spec(w["spec"])
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-13)
    assert not st.any()
    model = users[f"lin{n}"].model(per_series=False)
    o = tvi.Options(chunk=chunk, tol_abs=1e-13, precision=precision, adjoint_refine=2)
    y, _, status, rc = forward(tvi, model, w, o)
    assert rc == 0 and not status.any()
    assert relerr_series(y, ref).max() <= GATE[precision]
    g = workloads.random_grad_out(92, 8, 500, n)
    dA_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g)
    dA, dy0 = adjoint(tvi, model, w, o, ref, g)
    assert relerr(dA, dA_ref) <= GATE[precision]
    assert relerr(dy0, dy0_ref) <= GATE[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_user_mlp_n3(tvi, users, oracle_lib, precision):
    """A nonlinear user model of a size the built-in engines lack (n = 3, tanh
    MLP with hidden widths 2, 2; P = 23 shared)."""
    w = workloads.mlp_ode(B=8, N=600, n=3, hidden=(2, 2), seed=63, t_end=6.0)
    w["params"] = w["params"] + 0.3 * np.random.default_rng(64).standard_normal(
        w["params"].shape)  # non-zero biases
    m = OModel.from_spec(w["spec"])
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-13)
    assert not st.any()
    model = users["mlp3"].model(per_series=False)
    o = tvi.Options(chunk=128, tol_abs=1e-13, precision=precision, adjoint_refine=2)
    y, _, status, rc = forward(tvi, model, w, o)
    assert rc == 0 and not status.any()
    assert relerr_series(y, ref).max() <= GATE[precision]
    g = workloads.random_grad_out(93, 8, 600, 3)
    dp_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g)
    dp, dy0 = adjoint(tvi, model, w, o, ref, g)
    assert relerr(dp, dp_ref) <= GATE[precision]
    assert relerr(dy0, dy0_ref) <= GATE[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_user_forward_euler(tvi, users, oracle_lib, precision):
    w = workloads.vdp(B=8, N=1500, seed=65, mu_dt_max=0.2, mu_decades=(1.0, 2.0))
    m = OModel.from_spec(w["spec"])
    ref, st = oracle_lib.forward_euler(m, w["y0"], w["times"], w["params"])
    assert not st.any()
    model = users["vdp"].model(per_series=True)
    o = tvi.Options(chunk=64, tol_abs=1e-12, precision=precision, scheme="forward",
                    max_iter=60, adjoint_refine=2)
    y, _, status, rc = forward(tvi, model, w, o)
    assert rc == 0 and not status.any()
    # explicit recursion: residuals of 1e-12 grow with the recursion's conditioning
    est = fe_error_estimate(oracle_lib, m, w, ref, 1e-12)
    assert np.all(relerr_series(y, ref) <= np.maximum(GATE[precision], 10.0 * est))
    assert fe_step_errors(oracle_lib, m, w, y).max() <= STEP_GATE
    g = workloads.random_grad_out(94, 8, 1500, 2)
    dp_ref, dy0_ref = oracle_lib.adjoint_euler(m, w["times"], w["params"], ref, g)
    dp, dy0 = adjoint(tvi, model, w, o, ref, g)
    assert relerr(dp, dp_ref) <= GATE[precision]
    assert relerr(dy0, dy0_ref) <= GATE[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("u,chunk", [(1, 100), (2, 1000), (2, 7), (3, 300), (5, 1000), (10, 64),
                                     (10, 2000)])
def test_user_mds_matches_oracle(tvi, users, oracle_lib, precision, u, chunk):
    """Time-dependent right-hand side (the forcing f_a sin(2 pi t / T)): the
    mass-damper-spring chain of the paper's timing study, per-series parameters
    (table values, jittered so that series differ), zero initial state.  Up to
    2 units (n <= 4) on the fused small-state kernels, above on the large-state
    route (n = 6, 10, 20: the paper's n_unit 3, 5, 10)."""
    w = workloads.mds(B=16, N=2000, n_unit=u, jitter=0.1, seed=70 + u)
    m = OModel.from_spec(w["spec"])
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-18,
                                    max_iter=4)
    assert not st.any()
    model = users[f"mds{u}"].model(per_series=True)
    # |v| reaches 5e-3, so FP64 residuals bottom out near 1e-18: stop at 1e-17
    o = tvi.Options(chunk=chunk, tol_abs=1e-17, max_iter=20, precision=precision,
                    adjoint_refine=3)
    y, _, status, rc = forward(tvi, model, w, o)
    assert rc == 0 and not status.any()
    assert relerr_series(y, ref).max() <= GATE[precision]
    g = workloads.random_grad_out(96 + u, 16, 2000, 2 * u)
    dp_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g)
    dp, dy0 = adjoint(tvi, model, w, o, ref, g)
    e_p = np.abs(dp - dp_ref).max(axis=1) / np.abs(dp_ref).max(axis=1)
    assert e_p.max() <= GATE[precision], (e_p.argmax(), e_p.max())
    assert relerr(dy0, dy0_ref) <= GATE[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("which,chunk", [("lin5", 64), ("mlp5", 250)])
def test_user_large_shared_params(tvi, users, oracle_lib, precision, which, chunk):
    """Large-state route with shared parameters and a padded width (n = 5,
    vectors padded to 8): a linear system and a nonlinear tanh MLP."""
    if which == "lin5":
        w = workloads.linear_stiff(B=8, N=500, n=5, lam_decades=(0.0, 3.0))
    else:
        w = workloads.mlp_ode(B=8, N=500, n=5, hidden=(2, 1), seed=73, t_end=5.0)
        w["params"] = w["params"] + 0.3 * np.random.default_rng(74).standard_normal(
            w["params"].shape)
    m = OModel.from_spec(w["spec"])
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-13)
    assert not st.any()
    model = users[which].model(per_series=False)
    o = tvi.Options(chunk=chunk, tol_abs=1e-13, precision=precision, adjoint_refine=2)
    y, stats, status, rc = forward(tvi, model, w, o)
    assert rc == 0 and not status.any()
    assert relerr_series(y, ref).max() <= GATE[precision]
    g = workloads.random_grad_out(75, 8, 500, 5)
    dp_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g)
    dp, dy0 = adjoint(tvi, model, w, o, ref, g)
    assert relerr(dp, dp_ref) <= GATE[precision]
    assert relerr(dy0, dy0_ref) <= GATE[precision]


def test_user_large_padded_lengths_and_rejections(tvi, users, oracle_lib):
    import paper_2310_08649_gb300._lib as L
    w = workloads.mds(B=4, N=700, n_unit=3, jitter=0.1, seed=76)
    lens = np.array([700, 1, 0, 333], dtype=np.int32)
    m = OModel.from_spec(w["spec"])
    ref, _, _ = oracle_lib.forward(m, w["y0"], w["times"], w["params"], lengths=lens,
                                   tol_abs=1e-18, max_iter=4)
    model = users["mds3"].model(per_series=True)
    o = tvi.Options(chunk=128, tol_abs=1e-17, max_iter=20, precision="fp64")
    y, _, status, rc = forward(tvi, model, w, o, lengths=lens)
    assert rc == 0 and not status.any()
    for b, L_ in enumerate(lens):
        assert np.all(y[b, L_ + 1:] == y[b, L_])
    assert relerr_series(y, ref).max() <= 1e-10
    g = workloads.random_grad_out(77, 4, 700, 6)
    for b, L_ in enumerate(lens):
        g[b, L_ + 1:] = 0.0
    dp_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g, lengths=lens)
    dp, dy0 = adjoint(tvi, model, w, o, ref, g, lengths=lens)
    e_p = np.abs(dp - dp_ref).max(axis=1) / np.maximum(np.abs(dp_ref).max(axis=1), 1e-300)
    assert e_p.max() <= 1e-10 and relerr(dy0, dy0_ref) <= 1e-10
    # the allocation-free adjoint is a small-state feature
    lib = L.load()
    cm, co = model.c(), o.c()
    T, P, Y, G = dev(w["times"]), dev(w["params"]), dev(ref), dev(g)
    dpn = torch.empty_like(P)
    rc = lib.tvi_adjoint_noalloc(ctypes.byref(cm), ctypes.byref(co), 4, 700, T.data_ptr(), None,
                                 P.data_ptr(), Y.data_ptr(), G.data_ptr(), dpn.data_ptr(), None,
                                 None)
    assert rc == -7


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("u,chunk", [(1, 100), (2, 1000), (3, 250), (5, 1000)])
def test_user_chaboche_matches_oracle(tvi, users, oracle_lib, precision, u, chunk):
    """Chaboche viscoplasticity (nonsmooth flow rule, periodic strain rate): the
    paper's backstress counts 1 .. 5 (n = 3 .. 7; n > 4 on the large-state
    route), parameters from its table jittered per series, a loading strong
    enough to yield.  Gate per series: max(parity gate, 10 x the forward error
    that residuals of size tol leave after propagation)."""
    w = workloads.chaboche(B=12, N=2000, n_unit=u, jitter=0.1, seed=180 + u)
    w["params"][:, 6 + 2 * u] *= 3.0
    m = OModel.from_spec(w["spec"])
    tol = 1e-12
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=tol,
                                    max_iter=100)
    assert not st.any()
    assert np.abs(ref[:, :, 2:]).max() > 1e-2  # the backstresses moved: plastic flow
    est = oracle_lib.forward_error_estimate(m, w["times"], w["params"], ref, tol)
    model = users[f"chab{u}"].model(per_series=True)
    o = tvi.Options(chunk=chunk, tol_abs=tol, max_iter=60, precision=precision,
                    adjoint_refine=3)
    y, _, status, rc = forward(tvi, model, w, o)
    assert rc == 0 and not status.any()
    err = relerr_series(y, ref)
    bad = np.nonzero(err > np.maximum(GATE[precision], 10.0 * est))[0]
    assert bad.size == 0, (bad, err[bad], est[bad])
    assert be_step_errors(oracle_lib, m, w, y).max() <= STEP_GATE
    g = workloads.random_grad_out(190 + u, 12, 2000, 2 + u)
    dp_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g)
    dp, dy0 = adjoint(tvi, model, w, o, ref, g)
    e_p = np.abs(dp - dp_ref).max(axis=1) / np.abs(dp_ref).max(axis=1)
    assert e_p.max() <= GATE[precision], (e_p.argmax(), e_p.max())
    assert relerr(dy0, dy0_ref) <= GATE[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("u,chunk", [(1, 500), (2, 1000), (2, 64), (4, 1000), (6, 300),
                                     (7, 1000), (8, 64), (9, 250), (10, 1000)])
def test_user_neuron_matches_oracle(tvi, users, oracle_lib, precision, u, chunk):
    """Coupled neurons under a periodic current: one neuron (n = 4, fused
    kernels), two to ten (n = 8 .. 40, the large-state route; the paper's study
    runs 1 .. 10 neurons: ten have n = 40, blocks wider than a warp, and 151
    parameters, read from memory); n = 24 with FP32 blocks takes the tiled chain
    for these 16 series, n = 28 and 32 the sequential one; parameters from the
    paper's table jittered per series."""
    w = workloads.neuron(B=16, N=2000, n_unit=u, jitter=0.1, seed=230 + u)
    m = OModel.from_spec(w["spec"])
    tol = 1e-12
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=tol)
    assert not st.any()
    est = oracle_lib.forward_error_estimate(m, w["times"], w["params"], ref, tol)
    model = users[f"neuron{u}"].model(per_series=True)
    o = tvi.Options(chunk=chunk, tol_abs=tol, max_iter=60, precision=precision,
                    adjoint_refine=3)
    y, _, status, rc = forward(tvi, model, w, o)
    assert rc == 0 and not status.any()
    err = relerr_series(y, ref)
    bad = np.nonzero(err > np.maximum(GATE[precision], 10.0 * est))[0]
    assert bad.size == 0, (bad, err[bad], est[bad])
    assert be_step_errors(oracle_lib, m, w, y).max() <= STEP_GATE
    g = workloads.random_grad_out(240 + u, 16, 2000, 4 * u)
    dp_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g)
    dp, dy0 = adjoint(tvi, model, w, o, ref, g)
    e_p = np.abs(dp - dp_ref).max(axis=1) / np.abs(dp_ref).max(axis=1)
    assert e_p.max() <= GATE[precision], (e_p.argmax(), e_p.max())
    assert relerr(dy0, dy0_ref) <= GATE[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("which,chunk", [("chab3", 64), ("chab3", 1000), ("neuron2", 250)])
def test_user_large_forward_euler(tvi, users, oracle_lib, precision, which, chunk):
    """Forward Euler on the large-state route (blocks I + dt J without an
    inverse, the recurrence d_j = B_j d_{j-1} + R_j in the chain) against the
    step-by-step forward-Euler oracle: trajectory and both gradients."""
    if which == "chab3":
        w = workloads.chaboche(B=12, N=2000, n_unit=3, jitter=0.1, seed=250)
        w["params"][:, 12] *= 3.0  # strain-rate amplitude: the loading yields
    else:
        w = workloads.neuron(B=12, N=2000, n_unit=2, jitter=0.1, seed=251)
    m = OModel.from_spec(w["spec"])
    ref, st = oracle_lib.forward_euler(m, w["y0"], w["times"], w["params"])
    assert not st.any()
    model = users[which].model(per_series=True)
    o = tvi.Options(chunk=chunk, tol_abs=1e-12, precision=precision, scheme="forward",
                    max_iter=60, adjoint_refine=3)
    y, _, status, rc = forward(tvi, model, w, o)
    assert rc == 0 and not status.any()
    est = fe_error_estimate(oracle_lib, m, w, ref, 1e-12)
    err = relerr_series(y, ref)
    assert np.all(err <= np.maximum(GATE[precision], 10.0 * est)), (err.max(), est.max())
    assert fe_step_errors(oracle_lib, m, w, y).max() <= STEP_GATE
    n = w["spec"]["n"]
    g = workloads.random_grad_out(252, 12, 2000, n)
    dp_ref, dy0_ref = oracle_lib.adjoint_euler(m, w["times"], w["params"], ref, g)
    dp, dy0 = adjoint(tvi, model, w, o, ref, g)
    e_p = np.abs(dp - dp_ref).max(axis=1) / np.abs(dp_ref).max(axis=1)
    assert e_p.max() <= GATE[precision], (e_p.argmax(), e_p.max())
    assert relerr(dy0, dy0_ref) <= GATE[precision]


def test_user_large_chunk_halving(tvi, oracle_lib):
    """A stiff run-time compiled model on the large-state route (tanh MLP, n = 5,
    weights x5, 240 steps on [0, 12]) whose 240-step chunk needs more than 8 Newton
    updates: without halving the series report the iteration limit; with it they
    re-solve the chunk by halves and match the oracle, every step checked on its
    own."""
    import paper_2310_08649_gb300._lib as L
    w = workloads.mlp_ode(B=3, N=240, n=5, hidden=(3, 3), t_end=12.0, seed=62)
    w["params"] = w["params"] * 5.0
    m = OModel.from_spec(w["spec"])
    ref, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-12,
                                    max_iter=60)
    assert not st.any()
    user = tvi.UserModel(5, mlp_param_count(5, 3, 3), mlp_tanh(3, 3))
    model = user.model(per_series=False)
    o = tvi.Options(chunk=240, tol_abs=1e-12, precision="fp64", max_iter=8, retry_halving=False)
    _, _, status, rc = forward(tvi, model, w, o)
    assert rc == L.TVI_ENOTCONV and status.all()
    o = tvi.Options(chunk=240, tol_abs=1e-12, precision="fp64", max_iter=8)
    y, stats, status, rc = forward(tvi, model, w, o)
    assert rc == 0 and not status.any()
    assert stats[:, 2].min() >= 1  # every series halved at least once
    est = oracle_lib.forward_error_estimate(m, w["times"], w["params"], ref, 1e-12)
    assert np.all(relerr_series(y, ref) <= np.maximum(GATE["fp64"], 10.0 * est))
    assert be_step_errors(oracle_lib, m, w, y).max() <= STEP_GATE
    user.close()


def test_user_padded_lengths_and_noalloc(tvi, users, oracle_lib):
    import paper_2310_08649_gb300._lib as L
    w = workloads.vdp(B=4, N=700, seed=66)
    lens = np.array([700, 1, 0, 333], dtype=np.int32)
    m = OModel.from_spec(w["spec"])
    ref, _, _ = oracle_lib.forward(m, w["y0"], w["times"], w["params"], lengths=lens,
                                   tol_abs=1e-12)
    model = users["vdp"].model(per_series=True)
    o = tvi.Options(chunk=37, tol_abs=1e-12, precision="fp64")
    y, _, status, rc = forward(tvi, model, w, o, lengths=lens)
    assert rc == 0 and not status.any()
    for b, L_ in enumerate(lens):
        assert np.all(y[b, L_ + 1:] == y[b, L_])
    assert relerr_series(y, ref).max() <= 1e-9
    g = workloads.random_grad_out(95, 4, 700, 2)
    for b, L_ in enumerate(lens):
        g[b, L_ + 1:] = 0.0
    dp_ref, dy0_ref = oracle_lib.adjoint(m, w["times"], w["params"], ref, g, lengths=lens)
    dp, dy0 = adjoint(tvi, model, w, o, ref, g, lengths=lens)
    assert relerr(dp, dp_ref) <= 1e-10 and relerr(dy0, dy0_ref) <= 1e-10
    # the allocation-free adjoint takes user models too
    lib = L.load()
    cm, co = model.c(), o.c()
    T, P, Y, G = dev(w["times"]), dev(w["params"]), dev(ref), dev(g)
    LN = dev(lens, torch.int32)
    dpn = torch.empty_like(P)
    dy0n = torch.empty(4, 2, dtype=torch.float64, device="cuda")
    rc = lib.tvi_adjoint_noalloc(ctypes.byref(cm), ctypes.byref(co), 4, 700, T.data_ptr(),
                                 LN.data_ptr(), P.data_ptr(), Y.data_ptr(), G.data_ptr(),
                                 dpn.data_ptr(), dy0n.data_ptr(), None)
    torch.cuda.synchronize()
    assert rc == 0, L.last_error()
    assert np.array_equal(dpn.cpu().numpy(), dp) and np.array_equal(dy0n.cpu().numpy(), dy0)


def test_user_rejections_and_launch_count(tvi, users):
    import paper_2310_08649_gb300._lib as L
    lib = L.load()
    w = workloads.vdp(B=2, N=50, seed=67)
    model = users["vdp"].model(per_series=True)
    with pytest.raises(L.TviError) as e:
        forward_raise(tvi, model, w, tvi.Options(chunk=10, precision="bf16"))
    assert e.value.code == -7
    pred = torch.zeros(tvi_predictor_floats(lib), dtype=torch.float32, device="cuda")
    with pytest.raises(L.TviError) as e:
        forward_raise(tvi, model, w, tvi.Options(chunk=10, predictor=pred, predictor_chunk=10,
                                                 predictor_hidden=8))
    assert e.value.code == -7
    # kernels launched: one forward; adjoint with shared parameters adds the partial sum
    o = tvi.Options(chunk=10)
    y, _, _, rc = forward(tvi, model, w, o)
    k0 = lib.tvi_kernel_launches()
    forward(tvi, model, w, o)
    assert lib.tvi_kernel_launches() - k0 == 1
    lin = users["lin1"].model(per_series=False)
    wl = workloads.linear_stiff(B=3, N=40, n=1)
    yl, _, _, _ = forward(tvi, lin, wl, o)
    k0 = lib.tvi_kernel_launches()
    adjoint(tvi, lin, wl, o, yl, np.ones_like(yl))
    assert lib.tvi_kernel_launches() - k0 == 2


def forward_raise(tvi, model, w, o):
    return tvi.integrate(model, o, dev(w["y0"]), dev(w["times"]), dev(w["params"]))


def tvi_predictor_floats(lib):
    return lib.tvi_predictor_size(13, 8, 20)
