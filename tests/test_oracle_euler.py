"""Pins of the forward-Euler oracle (tvo_forward_euler / tvo_adjoint_euler)
against facts fixed by the mathematics:
  * forward on a linear system  -> y_k = Q diag((1 - dt lam)^k) Q^T y0 exactly
  * adjoint on a linear system  -> closed-form dL/dlambda and dL/dy0
  * nonlinear gradients         -> central finite differences of the discrete loss
  * padding (dt = 0)            -> the state and the gradients are unchanged
"""
import numpy as np

import workloads
from oracle import Model


def _relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _linear(B=4, N=300):
    # eigenvalues up to 100 with dt = 1/N: 1 - dt lam stays in (0, 1)
    return workloads.linear_stiff(B=B, N=N, lam_decades=(0.0, 2.0))


def test_linear_forward_closed_form(oracle_lib):
    w = _linear()
    m = Model.from_spec(w["spec"])
    y, st = oracle_lib.forward_euler(m, w["y0"], w["times"], w["params"])
    assert not st.any()
    Q, lam = w["Q"], w["lam"]
    dt = w["times"][0, 1] - w["times"][0, 0]
    d = 1.0 - dt * lam
    z0 = w["y0"] @ Q
    k = np.arange(w["times"].shape[1])
    exact = np.einsum("kn,bn,mn->bkm", d[None, :] ** k[:, None], z0, Q)
    assert _relerr(y, exact) < 1e-12


def test_linear_adjoint_closed_form(oracle_lib):
    """L = sum_b sum_{k>=1} |y_k|^2, y_k = Q D^k z0, D = diag(1 - dt lam):
    dL/dlam_m = -2 dt sum_b z0_m^2 sum_k k d_m^(2k-1), and dL/dlam_m = -q_m^T (dL/dA) q_m;
    dL/dy0 = 2 sum_{k>=1} Q D^(2k) Q^T y0."""
    w = _linear()
    m = Model.from_spec(w["spec"])
    y, _ = oracle_lib.forward_euler(m, w["y0"], w["times"], w["params"])
    g = 2.0 * y
    g[:, 0] = 0.0
    dA, dy0 = oracle_lib.adjoint_euler(m, w["times"], w["params"], y, g)
    Q, lam = w["Q"], w["lam"]
    dlam = -np.einsum("im,ij,jm->m", Q, dA.reshape(4, 4), Q)
    dt = w["times"][0, 1]
    d = 1.0 - dt * lam
    z0 = w["y0"] @ Q
    N = w["times"].shape[1] - 1
    k = np.arange(1, N + 1)[:, None]
    expect = -2.0 * dt * (z0 ** 2).sum(0) * (k * d[None, :] ** (2 * k - 1)).sum(0)
    assert _relerr(dlam, expect) < 1e-10
    s = (d[None, :] ** (2 * k)).sum(0)
    expect_y0 = 2.0 * (z0 * s[None, :]) @ Q.T
    assert _relerr(dy0, expect_y0) < 1e-10


def _loss(oracle_lib, m, w, y0, params, W):
    y, _ = oracle_lib.forward_euler(m, y0, w["times"], params, lengths=w.get("lengths"))
    return float((W * y).sum())


def _check_fd(oracle_lib, m, w, seed):
    g = np.random.default_rng(seed)
    B, n = w["y0"].shape
    N = w["times"].shape[1] - 1
    W = g.standard_normal((B, N + 1, n))
    y, st = oracle_lib.forward_euler(m, w["y0"], w["times"], w["params"],
                                     lengths=w.get("lengths"))
    assert not st.any()
    dp, dy0 = oracle_lib.adjoint_euler(m, w["times"], w["params"], y, W, lengths=w.get("lengths"))
    P = w["params"]
    flat = P.reshape(-1)
    for i in g.choice(flat.size, size=min(8, flat.size), replace=False):
        h = 1e-6 * max(1.0, abs(flat[i]))
        Pp, Pm = flat.copy(), flat.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (_loss(oracle_lib, m, w, w["y0"], Pp.reshape(P.shape), W)
              - _loss(oracle_lib, m, w, w["y0"], Pm.reshape(P.shape), W)) / (2 * h)
        assert abs(dp.reshape(-1)[i] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, dp.reshape(-1)[i], fd)
    for b in range(B):
        for i in range(n):
            h = 1e-6
            yp, ym = w["y0"].copy(), w["y0"].copy()
            yp[b, i] += h
            ym[b, i] -= h
            fd = (_loss(oracle_lib, m, w, yp, P, W) - _loss(oracle_lib, m, w, ym, P, W)) / (2 * h)
            assert abs(dy0[b, i] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_vdp_gradients_against_finite_differences(oracle_lib):
    # mu in [10, 100] on the shortened span of this workload: explicit steps stay bounded
    w = workloads.vdp(B=3, N=400, seed=23, mu_decades=(1.0, 2.0))
    _check_fd(oracle_lib, Model.from_spec(w["spec"]), w, 6)


def test_mlp_gradients_against_finite_differences(oracle_lib):
    w = workloads.mlp_ode(B=2, N=80, n=4, hidden=(6, 5), t_end=2.0)
    w["params"] = w["params"] + 0.05 * np.random.default_rng(7).standard_normal(
        w["params"].shape)
    _check_fd(oracle_lib, Model.from_spec(w["spec"]), w, 8)


def test_padding_keeps_state_and_gradient(oracle_lib):
    w = workloads.vdp(B=2, N=300, seed=24, mu_decades=(1.0, 2.0))
    m = Model.from_spec(w["spec"])
    lens = np.array([300, 170], dtype=np.int32)
    y, _ = oracle_lib.forward_euler(m, w["y0"], w["times"], w["params"], lengths=lens)
    assert np.all(y[1, 171:] == y[1, 170])
    short = dict(w, times=w["times"][1:2, :171], y0=w["y0"][1:2], params=w["params"][1:2])
    ys, _ = oracle_lib.forward_euler(m, short["y0"], short["times"], short["params"])
    assert np.array_equal(ys[0], y[1, :171])
    g = np.random.default_rng(9).standard_normal(y.shape)
    g[1, 171:] = 0.0
    dp, dy0 = oracle_lib.adjoint_euler(m, w["times"], w["params"], y, g, lengths=lens)
    dps, dy0s = oracle_lib.adjoint_euler(m, short["times"], short["params"], ys, g[1:2, :171])
    assert abs(dp[1, 0] - dps[0, 0]) <= 1e-12 * abs(dps[0, 0])
    assert np.allclose(dy0[1], dy0s[0], rtol=1e-12, atol=0)
