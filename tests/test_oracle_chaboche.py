"""Pins of the oracle's Chaboche viscoplastic model (TVO_CHABOCHE, Sec. 5.1.1)
against facts fixed by its mechanics and by the mathematics:

  * odd symmetry: (sigma, X, strain-rate amplitude) -> -(sigma, X, amplitude)
    maps h to (-sigma', K', -X') (a wrong sign or absolute value breaks it);
  * elastic range: below the yield surface |sigma - sum X| < K + sigma_0 the
    plastic rate vanishes, so sigma' is E times the applied strain rate, K
    relaxes and the backstresses stay put -- and the backward-Euler trajectory
    of an elastic loading is the explicit recursion of those linear equations;
  * steady state under a constant strain rate r: every backstress saturates
    at 2/3 C_i / g_i sign(r), K at K_inf, and |sigma - sum X| at
    K_inf + sigma_0 + eta r^(1/m) -- a fixed point that backward Euler keeps;
  * the Jacobian, the parameter VJP (all 2u + 8 parameters, the flow exponent
    included) and the adjoint gradient equal central differences.
"""
import numpy as np
import pytest

import workloads
from oracle import Model


def _model(u):
    return Model("chaboche", 2 + u, per_series=True)


def _params(u, seed, jitter=0.2):
    return workloads.chaboche(B=1, N=1, n_unit=u, jitter=jitter, seed=seed)["params"][0]


@pytest.mark.parametrize("u", [1, 3, 5])
def test_odd_symmetry(oracle_lib, u):
    g = np.random.default_rng(100 + u)
    m = _model(u)
    for trial in range(6):
        p = _params(u, 110 + trial)
        y = np.concatenate([[g.normal(0, 8)], [g.uniform(0, 5)], g.normal(0, 2, u)])
        t = g.uniform(0, 10)
        h = oracle_lib.rhs(m, p, y, t)
        pm = p.copy()
        pm[6 + 2 * u] = -p[6 + 2 * u]  # strain-rate amplitude
        ym = y.copy()
        ym[0], ym[2:] = -y[0], -y[2:]
        hm = oracle_lib.rhs(m, pm, ym, t)
        expect = np.concatenate([[-h[0]], [h[1]], -h[2:]])
        assert np.allclose(hm, expect, rtol=1e-14, atol=1e-14 * np.abs(h).max())


@pytest.mark.parametrize("u", [1, 2, 4])
def test_elastic_range(oracle_lib, u):
    g = np.random.default_rng(120 + u)
    m = _model(u)
    p = _params(u, 130 + u)
    E, s0, Kinf, tau = p[0], p[3], p[4], p[5]
    eda, T = p[6 + 2 * u], p[7 + 2 * u]
    for trial in range(5):
        K = g.uniform(0, 5)
        X = g.normal(0, 0.5, u)
        sigma = X.sum() + g.uniform(-1, 1) * 0.99 * (K + s0)  # inside the yield surface
        y = np.concatenate([[sigma], [K], X])
        t = g.uniform(0, 10)
        h = oracle_lib.rhs(m, p, y, t)
        assert h[0] == pytest.approx(E * eda * np.sin(2 * np.pi * t / T), rel=1e-14, abs=1e-15)
        assert h[1] == pytest.approx(tau * (Kinf - K), rel=1e-14)
        assert np.all(h[2:] == 0.0)


def test_elastic_trajectory_is_the_linear_recursion(oracle_lib):
    """Small amplitude: the loading never yields, so backward Euler reduces to
    sigma_k = sigma_{k-1} + dt E ed sin(2 pi t_k / T) and
    K_k = (K_{k-1} + dt tau K_inf) / (1 + dt tau), X_k = 0."""
    u = 2
    w = workloads.chaboche(B=3, N=500, n_unit=u, t_max=3.0)
    w["params"][:, 6 + 2 * u] = [0.01, 0.02, 0.05]
    m = _model(u)
    y, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-14)
    assert not st.any()
    for b in range(3):
        p = w["params"][b]
        E, Kinf, tau, eda, T = p[0], p[4], p[5], p[6 + 2 * u], p[7 + 2 * u]
        sig, K = 0.0, 0.0
        tb = w["times"][b]
        for k in range(1, tb.size):
            dt = tb[k] - tb[k - 1]
            sig += dt * E * eda * np.sin(2 * np.pi * tb[k] / T)
            K = (K + dt * tau * Kinf) / (1 + dt * tau)
            assert abs(y[b, k, 0] - sig) <= 1e-12 * max(1.0, abs(sig))
            assert abs(y[b, k, 1] - K) <= 1e-12 * max(1.0, abs(K))
        assert np.all(y[b, :, 2:] == 0.0)


@pytest.mark.parametrize("u", [1, 3])
def test_steady_state_under_constant_strain_rate(oracle_lib, u):
    """Times start at T/4 with T = 1e6, so the applied rate ed sin(2 pi t / T)
    stays within 1e-8 of ed over the span; the state must approach the closed-
    form fixed point."""
    m = _model(u)
    p = _params(u, 140 + u, jitter=0.0)
    T = 1e6
    p[7 + 2 * u] = T
    ed = 0.7
    p[6 + 2 * u] = ed
    N = 4000
    t0 = T / 4
    times = t0 + np.linspace(0.0, 200.0, N + 1)[None, :]
    y, _, st = oracle_lib.forward(m, np.zeros((1, 2 + u)), times, p[None, :], tol_abs=1e-12,
                                  max_iter=100)
    assert not st.any()
    E, mexp, eta, s0, Kinf = p[0], p[1], p[2], p[3], p[4]
    C, gm = p[6:6 + u], p[6 + u:6 + 2 * u]
    X_inf = 2.0 / 3.0 * C / gm
    s_inf = Kinf + s0 + eta * ed ** (1.0 / mexp)
    yN = y[0, -1]
    assert abs(yN[1] - Kinf) <= 1e-8 * Kinf
    assert np.allclose(yN[2:], X_inf, rtol=1e-6)
    assert abs((yN[0] - yN[2:].sum()) - s_inf) <= 1e-6 * s_inf


@pytest.mark.parametrize("side", [1.0, -1.0])  # sign of sigma - sum X
@pytest.mark.parametrize("u", [1, 4])
def test_jacobian_and_vjp_are_derivatives(oracle_lib, u, side):
    g = np.random.default_rng(150 + u)
    m = _model(u)
    p = _params(u, 160 + u)
    # a plastic state well away from the yield surface and from s = 0
    X = g.normal(0, 0.3, u)
    K = 2.0
    y = np.concatenate([[X.sum() + side * (K + p[3] + 1.5 * p[2]) * 1.3], [K], X])
    t = 0.37
    J = oracle_lib.jac(m, p, y, t)
    for c in range(2 + u):
        e = np.zeros(2 + u)
        e[c] = 1e-6
        fd = (oracle_lib.rhs(m, p, y + e, t) - oracle_lib.rhs(m, p, y - e, t)) / 2e-6
        assert np.allclose(J[:, c], fd, rtol=1e-6, atol=1e-7 * np.abs(J).max())
    a = g.standard_normal(2 + u)
    gp = oracle_lib.vjp_p(m, p, y, a, t)
    for q in range(2 * u + 8):
        hq = 1e-6 * abs(p[q])
        pp, pm = p.copy(), p.copy()
        pp[q] += hq
        pm[q] -= hq
        fd = a @ (oracle_lib.rhs(m, pp, y, t) - oracle_lib.rhs(m, pm, y, t)) / (2 * hq)
        assert abs(gp[q] - fd) <= 1e-6 * max(abs(fd), 1e-9 * np.abs(gp).max()), (q, gp[q], fd)


def test_adjoint_against_finite_differences(oracle_lib):
    u = 2
    w = workloads.chaboche(B=2, N=300, n_unit=u, t_max=1.5, jitter=0.1, seed=170)
    w["params"][:, 6 + 2 * u] *= 4.0  # strong loading: the trajectory yields
    m = _model(u)
    W = np.random.default_rng(171).standard_normal((2, 301, 2 + u))

    def loss(y0, params):
        y, _, _ = oracle_lib.forward(m, y0, w["times"], params, tol_abs=1e-14, max_iter=60)
        return float((W * y).sum())

    y, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-14,
                                  max_iter=60)
    assert not st.any()
    assert (np.abs(y[:, :, 2:]).max() > 1e-3)  # plastic flow happened
    dp, dy0 = oracle_lib.adjoint(m, w["times"], w["params"], y, W)
    P = w["params"]
    for b in range(2):
        for q in range(2 * u + 8):
            h = 1e-6 * abs(P[b, q])
            Pp, Pm = P.copy(), P.copy()
            Pp[b, q] += h
            Pm[b, q] -= h
            fd = (loss(w["y0"], Pp) - loss(w["y0"], Pm)) / (2 * h)
            assert abs(dp[b, q] - fd) <= 1e-5 * max(abs(fd), 1e-4 * np.abs(dp[b]).max()), \
                (b, q, dp[b, q], fd)
        for i in range(2 + u):
            h = 1e-6
            yp, ym = w["y0"].copy(), w["y0"].copy()
            yp[b, i] += h
            ym[b, i] -= h
            fd = (loss(yp, P) - loss(ym, P)) / (2 * h)
            assert abs(dy0[b, i] - fd) <= 1e-5 * max(abs(fd), 1.0)
