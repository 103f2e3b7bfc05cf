"""Pins of the oracle's mass-damper-spring model (TVO_MDS, Sec. 5.1.1) against
facts fixed by mechanics and by the mathematics, not by its own formulas:

  * work-energy theorem: for E = 1/2 sum M_i v_i^2 + 1/2 sum K_i (d_{i+1} - d_i)^2
    (d_{u+1} = 0), dE/dt along h equals minus the damper dissipation
    sum C_i (v_{i+1} - v_i)^2 plus the power M_1 v_1 f(t) of the applied forcing
    (a dropped term, a wrong sign or index in h breaks it);
  * the Jacobian and the parameter VJP are derivatives of h (central
    differences; h is linear in y, quadratic-free in K and C);
  * the backward-Euler trajectory of this linear forced system equals the
    modal recursion z_k = (z_{k-1} + dt c(t_k)) / (1 - dt lambda) in the
    eigenbasis of the matrix read off h by finite differences;
  * the adjoint gradient (all 3u + 2 parameters, and y0) equals central
    differences of the discrete loss.
"""
import numpy as np
import pytest

import workloads
from oracle import Model


def _model(u):
    return Model("mds", 2 * u, per_series=True)


def _random_state(g, u):
    return g.standard_normal(2 * u) * np.concatenate([np.full(u, 1e-3), np.full(u, 1e-1)])


def _params(u, seed):
    return workloads.mds(B=1, N=1, n_unit=u, jitter=0.3, seed=seed)["params"][0]


def _energy(u, p, y):
    K, M = p[:u], p[2 * u:3 * u]
    d, v = y[:u], y[u:]
    dn = np.append(d[1:], 0.0)
    return 0.5 * np.sum(M * v * v) + 0.5 * np.sum(K * (dn - d) ** 2)


@pytest.mark.parametrize("u", [1, 2, 3, 5])
def test_work_energy_theorem(oracle_lib, u):
    g = np.random.default_rng(10 + u)
    m = _model(u)
    for trial in range(5):
        p = _params(u, 20 + 7 * u + trial)
        y = _random_state(g, u)
        t = g.uniform(0.0, 1.0)
        h = oracle_lib.rhs(m, p, y, t)
        # dE/dt = grad E . h, gradient of E by central differences (E is quadratic: exact)
        grad = np.empty(2 * u)
        for i in range(2 * u):
            e = np.zeros(2 * u)
            e[i] = 1e-3 * max(abs(y[i]), 1e-6)
            grad[i] = (_energy(u, p, y + e) - _energy(u, p, y - e)) / (2 * e[i])
        C, M, fa, T = p[u:2 * u], p[2 * u:3 * u], p[3 * u], p[3 * u + 1]
        v = y[u:]
        vn = np.append(v[1:], 0.0)
        power = -np.sum(C * (vn - v) ** 2) + M[0] * v[0] * fa * np.sin(2 * np.pi * t / T)
        scale = np.sum(np.abs(grad * h)) + abs(power)
        assert abs(grad @ h - power) <= 1e-9 * scale, (u, trial, grad @ h, power)


@pytest.mark.parametrize("u", [1, 2, 4])
def test_jacobian_and_vjp_are_derivatives(oracle_lib, u):
    g = np.random.default_rng(30 + u)
    m = _model(u)
    p = _params(u, 40 + u)
    y = _random_state(g, u)
    t = 0.37
    J = oracle_lib.jac(m, p, y, t)
    for c in range(2 * u):
        e = np.zeros(2 * u)
        e[c] = 1e-4
        fd = (oracle_lib.rhs(m, p, y + e, t) - oracle_lib.rhs(m, p, y - e, t)) / 2e-4
        assert np.allclose(J[:, c], fd, rtol=1e-7, atol=1e-7 * np.abs(J).max())
    a = g.standard_normal(2 * u)
    gp = oracle_lib.vjp_p(m, p, y, a, t)
    for q in range(3 * u + 2):
        # h is linear in K, C and f_a (long steps: no truncation, less rounding);
        # M enters as 1/M, T through sin(2 pi t / T) with a phase of many radians
        rel = 1e-2 if (q < 2 * u or q == 3 * u) else (1e-7 if q == 3 * u + 1 else 1e-5)
        hq = rel * abs(p[q])
        pp, pm = p.copy(), p.copy()
        pp[q] += hq
        pm[q] -= hq
        fd = a @ (oracle_lib.rhs(m, pp, y, t) - oracle_lib.rhs(m, pm, y, t)) / (2 * hq)
        assert abs(gp[q] - fd) <= 1e-6 * max(abs(fd), 1e-12 * np.abs(gp).max()), (q, gp[q], fd)


@pytest.mark.parametrize("u", [1, 2, 3])
def test_trajectory_modal_closed_form(oracle_lib, u):
    w = workloads.mds(B=4, N=400, n_unit=u, t_max=0.2, jitter=0.2, seed=50 + u)
    m = _model(u)
    y, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-16)
    assert not st.any()
    n = 2 * u
    for b in range(4):
        p = w["params"][b]
        # matrix of the linear part and forcing vector, read off h
        zero = np.zeros(n)
        A = np.empty((n, n))
        for c in range(n):
            e = np.zeros(n)
            e[c] = 1.0
            A[:, c] = oracle_lib.rhs(m, p, e, 0.0) - oracle_lib.rhs(m, p, zero, 0.0)
        lam, V = np.linalg.eig(A)
        Vinv = np.linalg.inv(V)
        tb = w["times"][b]
        z = Vinv @ w["y0"][b].astype(complex)
        worst = 0.0
        for k in range(1, tb.size):
            dt = tb[k] - tb[k - 1]
            c = Vinv @ oracle_lib.rhs(m, p, zero, tb[k])
            z = (z + dt * c) / (1.0 - dt * lam)
            worst = max(worst, np.abs((V @ z).real - y[b, k]).max())
        assert worst <= 1e-9 * np.abs(y[b]).max(), (b, worst)


def test_adjoint_against_finite_differences(oracle_lib):
    u = 2
    w = workloads.mds(B=2, N=120, n_unit=u, t_max=0.05, jitter=0.2, seed=61)
    w["y0"] = np.random.default_rng(62).standard_normal((2, 2 * u)) * 1e-4
    m = _model(u)
    W = np.random.default_rng(63).standard_normal((2, 121, 2 * u))

    def loss(y0, params):
        y, _, _ = oracle_lib.forward(m, y0, w["times"], params, tol_abs=1e-18, max_iter=5)
        return float((W * y).sum())

    y, _, _ = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-18, max_iter=5)
    dp, dy0 = oracle_lib.adjoint(m, w["times"], w["params"], y, W)
    P = w["params"]
    for b in range(2):
        for q in range(3 * u + 2):
            h = 1e-6 * abs(P[b, q])
            Pp, Pm = P.copy(), P.copy()
            Pp[b, q] += h
            Pm[b, q] -= h
            fd = (loss(w["y0"], Pp) - loss(w["y0"], Pm)) / (2 * h)
            assert abs(dp[b, q] - fd) <= 2e-5 * max(abs(fd), 1e-3 * np.abs(dp[b]).max()), \
                (b, q, dp[b, q], fd)
        for i in range(2 * u):
            h = 1e-7
            yp, ym = w["y0"].copy(), w["y0"].copy()
            yp[b, i] += h
            ym[b, i] -= h
            fd = (loss(yp, P) - loss(ym, P)) / (2 * h)
            assert abs(dy0[b, i] - fd) <= 1e-6 * max(abs(fd), 1.0)
