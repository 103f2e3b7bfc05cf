"""Pins of the oracle's coupled neuron model (TVO_NEURON, Sec. 5.1.1):

  * the gating variables relax linearly and independently, so their backward-
    Euler values are the closed-form recursion m_k = (m_{k-1} + dt m_inf /
    tau_m) / (1 + dt / tau_m) (h and n alike);
  * with the gates started at their limits they stay there, the voltage
    equation of one neuron is linear with constant coefficients, and its
    backward-Euler trajectory is the closed-form recursion of that equation
    (pins the conductances, the reversal potentials and the applied current);
  * the coupling exchanges current only: sum_i C_i V_i' is unchanged by it
    when every neuron has the same coupling conductance, and two identical
    neurons started alike stay identical;
  * the Jacobian, the parameter VJP (all 15 u + 1) and the adjoint gradient
    equal central differences.
"""
import numpy as np
import pytest

import workloads
from oracle import Model


def _model(u):
    return Model("neuron", 4 * u, per_series=True)


def test_gating_closed_form(oracle_lib):
    u = 2
    w = workloads.neuron(B=3, N=400, n_unit=u, jitter=0.2, seed=200)
    m = _model(u)
    y, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-14)
    assert not st.any()
    for b in range(3):
        p = w["params"][b]
        tb = w["times"][b]
        for i in range(u):
            q = p[15 * i:15 * i + 15]
            for comp, (inf, tau) in enumerate([(q[7], q[8]), (q[9], q[10]), (q[11], q[12])]):
                v = 0.0
                for k in range(1, tb.size):
                    dt = tb[k] - tb[k - 1]
                    v = (v + dt * inf / tau) / (1 + dt / tau)
                    assert abs(y[b, k, 4 * i + 1 + comp] - v) <= 1e-13


def test_single_neuron_voltage_closed_form(oracle_lib):
    w = workloads.neuron(B=4, N=500, n_unit=1, jitter=0.2, seed=201)
    m = _model(1)
    p = w["params"]
    w["y0"][:, 1], w["y0"][:, 2], w["y0"][:, 3] = p[:, 7], p[:, 9], p[:, 11]  # gates at rest
    y, _, st = oracle_lib.forward(m, w["y0"], w["times"], p, tol_abs=1e-14)
    assert not st.any()
    for b in range(4):
        C, gNa, ENa, gK, EK, gL, EL = p[b, :7]
        m3h = p[b, 7] ** 3 * p[b, 9]
        n4 = p[b, 11] ** 4
        a = gNa * m3h + gK * n4 + gL
        c0 = gNa * m3h * ENa + gK * n4 * EK + gL * EL
        Ia, T = p[b, 15], p[b, 14]
        tb = w["times"][b]
        V = 0.0
        for k in range(1, tb.size):
            dt = tb[k] - tb[k - 1]
            V = (V + dt * (c0 + Ia * np.sin(2 * np.pi * tb[k] / T)) / C) / (1 + dt * a / C)
            assert abs(y[b, k, 0] - V) <= 1e-12 * max(1.0, abs(V))
        assert np.all(np.abs(y[b, :, 1:] - y[b, 0, 1:]) <= 1e-15)


def test_coupling_exchanges_current_only(oracle_lib):
    g = np.random.default_rng(202)
    u = 3
    m = _model(u)
    p = workloads.neuron(B=1, N=1, n_unit=u, jitter=0.2, seed=203)["params"][0]
    gc = p[13]
    for i in range(u):
        p[15 * i + 13] = gc  # one coupling conductance
    p0 = p.copy()
    for i in range(u):
        p0[15 * i + 13] = 0.0
    for trial in range(5):
        y = g.uniform(0.0, 1.0, 4 * u)
        y[0::4] = g.normal(0.0, 1.0, u)
        t = g.uniform(0.0, 10.0)
        C = p[0::15][:u]
        h1, h0 = oracle_lib.rhs(m, p, y, t), oracle_lib.rhs(m, p0, y, t)
        dq = (h1 - h0)[0::4] * C  # coupling currents (a difference of O(1) terms)
        scale = np.abs(h1[0::4] * C).max() + np.abs(h0[0::4] * C).max()
        assert abs(dq.sum()) <= 1e-14 * scale
        assert np.abs(dq).max() > 1e-6


def test_identical_neurons_stay_identical(oracle_lib):
    w = workloads.neuron(B=2, N=300, n_unit=2, jitter=0.0)
    q = w["params"][:, :15].copy()
    w["params"][:, 15:30] = q  # neuron 2 := neuron 1
    m = _model(2)
    y, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-14)
    assert not st.any()
    # equal up to the rounding of the dense LU, which orders the two neurons
    assert np.abs(y[:, :, :4] - y[:, :, 4:]).max() <= 1e-12 * np.abs(y).max()


@pytest.mark.parametrize("u", [1, 2])
def test_jacobian_and_vjp_are_derivatives(oracle_lib, u):
    g = np.random.default_rng(210 + u)
    m = _model(u)
    p = workloads.neuron(B=1, N=1, n_unit=u, jitter=0.2, seed=211)["params"][0]
    y = g.uniform(0.1, 0.9, 4 * u)
    y[0::4] = g.normal(0.0, 1.0, u)
    t = 0.77
    J = oracle_lib.jac(m, p, y, t)
    for c in range(4 * u):
        e = np.zeros(4 * u)
        e[c] = 1e-6
        fd = (oracle_lib.rhs(m, p, y + e, t) - oracle_lib.rhs(m, p, y - e, t)) / 2e-6
        assert np.allclose(J[:, c], fd, rtol=1e-6, atol=1e-8 * np.abs(J).max())
    a = g.standard_normal(4 * u)
    gp = oracle_lib.vjp_p(m, p, y, a, t)
    for q in range(15 * u + 1):
        hq = 1e-6 * abs(p[q])
        pp, pm = p.copy(), p.copy()
        pp[q] += hq
        pm[q] -= hq
        fd = a @ (oracle_lib.rhs(m, pp, y, t) - oracle_lib.rhs(m, pm, y, t)) / (2 * hq)
        assert abs(gp[q] - fd) <= 1e-6 * max(abs(fd), 1e-8 * np.abs(gp).max()), (q, gp[q], fd)


def test_adjoint_against_finite_differences(oracle_lib):
    u = 2
    w = workloads.neuron(B=2, N=150, n_unit=u, t_max=3.0, jitter=0.2, seed=220)
    m = _model(u)
    W = np.random.default_rng(221).standard_normal((2, 151, 4 * u))

    def loss(y0, params):
        y, _, _ = oracle_lib.forward(m, y0, w["times"], params, tol_abs=1e-14)
        return float((W * y).sum())

    y, _, _ = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-14)
    dp, dy0 = oracle_lib.adjoint(m, w["times"], w["params"], y, W)
    P = w["params"]
    for b in range(2):
        for q in range(15 * u + 1):
            h = 1e-6 * abs(P[b, q])
            Pp, Pm = P.copy(), P.copy()
            Pp[b, q] += h
            Pm[b, q] -= h
            fd = (loss(w["y0"], Pp) - loss(w["y0"], Pm)) / (2 * h)
            assert abs(dp[b, q] - fd) <= 1e-5 * max(abs(fd), 1e-4 * np.abs(dp[b]).max()), \
                (b, q, dp[b, q], fd)
        for i in range(4 * u):
            h = 1e-6
            yp, ym = w["y0"].copy(), w["y0"].copy()
            yp[b, i] += h
            ym[b, i] -= h
            fd = (loss(yp, P) - loss(ym, P)) / (2 * h)
            assert abs(dy0[b, i] - fd) <= 1e-5 * max(abs(fd), 1.0)
