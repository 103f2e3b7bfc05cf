"""Pins of the CPU oracle against facts fixed by the mathematics, not by itself.

Each test names what it pins:
  * backward-Euler forward on a linear system -> exact closed-form recursion
  * discrete adjoint on a linear system       -> closed-form dL/dlambda and dL/dy0
  * gradients of nonlinear models             -> central finite differences
  * model h, dh/dy, dh/dp                     -> torch library ops / autograd
  * nonlinear step root                       -> scipy.optimize.fsolve per step
  * independent step solves                   -> closed-form linear step, the forward
                                                 trajectory itself
  * forward-error estimate                    -> closed-form propagation on a
                                                 non-symmetric linear system; the
                                                 observed tol vs tol/1000 difference
  * padding (dt = 0) and series independence  -> invariants
"""
import numpy as np
import pytest

import workloads
from oracle import Model

TOL_TIGHT = 1e-13


def _relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# --------------------------------------------------------------------------
# Linear stiff system: y_k = Q diag((1 + dt lam)^-k) Q^T y0 (exact BE recursion,
# Sec. 2.2 Eq. backward-euler with h = A y, A = -Q diag(lam) Q^T).
# --------------------------------------------------------------------------
def test_linear_forward_closed_form(oracle_lib):
    w = workloads.linear_stiff()
    m = Model.from_spec(w["spec"])
    y, iters, status = oracle_lib.forward(m, w["y0"], w["times"], w["params"],
                                          tol_abs=TOL_TIGHT, max_iter=5)
    assert not status.any()
    # linear: one Newton update solves each step exactly (up to rounding)
    assert iters.max() <= 2
    Q, lam = w["Q"], w["lam"]
    dt = w["times"][0, 1] - w["times"][0, 0]
    d = 1.0 / (1.0 + dt * lam)
    z0 = w["y0"] @ Q  # [B][n] = Q^T y0 per series
    N = w["times"].shape[1] - 1
    k = np.arange(N + 1)
    exact = np.einsum("kn,bn,mn->bkm", d[None, :] ** k[:, None], z0, Q)
    assert _relerr(y, exact) < 1e-12


def test_linear_adjoint_closed_form(oracle_lib):
    """L = sum_b sum_{k>=1} |y_k|^2.  With z0 = Q^T y0 and d_m = 1/(1 + dt lam_m):
    dL/dlam_m = -2 dt sum_b z0_m^2 sum_k k d_m^(2k+1) and, since A = -Q diag(lam) Q^T,
    dL/dlam_m = -q_m^T (dL/dA) q_m.  Also dL/dy0 = 2 sum_k Q D^(2k) Q^T y0."""
    w = workloads.linear_stiff(B=4, N=300)
    m = Model.from_spec(w["spec"])
    y, _, status = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=TOL_TIGHT)
    assert not status.any()
    g = 2.0 * y
    g[:, 0] = 0.0
    dA, dy0 = oracle_lib.adjoint(m, w["times"], w["params"], y, g)
    Q, lam = w["Q"], w["lam"]
    G = dA.reshape(4, 4)
    dlam = -np.einsum("im,ij,jm->m", Q, G, Q)
    dt = w["times"][0, 1]
    d = 1.0 / (1.0 + dt * lam)
    z0 = w["y0"] @ Q
    kk = np.arange(1, 301)[:, None]
    exact = -2.0 * dt * (z0 ** 2).sum(0) * (kk * d[None, :] ** (2 * kk + 1)).sum(0)
    assert _relerr(dlam, exact) < 1e-10
    exact_dy0 = 2.0 * np.einsum("bm,m,im->bi", z0, (d[None, :] ** (2 * kk)).sum(0), Q)
    assert _relerr(dy0, exact_dy0) < 1e-10


# --------------------------------------------------------------------------
# Model functions against torch library ops and autograd.
# --------------------------------------------------------------------------
def _torch_mlp(p, n, hidden, kind):
    import torch
    h1, h2 = hidden
    sizes = [(h1, n), (h2, h1), (n, h2)]
    t = torch.tensor(p, dtype=torch.float64)
    layers, off = [], 0
    for (o, i) in sizes:
        W = t[off:off + o * i].reshape(o, i)
        off += o * i
        b = t[off:off + o]
        off += o
        layers.append((W, b))
    act = torch.tanh if kind == "mlp_tanh" else torch.nn.functional.silu

    def f(y, params_layers=layers):
        (W1, b1), (W2, b2), (W3, b3) = params_layers
        a = act(torch.nn.functional.linear(y, W1, b1))
        a = act(torch.nn.functional.linear(a, W2, b2))
        z = torch.nn.functional.linear(a, W3, b3)
        return torch.tanh(z) if kind == "mlp_tanh" else z
    return f, t


@pytest.mark.parametrize("kind,n,hidden", [("mlp_tanh", 16, (64, 64)), ("mlp_silu", 32, (128, 128)),
                                           ("mlp_tanh", 3, (5, 4)), ("mlp_silu", 2, (3, 7))])
def test_mlp_rhs_jac_vjp_against_torch(oracle_lib, kind, n, hidden):
    import torch
    g = np.random.default_rng(11)
    m = Model(kind, n, hidden)
    p = g.uniform(-0.6, 0.6, oracle_lib.param_count(m))
    f, pt = _torch_mlp(p, n, hidden, kind)
    for _ in range(3):
        y = g.standard_normal(n)
        yt = torch.tensor(y, dtype=torch.float64)
        assert _relerr(oracle_lib.rhs(m, p, y), f(yt).numpy()) < 1e-14
        J = torch.autograd.functional.jacobian(f, yt).numpy()
        assert _relerr(oracle_lib.jac(m, p, y), J) < 1e-13
        a = g.standard_normal(n)
        ptr = pt.clone().requires_grad_(True)
        f2, _ = _torch_mlp(p, n, hidden, kind)
        # rebuild layers from the differentiable flat vector
        h1, h2 = hidden
        off, layers = 0, []
        for (o, i) in [(h1, n), (h2, h1), (n, h2)]:
            W = ptr[off:off + o * i].reshape(o, i)
            off += o * i
            b = ptr[off:off + o]
            off += o
            layers.append((W, b))
        out = f2(yt, layers)
        (out * torch.tensor(a)).sum().backward()
        assert _relerr(oracle_lib.vjp_p(m, p, y, a, scale=0.5), 0.5 * ptr.grad.numpy()) < 1e-13


def test_vdp_and_linear_model_functions(oracle_lib):
    m = Model("vdp", 2, per_series=True)
    # h = [y2, mu (1 - y1^2) y2 - y1] at mu = 2, y = (0.5, 1): [1, 2 * 0.75 - 0.5] = [1, 1]
    assert np.allclose(oracle_lib.rhs(m, [2.0], [0.5, 1.0]), [1.0, 1.0], rtol=0, atol=1e-15)
    g = np.random.default_rng(3)
    for _ in range(5):
        mu, y = 10 ** g.uniform(1, 3), g.uniform(-2, 2, 2)
        eps = 1e-6
        J = np.stack([(oracle_lib.rhs(m, [mu], y + eps * e) - oracle_lib.rhs(m, [mu], y - eps * e))
                      / (2 * eps) for e in np.eye(2)], axis=1)
        assert _relerr(oracle_lib.jac(m, [mu], y), J) < 1e-8
        a = g.standard_normal(2)
        dmu = (oracle_lib.rhs(m, [mu + eps], y) - oracle_lib.rhs(m, [mu - eps], y)) / (2 * eps)
        assert np.isclose(oracle_lib.vjp_p(m, [mu], y, a)[0], a @ dmu, rtol=1e-8, atol=1e-12)
    ml = Model("linear", 4)
    A = g.standard_normal((4, 4))
    y = g.standard_normal(4)
    assert _relerr(oracle_lib.rhs(ml, A.ravel(), y), A @ y) < 1e-15
    assert _relerr(oracle_lib.jac(ml, A.ravel(), y), A) == 0
    a = g.standard_normal(4)
    assert _relerr(oracle_lib.vjp_p(ml, A.ravel(), y, a), np.outer(a, y).ravel()) < 1e-15


# --------------------------------------------------------------------------
# Nonlinear steps: each BE step against an independent library root finder.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["vdp", "mlp"])
def test_be_steps_against_scipy_fsolve(oracle_lib, which):
    from scipy.optimize import fsolve
    if which == "vdp":
        w = workloads.vdp(B=4, N=400)
    else:
        w = workloads.mlp_ode(B=2, N=60, n=4, hidden=(8, 8))
    m = Model.from_spec(w["spec"])
    y, _, status = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=TOL_TIGHT,
                                      max_iter=60)
    for b in range(w["y0"].shape[0]):
        p = w["params"][b] if m.per_series else w["params"]
        yp = w["y0"][b].copy()
        for k in range(1, w["times"].shape[1]):
            dt = w["times"][b, k] - w["times"][b, k - 1]

            def G(x, yp=yp, dt=dt):
                return x - yp - dt * oracle_lib.rhs(m, p, x)
            x = fsolve(G, yp, xtol=1e-14, full_output=False)
            scale = max(np.abs(x).max(), 1.0)
            assert np.abs(y[b, k] - x).max() <= 1e-9 * scale, (b, k)
            yp = x


# --------------------------------------------------------------------------
# Independent step solves: out_k solves step k from the GIVEN y_{k-1}.
# --------------------------------------------------------------------------
def _nonsym_linear(seed, n=4, lam_decades=(0.0, 3.0)):
    """A = -V diag(lam) V^-1 with V a seeded well-conditioned non-orthogonal matrix,
    so A != A^T (a transposed operand changes every result below)."""
    g = np.random.default_rng(seed)
    V = np.eye(n) + 0.4 * g.standard_normal((n, n))
    lam = 10.0 ** g.uniform(lam_decades[0], lam_decades[1], n)
    Vi = np.linalg.inv(V)
    return -(V * lam[None, :]) @ Vi, V, Vi, lam


def test_step_solves_linear_closed_form(oracle_lib):
    """Linear h = A y: the BE step from any state x is (I - dt A)^-1 x =
    V diag(1 / (1 + dt lam)) V^-1 x, here from states that are NOT a BE trajectory
    (random draws) and on per-series non-uniform grids."""
    A, V, Vi, lam = _nonsym_linear(101)
    B, N = 3, 40
    g = np.random.default_rng(102)
    yprev = g.standard_normal((B, N + 1, 4))
    times = workloads.random_times(103, B, N, t_end=0.05)
    m = Model("linear", 4)
    out, st = oracle_lib.step_solves(m, times, A.reshape(-1), yprev)
    assert not st.any()
    assert np.array_equal(out[:, 0], yprev[:, 0])
    dt = np.diff(times, axis=1)  # [B][N]
    z = np.einsum("ij,bkj->bki", Vi, yprev[:, :-1])  # V^-1 y_{k-1}
    exact = np.einsum("ij,bkj->bki", V, z / (1.0 + dt[..., None] * lam[None, None, :]))
    assert _relerr(out[:, 1:], exact) < 1e-12


@pytest.mark.parametrize("which", ["vdp", "mds"])
def test_step_solves_reproduce_forward(oracle_lib, which):
    """Fed the oracle's own trajectory, every independent step solve starts where the
    step-by-step integration started and runs the same Newton, so it reproduces the
    trajectory exactly (an index slip between y_{k-1}, t_k and dt_k would not);
    the time-dependent mass-damper-spring model checks t_k."""
    if which == "vdp":
        w = workloads.vdp(B=6, N=700, seed=104)
    else:
        w = workloads.mds(B=4, N=300, n_unit=2, jitter=0.2)
    m = Model.from_spec(w["spec"])
    tol = 1e-12 if which == "vdp" else 1e-18
    y, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=tol, max_iter=60)
    assert not st.any()
    out, st2 = oracle_lib.step_solves(m, w["times"], w["params"], y, tol_abs=tol, max_iter=60)
    assert not st2.any()
    assert np.array_equal(out, y)
    # shifting the states by one step breaks it
    shifted = y.copy()
    shifted[:, 1:] = y[:, :-1]
    out2, _ = oracle_lib.step_solves(m, w["times"], w["params"], shifted, tol_abs=tol)
    assert not np.array_equal(out2, y)


# --------------------------------------------------------------------------
# Forward-error estimate (random residuals propagated through the linearised
# BE recursion d_k = A_k^-1 (d_{k-1} + r_k)).
# --------------------------------------------------------------------------
def test_forward_error_estimate_linear_closed_form(oracle_lib):
    """On a linear system with uniform steps A_k = I - dt A for every k, so the
    propagated perturbation has the closed form d_k = sum_{m<=k} (I - dt A)^-(k-m+1) r_m,
    evaluated here as one lower-triangular Toeplitz product per eigenvalue of A
    (V^-1 r in, V out), from the same random draws as the estimate."""
    A, V, Vi, lam = _nonsym_linear(105, lam_decades=(0.0, 2.0))
    B, N, n, tol, trials, seed = 3, 60, 4, 1e-9, 3, 7
    times = workloads.uniform_times(B, N, 0.3)
    dt = times[0, 1]
    g = np.random.default_rng(106)
    y = g.standard_normal((B, N + 1, n))  # only its scale enters
    m = Model("linear", 4)
    est = oracle_lib.forward_error_estimate(m, times, A.reshape(-1), y, tol, trials=trials,
                                            seed=seed)
    rg = np.random.default_rng(seed)
    k = np.arange(N)
    expo = k[:, None] - k[None, :] + 1  # k - m + 1 for m <= k
    lower = expo >= 1
    want = np.zeros(B)
    for _ in range(trials):
        r = rg.uniform(-tol, tol, (B, N, n))
        s = np.einsum("ij,bmj->bmi", Vi, r)
        z = np.zeros((B, N, n), dtype=complex if np.iscomplexobj(lam) else float)
        for i in range(n):
            T = np.where(lower, (1.0 / (1.0 + dt * lam[i])) ** np.maximum(expo, 1), 0.0)
            z[:, :, i] = s[:, :, i] @ T.T
        d = np.einsum("ij,bkj->bki", V, z).real
        want = np.maximum(want, np.abs(d).max(axis=(1, 2)) / np.abs(y).max(axis=(1, 2)))
    assert _relerr(est, want) < 1e-10


def test_forward_error_estimate_brackets_observed(oracle_lib):
    """The estimate sets the van der Pol trajectory gates at 10x its value.  Against
    the difference actually observed between two oracle runs stopped at tol and at
    tol/1000, it must bound that difference within the factor 10 on every series,
    and not exceed it by more than 1000x where it is not negligible."""
    w = workloads.vdp(B=16, N=2000)
    m = Model.from_spec(w["spec"])
    for tol in (1e-8, 1e-10):
        y1, _, s1 = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=tol,
                                       max_iter=100)
        y2, _, s2 = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=tol / 1000,
                                       max_iter=100)
        assert not s1.any() and not s2.any()
        obs = np.abs(y1 - y2).max(axis=(1, 2)) / np.abs(y2).max(axis=(1, 2))
        est = oracle_lib.forward_error_estimate(m, w["times"], w["params"], y2, tol)
        assert np.all(obs <= 10.0 * est), (tol, obs / est)
        big = est >= 1e-3 * est.max()
        assert np.all(obs[big] >= est[big] / 1000.0), (tol, obs[big] / est[big])


# --------------------------------------------------------------------------
# Finite-difference gradients of the discrete loss L = sum_{b,k} w_bk . y_bk.
# --------------------------------------------------------------------------
def _loss(oracle_lib, m, w, y0, params, W):
    y, _, st = oracle_lib.forward(m, y0, w["times"], params, lengths=w["lengths"],
                                  tol_abs=1e-14, tol_rel=0.0, max_iter=60)
    return float((y * W).sum())


@pytest.mark.parametrize("which", ["vdp", "linear_ps", "mlp_tanh", "mlp_silu"])
def test_adjoint_against_finite_differences(oracle_lib, which):
    g = np.random.default_rng(5)
    if which == "vdp":
        w = workloads.vdp(B=3, N=300, seed=21)
    elif which == "linear_ps":
        w = workloads.linear_stiff(B=3, N=200)
        w["spec"] = dict(w["spec"], per_series=True)
        w["params"] = np.stack([w["params"] * s for s in (1.0, 0.5, 2.0)])
    elif which == "mlp_tanh":
        w = workloads.mlp_ode(B=2, N=80, n=4, hidden=(6, 5), t_end=2.0)
        w["params"] = w["params"] + 0.05 * g.standard_normal(w["params"].shape)
    else:
        w = workloads.mlp_ode(B=2, N=80, n=3, hidden=(5, 4), act="silu", t_end=2.0)
        w["params"] = w["params"] + 0.05 * g.standard_normal(w["params"].shape)
    m = Model.from_spec(w["spec"])
    B, n = w["y0"].shape
    N = w["times"].shape[1] - 1
    W = g.standard_normal((B, N + 1, n))
    y, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-14,
                                  max_iter=60)
    assert not st.any()
    dp, dy0 = oracle_lib.adjoint(m, w["times"], w["params"], y, W)
    P = w["params"]
    flat = P.reshape(-1)
    idx = g.choice(flat.size, size=min(8, flat.size), replace=False)
    for i in idx:
        h = 1e-6 * max(1.0, abs(flat[i]))
        Pp, Pm = flat.copy(), flat.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (_loss(oracle_lib, m, w, w["y0"], Pp.reshape(P.shape), W)
              - _loss(oracle_lib, m, w, w["y0"], Pm.reshape(P.shape), W)) / (2 * h)
        assert abs(dp.reshape(-1)[i] - fd) <= 1e-5 * max(1.0, abs(fd)), (i, dp.reshape(-1)[i], fd)
    # random directions in parameter space
    for _ in range(2):
        v = g.standard_normal(flat.size)
        h = 1e-6
        fd = (_loss(oracle_lib, m, w, w["y0"], (flat + h * v).reshape(P.shape), W)
              - _loss(oracle_lib, m, w, w["y0"], (flat - h * v).reshape(P.shape), W)) / (2 * h)
        an = dp.reshape(-1) @ v
        assert abs(an - fd) <= 1e-5 * max(1.0, abs(fd))
    # initial state
    for b in range(B):
        for i in range(n):
            h = 1e-6
            yp, ym = w["y0"].copy(), w["y0"].copy()
            yp[b, i] += h
            ym[b, i] -= h
            fd = (_loss(oracle_lib, m, w, yp, P, W) - _loss(oracle_lib, m, w, ym, P, W)) / (2 * h)
            assert abs(dy0[b, i] - fd) <= 1e-5 * max(1.0, abs(fd))


# --------------------------------------------------------------------------
# Invariants.
# --------------------------------------------------------------------------
def test_padding_with_zero_steps_changes_nothing(oracle_lib):
    w = workloads.mlp_ode(B=3, N=120, n=4, hidden=(6, 6), t_end=3.0)
    m = Model.from_spec(w["spec"])
    lengths = np.array([120, 70, 33], dtype=np.int32)
    y, iters, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], lengths=lengths,
                                      tol_abs=1e-13)
    g = workloads.random_grad_out(9, 3, 120, 4)
    for b, L in enumerate(lengths):
        g[b, L + 1:] = 0.0  # masked loss
    dp, dy0 = oracle_lib.adjoint(m, w["times"], w["params"], y, g, lengths=lengths)
    dp_sum = np.zeros_like(dp)
    for b, L in enumerate(lengths):
        yb, _, _ = oracle_lib.forward(m, w["y0"][b:b + 1], w["times"][b:b + 1, :L + 1],
                                      w["params"], tol_abs=1e-13)
        assert np.array_equal(y[b, :L + 1], yb[0])
        assert np.all(y[b, L + 1:] == y[b, L])  # padded steps keep the state
        assert np.all(iters[b, L:] == 0)
        dpb, dy0b = oracle_lib.adjoint(m, w["times"][b:b + 1, :L + 1], w["params"], yb,
                                       g[b:b + 1, :L + 1])
        assert _relerr(dy0[b], dy0b[0]) < 1e-14
        dp_sum += dpb
    assert _relerr(dp, dp_sum) < 1e-12


def test_series_independence_and_thread_count(oracle_lib):
    w = workloads.vdp(B=12, N=500)
    m = Model.from_spec(w["spec"])
    y, _, _ = oracle_lib.forward(m, w["y0"], w["times"], w["params"], nthreads=4)
    sub = [2, 7, 11]
    ys, _, _ = oracle_lib.forward(m, w["y0"][sub], w["times"][sub], w["params"][sub], nthreads=1)
    assert np.array_equal(y[sub], ys)


def test_nonfinite_and_nonconverged_status(oracle_lib):
    w = workloads.vdp(B=3, N=50)
    m = Model.from_spec(w["spec"])
    p = w["params"].copy()
    p[1, 0] = np.nan
    y, _, st = oracle_lib.forward(m, w["y0"], w["times"], p)
    assert st.tolist() == [0, 2, 0]
    _, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=1e-30, max_iter=1)
    assert np.all(st == 1)
