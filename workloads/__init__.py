"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws inputs (initial states, time grids, parameters, loss
gradients).  It holds none of the integration method's arithmetic, and both
the oracle and the CUDA path consume what it returns.  Every generator takes
an explicit seed (numpy PCG64) so that both sides see identical inputs.

Each generator returns a dict with
  spec    -- model description {"kind", "n", "hidden", "per_series"}
  y0      -- [B][n] float64
  times   -- [B][N+1] float64 (times[b][0] is the start time)
  params  -- float64, [B][P] when spec["per_series"] else [P]
  lengths -- [B] int32, or None when every series uses all N steps
plus generator-specific extras.

Default sizes are the paper-shaped workloads:
  linear_stiff  n=4 stiff linear system, 16 series, 1000 uniform steps on [0, 1]
  vdp           van der Pol n=2, 128 series, 10,000 log-spaced steps per series over
                [0, min(3 mu, 500 / mu)]
  mlp_ode       neural ODE n=16, MLP 16-64-64-16 tanh, 64 series, 2000 steps on [0, 10]
  mlp_large     neural ODE n=32, MLP 32-128-128-32 SiLU, 512 series, 20,000 padded
                steps with per-series lengths uniform in [2000, 20000]
  mds           mass-damper-spring chain (n = 2 n_unit), the parameter table of the
                paper's timing study, 100 series, 2000 uniform steps on [0, 1]
  chaboche      Chaboche viscoplasticity (n = 2 + n_unit), the paper's parameter
                table, 50 series, 2000 uniform steps on [0, 10]
  neuron        coupled neurons (n = 4 n_unit), the paper's parameter table,
                50 series, 2000 uniform steps on [0, 10]
"""
import numpy as np

SEED_LINEAR, SEED_VDP, SEED_MLP, SEED_PREDICTOR, SEED_MLP_LARGE = 1001, 1002, 1003, 1004, 1005
SEED_MDS, SEED_CHABOCHE, SEED_NEURON = 1006, 1007, 1008


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def uniform_times(B, N, t_end):
    """t_k = k t_end / N for every series."""
    return np.tile(np.linspace(0.0, t_end, N + 1), (B, 1))


def log_times(B, N, t_end, decades=6.0):
    """t_0 = 0 and t_k = t_end 10^(-decades + decades (k-1)/(N-1)), k = 1..N:
    a geometric grid from t_end 10^-decades up to t_end."""
    k = np.arange(1, N + 1, dtype=np.float64)
    t = np.empty(N + 1)
    t[0] = 0.0
    t[1:] = t_end * 10.0 ** (-decades + decades * (k - 1) / max(N - 1, 1))
    return np.tile(t, (B, 1))


def linear_stiff(seed=SEED_LINEAR, B=16, N=1000, n=4, t_end=1.0, lam_decades=(0.0, 4.0)):
    """dy/dt = A y with A = -Q diag(lam) Q^T, Q a seeded random orthogonal matrix
    (QR of a Gaussian matrix, signs fixed so diag(R) > 0) and lam log-uniform in
    [10^lam_decades[0], 10^lam_decades[1]].  One A shared by all series."""
    g = _rng(seed)
    X = g.standard_normal((n, n))
    Q, R = np.linalg.qr(X)
    Q = Q * np.sign(np.diag(R))[None, :]
    lam = 10.0 ** g.uniform(lam_decades[0], lam_decades[1], n)
    A = -(Q * lam[None, :]) @ Q.T
    y0 = g.standard_normal((B, n))
    return {"spec": {"kind": "linear", "n": n, "hidden": (0, 0), "per_series": False},
            "y0": y0, "times": uniform_times(B, N, t_end), "params": A.reshape(-1).copy(),
            "lengths": None, "Q": Q, "lam": lam}


def vdp(seed=SEED_VDP, B=128, N=10000, span_mu=3.0, t_max=None, mu_dt_max=0.69,
        mu_decades=(1.0, 3.0)):
    """van der Pol, mu log-uniform in [10, 1000] per series, y0 uniform in [-2, 2]^2,
    N log-spaced steps (6 decades) over [0, span_mu * mu].  The largest log step
    is about t_end 6 ln(10) / (N - 1), so series b ends at
        t_end = min(span_mu mu_b, mu_dt_max (N - 1) / (6 ln(10) mu_b))
    (= min(3 mu_b, 500 / mu_b) at N = 10,000): mu dt <= mu_dt_max at every step and
    the grid resolves the fast time scale 1/mu everywhere.  t_max, when given, caps
    t_end further.  Times differ per series."""
    g = _rng(seed)
    mu = 10.0 ** g.uniform(mu_decades[0], mu_decades[1], B)
    y0 = g.uniform(-2.0, 2.0, (B, 2))
    resolve = 500.0 * (N - 1) / 9999.0 * (mu_dt_max / 0.69)
    t_end = np.minimum(span_mu * mu, resolve / mu)
    if t_max is not None:
        t_end = np.minimum(t_end, t_max)
    times = log_times(B, N, 1.0) * t_end[:, None]
    return {"spec": {"kind": "vdp", "n": 2, "hidden": (0, 0), "per_series": True},
            "y0": y0, "times": times, "params": mu.reshape(B, 1).copy(), "lengths": None}


def xavier_mlp(g, n, hidden):
    """Flat MLP parameters W1 b1 W2 b2 W3 b3 (W row-major out x in): Xavier-uniform
    weights U(-a, a), a = sqrt(6 / (fan_in + fan_out)); zero biases."""
    sizes = [n, hidden[0], hidden[1], n]
    parts = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        a = np.sqrt(6.0 / (fan_in + fan_out))
        parts.append(g.uniform(-a, a, (fan_out, fan_in)).reshape(-1))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts)


def mlp_ode(seed=SEED_MLP, B=64, N=2000, n=16, hidden=(64, 64), act="tanh", t_end=10.0,
            lengths_range=None):
    """Neural ODE dy/dt = MLP(y).  y0 ~ N(0, 1).  'params' is the trained model,
    'target_params' a second seeded network of the same architecture whose
    trajectory from the same y0 serves as the regression target."""
    g = _rng(seed)
    params = xavier_mlp(g, n, hidden)
    target = xavier_mlp(g, n, hidden)
    y0 = g.standard_normal((B, n))
    lengths = None
    if lengths_range is not None:
        lengths = g.integers(lengths_range[0], lengths_range[1] + 1, B).astype(np.int32)
    kind = "mlp_tanh" if act == "tanh" else "mlp_silu"
    return {"spec": {"kind": kind, "n": n, "hidden": tuple(hidden), "per_series": False},
            "y0": y0, "times": uniform_times(B, N, t_end), "params": params,
            "target_params": target, "lengths": lengths}


def mlp_large(seed=SEED_MLP_LARGE, B=512, N=20000, n=32, hidden=(128, 128), t_end=10.0,
              lengths_range=(2000, 20000)):
    """n = 32 SiLU neural ODE, per-series random lengths padded into one launch."""
    return mlp_ode(seed=seed, B=B, N=N, n=n, hidden=hidden, act="silu", t_end=t_end,
                   lengths_range=lengths_range)


def mds(seed=SEED_MDS, B=100, N=2000, n_unit=2, t_max=1.0, jitter=0.0):
    """Mass-damper-spring chain (Sec. 5.1.1, Table mass-params): K_i, C_i, M_i
    linspace over the units in [1e-2, 1], [1e-6, 1e-4], [1e-7, 1e-5]; f_a = 1;
    forcing period T linspace over the series in [1e-2, 1]; zero initial
    state; N uniform steps on [0, t_max].  Per-series parameter vectors
    [K_1..K_u, C_1..C_u, M_1..M_u, f_a, T].  jitter > 0 multiplies every
    parameter by a seeded factor exp(jitter * N(0, 1)) (distinct series for
    tests); 0 keeps the table's values."""
    u = int(n_unit)
    base = np.concatenate([np.linspace(1e-2, 1.0, u), np.linspace(1e-6, 1e-4, u),
                           np.linspace(1e-7, 1e-5, u), [1.0]])
    T = np.linspace(1e-2, 1.0, B)
    params = np.concatenate([np.tile(base, (B, 1)), T[:, None]], axis=1)
    if jitter > 0.0:
        params = params * np.exp(jitter * _rng(seed).standard_normal(params.shape))
    return {"spec": {"kind": "mds", "n": 2 * u, "hidden": (0, 0), "per_series": True},
            "y0": np.zeros((B, 2 * u)), "times": uniform_times(B, N, t_max),
            "params": params, "lengths": None}


def chaboche(seed=SEED_CHABOCHE, B=50, N=2000, n_unit=3, t_max=10.0, jitter=0.0):
    """Chaboche viscoplasticity (Sec. 5.1.1, Table chaboche-params): E = 10,
    flow exponent 5, eta = 2, sigma_0 = 1, K_inf = 10, tau = 1, C_i and g_i
    linspace over the backstresses in [0.1, 1] and [0.1, 0.5], strain-rate
    amplitude linspace over the series in [0.1, 1], period T = 1; zero initial
    state; N uniform steps on [0, t_max].  Per-series parameter vectors
    [E, m, eta, sigma_0, K_inf, tau, C_1..C_u, g_1..g_u, ed_a, T].  jitter > 0
    multiplies every parameter by a seeded factor exp(jitter * N(0, 1))."""
    u = int(n_unit)
    base = np.concatenate([[10.0, 5.0, 2.0, 1.0, 10.0, 1.0], np.linspace(0.1, 1.0, u),
                           np.linspace(0.1, 0.5, u)])
    eda = np.linspace(0.1, 1.0, B)
    params = np.concatenate([np.tile(base, (B, 1)), eda[:, None], np.ones((B, 1))], axis=1)
    if jitter > 0.0:
        params = params * np.exp(jitter * _rng(seed).standard_normal(params.shape))
    return {"spec": {"kind": "chaboche", "n": 2 + u, "hidden": (0, 0), "per_series": True},
            "y0": np.zeros((B, 2 + u)), "times": uniform_times(B, N, t_max),
            "params": params, "lengths": None}


def neuron(seed=SEED_NEURON, B=50, N=2000, n_unit=1, t_max=10.0, jitter=0.0):
    """Coupled neurons (Sec. 5.1.1, Table neuron-params): per neuron C, gNa, ENa,
    gK, EK, gL, EL, m_inf, h_inf, n_inf linspace over the neurons in [0.1, 1];
    tau_m, tau_h, tau_n in [0.5, 5], [1.5, 15], [1, 10]; gC in [1e-3, 1e-2];
    period T in [0.5, 2]; applied amplitude I_a linspace over the series in
    [0.1, 1]; zero initial state; N uniform steps on [0, t_max].  Per-series
    parameter vectors: 15 per neuron [C, gNa, ENa, gK, EK, gL, EL, m_inf, tau_m,
    h_inf, tau_h, n_inf, tau_n, gC, T], then I_a.  jitter > 0 multiplies every
    parameter by a seeded factor exp(jitter * N(0, 1))."""
    u = int(n_unit)
    ls = lambda a, b: np.linspace(a, b, u)  # noqa: E731
    cols = [ls(0.1, 1.0)] * 7 + [ls(0.1, 1.0), ls(0.5, 5.0), ls(0.1, 1.0), ls(1.5, 15.0),
                                 ls(0.1, 1.0), ls(1.0, 10.0), ls(1e-3, 1e-2), ls(0.5, 2.0)]
    per_unit = np.stack(cols, axis=1).reshape(-1)  # [u][15]
    Ia = np.linspace(0.1, 1.0, B)
    params = np.concatenate([np.tile(per_unit, (B, 1)), Ia[:, None]], axis=1)
    if jitter > 0.0:
        params = params * np.exp(jitter * _rng(seed).standard_normal(params.shape))
    return {"spec": {"kind": "neuron", "n": 4 * u, "hidden": (0, 0), "per_series": True},
            "y0": np.zeros((B, 4 * u)), "times": uniform_times(B, N, t_max),
            "params": params, "lengths": None}


def random_grad_out(seed, B, N, n, scale=1.0):
    """A seeded dL/dy for every output [B][N+1][n] (adjoint parity inputs)."""
    return scale * _rng(seed).standard_normal((B, N + 1, n))


def random_times(seed, B, N, t_end=1.0, spread=0.5):
    """Per-series non-uniform grids: positive steps drawn U(1-spread, 1+spread),
    rescaled per series to end at t_end times a per-series factor in [0.5, 1.5]."""
    g = _rng(seed)
    steps = g.uniform(1.0 - spread, 1.0 + spread, (B, N))
    ends = t_end * g.uniform(0.5, 1.5, B)
    steps = steps / steps.sum(axis=1, keepdims=True) * ends[:, None]
    t = np.zeros((B, N + 1))
    t[:, 1:] = np.cumsum(steps, axis=1)
    return t
