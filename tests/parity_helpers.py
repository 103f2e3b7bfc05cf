"""Step-by-step parity checks shared by the GPU tests (test infrastructure).

Two correct solvers that stop Newton at a residual tolerance can drift apart
over a trajectory by the problem's conditioning times that tolerance (van der
Pol's relaxation jumps amplify strongly).  These checks remove the drift: every
step of the GPU trajectory is compared with the oracle's solution of that step
from the GPU's OWN previous state, so only one step's conditioning enters,
||A_k^-1|| with A_k = I - dt_k j(y_k) for backward Euler and none at all for
forward Euler.  Errors are per series, max_k |y_k - y*_k|_inf / max_k |y*_k|_inf.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np

STEP_GATE = 1e-10  # every step, FP64 and mixed-precision blocks alike (FP64 residuals)


def relerr_series(a, b):
    return np.abs(a - b).max(axis=(1, 2)) / np.maximum(np.abs(b).max(axis=(1, 2)), 1e-300)


def be_step_errors(oracle_lib, m, w, y, lengths=None, tol=1e-13):
    """Backward Euler: y*_k is the oracle's one-step Newton solve from the GPU's
    y_{k-1} (oracle.step_solves), stopped at tol x max(1, max_k |y_k|_inf) for each
    series (FP64 rounding of states near 1e3 sits near 1e-13).  One oracle call
    per series, on a thread pool (the calls release the interpreter lock)."""
    B = y.shape[0]
    one = np.empty_like(y)

    def solve(b):
        p = w["params"][b:b + 1] if m.per_series else w["params"]
        lens = None if lengths is None else lengths[b:b + 1]
        tb = tol * max(1.0, float(np.abs(y[b]).max()))
        one[b:b + 1], st = oracle_lib.step_solves(m, w["times"][b:b + 1], p, y[b:b + 1],
                                                  lengths=lens, tol_abs=tb, max_iter=100,
                                                  nthreads=1)
        return int(st[0])
    with ThreadPoolExecutor(max_workers=max(1, oracle_lib.max_threads())) as ex:
        status = list(ex.map(solve, range(B)))
    assert not any(status), status
    return relerr_series(y, one)


def be_step_bound(oracle_lib, m, w, y, tol, lengths=None):
    """Largest per-series step error that GPU residuals of size tol can leave:
    1.5 tol max_k ||A_k^-1||_inf / max_k |y_k|_inf (1.5: the Newton iterate's A_k
    is taken at y_k rather than at the exact root)."""
    A = oracle_lib.step_matrices(m, w["times"], w["params"], y, lengths)
    inv_norm = np.abs(np.linalg.inv(A)).sum(-1).max(-1).max(-1)  # [B]
    return 1.5 * tol * inv_norm / np.maximum(np.abs(y).max(axis=(1, 2)), 1e-300)


def fe_step_errors(oracle_lib, m, w, y, lengths=None):
    """Forward Euler: y*_k = y_{k-1} + dt_k h(y_{k-1}, t_{k-1}) from the GPU's
    y_{k-1}, by the oracle's explicit recursion run for one step from every state
    (steps past a series' length have dt = 0)."""
    B, Np1, n = y.shape
    N = Np1 - 1
    if N == 0:
        return np.zeros(B)
    times = np.array(w["times"], dtype=np.float64, copy=True)
    if lengths is not None:
        for b, L in enumerate(lengths):
            times[b, L + 1:] = times[b, L]
    pairs = np.stack([times[:, :-1], times[:, 1:]], axis=-1).reshape(B * N, 2)
    starts = y[:, :-1].reshape(B * N, n)
    params = np.repeat(w["params"], N, axis=0) if m.per_series else w["params"]
    one, st = oracle_lib.forward_euler(m, starts, pairs, params)
    assert not st.any()
    ystar = np.concatenate([y[:, :1], one[:, 1].reshape(B, N, n)], axis=1)
    return relerr_series(y, ystar)
