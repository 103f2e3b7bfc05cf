"""Alg. 1, chunked backward-Euler Newton integration (TEST INFRASTRUCTURE ONLY).

Plain numpy, small cases only: used to show that solving the chunked
equations (Eq. batched-backward-euler) with any of the Sec. 3 solvers gives
the same trajectory as step-by-step integration.  Model functions come from
the C oracle one point at a time.

Per chunk of c steps starting at y_i (Sec. 2.3):
  unknowns  dy_j, j = 1..c, with y_{i+j} = y_i + dy_j and dy_0 = 0
  residual  R_j = dy_j - dy_{j-1} - dt_{i+j} h(y_i + dy_j, t_{i+j}; p)
  Jacobian  block lower-bidiagonal, diagonal I - dt_{i+j} j(y_i + dy_j),
            sub-diagonal -I (Eq. batched-update, with the dt factor of Sec. 2.2)
  guess     dy = 0 (Sec. 2.3)
Convergence (Alg. 1 as read here): series b is converged once
||R_b||_inf <= tol_abs or ||R_b||_inf <= tol_rel ||R_b^0||_inf, the norm taken
over the whole chunk; converged series are frozen; iterate while any is not.
"""
import numpy as np

from . import core, solvers

SOLVERS = {"dense": solvers.dense_solve, "thomas": solvers.thomas, "pcr": solvers.pcr}


def forward_chunked(model, y0, times, params, chunk, solver="thomas", lengths=None,
                    tol_abs=1e-10, tol_rel=0.0, max_iter=50):
    """Returns (y [B][N+1][n], iters per chunk [B][n_chunks])."""
    y0, times, params = (np.asarray(a, float) for a in (y0, times, params))
    B, n = y0.shape
    N = times.shape[1] - 1
    P = core.param_count(model)
    solve = SOLVERS[solver]
    y = np.empty((B, N + 1, n))
    n_chunks = (N + chunk - 1) // chunk
    iters = np.zeros((B, n_chunks), dtype=np.int64)
    for b in range(B):
        p = params[b] if model.per_series else params
        assert p.size == P
        y[b, 0] = y0[b]
        yi = y0[b].copy()
        for ci, i in enumerate(range(0, N, chunk)):
            ce = min(chunk, N - i)
            ks = np.arange(i + 1, i + ce + 1)
            dt = times[b, ks] - times[b, ks - 1]
            if lengths is not None:
                dt = np.where(ks > lengths[b], 0.0, dt)
            tk = times[b, ks]
            dy = np.zeros((ce, n))
            norm0 = None
            it = 0
            while True:
                prev = np.vstack([np.zeros((1, n)), dy[:-1]])
                R = np.stack([dy[j] - prev[j] - dt[j] * core.rhs(model, p, yi + dy[j], tk[j])
                              for j in range(ce)])
                nr = np.abs(R).max()
                if norm0 is None:
                    norm0 = nr
                if nr <= tol_abs or nr <= tol_rel * norm0 or it >= max_iter or not np.isfinite(nr):
                    break
                A = np.stack([np.eye(n) - dt[j] * core.jac(model, p, yi + dy[j], tk[j])
                              for j in range(ce)])
                Bsub = np.stack([-np.eye(n)] * (ce - 1)) if ce > 1 else np.zeros((0, n, n))
                dy = dy - solve(A, Bsub, R)
                it += 1
            iters[b, ci] = it
            y[b, i + 1:i + ce + 1] = yi + dy
            yi = yi + dy[-1]
    return y, iters
