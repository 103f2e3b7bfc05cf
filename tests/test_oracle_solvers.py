"""Pins of the oracle's block-bidiagonal solvers (Sec. 3) and of Alg. 1.

* Thomas (Alg. 2) and PCR (Alg. 3) against a dense library solve of the
  assembled (c n) x (c n) matrix, for many chunk sizes including non-powers of two.
* One PCR level against the paper's four-block splitting example (Sec. 3.2).
* Alg. 1 (chunked Newton) against step-by-step integration: chunk-size invariance.
"""
import numpy as np
import pytest

import workloads
from oracle import Model, chunked, solvers


def _system(g, c, n):
    A = np.stack([np.eye(n) * (2.0 + g.uniform()) + 0.3 * g.standard_normal((n, n))
                  for _ in range(c)])
    Bsub = 0.7 * g.standard_normal((max(c - 1, 0), n, n))
    y = g.standard_normal((c, n))
    return A, Bsub, y


@pytest.mark.parametrize("c", [1, 2, 3, 4, 5, 7, 8, 9, 16, 33])
@pytest.mark.parametrize("n", [1, 2, 4])
def test_thomas_and_pcr_match_dense(c, n):
    g = np.random.default_rng(100 * c + n)
    A, Bsub, y = _system(g, c, n)
    x = solvers.dense_solve(A, Bsub, y)
    assert np.abs(solvers.thomas(A, Bsub, y) - x).max() <= 1e-12 * max(1, np.abs(x).max())
    assert np.abs(solvers.pcr(A, Bsub, y) - x).max() <= 1e-12 * max(1, np.abs(x).max())


def test_pcr_one_level_matches_four_block_example():
    """Sec. 3.2: one splitting of the 4-block system gives row 2 coupling 0 and
    rhs y2 - B1 A1^-1 y1, row 3 coupling -B2 A2^-1 B1 (to x1) and rhs
    y3 - B2 A2^-1 y2, row 4 coupling -B3 A3^-1 B2 (to x2) and rhs y4 - B3 A3^-1 y3;
    row 1 and all diagonal blocks are unchanged."""
    g = np.random.default_rng(4)
    A, Bsub, y = _system(g, 4, 3)
    C = np.zeros_like(A)
    C[1:] = Bsub
    C1, y1 = solvers.pcr_level(A, C, y, 1)
    inv = np.linalg.inv
    B1, B2, B3 = Bsub
    assert np.allclose(C1[0], 0) and np.allclose(C1[1], 0)
    assert np.allclose(C1[2], -B2 @ inv(A[1]) @ B1, atol=1e-14)
    assert np.allclose(C1[3], -B3 @ inv(A[2]) @ B2, atol=1e-14)
    assert np.array_equal(y1[0], y[0])
    assert np.allclose(y1[1], y[1] - B1 @ inv(A[0]) @ y[0], atol=1e-14)
    assert np.allclose(y1[2], y[2] - B2 @ inv(A[1]) @ y[1], atol=1e-14)
    assert np.allclose(y1[3], y[3] - B3 @ inv(A[2]) @ y[2], atol=1e-14)
    # the red (rows 1, 3) and green (rows 2, 4) systems are now independent:
    # solving them separately reproduces the full solution
    x = solvers.dense_solve(A, Bsub, y)
    red = solvers.dense_solve(A[[0, 2]], C1[[2]], y1[[0, 2]])
    green = solvers.dense_solve(A[[1, 3]], C1[[3]], y1[[1, 3]])
    assert np.allclose(red, x[[0, 2]], atol=1e-12) and np.allclose(green, x[[1, 3]], atol=1e-12)


def test_pcr_level_count_is_ceil_log2():
    """After ceil(log2 c) levels every coupling block is zero (and not before)."""
    g = np.random.default_rng(8)
    for c in [2, 3, 5, 8, 13, 64, 100]:
        A, Bsub, y = _system(g, c, 2)
        C = np.zeros_like(A)
        C[1:] = Bsub
        s, levels = 1, 0
        while np.any(C):
            C, y = solvers.pcr_level(A, C, y, s)
            s *= 2
            levels += 1
        assert levels == int(np.ceil(np.log2(c)))


@pytest.mark.parametrize("which", ["linear", "vdp", "mlp"])
def test_chunked_newton_matches_step_by_step(oracle_lib, which):
    if which == "linear":
        w = workloads.linear_stiff(B=2, N=130)
        tol = 1e-12
    elif which == "vdp":
        # resolved grid (mu dt <= 0.7): plain Newton from the zero guess converges
        w = workloads.vdp(B=3, N=300, seed=31, t_max=0.5, mu_decades=(1.0, 1.5))
        tol = 1e-12
    else:
        w = workloads.mlp_ode(B=2, N=90, n=3, hidden=(5, 5), t_end=3.0)
        tol = 1e-12
    m = Model.from_spec(w["spec"])
    ys, _, st = oracle_lib.forward(m, w["y0"], w["times"], w["params"], tol_abs=tol, max_iter=60)
    assert not st.any()
    N = w["times"].shape[1] - 1
    for c, solver in [(1, "thomas"), (7, "pcr"), (32, "thomas"), (N, "pcr"), (13, "dense")]:
        yc, it = chunked.forward_chunked(m, w["y0"], w["times"], w["params"], c, solver,
                                         tol_abs=tol, max_iter=60)
        scale = np.abs(ys).max()
        assert np.abs(yc - ys).max() <= 1e-10 * scale, (c, solver, np.abs(yc - ys).max())
