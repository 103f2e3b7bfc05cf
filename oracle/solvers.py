"""Block lower-bidiagonal solvers of paper Sec. 3 (TEST INFRASTRUCTURE ONLY).

System (Sec. 3, first equation), c diagonal blocks A_1..A_c (n x n) and c-1
sub-diagonal blocks B_1..B_{c-1} (B_i sits in block row i+1, column i):

    A_1 x_1                 = y_1
    B_i x_i + A_{i+1} x_{i+1} = y_{i+1},   i = 1..c-1

Arrays are zero-based: A[c][n][n], Bsub[c-1][n][n], y[c][n].
"""
import numpy as np


def dense_solve(A, Bsub, y):
    """Assemble the full (c n) x (c n) matrix and call a dense library solve."""
    A, Bsub, y = np.asarray(A, float), np.asarray(Bsub, float), np.asarray(y, float)
    c, n, _ = A.shape
    M = np.zeros((c * n, c * n))
    for i in range(c):
        M[i * n:(i + 1) * n, i * n:(i + 1) * n] = A[i]
        if i > 0:
            M[i * n:(i + 1) * n, (i - 1) * n:i * n] = Bsub[i - 1]
    return np.linalg.solve(M, y.reshape(-1)).reshape(c, n)


def thomas(A, Bsub, y):
    """Alg. 2: block forward substitution, x_1 = A_1^-1 y_1, x_{i+1} = A_{i+1}^-1 (y_{i+1} - B_i x_i)."""
    A, Bsub, y = np.asarray(A, float), np.asarray(Bsub, float), np.asarray(y, float)
    c = A.shape[0]
    x = np.empty_like(y)
    x[0] = np.linalg.solve(A[0], y[0])
    for i in range(1, c):
        x[i] = np.linalg.solve(A[i], y[i] - Bsub[i - 1] @ x[i - 1])
    return x


def pcr_level(A, C, y, s):
    """One splitting level of PCR (Sec. 3.2, the four-block example).

    Row k reads  A_k x_k + C_k x_{k-s} = y_k  (C_k = 0 where there is no
    partner).  Substituting row k-s eliminates x_{k-s} and couples row k to
    x_{k-2s}:

        C_k <- -C_k A_{k-s}^-1 C_{k-s}
        y_k <-  y_k - C_k A_{k-s}^-1 y_{k-s}

    Every row uses the values from before the level; diagonal blocks never
    change.  Rows k <= s (zero-based k < s) have no partner and are untouched.
    """
    c = A.shape[0]
    C_new, y_new = C.copy(), y.copy()
    for k in range(s, c):
        CkAinv = C[k] @ np.linalg.inv(A[k - s])
        C_new[k] = -CkAinv @ C[k - s]
        y_new[k] = y[k] - CkAinv @ y[k - s]
    return C_new, y_new


def pcr(A, Bsub, y):
    """Alg. 3 (read with the four-block example as authority): levels with
    stride s = 1, 2, 4, ... while s < c, i.e. ceil(log2 c) levels, which leaves
    a block-diagonal system; then x_k = A_k^-1 y_k.  Any c works: rows without
    a partner at a level are left unchanged."""
    A, Bsub, y = np.asarray(A, float), np.asarray(Bsub, float), np.asarray(y, float)
    c, n, _ = A.shape
    C = np.zeros_like(A)
    C[1:] = Bsub
    s = 1
    while s < c:
        C, y = pcr_level(A, C, y, s)
        s *= 2
    assert not np.any(C), "PCR left a coupling block behind"
    return np.stack([np.linalg.solve(A[k], y[k]) for k in range(c)])
