"""CPU FP64 oracle for time-vectorized backward-Euler integration.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product library never does.  It
shares no code with the CUDA path.

* ``forward`` / ``adjoint`` / ``rhs`` / ``jac`` / ``vjp_p`` wrap the C library
  (tvi_oracle.c): step-by-step Newton with dense LU, and the discrete adjoint
  (paper Sec. 2.2 and App. A.1).  ``step_solves`` runs the same one-step Newton
  from every state of a given trajectory (a check of each step on its own).
* ``solvers`` holds the block lower-bidiagonal solvers used only to pin the
  method's linear algebra: a dense solve, Thomas's algorithm (Alg. 2) and
  parallel cyclic reduction (Alg. 3).
* ``chunked`` holds Alg. 1 (chunked backward-Euler Newton) in plain numpy for
  chunk-size invariance checks.
* ``predictor`` holds the FP64 reference of the Newton-predictor MLP.
"""
from .core import (KIND_IDS, Model, adjoint, adjoint_euler, forward, forward_error_estimate,
                   forward_euler, jac, max_threads, param_count, rhs, step_matrices, step_solves,
                   vjp_p)

__all__ = ["KIND_IDS", "Model", "adjoint", "adjoint_euler", "forward", "forward_euler",
           "forward_error_estimate", "jac",
           "max_threads", "param_count", "rhs", "step_matrices", "step_solves", "vjp_p"]
