"""Time-vectorized implicit ODE integration on GB300 (sm_103a).

Chunked backward-Euler Newton integration batched over independent series and
over a chunk of sequential steps, with the block-bidiagonal Newton systems
solved by parallel cyclic reduction, and the discrete adjoint for parameter
gradients.  The computation lives in the CUDA library built from csrc/ (C ABI
in include/tvi.h); this package is its thin Python binding.
"""
from .api import Integrate, Model, Options, UserModel, adjoint, effective_chunk, integrate, \
    make_workspace, odeint, workspace_bytes

__all__ = ["Integrate", "Model", "Options", "UserModel", "adjoint", "effective_chunk",
           "integrate", "make_workspace", "odeint", "workspace_bytes"]
