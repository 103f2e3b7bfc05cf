"""ctypes binding of libtvi.so (the C ABI of include/tvi.h).

Argument marshalling only: every step of the integration runs in the CUDA
library.  There is no CPU fallback -- loading fails loudly when the library
has not been built.
"""
import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libtvi.so")

MODEL_KINDS = {"linear": 0, "vdp": 1, "mlp_tanh": 2, "mlp_silu": 3, "user": 4}
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16": 2}
SCHEMES = {"backward": 0, "forward": 1}
STATUS = {0: "TVI_OK", -1: "TVI_EINVAL", -2: "TVI_EWORKSPACE", -3: "TVI_ECUDA",
          -4: "TVI_ENOTCONV", -5: "TVI_ENONFINITE", -6: "TVI_ETIMEOUT", -7: "TVI_EUNSUPPORTED"}
TVI_ENOTCONV, TVI_ENONFINITE, TVI_ETIMEOUT = -4, -5, -6

# every symbol include/tvi.h declares
EXPORTS = ("tvi_default_options", "tvi_param_count", "tvi_workspace_bytes",
           "tvi_effective_chunk", "tvi_integrate",
           "tvi_adjoint", "tvi_adjoint_noalloc", "tvi_predictor_size", "tvi_predictor_forward",
           "tvi_predictor_workspace_bytes", "tvi_predictor_train_step", "tvi_user_model_create",
           "tvi_user_model_prepare", "tvi_user_model_destroy", "tvi_kernel_launches",
           "tvi_last_error", "tvi_version")
STATS = 6  # per-series statistics columns of tvi_integrate


class TviModel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("hidden1", ctypes.c_int),
                ("hidden2", ctypes.c_int), ("per_series", ctypes.c_int),
                ("user", ctypes.c_void_p)]


class TviOptions(ctypes.Structure):
    _fields_ = [("chunk", ctypes.c_int), ("tol_abs", ctypes.c_double),
                ("tol_rel", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("precision", ctypes.c_int), ("retry_halving", ctypes.c_int),
                ("adjoint_refine", ctypes.c_int), ("rows_per_thread", ctypes.c_int),
                ("sync_status", ctypes.c_int), ("predictor", ctypes.c_void_p),
                ("predictor_chunk", ctypes.c_int), ("predictor_hidden", ctypes.c_int),
                ("scheme", ctypes.c_int)]


class TviError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def load():
    """Load libtvi.so once; raise if it is missing (build it with build.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                                  "(python -m paper_2310_08649_gb300.build)")
            lib = ctypes.CDLL(LIB_PATH)
            vp, sz = ctypes.c_void_p, ctypes.c_size_t
            mp, op = ctypes.POINTER(TviModel), ctypes.POINTER(TviOptions)
            lib.tvi_default_options.argtypes = [op]
            lib.tvi_default_options.restype = None
            lib.tvi_param_count.argtypes = [mp]
            lib.tvi_param_count.restype = ctypes.c_int
            lib.tvi_workspace_bytes.argtypes = [mp, op, ctypes.c_int, ctypes.c_int]
            lib.tvi_workspace_bytes.restype = sz
            lib.tvi_effective_chunk.argtypes = [mp, op, ctypes.c_int]
            lib.tvi_effective_chunk.restype = ctypes.c_int
            lib.tvi_integrate.argtypes = [mp, op, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp,
                                          vp, vp, vp, sz, vp]
            lib.tvi_integrate.restype = ctypes.c_int
            lib.tvi_adjoint.argtypes = [mp, op, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp,
                                        vp, vp, vp, sz, vp]
            lib.tvi_adjoint.restype = ctypes.c_int
            lib.tvi_adjoint_noalloc.argtypes = [mp, op, ctypes.c_int, ctypes.c_int, vp, vp, vp,
                                                vp, vp, vp, vp, vp]
            lib.tvi_adjoint_noalloc.restype = ctypes.c_int
            ci = ctypes.c_int
            lib.tvi_predictor_size.argtypes = [ci, ci, ci]
            lib.tvi_predictor_size.restype = ci
            lib.tvi_predictor_forward.argtypes = [vp, ci, ci, ci, ci, vp, vp, vp]
            lib.tvi_predictor_forward.restype = ci
            lib.tvi_predictor_workspace_bytes.argtypes = [ci, ci, ci, ci]
            lib.tvi_predictor_workspace_bytes.restype = sz
            lib.tvi_predictor_train_step.argtypes = [vp, vp, vp, ci, ci, ci, ci, vp, vp, vp,
                                                     ctypes.c_float, ci, vp, vp, sz, vp]
            lib.tvi_predictor_train_step.restype = ci
            lib.tvi_user_model_create.argtypes = [ci, ci, ctypes.c_char_p,
                                                  ctypes.POINTER(ctypes.c_void_p)]
            lib.tvi_user_model_create.restype = ci
            lib.tvi_user_model_prepare.argtypes = [vp, ci]
            lib.tvi_user_model_prepare.restype = ci
            lib.tvi_user_model_destroy.argtypes = [vp]
            lib.tvi_user_model_destroy.restype = None
            lib.tvi_kernel_launches.argtypes = []
            lib.tvi_kernel_launches.restype = ctypes.c_ulonglong
            lib.tvi_last_error.argtypes = []
            lib.tvi_last_error.restype = ctypes.c_char_p
            lib.tvi_version.argtypes = []
            lib.tvi_version.restype = ctypes.c_char_p
            _lib = lib
    return _lib


def last_error():
    return load().tvi_last_error().decode()
