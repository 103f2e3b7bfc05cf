"""The C-ABI library builds, loads, exports every symbol include/tvi.h declares,
and its host-side logic (argument checks, sizes) works without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_08649_gb300 import _lib, build
    build.build()
    return _lib.load()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "tvi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tvi_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2310_08649_gb300 import _lib
    declared = _declared_functions()
    assert declared, "no declarations parsed"
    assert set(declared) == set(_lib.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
    assert lib.tvi_version().decode().startswith("tvi")


def test_defaults_param_counts_and_workspace(lib):
    from paper_2310_08649_gb300 import Model, Options, _lib
    o = _lib.TviOptions()
    lib.tvi_default_options(ctypes.byref(o))
    assert (o.chunk, o.tol_abs, o.max_iter, o.precision, o.retry_halving, o.sync_status) == \
        (1, 1e-8, 50, 0, 1, 1)
    assert Model("vdp", 2, per_series=True).param_count() == 1
    assert Model("linear", 4).param_count() == 16
    assert Model("mlp_tanh", 16, (64, 64)).param_count() == 6288
    assert Model("mlp_silu", 32, (128, 128)).param_count() == 24864
    assert Model("vdp", 3).param_count() == -1
    from paper_2310_08649_gb300 import workspace_bytes
    ws = workspace_bytes(Model("linear", 4), Options(chunk=50), 16, 1000)
    assert ws >= 256 + 16 * 16 * 8 and ws % 256 == 0


def test_effective_chunk(lib):
    """The small-state engine solves at most 1024 steps together; every engine stops at N."""
    from paper_2310_08649_gb300 import Model, Options, effective_chunk
    vdp = Model("vdp", 2, per_series=True)
    assert effective_chunk(vdp, Options(chunk=4096), 10000) == 1024
    assert effective_chunk(vdp, Options(chunk=1000), 10000) == 1000
    assert effective_chunk(vdp, Options(chunk=100), 50) == 50
    assert effective_chunk(vdp, Options(chunk=7), 0) == 7
    mlp = Model("mlp_tanh", 16, (64, 64))
    assert effective_chunk(mlp, Options(chunk=5000), 2000) == 2000
    assert effective_chunk(mlp, Options(chunk=3000), 20000) == 3000
    assert effective_chunk(Model("vdp", 3), Options(chunk=10), 10) == -1
    assert effective_chunk(vdp, Options(chunk=0), 10) == -1


def test_argument_errors_are_returned_without_touching_the_gpu(lib):
    """Validation happens before any CUDA call, so these run on a CPU-only host."""
    from paper_2310_08649_gb300 import Model, Options, _lib
    m = Model("vdp", 2, per_series=True).c()
    vp = ctypes.c_void_p(16)  # never dereferenced: every call below fails validation first

    def call(model, opts, B=4, N=10, y0=vp, ws=vp, ws_bytes=1 << 20):
        return lib.tvi_integrate(ctypes.byref(model), ctypes.byref(opts), B, N, y0, vp, None, vp,
                                 vp, None, None, ws, ws_bytes, None)
    assert call(m, Options(chunk=0).c()) == -1
    assert call(m, Options(tol_abs=-1.0).c()) == -1
    assert call(m, Options(precision="bf16").c()) == -7  # BF16 blocks: MLP path only
    bf = Options(precision="bf16").c()
    assert call(Model("mlp_tanh", 8, (64, 64)).c(), bf) == -7    # n < 16
    assert call(Model("mlp_tanh", 16, (48, 36)).c(), bf) == -7   # 36 not a multiple of 16
    assert call(Model("mlp_silu", 32, (64, 64)).c(), bf) == -7   # max(hidden) < 4 n
    assert call(Model("mlp_silu", 32, (128, 128)).c(), bf, ws=None) == -2  # accepted, then ws
    unknown = Options().c()
    unknown.precision = 7
    assert call(m, unknown) == -1
    assert call(Model("vdp", 3).c(), Options().c()) == -1
    assert call(Model("linear", 3).c(), Options().c()) == -7
    assert call(m, Options().c(), B=-1) == -1
    assert call(m, Options().c(), y0=None) == -1
    assert call(m, Options().c(), ws=None) == -2
    assert call(m, Options().c(), ws_bytes=8) == -2
    assert "workspace" in lib.tvi_last_error().decode()
    assert call(m, Options().c(), B=0) == 0


C_PROGRAM = r"""
/* A C99 caller of the ABI: options, parameter counts, argument errors and a
 * user model compiled from device source, all without a GPU. */
#include <stdio.h>
#include <string.h>
#include "tvi.h"

static const char* kSource =
    "__device__ void tvi_rhs(const double* y, double t, const double* p, double* h) {\n"
    "  h[0] = -p[0] * y[0];\n"
    "}\n"
    "__device__ void tvi_jac(const double* y, double t, const double* p, double* J) {\n"
    "  J[0] = -p[0];\n"
    "}\n"
    "__device__ void tvi_vjp_p(const double* y, double t, const double* p, const double* a,\n"
    "                          double* g) {\n"
    "  g[0] = -a[0] * y[0];\n"
    "}\n";

int main(void) {
  tvi_options o;
  tvi_model m;
  tvi_user_model* u = NULL;
  tvi_default_options(&o);
  if (o.chunk != 1 || o.precision != TVI_PREC_FP64 || o.scheme != TVI_BACKWARD_EULER) return 1;
  memset(&m, 0, sizeof m);
  m.kind = TVI_MODEL_VDP;
  m.n = 2;
  if (tvi_param_count(&m) != 1) return 2;
  if (tvi_integrate(&m, &o, -1, 10, NULL, NULL, NULL, NULL, NULL, NULL, NULL, NULL, 0, NULL)
      != TVI_EINVAL)
    return 3;
  if (tvi_user_model_create(1, 1, kSource, &u) != TVI_OK || u == NULL) {
    printf("%s\n", tvi_last_error());
    return 4;
  }
  m.kind = TVI_MODEL_USER;
  m.n = 1;
  m.user = u;
  if (tvi_param_count(&m) != 1) return 5;
  if (tvi_user_model_prepare(u, TVI_PREC_FP32) != TVI_OK) return 6;
  tvi_user_model_destroy(u);
  printf("ok %s\n", tvi_version());
  return 0;
}
"""


def test_header_is_c99_and_the_library_links_from_c(lib, tmp_path):
    """include/tvi.h compiles as strict C99 and a C program linked against
    libtvi.so runs the host side of the ABI (NVRTC needed for the user model)."""
    import shutil
    import subprocess
    from paper_2310_08649_gb300 import _lib
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "caller.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(_lib.LIB_PATH)
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
           "-L", libdir, "-ltvi", "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    if r.returncode == 4 and "could not be loaded" in r.stdout:
        pytest.skip("NVRTC is not available")
    assert r.returncode == 0 and r.stdout.startswith("ok tvi"), (r.returncode, r.stdout,
                                                                  r.stderr)
