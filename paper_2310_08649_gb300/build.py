"""Build the CUDA library paper_2310_08649_gb300/_build/libtvi.so for sm_103a.

Every translation unit under csrc/ is compiled by nvcc in parallel, then linked
into one shared library exporting the C ABI of include/tvi.h.  Nothing is
installed: the library stays in-tree and the Python binding loads it by path.
The headers that user models are compiled against at run time (NVRTC) are
embedded into the library as string literals (_build/tvi_jit_headers.inc).
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libtvi.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC, "-I", OUT_DIR] + ARCH

# headers the run-time compiled user-model kernels include (tvi_jit.cu)
JIT_HEADERS = ["tvi_device.cuh", "tvi_internal.h", "tvi_predictor.cuh", "tvi_small_kernels.cuh",
               "tvi_large_kernels.cuh"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtvi.so")
    return exe


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return files + [os.path.abspath(__file__)]


def write_jit_headers():
    """Write _build/tvi_jit_headers.inc: the JIT_HEADERS as C++ raw string
    literals with their include names, for nvrtcCreateProgram."""
    names, bodies = [], []
    for h in JIT_HEADERS:
        with open(os.path.join(CSRC, h)) as f:
            text = f.read()
        if ")tvi_hdr\"" in text:
            raise RuntimeError(f"{h} contains the raw-string delimiter")
        names.append(f'"{h}"')
        bodies.append(f'R"tvi_hdr({text})tvi_hdr"')
    out = ("// generated by build.py from csrc/: headers of the run-time compiled kernels\n"
           f"static const int kJitHeaderCount = {len(names)};\n"
           f"static const char* const kJitHeaderNames[] = {{{', '.join(names)}}};\n"
           "static const char* const kJitHeaderSources[] = {\n" + ",\n".join(bodies) + "};\n")
    path = os.path.join(OUT_DIR, "tvi_jit_headers.inc")
    if not os.path.exists(path) or open(path).read() != out:
        with open(path, "w") as f:
            f.write(out)
    return path


def _compile(src, extra):
    obj = os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc()] + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(force=False, verbose_ptxas=False):
    os.makedirs(OUT_DIR, exist_ok=True)
    write_jit_headers()  # rewritten only when a header changed
    newest = max(os.path.getmtime(p) for p in _deps())
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    srcs = sources()
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        results = list(ex.map(lambda s: _compile(s, extra), srcs))
    if verbose_ptxas:
        for _, err in results:
            sys.stderr.write(err)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
