// tvi_jit.cu -- user-defined small-state models, compiled at run time.
//
// The fused small-state kernels (tvi_small_kernels.cuh) are templates over a
// model type that supplies h(y; p), the step Jacobian I - dt j(y) (Sec. 2.2)
// and the parameter vector-Jacobian product (App. A.1).  For a user model the
// caller's device functions tvi_rhs / tvi_jac / tvi_vjp_p are wrapped into such
// a type and compiled with NVRTC together with the kernel templates, one
// program per (block precision, steps per thread), so the user's right-hand
// side runs inside the same one-block-per-series solver as the built-in
// models, with nothing but an inlined function call between them.
//
// Models with n > 4 use the large-state kernels instead (tvi_large_kernels.cuh,
// one program per block precision) inside the Newton and adjoint loops of
// tvi_large.cu.  The cubins are loaded as context-independent libraries
// (cudaLibraryLoadData) and launched with the same argument blocks as the
// built-in kernels.  NVRTC is opened with dlopen on first use: the library
// loads, and every other entry point works, where NVRTC is absent.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdlib>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "tvi.h"
#include "tvi_internal.h"
#include "tvi_jit_headers.inc"  // generated at build time: kJitHeaderCount, names, sources

namespace {

constexpr unsigned kUserMagic = 0x74766975u;
constexpr int kRptCount = 4;  // steps per thread 1, 2, 4, 8
constexpr int kPrecCount = 2; // FP64, FP32 blocks
// large-state kernels: residual, block, adjoint residual, parameter VJP, forward
// Euler's dL/dy0
constexpr int kLargeKernels = 5;

int rpt_index(int rpt) { return rpt == 1 ? 0 : rpt == 2 ? 1 : rpt == 4 ? 2 : rpt == 8 ? 3 : -1; }

}  // namespace

// One compiled user model.  Immutable after creation except for the caches,
// which fill under `mu` and are never replaced once set.
struct tvi_user_model {
  unsigned magic;
  int n, P;
  std::string source;
  std::mutex mu;
  bool compiled[kPrecCount][kRptCount];
  std::vector<char> cubin[kPrecCount][kRptCount];
  std::string fwd_name[kPrecCount][kRptCount], adj_name[kPrecCount][kRptCount];
  cudaLibrary_t lib[kPrecCount][kRptCount];
  cudaKernel_t fwd[kPrecCount][kRptCount], adj[kPrecCount][kRptCount];
  // large-state kernels (n > 4): residual, Jacobian, adjoint residual, parameter VJP
  bool lcompiled[kPrecCount];
  std::vector<char> lcubin[kPrecCount];
  std::string lname[kPrecCount][kLargeKernels];
  cudaLibrary_t llib[kPrecCount];
  cudaKernel_t lk[kPrecCount][kLargeKernels];
};

namespace tvi {
namespace {

// ---------------------------------------------------------------------------
// NVRTC entry points, resolved once with dlopen.
// ---------------------------------------------------------------------------
struct Nvrtc {
  bool ok = false;
  std::string why;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcAddNameExpression) add_name = nullptr;
  decltype(&nvrtcGetLoweredName) lowered = nullptr;
  decltype(&nvrtcGetErrorString) error_string = nullptr;
};

Nvrtc load_nvrtc() {
  Nvrtc api;
  std::vector<std::string> candidates = {"libnvrtc.so.13", "libnvrtc.so"};
  if (const char* home = std::getenv("CUDA_HOME"))
    candidates.push_back(std::string(home) + "/lib64/libnvrtc.so.13");
  candidates.push_back("/usr/local/cuda/lib64/libnvrtc.so.13");
  void* h = nullptr;
  for (const std::string& c : candidates)
    if ((h = dlopen(c.c_str(), RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
  if (!h) {
    const char* e = dlerror();
    api.why = std::string("NVRTC (libnvrtc.so.13) could not be loaded: ") + (e ? e : "not found");
    return api;
  }
  bool all = true;
  auto sym = [&](auto& fn, const char* name) {
    fn = reinterpret_cast<std::remove_reference_t<decltype(fn)>>(dlsym(h, name));
    if (!fn) {
      all = false;
      api.why = std::string("NVRTC lacks ") + name;
    }
  };
  sym(api.create, "nvrtcCreateProgram");
  sym(api.destroy, "nvrtcDestroyProgram");
  sym(api.compile, "nvrtcCompileProgram");
  sym(api.log_size, "nvrtcGetProgramLogSize");
  sym(api.log, "nvrtcGetProgramLog");
  sym(api.cubin_size, "nvrtcGetCUBINSize");
  sym(api.cubin, "nvrtcGetCUBIN");
  sym(api.add_name, "nvrtcAddNameExpression");
  sym(api.lowered, "nvrtcGetLoweredName");
  sym(api.error_string, "nvrtcGetErrorString");
  api.ok = all;
  return api;
}

const Nvrtc& nvrtc() {
  static const Nvrtc api = load_nvrtc();
  return api;
}

// ---------------------------------------------------------------------------
// Program text.  The kernel templates come first, then the user's functions
// (with their own line numbers for the compiler log), then the model type
// that adapts them to the kernels' model interface.
// ---------------------------------------------------------------------------
const char* const kAdapter = R"tvi_src(
// true when tvi_jac accepts element type T for y and J (a template over T)
template <class...> struct TviVoid { typedef void type; };
template <class T> T&& tvi_declval();
template <class T, class = void> struct TviTypedJac { static constexpr bool value = false; };
template <class T>
struct TviTypedJac<T, typename TviVoid<decltype(tvi_jac(tvi_declval<const T*>(), 0.0,
                                                        tvi_declval<const double*>(),
                                                        tvi_declval<T*>()))>::type> {
  static constexpr bool value = true;
};

// the series' parameters: copied to registers up to 32, else read where they lie
template <int NP_, bool kInRegs>
struct TviParams {
  double v[NP_];
  __device__ __forceinline__ void load(const double* src) {
#pragma unroll
    for (int q = 0; q < NP_; ++q) v[q] = src[q];
  }
  __device__ __forceinline__ operator const double*() const { return v; }
};
template <int NP_>
struct TviParams<NP_, false> {
  const double* v;
  __device__ __forceinline__ void load(const double* src) { v = src; }
  __device__ __forceinline__ operator const double*() const { return v; }
};

struct TviUserModel {
  static constexpr int NS = TVI_N;
  static constexpr int NP = TVI_P;
  static constexpr bool kPredictable = false;  // no learned predictor for user models
  static constexpr bool kUsesTime = true;
  TviParams<NP, (NP <= 32)> p;

  __device__ __forceinline__ float param_feature() const { return 0.0f; }
  __device__ __forceinline__ void load(const double* params, int b, int per_series) {
    p.load(params + (per_series ? static_cast<unsigned long long>(b) * NP : 0ull));
  }
  __device__ __forceinline__ void rhs(const double (&y)[NS], double t, double (&h)[NS]) const {
    tvi_rhs(y, t, p, h);
  }
  // A = I - dt J, J = dh/dy evaluated in the block type T when tvi_jac is a
  // template over it, else in FP64 and rounded to T (integer-pipe conversions)
  template <typename T>
  __device__ __forceinline__ void step_matrix(const T (&y)[NS], double t, T dt,
                                              T (&A)[NS][NS]) const {
    if constexpr (TviTypedJac<T>::value) {
      T J[NS * NS];
      tvi_jac(y, t, p, J);
#pragma unroll
      for (int r = 0; r < NS; ++r)
#pragma unroll
        for (int c = 0; c < NS; ++c) A[r][c] = fma(-dt, J[r * NS + c], r == c ? T(1) : T(0));
    } else {
      double yd[NS], J[NS * NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) yd[s] = tvi::widen(y[s]);
      tvi_jac(yd, t, p, J);
#pragma unroll
      for (int r = 0; r < NS; ++r)
#pragma unroll
        for (int c = 0; c < NS; ++c)
          A[r][c] = fma(-dt, tvi::narrow<T>(J[r * NS + c]), r == c ? T(1) : T(0));
    }
  }
  // J = dh/dy at (y, t), row-major n x n, in T (the large-state kernels)
  template <typename T>
  __device__ __forceinline__ void jacobian(const double (&y)[NS], double t, T* J) const {
    if constexpr (TviTypedJac<T>::value) {
      T yt[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) yt[s] = tvi::narrow<T>(y[s]);
      tvi_jac(yt, t, p, J);
    } else {
      double Jd[NS * NS];
      tvi_jac(y, t, p, Jd);
#pragma unroll
      for (int k = 0; k < NS * NS; ++k) J[k] = tvi::narrow<T>(Jd[k]);
    }
  }
  // acc += scale (dh/dp)^T a
  __device__ __forceinline__ void vjp_p(const double (&y)[NS], double t, const double (&a)[NS],
                                        double scale, double (&acc)[NP]) const {
    double g[NP];
    tvi_vjp_p(y, t, p, a, g);
#pragma unroll
    for (int q = 0; q < NP; ++q) acc[q] = fma(scale, g[q], acc[q]);
  }
};
)tvi_src";

// Kernel that calls each user function once: compiling it checks the source
// without instantiating the solver templates.
const char* const kCheck = R"tvi_src(
__global__ void tvi_user_check(const double* y, double t, const double* p, const double* a,
                               double* out) {
  double h[TVI_N], J[TVI_N * TVI_N], g[TVI_P];
  tvi_rhs(y, t, p, h);
  tvi_jac(y, t, p, J);
  tvi_vjp_p(y, t, p, a, g);
  for (int i = 0; i < TVI_N; ++i) out[i] = h[i];
  for (int i = 0; i < TVI_N * TVI_N; ++i) out[TVI_N + i] = J[i];
  for (int i = 0; i < TVI_P; ++i) out[TVI_N + TVI_N * TVI_N + i] = g[i];
}
)tvi_src";

bool is_large(const tvi_user_model& m) { return m.n > kUserSmallMaxN; }

// solver = false: the check kernel only; true: the adapter, with the kernel
// templates of the model's route
std::string program_text(const tvi_user_model& m, bool solver) {
  std::string s;
  s += "#define TVI_N " + std::to_string(m.n) + "\n";
  s += "#define TVI_P " + std::to_string(m.P) + "\n";
  s += is_large(m) ? "#include \"tvi_large_kernels.cuh\"\n" : "#include \"tvi_small_kernels.cuh\"\n";
  s += "#line 1 \"user_model.cu\"\n";
  s += m.source;
  s += "\n#line 1 \"tvi_user_adapter.cu\"\n";
  s += solver ? kAdapter : kCheck;
  return s;
}

std::string large_kernel_name(int which, int precision, int n) {
  switch (which) {
    case 0: return "tvi::klarge::large_residual_kernel<TviUserModel>";
    case 1:
      return std::string("tvi::klarge::large_block_kernel<TviUserModel, ") +
             (precision == kPrecFp64 ? "double, " : "float, ") + std::to_string((n + 3) / 4 * 4) +
             ">";
    case 2: return "tvi::klarge::large_adj_residual_kernel<TviUserModel>";
    case 3: return "tvi::klarge::large_param_kernel<TviUserModel>";
    default: return "tvi::klarge::large_fe_dy0_kernel<TviUserModel>";
  }
}

std::string kernel_name(bool forward, int precision, int rpt) {
  return std::string(forward ? "tvi::kern::forward_small_kernel<TviUserModel, "
                             : "tvi::kern::adjoint_small_kernel<TviUserModel, ") +
         (precision == kPrecFp64 ? "double, " : "float, ") + std::to_string(rpt) + ">";
}

// Compile one program; on success returns 0 and (when `names` is given) the
// cubin and the lowered kernel names.  Errors: kJitNoNvrtc, kJitCompile.
int compile(const std::string& text, const std::vector<std::string>& names,
            std::vector<char>* cubin, std::vector<std::string>* lowered, std::string* err) {
  const Nvrtc& api = nvrtc();
  if (!api.ok) {
    *err = api.why;
    return kJitNoNvrtc;
  }
  nvrtcProgram prog = nullptr;
  nvrtcResult r = api.create(&prog, text.c_str(), "tvi_user_program.cu", kJitHeaderCount,
                             kJitHeaderSources, kJitHeaderNames);
  if (r != NVRTC_SUCCESS) {
    *err = std::string("nvrtcCreateProgram: ") + api.error_string(r);
    return kJitCompile;
  }
  for (const std::string& nm : names) api.add_name(prog, nm.c_str());
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-default-device"};
  r = api.compile(prog, 3, opts);
  if (r != NVRTC_SUCCESS) {
    size_t n = 0;
    api.log_size(prog, &n);
    std::string log(n, '\0');
    if (n) api.log(prog, &log[0]);
    while (!log.empty() && (log.back() == '\0' || log.back() == '\n')) log.pop_back();
    *err = std::string("user model does not compile (") + api.error_string(r) + "):\n" + log;
    api.destroy(&prog);
    return kJitCompile;
  }
  if (cubin) {
    size_t n = 0;
    api.cubin_size(prog, &n);
    cubin->resize(n);
    if (n) api.cubin(prog, cubin->data());
  }
  if (lowered) {
    lowered->clear();
    for (const std::string& nm : names) {
      const char* low = nullptr;
      api.lowered(prog, nm.c_str(), &low);
      lowered->push_back(low ? low : "");
    }
  }
  api.destroy(&prog);
  return kJitOk;
}

// Compile the solver kernels of (precision, rpt) unless done; caller holds m->mu.
int ensure_compiled(tvi_user_model* m, int pi, int ri, std::string* err) {
  if (m->compiled[pi][ri]) return kJitOk;
  const int precision = pi == 0 ? kPrecFp64 : kPrecFp32;
  const int rpt = 1 << ri;
  std::vector<std::string> names = {kernel_name(true, precision, rpt),
                                    kernel_name(false, precision, rpt)};
  std::vector<std::string> low;
  std::vector<char> cubin;
  int rc = compile(program_text(*m, true), names, &cubin, &low, err);
  if (rc != kJitOk) return rc;
  m->cubin[pi][ri].swap(cubin);
  m->fwd_name[pi][ri] = low[0];
  m->adj_name[pi][ri] = low[1];
  m->compiled[pi][ri] = true;
  return kJitOk;
}

// Kernels of (precision, rpt), compiled and loaded on first use.
int kernels(const tvi_user_model* cm, int precision, int rpt, cudaKernel_t* fwd, cudaKernel_t* adj,
            std::string* err) {
  tvi_user_model* m = const_cast<tvi_user_model*>(cm);
  const int pi = precision == kPrecFp64 ? 0 : 1;
  const int ri = rpt_index(rpt);
  if (ri < 0 || (precision != kPrecFp64 && precision != kPrecFp32)) {
    *err = "user models run with FP64 or FP32 blocks and 1, 2, 4 or 8 steps per thread";
    return kJitCompile;
  }
  std::lock_guard<std::mutex> lock(m->mu);
  if (!m->lib[pi][ri]) {
    int rc = ensure_compiled(m, pi, ri, err);
    if (rc != kJitOk) return rc;
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, m->cubin[pi][ri].data(), nullptr, nullptr, 0,
                                        nullptr, nullptr, 0);
    cudaKernel_t kf = nullptr, ka = nullptr;
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&kf, lib, m->fwd_name[pi][ri].c_str());
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&ka, lib, m->adj_name[pi][ri].c_str());
    if (e != cudaSuccess) {
      if (lib) cudaLibraryUnload(lib);
      *err = std::string("loading the user model's kernels: ") + cudaGetErrorString(e);
      return kJitCuda;
    }
    m->fwd[pi][ri] = kf;
    m->adj[pi][ri] = ka;
    m->lib[pi][ri] = lib;
  }
  *fwd = m->fwd[pi][ri];
  *adj = m->adj[pi][ri];
  return kJitOk;
}

// Compile the large-state kernels of one precision unless done; caller holds m->mu.
int ensure_large_compiled(tvi_user_model* m, int pi, std::string* err) {
  if (m->lcompiled[pi]) return kJitOk;
  const int precision = pi == 0 ? kPrecFp64 : kPrecFp32;
  std::vector<std::string> names;
  for (int w = 0; w < kLargeKernels; ++w) names.push_back(large_kernel_name(w, precision, m->n));
  std::vector<std::string> low;
  std::vector<char> cubin;
  int rc = compile(program_text(*m, true), names, &cubin, &low, err);
  if (rc != kJitOk) return rc;
  m->lcubin[pi].swap(cubin);
  for (int w = 0; w < kLargeKernels; ++w) m->lname[pi][w] = low[w];
  m->lcompiled[pi] = true;
  return kJitOk;
}

int large_kernels(const tvi_user_model* cm, int precision, LargeKernels* out, std::string* err) {
  tvi_user_model* m = const_cast<tvi_user_model*>(cm);
  if (precision != kPrecFp64 && precision != kPrecFp32) {
    *err = "user models run with FP64 or FP32 blocks";
    return kJitCompile;
  }
  const int pi = precision == kPrecFp64 ? 0 : 1;
  std::lock_guard<std::mutex> lock(m->mu);
  if (!m->llib[pi]) {
    int rc = ensure_large_compiled(m, pi, err);
    if (rc != kJitOk) return rc;
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, m->lcubin[pi].data(), nullptr, nullptr, 0,
                                        nullptr, nullptr, 0);
    cudaKernel_t k[kLargeKernels] = {};
    for (int w = 0; w < kLargeKernels && e == cudaSuccess; ++w)
      e = cudaLibraryGetKernel(&k[w], lib, m->lname[pi][w].c_str());
    if (e != cudaSuccess) {
      if (lib) cudaLibraryUnload(lib);
      *err = std::string("loading the user model's kernels: ") + cudaGetErrorString(e);
      return kJitCuda;
    }
    for (int w = 0; w < kLargeKernels; ++w) m->lk[pi][w] = k[w];
    m->llib[pi] = lib;
  }
  out->residual = reinterpret_cast<const void*>(m->lk[pi][0]);
  out->block = reinterpret_cast<const void*>(m->lk[pi][1]);
  out->adj_residual = reinterpret_cast<const void*>(m->lk[pi][2]);
  out->param = reinterpret_cast<const void*>(m->lk[pi][3]);
  out->fe_dy0 = reinterpret_cast<const void*>(m->lk[pi][4]);
  return kJitOk;
}

}  // namespace

bool user_valid(const tvi_user_model* m) { return m && m->magic == kUserMagic; }
int user_n(const tvi_user_model* m) { return m->n; }
int user_P(const tvi_user_model* m) { return m->P; }

int user_create(int n, int P, const char* source, tvi_user_model** out, std::string* err) {
  tvi_user_model* m = new tvi_user_model();
  m->magic = kUserMagic;
  m->n = n;
  m->P = P;
  m->source = source;
  for (int i = 0; i < kPrecCount; ++i) {
    for (int j = 0; j < kRptCount; ++j) {
      m->compiled[i][j] = false;
      m->lib[i][j] = nullptr;
      m->fwd[i][j] = m->adj[i][j] = nullptr;
    }
    m->lcompiled[i] = false;
    m->llib[i] = nullptr;
    for (int w = 0; w < kLargeKernels; ++w) m->lk[i][w] = nullptr;
  }
  int rc = compile(program_text(*m, false), {}, nullptr, nullptr, err);
  if (rc != kJitOk) {
    m->magic = 0;
    delete m;
    return rc;
  }
  *out = m;
  return kJitOk;
}

void user_destroy(tvi_user_model* m) {
  if (!user_valid(m)) return;
  for (int i = 0; i < kPrecCount; ++i) {
    for (int j = 0; j < kRptCount; ++j)
      if (m->lib[i][j]) cudaLibraryUnload(m->lib[i][j]);
    if (m->llib[i]) cudaLibraryUnload(m->llib[i]);
  }
  m->magic = 0;
  delete m;
}

// Compile every steps-per-thread variant of one precision, in parallel threads.
int user_prepare(tvi_user_model* m, int precision, std::string* err) {
  if (precision != kPrecFp64 && precision != kPrecFp32) {
    *err = "user models run with FP64 or FP32 blocks";
    return kJitCompile;
  }
  const int pi = precision == kPrecFp64 ? 0 : 1;
  std::lock_guard<std::mutex> lock(m->mu);
  if (is_large(*m)) return ensure_large_compiled(m, pi, err);
  int rc[kRptCount] = {kJitOk, kJitOk, kJitOk, kJitOk};
  std::string errs[kRptCount];
  std::vector<std::thread> pool;
  for (int ri = 0; ri < kRptCount; ++ri)
    pool.emplace_back([&, ri] { rc[ri] = ensure_compiled(m, pi, ri, &errs[ri]); });
  for (std::thread& t : pool) t.join();
  for (int ri = 0; ri < kRptCount; ++ri)
    if (rc[ri] != kJitOk) {
      *err = errs[ri];
      return rc[ri];
    }
  return kJitOk;
}

int user_forward(const tvi_user_model* m, int precision, int rpt, int threads, const FwdArgs& a,
                 cudaStream_t s, std::string* err) {
  cudaKernel_t kf = nullptr, ka = nullptr;
  int rc = kernels(m, precision, rpt, &kf, &ka, err);
  if (rc != kJitOk) return rc;
  FwdArgs args = a;
  void* params[] = {&args};
  note_launch();
  cudaError_t e = cudaLaunchKernel(reinterpret_cast<const void*>(kf), dim3(a.B), dim3(threads),
                                   params, 0, s);
  if (e != cudaSuccess) {
    *err = std::string("user model forward launch: ") + cudaGetErrorString(e);
    return kJitCuda;
  }
  return kJitOk;
}

int user_adjoint(const tvi_user_model* m, int precision, int rpt, int threads, const AdjArgs& a,
                 cudaStream_t s, std::string* err) {
  cudaKernel_t kf = nullptr, ka = nullptr;
  int rc = kernels(m, precision, rpt, &kf, &ka, err);
  if (rc != kJitOk) return rc;
  AdjArgs args = a;
  void* params[] = {&args};
  note_launch();
  cudaError_t e = cudaLaunchKernel(reinterpret_cast<const void*>(ka), dim3(a.B), dim3(threads),
                                   params, 0, s);
  if (e == cudaSuccess && !a.per_series) e = small_sum_partials(a, m->P, s);
  if (e != cudaSuccess) {
    *err = std::string("user model adjoint launch: ") + cudaGetErrorString(e);
    return kJitCuda;
  }
  return kJitOk;
}

bool user_large(const tvi_user_model* m) { return is_large(*m); }

size_t user_workspace_bytes(const tvi_user_model* m, int B, int chunk, int precision) {
  return large_workspace_bytes(m->n, m->P, B, chunk, precision);
}

int user_large_forward(const tvi_user_model* m, int precision, const FwdArgs& a, void* workspace,
                       cudaStream_t s, int* host_worst, std::string* err) {
  LargeKernels k{};
  int rc = large_kernels(m, precision, &k, err);
  if (rc != kJitOk) return rc;
  cudaError_t e = large_forward(k, m->n, m->P, precision, a, workspace, s, host_worst);
  if (e != cudaSuccess) {
    *err = std::string("user model forward (large-state kernels): ") + cudaGetErrorString(e);
    return kJitCuda;
  }
  return kJitOk;
}

int user_large_adjoint(const tvi_user_model* m, int precision, const AdjArgs& a, void* workspace,
                       cudaStream_t s, std::string* err) {
  LargeKernels k{};
  int rc = large_kernels(m, precision, &k, err);
  if (rc != kJitOk) return rc;
  cudaError_t e = large_adjoint(k, m->n, m->P, precision, a, workspace, s);
  if (e != cudaSuccess) {
    *err = std::string("user model adjoint (large-state kernels): ") + cudaGetErrorString(e);
    return kJitCuda;
  }
  return kJitOk;
}

}  // namespace tvi
