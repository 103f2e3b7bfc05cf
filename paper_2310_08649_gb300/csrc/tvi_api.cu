// tvi_api.cu -- the C ABI declared in include/tvi.h: argument checks, workspace
// layout, kernel dispatch and status read-back.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "tvi.h"
#include "tvi_internal.h"

namespace {

thread_local std::string g_last_error;
std::atomic<unsigned long long> g_launches{0};

tvi_status fail(tvi_status code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
tvi_status fail(tvi_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

tvi_status cuda_fail(cudaError_t e, const char* where) {
  return fail(TVI_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Workspace layout (all offsets 256-byte aligned):
//   [0]        int worst status word
//   [256]      double partials [B][P]  (adjoint, shared parameters)
struct Layout {
  size_t worst, partials, total;
};

Layout layout(int B, int P) {
  Layout l;
  l.worst = 0;
  l.partials = 256;
  l.total = l.partials + align256(static_cast<size_t>(B) * static_cast<size_t>(P) * sizeof(double));
  return l;
}

bool is_mlp(const tvi_model* m) {
  return m->kind == TVI_MODEL_MLP_TANH || m->kind == TVI_MODEL_MLP_SILU;
}

// user models with n > 4 take the large-state route (workspace, no halving)
bool is_large_user(const tvi_model* m) {
  return m->kind == TVI_MODEL_USER && tvi::user_large(m->user);
}

// a user-model error from tvi_jit.cu: the full text (a compiler log can be long)
tvi_status jit_fail(int kind, const std::string& text) {
  g_last_error = text;
  return kind == tvi::kJitNoNvrtc ? TVI_EUNSUPPORTED
         : kind == tvi::kJitCuda  ? TVI_ECUDA
                                  : TVI_EINVAL;
}

// fused small-state forward kernel of a built-in or user model
tvi_status small_forward(const tvi_model* m, int precision, int rpt, int threads,
                         const tvi::FwdArgs& a, cudaStream_t s) {
  if (m->kind == TVI_MODEL_USER) {
    std::string err;
    int rc = tvi::user_forward(m->user, precision, rpt, threads, a, s, &err);
    return rc == tvi::kJitOk ? TVI_OK : jit_fail(rc, "tvi_integrate: " + err);
  }
  cudaError_t e = tvi::small_forward(m->kind, m->n, precision, rpt, threads, a, s);
  return e == cudaSuccess ? TVI_OK : cuda_fail(e, "tvi_integrate: kernel launch");
}

tvi_status small_adjoint(const tvi_model* m, int precision, int rpt, int threads,
                         const tvi::AdjArgs& a, int P, cudaStream_t s, const char* who) {
  if (m->kind == TVI_MODEL_USER) {
    std::string err;
    int rc = tvi::user_adjoint(m->user, precision, rpt, threads, a, s, &err);
    return rc == tvi::kJitOk ? TVI_OK : jit_fail(rc, std::string(who) + ": " + err);
  }
  cudaError_t e = tvi::small_adjoint(m->kind, m->n, precision, rpt, threads, a, P, s);
  return e == cudaSuccess ? TVI_OK : cuda_fail(e, who);
}

tvi_status check_model(const tvi_model* m) {
  if (!m) return fail(TVI_EINVAL, "model is NULL");
  if (m->kind == TVI_MODEL_USER && (!tvi::user_valid(m->user) || m->n != tvi::user_n(m->user)))
    return fail(TVI_EINVAL, "user model: tvi_model.user must be a live model of n = %d", m->n);
  if (tvi_param_count(m) < 0)
    return fail(TVI_EINVAL, "bad model (kind %d, n %d, hidden %d/%d)", m->kind, m->n, m->hidden1,
                m->hidden2);
  if (is_mlp(m)) {
    if (m->per_series)
      return fail(TVI_EUNSUPPORTED, "MLP models take one shared parameter vector");
    if (!tvi::mlp_supported(m->n, m->hidden1, m->hidden2))
      return fail(TVI_EUNSUPPORTED,
                  "MLP sizes n %d, hidden %d/%d not built (n in {4, 8, 16, 32}, hidden <= 128 "
                  "and a multiple of 4)",
                  m->n, m->hidden1, m->hidden2);
    return TVI_OK;
  }
  if (m->kind == TVI_MODEL_USER) return TVI_OK;  // sizes fixed at creation
  if (!tvi::small_supported(m->kind, m->n))
    return fail(TVI_EUNSUPPORTED, "model kind %d with n = %d is not built", m->kind, m->n);
  return TVI_OK;
}

// BF16 block products run on the tensor cores of the MLP path only
tvi_status check_precision(const tvi_model* m, const tvi_options* o) {
  if (o->scheme == TVI_FORWARD_EULER &&
      ((is_mlp(m) && o->precision == tvi::kPrecBf16) || o->predictor))
    return fail(TVI_EUNSUPPORTED,
                "forward Euler runs with FP64 or FP32 blocks (no tensor-core blocks) and "
                "without a predictor");
  if (m->kind == TVI_MODEL_USER && o->precision == tvi::kPrecBf16)
    return fail(TVI_EUNSUPPORTED, "user models run with FP64 or FP32 blocks");
  if (o->precision != tvi::kPrecBf16) return TVI_OK;
  if (!is_mlp(m) || !tvi::mlp_tc_supported(m->n, m->hidden1, m->hidden2))
    return fail(TVI_EUNSUPPORTED,
                "BF16 blocks are built for MLP models with n in {16, 32}, hidden sizes multiples "
                "of 16 in [16, 128] and max(hidden) >= 4 n (got kind %d, n %d, hidden %d/%d)",
                m->kind, m->n, m->hidden1, m->hidden2);
  return TVI_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// chunk the MLP path runs with: the requested one, at most N (and at least 1)
int mlp_chunk(const tvi_options* o, int N) {
  const int c = o->chunk < N ? o->chunk : N;
  return c < 1 ? 1 : c;
}

tvi_status check_opt(const tvi_options* o) {
  if (!o) return fail(TVI_EINVAL, "options are NULL");
  if (o->chunk < 1) return fail(TVI_EINVAL, "chunk must be >= 1 (got %d)", o->chunk);
  if (o->max_iter < 0) return fail(TVI_EINVAL, "max_iter must be >= 0");
  if (!(o->tol_abs >= 0.0) || !(o->tol_rel >= 0.0))
    return fail(TVI_EINVAL, "tolerances must be >= 0");
  if (o->precision != tvi::kPrecFp64 && o->precision != tvi::kPrecFp32 &&
      o->precision != tvi::kPrecBf16)
    return fail(TVI_EINVAL, "unknown precision %d", o->precision);
  if (o->predictor &&
      (o->predictor_chunk < 1 || o->predictor_chunk > tvi::kPredMaxChunk ||
       o->predictor_hidden < 2 || o->predictor_hidden > tvi::kPredMaxHidden ||
       o->predictor_hidden % 2 != 0))
    return fail(TVI_EINVAL, "predictor needs 1 <= predictor_chunk <= %d and an even "
                "predictor_hidden <= %d", tvi::kPredMaxChunk, tvi::kPredMaxHidden);
  if (o->adjoint_refine < 0 || o->adjoint_refine > 16)
    return fail(TVI_EINVAL, "adjoint_refine must be in [0, 16]");
  if (o->scheme != TVI_BACKWARD_EULER && o->scheme != TVI_FORWARD_EULER)
    return fail(TVI_EINVAL, "unknown scheme %d", o->scheme);
  return TVI_OK;
}

}  // namespace

void tvi::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

extern "C" {

void tvi_default_options(tvi_options* opt) {
  if (!opt) return;
  opt->chunk = 1;
  opt->tol_abs = 1e-8;
  opt->tol_rel = 0.0;
  opt->max_iter = 50;
  opt->precision = TVI_PREC_FP64;
  opt->retry_halving = 1;
  opt->adjoint_refine = 2;
  opt->rows_per_thread = 0;
  opt->sync_status = 1;
  opt->predictor = nullptr;
  opt->predictor_chunk = 0;
  opt->predictor_hidden = 0;
  opt->scheme = TVI_BACKWARD_EULER;
}

int tvi_param_count(const tvi_model* m) {
  if (!m || m->n <= 0) return -1;
  switch (m->kind) {
    case TVI_MODEL_LINEAR: return m->n * m->n;
    case TVI_MODEL_VDP: return m->n == 2 ? 1 : -1;
    case TVI_MODEL_MLP_TANH:
    case TVI_MODEL_MLP_SILU:
      if (m->hidden1 <= 0 || m->hidden2 <= 0) return -1;
      return m->hidden1 * m->n + m->hidden1 + m->hidden2 * m->hidden1 + m->hidden2 +
             m->n * m->hidden2 + m->n;
    case TVI_MODEL_USER:
      if (!tvi::user_valid(m->user) || m->n != tvi::user_n(m->user)) return -1;
      return tvi::user_P(m->user);
    default: return -1;
  }
}

size_t tvi_workspace_bytes(const tvi_model* model, const tvi_options* opt, int B, int N) {
  int P = tvi_param_count(model);
  if (P < 0 || B < 0 || N < 0) return 0;
  if (is_mlp(model)) {
    if (!opt || !tvi::mlp_supported(model->n, model->hidden1, model->hidden2)) return 0;
    return tvi::mlp_workspace_bytes(model->n, model->hidden1, model->hidden2, B, mlp_chunk(opt, N),
                                    opt->precision);
  }
  if (is_large_user(model)) {
    if (!opt) return 0;
    return tvi::user_workspace_bytes(model->user, B, mlp_chunk(opt, N), opt->precision);
  }
  return layout(B, P).total;
}

int tvi_effective_chunk(const tvi_model* model, const tvi_options* opt, int N) {
  if (tvi_param_count(model) < 0 || !opt || opt->chunk < 1 || N < 0) return -1;
  if (is_mlp(model) || is_large_user(model)) return mlp_chunk(opt, N);
  int c = opt->chunk < tvi::kSmallMaxChunk ? opt->chunk : tvi::kSmallMaxChunk;
  if (N >= 1 && c > N) c = N;
  return c;
}

tvi_status tvi_integrate(const tvi_model* model, const tvi_options* opt, int B, int N,
                         const double* y0, const double* times, const int* lengths,
                         const double* params, double* y_out, int* stats, int* series_status,
                         void* workspace, size_t workspace_bytes, void* stream) {
  g_last_error.clear();
  tvi_status r = check_model(model);
  if (r != TVI_OK) return r;
  if ((r = check_opt(opt)) != TVI_OK) return r;
  if ((r = check_precision(model, opt)) != TVI_OK) return r;
  if (B < 0 || N < 0) return fail(TVI_EINVAL, "B and N must be >= 0 (got %d, %d)", B, N);
  if (B == 0) return TVI_OK;
  if (!y0 || !times || !params || !y_out)
    return fail(TVI_EINVAL, "y0, times, params and y_out must not be NULL");
  const int P = tvi_param_count(model);
  const Layout l = layout(B, P);
  const size_t need = tvi_workspace_bytes(model, opt, B, N);
  if (!workspace || workspace_bytes < need)
    return fail(TVI_EWORKSPACE, "workspace of %zu bytes needed (got %zu)", need,
                workspace ? workspace_bytes : static_cast<size_t>(0));
  if (!aligned16(workspace)) return fail(TVI_EWORKSPACE, "workspace must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);

  tvi::FwdArgs a;
  a.B = B;
  a.N = N;
  a.chunk = opt->chunk < tvi::kSmallMaxChunk ? opt->chunk : tvi::kSmallMaxChunk;
  a.max_iter = opt->max_iter;
  a.retry_halving = opt->retry_halving ? 1 : 0;
  a.per_series = model->per_series ? 1 : 0;
  a.tol_abs = opt->tol_abs;
  a.tol_rel = opt->tol_rel;
  a.y0 = y0;
  a.times = times;
  a.lengths = lengths;
  a.params = params;
  a.y_out = y_out;
  a.stats = stats;
  a.series_status = series_status;
  a.worst = reinterpret_cast<int*>(ws + l.worst);
  a.pred = opt->predictor;
  a.pred_chunk = opt->predictor_chunk;
  a.pred_hid = opt->predictor_hidden;
  a.scheme = opt->scheme;
  if (a.pred && model->kind != TVI_MODEL_VDP)
    return fail(TVI_EUNSUPPORTED, "the Newton predictor is built for the van der Pol model");

  if (is_mlp(model)) {
    a.chunk = mlp_chunk(opt, N);
    int worst = 0;
    cudaError_t e = tvi::mlp_forward(model->kind, model->n, model->hidden1, model->hidden2,
                                     opt->precision, a, workspace, s,
                                     opt->sync_status ? &worst : nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "tvi_integrate (MLP path)");
    if (worst == 3) return fail(TVI_ETIMEOUT, "a tensor-core wait gave up; results are invalid");
    if (worst == 2) return fail(TVI_ENONFINITE, "a series produced a non-finite residual");
    if (worst == 1) return fail(TVI_ENOTCONV, "a series hit the Newton iteration limit");
    return TVI_OK;
  }
  if (is_large_user(model)) {
    a.chunk = mlp_chunk(opt, N);
    int worst = 0;
    std::string err;
    int rc = tvi::user_large_forward(model->user, opt->precision, a, workspace, s,
                                     opt->sync_status ? &worst : nullptr, &err);
    if (rc != tvi::kJitOk) return jit_fail(rc, "tvi_integrate: " + err);
    if (worst == 3) return fail(TVI_ETIMEOUT, "a bounded wait gave up; results are invalid");
    if (worst == 2) return fail(TVI_ENONFINITE, "a series produced a non-finite residual");
    if (worst == 1) return fail(TVI_ENOTCONV, "a series hit the Newton iteration limit");
    return TVI_OK;
  }
  cudaError_t e = cudaMemsetAsync(a.worst, 0, sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(e, "tvi_integrate: clearing the status word");
  int rpt, threads;
  tvi::small_launch_shape(a.chunk, opt->rows_per_thread, &rpt, &threads);
  // the predictor's layers are latency-bound GEMVs: give them every warp the block can hold
  if (a.pred) threads = tvi::small_max_threads(rpt);
  if ((r = small_forward(model, opt->precision, rpt, threads, a, s)) != TVI_OK) return r;
  if (!opt->sync_status) return TVI_OK;
  int worst = 0;
  e = cudaMemcpyAsync(&worst, a.worst, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "tvi_integrate: status read-back");
  if (worst == 2) return fail(TVI_ENONFINITE, "a series produced a non-finite residual");
  if (worst == 1) return fail(TVI_ENOTCONV, "a series hit the Newton iteration limit");
  return TVI_OK;
}

tvi_status tvi_adjoint(const tvi_model* model, const tvi_options* opt, int B, int N,
                       const double* times, const int* lengths, const double* params,
                       const double* y, const double* grad_out, double* dparams, double* dy0,
                       void* workspace, size_t workspace_bytes, void* stream) {
  g_last_error.clear();
  tvi_status r = check_model(model);
  if (r != TVI_OK) return r;
  if ((r = check_opt(opt)) != TVI_OK) return r;
  if ((r = check_precision(model, opt)) != TVI_OK) return r;
  if (B < 0 || N < 0) return fail(TVI_EINVAL, "B and N must be >= 0 (got %d, %d)", B, N);
  if (B == 0) return TVI_OK;
  if (!times || !params || !y || !grad_out || !dparams)
    return fail(TVI_EINVAL, "times, params, y, grad_out and dparams must not be NULL");
  const int P = tvi_param_count(model);
  const Layout l = layout(B, P);
  const size_t need = tvi_workspace_bytes(model, opt, B, N);
  if (!workspace || workspace_bytes < need)
    return fail(TVI_EWORKSPACE, "workspace of %zu bytes needed (got %zu)", need,
                workspace ? workspace_bytes : static_cast<size_t>(0));
  if (!aligned16(workspace)) return fail(TVI_EWORKSPACE, "workspace must be 16-byte aligned");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);

  tvi::AdjArgs a;
  a.B = B;
  a.N = N;
  a.chunk = opt->chunk < tvi::kSmallMaxChunk ? opt->chunk : tvi::kSmallMaxChunk;
  a.refine = opt->precision == tvi::kPrecFp64 ? 0 : opt->adjoint_refine;
  a.scheme = opt->scheme;
  a.per_series = model->per_series ? 1 : 0;
  a.times = times;
  a.lengths = lengths;
  a.params = params;
  a.y = y;
  a.grad_out = grad_out;
  a.dparams = dparams;
  a.dy0 = dy0;
  a.partials = reinterpret_cast<double*>(ws + l.partials);
  if (is_mlp(model)) {
    if (!aligned16(grad_out)) return fail(TVI_EINVAL, "grad_out must be 16-byte aligned");
    a.chunk = mlp_chunk(opt, N);
    cudaError_t e = tvi::mlp_adjoint(model->kind, model->n, model->hidden1, model->hidden2,
                                     opt->precision, a, workspace, s);
    return e == cudaSuccess ? TVI_OK : cuda_fail(e, "tvi_adjoint (MLP path)");
  }
  if (is_large_user(model)) {
    a.chunk = mlp_chunk(opt, N);
    std::string err;
    int rc = tvi::user_large_adjoint(model->user, opt->precision, a, workspace, s, &err);
    return rc == tvi::kJitOk ? TVI_OK : jit_fail(rc, "tvi_adjoint: " + err);
  }
  if (N == 0) {
    // no steps: dL/dp = 0 and dL/dy0 = grad_out[:, 0]
    size_t dp_bytes = (a.per_series ? static_cast<size_t>(B) : 1u) * P * sizeof(double);
    cudaError_t e = cudaMemsetAsync(dparams, 0, dp_bytes, s);
    if (e == cudaSuccess && dy0)
      e = cudaMemcpyAsync(dy0, grad_out, static_cast<size_t>(B) * model->n * sizeof(double),
                          cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? TVI_OK : cuda_fail(e, "tvi_adjoint: empty integration");
  }
  int rpt, threads;
  tvi::small_launch_shape(a.chunk, opt->rows_per_thread, &rpt, &threads);
  return small_adjoint(model, opt->precision, rpt, threads, a, P, s, "tvi_adjoint: kernel launch");
}

tvi_status tvi_user_model_create(int n, int P, const char* source, tvi_user_model** out) {
  g_last_error.clear();
  if (!out || !source) return fail(TVI_EINVAL, "tvi_user_model_create: NULL source or out");
  const int pmax = n <= tvi::kUserSmallMaxN ? tvi::kUserMaxP : tvi::kUserMaxPLarge;
  if (n < 1 || n > tvi::kUserMaxN || P < 1 || P > pmax)
    return fail(TVI_EINVAL,
                "user models take 1 <= n <= %d and 1 <= P <= %d (%d for n <= %d; got n %d, "
                "P %d)",
                tvi::kUserMaxN, tvi::kUserMaxPLarge, tvi::kUserMaxP, tvi::kUserSmallMaxN, n, P);
  std::string err;
  tvi_user_model* m = nullptr;
  int rc = tvi::user_create(n, P, source, &m, &err);
  if (rc != tvi::kJitOk) return jit_fail(rc, "tvi_user_model_create: " + err);
  *out = m;
  return TVI_OK;
}

tvi_status tvi_user_model_prepare(tvi_user_model* model, int precision) {
  g_last_error.clear();
  if (!tvi::user_valid(model)) return fail(TVI_EINVAL, "tvi_user_model_prepare: not a live model");
  if (precision != TVI_PREC_FP64 && precision != TVI_PREC_FP32)
    return fail(TVI_EUNSUPPORTED, "user models run with FP64 or FP32 blocks (got %d)", precision);
  std::string err;
  int rc = tvi::user_prepare(model, precision, &err);
  return rc == tvi::kJitOk ? TVI_OK : jit_fail(rc, "tvi_user_model_prepare: " + err);
}

void tvi_user_model_destroy(tvi_user_model* model) { tvi::user_destroy(model); }

const char* tvi_last_error(void) { return g_last_error.c_str(); }

unsigned long long tvi_kernel_launches(void) {
  return g_launches.load(std::memory_order_relaxed);
}

const char* tvi_version(void) { return "tvi sm_103a"; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free adjoint.
//
// Some callers cannot allocate device memory at all: code running where
// cudaMalloc is forbidden or unavailable (inside a host callback or a
// real-time loop that must not block on the allocator, a plugin whose host
// application owns every allocation, a process running under an allocator
// that has already reserved the whole device).  tvi_adjoint needs a caller-
// provided workspace for the per-series partial gradients of shared
// parameters; this variant keeps that scratch in a fixed array that lives in
// the library's device image instead.
//
// The array is part of the library's GPU code, so every GPU that runs that
// code holds its kNoAllocScratchBytes until the process exits.  With lazy
// module loading (the CUDA default since 12.2) the module, and with it the
// 4 MiB, is committed on the first call that needs it on a device -- the
// first call of this entry point there -- not when the library is loaded: a
// caller whose allocator will reserve the whole device should make that first
// call before it does.  Host code cannot use the array's name as a device
// address (on the host it names a shadow variable), so the device address is
// looked up with cudaGetSymbolAddress once per CUDA context, with its device
// current, on the first call made in that context; make that first call
// before any stream capture.  The cache is keyed by the context's unique id,
// so a context created after cudaDeviceReset gets its own lookup instead of a
// stale address.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchDoubles = static_cast<size_t>(1) << 19;  // 4 MiB
constexpr int kNoAllocMaxDevices = 64;

std::mutex g_noalloc_mu;
double* g_noalloc_addr[kNoAllocMaxDevices] = {};
unsigned long long g_noalloc_ctx[kNoAllocMaxDevices] = {};

// Unique id of the calling thread's current context (cuCtxGetId, reached through
// the runtime's driver entry points), or 0 when it cannot be read.
unsigned long long current_context_id() {
  using GetCurrent = int (*)(void**);
  using GetId = int (*)(void*, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    // both functions exist with these signatures since CUDA 12.0
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    looked_up = true;
  }
  void* ctx = nullptr;
  unsigned long long id = 0;
  if (get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) return id;
  return 0;
}

}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

namespace {

// Device address of g_noalloc_scratch in the current context (looked up once per
// context).
tvi_status noalloc_scratch(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "tvi_adjoint_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(TVI_EUNSUPPORTED, "tvi_adjoint_noalloc: device %d beyond the supported %d", dev,
                kNoAllocMaxDevices);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  // no context may be current yet on a fresh thread (id 0): the lookup then binds
  // the device's primary context, and its id is read after it
  const unsigned long long ctx = current_context_id();
  if (!g_noalloc_addr[dev] || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return cuda_fail(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                       "tvi_adjoint_noalloc: cudaGetSymbolAddress of the scratch array");
    g_noalloc_addr[dev] = static_cast<double*>(p);
    g_noalloc_ctx[dev] = current_context_id();
  }
  *out = g_noalloc_addr[dev];
  return TVI_OK;
}

}  // namespace

extern "C" tvi_status tvi_adjoint_noalloc(const tvi_model* model, const tvi_options* opt, int B,
                                          int N, const double* times, const int* lengths,
                                          const double* params, const double* y,
                                          const double* grad_out, double* dparams, double* dy0,
                                          void* stream) {
  g_last_error.clear();
  tvi_status r = check_model(model);
  if (r != TVI_OK) return r;
  if (is_mlp(model) || is_large_user(model))
    return fail(TVI_EUNSUPPORTED,
                "tvi_adjoint_noalloc covers the small-state engine (linear, van der Pol and user "
                "models with n <= 4)");
  if ((r = check_opt(opt)) != TVI_OK) return r;
  if ((r = check_precision(model, opt)) != TVI_OK) return r;
  if (B < 0 || N < 0) return fail(TVI_EINVAL, "B and N must be >= 0 (got %d, %d)", B, N);
  if (B == 0) return TVI_OK;
  if (!times || !params || !y || !grad_out || !dparams)
    return fail(TVI_EINVAL, "times, params, y, grad_out and dparams must not be NULL");
  const int P = tvi_param_count(model);
  const size_t need = model->per_series ? 0 : static_cast<size_t>(B) * static_cast<size_t>(P);
  if (need > kNoAllocScratchDoubles)
    return fail(TVI_EINVAL,
                "tvi_adjoint_noalloc: B * P = %zu partial gradients exceed the fixed scratch of "
                "%zu doubles (%zu bytes); use tvi_adjoint with a workspace",
                need, kNoAllocScratchDoubles, kNoAllocScratchDoubles * sizeof(double));
  double* scratch = nullptr;
  if ((r = noalloc_scratch(&scratch)) != TVI_OK) return r;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  tvi::AdjArgs a;
  a.B = B;
  a.N = N;
  a.chunk = opt->chunk < tvi::kSmallMaxChunk ? opt->chunk : tvi::kSmallMaxChunk;
  a.refine = opt->precision == tvi::kPrecFp64 ? 0 : opt->adjoint_refine;
  a.scheme = opt->scheme;
  a.per_series = model->per_series ? 1 : 0;
  a.times = times;
  a.lengths = lengths;
  a.params = params;
  a.y = y;
  a.grad_out = grad_out;
  a.dparams = dparams;
  a.dy0 = dy0;
  // Every series block writes all P entries of its own row before the
  // reduction reads them, so the scratch needs no clearing between calls.
  a.partials = scratch;
  if (N == 0) {
    size_t dp_bytes = (a.per_series ? static_cast<size_t>(B) : 1u) * P * sizeof(double);
    cudaError_t e = cudaMemsetAsync(dparams, 0, dp_bytes, s);
    if (e == cudaSuccess && dy0)
      e = cudaMemcpyAsync(dy0, grad_out, static_cast<size_t>(B) * model->n * sizeof(double),
                          cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? TVI_OK : cuda_fail(e, "tvi_adjoint_noalloc: empty integration");
  }
  int rpt, threads;
  tvi::small_launch_shape(a.chunk, opt->rows_per_thread, &rpt, &threads);
  return small_adjoint(model, opt->precision, rpt, threads, a, P, s,
                       "tvi_adjoint_noalloc: kernel launch");
}
