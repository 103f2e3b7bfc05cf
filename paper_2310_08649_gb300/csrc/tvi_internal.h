// tvi_internal.h -- argument blocks and launchers shared by the C-ABI layer and
// the kernel translation units.  Not part of the public interface.
#pragma once

#ifndef __CUDACC_RTC__  // host compile (NVRTC provides the device built-ins)
#include <cuda_runtime.h>
#include <stddef.h>

#include <string>

struct tvi_user_model;  // a run-time compiled user model (tvi_jit.cu)
#endif

namespace tvi {

enum { kKindLinear = 0, kKindVdp = 1, kKindMlpTanh = 2, kKindMlpSilu = 3, kKindUser = 4 };
enum { kPrecFp64 = 0, kPrecFp32 = 1, kPrecBf16 = 2 };
// integration schemes (Sec. 2.2): backward Euler, forward Euler
enum { kSchemeBackward = 0, kSchemeForward = 1 };

// Largest chunk the fused small-state kernels hold on chip; a larger requested
// chunk is solved as chunks of this size (same equations, same result).
constexpr int kSmallMaxChunk = 1024;

// Thread bound of the fused kernels by steps per thread: more steps per thread
// need more registers, so fewer threads (the block always holds 1024 steps).
__host__ __device__ constexpr int small_max_threads(int rpt) {
  return rpt == 1 ? 512 : 1024 / rpt;
}

struct FwdArgs {
  int B, N, chunk, max_iter, retry_halving, per_series;
  double tol_abs, tol_rel;
  const double* y0;
  const double* times;
  const int* lengths;
  const double* params;
  double* y_out;
  int* stats;          // [B][kStats] or null
  int* series_status;  // [B] or null
  int* worst;          // device word: max status over series
  const float* pred;   // packed Newton predictor or null
  int pred_chunk, pred_hid;
  int scheme;          // kSchemeBackward / kSchemeForward
};

// per-series statistics: updates, chunks, retries, max updates of a chunk,
// chunks started from the predictor, predictor guesses rejected
constexpr int kStats = 6;
constexpr int kPredMaxChunk = 128;
constexpr int kPredMaxHidden = 256;

struct AdjArgs {
  int B, N, chunk, refine, per_series;
  const double* times;
  const int* lengths;
  const double* params;
  const double* y;
  const double* grad_out;
  double* dparams;
  double* dy0;       // [B][n] or null
  double* partials;  // [B][P] per-series gradient partials (shared parameters)
  int scheme;        // kSchemeBackward / kSchemeForward
};

#ifndef __CUDACC_RTC__
// Host-side count of the kernels this library has enqueued (every host thread),
// read through tvi_kernel_launches(); called right before each launch.
void note_launch();

bool small_supported(int kind, int n);
void small_launch_shape(int chunk, int preferred, int* rpt, int* threads);
cudaError_t small_forward(int kind, int n, int precision, int rpt, int threads, const FwdArgs& a,
                          cudaStream_t s);
cudaError_t small_adjoint(int kind, int n, int precision, int rpt, int threads, const AdjArgs& a,
                          int P, cudaStream_t s);
// dparams = sum over series of the per-series partials (shared parameters)
cudaError_t small_sum_partials(const AdjArgs& a, int P, cudaStream_t s);

// User models (tvi_jit.cu): the small-state kernels compiled at run time with
// the caller's right-hand side.  Return kJitOk or an error kind, with the text
// (the compiler log for kJitCompile) in *err.
enum { kJitOk = 0, kJitNoNvrtc = 1, kJitCompile = 2, kJitCuda = 3 };
constexpr int kUserMaxN = 4;
constexpr int kUserMaxP = 32;
bool user_valid(const tvi_user_model* m);
int user_n(const tvi_user_model* m);
int user_P(const tvi_user_model* m);
int user_create(int n, int P, const char* source, tvi_user_model** out, std::string* err);
void user_destroy(tvi_user_model* m);
int user_prepare(tvi_user_model* m, int precision, std::string* err);
int user_forward(const tvi_user_model* m, int precision, int rpt, int threads, const FwdArgs& a,
                 cudaStream_t s, std::string* err);
int user_adjoint(const tvi_user_model* m, int precision, int rpt, int threads, const AdjArgs& a,
                 cudaStream_t s, std::string* err);

// Neural-ODE (MLP right-hand side) path: shared parameters, n <= 32 and hidden
// widths <= 128, all multiples of 4.  The chunk in the argument blocks is the
// effective one (<= N); workspace as sized by mlp_workspace_bytes.
bool mlp_supported(int n, int h1, int h2);
// BF16 tensor-core blocks: n in {16, 32}, hidden multiples of 16 in [16, 128],
// max(h1, h2) >= 4 n
bool mlp_tc_supported(int n, int h1, int h2);
size_t mlp_workspace_bytes(int n, int h1, int h2, int B, int chunk, int precision);
cudaError_t mlp_forward(int kind, int n, int h1, int h2, int precision, const FwdArgs& a,
                        void* workspace, cudaStream_t s, int* host_worst);
cudaError_t mlp_adjoint(int kind, int n, int h1, int h2, int precision, const AdjArgs& a,
                        void* workspace, cudaStream_t s);

#endif  // __CUDACC_RTC__

}  // namespace tvi
