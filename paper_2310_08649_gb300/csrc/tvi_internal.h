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
// Host-driven Newton loops (large-state engines): the host reads the number of
// series still iterating once per this many passes instead of after each one.
constexpr int kHostCheckEvery = 4;
// Deepest recursion of chunk halving on those engines (a chunk of up to 2^31
// steps halves to one step within it).
constexpr int kHalvingDepth = 32;

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

// Block chain solve of the large-state engines (mlp_chain_kernel): per series
// d_j = M_j (d_{j-1} + rhs_j), j = 0..L-1, with x updated by mode.
struct ChainArgs {
  int B, n, L, c, N, i0, reverse;
  const void* M;           // [B][c][n][n] in T, each block transposed
  const double* rhs_buf;   // [B][c][n] rhs by row, or null
  const double* rhs_traj;  // [B][N+1][n] rhs by step (adjoint dL/dy), or null
  const double* x_init;    // [B][n] d_{-1}, or null (zero)
  const int* active;       // [B] or null
  double* x;               // [B][c][n]
  int mode;                // 0: x -= d   1: x = d   2: x += d
  int* err;                // set when a bounded wait for staged data gives up
  int post_add;            // 1: d_j = M_j d_{j-1} + rhs_j (forward Euler's recurrence)
};

// Argument block of the run-time compiled kernels of user models with n > 4
// (tvi_large_kernels.cuh).  Rows j of the chunk are steps i0 + 1 + j (forward)
// or i0 + L - j (reverse, the adjoint); state vectors are padded to n4 (a
// multiple of 4) in the workspace buffers.
struct LargeArgs {
  int B, N, i0, L, c, n4, per_series, reverse;
  int fwd_euler;            // scheme: forward Euler (h at y_{k-1}; blocks I + dt J)
  const double* times;      // [B][N+1]
  const int* lengths;       // [B] or null
  const double* params;     // [B][P] or [P]
  const double* yi;         // [B][n4] chunk start (forward)
  const double* dy;         // [B][c][n4] Newton iterate (forward)
  const double* ytraj;      // [B][N+1][n] trajectory (adjoint)
  const double* g;          // [B][N+1][n] dL/dy (adjoint)
  const double* av;         // [B][c][n4] adjoint rows (adjoint)
  const double* carry;      // [B][n4] adjoint of the step after the chunk (adjoint)
  double* R;                // [B][c][n4] residual rows (output)
  void* J;                  // [B][c] block slots of n4 x n4 T (the chain's M)
  double* acc;              // [B][P] gradient accumulators (adjoint)
  unsigned long long* norm; // [B] max |R| bits (forward)
  const int* active;        // [B] or null
  double* dy0;              // [B][n] dL/dy0 (forward Euler's final adjoint row)
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
constexpr int kUserSmallMaxN = 4;  // fused one-block-per-series kernels up to here
constexpr int kUserMaxN = 40;       // large-state kernels above (blocks of up to 40 x 40)
constexpr int kUserMaxP = 32;       // parameters of fused-kernel models (held in registers)
constexpr int kUserMaxPLarge = 160; // parameters of large-state models (read from memory
                                    // above 32)
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
// n > kUserSmallMaxN: the large-state route, with a caller workspace
bool user_large(const tvi_user_model* m);
size_t user_workspace_bytes(const tvi_user_model* m, int B, int chunk, int precision);
int user_large_forward(const tvi_user_model* m, int precision, const FwdArgs& a, void* workspace,
                       cudaStream_t s, int* host_worst, std::string* err);
int user_large_adjoint(const tvi_user_model* m, int precision, const AdjArgs& a, void* workspace,
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
// pieces of the MLP engine shared with large-state user models
cudaError_t mlp_launch_chain(int precision, const ChainArgs& ch, cudaStream_t s);
cudaError_t mlp_launch_check(int B, int it, int max_iter, double tol_abs, double tol_rel,
                             unsigned long long* norm, double* norm0, int* active, int* status,
                             int* iters, int* remaining, cudaStream_t s);
// chunk halving: an attempt's start for the series of `mask` (all when null), and
// after it the failed ones into `fail` (their status restored, one retry counted)
cudaError_t mlp_launch_chunk_begin(int B, int rowlen, int c, const int* mask, double* dy,
                                   int* active, unsigned long long* norm, int* iters,
                                   const int* status, int* status0, cudaStream_t s);
cudaError_t mlp_launch_chunk_fail(int B, const int* mask, int* status, const int* status0,
                                  int* fail, int* nfail, int* stats, cudaStream_t s);

// Large-state user models (tvi_large.cu): n in 5..32, the run-time compiled
// kernels of tvi_large_kernels.cuh around the pieces above.
struct LargeKernels {
  const void* residual;      // large_residual_kernel<Model>
  const void* block;         // large_block_kernel<Model, T, n4>
  const void* adj_residual;  // large_adj_residual_kernel<Model>
  const void* param;         // large_param_kernel<Model>
  const void* fe_dy0;        // large_fe_dy0_kernel<Model>
};
size_t large_workspace_bytes(int n, int P, int B, int chunk, int precision);
cudaError_t large_forward(const LargeKernels& k, int n, int P, int precision, const FwdArgs& a,
                          void* workspace, cudaStream_t s, int* host_worst);
cudaError_t large_adjoint(const LargeKernels& k, int n, int P, int precision, const AdjArgs& a,
                          void* workspace, cudaStream_t s);

#endif  // __CUDACC_RTC__

}  // namespace tvi
