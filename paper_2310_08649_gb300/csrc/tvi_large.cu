// tvi_large.cu -- host side of user models with 4 < n <= 40 (the large-state
// route): workspace, the model-independent kernels, and the Newton and adjoint
// loops around the run-time compiled kernels of tvi_large_kernels.cuh.
//
// Forward, per chunk (Alg. 1), all series at once, converged series skipped:
//   residual (user) -> convergence check (mlp_launch_check; the host reads how
//   many series still iterate) -> blocks: Jacobian and inverse (user) -> block
//   forward substitution dy -= d (mlp_launch_chain)
// Adjoint (App. A.2), chunks in reverse: dL/dy rows gathered in row order ->
// A^-T blocks at the trajectory (user) -> a = substitution; FP64 refinement
// residuals (user) and corrections; parameter gradient (user).
// State vectors are padded to n4 = 4 ceil(n / 4) (the chain's vector width).
#include <cuda_runtime.h>

#include <functional>

#include "tvi_device.cuh"
#include "tvi_internal.h"

namespace tvi {

namespace {

constexpr int kThreads = 128;  // kLargeThreads of the run-time compiled kernels

int pad4(int n) { return (n + 3) / 4 * 4; }
size_t al(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct LWs {
  int *worst, *remaining, *err, *active, *status, *iters;
  int *status0, *nfail, *fail;  // chunk halving: status before an attempt, failures, masks
  double *yi, *carry, *norm0, *dy, *R, *acc;
  unsigned long long* norm;
  void* M;
  size_t total;
};

LWs carve(char* base, int n, int P, int B, int c, int precision) {
  LWs w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += al(bytes);
    return p;
  };
  const int n4 = pad4(n);
  const size_t bc = static_cast<size_t>(B) * c;
  const size_t tsz = precision == kPrecFp64 ? sizeof(double) : sizeof(float);
  w.worst = reinterpret_cast<int*>(take(sizeof(int)));
  w.remaining = reinterpret_cast<int*>(take(sizeof(int)));
  w.err = reinterpret_cast<int*>(take(sizeof(int)));
  w.active = reinterpret_cast<int*>(take(sizeof(int) * B));
  w.status = reinterpret_cast<int*>(take(sizeof(int) * B));
  w.iters = reinterpret_cast<int*>(take(sizeof(int) * B));
  w.status0 = reinterpret_cast<int*>(take(sizeof(int) * B));
  w.nfail = reinterpret_cast<int*>(take(sizeof(int)));
  w.fail = reinterpret_cast<int*>(take(sizeof(int) * B * kHalvingDepth));
  w.norm = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * B));
  w.norm0 = reinterpret_cast<double*>(take(sizeof(double) * B));
  w.yi = reinterpret_cast<double*>(take(sizeof(double) * B * n4));
  w.carry = reinterpret_cast<double*>(take(sizeof(double) * B * n4));
  w.acc = reinterpret_cast<double*>(take(sizeof(double) * B * P));
  w.dy = reinterpret_cast<double*>(take(sizeof(double) * bc * n4));
  w.R = reinterpret_cast<double*>(take(sizeof(double) * bc * n4));
  w.M = take(tsz * bc * n4 * n4);
  w.total = off;
  return w;
}

__global__ void large_start_kernel(int B, int n, int n4, int Np1, const double* y0,
                                   double* y_out, double* yi, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B * n4) {
    const int b = i / n4, s = i % n4;
    const double v = s < n ? y0[b * n + s] : 0.0;
    yi[i] = v;
    if (s < n) y_out[static_cast<size_t>(b) * Np1 * n + s] = v;
  }
  if (i < B) status[i] = 0;
}

// y_{i0+1..i0+L} = y_i + dy; carry y_{i0+L}; one block per series.  Padded
// steps (k > length) keep the last real state exactly (reading C-14), whatever
// rounding Newton left in their identity rows.
__global__ void large_store_kernel(int n, int n4, int L, int c, int N, int i0, const int* lengths,
                                   const double* dy, double* yi, double* y_out, const int* iters,
                                   int* stats, const int* mask, const int* fail) {
  const int b = blockIdx.x;
  // only the attempt's series (mask), and not those re-solving it by halves
  if ((mask && !mask[b]) || (fail && fail[b])) return;
  const int len = lengths ? min(max(lengths[b], 0), N) : N;
  const int jl = min(L, max(len - i0, 0)) - 1;  // last real row of the chunk, -1 if none
  const double* dyb = dy + static_cast<size_t>(b) * c * n4;
  double* yb = y_out + static_cast<size_t>(b) * (N + 1) * n;
  for (int e = threadIdx.x; e < L * n; e += blockDim.x) {
    const int j = e / n, s = e % n;
    const int jr = min(j, jl);
    yb[static_cast<size_t>(i0 + 1 + j) * n + s] =
        yi[b * n4 + s] + (jr >= 0 ? dyb[jr * n4 + s] : 0.0);
  }
  __syncthreads();
  if (threadIdx.x < n && jl >= 0) yi[b * n4 + threadIdx.x] += dyb[jl * n4 + threadIdx.x];
  if (threadIdx.x == 0 && stats) {
    int* o = stats + b * kStats;
    o[0] += iters[b];
    o[1] += 1;
    o[3] = max(o[3], iters[b]);
  }
}

__global__ void large_worst_kernel(int B, const int* status, const int* err, int* series_status,
                                   int* worst) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int st = *err ? 3 : status[b];
  if (series_status) series_status[b] = st;
  if (st) atomicMax(worst, st);
}

// dL/dy rows of the chunk in row order (row j = step i0 + L - j), padded
__global__ void large_gather_kernel(int B, int n, int n4, int N, int i0, int L, int c,
                                    const double* g, double* out) {
  const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<size_t>(B) * L * n4) return;
  const int s = static_cast<int>(i % n4);
  const int j = static_cast<int>((i / n4) % L);
  const int b = static_cast<int>(i / (static_cast<size_t>(n4) * L));
  const int k = i0 + L - j;
  out[(static_cast<size_t>(b) * c + j) * n4 + s] =
      s < n ? g[(static_cast<size_t>(b) * (N + 1) + k) * n + s] : 0.0;
}

// carry a_{i0+1} (row L-1) to the earlier chunk
__global__ void large_carry_kernel(int B, int n4, int L, int c, const double* av, double* carry) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B * n4) carry[i] = av[(static_cast<size_t>(i / n4) * c + (L - 1)) * n4 + (i % n4)];
}

// dL/dy0 = a_1 + dL/dy_0; dL/dp per series, or summed over the series in order
// (shared parameters); NaN when a bounded wait gave up
// (forward Euler: dL/dy0 was written by large_fe_dy0_kernel and is only
// replaced by NaN here)
__global__ void large_adjoint_end_kernel(int B, int n, int n4, int Np1, int P, int per_series,
                                         int fwd_euler, const double* carry, const double* g,
                                         const double* acc, double* dy0, double* dparams,
                                         const int* err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool bad = *err != 0;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  if (dy0 && i < B * n) {
    const int b = i / n, s = i % n;
    if (bad) dy0[i] = nan;
    else if (!fwd_euler) dy0[i] = carry[b * n4 + s] + g[static_cast<size_t>(b) * Np1 * n + s];
  }
  if (per_series) {
    if (i < B * P) dparams[i] = bad ? nan : acc[i];
  } else if (i < P) {
    double v = 0.0;
    for (int b = 0; b < B; ++b) v += acc[static_cast<size_t>(b) * P + i];
    dparams[i] = bad ? nan : v;
  }
}

cudaError_t launch_user(const void* kernel, dim3 grid, const LargeArgs& a, cudaStream_t s) {
  LargeArgs args = a;
  void* params[] = {&args};
  note_launch();
  return cudaLaunchKernel(kernel, grid, dim3(kThreads), params, 0, s);
}

// the block kernel: four warps per block, each forming 32 / SEG blocks (SEG the
// lanes of one block: 8, 16 or 32 for n4 up to 8, 16, 32; above, one block per warp
// with two rows a lane)
dim3 block_grid(int L, int B, int n4) {
  const int per_warp = n4 <= 8 ? 4 : (n4 <= 16 ? 2 : 1);
  const int per_block = 4 * per_warp;
  return dim3((L + per_block - 1) / per_block, B);
}

#define TVI_TRY(x)                    \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

unsigned blocks_for(size_t count, int threads) {
  return static_cast<unsigned>((count + threads - 1) / threads);
}

}  // namespace

size_t large_workspace_bytes(int n, int P, int B, int chunk, int precision) {
  return carve(nullptr, n, P, B, chunk, precision).total;
}

cudaError_t large_forward(const LargeKernels& k, int n, int P, int precision, const FwdArgs& a,
                          void* workspace, cudaStream_t s, int* host_worst) {
  const int B = a.B, N = a.N, c = a.chunk, n4 = pad4(n);
  LWs w = carve(static_cast<char*>(workspace), n, P, B, c, precision);
  TVI_TRY(cudaMemsetAsync(w.worst, 0, sizeof(int), s));
  TVI_TRY(cudaMemsetAsync(w.err, 0, sizeof(int), s));
  note_launch();
  large_start_kernel<<<blocks_for(static_cast<size_t>(B) * n4, 256), 256, 0, s>>>(
      B, n, n4, N + 1, a.y0, a.y_out, w.yi, w.status);
  TVI_TRY(cudaGetLastError());
  if (a.stats) TVI_TRY(cudaMemsetAsync(a.stats, 0, sizeof(int) * kStats * B, s));
  // One attempt over steps i0 + 1 .. i0 + L for the series in `mask` (all when
  // null); with retry_halving the series whose attempt failed re-solve the same
  // steps as two halves, recursively down to one step (as in the MLP engine).
  std::function<cudaError_t(int, int, const int*, int)> solve =
      [&](int i0, int L, const int* mask, int depth) -> cudaError_t {
    const bool halve = a.retry_halving && L > 1 && depth < kHalvingDepth;
    TVI_TRY(mlp_launch_chunk_begin(B, n4, c, mask, w.dy, w.active, w.norm, w.iters, w.status,
                                   w.status0, s));
    LargeArgs la{};
    la.B = B; la.N = N; la.i0 = i0; la.L = L; la.c = c; la.n4 = n4;
    la.per_series = a.per_series; la.reverse = 0; la.fwd_euler = a.scheme == kSchemeForward;
    la.times = a.times; la.lengths = a.lengths; la.params = a.params;
    la.yi = w.yi; la.dy = w.dy; la.R = w.R; la.J = w.M; la.norm = w.norm; la.active = w.active;
    const dim3 grid((L + kThreads - 1) / kThreads, B);
    for (int it = 0;; ++it) {
      TVI_TRY(launch_user(k.residual, grid, la, s));
      TVI_TRY(cudaMemsetAsync(w.remaining, 0, sizeof(int), s));
      TVI_TRY(mlp_launch_check(B, it, a.max_iter, a.tol_abs, a.tol_rel, w.norm, w.norm0, w.active,
                               w.status, w.iters, w.remaining, s));
      // the host reads how many series still iterate only every kHostCheckEvery
      // passes (and at the iteration limit, where the check stops every series);
      // passes enqueued after the last series stopped find none active and return
      if ((it + 1) % kHostCheckEvery == 0 || it >= a.max_iter) {
        int remaining = 0;
        TVI_TRY(cudaMemcpyAsync(&remaining, w.remaining, sizeof(int), cudaMemcpyDeviceToHost, s));
        TVI_TRY(cudaStreamSynchronize(s));
        if (remaining == 0) break;
      }
      TVI_TRY(launch_user(k.block, block_grid(L, B, n4), la, s));
      ChainArgs ch{};
      ch.B = B; ch.n = n4; ch.L = L; ch.c = c; ch.N = N; ch.i0 = i0; ch.reverse = 0; ch.M = w.M;
      ch.rhs_buf = w.R; ch.active = w.active; ch.x = w.dy; ch.mode = 0; ch.err = w.err;
      ch.post_add = la.fwd_euler;  // forward Euler: d_j = (I + dt J) d_{j-1} + R_j
      TVI_TRY(mlp_launch_chain(precision, ch, s));
    }
    int* fail = halve ? w.fail + static_cast<size_t>(depth) * B : nullptr;
    int nfail = 0;
    if (halve) {
      TVI_TRY(mlp_launch_chunk_fail(B, mask, w.status, w.status0, fail, w.nfail, a.stats, s));
      TVI_TRY(cudaMemcpyAsync(&nfail, w.nfail, sizeof(int), cudaMemcpyDeviceToHost, s));
      TVI_TRY(cudaStreamSynchronize(s));
    }
    note_launch();
    large_store_kernel<<<B, 128, 0, s>>>(n, n4, L, c, N, i0, a.lengths, w.dy, w.yi, a.y_out,
                                         w.iters, a.stats, mask, fail);
    TVI_TRY(cudaGetLastError());
    if (nfail > 0) {
      const int L1 = (L + 1) / 2;
      TVI_TRY(solve(i0, L1, fail, depth + 1));
      TVI_TRY(solve(i0 + L1, L - L1, fail, depth + 1));
    }
    return cudaSuccess;
  };
  for (int i0 = 0; i0 < N; i0 += c) TVI_TRY(solve(i0, (N - i0 < c) ? N - i0 : c, nullptr, 0));
  note_launch();
  large_worst_kernel<<<blocks_for(B, 128), 128, 0, s>>>(B, w.status, w.err, a.series_status,
                                                        w.worst);
  TVI_TRY(cudaGetLastError());
  if (host_worst) {
    TVI_TRY(cudaMemcpyAsync(host_worst, w.worst, sizeof(int), cudaMemcpyDeviceToHost, s));
    TVI_TRY(cudaStreamSynchronize(s));
  }
  return cudaSuccess;
}

cudaError_t large_adjoint(const LargeKernels& k, int n, int P, int precision, const AdjArgs& a,
                          void* workspace, cudaStream_t s) {
  const int B = a.B, N = a.N, c = a.chunk, n4 = pad4(n);
  LWs w = carve(static_cast<char*>(workspace), n, P, B, c, precision);
  TVI_TRY(cudaMemsetAsync(w.err, 0, sizeof(int), s));
  TVI_TRY(cudaMemsetAsync(w.carry, 0, sizeof(double) * B * n4, s));  // a_{N+1} = 0
  TVI_TRY(cudaMemsetAsync(w.acc, 0, sizeof(double) * B * P, s));
  const int refine = precision == kPrecFp64 ? 0 : a.refine;
  const int nch = (N + c - 1) / c;
  for (int ci = nch - 1; ci >= 0; --ci) {
    const int i0 = ci * c;
    const int L = (N - i0 < c) ? N - i0 : c;
    LargeArgs la{};
    la.B = B; la.N = N; la.i0 = i0; la.L = L; la.c = c; la.n4 = n4;
    la.per_series = a.per_series; la.reverse = 1; la.fwd_euler = a.scheme == kSchemeForward;
    la.times = a.times; la.lengths = a.lengths; la.params = a.params;
    la.ytraj = a.y; la.g = a.grad_out; la.av = w.dy; la.carry = w.carry; la.R = w.R; la.J = w.M;
    la.acc = w.acc;
    const dim3 grid((L + kThreads - 1) / kThreads, B);
    note_launch();
    large_gather_kernel<<<blocks_for(static_cast<size_t>(B) * L * n4, 256), 256, 0, s>>>(
        B, n, n4, N, i0, L, c, a.grad_out, w.R);
    TVI_TRY(cudaGetLastError());
    TVI_TRY(launch_user(k.block, block_grid(L, B, n4), la, s));
    // a_j = A^-T (a_{j-1} + g_k) (backward Euler) or (I + dt J)^T a_{j-1} + g_k
    // (forward Euler), a_{-1} = carry
    ChainArgs ch{};
    ch.B = B; ch.n = n4; ch.L = L; ch.c = c; ch.N = N; ch.i0 = i0; ch.reverse = 1; ch.M = w.M;
    ch.rhs_buf = w.R; ch.x_init = w.carry; ch.x = w.dy; ch.mode = 1; ch.err = w.err;
    ch.post_add = la.fwd_euler;
    TVI_TRY(mlp_launch_chain(precision, ch, s));
    for (int it = 0; it < refine; ++it) {
      TVI_TRY(launch_user(k.adj_residual, grid, la, s));
      ChainArgs cr = ch;
      cr.x_init = nullptr;
      cr.mode = 2;  // a += correction
      TVI_TRY(mlp_launch_chain(precision, cr, s));
    }
    TVI_TRY(launch_user(k.param, dim3(B), la, s));
    note_launch();
    large_carry_kernel<<<blocks_for(static_cast<size_t>(B) * n4, 256), 256, 0, s>>>(
        B, n4, L, c, w.dy, w.carry);
    TVI_TRY(cudaGetLastError());
  }
  const bool fe = a.scheme == kSchemeForward;
  if (fe && a.dy0) {  // dL/dy0 = g_0 + (I + dt_1 J(y_0))^T a_1
    LargeArgs la{};
    la.B = B; la.N = N; la.n4 = n4; la.per_series = a.per_series; la.fwd_euler = 1;
    la.times = a.times; la.lengths = a.lengths; la.params = a.params;
    la.ytraj = a.y; la.g = a.grad_out; la.carry = w.carry; la.dy0 = a.dy0;
    TVI_TRY(launch_user(k.fe_dy0, dim3(blocks_for(B, kThreads)), la, s));
  }
  const int per = a.per_series ? B * P : P;
  const int cnt = B * n > per ? B * n : per;
  note_launch();
  large_adjoint_end_kernel<<<blocks_for(cnt, 256), 256, 0, s>>>(
      B, n, n4, N + 1, P, a.per_series, fe ? 1 : 0, w.carry, a.grad_out, w.acc, a.dy0,
      a.dparams, w.err);
  return cudaGetLastError();
}

}  // namespace tvi
