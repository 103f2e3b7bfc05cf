// tvi_small.cu -- fused per-series kernels for small state sizes (n <= 4).
//
// One thread block owns one series for the whole integration: it marches
// through the chunks (Alg. 1 outer loop), runs the Newton loop of each chunk
// on-chip (residual assembly, convergence norm, block inverses, cyclic
// reduction, update), writes the converged chunk to the trajectory and
// carries y_{i+c} to the next chunk.  Series are independent (Sec. 2.1), so
// blocks never wait on one another and a converged series stops iterating
// while others continue (the per-series freezing reading of Alg. 1).
//
// Thread t holds the RPT consecutive steps t*RPT .. t*RPT+RPT-1 of the chunk.
// Per Newton iteration:
//   residual   R_j = dy_j - dy_{j-1} - dt_j h(y_i + dy_j)     FP64 (Eq. batched-backward-euler)
//   norm       ||R||_inf over the chunk, block max             FP64 bits, integer pipe
//   blocks     A_j = I - dt_j j(y_i + dy_j), M_j = A_j^-1, v_j = M_j R_j      in T
//   reduction  d_j = M_j d_{j-1} + v_j  by serial runs + cyclic reduction  in T
//   update     dy_j -= d_j                                   FP64
// T = double (FP64 mode) or float (mixed mode: the FP64 residual makes Newton
// an iterative refinement that converges to the FP64 solution).  The iterate is
// held as y_j = y_i + dy_j itself.  Forward Euler (Sec. 2.2, explicit methods)
// uses the same loop with h and j taken at y_{j-1}: R_j = y_j - y_{j-1} -
// dt_j h(y_{j-1}) and d_j = (I + dt_j j(y_{j-1})) d_{j-1} + R_j (no inverse).
#include "tvi_device.cuh"
#include "tvi_internal.h"
#include "tvi_models.cuh"
#include "tvi_small_kernels.cuh"

namespace tvi {

namespace {

using kern::adjoint_small_kernel;
using kern::forward_small_kernel;

template <class Model, typename T, int RPT>
cudaError_t launch_fwd(const FwdArgs& a, int threads, cudaStream_t s) {
  note_launch();
  forward_small_kernel<Model, T, RPT><<<a.B, threads, 0, s>>>(a);
  return cudaGetLastError();
}

template <class Model, typename T, int RPT>
cudaError_t launch_adj(const AdjArgs& a, int threads, cudaStream_t s) {
  note_launch();
  adjoint_small_kernel<Model, T, RPT><<<a.B, threads, 0, s>>>(a);
  return cudaGetLastError();
}

template <class Model, typename T>
cudaError_t dispatch_fwd_rpt(const FwdArgs& a, int rpt, int threads, cudaStream_t s) {
  switch (rpt) {
    case 1: return launch_fwd<Model, T, 1>(a, threads, s);
    case 2: return launch_fwd<Model, T, 2>(a, threads, s);
    case 4: return launch_fwd<Model, T, 4>(a, threads, s);
    case 8: return launch_fwd<Model, T, 8>(a, threads, s);
    default: return cudaErrorInvalidValue;
  }
}

template <class Model, typename T>
cudaError_t dispatch_adj_rpt(const AdjArgs& a, int rpt, int threads, cudaStream_t s) {
  switch (rpt) {
    case 1: return launch_adj<Model, T, 1>(a, threads, s);
    case 2: return launch_adj<Model, T, 2>(a, threads, s);
    case 4: return launch_adj<Model, T, 4>(a, threads, s);
    case 8: return launch_adj<Model, T, 8>(a, threads, s);
    default: return cudaErrorInvalidValue;
  }
}

__global__ void sum_partials_kernel(const double* partials, int B, int P, double* out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double s = 0.0;
  for (int b = 0; b < B; ++b) s += partials[static_cast<size_t>(b) * P + p];  // series order
  out[p] = s;
}

}  // namespace

bool small_supported(int kind, int n) {
  if (kind == kKindVdp) return n == 2;
  if (kind == kKindLinear) return n == 2 || n == 4;
  return false;
}

// Steps per thread: the smallest power of two whose block fits the kernel's
// thread bound, raised to `preferred` when given; threads = ceil(c / rpt)
// rounded up to a whole warp.  Every shape holds up to kSmallMaxChunk steps.
void small_launch_shape(int chunk, int preferred, int* rpt, int* threads) {
  int r = 1;
  while (r < 8 && (chunk + r - 1) / r > small_max_threads(r)) r *= 2;
  if (preferred == 1 || preferred == 2 || preferred == 4 || preferred == 8) r = r > preferred ? r : preferred;
  int t = (chunk + r - 1) / r;
  t = ((t + 31) / 32) * 32;
  if (t > small_max_threads(r)) t = small_max_threads(r);
  *rpt = r;
  *threads = t;
}

cudaError_t small_forward(int kind, int n, int precision, int rpt, int threads, const FwdArgs& a,
                          cudaStream_t s) {
  const bool f64 = precision == kPrecFp64;
  if (kind == kKindVdp)
    return f64 ? dispatch_fwd_rpt<ModelVdp, double>(a, rpt, threads, s)
               : dispatch_fwd_rpt<ModelVdp, float>(a, rpt, threads, s);
  if (n == 2)
    return f64 ? dispatch_fwd_rpt<ModelLinear<2>, double>(a, rpt, threads, s)
               : dispatch_fwd_rpt<ModelLinear<2>, float>(a, rpt, threads, s);
  return f64 ? dispatch_fwd_rpt<ModelLinear<4>, double>(a, rpt, threads, s)
             : dispatch_fwd_rpt<ModelLinear<4>, float>(a, rpt, threads, s);
}

cudaError_t small_adjoint(int kind, int n, int precision, int rpt, int threads, const AdjArgs& a,
                          int P, cudaStream_t s) {
  const bool f64 = precision == kPrecFp64;
  cudaError_t e;
  if (kind == kKindVdp)
    e = f64 ? dispatch_adj_rpt<ModelVdp, double>(a, rpt, threads, s)
            : dispatch_adj_rpt<ModelVdp, float>(a, rpt, threads, s);
  else if (n == 2)
    e = f64 ? dispatch_adj_rpt<ModelLinear<2>, double>(a, rpt, threads, s)
            : dispatch_adj_rpt<ModelLinear<2>, float>(a, rpt, threads, s);
  else
    e = f64 ? dispatch_adj_rpt<ModelLinear<4>, double>(a, rpt, threads, s)
            : dispatch_adj_rpt<ModelLinear<4>, float>(a, rpt, threads, s);
  if (e != cudaSuccess) return e;
  return a.per_series ? cudaSuccess : small_sum_partials(a, P, s);
}

cudaError_t small_sum_partials(const AdjArgs& a, int P, cudaStream_t s) {
  note_launch();
  sum_partials_kernel<<<(P + 127) / 128, 128, 0, s>>>(a.partials, a.B, P, a.dparams);
  return cudaGetLastError();
}

}  // namespace tvi
