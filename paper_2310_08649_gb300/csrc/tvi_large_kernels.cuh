// tvi_large_kernels.cuh -- the model-dependent kernels of user models with
// 4 < n <= 40, compiled at run time together with the user's functions.
//
// Above n = 4 a step's n x n block no longer fits one thread's registers, so
// these models take the large-state route of the MLP engine: every (series,
// step) pair of the chunk is a thread here, the blocks are formed by one warp
// each, and the chunk system is solved by the chain solve of tvi_mlp.cu, chosen
// by width (the tiled hybrid of Sec. 3.3 up to n = 16, block forward
// substitution -- Thomas's algorithm, which the paper finds faster for larger
// systems, Sec. 5.3 -- above).  One Newton iteration (Alg. 1):
//   large_residual_kernel    R_j = dy_j - dy_{j-1} - dt_k h(y_i + dy_j, t_k) in
//                            FP64 (forward Euler: h at y_{k-1}, t_{k-1}),
//                            per-series max |R| (integer atomics on bits)
//   large_block_kernel       J = dh/dy in the block type; A = I - dt J inverted
//                            in registers, one warp per pair (forward Euler:
//                            B = I + dt J, no inverse)
// and the adjoint (App. A.2), chunks in reverse over the stored trajectory:
//   large_block_kernel       (reverse rows) the A^-T blocks (B^T)
//   large_adj_residual_kernel  the FP64 residual of the adjoint recurrence
//                            (refinement of the mixed-precision solve)
//   large_param_kernel       acc_b += sum_k dt_k (dh/dp)^T a_k, one block per
//                            series, fixed summation order
//   large_fe_dy0_kernel      forward Euler's dL/dy0 through the first step
// Model is the adapter of the user's functions (tvi_jit.cu).
#pragma once

#include "tvi_device.cuh"
#include "tvi_internal.h"

namespace tvi {
namespace klarge {

constexpr int kLargeThreads = 128;

__device__ __forceinline__ int step_index(int reverse, int i0, int L, int j) {
  return reverse ? i0 + L - j : i0 + 1 + j;
}

__device__ __forceinline__ int series_len(const LargeArgs& a, int b) {
  return a.lengths ? min(max(a.lengths[b], 0), a.N) : a.N;
}

// dt of step k; padded steps (k > len) have dt = 0 (identity rows)
__device__ __forceinline__ double step_dt_of(const double* tb, int len, int k) {
  return (k >= 1 && k <= len) ? tb[k] - tb[k - 1] : 0.0;
}

template <class Model>
__global__ void __launch_bounds__(kLargeThreads) large_residual_kernel(LargeArgs a) {
  constexpr int NS = Model::NS;
  const int b = blockIdx.y;
  if (a.active && !a.active[b]) return;  // block-uniform
  const int j = blockIdx.x * kLargeThreads + threadIdx.x;
  unsigned long long mx = 0ull;
  if (j < a.L) {
    Model mdl;
    mdl.load(a.params, b, a.per_series);
    const double* tb = a.times + static_cast<size_t>(b) * (a.N + 1);
    const int k = a.i0 + 1 + j;
    const double dt = step_dt_of(tb, series_len(a, b), k);
    const double* yi = a.yi + static_cast<size_t>(b) * a.n4;
    const double* dyj = a.dy + (static_cast<size_t>(b) * a.c + j) * a.n4;
    double y[NS], h[NS];
    // backward Euler evaluates h at (y_k, t_k), forward Euler at (y_{k-1}, t_{k-1})
    if (a.fwd_euler) {
#pragma unroll
      for (int s = 0; s < NS; ++s) y[s] = yi[s] + (j > 0 ? dyj[s - a.n4] : 0.0);
    } else {
#pragma unroll
      for (int s = 0; s < NS; ++s) y[s] = yi[s] + dyj[s];
    }
    mdl.rhs(y, a.fwd_euler ? tb[k - 1] : tb[k], h);
    double* Rj = a.R + (static_cast<size_t>(b) * a.c + j) * a.n4;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const double prev = j > 0 ? dyj[s - a.n4] : 0.0;
      const double R = fma(-dt, h[s], dyj[s] - prev);
      Rj[s] = R;
      mx = umax64(mx, abs_bits(R));
    }
    for (int s = NS; s < a.n4; ++s) Rj[s] = 0.0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = umax64(mx, __shfl_xor_sync(kFull, mx, o));
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(a.norm + b, mx);
}

// lanes that form one block: a power of two >= N4 up to a warp (a warp holds
// 32 / SEG blocks); wider blocks give each lane RPL = ceil(N4 / 32) rows
template <int N4>
constexpr int block_lanes() {
  return N4 <= 8 ? 8 : (N4 <= 16 ? 16 : 32);
}

// Block of pair j: A = I - dt_k J(y_j, t_k) inverted by Gauss-Jordan with
// partial pivoting, stored in the pair's slot as the chain reads it (A^-1
// transposed; A^-T when reverse), padded to N4 with the identity.  A group of
// SEG lanes forms one block, so a warp forms 32 / SEG at once (4 at N4 = 8).
// The group's first lane evaluates J into shared memory; lane r < N4 of the
// group then keeps row r of [A | I] in registers.  Pivoting without row swaps:
// step k takes the unused row of largest |A[r][k]| (a butterfly argmax within
// the group, first of equal maxima), the pivot row is broadcast by shuffles,
// and every row takes one FMA per entry: row_r -= (A[r][k] / piv) row_p, and
// the pivot row -= (1 - 1 / piv) itself, which scales it.  The row that pivoted
// at step k holds row k of A^-1 in its right half.  The result leaves through
// shared memory (coalesced stores).  Forward Euler's blocks B = I + dt J need no
// inverse.  Groups past the chunk's end run the elimination on the identity
// (their lanes take part in the shuffles) and store nothing.
template <class Model, typename T, int N4>
__global__ void __launch_bounds__(128) large_block_kernel(LargeArgs a) {
  constexpr int NS = Model::NS;
  constexpr int SEG = block_lanes<N4>();
  constexpr int G = 32 / SEG;   // blocks per warp
  constexpr int LD = N4 + 1;    // padded row stride of the staging buffer
  // blocks wider than a warp stage J in their own output slot (global memory)
  // and store the result from registers: a shared buffer per warp would exceed
  // the static shared memory of four warps
  constexpr bool kWide = N4 > 32;
  __shared__ T s_buf[4][G][kWide ? 1 : N4 * LD];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / SEG, lg = lane - grp * SEG;
  const int b = blockIdx.y;
  if (a.active && !a.active[b]) return;  // block-uniform
  const int jw = (blockIdx.x * 4 + warp) * G;  // first pair of the warp
  if (jw >= a.L) return;                       // warp-uniform
  const int j = jw + grp;
  const bool live = j < a.L;
  const int jc = live ? j : jw;  // a valid row for the index arithmetic
  T* slot = static_cast<T*>(a.J) + (static_cast<size_t>(b) * a.c + jc) * N4 * N4;
  T* buf = kWide ? slot : s_buf[warp][grp];
  const double* tb = a.times + static_cast<size_t>(b) * (a.N + 1);
  const int k = step_index(a.reverse, a.i0, a.L, jc);
  // forward Euler couples a_k to a_{k+1} through step k+1 in the adjoint
  const int len = series_len(a, b);
  const T dt = live ? static_cast<T>(step_dt_of(tb, len, a.fwd_euler && a.reverse ? k + 1 : k))
                    : T(0);
  if (lg == 0 && live) {
    Model mdl;
    mdl.load(a.params, b, a.per_series);
    double y[NS];
    // J at (y_k, t_k), except forward Euler's forward blocks: at (y_{k-1}, t_{k-1})
    const bool prev = a.fwd_euler && !a.reverse;
    if (a.reverse) {
      const double* yk = a.ytraj + (static_cast<size_t>(b) * (a.N + 1) + k) * NS;
#pragma unroll
      for (int s = 0; s < NS; ++s) y[s] = yk[s];
    } else {
      const double* yi = a.yi + static_cast<size_t>(b) * a.n4;
      const double* dyj = a.dy + (static_cast<size_t>(b) * a.c + j) * a.n4;
      const int jj = prev ? j - 1 : j;
#pragma unroll
      for (int s = 0; s < NS; ++s) y[s] = yi[s] + (jj >= 0 ? dyj[(jj - j) * a.n4 + s] : 0.0);
    }
    mdl.template jacobian<T>(y, prev ? tb[k - 1] : tb[k], buf);  // J, NS x NS row-major
  }
  __syncwarp();
  if (a.fwd_euler && kWide) {
    // lane lg holds rows rr = lg + 32 u of B = I + dt J; every lane reads J before
    // any lane overwrites the slot
    T Bv[(N4 + 31) / 32][N4];
#pragma unroll
    for (int u = 0; u < (N4 + 31) / 32; ++u) {
      const int rr = lg + 32 * u;
#pragma unroll
      for (int q = 0; q < N4; ++q) {
        const T Jv = (rr < NS && q < NS) ? buf[rr * NS + q] : T(0);
        Bv[u][q] = fma(dt, Jv, rr == q ? T(1) : T(0));
      }
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < (N4 + 31) / 32; ++u) {
      const int rr = lg + 32 * u;
      if (rr < N4)
#pragma unroll
        for (int q = 0; q < N4; ++q) {
          if (a.reverse) slot[rr * N4 + q] = Bv[u][q];
          else slot[q * N4 + rr] = Bv[u][q];
        }
    }
    return;
  }
  if (a.fwd_euler) {
    // no inverse: the block is B = I + dt J (forward, stored transposed as the chain
    // reads it) or B^T (adjoint), slot[r][q] = B[q][r] or B[r][q]
    if (live) {
      for (int i = lg; i < N4 * N4; i += SEG) {
        const int r = i / N4, q = i - r * N4;
        const int rr = a.reverse ? r : q, cc = a.reverse ? q : r;  // B[rr][cc]
        const T Jv = (rr < NS && cc < NS) ? buf[rr * NS + cc] : T(0);
        slot[i] = fma(dt, Jv, rr == cc ? T(1) : T(0));
      }
    }
    return;
  }
  // lane lg keeps rows lg + SEG * u (u < RPL) of [A | I]
  constexpr int RPL = (N4 + SEG - 1) / SEG;
  T row[RPL][2 * N4];
  bool used[RPL];
  int myk[RPL];
#pragma unroll
  for (int u = 0; u < RPL; ++u) {
    const int rr = lg + SEG * u;
#pragma unroll
    for (int q = 0; q < N4; ++q) {
      const T Jv = (live && rr < NS && q < NS) ? buf[rr * NS + q] : T(0);
      row[u][q] = rr < N4 ? fma(-dt, Jv, rr == q ? T(1) : T(0)) : T(0);
      row[u][N4 + q] = rr == q ? T(1) : T(0);
    }
    used[u] = rr >= N4;  // lanes without a row never pivot
    myk[u] = 0;
  }
  __syncwarp();  // buf is reused for the result
#pragma unroll
  for (int kk = 0; kk < N4; ++kk) {
    // NaN rows sort high (and stay NaN): every lane of the group agrees on the pivot
    T v = T(-1);
    int p = N4;
#pragma unroll
    for (int u = 0; u < RPL; ++u) {
      const T x = fabs(row[u][kk]);
      const T xv = used[u] ? T(-1) : (x == x ? x : static_cast<T>(__int_as_float(0x7f800000)));
      if (xv > v) {
        v = xv;
        p = lg + SEG * u;
      }
    }
#pragma unroll
    for (int o = SEG / 2; o > 0; o >>= 1) {
      const T ov = __shfl_xor_sync(kFull, v, o, SEG);
      const int op = __shfl_xor_sync(kFull, p, o, SEG);
      if (ov > v || (ov == v && op < p)) {
        v = ov;
        p = op;
      }
    }
    const int pl = p % SEG, pu = p / SEG;  // owner lane and its row slot
#pragma unroll
    for (int u = 0; u < RPL; ++u)
      if (lg == pl && u == pu) {
        used[u] = true;
        myk[u] = kk;
      }
    // the pivot row, broadcast entry by entry from its owner
    T prow[2 * N4];
#pragma unroll
    for (int q = 0; q < 2 * N4; ++q) {
      T src = row[0][q];
#pragma unroll
      for (int u = 1; u < RPL; ++u) src = (pu == u) ? row[u][q] : src;
      prow[q] = __shfl_sync(kFull, src, pl, SEG);
    }
    const T inv = T(1) / prow[kk];
#pragma unroll
    for (int u = 0; u < RPL; ++u) {
      const bool piv = lg == pl && u == pu;
      const T f = piv ? T(1) - inv : row[u][kk] * inv;
#pragma unroll
      for (int q = 0; q < 2 * N4; ++q) row[u][q] = fma(-f, prow[q], row[u][q]);
    }
  }
  if constexpr (kWide) {
    // rows myk of A^-1 straight from registers: forward slot[q][myk] (transposed),
    // reverse slot[myk][q]
#pragma unroll
    for (int u = 0; u < RPL; ++u)
      if (lg + SEG * u < N4) {
#pragma unroll
        for (int q = 0; q < N4; ++q) {
          if (a.reverse) slot[myk[u] * N4 + q] = row[u][N4 + q];
          else slot[q * N4 + myk[u]] = row[u][N4 + q];
        }
      }
    return;
  }
#pragma unroll
  for (int u = 0; u < RPL; ++u)
    if (lg + SEG * u < N4) {
#pragma unroll
      for (int q = 0; q < N4; ++q) buf[myk[u] * LD + q] = row[u][N4 + q];  // A^-1[myk][q]
    }
  __syncwarp();
  if (live) {
    for (int i = lg; i < N4 * N4; i += SEG) {
      const int r = i / N4, q = i - r * N4;
      // forward: slot[r][q] = A^-1[q][r] (transposed); reverse: slot[r][q] = A^-1[r][q]
      slot[i] = a.reverse ? buf[r * LD + q] : buf[q * LD + r];
    }
  }
}

template <class Model>
__global__ void __launch_bounds__(kLargeThreads) large_adj_residual_kernel(LargeArgs a) {
  constexpr int NS = Model::NS;
  const int b = blockIdx.y;
  const int j = blockIdx.x * kLargeThreads + threadIdx.x;
  if (j >= a.L) return;
  Model mdl;
  mdl.load(a.params, b, a.per_series);
  const double* tb = a.times + static_cast<size_t>(b) * (a.N + 1);
  const int k = a.i0 + a.L - j;
  // backward Euler: (I - dt_k J_k)^T a_k = a_{k+1} + g_k; forward Euler:
  // a_k = g_k + (I + dt_{k+1} J_k)^T a_{k+1}, J_k = dh/dy at (y_k, t_k) in both
  const double dt = step_dt_of(tb, series_len(a, b), a.fwd_euler ? k + 1 : k);
  double y[NS], J[NS * NS];
  const double* yk = a.ytraj + (static_cast<size_t>(b) * (a.N + 1) + k) * NS;
#pragma unroll
  for (int s = 0; s < NS; ++s) y[s] = yk[s];
  mdl.template jacobian<double>(y, tb[k], J);
  const double* aj = a.av + (static_cast<size_t>(b) * a.c + j) * a.n4;
  const double* ap = j > 0 ? aj - a.n4 : a.carry + static_cast<size_t>(b) * a.n4;
  const double* gk = a.g + (static_cast<size_t>(b) * (a.N + 1) + k) * NS;
  const double* ax = a.fwd_euler ? ap : aj;  // the adjoint row J^T multiplies
  double* rj = a.R + (static_cast<size_t>(b) * a.c + j) * a.n4;
  for (int p = 0; p < NS; ++p) {
    double s = 0.0;
    for (int q = 0; q < NS; ++q) s = fma(J[q * NS + p], ax[q], s);  // (J^T a)_p
    rj[p] = fma(dt, s, gk[p] + ap[p] - aj[p]);
  }
  for (int p = NS; p < a.n4; ++p) rj[p] = 0.0;
}

template <class Model>
__global__ void __launch_bounds__(kLargeThreads) large_param_kernel(LargeArgs a) {
  constexpr int NS = Model::NS;
  constexpr int NP = Model::NP;
  __shared__ double s_part[kLargeThreads / 32][NP];
  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  Model mdl;
  mdl.load(a.params, b, a.per_series);
  const double* tb = a.times + static_cast<size_t>(b) * (a.N + 1);
  const int len = series_len(a, b);
  double acc[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) acc[q] = 0.0;
  for (int j = tid; j < a.L; j += kLargeThreads) {
    const int k = a.i0 + a.L - j;
    const double dt = step_dt_of(tb, len, k);
    if (dt == 0.0) continue;
    double y[NS], av[NS];
    // step k evaluates h at (y_k, t_k) (backward Euler) or (y_{k-1}, t_{k-1})
    const int ke = a.fwd_euler ? k - 1 : k;
    const double* yk = a.ytraj + (static_cast<size_t>(b) * (a.N + 1) + ke) * NS;
    const double* aj = a.av + (static_cast<size_t>(b) * a.c + j) * a.n4;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      y[s] = yk[s];
      av[s] = aj[s];
    }
    mdl.vjp_p(y, tb[ke], av, dt, acc);
  }
  // deterministic block sum: warp tree, then the warps in order
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0) s_part[warp][q] = v;
  }
  __syncthreads();
  for (int q = tid; q < NP; q += kLargeThreads) {  // NP may exceed the block's threads
    double v = 0.0;
    for (int w = 0; w < kLargeThreads / 32; ++w) v += s_part[w][q];
    a.acc[static_cast<size_t>(b) * NP + q] += v;
  }
}

// Forward Euler's dL/dy0 = g_0 + (I + dt_1 J(y_0, t_0))^T a_1, a_1 = the carry
// after the first chunk; one thread per series.
template <class Model>
__global__ void __launch_bounds__(kLargeThreads) large_fe_dy0_kernel(LargeArgs a) {
  constexpr int NS = Model::NS;
  const int b = blockIdx.x * kLargeThreads + threadIdx.x;
  if (b >= a.B) return;
  Model mdl;
  mdl.load(a.params, b, a.per_series);
  const double* tb = a.times + static_cast<size_t>(b) * (a.N + 1);
  const double dt = a.N >= 1 ? step_dt_of(tb, series_len(a, b), 1) : 0.0;
  double y[NS], J[NS * NS];
  const double* y0 = a.ytraj + static_cast<size_t>(b) * (a.N + 1) * NS;
#pragma unroll
  for (int s = 0; s < NS; ++s) y[s] = y0[s];
  mdl.template jacobian<double>(y, tb[0], J);
  const double* cr = a.carry + static_cast<size_t>(b) * a.n4;
  const double* g0 = a.g + static_cast<size_t>(b) * (a.N + 1) * NS;
  for (int p = 0; p < NS; ++p) {
    double s = 0.0;
    for (int q = 0; q < NS; ++q) s = fma(J[q * NS + p], cr[q], s);
    a.dy0[static_cast<size_t>(b) * NS + p] = fma(dt, s, g0[p] + cr[p]);
  }
}

}  // namespace klarge
}  // namespace tvi
