// tvi_mlp.cu -- neural-ODE models (h = MLP(y)), state sizes up to 32.
//
// The right-hand side is the three-layer MLP of the paper's neural ODE (Sec.
// 5.1.1): tanh after every layer, or SiLU after the two hidden layers with a
// linear output.  Evaluating it in FP64 for the Newton residual costs
// 2 (n h1 + h1 h2 + h2 n) FP64 flops per (series, step) -- 12.3k at n = 16,
// 49k at n = 32 -- which on GB300 (FP64 at 1/64 of FP32) outweighs the rest of
// an iteration, so this path spreads the steps of all series over the whole GPU
// instead of giving each series one block.  One Newton iteration of a chunk
// (Alg. 1), all series at once, converged series skipped:
//   mlp_residual_kernel  FP64 MLP at y_i + dy_j -> R_j (Eq. batched-backward-
//                        euler), per-series max |R| (integer atomics on FP64
//                        bits), activation derivatives (FP64, so FP64 blocks
//                        are exact)
//   mlp_check_kernel     per-series convergence (reading C-4); the host reads
//                        how many series still iterate
//   mlp_blocks_kernel    J = D3 W3 D2 W2 D1 W1, A = I - dt J, M = A^-1 in the
//                        block precision (Sec. 3.2: factorise the diagonal blocks)
//   mlp_chain_kernel     d_j = M_j (d_{j-1} + R_j) per series, dy -= d (FP64)
// The adjoint (App. A.2) runs the chunks in reverse with transposed blocks: a
// derivative pass at the stored trajectory (mlp_residual_kernel in reverse
// mode, which also keeps the activations), refinement residuals
// r = g + a_next - a + dt J^T a assembled in FP64 around a backward-only
// vector-Jacobian product (mlp_vjp_kernel), and the parameter gradient
// sum_k dt_k (dh/dp)^T a_k as tiled outer-product sums (mlp_param_grad_kernel).
// With FP64 blocks every MLP pass is FP64; with FP32 / BF16 blocks the
// adjoint's MLP passes run in FP32 (64x the FP64 rate on this part), which
// bounds the gradient's relative error near 1e-7 instead of 1e-15.
#include <cstdlib>
#include <functional>
#include <cuda_runtime.h>

#include "tvi_device.cuh"
#include "tvi_internal.h"
#include "tvi_tc.cuh"

namespace tvi {

namespace {

constexpr int kTileThreads = 256;

struct MlpDims {
  int n, h1, h2, P;
};

template <typename T>
struct MlpW {
  const T *W1, *b1, *W2, *b2, *W3, *b3;
};

template <typename T>
__device__ __forceinline__ MlpW<T> mlp_split(const T* p, const MlpDims& d) {
  MlpW<T> w;
  w.W1 = p;
  w.b1 = w.W1 + d.h1 * d.n;
  w.W2 = w.b1 + d.h1;
  w.b2 = w.W2 + d.h2 * d.h1;
  w.W3 = w.b2 + d.h2;
  w.b3 = w.W3 + d.n * d.h2;
  return w;
}

// activation and its derivative, in the arithmetic of T (FP64 or FP32)
__device__ __forceinline__ double tanh_t(double z) { return tanh(z); }
__device__ __forceinline__ float tanh_t(float z) { return tanhf(z); }
__device__ __forceinline__ double exp_t(double z) { return exp(z); }
__device__ __forceinline__ float exp_t(float z) { return expf(z); }

template <int KIND, typename T>
__device__ __forceinline__ void act_hidden(T z, T& a, T& da) {
  if constexpr (KIND == kKindMlpTanh) {
    a = tanh_t(z);
    da = T(1) - a * a;
  } else {
    const T s = T(1) / (T(1) + exp_t(-z));
    a = z * s;
    da = s + z * s * (T(1) - s);
  }
}

template <int KIND, typename T>
__device__ __forceinline__ void act_out(T z, T& a, T& da) {
  if constexpr (KIND == kKindMlpTanh) {
    a = tanh_t(z);
    da = T(1) - a * a;
  } else {
    a = z;
    da = T(1);
  }
}

__device__ __forceinline__ int step_of(int reverse, int i0, int L, int j) {
  return reverse ? i0 + L - j : i0 + 1 + j;
}

// dt of step k (1 <= k <= len); 0 for padded steps and for k = 0, the state
// y_0 that the forward-Euler adjoint's one-row pass visits (no read of tb[-1])
__device__ __forceinline__ double step_dt(const double* tb, int len, int k) {
  return (k >= 1 && k <= len) ? tb[k] - tb[k - 1] : 0.0;
}

// ---------------------------------------------------------------------------
// FP32 products of a tile of TP pairs: out(r, p) = sum_k A(r, k) X[k][p] for
// r < R (a multiple of 4), with A(r, k) = Wg[r sr + k sk] read through the
// read-only cache and X [K][TP] in shared memory.  Each thread owns 4 x 4
// output tiles; the lanes of a warp share a row group, so the weight loads are
// broadcasts.  The weights of a k come in one 16-byte load when the four rows
// are adjacent (kRowsAdjacent: sr = 1, the transposed products of the adjoint),
// else those of four k at once per row when K is contiguous (sk = 1, K a
// multiple of 4); k runs in ascending order either way.  epi(r, p, value)
// receives every result.
// ---------------------------------------------------------------------------
template <int TP, bool kRowsAdjacent, typename Epi>
__device__ __forceinline__ void tile_mm_f32(const float* __restrict__ Wg, int sr, int sk, int R,
                                            int K, const float* X, Epi epi) {
  constexpr int PG = TP / 4;
  const int tiles = (R / 4) * PG;
  for (int tt = threadIdx.x; tt < tiles; tt += kTileThreads) {
    const int r0 = (tt / PG) * 4, p0 = (tt % PG) * 4;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    const float* w0 = Wg + static_cast<size_t>(r0) * sr;
    auto step = [&](const float (&w)[4], const float4& x) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        acc[i][0] = fmaf(w[i], x.x, acc[i][0]);
        acc[i][1] = fmaf(w[i], x.y, acc[i][1]);
        acc[i][2] = fmaf(w[i], x.z, acc[i][2]);
        acc[i][3] = fmaf(w[i], x.w, acc[i][3]);
      }
    };
    if constexpr (kRowsAdjacent) {  // sr = 1: A(r0 .. r0 + 3, k) adjacent
#pragma unroll 2
      for (int k = 0; k < K; ++k) {
        const float4 x = *reinterpret_cast<const float4*>(X + k * TP + p0);
        const float4 wv = __ldg(reinterpret_cast<const float4*>(w0 + static_cast<size_t>(k) * sk));
        const float w[4] = {wv.x, wv.y, wv.z, wv.w};
        step(w, x);
      }
    } else {  // sk = 1: A(r, k .. k + 3) adjacent
      for (int k = 0; k < K; k += 4) {
        float4 wr[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          wr[i] = __ldg(reinterpret_cast<const float4*>(w0 + static_cast<size_t>(i) * sr + k));
        const float wk0[4] = {wr[0].x, wr[1].x, wr[2].x, wr[3].x};
        const float wk1[4] = {wr[0].y, wr[1].y, wr[2].y, wr[3].y};
        const float wk2[4] = {wr[0].z, wr[1].z, wr[2].z, wr[3].z};
        const float wk3[4] = {wr[0].w, wr[1].w, wr[2].w, wr[3].w};
        step(wk0, *reinterpret_cast<const float4*>(X + k * TP + p0));
        step(wk1, *reinterpret_cast<const float4*>(X + (k + 1) * TP + p0));
        step(wk2, *reinterpret_cast<const float4*>(X + (k + 2) * TP + p0));
        step(wk3, *reinterpret_cast<const float4*>(X + (k + 3) * TP + p0));
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) epi(r0 + i, p0 + j, acc[i][j]);
  }
}

// ---------------------------------------------------------------------------
// Forward pass (in T: FP64, or FP32 for the mixed-precision adjoint) for a tile
// of TP pairs held in shared memory.  Thread t takes pair p = t % TP and every
// G-th output row (G = threads / TP), so the lanes of a warp read the same
// weight row (broadcast through the read-only cache).  Layouts [row][TP] keep
// the pairs contiguous (no bank conflicts).
//   sy [n][TP] in; sa1 [h1][TP], sa2 [h2][TP], sz3 [n][TP] out;
//   dv_tile (optional) receives act'(z) of the hidden layers ([pair][dvs], FP64).
// ---------------------------------------------------------------------------
template <int KIND, int TP, typename T>
__device__ __forceinline__ void mlp_tile_forward(const MlpW<T>& w, const MlpDims& d, const T* sy,
                                                 T* sa1, T* sa2, T* sz3, int np, double* dv_tile,
                                                 int dvs) {
  if constexpr (sizeof(T) == sizeof(float)) {
    tile_mm_f32<TP, false>(w.W1, d.n, 1, d.h1, d.n, sy, [&](int r, int p, float z) {
      float a, da;
      act_hidden<KIND>(z + __ldg(w.b1 + r), a, da);
      sa1[r * TP + p] = a;
      if (dv_tile && p < np) dv_tile[p * dvs + r] = widen(da);
    });
    __syncthreads();
    tile_mm_f32<TP, false>(w.W2, d.h1, 1, d.h2, d.h1, sa1, [&](int r, int p, float z) {
      float a, da;
      act_hidden<KIND>(z + __ldg(w.b2 + r), a, da);
      sa2[r * TP + p] = a;
      if (dv_tile && p < np) dv_tile[p * dvs + d.h1 + r] = widen(da);
    });
    __syncthreads();
    tile_mm_f32<TP, false>(w.W3, d.h2, 1, d.n, d.h2, sa2,
                    [&](int r, int p, float z) { sz3[r * TP + p] = z + __ldg(w.b3 + r); });
    __syncthreads();
    return;
  }
  constexpr int G = kTileThreads / TP;
  const int t = threadIdx.x, p = t % TP, g = t / TP;
  const bool live = p < np;
  for (int r = g; r < d.h1; r += G) {
    T acc = w.b1[r];
    const T* wr = w.W1 + r * d.n;
    for (int c = 0; c < d.n; ++c) acc = fma(__ldg(wr + c), sy[c * TP + p], acc);
    T a, da;
    act_hidden<KIND>(acc, a, da);
    sa1[r * TP + p] = a;
    if (dv_tile && live) dv_tile[p * dvs + r] = static_cast<double>(da);
  }
  __syncthreads();
  for (int r = g; r < d.h2; r += G) {
    T acc = w.b2[r];
    const T* wr = w.W2 + r * d.h1;
    for (int c = 0; c < d.h1; ++c) acc = fma(__ldg(wr + c), sa1[c * TP + p], acc);
    T a, da;
    act_hidden<KIND>(acc, a, da);
    sa2[r * TP + p] = a;
    if (dv_tile && live) dv_tile[p * dvs + d.h1 + r] = static_cast<double>(da);
  }
  __syncthreads();
  for (int r = g; r < d.n; r += G) {
    T acc = w.b3[r];
    const T* wr = w.W3 + r * d.h2;
    for (int c = 0; c < d.h2; ++c) acc = fma(__ldg(wr + c), sa2[c * TP + p], acc);
    sz3[r * TP + p] = acc;
  }
  __syncthreads();
}

__global__ void convert_weights_kernel(const double* p, float* f, int P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P) f[i] = static_cast<float>(p[i]);
}

// ---------------------------------------------------------------------------
// Residual (forward) or activation derivatives at the stored trajectory
// (adjoint).  Grid: (ceil(L / TP), B).
// ---------------------------------------------------------------------------
struct ResidualArgs {
  MlpDims d;
  int B, N, i0, L, c;
  int reverse;               // 1: adjoint -- y from the trajectory at step i0 + L - j, no R
  int fe;                    // forward Euler (forward pass): h and its derivatives at y_{j-1}
  const double* times;
  const int* lengths;
  const double* params;      // FP64 parameters (T = double)
  const float* Wf;           // FP32 copy (T = float: the mixed-precision adjoint)
  const double* yi;          // [B][n] chunk start (forward)
  const double* dy;          // [B][c][n] (forward)
  const double* ytraj;       // [B][N+1][n] (adjoint)
  double* R;                 // [B][c][n] (forward)
  double* dv;                // [B][c][h1+h2+n]
  unsigned long long* norm;  // [B] max |R| bits (forward)
  const int* active;         // [B] or null
  double* act;               // [B][c][n+h1+h2+3] (y, 1, a1, 1, a2, 1) or null (adjoint)
};

// T = double: the Newton residual (forward) or the FP64 adjoint's derivative
// pass; T = float: the derivative pass of the mixed-precision adjoint.
template <int KIND, int TP, typename T>
__global__ void __launch_bounds__(kTileThreads) mlp_residual_kernel(ResidualArgs a) {
  extern __shared__ double smem[];
  const int b = blockIdx.y;
  if (a.active && !a.active[b]) return;
  const MlpDims d = a.d;
  const int j0 = blockIdx.x * TP;
  const int np = min(TP, a.L - j0);
  T* sy = reinterpret_cast<T*>(smem);
  T* sa1 = sy + d.n * TP;
  T* sa2 = sa1 + d.h1 * TP;
  T* sz3 = sa2 + d.h2 * TP;
  MlpW<T> w;
  if constexpr (sizeof(T) == sizeof(double)) w = mlp_split(a.params, d);
  else w = mlp_split(a.Wf, d);
  const double* tb = a.times + static_cast<size_t>(b) * (a.N + 1);
  const int len = a.lengths ? min(max(a.lengths[b], 0), a.N) : a.N;
  const double* dyb = a.dy ? a.dy + static_cast<size_t>(b) * a.c * d.n : nullptr;
  if (!a.reverse && a.i0 + 1 + j0 > len) {
    // every step of the tile lies past the series' length: dt = 0, so R_j =
    // dy_j - dy_{j-1} without the network (a finite h times dt = 0 adds nothing);
    // the activation derivatives are written as zeros (the blocks of these steps
    // are the identity whatever J is)
    const int dvs = d.h1 + d.h2 + d.n;
    double* dv_tile = a.dv + (static_cast<size_t>(b) * a.c + j0) * dvs;
    for (int e = threadIdx.x; e < np * dvs; e += kTileThreads) dv_tile[e] = 0.0;
    unsigned long long mx = 0ull;
    for (int e = threadIdx.x; e < np * d.n; e += kTileThreads) {
      const int j = j0 + e / d.n, r = e % d.n;
      const double prev = (j > 0) ? dyb[(j - 1) * d.n + r] : 0.0;
      const double R = dyb[j * d.n + r] - prev;
      a.R[(static_cast<size_t>(b) * a.c + j) * d.n + r] = R;
      mx = umax64(mx, abs_bits(R));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = umax64(mx, __shfl_xor_sync(kFull, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(a.norm + b, mx);
    return;
  }
  for (int e = threadIdx.x; e < d.n * TP; e += kTileThreads) {
    const int c = e / TP, p = e % TP;
    double v = 0.0;
    if (p < np) {
      const int j = j0 + p;
      if (a.reverse)
        v = a.ytraj[(static_cast<size_t>(b) * (a.N + 1) + step_of(1, a.i0, a.L, j)) * d.n + c];
      else if (a.fe)  // R_j = dy_j - dy_{j-1} - dt_j h(y_{j-1})
        v = a.yi[b * d.n + c] + (j > 0 ? dyb[(j - 1) * d.n + c] : 0.0);
      else
        v = a.yi[b * d.n + c] + dyb[j * d.n + c];
    }
    sy[e] = narrow<T>(v);
  }
  __syncthreads();
  const int dvs = d.h1 + d.h2 + d.n;
  double* dv_tile = a.dv + (static_cast<size_t>(b) * a.c + j0) * dvs;
  mlp_tile_forward<KIND, TP, T>(w, d, sy, sa1, sa2, sz3, np, dv_tile, dvs);
  constexpr int G = kTileThreads / TP;
  const int t = threadIdx.x, p = t % TP, g = t / TP;
  if (a.act && p < np) {  // activations for the parameter gradient (adjoint)
    const int aw = d.n + d.h1 + d.h2 + 3;
    double* ar = a.act + (static_cast<size_t>(b) * a.c + j0 + p) * aw;
    const double* yt = a.ytraj + (static_cast<size_t>(b) * (a.N + 1) +
                                  step_of(1, a.i0, a.L, j0 + p)) * d.n;
    for (int c = g; c < d.n; c += G) ar[c] = yt[c];
    for (int c = g; c < d.h1; c += G) ar[d.n + 1 + c] = widen(sa1[c * TP + p]);
    for (int c = g; c < d.h2; c += G) ar[d.n + 1 + d.h1 + 1 + c] = widen(sa2[c * TP + p]);
    if (g == 0) {
      ar[d.n] = 1.0;
      ar[d.n + 1 + d.h1] = 1.0;
      ar[d.n + 1 + d.h1 + 1 + d.h2] = 1.0;
    }
  }
  unsigned long long mx = 0ull;
  if (p < np) {
    const int j = j0 + p;
    const double dt = step_dt(tb, len, step_of(a.reverse, a.i0, a.L, j));
    for (int r = g; r < d.n; r += G) {
      T h, dh;
      act_out<KIND>(sz3[r * TP + p], h, dh);
      dv_tile[p * dvs + d.h1 + d.h2 + r] = widen(dh);
      if constexpr (sizeof(T) == sizeof(double)) {
        if (!a.reverse) {
          const double prev = (j > 0) ? dyb[(j - 1) * d.n + r] : 0.0;
          const double R = fma(-dt, h, dyb[j * d.n + r] - prev);
          a.R[(static_cast<size_t>(b) * a.c + j) * d.n + r] = R;
          mx = umax64(mx, abs_bits(R));
        }
      }
    }
  }
  if (!a.reverse) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = umax64(mx, __shfl_xor_sync(kFull, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(a.norm + b, mx);
  }
}

// First residual of a chunk attempt (forward pass).  The attempt starts from
// dy = 0 (Sec. 2.3), so every step of the chunk evaluates the network at the
// same point y_i + 0 (backward Euler at y_i + dy_j, forward Euler at
// y_i + dy_{j-1}).  One block per series evaluates it once -- the FP64 code and
// summation order of the per-pair tiles, so the values are the same -- and
// writes R_j = dy_j - dy_{j-1} - dt_j h = -dt_j h and the activation
// derivatives of every step of the chunk.  Grid: B.
template <int KIND>
__global__ void __launch_bounds__(kTileThreads) mlp_residual_start_kernel(ResidualArgs a) {
  __shared__ double sy[32], sa1[128], sa2[128], sz3[32], sh[32], sdv[128 + 128 + 32];
  const int b = blockIdx.x;
  if (a.active && !a.active[b]) return;
  const MlpDims d = a.d;
  const int tid = threadIdx.x;
  const MlpW<double> w = mlp_split(a.params, d);
  const double* dyb = a.dy + static_cast<size_t>(b) * a.c * d.n;
  for (int c = tid; c < d.n; c += kTileThreads) sy[c] = a.yi[b * d.n + c] + dyb[c];
  __syncthreads();
  const int dvs = d.h1 + d.h2 + d.n;
  mlp_tile_forward<KIND, 1, double>(w, d, sy, sa1, sa2, sz3, 1, sdv, dvs);
  for (int r = tid; r < d.n; r += kTileThreads) {
    double h, dh;
    act_out<KIND>(sz3[r], h, dh);
    sdv[d.h1 + d.h2 + r] = dh;
    sh[r] = h;
  }
  __syncthreads();
  // the same derivatives for every step (dvs is even: h1, h2 are multiples of 4)
  const int half = dvs / 2;
  double2* dv2 = reinterpret_cast<double2*>(a.dv + static_cast<size_t>(b) * a.c * dvs);
  for (int e = tid; e < a.L * half; e += kTileThreads) {
    const int q = e % half;
    dv2[e] = make_double2(sdv[2 * q], sdv[2 * q + 1]);
  }
  const double* tb = a.times + static_cast<size_t>(b) * (a.N + 1);
  const int len = a.lengths ? min(max(a.lengths[b], 0), a.N) : a.N;
  double* Rb = a.R + static_cast<size_t>(b) * a.c * d.n;
  unsigned long long mx = 0ull;
  for (int e = tid; e < a.L * d.n; e += kTileThreads) {
    const int j = e / d.n, r = e - j * d.n;
    const double R = fma(-step_dt(tb, len, a.i0 + 1 + j), sh[r], 0.0);
    Rb[e] = R;
    mx = umax64(mx, abs_bits(R));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = umax64(mx, __shfl_xor_sync(kFull, mx, o));
  if ((tid & 31) == 0 && mx) atomicMax(a.norm + b, mx);
}

struct CheckArgs {
  int B, it, max_iter;
  double tol_abs, tol_rel;
  unsigned long long* norm;  // [B] cleared here for the next iteration
  double* norm0;             // [B]
  int* active;               // [B]
  int* status;               // [B] (sticky)
  int* iters;                // [B] Newton updates of the current chunk
  int* remaining;            // device word: series still iterating
};

// Alg. 1 convergence test per series; counts the series that need another update.
__global__ void mlp_check_kernel(CheckArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.B || !a.active[b]) return;
  const unsigned long long nb = a.norm[b];
  a.norm[b] = 0ull;
  const double nr = __longlong_as_double(static_cast<long long>(nb));
  if (a.it == 0) a.norm0[b] = nr;
  bool stop = false;
  if (nb >= kNonFiniteBits) {
    a.status[b] = 2;
    stop = true;
  } else if (nr <= a.tol_abs || nr <= a.tol_rel * a.norm0[b]) {
    stop = true;
  } else if (a.it >= a.max_iter) {
    if (a.status[b] == 0) a.status[b] = 1;
    stop = true;
  }
  if (stop) {
    a.active[b] = 0;
  } else {
    a.iters[b] = a.it + 1;
    atomicAdd(a.remaining, 1);
  }
}

// ---------------------------------------------------------------------------
// Blocks: per pair J = D3 W3 D2 W2 D1 W1, A = I - dt J, M = A^-1 (A^-T when
// reverse) in the block precision T.  A thread block takes TP consecutive steps
// of one series and forms the products for all of them as two register-tiled
// GEMMs over the columns (pair, input component):
//     G [h2][TP n] = W2 [h2][h1] . U [h1][TP n],   U[q][(p, c)] = d1[p][q] W1[q][c]
//     J [n][TP n]  = W3 [n][h2]  . (D2 G)
// (4 x 4 outputs per thread; weights through the read-only cache; U and G in
// shared memory).  Each warp then inverts pairs by Gauss-Jordan with partial
// pivoting on [A | I] in shared memory.  Needs n, h1, h2 multiples of 4.
// ---------------------------------------------------------------------------
struct BlocksArgs {
  MlpDims d;
  int B, N, i0, L, c;
  int reverse;
  const double* times;
  const int* lengths;
  const float* Wf;    // FP32 copy of the parameters (same layout), FP32 blocks
  const double* Wd;   // the FP64 parameters, FP64 blocks
  const double* dv;   // [B][c][h1+h2+n]
  const int* active;  // [B] or null
  void* M;            // [B][c][n][n] in T
  int first_wait_polls;  // tensor-core kernel: poll limit of each block's first data wait
  int fe;             // forward Euler: B = I + dt J (no inverse); reverse rows take dt_{k+1}
};

// weight i of the flat parameter vector in the block precision
template <typename T>
__device__ __forceinline__ T wget(const BlocksArgs& a, int i) {
  if constexpr (sizeof(T) == sizeof(double)) return __ldg(a.Wd + i);
  else return __ldg(a.Wf + i);
}

// Gauss-Jordan inverse of one augmented block [A | I] (n x 2n, shared memory)
// by one warp, partial pivoting, then M = A^-1 stored transposed to Mo
// (Mo[col][r] = M[r][col]; the adjoint's blocks are M^T, stored untransposed).
template <typename T>
__device__ __forceinline__ void gj_invert_store(T* Ap, int n, int lane, T* Mo, int reverse) {
  for (int kk = 0; kk < n; ++kk) {
    T best = (lane >= kk && lane < n) ? fabs(Ap[lane * 2 * n + kk]) : T(-1);
    int piv = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(kFull, best, o);
      const int op = __shfl_xor_sync(kFull, piv, o);
      if (ob > best || (ob == best && op < piv)) {
        best = ob;
        piv = op;
      }
    }
    if (piv != kk) {
      for (int col = lane; col < 2 * n; col += 32) {
        const T tmp = Ap[kk * 2 * n + col];
        Ap[kk * 2 * n + col] = Ap[piv * 2 * n + col];
        Ap[piv * 2 * n + col] = tmp;
      }
    }
    __syncwarp();
    const T inv = T(1) / Ap[kk * 2 * n + kk];
    __syncwarp();
    for (int col = lane; col < 2 * n; col += 32) Ap[kk * 2 * n + col] *= inv;
    __syncwarp();
    // each lane updates the columns it owns; column kk is read, not written
    for (int col = lane; col < 2 * n; col += 32) {
      if (col == kk) continue;
      const T pk = Ap[kk * 2 * n + col];
      for (int r = 0; r < n; ++r)
        if (r != kk) Ap[r * 2 * n + col] = fma(-Ap[r * 2 * n + kk], pk, Ap[r * 2 * n + col]);
    }
    __syncwarp();
    for (int r = lane; r < n; r += 32)
      if (r != kk) Ap[r * 2 * n + kk] = T(0);
    __syncwarp();
  }
  for (int r = 0; r < n; ++r)
    for (int col = lane; col < n; col += 32)
      // stored transposed (Mo[col][r] = M[r][col]) for the chain's conflict-free reads
      Mo[col * n + r] = reverse ? Ap[col * 2 * n + n + r] : Ap[r * 2 * n + n + col];
  __syncwarp();
}

template <typename T>
__global__ void __launch_bounds__(kTileThreads) mlp_blocks_kernel(BlocksArgs a, int TP,
                                                                  int stage_w2) {
  extern __shared__ unsigned char smem_raw[];
  const MlpDims d = a.d;
  const int n = d.n, h1 = d.h1, h2 = d.h2;
  const int NT = TP * n;
  const int b = blockIdx.y;
  if (a.active && !a.active[b]) return;
  const int j0 = blockIdx.x * TP;
  const int np = min(TP, a.L - j0);
  // W2 transposed ([h1][h2]) when it fits: 4-wide shared loads in the inner loop
  T* sW2t = reinterpret_cast<T*>(smem_raw);
  T* sU = sW2t + (stage_w2 ? h1 * h2 : 0);  // [h1][NT]
  T* sG = sU + h1 * NT;                     // [h2][NT]
  T* sA = sG + h2 * NT;                     // [TP][n][2n]
  T* sdt = sA + TP * n * 2 * n;             // [TP]
  const int oW2 = h1 * n + h1;            // offsets in the flat parameter vector
  const int oW3 = oW2 + h2 * h1 + h2;
  const int dvs = h1 + h2 + n;
  const double* dvt = a.dv + (static_cast<size_t>(b) * a.c + j0) * dvs;
  const int tid = threadIdx.x;
  const int len = a.lengths ? min(max(a.lengths[b], 0), a.N) : a.N;
  const double* tb = a.times + static_cast<size_t>(b) * (a.N + 1);
  // forward Euler's adjoint couples a_k to a_{k+1} through step k + 1
  const int kshift = (a.fe && a.reverse) ? 1 : 0;
  for (int p = tid; p < TP; p += kTileThreads)
    sdt[p] = static_cast<T>(
        p < np ? step_dt(tb, len, step_of(a.reverse, a.i0, a.L, j0 + p) + kshift) : 0.0);
  const int ln = __ffs(n) - 1;    // n and NT are powers of two
  const int lnt = __ffs(NT) - 1;
  for (int e = tid; e < h1 * NT; e += kTileThreads) {
    const int q = e >> lnt, col = e & (NT - 1), p = col >> ln, c = col & (n - 1);
    sU[e] = (p < np) ? narrow<T>(dvt[p * dvs + q]) * wget<T>(a, q * n + c) : T(0);
  }
  if (stage_w2)
    for (int e = tid; e < h1 * h2; e += kTileThreads) {
      const int r = e / h1, q = e - r * h1;
      sW2t[q * h2 + r] = wget<T>(a, oW2 + e);
    }
  __syncthreads();
  {  // G = D2 W2 U
    const int tn = NT / 4, tiles = (h2 / 4) * tn;
    for (int tt = tid; tt < tiles; tt += kTileThreads) {
      const int r0 = (tt / tn) * 4, c0 = (tt % tn) * 4;
      T acc[4][4] = {};
      for (int q = 0; q < h1; ++q) {
        T wv[4], uv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          wv[i] = stage_w2 ? sW2t[q * h2 + r0 + i] : wget<T>(a, oW2 + (r0 + i) * h1 + q);
#pragma unroll
        for (int i = 0; i < 4; ++i) uv[i] = sU[q * NT + c0 + i];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int k2 = 0; k2 < 4; ++k2) acc[i][k2] = fma(wv[i], uv[k2], acc[i][k2]);
      }
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) {
        const int p = (c0 + k2) >> ln;
        const bool live = p < np;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const T d2v = live ? narrow<T>(dvt[p * dvs + h1 + r0 + i]) : T(0);
          sG[(r0 + i) * NT + c0 + k2] = d2v * acc[i][k2];
        }
      }
    }
  }
  __syncthreads();
  {  // A = I - dt D3 W3 G, augmented with I
    const int tn = NT / 4, tiles = (n / 4) * tn;
    for (int tt = tid; tt < tiles; tt += kTileThreads) {
      const int r0 = (tt / tn) * 4, c0 = (tt % tn) * 4;
      T acc[4][4] = {};
      for (int q = 0; q < h2; ++q) {
        T wv[4], gv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) wv[i] = wget<T>(a, oW3 + (r0 + i) * h2 + q);
#pragma unroll
        for (int i = 0; i < 4; ++i) gv[i] = sG[q * NT + c0 + i];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int k2 = 0; k2 < 4; ++k2) acc[i][k2] = fma(wv[i], gv[k2], acc[i][k2]);
      }
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) {
        const int col = c0 + k2, p = col >> ln, c = col & (n - 1);
        if (p >= np) continue;
        T* Ap = sA + p * n * 2 * n;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = r0 + i;
          const T J = narrow<T>(dvt[p * dvs + h1 + h2 + r]) * acc[i][k2];
          // backward Euler A = I - dt J (inverted below); forward Euler B = I + dt J
          Ap[r * 2 * n + c] = ((r == c) ? T(1) : T(0)) + (a.fe ? sdt[p] : -sdt[p]) * J;
          Ap[r * 2 * n + n + c] = (r == c) ? T(1) : T(0);
        }
      }
    }
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  if (a.fe) {
    // no inverse: B stored as the chain reads it (Mo[col][r] = B[r][col]; the
    // adjoint's B^T untransposed, Mo[col][r] = B[col][r])
    for (int e = tid; e < np * n * n; e += kTileThreads) {
      const int p = e / (n * n), rc = e - p * n * n, col = rc / n, r = rc - col * n;
      const T* Ap = sA + p * n * 2 * n;
      static_cast<T*>(a.M)[(static_cast<size_t>(b) * a.c + j0 + p) * n * n + rc] =
          a.reverse ? Ap[col * 2 * n + r] : Ap[r * 2 * n + col];
    }
    return;
  }
  for (int p = warp; p < np; p += kTileThreads / 32)
    gj_invert_store<T>(sA + p * n * 2 * n, n, lane,
                       static_cast<T*>(a.M) + (static_cast<size_t>(b) * a.c + j0 + p) * n * n,
                       a.reverse);
}

// ---------------------------------------------------------------------------
// Jacobian blocks on the tensor cores (precision BF16: BF16 operands, FP32
// accumulation in tensor memory), n in {16, 32}.  A tile is 128 rows (p, c):
// TP = 128 / n steps x n Jacobian columns, the M of one tcgen05 MMA.
//   GEMM 1  G^T[(p,c)][r] = sum_q U^T[(p,c)][q] W2[r][q],  U^T[(p,c)][q] = d1[p][q] W1[q][c]
//   scale   G^T[(p,c)][r] *= d2[p][r], rounded to BF16 (operand of GEMM 2)
//   GEMM 2  J^T[(p,c)][r] = sum_s G^T[(p,c)][s] W3[r][s]
//   blocks  A_p[r][c] = delta_rc - dt_p d3[p][r] J^T[(p,c)][r] in FP32, inverted by
//           Gauss-Jordan as in mlp_blocks_kernel.
// Persistent blocks of 128 threads: W2 and W3 (BF16, operand layout) and W1^T
// (FP32) are staged once, then tiles are taken in turn.  Thread 0 issues the
// MMAs and commits them to an mbarrier; the four warps (the four TMEM lane
// quarters) drain the accumulator, warp w reading rows 32 w .. 32 w + 31.  The
// A operands of the two GEMMs and then the FP32 blocks share one region.  Every wait is bounded: a timeout sets *err and ends the block
// after a second bounded wait for its MMAs, with the tensor memory freed.
// ---------------------------------------------------------------------------
constexpr int kTcThreads = 128;
constexpr int kTcRows = 128;          // MMA M
constexpr uint32_t kTcCols = 128;     // TMEM columns: GEMM 1 needs h2 <= 128, GEMM 2 n
constexpr int kTcWaitLimit = 1 << 24; // mbarrier polls before giving up
constexpr size_t kTcMinSmem = 58 * 1024;  // <= 3 blocks per SM: 3 x 128 TMEM columns fit

struct TcLayout {
  uint32_t w2, w3, ug, w1t, dv, dvraw, total;  // byte offsets in dynamic shared memory
};

// The A operands of the two GEMMs share one region (U is dead once GEMM 1 has
// completed), and the FP32 blocks [TP][n][2n] reuse it once GEMM 2 has.
__host__ __device__ inline TcLayout tc_layout(const MlpDims& d) {
  TcLayout L;
  const int tp = kTcRows / d.n;
  const int hmax = d.h1 > d.h2 ? d.h1 : d.h2;
  L.w2 = 0;                                   // [h2][h1] BF16, operand layout
  L.w3 = L.w2 + 2u * d.h2 * d.h1;             // [n][h2] BF16, operand layout
  L.ug = L.w3 + 2u * d.n * d.h2;              // [128][h1] then [128][h2] BF16, operand layout
  L.w1t = L.ug + 2u * kTcRows * hmax;         // [n][h1 + 4] FP32 (rows padded by 16 B)
  L.dv = L.w1t + 4u * d.n * (d.h1 + 4);       // [TP][h1+h2+n] FP32
  L.dvraw = L.dv + 4u * tp * (d.h1 + d.h2 + d.n);  // 2 x [TP][h1+h2+n] FP64, bulk-copied
  L.total = L.dvraw + 2u * 8u * tp * (d.h1 + d.h2 + d.n);
  return L;
}

// the FP32 blocks fit the operand region: 4 * 128 * 2n <= 2 * 128 * max(h1, h2)
bool tc_supported(const MlpDims& d) {
  const int hmax = d.h1 > d.h2 ? d.h1 : d.h2;
  return (d.n == 16 || d.n == 32) && d.h1 % 16 == 0 && d.h2 % 16 == 0 && d.h1 >= 16 &&
         d.h2 >= 16 && d.h1 <= 128 && d.h2 <= 128 && hmax >= 4 * d.n;
}

constexpr float kNeumannMaxNorm = 0.125f;

// The NN x NN diagonal block of a 128 x 128 accumulator for row `32 warp + lane`:
// columns NN p .. NN p + NN - 1 of its step p.  A warp's rows cover columns
// 32 warp .. 32 warp + 31; for NN = 16 the two half-warps take one half each.
template <int NN>
__device__ __forceinline__ void tmem_diag_block(uint32_t tmem_rows, int warp, int lane,
                                                float (&q)[NN]) {
  float lo[16], hi[16];
  tc::tmem_ld16(tmem_rows + 32u * warp, lo);
  tc::tmem_ld16(tmem_rows + 32u * warp + 16u, hi);
  if constexpr (NN == 32) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      q[i] = lo[i];
      q[16 + i] = hi[i];
    }
  } else {
    const bool upper = lane >= 16;
#pragma unroll
    for (int i = 0; i < 16; ++i) q[i] = upper ? hi[i] : lo[i];
  }
}

template <int NN>
__global__ void __launch_bounds__(kTcThreads) mlp_blocks_tc_kernel(BlocksArgs a, int* err) {
  extern __shared__ __align__(128) unsigned char tsm[];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ __align__(8) uint64_t s_dvbar[2];
  __shared__ uint32_t s_tmem;
  __shared__ float s_dt[kTcRows / NN];
  __shared__ int s_stop;
  const MlpDims d = a.d;
  constexpr int n = NN, TP = kTcRows / NN, ln = NN == 16 ? 4 : 5;
  const int h1 = d.h1, h2 = d.h2;
  const int dvs = h1 + h2 + n;
  const TcLayout Lo = tc_layout(d);
  unsigned char* sW2 = tsm + Lo.w2;
  unsigned char* sW3 = tsm + Lo.w3;
  unsigned char* sU = tsm + Lo.ug;
  unsigned char* sG = tsm + Lo.ug;
  float* sW1t = reinterpret_cast<float*>(tsm + Lo.w1t);
  float* sdv = reinterpret_cast<float*>(tsm + Lo.dv);
  float* sA = reinterpret_cast<float*>(tsm + Lo.ug);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int oW2 = h1 * n + h1, oW3 = oW2 + h2 * h1 + h2;

  // ---- once per block: weights into shared memory ----
  for (int e = tid; e < (h2 * h1) >> 1; e += kTcThreads) {
    const int r = (2 * e) / h1, q = 2 * e - r * h1;
    *reinterpret_cast<uint32_t*>(sW2 + tc::kmajor_offset(r, q, h1)) =
        tc::pack_bf16(a.Wf[oW2 + r * h1 + q], a.Wf[oW2 + r * h1 + q + 1]);
  }
  for (int e = tid; e < (n * h2) >> 1; e += kTcThreads) {
    const int r = (2 * e) / h2, q = 2 * e - r * h2;
    *reinterpret_cast<uint32_t*>(sW3 + tc::kmajor_offset(r, q, h2)) =
        tc::pack_bf16(a.Wf[oW3 + r * h2 + q], a.Wf[oW3 + r * h2 + q + 1]);
  }
  const int h1p = h1 + 4;  // padded rows: the 8 rows a quarter-warp reads hit distinct banks
  for (int e = tid; e < n * h1; e += kTcThreads) {
    const int q = e >> ln, c = e & (n - 1);
    sW1t[c * h1p + q] = a.Wf[e];  // W1[q][c]
  }
  if (tid == 0) {
    tc::mbar_init(&s_bar, 1);
    tc::mbar_init(&s_dvbar[0], 1);
    tc::mbar_init(&s_dvbar[1], 1);
    s_stop = 0;
  }
  if (warp == 0) tc::tmem_alloc(&s_tmem, kTcCols);
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;
  const uint32_t tmem_rows = tmem + (static_cast<uint32_t>(warp * 32) << 16);
  const uint32_t aU = tc::smem_u32(sU), aG = tc::smem_u32(sG);
  const uint32_t aW2 = tc::smem_u32(sW2), aW3 = tc::smem_u32(sW3);
  const uint32_t id1 = tc::idesc_bf16(kTcRows, h2), id2 = tc::idesc_bf16(kTcRows, n);
  const uint32_t id3 = tc::idesc_bf16(kTcRows, kTcRows);
  uint32_t phase = 0;
  const int row = tid, p_row = row >> ln, c_row = row & (n - 1);
  const int tiles_per = (a.L + TP - 1) / TP;
  const int total = a.B * tiles_per;

  // The activation derivatives of a tile (np x dvs FP64, contiguous) arrive by a
  // bulk copy issued while the previous tile is processed (two buffers, one
  // mbarrier each); inactive series' tiles are skipped.
  double* dvraw = reinterpret_cast<double*>(tsm + Lo.dvraw);
  auto next_tile = [&](int t) {
    while (t < total && a.active && !a.active[t / tiles_per]) t += gridDim.x;
    return t;
  };
  auto issue_dv = [&](int t, int bf) {  // thread 0
    const int bb = t / tiles_per, jj = (t - bb * tiles_per) * TP;
    const int npp = min(TP, a.L - jj);
    const uint32_t bytes = static_cast<uint32_t>(8 * npp * dvs);
    tc::fence_smem_to_async();  // earlier reads of this buffer precede the refill
    tc::mbar_expect_tx(&s_dvbar[bf], bytes);
    tc::bulk_g2s(dvraw + bf * TP * dvs, a.dv + (static_cast<size_t>(bb) * a.c + jj) * dvs, bytes,
                 &s_dvbar[bf]);
  };
  int buf = 0, nxt = 0;
  uint32_t dvphase = 0;  // bit bf: parity of buffer bf's next completion
  uint32_t outst = 0;    // bit bf: a copy into buffer bf is in flight
  const int first = next_tile(blockIdx.x);
  if (first < total) {
    if (tid == 0) issue_dv(first, 0);
    outst |= 1u;
  }
  for (int tile = first; tile < total; tile = nxt, buf ^= 1) {
    const int b = tile / tiles_per;
    const int j0 = (tile - b * tiles_per) * TP;
    const int np = min(TP, a.L - j0);
    nxt = next_tile(tile + gridDim.x);
    if (nxt < total) {
      if (tid == 0) issue_dv(nxt, buf ^ 1);
      outst |= 1u << (buf ^ 1);
    }
    const int len = a.lengths ? min(max(a.lengths[b], 0), a.N) : a.N;
    const double* tb = a.times + static_cast<size_t>(b) * (a.N + 1);
    if (tid < TP)
      s_dt[tid] = tid < np ? narrow<float>(step_dt(tb, len, step_of(a.reverse, a.i0, a.L, j0 + tid)))
                           : 0.0f;
    if (tc::mbar_wait_bounded(&s_dvbar[buf], (dvphase >> buf) & 1u,
                              tile == first ? a.first_wait_polls : kTcWaitLimit))
      outst &= ~(1u << buf);
    else
      s_stop = 1;
    dvphase ^= 1u << buf;
    __syncthreads();
    if (s_stop) break;
    const double* dvt = dvraw + buf * TP * dvs;
    for (int e = tid; e < TP * dvs; e += kTcThreads)
      sdv[e] = e < np * dvs ? narrow<float>(dvt[e]) : 0.0f;
    __syncthreads();
    // U^T in the operand layout: 8 consecutive threads fill one core matrix
    const int kch = h1 >> 3;
    for (int e = tid; e < kTcRows * kch; e += kTcThreads) {
      const int r8 = e & 7, rest = e >> 3;
      const int kg = rest % kch, rg = rest / kch;
      const int r = rg * 8 + r8, p = r >> ln, c = r & (n - 1);
      const float4* d1 = reinterpret_cast<const float4*>(sdv + p * dvs + kg * 8);
      const float4* w1 = reinterpret_cast<const float4*>(sW1t + c * h1p + kg * 8);
      const float4 da = d1[0], db = d1[1], wa = w1[0], wb = w1[1];
      uint4 v;
      v.x = tc::pack_bf16(da.x * wa.x, da.y * wa.y);
      v.y = tc::pack_bf16(da.z * wa.z, da.w * wa.w);
      v.z = tc::pack_bf16(db.x * wb.x, db.y * wb.y);
      v.w = tc::pack_bf16(db.z * wb.z, db.w * wb.w);
      *reinterpret_cast<uint4*>(sU + tc::kmajor_offset(r, kg * 8, h1)) = v;
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {  // GEMM 1
      tc::fence_after_sync();
      for (int s = 0; s < (h1 >> 4); ++s)
        tc::mma_bf16(tmem, tc::smem_desc(aU + 256u * s, 128u, 16u * h1),
                     tc::smem_desc(aW2 + 256u * s, 128u, 16u * h1), id1, s > 0);
      tc::mma_commit(&s_bar);
    }
    if (!tc::mbar_wait_bounded(&s_bar, phase, kTcWaitLimit)) s_stop = 1;
    phase ^= 1u;
    tc::fence_after_sync();
    __syncthreads();
    if (s_stop) break;
    // scale by d2 and round to BF16: row `row` of G^T (over U, consumed by GEMM 1)
    for (int r0 = 0; r0 < h2; r0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem_rows + r0, v);
      const float* d2 = sdv + p_row * dvs + h1 + r0;
      uint4 lo, hi;
      lo.x = tc::pack_bf16(v[0] * d2[0], v[1] * d2[1]);
      lo.y = tc::pack_bf16(v[2] * d2[2], v[3] * d2[3]);
      lo.z = tc::pack_bf16(v[4] * d2[4], v[5] * d2[5]);
      lo.w = tc::pack_bf16(v[6] * d2[6], v[7] * d2[7]);
      hi.x = tc::pack_bf16(v[8] * d2[8], v[9] * d2[9]);
      hi.y = tc::pack_bf16(v[10] * d2[10], v[11] * d2[11]);
      hi.z = tc::pack_bf16(v[12] * d2[12], v[13] * d2[13]);
      hi.w = tc::pack_bf16(v[14] * d2[14], v[15] * d2[15]);
      *reinterpret_cast<uint4*>(sG + tc::kmajor_offset(row, r0, h2)) = lo;
      *reinterpret_cast<uint4*>(sG + tc::kmajor_offset(row, r0 + 8, h2)) = hi;
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {  // GEMM 2 (overwrites TMEM columns 0 .. n-1, already drained)
      tc::fence_after_sync();
      for (int s = 0; s < (h2 >> 4); ++s)
        tc::mma_bf16(tmem, tc::smem_desc(aG + 256u * s, 128u, 16u * h2),
                     tc::smem_desc(aW3 + 256u * s, 128u, 16u * h2), id2, s > 0);
      tc::mma_commit(&s_bar);
    }
    if (!tc::mbar_wait_bounded(&s_bar, phase, kTcWaitLimit)) s_stop = 1;
    phase ^= 1u;
    tc::fence_after_sync();
    __syncthreads();
    if (s_stop) break;
    // X_p = dt_p D3 J_p; thread (p, c) holds column c of X_p in FP32
    float x[NN];
#pragma unroll
    for (int r0 = 0; r0 < NN; r0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem_rows + r0, v);
      const float dtp = s_dt[p_row];
#pragma unroll
      for (int i = 0; i < 16; ++i)
        x[r0 + i] = p_row < np ? dtp * (sdv[p_row * dvs + h1 + h2 + r0 + i] * v[i]) : 0.0f;
    }
    // ||X_p||_1 (largest column sum) over the NN lanes holding step p
    float cs = 0.0f;
#pragma unroll
    for (int r = 0; r < NN; ++r) cs += fabsf(x[r]);
#pragma unroll
    for (int o = NN / 2; o > 0; o >>= 1) cs = fmaxf(cs, __shfl_xor_sync(kFull, cs, o));
    tc::fence_before_sync();
    if (__syncthreads_or(!(cs <= kNeumannMaxNorm))) {
      // a step with ||X||_1 > 1/8 (or not finite): Gauss-Jordan on A = I - X for the tile
      if (p_row < np) {
        float* Ap = sA + p_row * n * 2 * n;
#pragma unroll
        for (int r = 0; r < NN; ++r) {
          Ap[r * 2 * n + c_row] = (r == c_row ? 1.0f : 0.0f) - x[r];
          Ap[r * 2 * n + n + c_row] = r == c_row ? 1.0f : 0.0f;
        }
      }
      __syncthreads();
      for (int p = warp; p < np; p += kTcThreads / 32)
        gj_invert_store<float>(sA + p * n * 2 * n, n, lane,
                               static_cast<float*>(a.M) + (static_cast<size_t>(b) * a.c + j0 + p) * n * n,
                               a.reverse);
      __syncthreads();
      continue;
    }
    // Neumann series A^-1 = I + X + X^2 + X^3 + O(||X||^4) (<= 2.9e-4 at ||X||_1 <= 1/8),
    // in the transposed form Y = X^T so that every thread keeps its column of X:
    //   P1 = Y Y, P2 = Y^2 (I + Y) on the tensor cores (block-diagonal parts of
    //   128 x 128 products), then column c of M = e_c + X[.][c] + row c of P2.
    unsigned char* sAY = tsm + Lo.ug;         // rows (p, c): Y_p[c][k] = X_p[k][c]
    unsigned char* sBX = sAY + 256 * NN;      // rows (p, j): X_p[j][k]       (B of P1)
    unsigned char* sBIX = sBX + 256 * NN;     // rows (p, j): (I + X_p)[j][k] (B of P2)
    unsigned char* sAY2 = sBIX + 256 * NN;    // rows (p, c): (Y_p^2)[c][k]   (A of P2)
#pragma unroll
    for (int k0 = 0; k0 < NN; k0 += 8) {
      uint4 v;
      v.x = tc::pack_bf16(x[k0], x[k0 + 1]);
      v.y = tc::pack_bf16(x[k0 + 2], x[k0 + 3]);
      v.z = tc::pack_bf16(x[k0 + 4], x[k0 + 5]);
      v.w = tc::pack_bf16(x[k0 + 6], x[k0 + 7]);
      *reinterpret_cast<uint4*>(sAY + tc::kmajor_offset(row, k0, NN)) = v;
    }
#pragma unroll
    for (int j = 0; j < NN; ++j) {
      const int rj = p_row * NN + j;
      const uint32_t two = tc::pack_bf16(x[j], x[j] + (j == c_row ? 1.0f : 0.0f));
      *reinterpret_cast<uint16_t*>(sBX + tc::kmajor_offset(rj, c_row, NN)) =
          static_cast<uint16_t>(two & 0xFFFFu);
      *reinterpret_cast<uint16_t*>(sBIX + tc::kmajor_offset(rj, c_row, NN)) =
          static_cast<uint16_t>(two >> 16);
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {  // P1 = Y Y
      tc::fence_after_sync();
#pragma unroll
      for (int s = 0; s < NN / 16; ++s)
        tc::mma_bf16(tmem, tc::smem_desc(tc::smem_u32(sAY) + 256u * s, 128u, 16u * NN),
                     tc::smem_desc(tc::smem_u32(sBX) + 256u * s, 128u, 16u * NN), id3, s > 0);
      tc::mma_commit(&s_bar);
    }
    if (!tc::mbar_wait_bounded(&s_bar, phase, kTcWaitLimit)) s_stop = 1;
    phase ^= 1u;
    tc::fence_after_sync();
    __syncthreads();
    if (s_stop) break;
    {  // row c of Y^2 -> A operand of P2
      float q[NN];
      tmem_diag_block<NN>(tmem_rows, warp, lane, q);
#pragma unroll
      for (int k0 = 0; k0 < NN; k0 += 8) {
        uint4 v;
        v.x = tc::pack_bf16(q[k0], q[k0 + 1]);
        v.y = tc::pack_bf16(q[k0 + 2], q[k0 + 3]);
        v.z = tc::pack_bf16(q[k0 + 4], q[k0 + 5]);
        v.w = tc::pack_bf16(q[k0 + 6], q[k0 + 7]);
        *reinterpret_cast<uint4*>(sAY2 + tc::kmajor_offset(row, k0, NN)) = v;
      }
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {  // P2 = Y^2 (I + Y)
      tc::fence_after_sync();
#pragma unroll
      for (int s = 0; s < NN / 16; ++s)
        tc::mma_bf16(tmem, tc::smem_desc(tc::smem_u32(sAY2) + 256u * s, 128u, 16u * NN),
                     tc::smem_desc(tc::smem_u32(sBIX) + 256u * s, 128u, 16u * NN), id3, s > 0);
      tc::mma_commit(&s_bar);
    }
    if (!tc::mbar_wait_bounded(&s_bar, phase, kTcWaitLimit)) s_stop = 1;
    phase ^= 1u;
    tc::fence_after_sync();
    __syncthreads();
    if (s_stop) break;
    {  // column c of M: M[j][c] = delta_jc + X[j][c] + (X^2 (I + X))[j][c]
      float q[NN];
      tmem_diag_block<NN>(tmem_rows, warp, lane, q);
      if (p_row < np) {
        float* Mo = static_cast<float*>(a.M) + (static_cast<size_t>(b) * a.c + j0 + p_row) * n * n;
        auto mv = [&](int j) { return (j == c_row ? 1.0f : 0.0f) + x[j] + q[j]; };
        // forward blocks stored transposed (Mo[c][j] = M[j][c]: the thread's own
        // 16-byte aligned row, 16-byte stores); adjoint blocks M^T (lanes coalesced)
        if (a.reverse) {
#pragma unroll
          for (int j = 0; j < NN; ++j) Mo[j * n + c_row] = mv(j);
        } else {
          float4* row4 = reinterpret_cast<float4*>(Mo + c_row * n);
#pragma unroll
          for (int j = 0; j < NN; j += 4) row4[j / 4] = make_float4(mv(j), mv(j + 1), mv(j + 2), mv(j + 3));
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();  // blocks (aliasing U, G) consumed before the next tile writes U
  }
  if (s_stop) {
    if (tid == 0) atomicExch(err, 1);
    tc::mbar_wait_bounded(&s_bar, phase ^ 1u, kTcWaitLimit);  // the MMAs that timed out
    for (int bf = 0; bf < 2; ++bf)  // derivative copies still in flight
      if (outst & (1u << bf)) {
        const uint32_t par = (dvphase >> bf) & 1u;
        // the buffer being waited on when the timeout hit has already flipped its parity
        tc::mbar_wait_bounded(&s_dvbar[bf], bf == buf ? par ^ 1u : par, kTcWaitLimit);
      }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTcCols);
}

// ---------------------------------------------------------------------------
// Block substitution d_j = M_j (d_{j-1} + rhs_j), d_{-1} = x_init (Alg. 2 on the
// normalised blocks): one warp per series, lane r owns component r.  For
// n = 16-32 this is n^2 work per step against the n^3 per step of a cyclic
// reduction, the trade-off the paper reports for larger systems (Sec. 5.3).
// The chain is latency bound (one dependent mat-vec per step), so everything
// that does not depend on d_{j-1} -- the block M_j (stored transposed), rhs_j
// and the accumulator row x_j -- is staged D steps ahead into a per-warp ring
// of shared-memory slots by bulk copies, and d_{j-1} + rhs_j is broadcast
// through shared memory.
// ---------------------------------------------------------------------------
// (ChainArgs is declared in tvi_internal.h: the large-state user models use
// this kernel too.)
constexpr int kChainWarps = 4;
constexpr int kChainOneWarpMaxSeries = 256;
constexpr int kChainWaitLimit = 1 << 22;

// ring slot: the block (N x N in T), the rhs row and the x row (FP64)
template <typename T, int N>
constexpr size_t chain_slot_bytes() {
  return sizeof(T) * N * N + 2 * sizeof(double) * N;
}
// the deepest ring (64 .. 4 steps) whose W warps fit in 200 KB: half a ring's
// copies are in flight while the other half is consumed
template <typename T, int N, int W>
constexpr int chain_depth() {
  return W * 64 * chain_slot_bytes<T, N>() <= 200 * 1024   ? 64
         : W * 32 * chain_slot_bytes<T, N>() <= 200 * 1024 ? 32
         : W * 16 * chain_slot_bytes<T, N>() <= 200 * 1024 ? 16
         : W * 8 * chain_slot_bytes<T, N>() <= 200 * 1024  ? 8
                                                            : 4;
}

// Lane 0 of each warp stages step j's block, rhs row and x row into ring slot
// j % D with bulk copies (the TMA unit) that complete on the mbarrier of the
// slot's half of the ring.  Every source is 16-byte aligned and every size a
// multiple of 16 (N a multiple of 4; workspace buffers by construction, caller
// arrays checked by the C ABI).  The width N is a template parameter so the
// mat-vec unrolls: the block's column loads do not depend on d_{j-1} and are
// issued before it, leaving one shared-memory round trip and N/4 dependent
// FMAs on the step-to-step path.  Lane l owns components l and, for N > 32,
// l + 32 (KC components per lane).
template <typename T, int N, int W>
__global__ void __launch_bounds__(32 * W) mlp_chain_kernel(ChainArgs a) {
  constexpr int KC = (N + 31) / 32;
  constexpr int D = chain_depth<T, N, W>();
  constexpr int H = D / 2;
  constexpr uint32_t mbytes = static_cast<uint32_t>(sizeof(T) * N * N);
  constexpr uint32_t vbytes = static_cast<uint32_t>(sizeof(double) * N);
  constexpr size_t slot_bytes = chain_slot_bytes<T, N>();
  extern __shared__ __align__(16) unsigned char chain_smem[];
  __shared__ T s_u[W][32 * KC];
  __shared__ __align__(8) uint64_t s_bar[W][2];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int b = blockIdx.x * W + wib;
  // warp-uniform exit: the kernel synchronises only within a warp
  if (b >= a.B || (a.active && !a.active[b])) return;
  bool own[KC];
#pragma unroll
  for (int kc = 0; kc < KC; ++kc) own[kc] = lane + 32 * kc < N;
  unsigned char* ring = chain_smem + static_cast<size_t>(wib) * D * slot_bytes;
  uint64_t* bars = s_bar[wib];
  const unsigned char* Mb = static_cast<const unsigned char*>(a.M) +
                            static_cast<size_t>(b) * a.c * mbytes;
  double* xb = a.x + static_cast<size_t>(b) * a.c * N;
  T* su = s_u[wib];
  if (lane == 0)
    for (int k = 0; k < 2; ++k) tc::mbar_init(&bars[k], 1);
  __syncwarp();
  // The ring is two halves of H steps, each with one mbarrier: a half is staged
  // by one fence, one expect_tx and its steps' bulk copies, waited on once, and
  // refilled with the steps D later as soon as its last step is used.
  const uint32_t step_bytes = mbytes + vbytes + (a.mode != 1 ? vbytes : 0u);
  unsigned ph = 0u;    // bit h: parity of half h's next phase
  unsigned pend = 0u;  // bit h: half h staged and not yet waited on
  auto issue_half = [&](int j0) {  // warp-uniform: stage steps j0 .. j0 + H - 1
    const int cnt = min(H, a.L - j0);
    if (cnt <= 0) return;
    const int h = (j0 % D) / H;
    pend |= 1u << h;
    if (lane != 0) return;
    tc::fence_smem_to_async();  // the warp's reads of these slots precede the refill
    tc::mbar_expect_tx(&bars[h], step_bytes * static_cast<uint32_t>(cnt));
    for (int q = 0; q < cnt; ++q) {
      const int j = j0 + q;
      unsigned char* slot = ring + static_cast<size_t>(j % D) * slot_bytes;
      const double* gr =
          a.rhs_buf ? a.rhs_buf + (static_cast<size_t>(b) * a.c + j) * N
                    : a.rhs_traj + (static_cast<size_t>(b) * (a.N + 1) +
                                    step_of(a.reverse, a.i0, a.L, j)) * N;
      tc::bulk_g2s(slot, Mb + static_cast<size_t>(j) * mbytes, mbytes, &bars[h]);
      tc::bulk_g2s(slot + mbytes, gr, vbytes, &bars[h]);
      if (a.mode != 1)
        tc::bulk_g2s(slot + mbytes + vbytes, xb + static_cast<size_t>(j) * N, vbytes, &bars[h]);
    }
  };
  issue_half(0);
  issue_half(H);
  T dprev[KC];
#pragma unroll
  for (int kc = 0; kc < KC; ++kc)
    dprev[kc] = (a.x_init && own[kc]) ? static_cast<T>(a.x_init[b * N + lane + 32 * kc]) : T(0);
#pragma unroll 1
  for (int j = 0; j < a.L; ++j) {
    if (j % H == 0) {
      const int h = (j % D) / H;
      const bool ok =
          __all_sync(kFull, tc::mbar_wait_bounded(&bars[h], (ph >> h) & 1u, kChainWaitLimit));
      if (!ok) {
        if (lane == 0) atomicExch(a.err, 1);
        break;
      }
      ph ^= 1u << h;
      pend &= ~(1u << h);
    }
    const unsigned char* slot = ring + static_cast<size_t>(j % D) * slot_bytes;
    const T* Mt = reinterpret_cast<const T*>(slot);  // Mt[q * N + r] = M_j[r][q]
    const double* rr = reinterpret_cast<const double*>(slot + mbytes);
    // independent of d_{j-1}: rows `lane` (+ 32) of M_j, the rhs and the x entries
    T m[KC][N], rc[KC];
    double x_cur[KC];
#pragma unroll
    for (int kc = 0; kc < KC; ++kc) {
      const int r = lane + 32 * kc;
#pragma unroll
      for (int q = 0; q < N; ++q) m[kc][q] = own[kc] ? Mt[q * N + r] : T(0);
      rc[kc] = own[kc] ? static_cast<T>(rr[r]) : T(0);
      x_cur[kc] = (own[kc] && a.mode != 1) ? rr[N + r] : 0.0;
      // component r of d_{j-1} + rhs_j (of d_{j-1} alone with post_add)
      if (own[kc]) su[r] = a.post_add ? dprev[kc] : dprev[kc] + rc[kc];
    }
    __syncwarp();
    T acc[KC];
#pragma unroll
    for (int kc = 0; kc < KC; ++kc) {
      T acc0 = T(0), acc1 = T(0), acc2 = T(0), acc3 = T(0);
#pragma unroll
      for (int q = 0; q < N; q += 4) {
        acc0 = fma(m[kc][q], su[q], acc0);
        acc1 = fma(m[kc][q + 1], su[q + 1], acc1);
        acc2 = fma(m[kc][q + 2], su[q + 2], acc2);
        acc3 = fma(m[kc][q + 3], su[q + 3], acc3);
      }
      acc[kc] = (acc0 + acc1) + (acc2 + acc3) + (a.post_add ? rc[kc] : T(0));
    }
    __syncwarp();  // su and (at a half's end) its slots are free again
    if (j % H == H - 1) issue_half(j + 1 - H + D);
#pragma unroll
    for (int kc = 0; kc < KC; ++kc) {
      dprev[kc] = own[kc] ? acc[kc] : T(0);
      if (own[kc]) {
        const double dd = static_cast<double>(acc[kc]);
        xb[static_cast<size_t>(j) * N + lane + 32 * kc] =
            (a.mode == 0) ? x_cur[kc] - dd : (a.mode == 1 ? dd : x_cur[kc] + dd);
      }
    }
  }
  // after a timeout: give the halves still in flight a second bounded wait
  // before the block's shared memory goes away
  for (int h = 0; h < 2; ++h)
    if ((pend >> h) & 1u) tc::mbar_wait_bounded(&bars[h], (ph >> h) & 1u, kChainWaitLimit);
}

// ---------------------------------------------------------------------------
// Vector-Jacobian product at the stored trajectory (adjoint), backward pass
// only: the derivative pass stored act'(z1), act'(z2), h'(z3) in dv.  For each
// pair (row j = step k = i0 + L - j) with adjoint a_j:
//   delta3 = a * h'(z3), delta2 = (W3^T delta3) * act'(z2),
//   delta1 = (W2^T delta2) * act'(z1), J^T a = W1^T delta1.
// The products run in T (FP64, or FP32 in the mixed-precision adjoint); the
// residual is assembled in FP64 around them.  Outputs (each optional):
//   res  r_j = g_k + a_{j-1} - a_j + dt_k J^T a_j  (a_{-1} = carry): the
//        residual of the chunk's adjoint system, for refinement
//   del  [pair][h1+h2+n] = dt_k (delta1, delta2, delta3): with the activations
//        the derivative pass stored, the factors of dt_k (dh/dp)^T a_k
// Grid: (ceil(L / TP), B).
// ---------------------------------------------------------------------------
struct VjpArgs {
  MlpDims d;
  int B, N, i0, L, c;
  const double* times;
  const int* lengths;
  const double* params;    // FP64 weights (T = double)
  const float* Wf;         // FP32 weights (T = float)
  const double* g;         // [B][N+1][n]
  const double* carry;     // [B][n]
  const double* av;        // [B][c][n] adjoint by row
  const double* dv;        // [B][c][h1+h2+n] activation derivatives
  double* res;             // [B][c][n] or null
  double* del;             // [B*c][h1+h2+n] or null
  int fe;                  // forward Euler: the products take a_{k+1} (row j-1, or the
                           // carry) and dt_{k+1}: r_j = g_k + a_{j-1} - a_j + dt_{k+1} J^T
                           // a_{j-1}, del = dt_{k+1} (delta's of a_{j-1}) at y_k
  const int* active;       // [B] or null: series whose chunk is skipped write nothing
};

template <int KIND, int TP, typename T>
__global__ void __launch_bounds__(kTileThreads) mlp_vjp_kernel(VjpArgs a) {
  extern __shared__ double smem[];
  const MlpDims d = a.d;
  const int n = d.n, h1 = d.h1, h2 = d.h2;
  const int b = blockIdx.y;
  if (a.active && !a.active[b]) return;  // block-uniform
  const int j0 = blockIdx.x * TP;
  const int np = min(TP, a.L - j0);
  T* sd1 = reinterpret_cast<T*>(smem);  // [h1][TP] act'(z1), then delta1
  T* sd2 = sd1 + h1 * TP;               // [h2][TP] act'(z2), then delta2
  T* sz3 = sd2 + h2 * TP;               // [n][TP]  h'(z3), then delta3
  MlpW<T> w;
  if constexpr (sizeof(T) == sizeof(double)) w = mlp_split(a.params, d);
  else w = mlp_split(a.Wf, d);
  const double* tb = a.times + static_cast<size_t>(b) * (a.N + 1);
  const int len = a.lengths ? min(max(a.lengths[b], 0), a.N) : a.N;
  constexpr int G = kTileThreads / TP;
  const int t = threadIdx.x, p = t % TP, g = t / TP;
  const bool live = p < np;
  const int j = j0 + p;
  const double* avb = a.av + static_cast<size_t>(b) * a.c * n;
  const int dvs = h1 + h2 + n;
  const double* dvt = a.dv + (static_cast<size_t>(b) * a.c + j0) * dvs;
  for (int e = threadIdx.x; e < dvs * TP; e += kTileThreads) {
    const int pp = e / dvs, q = e - pp * dvs;  // consecutive threads read one row
    const T v = pp < np ? narrow<T>(dvt[pp * dvs + q]) : T(0);
    if (q < h1) sd1[q * TP + pp] = v;
    else if (q < h1 + h2) sd2[(q - h1) * TP + pp] = v;
    else sz3[(q - h1 - h2) * TP + pp] = v;
  }
  __syncthreads();
  // delta3 = a * h'(z3): a_j, or a_{j-1} (the carry for row 0) for forward Euler
  for (int r = g; r < n; r += G) {
    double av = 0.0;
    if (live) av = !a.fe ? avb[j * n + r] : (j > 0 ? avb[(j - 1) * n + r] : a.carry[b * n + r]);
    sz3[r * TP + p] = live ? narrow<T>(av) * sz3[r * TP + p] : T(0);
  }
  const int kshift = a.fe ? 1 : 0;  // forward Euler: dt_{k+1}
  __syncthreads();
  if constexpr (sizeof(T) == sizeof(float)) {
    // register-tiled products; then outputs with one thread per element
    tile_mm_f32<TP, true>(w.W3, 1, h2, h2, n, sz3, [&](int c, int pp, float v) { sd2[c * TP + pp] *= v; });
    __syncthreads();
    tile_mm_f32<TP, true>(w.W2, 1, h1, h1, h2, sd2, [&](int c, int pp, float v) { sd1[c * TP + pp] *= v; });
    __syncthreads();
    if (a.res) {
      float* sjt = sz3 + n * TP;  // J^T a, [n][TP]
      tile_mm_f32<TP, true>(w.W1, 1, n, n, h1, sd1, [&](int c, int pp, float v) { sjt[c * TP + pp] = v; });
      __syncthreads();
      for (int e = threadIdx.x; e < n * TP; e += kTileThreads) {
        const int c = e / TP, pp = e - c * TP;
        if (pp >= np) continue;
        const int jj = j0 + pp, kk = step_of(1, a.i0, a.L, jj);
        const double prev = (jj > 0) ? avb[(jj - 1) * n + c] : a.carry[b * n + c];
        const double gk = a.g[(static_cast<size_t>(b) * (a.N + 1) + kk) * n + c];
        a.res[(static_cast<size_t>(b) * a.c + jj) * n + c] =
            fma(step_dt(tb, len, kk + kshift), widen(sjt[c * TP + pp]),
                gk + prev - avb[jj * n + c]);
      }
    }
    if (a.del) {
      const int dw = h1 + h2 + n;
      for (int e = threadIdx.x; e < dw * TP; e += kTileThreads) {
        const int pp = e / dw, q = e - pp * dw;  // consecutive threads fill one row
        if (pp >= np) continue;
        const int jj = j0 + pp;
        const float v = q < h1 ? sd1[q * TP + pp]
                               : (q < h1 + h2 ? sd2[(q - h1) * TP + pp] : sz3[(q - h1 - h2) * TP + pp]);
        a.del[(static_cast<size_t>(b) * a.c + jj) * dw + q] =
            step_dt(tb, len, step_of(1, a.i0, a.L, jj) + kshift) * widen(v);
      }
    }
  } else {  // FP64: one output element a thread
    // delta2 = (W3^T delta3) * act'(z2)
    for (int c = g; c < h2; c += G) {
      T acc = T(0);
      for (int r = 0; r < n; ++r) acc = fma(__ldg(w.W3 + r * h2 + c), sz3[r * TP + p], acc);
      sd2[c * TP + p] *= acc;
    }
    __syncthreads();
    // delta1 = (W2^T delta2) * act'(z1)
    for (int c = g; c < h1; c += G) {
      T acc = T(0);
      for (int r = 0; r < h2; ++r) acc = fma(__ldg(w.W2 + r * h1 + c), sd2[r * TP + p], acc);
      sd1[c * TP + p] *= acc;
    }
    __syncthreads();
    if (!live) return;
    const int k = step_of(1, a.i0, a.L, j);
    const double dt = step_dt(tb, len, k + kshift);
    if (a.res) {
      // r_j = g_k + a_{j-1} - a_j + dt (W1^T delta1), assembled in FP64
      for (int c = g; c < n; c += G) {
        T acc = T(0);
        for (int r = 0; r < h1; ++r) acc = fma(__ldg(w.W1 + r * n + c), sd1[r * TP + p], acc);
        const double prev = (j > 0) ? avb[(j - 1) * n + c] : a.carry[b * n + c];
        const double gk = a.g[(static_cast<size_t>(b) * (a.N + 1) + k) * n + c];
        a.res[(static_cast<size_t>(b) * a.c + j) * n + c] =
            fma(dt, widen(acc), gk + prev - avb[j * n + c]);
      }
    }
    if (a.del) {
      const int dw = h1 + h2 + n;
      double* dr = a.del + (static_cast<size_t>(b) * a.c + j) * dw;
      for (int c = g; c < h1; c += G) dr[c] = dt * widen(sd1[c * TP + p]);
      for (int c = g; c < h2; c += G) dr[h1 + c] = dt * widen(sd2[c * TP + p]);
      for (int c = g; c < n; c += G) dr[h1 + h2 + c] = dt * widen(sz3[c * TP + p]);
    }
  }
}

// ---------------------------------------------------------------------------
// Parameter gradient of one chunk: for each layer l, the [rows][cols + 1] block
// (weights and bias) += sum over the chunk's pairs of del_l[pair][row] *
// act_l[pair][col] (act's extra column is 1 for the bias).  Each thread block
// owns a 32 x 32 output tile (no atomics: a fixed summation order), stages 64
// pairs at a time in shared memory, forms products in T and adds every
// 64-pair partial sum into an FP64 accumulator.
// ---------------------------------------------------------------------------
struct ParamArgs {
  MlpDims d;
  int B, L, c;
  const double* act;  // [B*c][n+h1+h2+3]
  const double* del;  // [B*c][h1+h2+n]
  double* part;       // [nsplit][P] partial sums, one per range of pairs (grid.y)
  int per;            // pairs per range (multiple of 64)
  const int* active;  // [B] or null: pairs of series whose chunk is skipped add nothing
};

template <typename T>
__global__ void __launch_bounds__(256) mlp_param_grad_kernel(ParamArgs a) {
  __shared__ T sX[64][33];
  __shared__ T sY[64][33];
  const MlpDims d = a.d;
  const int n = d.n, h1 = d.h1, h2 = d.h2;
  const int aw = n + h1 + h2 + 3, dw = h1 + h2 + n;
  // layer geometry: rows, cols (incl. bias), del offset, act offset, W offset, bias offset
  int rows[3] = {h1, h2, n}, cols[3] = {n + 1, h1 + 1, h2 + 1};
  int doff[3] = {0, h1, h1 + h2}, aoff[3] = {0, n + 1, n + 1 + h1 + 1};
  int woff[3] = {0, h1 * n + h1, h1 * n + h1 + h2 * h1 + h2};
  int tiles[3];
  for (int l = 0; l < 3; ++l) tiles[l] = ((rows[l] + 31) / 32) * ((cols[l] + 31) / 32);
  int tile = blockIdx.x, l = 0;
  while (l < 2 && tile >= tiles[l]) tile -= tiles[l++];
  const int tcols = (cols[l] + 31) / 32;
  const int r0 = (tile / tcols) * 32, c0 = (tile % tcols) * 32;
  const int tid = threadIdx.x;
  const int tr = tid / 8, tc = (tid % 8) * 4;  // 32 rows x (8 x 4) cols
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int pbeg = blockIdx.y * a.per;
  const int npairs = min(a.B * a.L, pbeg + a.per);
  for (int p0 = pbeg; p0 < npairs; p0 += 64) {
    for (int e = tid; e < 64 * 32; e += 256) {
      const int pp = e / 32, q = e % 32;
      const int pi = p0 + pp;
      T xv = T(0), yv = T(0);
      if (pi < npairs && (!a.active || a.active[pi / a.L])) {
        const size_t row = static_cast<size_t>(pi / a.L) * a.c + (pi % a.L);
        if (r0 + q < rows[l]) xv = static_cast<T>(a.del[row * dw + doff[l] + r0 + q]);
        if (c0 + q < cols[l]) yv = static_cast<T>(a.act[row * aw + aoff[l] + c0 + q]);
      }
      sX[pp][q] = xv;
      sY[pp][q] = yv;
    }
    __syncthreads();
    T part[4] = {T(0), T(0), T(0), T(0)};
    for (int pp = 0; pp < 64; ++pp) {
      const T xv = sX[pp][tr];
#pragma unroll
      for (int i = 0; i < 4; ++i) part[i] = fma(xv, sY[pp][tc + i], part[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] += static_cast<double>(part[i]);
    __syncthreads();
  }
  const int r = r0 + tr;
  if (r >= rows[l]) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int c = c0 + tc + i;
    if (c >= cols[l]) continue;
    const int idx = (c < cols[l] - 1) ? woff[l] + r * (cols[l] - 1) + c
                                      : woff[l] + rows[l] * (cols[l] - 1) + r;
    a.part[static_cast<size_t>(blockIdx.y) * d.P + idx] = acc[i];
  }
}

// acc[q] += sum over ranges s = 0..nsplit-1 of part[s][q], in range order
__global__ void mlp_param_reduce_kernel(int P, int nsplit, const double* part, double* acc) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P) return;
  double s = 0.0;
  for (int k = 0; k < nsplit; ++k) s += part[static_cast<size_t>(k) * P + q];
  acc[q] += s;
}

constexpr int kMaxParamSplits = 64;

int param_grad_tiles(const MlpDims& d) {
  auto t = [](int r, int c) { return ((r + 31) / 32) * ((c + 31) / 32); };
  return t(d.h1, d.n + 1) + t(d.h2, d.h1 + 1) + t(d.n, d.h2 + 1);
}

// ---------------------------------------------------------------------------
// Small bookkeeping kernels.
// ---------------------------------------------------------------------------
__global__ void mlp_start_kernel(int B, int n, int Np1, const double* y0, double* y_out,
                                 double* yi, int* status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B * n) {
    const int b = i / n, s = i % n;
    y_out[static_cast<size_t>(b) * Np1 * n + s] = y0[i];
    yi[i] = y0[i];
  }
  if (i < B) status[i] = 0;
}

// Start of a chunk attempt for the series in `mask` (every series when null):
// dy = 0 (the Sec. 2.3 guess), the series active, its status remembered so that
// a failure of this attempt can be told apart from an earlier one.
__global__ void chunk_begin_kernel(int B, int rowlen, int c, const int* mask, double* dy,
                                   int* active, unsigned long long* norm, int* iters,
                                   const int* status, int* status0) {
  const size_t i = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < static_cast<size_t>(B) * c * rowlen) dy[i] = 0.0;
  if (i < static_cast<size_t>(B)) {
    active[i] = mask ? mask[i] : 1;
    norm[i] = 0ull;
    iters[i] = 0;
    status0[i] = status[i];
  }
}

// After an attempt that may be halved: the series of `mask` whose attempt failed
// (status set by it) go into `fail`, get their earlier status back (the halves
// re-solve the same steps) and count one retry; *nfail counts them.
__global__ void chunk_fail_kernel(int B, const int* mask, int* status, const int* status0,
                                  int* fail, int* nfail, int* stats) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const bool failed = (!mask || mask[b]) && status[b] != status0[b];
  fail[b] = failed ? 1 : 0;
  if (failed) {
    status[b] = status0[b];
    atomicAdd(nfail, 1);
    if (stats) stats[b * kStats + 2] += 1;
  }
}

// Write y_{i0+1..i0+L} = y_i + dy and carry y_{i0+L}; one block per series.
// Padded steps (k > length) keep the last real state exactly (reading C-14),
// whatever rounding Newton left in their identity rows.
__global__ void mlp_store_kernel(int n, int L, int c, int N, int i0, const int* lengths,
                                 const double* dy, double* yi, double* y_out, const int* iters,
                                 int* stats, const int* mask, const int* fail) {
  const int b = blockIdx.x;
  // only the attempt's series (mask), and not those re-solving it by halves
  if ((mask && !mask[b]) || (fail && fail[b])) return;
  const int len = lengths ? min(max(lengths[b], 0), N) : N;
  const int jl = min(L, max(len - i0, 0)) - 1;  // last real row of the chunk, -1 if none
  const double* dyb = dy + static_cast<size_t>(b) * c * n;
  double* yb = y_out + static_cast<size_t>(b) * (N + 1) * n;
  for (int e = threadIdx.x; e < L * n; e += blockDim.x) {
    const int j = e / n, s = e % n;
    const int jr = min(j, jl);
    yb[static_cast<size_t>(i0 + 1 + j) * n + s] =
        yi[b * n + s] + (jr >= 0 ? dyb[jr * n + s] : 0.0);
  }
  __syncthreads();
  if (threadIdx.x < n && jl >= 0) yi[b * n + threadIdx.x] += dyb[jl * n + threadIdx.x];
  if (threadIdx.x == 0 && stats) {
    int* o = stats + b * kStats;
    o[0] += iters[b];
    o[1] += 1;
    o[3] = max(o[3], iters[b]);
  }
}

// status 3 for every series when a tensor-core wait gave up (results invalid)
__global__ void mlp_worst_kernel(int B, const int* status, const int* tcerr, int* series_status,
                                 int* worst) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int st = *tcerr ? 3 : status[b];
  if (series_status) series_status[b] = st;
  if (st) atomicMax(worst, st);
}

// carry a_{i0+1} (row L-1) to the next (earlier) chunk
__global__ void mlp_carry_kernel(int B, int n, int L, int c, const double* av, double* carry,
                                 const int* active) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B * n && (!active || active[i / n]))
    carry[i] = av[(static_cast<size_t>(i / n) * c + (L - 1)) * n + (i % n)];
}

// Adjoint chunk of steps i0 + 1 .. i0 + L: a series takes part unless every step
// lies past its length (dt = 0: identity blocks, no parameter terms) and dL/dy is
// zero on all of them -- then a_k = a_{k+1} on every row and its carry passes
// through unchanged, so skipping the chunk changes no result.  Grid: B.
__global__ void mlp_adj_active_kernel(int n, int Np1, int i0, int L, const int* lengths,
                                      const double* g, int* active) {
  const int b = blockIdx.x;
  const int len = min(max(lengths[b], 0), Np1 - 1);
  bool any = i0 + 1 <= len;
  if (!any) {  // n is a multiple of 4: rows are 16-byte aligned, read two values a load
    const double2* gb = reinterpret_cast<const double2*>(g + (static_cast<size_t>(b) * Np1 + i0 + 1) * n);
    const int m = L * n / 2;
#pragma unroll 4
    for (int e = threadIdx.x; e < m; e += blockDim.x) {
      const double2 v = gb[e];
      if (v.x != 0.0 || v.y != 0.0) any = true;  // NaN counts as nonzero
    }
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) active[b] = any ? 1 : 0;
}

// gradients are NaN when a tensor-core wait gave up (results invalid)
// dL/dy0 = a_1 + dL/dy_0 (backward Euler), or row 0 of `row0` [B][c][n] (forward
// Euler: the y_0 pass's residual)
__global__ void mlp_adjoint_end_kernel(int B, int n, int Np1, int c, const double* carry,
                                       const double* g, const double* row0, double* dy0,
                                       const double* acc, double* dparams, int P,
                                       const int* tcerr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool bad = *tcerr != 0;
  if (dy0 && i < B * n)
    dy0[i] = bad ? __longlong_as_double(0x7ff8000000000000LL)
           : row0 ? row0[static_cast<size_t>(i / n) * c * n + (i % n)]
                  : carry[i] + g[static_cast<size_t>(i / n) * Np1 * n + (i % n)];
  if (i < P) dparams[i] = bad ? __longlong_as_double(0x7ff8000000000000LL) : acc[i];
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
size_t al(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct Ws {
  float* Wf;
  double *yi, *dy, *R, *carry, *acc, *part, *act, *del, *norm0;
  double* dv;
  void* M;
  unsigned long long* norm;
  int *active, *status, *iters, *remaining, *worst, *tcerr;
  int *status0, *nfail, *fail;  // chunk halving: status before an attempt, failures, masks
  size_t total;
};

Ws carve(char* base, int B, int c, const MlpDims& d, int precision, bool adjoint_bufs) {
  Ws w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += al(bytes);
    return p;
  };
  const size_t bc = static_cast<size_t>(B) * c;
  const size_t tsz = precision == kPrecFp64 ? sizeof(double) : sizeof(float);
  w.worst = reinterpret_cast<int*>(take(sizeof(int)));
  w.remaining = reinterpret_cast<int*>(take(sizeof(int)));
  w.tcerr = reinterpret_cast<int*>(take(sizeof(int)));
  w.Wf = reinterpret_cast<float*>(take(sizeof(float) * d.P));
  w.yi = reinterpret_cast<double*>(take(sizeof(double) * B * d.n));
  w.carry = reinterpret_cast<double*>(take(sizeof(double) * B * d.n));
  w.norm = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * B));
  w.norm0 = reinterpret_cast<double*>(take(sizeof(double) * B));
  w.active = reinterpret_cast<int*>(take(sizeof(int) * B));
  w.status = reinterpret_cast<int*>(take(sizeof(int) * B));
  w.iters = reinterpret_cast<int*>(take(sizeof(int) * B));
  w.status0 = reinterpret_cast<int*>(take(sizeof(int) * B));
  w.nfail = reinterpret_cast<int*>(take(sizeof(int)));
  w.fail = reinterpret_cast<int*>(take(sizeof(int) * B * kHalvingDepth));
  w.dy = reinterpret_cast<double*>(take(sizeof(double) * bc * d.n));
  w.R = reinterpret_cast<double*>(take(sizeof(double) * bc * d.n));
  w.dv = reinterpret_cast<double*>(take(sizeof(double) * bc * (d.h1 + d.h2 + d.n)));
  w.M = take(tsz * bc * d.n * d.n);
  if (adjoint_bufs) {
    w.acc = reinterpret_cast<double*>(take(sizeof(double) * d.P));
    w.part = reinterpret_cast<double*>(take(sizeof(double) * d.P * kMaxParamSplits));
    w.act = reinterpret_cast<double*>(take(sizeof(double) * bc * (d.n + d.h1 + d.h2 + 3)));
    w.del = reinterpret_cast<double*>(take(sizeof(double) * bc * (d.h1 + d.h2 + d.n)));
  }
  w.total = off;
  return w;
}

MlpDims dims_of(int n, int h1, int h2) {
  MlpDims d;
  d.n = n;
  d.h1 = h1;
  d.h2 = h2;
  d.P = h1 * n + h1 + h2 * h1 + h2 + n * h2 + n;
  return d;
}

constexpr size_t kMaxDynSmem = 227 * 1024;  // per-block shared memory limit
// pairs per residual tile: 64 for the FP32 derivative pass of the adjoint; 32
// for the FP64 passes, whose time is the FP64 pipe's, so that smaller tiles
// spread a chunk's pairs evenly over the SMs (n = 16, 64 x 200 pairs: 448 tiles
// instead of 256 on 152 SMs) with half the shared memory per block
template <typename T>
constexpr int res_tp() {
  return sizeof(T) == sizeof(double) ? 32 : 64;
}
constexpr int kVjpTP = 32;  // pairs per vector-Jacobian tile

size_t residual_smem(const MlpDims& d, int tp) {
  return sizeof(double) * (2 * d.n + d.h1 + d.h2) * tp;
}
size_t vjp_smem(const MlpDims& d) {
  return sizeof(double) * (d.n + d.h1 + d.h2) * kVjpTP;
}

// pairs per Jacobian tile: about 32k bytes of U per block, at least 1
int blocks_tp(const MlpDims& d, int precision) {
  const int tsz = precision == kPrecFp64 ? 8 : 4;
  const int hmax = d.h1 > d.h2 ? d.h1 : d.h2;
  int nt = 32768 / (hmax * tsz);
  int tp = nt / d.n;
  tp = tp < 1 ? 1 : (tp > 64 ? 64 : tp);
  while (tp & (tp - 1)) tp &= tp - 1;  // power of two: tile columns TP * n index by shifts
  return tp;
}
size_t blocks_smem(const MlpDims& d, int precision, int tp) {
  const size_t tsz = precision == kPrecFp64 ? 8 : 4;
  return tsz * (static_cast<size_t>(d.h1 + d.h2) * tp * d.n + static_cast<size_t>(tp) * d.n * 2 * d.n + tp);
}

template <typename K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(bytes));
}

template <int KIND, typename T>
cudaError_t launch_residual_t(const ResidualArgs& r, cudaStream_t s) {
  constexpr int TP = res_tp<T>();
  const size_t sm = residual_smem(r.d, TP);
  cudaError_t e = set_smem(mlp_residual_kernel<KIND, TP, T>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((r.L + TP - 1) / TP, r.B);
  note_launch();
  mlp_residual_kernel<KIND, TP, T><<<grid, kTileThreads, sm, s>>>(r);
  return cudaGetLastError();
}

// first residual of a chunk attempt: the network once per series
cudaError_t launch_residual_start(int kind, const ResidualArgs& r, cudaStream_t s) {
  note_launch();
  if (kind == kKindMlpTanh)
    mlp_residual_start_kernel<kKindMlpTanh><<<r.B, kTileThreads, 0, s>>>(r);
  else
    mlp_residual_start_kernel<kKindMlpSilu><<<r.B, kTileThreads, 0, s>>>(r);
  return cudaGetLastError();
}

// FP64 always for the Newton residual; the adjoint's derivative pass in FP32
// when the blocks are FP32 / BF16
cudaError_t launch_residual(int kind, bool fp32, const ResidualArgs& r, cudaStream_t s) {
  if (kind == kKindMlpTanh)
    return fp32 ? launch_residual_t<kKindMlpTanh, float>(r, s)
                : launch_residual_t<kKindMlpTanh, double>(r, s);
  return fp32 ? launch_residual_t<kKindMlpSilu, float>(r, s)
              : launch_residual_t<kKindMlpSilu, double>(r, s);
}

template <int KIND, typename T>
cudaError_t launch_vjp_t(const VjpArgs& v, cudaStream_t s) {
  const size_t sm = vjp_smem(v.d);
  cudaError_t e = set_smem(mlp_vjp_kernel<KIND, kVjpTP, T>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((v.L + kVjpTP - 1) / kVjpTP, v.B);
  note_launch();
  mlp_vjp_kernel<KIND, kVjpTP, T><<<grid, kTileThreads, sm, s>>>(v);
  return cudaGetLastError();
}

cudaError_t launch_vjp(int kind, bool fp32, const VjpArgs& v, cudaStream_t s) {
  if (kind == kKindMlpTanh)
    return fp32 ? launch_vjp_t<kKindMlpTanh, float>(v, s) : launch_vjp_t<kKindMlpTanh, double>(v, s);
  return fp32 ? launch_vjp_t<kKindMlpSilu, float>(v, s) : launch_vjp_t<kKindMlpSilu, double>(v, s);
}

template <typename T>
cudaError_t launch_blocks(const BlocksArgs& bk, int precision, cudaStream_t s) {
  const int tp = blocks_tp(bk.d, precision);
  size_t sm = blocks_smem(bk.d, precision, tp);
  // W2 goes to shared memory only when that keeps two blocks per SM (measured:
  // losing the second block costs more than the cached loads it saves)
  const size_t w2 = sizeof(T) * bk.d.h1 * bk.d.h2;
  const int stage = 2 * (sm + w2) <= kMaxDynSmem ? 1 : 0;
  if (stage) sm += w2;
  cudaError_t e = set_smem(mlp_blocks_kernel<T>, sm);
  if (e != cudaSuccess) return e;
  dim3 grid((bk.L + tp - 1) / tp, bk.B);
  note_launch();
  mlp_blocks_kernel<T><<<grid, kTileThreads, sm, s>>>(bk, tp, stage);
  return cudaGetLastError();
}

// Poll limit of the first derivative-copy wait of each tensor-core block: the
// full limit, unless the environment variable TVI_TEST_TC_FIRST_WAIT_POLLS sets
// another (a test hook: 0 makes that wait give up at once, so the timeout path --
// error flag, drain of the copies in flight, tensor memory freed -- runs without
// any fault).
int tc_first_wait_polls() {
  const char* v = std::getenv("TVI_TEST_TC_FIRST_WAIT_POLLS");
  if (!v || !*v) return kTcWaitLimit;
  char* end = nullptr;
  const long x = std::strtol(v, &end, 10);
  if (end == v || x < 0 || x > kTcWaitLimit) return kTcWaitLimit;
  return static_cast<int>(x);
}

cudaError_t launch_blocks_tc(const BlocksArgs& bk_in, int* err, cudaStream_t s) {
  BlocksArgs bk = bk_in;
  bk.first_wait_polls = tc_first_wait_polls();
  const TcLayout Lo = tc_layout(bk.d);
  const size_t sm = Lo.total < kTcMinSmem ? kTcMinSmem : Lo.total;
  cudaError_t e = bk.d.n == 16 ? set_smem(mlp_blocks_tc_kernel<16>, sm)
                                : set_smem(mlp_blocks_tc_kernel<32>, sm);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int tp = kTcRows / bk.d.n;
  const int tiles = bk.B * ((bk.L + tp - 1) / tp);
  const int per_sm = static_cast<int>(kMaxDynSmem / sm) >= 2 ? 2 : 1;
  const int grid = tiles < per_sm * sms ? tiles : per_sm * sms;
  if (grid < 1) return cudaSuccess;
  if (bk.d.n == 16) {
    note_launch();
    mlp_blocks_tc_kernel<16><<<grid, kTcThreads, sm, s>>>(bk, err);
  } else {
    note_launch();
    mlp_blocks_tc_kernel<32><<<grid, kTcThreads, sm, s>>>(bk, err);
  }
  return cudaGetLastError();
}

// Jacobian blocks in the precision's arithmetic: FP64 / FP32 on the FMA pipes,
// BF16 products on the tensor cores (blocks and chain then in FP32)
cudaError_t launch_blocks_any(const BlocksArgs& bk, int precision, int* err, cudaStream_t s) {
  if (precision == kPrecFp64) return launch_blocks<double>(bk, precision, s);
  if (precision == kPrecBf16) return launch_blocks_tc(bk, err, s);
  return launch_blocks<float>(bk, precision, s);
}

// ---------------------------------------------------------------------------
// Tiled chain solve (the hybrid of Sec. 3.3): the chunk's L steps are split
// into W tiles, one warp each.
//   pass A (tiles in parallel)  warp w composes its tile's affine map
//                               d_end = P_w d_in + q_w  (P <- M_j P, q <- M_j (q + r_j);
//                               q <- M_j q + r_j for forward Euler's recurrence)
//   pass B (one warp)           d_in of every tile from x_init by the W maps
//   pass C (tiles in parallel)  warp w sweeps its tile from its d_in:
//                               d_j = M_j (d_{j-1} + r_j), x updated by mode
// Sequential depth per series: L / W + W steps instead of L, for n^3 / 32
// FMAs a lane per step in pass A.  Blocks and rhs rows are read from global
// memory (pass C reads them a second time, mostly from L2).  Shared memory per
// warp: P (two buffers), the staged block M_j (rows padded to N + 1), q, d_in.
// ---------------------------------------------------------------------------
// four consecutive T (16-byte aligned) in shared memory
__device__ __forceinline__ void ld4(const float* p, float (&u)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  u[0] = v.x; u[1] = v.y; u[2] = v.z; u[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&u)[4]) {
  const double2 v0 = reinterpret_cast<const double2*>(p)[0];
  const double2 v1 = reinterpret_cast<const double2*>(p)[1];
  u[0] = v0.x; u[1] = v0.y; u[2] = v1.x; u[3] = v1.y;
}
__device__ __forceinline__ void st4(float* p, const float (&u)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(u[0], u[1], u[2], u[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&u)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(u[0], u[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(u[2], u[3]);
}

// rows of P <- M_j P a lane forms in pass A: the fewest (dividing N) that fit
// the N x N outputs into 32 lanes of RT x 4 tiles (1 at N <= 8, 2 at 12-16, 4 at
// 20, 6 at 24)
constexpr int tile_rows_per_lane(int N) {
  int rt = 1;
  while (N % rt != 0 || (N / rt) * (N / 4) > 32) ++rt;
  return rt;
}

template <typename T, int N>
constexpr size_t tile_warp_bytes() {
  return sizeof(T) * (2 * N * N + N * (N + 1) + 2 * N + 32);
}

template <typename T, int N, int W>
__global__ void __launch_bounds__(32 * W) tile_chain_kernel(ChainArgs a) {
  constexpr int LDM = N + 1;
  extern __shared__ __align__(16) unsigned char tile_smem[];
  const int b = blockIdx.x;
  if (a.active && !a.active[b]) return;  // block-uniform
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* wbase = reinterpret_cast<T*>(tile_smem + static_cast<size_t>(warp) * tile_warp_bytes<T, N>());
  T* P0 = wbase;
  T* P1 = P0 + N * N;
  T* sM = P1 + N * N;    // [N][LDM]
  T* sq = sM + N * LDM;  // [N]
  T* sd = sq + N;        // [N] d_in of the tile
  T* su = sd + N;        // [32] q + r_j
  const int Lt = (a.L + W - 1) / W;
  const int j0 = min(a.L, warp * Lt), j1 = min(a.L, j0 + Lt);
  const T* Mb = static_cast<const T*>(a.M) + static_cast<size_t>(b) * a.c * N * N;
  double* xb = a.x + static_cast<size_t>(b) * a.c * N;
  auto rhs_row = [&](int j) -> const double* {
    return a.rhs_buf ? a.rhs_buf + (static_cast<size_t>(b) * a.c + j) * N
                     : a.rhs_traj + (static_cast<size_t>(b) * (a.N + 1) +
                                     step_of(a.reverse, a.i0, a.L, j)) * N;
  };
  // Each pass reads a step's block and rhs row PF steps ahead into registers
  // (a ring indexed at compile time), so the loads' latency overlaps the
  // dependent arithmetic of the steps in between.
  constexpr int PF = N * sizeof(T) <= 32 ? 4 : 2;  // the deeper ring only where it fits
  constexpr int E = (N * N + 31) / 32;  // block entries a lane stages in pass A
  constexpr int RT = tile_rows_per_lane(N);  // pass A register tile: RT rows x 4 columns
  constexpr int NCQ = N / 4;
  constexpr int kLanesA = (N / RT) * NCQ;    // <= 32
  static_assert(N % 4 == 0 && N % RT == 0 && kLanesA <= 32, "tile chain widths: multiples of 4 up to 24");
  // ---- pass A: (P, q) = composite of the tile's maps, starting from (I, 0) ----
  for (int e = lane; e < N * N; e += 32) P0[e] = (e / N == e % N) ? T(1) : T(0);
  if (lane < N) sq[lane] = T(0);
  __syncwarp();
  T* Pc = P0;
  T* Pn = P1;
  {
    T mreg[PF][E];
    double rreg[PF];
    auto load_a = [&](int j, T (&mr)[E], double& rv) {
      if (j < j1) {
        const T* Mt = Mb + static_cast<size_t>(j) * N * N;
#pragma unroll
        for (int i = 0; i < E; ++i) {
          const int e = lane + 32 * i;
          mr[i] = e < N * N ? Mt[e] : T(0);
        }
        rv = lane < N ? rhs_row(j)[lane] : 0.0;
      }
    };
#pragma unroll
    for (int q = 0; q < PF; ++q) load_a(j0 + q, mreg[q], rreg[q]);
#pragma unroll 1
    for (int jb = j0; jb < j1; jb += PF) {
#pragma unroll
      for (int q = 0; q < PF; ++q) {
        const int j = jb + q;
        if (j < j1) {  // warp-uniform
          // stage M_j row-major (sM[r][k] = M_j[r][k] = Mt[k * N + r]) and u = q + r_j
#pragma unroll
          for (int i = 0; i < E; ++i) {
            const int e = lane + 32 * i;
            if (e < N * N) {
              const int k = e / N, r = e - k * N;
              sM[r * LDM + k] = mreg[q][i];
            }
          }
          const T rj = lane < N ? static_cast<T>(rreg[q]) : T(0);
          // u = q + r_j, or q alone with post_add (then r_j is added after the product)
          if (lane < N) su[lane] = a.post_add ? sq[lane] : sq[lane] + rj;
          load_a(j + PF, mreg[q], rreg[q]);
          __syncwarp();
          // P <- M_j P in register tiles: lane (rg, cq) forms rows RT rg .. RT rg + RT - 1
          // and columns 4 cq .. 4 cq + 3 from 16-byte loads of P and broadcast loads
          // of M_j's rows (k ascending, as a plain dot product)
          if (lane < kLanesA) {
            const int rg = lane / NCQ, cq = lane - rg * NCQ;
            T acc[RT][4];
#pragma unroll
            for (int rr = 0; rr < RT; ++rr)
#pragma unroll
              for (int i = 0; i < 4; ++i) acc[rr][i] = T(0);
#pragma unroll
            for (int k = 0; k < N; ++k) {
              T b4[4];
              ld4(Pc + k * N + 4 * cq, b4);
#pragma unroll
              for (int rr = 0; rr < RT; ++rr) {
                const T av = sM[(RT * rg + rr) * LDM + k];
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[rr][i] = fma(av, b4[i], acc[rr][i]);
              }
            }
#pragma unroll
            for (int rr = 0; rr < RT; ++rr) st4(Pn + (RT * rg + rr) * N + 4 * cq, acc[rr]);
          }
          if (lane < N) {
            T acc = a.post_add ? rj : T(0);
#pragma unroll
            for (int k = 0; k < N; ++k) acc = fma(sM[lane * LDM + k], su[k], acc);
            sq[lane] = acc;
          }
          __syncwarp();
          T* t = Pc;
          Pc = Pn;
          Pn = t;
        }
      }
    }
  }
  if (Pc != P0) {
    for (int e = lane; e < N * N; e += 32) P0[e] = Pc[e];
    __syncwarp();
  }
  __syncthreads();
  // ---- pass B: tile inputs d_in, in tile order ----
  if (warp == 0) {
    T d = (a.x_init && lane < N) ? static_cast<T>(a.x_init[b * N + lane]) : T(0);
    for (int w = 0; w < W; ++w) {
      T* wb = reinterpret_cast<T*>(tile_smem + static_cast<size_t>(w) * tile_warp_bytes<T, N>());
      const T* Pw = wb;
      const T* qw = wb + 2 * N * N + N * LDM;
      T* dw = wb + 2 * N * N + N * LDM + N;
      if (lane < N) dw[lane] = d;
      T acc = lane < N ? qw[lane] : T(0);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const T dk = __shfl_sync(kFull, d, k);
        if (lane < N) acc = fma(Pw[lane * N + k], dk, acc);
      }
      d = acc;
    }
  }
  __syncthreads();
  // ---- pass C: sweep the tile from its input ----
  T d = lane < N ? sd[lane] : T(0);
  {
    T mrow[PF][N];  // row `lane` of M_j: Mt[k * N + lane]
    double rreg[PF], xreg[PF];
    auto load_c = [&](int j, T (&mr)[N], double& rv, double& xv) {
      if (j < j1 && lane < N) {
        const T* Mt = Mb + static_cast<size_t>(j) * N * N;
#pragma unroll
        for (int k = 0; k < N; ++k) mr[k] = Mt[k * N + lane];
        rv = rhs_row(j)[lane];
        xv = a.mode != 1 ? xb[static_cast<size_t>(j) * N + lane] : 0.0;
      }
    };
#pragma unroll
    for (int q = 0; q < PF; ++q) load_c(j0 + q, mrow[q], rreg[q], xreg[q]);
#pragma unroll 1
    for (int jb = j0; jb < j1; jb += PF) {
#pragma unroll
      for (int q = 0; q < PF; ++q) {
        const int j = jb + q;
        if (j < j1) {  // warp-uniform
          const T rj = lane < N ? static_cast<T>(rreg[q]) : T(0);
          const T u = lane < N ? (a.post_add ? d : d + rj) : T(0);
          T acc0 = a.post_add ? rj : T(0), acc1 = T(0);
#pragma unroll
          for (int k = 0; k < N; k += 2) {
            const T u0 = __shfl_sync(kFull, u, k);
            const T u1 = __shfl_sync(kFull, u, k + 1);
            acc0 = fma(mrow[q][k], u0, acc0);
            acc1 = fma(mrow[q][k + 1], u1, acc1);
          }
          const T acc = acc0 + acc1;
          d = lane < N ? acc : T(0);
          if (lane < N) {
            const double dd = static_cast<double>(acc);
            xb[static_cast<size_t>(j) * N + lane] =
                (a.mode == 0) ? xreg[q] - dd : (a.mode == 1 ? dd : xreg[q] + dd);
          }
          load_c(j + PF, mrow[q], rreg[q], xreg[q]);
        }
      }
    }
  }
}

template <typename T, int N, int W>
cudaError_t launch_tile_chain(const ChainArgs& ch, cudaStream_t s) {
  const size_t sm = static_cast<size_t>(W) * tile_warp_bytes<T, N>();
  cudaError_t e = set_smem(tile_chain_kernel<T, N, W>, sm);
  if (e != cudaSuccess) return e;
  note_launch();
  tile_chain_kernel<T, N, W><<<ch.B, 32 * W, sm, s>>>(ch);
  return cudaGetLastError();
}

// tiles per series: 16 warps while their shared memory fits 200 KB, else 8
template <typename T, int N>
cudaError_t launch_tile_n(const ChainArgs& ch, cudaStream_t s) {
  if (16 * tile_warp_bytes<T, N>() <= 200 * 1024) return launch_tile_chain<T, N, 16>(ch, s);
  return launch_tile_chain<T, N, 8>(ch, s);
}

template <typename T, int N, int W>
cudaError_t launch_chain_n(const ChainArgs& ch, cudaStream_t s) {
  const dim3 grid((ch.B + W - 1) / W);
  const size_t sm = static_cast<size_t>(W) * chain_depth<T, N, W>() * chain_slot_bytes<T, N>();
  cudaError_t e = set_smem(mlp_chain_kernel<T, N, W>, sm);
  if (e != cudaSuccess) return e;
  note_launch();
  mlp_chain_kernel<T, N, W><<<grid, 32 * W, sm, s>>>(ch);
  return cudaGetLastError();
}

template <typename T, int W>
cudaError_t launch_chain_w(const ChainArgs& ch, cudaStream_t s) {
  switch (ch.n) {
    case 4: return launch_chain_n<T, 4, W>(ch, s);
    case 8: return launch_chain_n<T, 8, W>(ch, s);
    case 12: return launch_chain_n<T, 12, W>(ch, s);
    case 16: return launch_chain_n<T, 16, W>(ch, s);
    case 20: return launch_chain_n<T, 20, W>(ch, s);
    case 24: return launch_chain_n<T, 24, W>(ch, s);
    case 28: return launch_chain_n<T, 28, W>(ch, s);
    case 32: return launch_chain_n<T, 32, W>(ch, s);
    case 36: return launch_chain_n<T, 36, W>(ch, s);
    case 40: return launch_chain_n<T, 40, W>(ch, s);
    default: return cudaErrorInvalidValue;
  }
}

// One warp per series.  With few series, one warp per block spreads them over
// as many SMs; with many, four per block.
template <typename T>
cudaError_t launch_seq_chain(const ChainArgs& ch, cudaStream_t s) {
  return ch.B <= kChainOneWarpMaxSeries ? launch_chain_w<T, 1>(ch, s)
                                        : launch_chain_w<T, kChainWarps>(ch, s);
}

// Chain solve, chosen by block width (the paper's Thomas-versus-PCR trade-off,
// Sec. 5.3): the tiled hybrid (sequential depth L / W + W, n^3 / 32 FMAs a lane
// per step to compose the tiles) up to n = 16 -- n = 8 in FP64, whose products
// run on the 1/64-rate pipe -- and the sequential substitution (n^2 per step)
// above.  Measured on GB300 (FP32 blocks, series*steps/s of a whole step):
// n = 8 Chaboche 2.26e7 -> 4.38e7 (6.0e7 with the blocks read ahead), n = 16
// neural ODE 5.70e6 -> 6.06e6 with the tiles; n = 20 mass-damper-spring
// 1.79e7 -> 1.57e7 (1.84e7 with the blocks read ahead: even, at slightly more
// Newton updates) and n = 32 neural ODE 3.02e6 -> 2.42e6 (2.46e6), so the wider
// blocks keep the sequential solve.  Those figures predate the register tiles of
// pass A (one output a lane and iteration before, two shared loads per FMA); with
// them the tiles also take FP32 widths 20 and 24 whenever every series gets its
// own SM (the tiled kernel runs one block of W warps per series; the sequential
// one packs one warp per series, so it keeps large batches): measured, n = 20
// mass-damper-spring (100 series) 1.60e7 -> 2.16e7 and n = 24 coupled neurons
// (50 series) 8.47e6 -> 1.11e7, while n = 32 lost 3-5 % (50 and 128 series).
template <typename T>
cudaError_t launch_chain(const ChainArgs& ch, cudaStream_t s) {
  const int tile_max = sizeof(T) == sizeof(double) ? 8 : 16;
  if (ch.n > tile_max) {
    if constexpr (sizeof(T) == sizeof(float)) {
      int dev = 0, sms = 0;
      if (ch.n <= 24 && cudaGetDevice(&dev) == cudaSuccess &&
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
          ch.B <= sms) {
        switch (ch.n) {
          case 20: return launch_tile_n<T, 20>(ch, s);
          case 24: return launch_tile_n<T, 24>(ch, s);
          default: break;
        }
      }
    }
    return launch_seq_chain<T>(ch, s);
  }
  switch (ch.n) {
    case 4: return launch_tile_n<T, 4>(ch, s);
    case 8: return launch_tile_n<T, 8>(ch, s);
    case 12: return launch_tile_n<T, 12>(ch, s);
    case 16: return launch_tile_n<T, 16>(ch, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t mlp_launch_chain(int precision, const ChainArgs& ch, cudaStream_t s) {
  return precision == kPrecFp64 ? launch_chain<double>(ch, s) : launch_chain<float>(ch, s);
}

cudaError_t mlp_launch_check(int B, int it, int max_iter, double tol_abs, double tol_rel,
                             unsigned long long* norm, double* norm0, int* active, int* status,
                             int* iters, int* remaining, cudaStream_t s) {
  CheckArgs ck{B, it, max_iter, tol_abs, tol_rel, norm, norm0, active, status, iters, remaining};
  note_launch();
  mlp_check_kernel<<<(B + 127) / 128, 128, 0, s>>>(ck);
  return cudaGetLastError();
}

cudaError_t mlp_launch_chunk_begin(int B, int rowlen, int c, const int* mask, double* dy,
                                   int* active, unsigned long long* norm, int* iters,
                                   const int* status, int* status0, cudaStream_t s) {
  note_launch();
  chunk_begin_kernel<<<(static_cast<unsigned>(B) * c * rowlen + 255) / 256, 256, 0, s>>>(
      B, rowlen, c, mask, dy, active, norm, iters, status, status0);
  return cudaGetLastError();
}

cudaError_t mlp_launch_chunk_fail(int B, const int* mask, int* status, const int* status0,
                                  int* fail, int* nfail, int* stats, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(nfail, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  note_launch();
  chunk_fail_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, mask, status, status0, fail, nfail, stats);
  return cudaGetLastError();
}

bool mlp_supported(int n, int h1, int h2) {
  const bool n_ok = n == 4 || n == 8 || n == 16 || n == 32;  // index math uses shifts
  return n_ok && h1 >= 4 && h1 <= 128 && h1 % 4 == 0 && h2 >= 4 && h2 <= 128 && h2 % 4 == 0;
}

bool mlp_tc_supported(int n, int h1, int h2) {
  return mlp_supported(n, h1, h2) && tc_supported(dims_of(n, h1, h2));
}

size_t mlp_workspace_bytes(int n, int h1, int h2, int B, int chunk, int precision) {
  return carve(nullptr, B, chunk, dims_of(n, h1, h2), precision, true).total;
}

#define TVI_TRY(x)                          \
  do {                                      \
    cudaError_t e_ = (x);                   \
    if (e_ != cudaSuccess) return e_;       \
  } while (0)

// An attempt's first residual comes from mlp_residual_start_kernel unless the
// environment variable TVI_TEST_PER_PAIR_FIRST_PASS is set to 1 (a test hook:
// the per-pair kernel then evaluates every step, and the results must be the
// same bit for bit).
bool per_pair_first_pass() {
  const char* v = std::getenv("TVI_TEST_PER_PAIR_FIRST_PASS");
  return v && v[0] == '1' && v[1] == '\0';
}

cudaError_t mlp_forward(int kind, int n, int h1, int h2, int precision, const FwdArgs& a,
                        void* workspace, cudaStream_t s, int* host_worst) {
  const MlpDims d = dims_of(n, h1, h2);
  const bool start_pass = !per_pair_first_pass();
  const int B = a.B, N = a.N, c = a.chunk;
  const int fe = a.scheme == kSchemeForward ? 1 : 0;
  Ws w = carve(static_cast<char*>(workspace), B, c, d, precision, false);
  TVI_TRY(cudaMemsetAsync(w.worst, 0, sizeof(int), s));
  TVI_TRY(cudaMemsetAsync(w.tcerr, 0, sizeof(int), s));
  note_launch();
  convert_weights_kernel<<<(d.P + 255) / 256, 256, 0, s>>>(a.params, w.Wf, d.P);
  note_launch();
  mlp_start_kernel<<<(B * n + 255) / 256, 256, 0, s>>>(B, n, N + 1, a.y0, a.y_out, w.yi, w.status);
  TVI_TRY(cudaGetLastError());
  if (a.stats) TVI_TRY(cudaMemsetAsync(a.stats, 0, sizeof(int) * kStats * B, s));
  // One attempt over steps i0 + 1 .. i0 + L for the series in `mask` (all when
  // null).  With retry_halving, the series whose attempt failed (iteration limit
  // or non-finite residual) re-solve the same steps as two halves, recursively
  // down to one step (the same equations to the same tolerance: only where
  // Newton starts changes); a one-step failure sets the series' status.
  std::function<cudaError_t(int, int, const int*, int)> solve =
      [&](int i0, int L, const int* mask, int depth) -> cudaError_t {
    const bool halve = a.retry_halving && L > 1 && depth < kHalvingDepth;
    TVI_TRY(mlp_launch_chunk_begin(B, n, c, mask, w.dy, w.active, w.norm, w.iters, w.status,
                                   w.status0, s));
    for (int it = 0;; ++it) {
      ResidualArgs r{};
      r.d = d; r.B = B; r.N = N; r.i0 = i0; r.L = L; r.c = c; r.reverse = 0; r.fe = fe;
      r.times = a.times; r.lengths = a.lengths; r.params = a.params; r.yi = w.yi; r.dy = w.dy;
      r.R = w.R; r.dv = w.dv; r.norm = w.norm; r.active = w.active;
      TVI_TRY(it == 0 && start_pass ? launch_residual_start(kind, r, s)
                                    : launch_residual(kind, false, r, s));
      TVI_TRY(cudaMemsetAsync(w.remaining, 0, sizeof(int), s));
      CheckArgs ck{B, it, a.max_iter, a.tol_abs, a.tol_rel, w.norm, w.norm0, w.active, w.status,
                   w.iters, w.remaining};
      note_launch();
      mlp_check_kernel<<<(B + 127) / 128, 128, 0, s>>>(ck);
      TVI_TRY(cudaGetLastError());
      // the host reads how many series still iterate only every kHostCheckEvery
      // passes (and at the iteration limit, where the check stops every series);
      // passes enqueued after the last series stopped find none active and return
      if ((it + 1) % kHostCheckEvery == 0 || it >= a.max_iter) {
        int remaining = 0;
        TVI_TRY(cudaMemcpyAsync(&remaining, w.remaining, sizeof(int), cudaMemcpyDeviceToHost, s));
        TVI_TRY(cudaStreamSynchronize(s));
        if (remaining == 0) break;
      }
      BlocksArgs bk{};
      bk.d = d; bk.B = B; bk.N = N; bk.i0 = i0; bk.L = L; bk.c = c; bk.reverse = 0;
      bk.times = a.times; bk.lengths = a.lengths; bk.Wf = w.Wf; bk.Wd = a.params; bk.dv = w.dv;
      bk.active = w.active; bk.M = w.M; bk.fe = fe;
      ChainArgs ch{};
      ch.B = B; ch.n = n; ch.L = L; ch.c = c; ch.N = N; ch.i0 = i0; ch.reverse = 0; ch.M = w.M;
      ch.rhs_buf = w.R; ch.active = w.active; ch.x = w.dy; ch.mode = 0; ch.err = w.tcerr;
      ch.post_add = fe;  // forward Euler: d_j = (I + dt J) d_{j-1} + R_j
      TVI_TRY(launch_blocks_any(bk, precision, w.tcerr, s));
      TVI_TRY(precision == kPrecFp64 ? launch_chain<double>(ch, s) : launch_chain<float>(ch, s));
    }
    int* fail = halve ? w.fail + static_cast<size_t>(depth) * B : nullptr;
    int nfail = 0;
    if (halve) {
      TVI_TRY(mlp_launch_chunk_fail(B, mask, w.status, w.status0, fail, w.nfail, a.stats, s));
      TVI_TRY(cudaMemcpyAsync(&nfail, w.nfail, sizeof(int), cudaMemcpyDeviceToHost, s));
      TVI_TRY(cudaStreamSynchronize(s));
    }
    note_launch();
    mlp_store_kernel<<<B, 128, 0, s>>>(n, L, c, N, i0, a.lengths, w.dy, w.yi, a.y_out, w.iters,
                                       a.stats, mask, fail);
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
  mlp_worst_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, w.status, w.tcerr, a.series_status, w.worst);
  TVI_TRY(cudaGetLastError());
  if (host_worst) {
    TVI_TRY(cudaMemcpyAsync(host_worst, w.worst, sizeof(int), cudaMemcpyDeviceToHost, s));
    TVI_TRY(cudaStreamSynchronize(s));
  }
  return cudaSuccess;
}

cudaError_t mlp_adjoint(int kind, int n, int h1, int h2, int precision, const AdjArgs& a,
                        void* workspace, cudaStream_t s) {
  const MlpDims d = dims_of(n, h1, h2);
  const int B = a.B, N = a.N, c = a.chunk;
  const int fe = a.scheme == kSchemeForward ? 1 : 0;
  Ws w = carve(static_cast<char*>(workspace), B, c, d, precision, true);
  TVI_TRY(cudaMemsetAsync(w.tcerr, 0, sizeof(int), s));
  note_launch();
  convert_weights_kernel<<<(d.P + 255) / 256, 256, 0, s>>>(a.params, w.Wf, d.P);
  TVI_TRY(cudaMemsetAsync(w.carry, 0, sizeof(double) * B * n, s));  // a_{N+1} = 0
  TVI_TRY(cudaMemsetAsync(w.acc, 0, sizeof(double) * d.P, s));
  const int refine = precision == kPrecFp64 ? 0 : a.refine;
  // mixed precision: every MLP pass of the adjoint in FP32 (the refinement
  // residual is still assembled in FP64); FP64 blocks: FP64 throughout
  const bool mixed = precision != kPrecFp64;
  // dL/dp += sum over the L rows of the activations x the factors in del
  auto param_grad = [&](int L, const int* active) -> cudaError_t {
    // pairs split into up to kMaxParamSplits ranges of >= 1024 so the tiles fill the GPU
    const int npairs = B * L;
    int nsplit = (npairs + 1023) / 1024;
    nsplit = nsplit < 1 ? 1 : (nsplit > kMaxParamSplits ? kMaxParamSplits : nsplit);
    const int per = ((npairs + nsplit - 1) / nsplit + 63) / 64 * 64;
    nsplit = (npairs + per - 1) / per;
    ParamArgs pa{d, B, L, c, w.act, w.del, w.part, per, active};
    const dim3 pgrid(param_grad_tiles(d), nsplit);
    if (precision == kPrecFp64) {
      note_launch();
      mlp_param_grad_kernel<double><<<pgrid, 256, 0, s>>>(pa);
    } else {
      note_launch();
      mlp_param_grad_kernel<float><<<pgrid, 256, 0, s>>>(pa);
    }
    note_launch();
    mlp_param_reduce_kernel<<<(d.P + 255) / 256, 256, 0, s>>>(d.P, nsplit, w.part, w.acc);
    return cudaGetLastError();
  };
  const int nch = (N + c - 1) / c;
  for (int ci = nch - 1; ci >= 0; --ci) {
    const int i0 = ci * c;
    const int L = (N - i0 < c) ? N - i0 : c;
    // with per-series lengths, the series whose chunk lies wholly past its length
    // with zero dL/dy there skip it (their carry passes through)
    int* act_mask = nullptr;
    if (a.lengths) {
      note_launch();
      mlp_adj_active_kernel<<<B, 256, 0, s>>>(n, N + 1, i0, L, a.lengths, a.grad_out, w.active);
      TVI_TRY(cudaGetLastError());
      act_mask = w.active;
    }
    // activation derivatives at the stored trajectory, rows in reverse step order
    ResidualArgs r{};
    r.d = d; r.B = B; r.N = N; r.i0 = i0; r.L = L; r.c = c; r.reverse = 1;
    r.times = a.times; r.lengths = a.lengths; r.params = a.params; r.ytraj = a.y; r.dv = w.dv;
    r.act = w.act; r.Wf = w.Wf; r.active = act_mask;
    TVI_TRY(launch_residual(kind, mixed, r, s));
    BlocksArgs bk{};
    bk.d = d; bk.B = B; bk.N = N; bk.i0 = i0; bk.L = L; bk.c = c; bk.reverse = 1;
    bk.times = a.times; bk.lengths = a.lengths; bk.Wf = w.Wf; bk.Wd = a.params; bk.dv = w.dv;
    bk.M = w.M; bk.fe = fe; bk.active = act_mask;
    // a_j = A^-T (a_{j-1} + g_k), a_{-1} = carry (forward Euler: a_j = B^T a_{j-1} + g_k)
    ChainArgs ch{};
    ch.B = B; ch.n = n; ch.L = L; ch.c = c; ch.N = N; ch.i0 = i0; ch.reverse = 1; ch.M = w.M;
    ch.rhs_traj = a.grad_out; ch.x_init = w.carry; ch.x = w.dy; ch.mode = 1; ch.err = w.tcerr;
    ch.post_add = fe; ch.active = act_mask;
    TVI_TRY(launch_blocks_any(bk, precision, w.tcerr, s));
    TVI_TRY(precision == kPrecFp64 ? launch_chain<double>(ch, s) : launch_chain<float>(ch, s));
    VjpArgs v{};
    v.d = d; v.B = B; v.N = N; v.i0 = i0; v.L = L; v.c = c; v.times = a.times;
    v.lengths = a.lengths; v.params = a.params; v.Wf = w.Wf; v.g = a.grad_out;
    v.carry = w.carry; v.av = w.dy; v.fe = fe; v.active = act_mask;
    v.dv = w.dv;  // backward passes only: the derivative pass above stored act' and h'
    for (int it = 0; it < refine; ++it) {
      v.res = w.R;
      v.del = nullptr;
      TVI_TRY(launch_vjp(kind, mixed, v, s));
      ChainArgs cr = ch;
      cr.rhs_traj = nullptr;
      cr.rhs_buf = w.R;
      cr.x_init = nullptr;
      cr.mode = 2;  // a += correction
      TVI_TRY(precision == kPrecFp64 ? launch_chain<double>(cr, s) : launch_chain<float>(cr, s));
    }
    // parameter gradient factors at the final a, then the tiled sums
    v.res = nullptr;
    v.del = w.del;  // the activations were stored by the derivative pass
    TVI_TRY(launch_vjp(kind, mixed, v, s));
    TVI_TRY(param_grad(L, act_mask));
    note_launch();
    mlp_carry_kernel<<<(B * n + 255) / 256, 256, 0, s>>>(B, n, L, c, w.dy, w.carry, act_mask);
    TVI_TRY(cudaGetLastError());
  }
  if (fe && N > 0) {
    // Forward Euler's step 1 evaluates h at y_0, so its terms sit outside every
    // chunk: a one-row pass at y_0 with the VJP of a_1 (the carry) gives
    // dt_1 (dh/dp)^T a_1 for the gradient and, with that row's own a set to 0,
    // the residual g_0 + a_1 + dt_1 J(y_0)^T a_1 = dL/dy0 (App. A, explicit form).
    ResidualArgs r{};
    r.d = d; r.B = B; r.N = N; r.i0 = -1; r.L = 1; r.c = c; r.reverse = 1;
    r.times = a.times; r.lengths = a.lengths; r.params = a.params; r.ytraj = a.y; r.dv = w.dv;
    r.act = w.act; r.Wf = w.Wf;
    TVI_TRY(launch_residual(kind, mixed, r, s));
    TVI_TRY(cudaMemset2DAsync(w.dy, sizeof(double) * c * n, 0, sizeof(double) * n, B, s));
    VjpArgs v{};
    v.d = d; v.B = B; v.N = N; v.i0 = -1; v.L = 1; v.c = c; v.times = a.times;
    v.lengths = a.lengths; v.params = a.params; v.Wf = w.Wf; v.g = a.grad_out;
    v.carry = w.carry; v.av = w.dy; v.dv = w.dv; v.fe = 1; v.res = w.R; v.del = w.del;
    TVI_TRY(launch_vjp(kind, mixed, v, s));
    TVI_TRY(param_grad(1, nullptr));
  }
  const int cnt = (B * n > d.P) ? B * n : d.P;
  note_launch();
  mlp_adjoint_end_kernel<<<(cnt + 255) / 256, 256, 0, s>>>(
      B, n, N + 1, c, w.carry, a.grad_out, (fe && N > 0) ? w.R : nullptr, a.dy0, w.acc, a.dparams,
      d.P, w.tcerr);
  return cudaGetLastError();
}

}  // namespace tvi
