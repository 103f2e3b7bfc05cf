// tvi_small_kernels.cuh -- the fused per-series kernels of the small-state
// engine as templates over the model (see tvi_small.cu for the scheme).  Included
// by tvi_small.cu for the built-in models and compiled at run time (NVRTC) for
// models whose right-hand side the caller supplies as source (tvi_jit.cu).
#pragma once

#include "tvi_device.cuh"
#include "tvi_internal.h"
#include "tvi_predictor.cuh"

namespace tvi {
namespace kern {

// time t_k of a model evaluation; models that ignore t (Model::kUsesTime false)
// get 0 without a load, so the time lookups leave their kernels unchanged
template <class Model>
__device__ __forceinline__ double model_time(const double* tb, int k) {
  if constexpr (Model::kUsesTime) return tb[k];
  else return 0.0;
}

// Infinity norm of the chunk residual R_j = dy_j - dy_{j-1} - dt_j h(y_i + dy_j)
// for increments dyv, over the whole block (every thread calls it; full-block
// barriers).  Returns the FP64 bit pattern of the max (NaN/Inf compare high).
template <class Model, int RPT>
__device__ __forceinline__ unsigned long long residual_norm_block(
    const Model& mdl, const double (&yi)[Model::NS], const double (&dyv)[RPT][Model::NS],
    const double (&dt)[RPT], const bool (&act)[RPT], int rpa, const double* tb, int k0,
    double (*s_wlast)[Model::NS], unsigned long long* s_red, int lane, int warp) {
  constexpr int NS = Model::NS;
  const int nwarps = static_cast<int>(blockDim.x >> 5);
  double prev[NS], mine[NS];
  last_row<RPT, NS>(dyv, rpa, mine);
#pragma unroll
  for (int s = 0; s < NS; ++s) prev[s] = __shfl_up_sync(kFull, mine[s], 1);
  if (lane == 31) {
#pragma unroll
    for (int s = 0; s < NS; ++s) s_wlast[warp][s] = mine[s];
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) prev[s] = (warp > 0) ? s_wlast[warp - 1][s] : 0.0;
  }
  unsigned long long mx = 0ull;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    if (r >= rpa) break;  // block-uniform
    double y[NS], h[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) y[s] = yi[s] + dyv[r][s];
    mdl.rhs(y, act[r] ? model_time<Model>(tb, k0 + r) : 0.0, h);  // row r is step k0 + r
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const double pv = (r == 0) ? prev[s] : dyv[r - 1][s];
      if (act[r]) mx = umax64(mx, abs_bits(fma(-dt[r], h[s], dyv[r][s] - pv)));
    }
  }
  const unsigned long long nb = block_max_u64(mx, s_red, lane, warp, nwarps);
  __syncthreads();  // s_wlast and s_red are reused by the next call
  return nb;
}

// Newton outcome of one chunk attempt.
enum { kConv = 0, kMaxIter = 1, kNonFinite = 2, kDiverged = 3 };

// shortest converged prefix of a failed chunk attempt that is kept
constexpr int kMinPrefix = 8;

template <class Model, typename T, int RPT>
__global__ void __launch_bounds__(small_max_threads(RPT)) forward_small_kernel(FwdArgs a) {
  constexpr int NS = Model::NS;
  constexpr bool kMixed = sizeof(T) != sizeof(double);
  __shared__ Aff<NS, T> s_wtot[32];
  __shared__ double s_wlast[32][NS];
  __shared__ unsigned long long s_red[32];
  __shared__ double s_carry[NS];
  __shared__ int s_ctl[3];  // outcome, Newton updates and converged prefix of the last attempt
  // predictor features, hidden activations and outputs (van der Pol only)
  __shared__ float s_pred[Model::kPredictable
                              ? (NS + 1 + kPredMaxChunk) + 2 * kPredMaxHidden + NS * kPredMaxChunk
                              : 1];

  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int pred_used = 0, pred_rejected = 0;
  int pred_wait = 0, pred_streak = 0;  // back-off after rejected guesses
  const bool fwd_euler = a.scheme == kSchemeForward;
  const int N = a.N;
  const double* tb = a.times + static_cast<size_t>(b) * (N + 1);
  double* yb = a.y_out + static_cast<size_t>(b) * (N + 1) * NS;
  const int len = a.lengths ? min(max(a.lengths[b], 0), N) : N;

  Model mdl;
  mdl.load(a.params, b, a.per_series);

  double yi[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) yi[s] = a.y0[static_cast<size_t>(b) * NS + s];
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) yb[s] = yi[s];
  }

  int st = 0, tot_iters = 0, n_chunks = 0, retries = 0, max_it = 0, streak = 0;
  int i = 0, c_cur = a.chunk;
  while (i < N) {
    const int L = min(c_cur, N - i);
    // rows per thread of this attempt: one while the attempt fits the block's
    // threads, else RPT.  A warp's FP64 instructions issue one per 64 cycles
    // whatever its active lanes, so a short attempt spread one row per thread
    // runs half the FP64 instructions per warp (and more warps in parallel).
    const int rpa = (L + static_cast<int>(blockDim.x) - 1) / static_cast<int>(blockDim.x);
    // warps holding at least one step of this attempt; the rest skip all work
    const int nwa = ((L + rpa - 1) / rpa + 31) / 32;
    const bool wact = warp < nwa;
    const bool can_halve = a.retry_halving && c_cur > 1;
    // ---- per-thread rows of this chunk attempt ----
    // the iterate is held as y_j = y_i + dy_j itself (FP64), so the residual needs
    // no y_i + dy_j adds: 9 FP64 operations per step and pass (van der Pol)
    double dt[RPT], yv[RPT][NS];
    T dtT[RPT], yiT[NS], yT[RPT][NS];  // block-precision shadows (mixed mode)
    bool act[RPT];
#pragma unroll
    for (int s = 0; s < NS; ++s) yiT[s] = narrow<T>(yi[s]);
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int j = tid * rpa + r;
      const int k = i + 1 + j;
      act[r] = r < rpa && j < L;
      dt[r] = (act[r] && k <= len) ? (tb[k] - tb[k - 1]) : 0.0;
      dtT[r] = narrow<T>(dt[r]);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        yv[r][s] = yi[s];  // Sec. 2.3 guess: dy = 0
        yT[r][s] = yiT[s];
      }
    }

    // ---- learned Newton predictor: replace dy = 0 by the proposed increments
    // when their FP64 residual is smaller (results unchanged: Newton still runs
    // to the tolerance) ----
    if constexpr (Model::kPredictable) {
      const bool pred_try = a.pred && L == a.pred_chunk && pred_wait == 0;
      if (a.pred && L == a.pred_chunk && pred_wait > 0) --pred_wait;
      if (pred_try) {
        const PredDims pd{NS + 1 + L, a.pred_hid, NS * L};
        float* feat = s_pred;
        float* h1 = feat + pd.in;
        float* h2 = h1 + pd.hid;
        float* outv = h2 + pd.hid;
        if (tid < NS) feat[tid] = static_cast<float>(yi[tid]);
        if (tid == 0) feat[NS] = mdl.param_feature();
#pragma unroll
        for (int r = 0; r < RPT; ++r)
          if (act[r]) feat[NS + 1 + tid * rpa + r] = log10f(fmaxf(static_cast<float>(dt[r]), 1e-30f));
        __syncthreads();
        pred_infer_block(a.pred, pd, feat, h1, h2, outv);
        // the network proposes per-step slopes s_j; the guess is their running
        // sum dy_j = sum_{l <= j} dt_l s_l (warp 0 scans, FP64 sums)
#pragma unroll
        for (int r = 0; r < RPT; ++r)
          if (act[r])
#pragma unroll
            for (int s = 0; s < NS; ++s) outv[(tid * rpa + r) * NS + s] *= static_cast<float>(dt[r]);
        __syncthreads();
        if (warp == 0) {
          constexpr int kPer = (kPredMaxChunk + 31) / 32;
          const int j0 = lane * kPer;
          double own[NS], incl[NS];
#pragma unroll
          for (int s = 0; s < NS; ++s) own[s] = 0.0;
#pragma unroll
          for (int q = 0; q < kPer; ++q)
            if (j0 + q < L)
#pragma unroll
              for (int s = 0; s < NS; ++s) own[s] += outv[(j0 + q) * NS + s];
#pragma unroll
          for (int s = 0; s < NS; ++s) incl[s] = own[s];
#pragma unroll
          for (int off = 1; off < 32; off <<= 1)
#pragma unroll
            for (int s = 0; s < NS; ++s) {
              const double v = __shfl_up_sync(0xffffffffu, incl[s], off);
              if (lane >= off) incl[s] += v;
            }
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            const double prev = __shfl_up_sync(0xffffffffu, incl[s], 1);
            own[s] = lane > 0 ? prev : 0.0;  // sum over the lanes before this one
          }
#pragma unroll
          for (int q = 0; q < kPer; ++q)
            if (j0 + q < L)
#pragma unroll
              for (int s = 0; s < NS; ++s) {
                own[s] += outv[(j0 + q) * NS + s];
                outv[(j0 + q) * NS + s] = static_cast<float>(own[s]);
              }
        }
        __syncthreads();
        double dyp[RPT][NS];
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
          for (int s = 0; s < NS; ++s)
            dyp[r][s] = act[r] ? static_cast<double>(outv[(tid * rpa + r) * NS + s]) : 0.0;
        double dz[RPT][NS];
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
          for (int s = 0; s < NS; ++s) dz[r][s] = 0.0;
        const unsigned long long n_zero =
            residual_norm_block<Model, RPT>(mdl, yi, dz, dt, act, rpa, tb, i + 1 + tid * rpa,
                                            s_wlast, s_red, lane, warp);
        const unsigned long long n_pred =
            residual_norm_block<Model, RPT>(mdl, yi, dyp, dt, act, rpa, tb, i + 1 + tid * rpa,
                                            s_wlast, s_red, lane, warp);
        if (n_pred < n_zero) {  // both finite bit patterns compare as values
#pragma unroll
          for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int s = 0; s < NS; ++s) {
              yv[r][s] = yi[s] + dyp[r][s];
              yT[r][s] = narrow<T>(yv[r][s]);
            }
          ++pred_used;
          pred_streak = 0;
        } else {
          // k rejections in a row: skip the predictor on the next 2^k - 1 eligible
          // chunks (k <= 5); n_pred and n_zero are block-wide, so all threads agree
          ++pred_rejected;
          pred_streak = min(pred_streak + 1, 5);
          pred_wait = (1 << pred_streak) - 1;
        }
      }
    }

    int it = 0, outcome = kConv;
    // Convergence and divergence are decided on FP64 bit patterns (ordered like
    // the values for non-negative doubles) against thresholds formed once per
    // attempt from its first residual, so no FP64 instruction sits in a pass's
    // control flow.
    unsigned long long thr_bits = 0ull, div_bits = 0ull;
    // Only the nwa warps holding steps run the Newton loop; they synchronise on
    // a named barrier among themselves, the others wait at the barrier after it.
    if (wact) {
    for (;;) {
      // y_{j-1} of the first own row: last row of the previous thread
      double prev[NS], mine[NS];
      last_row<RPT, NS>(yv, rpa, mine);
#pragma unroll
      for (int s = 0; s < NS; ++s) prev[s] = __shfl_up_sync(kFull, mine[s], 1);
      if (lane == 31) {
#pragma unroll
        for (int s = 0; s < NS; ++s) s_wlast[warp][s] = mine[s];
      }
      sync_first(32 * nwa);
      if (lane == 0) {  // the row before row 0 is the chunk start y_i
#pragma unroll
        for (int s = 0; s < NS; ++s) prev[s] = (warp > 0) ? s_wlast[warp - 1][s] : yi[s];
      }
      // ---- residual, FP64 ----
      double R[RPT][NS];
      unsigned long long mx = 0ull;
#pragma unroll
      for (int r = 0; r < RPT; ++r)
#pragma unroll
        for (int s = 0; s < NS; ++s) R[r][s] = 0.0;
      if (wact) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          if (r >= rpa) break;  // block-uniform: no FP64 work for rows this attempt lacks
          // backward Euler evaluates h at y_j, forward Euler at y_{j-1} (Sec. 2.2)
          double yp[NS], yh[NS], h[NS];
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            yp[s] = (r == 0) ? prev[s] : yv[r - 1][s];
            yh[s] = fwd_euler ? yp[s] : yv[r][s];
          }
          const int k = i + 1 + tid * rpa + r;
          mdl.rhs(yh, act[r] ? model_time<Model>(tb, fwd_euler ? k - 1 : k) : 0.0, h);
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            // rows past the attempt's end compute a value that nothing reads (every
            // later use of R is guarded by act): no select on the FP64 result
            R[r][s] = fma(-dt[r], h[s], yv[r][s] - yp[s]);
            if (act[r]) mx = umax64(mx, abs_bits(R[r][s]));
          }
        }
      }
      const unsigned long long nb = block_max_u64(mx, s_red, lane, warp, nwa);
      if (it == 0) {  // this attempt's thresholds, from its first residual
        const double nr0 = __longlong_as_double(static_cast<long long>(nb));
        thr_bits = abs_bits(fmax(a.tol_abs, a.tol_rel * nr0));
        div_bits = abs_bits(10.0 * nr0);
      }
      if (nb <= thr_bits) {  // finite and within tol_abs or tol_rel ||R_0||
        outcome = kConv;
        break;
      }
      // When a smaller chunk can still be tried, an attempt whose residual is
      // still above 10x its starting value after 4 updates is abandoned early
      // (a heuristic for speed only: the retry solves the same equations).
      const int fail = nb >= kNonFiniteBits                      ? kNonFinite
                       : it >= a.max_iter                        ? kMaxIter
                       : (can_halve && it >= 4 && nb > div_bits) ? kDiverged
                                                                 : kConv;
      if (fail != kConv) {
        outcome = fail;
        if (can_halve) {
          // Rows whose backward-Euler residual is already within the tolerance form
          // a solution of their steps (row j involves only y_{j-1} and y_j), so the
          // attempt's longest such prefix is kept: first row index over tolerance.
          unsigned long long v = 0ull;  // ~j of the first row over tolerance, max-reduced
#pragma unroll
          for (int r = 0; r < RPT; ++r) {
            bool over = false;
#pragma unroll
            for (int s = 0; s < NS; ++s) over = over || abs_bits(R[r][s]) > thr_bits;
            if (act[r] && over) v = umax64(v, ~static_cast<unsigned long long>(tid * rpa + r));
          }
          sync_first(32 * nwa);  // s_red reuse
          const unsigned long long m = block_max_u64(v, s_red, lane, warp, nwa);
          if (tid == 0) s_ctl[2] = m ? static_cast<int>(~m) : L;
        }
        break;
      }

      // ---- blocks, their inverses, and the cyclic-reduction solve ----
      Aff<NS, T> f[RPT];
      T d[RPT][NS];
      if (wact) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          if (act[r]) {
            T yt[NS], A[NS][NS];
#pragma unroll
            for (int s = 0; s < NS; ++s) {
              if (fwd_euler) {  // the Jacobian block of forward Euler is taken at y_{j-1}
                if constexpr (kMixed) yt[s] = (r == 0) ? narrow<T>(prev[s]) : yT[r - 1][s];
                else yt[s] = (r == 0) ? prev[s] : yv[r - 1][s];
              } else {
                if constexpr (kMixed) yt[s] = yT[r][s];
                else yt[s] = yv[r][s];
              }
            }
            const int k = i + 1 + tid * rpa + r;
            mdl.step_matrix(yt, model_time<Model>(tb, fwd_euler ? k - 1 : k), dtT[r],
                            A);  // A = I - dt j
            T Rt[NS];
#pragma unroll
            for (int q = 0; q < NS; ++q) Rt[q] = narrow<T>(R[r][q]);
            if (fwd_euler) {
              // diagonal block I, sub-diagonal -(I + dt j): d_j = (2I - A) d_{j-1} + R_j
#pragma unroll
              for (int p = 0; p < NS; ++p) {
#pragma unroll
                for (int q = 0; q < NS; ++q) f[r].M[p][q] = (p == q ? T(2) : T(0)) - A[p][q];
                f[r].v[p] = Rt[p];
              }
            } else {
              block_inverse<NS, T>(A, f[r].M);
#pragma unroll
              for (int p = 0; p < NS; ++p) {
                T sacc = T(0);
#pragma unroll
                for (int q = 0; q < NS; ++q) sacc = fma(f[r].M[p][q], Rt[q], sacc);
                f[r].v[p] = sacc;
              }
            }
          } else {
            aff_identity(f[r]);
          }
        }
      }
      solve_chain<NS, T, RPT>(f, d, s_wtot, lane, warp, nwa, rpa,
                              nwa > 1 ? 32 : (L + rpa - 1) / rpa);
      // ---- Newton update, FP64 accumulate ----
      if (wact) {
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
          for (int s = 0; s < NS; ++s)
            if (r < rpa && act[r]) {
              yv[r][s] -= widen<T>(d[r][s]);
              if constexpr (kMixed) yT[r][s] -= d[r][s];
            }
      }
      ++it;
    }
    if (tid == 0) {
      s_ctl[0] = outcome;
      s_ctl[1] = it;
    }
    }  // wact
    __syncthreads();
    outcome = s_ctl[0];
    it = s_ctl[1];

    if (outcome != kConv && can_halve) {
      // keep a converged prefix of at least kMinPrefix steps, then re-solve the rest
      // of the chunk from its end with half the steps
      const int K = s_ctl[2];
      if (K >= kMinPrefix) {
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          const int j = tid * rpa + r;
          if (act[r] && j < K) {
            double* out = yb + static_cast<size_t>(i + 1 + j) * NS;
#pragma unroll
            for (int s = 0; s < NS; ++s) out[s] = yv[r][s];
          }
          if (act[r] && j == K - 1) {
#pragma unroll
            for (int s = 0; s < NS; ++s) s_carry[s] = yv[r][s];
          }
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < NS; ++s) yi[s] = s_carry[s];
        i += K;
        tot_iters += it;
        ++n_chunks;
        max_it = max(max_it, it);
      }
      c_cur = (c_cur + 1) / 2;
      ++retries;
      streak = 0;
      __syncthreads();  // s_wlast / s_red / s_carry reuse
      continue;
    }
    if (outcome == kNonFinite) st = 2;
    else if (outcome != kConv && st == 0) st = 1;
    tot_iters += it;
    ++n_chunks;
    max_it = max(max_it, it);

    // ---- write the chunk's trajectory and carry y_{i+L} ----
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int j = tid * rpa + r;
      if (act[r]) {
        double* out = yb + static_cast<size_t>(i + 1 + j) * NS;
#pragma unroll
        for (int s = 0; s < NS; ++s) out[s] = yv[r][s];
      }
      if (act[r] && j == L - 1) {
#pragma unroll
        for (int s = 0; s < NS; ++s) s_carry[s] = yv[r][s];
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < NS; ++s) yi[s] = s_carry[s];
    __syncthreads();
    i += L;
    // after two successes in a row the chunk grows back by doubling, up to
    // the requested size (as in step-size control)
    if (++streak >= 2) {
      c_cur = min(a.chunk, 2 * c_cur);
      streak = 0;
    }
  }

  if (tid == 0) {
    if (a.stats) {
      int* o = a.stats + static_cast<size_t>(b) * kStats;
      o[0] = tot_iters;
      o[1] = n_chunks;
      o[2] = retries;
      o[3] = max_it;
      o[4] = pred_used;
      o[5] = pred_rejected;
    }
    if (a.series_status) a.series_status[b] = st;
    if (st) atomicMax(a.worst, st);
  }
}

// Adjoint of one series, chunks in reverse (App. A.2).  Within a chunk of L
// steps k = i+1..i+L the unknowns are taken in reverse order, q = i+L+1-k, so
//     A_k^T a_k - a_{k+1} = g_k    becomes    x_q = A_k^-T x_{q-1} + A_k^-T g_k,
// x_{-1} = a_{i+L+1} (the carry from the later chunk, folded into row 0) -- the
// same chain as the forward pass with transposed blocks.  In mixed precision
// the chain is solved in T and refined with FP64 residuals
//     r_k = g_k + a_{k+1} - A_k^T a_k   (A_k in FP64).
template <class Model, typename T, int RPT>
__global__ void __launch_bounds__(small_max_threads(RPT)) adjoint_small_kernel(AdjArgs a) {
  constexpr int NS = Model::NS;
  constexpr int NP = Model::NP;
  __shared__ Aff<NS, T> s_wtot[32];
  __shared__ double s_wlast[32][NS];
  __shared__ double s_carry[NS];
  __shared__ double s_acc[32][NP];

  const int b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int N = a.N, c = a.chunk;
  const bool fwd_euler = a.scheme == kSchemeForward;
  const double* tb = a.times + static_cast<size_t>(b) * (N + 1);
  const double* yb = a.y + static_cast<size_t>(b) * (N + 1) * NS;
  const double* gb = a.grad_out + static_cast<size_t>(b) * (N + 1) * NS;
  const int len = a.lengths ? min(max(a.lengths[b], 0), N) : N;

  Model mdl;
  mdl.load(a.params, b, a.per_series);

  double carry[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) carry[s] = 0.0;  // a_{N+1} = 0
  double acc[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) acc[p] = 0.0;

  const int n_chunks = (N + c - 1) / c;
  for (int ci = n_chunks - 1; ci >= 0; --ci) {
    const int i = ci * c;
    const int L = min(c, N - i);
    const int nwa = ((L + RPT - 1) / RPT + 31) / 32;
    double yk[RPT][NS], gk[RPT][NS], dt[RPT], dtb[RPT], av[RPT][NS];
    bool act[RPT];
    Aff<NS, T> f[RPT];
    // warps holding no step of a short (last) chunk skip to the carry barrier
    const bool wact = warp < nwa;
    if (wact) {
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int q = tid * RPT + r;
      act[r] = q < L;
      const int k = i + L - q;
      dt[r] = (act[r] && k <= len) ? (tb[k] - tb[k - 1]) : 0.0;
      // the step whose block couples a_k to a_{k+1}: backward Euler dt_k at y_k;
      // forward Euler dt_{k+1} at y_k (a_k = g_k + (I + dt_{k+1} j_k)^T a_{k+1})
      dtb[r] = !fwd_euler ? dt[r] : ((act[r] && k + 1 <= len) ? (tb[k + 1] - tb[k]) : 0.0);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        yk[r][s] = act[r] ? yb[static_cast<size_t>(k) * NS + s] : 0.0;
        gk[r][s] = act[r] ? gb[static_cast<size_t>(k) * NS + s] : 0.0;
      }
      if (act[r]) {
        T yt[NS], A[NS][NS], Ai[NS][NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) yt[s] = narrow<T>(yk[r][s]);
        mdl.step_matrix(yt, model_time<Model>(tb, k), narrow<T>(dtb[r]),
                        A);  // A = I - dt j(y_k, t_k)
        if (fwd_euler) {
          // x_q = (2I - A)^T x_{q-1} + g_k, the carry a_{i+L+1} entering row 0
#pragma unroll
          for (int p = 0; p < NS; ++p)
#pragma unroll
            for (int q2 = 0; q2 < NS; ++q2) f[r].M[p][q2] = (p == q2 ? T(2) : T(0)) - A[q2][p];
#pragma unroll
          for (int p = 0; p < NS; ++p) {
            T sacc = narrow<T>(gk[r][p]);
            if (q == 0)
#pragma unroll
              for (int q2 = 0; q2 < NS; ++q2) sacc = fma(f[r].M[p][q2], narrow<T>(carry[q2]), sacc);
            f[r].v[p] = sacc;
          }
        } else {
          block_inverse<NS, T>(A, Ai);
#pragma unroll
          for (int p = 0; p < NS; ++p)
#pragma unroll
            for (int q2 = 0; q2 < NS; ++q2) f[r].M[p][q2] = Ai[q2][p];  // A^-T
          double rhs[NS];
#pragma unroll
          for (int s = 0; s < NS; ++s) rhs[s] = gk[r][s] + ((q == 0) ? carry[s] : 0.0);
#pragma unroll
          for (int p = 0; p < NS; ++p) {
            T sacc = T(0);
#pragma unroll
            for (int q2 = 0; q2 < NS; ++q2) sacc = fma(f[r].M[p][q2], narrow<T>(rhs[q2]), sacc);
            f[r].v[p] = sacc;
          }
        }
      } else {
        aff_identity(f[r]);
      }
    }
    {
      T x[RPT][NS];
      solve_chain<NS, T, RPT>(f, x, s_wtot, lane, warp, nwa);
#pragma unroll
      for (int r = 0; r < RPT; ++r)
#pragma unroll
        for (int s = 0; s < NS; ++s) av[r][s] = act[r] ? widen<T>(x[r][s]) : 0.0;
    }
    // ---- FP64-residual refinement (mixed precision) ----
    for (int ref = 0; ref < a.refine; ++ref) {
      double nxt[NS];  // a_{k+1} of the first own row: last row of the previous thread
#pragma unroll
      for (int s = 0; s < NS; ++s) nxt[s] = __shfl_up_sync(kFull, av[RPT - 1][s], 1);
      if (lane == 31) {
#pragma unroll
        for (int s = 0; s < NS; ++s) s_wlast[warp][s] = av[RPT - 1][s];
      }
      sync_first(32 * nwa);
      if (lane == 0) {
#pragma unroll
        for (int s = 0; s < NS; ++s) nxt[s] = (warp > 0) ? s_wlast[warp - 1][s] : 0.0;
      }
      if (tid == 0) {
#pragma unroll
        for (int s = 0; s < NS; ++s) nxt[s] = carry[s];
      }
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        double A[NS][NS];
        const int k = i + L - (tid * RPT + r);
        mdl.step_matrix(yk[r], act[r] ? model_time<Model>(tb, k) : 0.0, dtb[r], A);
        double res[NS];
#pragma unroll
        for (int p = 0; p < NS; ++p) {
          double sacc;
          if (fwd_euler) {  // g_k + (2I - A)^T a_{k+1} - a_k
            sacc = gk[r][p] - av[r][p];
#pragma unroll
            for (int q2 = 0; q2 < NS; ++q2) {
              const double an = (r == 0) ? nxt[q2] : av[r - 1][q2];
              sacc = fma((p == q2 ? 2.0 : 0.0) - A[q2][p], an, sacc);
            }
          } else {  // g_k + a_{k+1} - A^T a_k
            sacc = gk[r][p] + ((r == 0) ? nxt[p] : av[r - 1][p]);
#pragma unroll
            for (int q2 = 0; q2 < NS; ++q2) sacc = fma(-A[q2][p], av[r][q2], sacc);
          }
          res[p] = act[r] ? sacc : 0.0;
        }
#pragma unroll
        for (int p = 0; p < NS; ++p) {
          T sacc = T(0);
#pragma unroll
          for (int q2 = 0; q2 < NS; ++q2) sacc = fma(f[r].M[p][q2], narrow<T>(res[q2]), sacc);
          f[r].v[p] = act[r] ? sacc : T(0);
        }
      }
      T x[RPT][NS];
      solve_chain<NS, T, RPT>(f, x, s_wtot, lane, warp, nwa);
#pragma unroll
      for (int r = 0; r < RPT; ++r)
#pragma unroll
        for (int s = 0; s < NS; ++s) av[r][s] += act[r] ? widen<T>(x[r][s]) : 0.0;
      sync_first(32 * nwa);  // s_wlast reuse
    }
    // ---- parameter VJP: acc += dt_k (dh/dp)^T a_k ----
#pragma unroll
    for (int r = 0; r < RPT; ++r)
      if (act[r] && dt[r] != 0.0) {
        if (fwd_euler) {  // forward Euler's step k evaluates h at y_{k-1}
          const int k = i + L - (tid * RPT + r);
          double ykm[NS];
#pragma unroll
          for (int s = 0; s < NS; ++s) ykm[s] = yb[static_cast<size_t>(k - 1) * NS + s];
          mdl.vjp_p(ykm, model_time<Model>(tb, k - 1), av[r], dt[r], acc);
        } else {
          mdl.vjp_p(yk[r], model_time<Model>(tb, i + L - (tid * RPT + r)), av[r], dt[r], acc);
        }
      }
    }  // wact
    // ---- carry a_{i+1} (row L-1) to the earlier chunk ----
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (tid * RPT + r == L - 1) {
#pragma unroll
        for (int s = 0; s < NS; ++s) s_carry[s] = av[r][s];
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < NS; ++s) carry[s] = s_carry[s];
    __syncthreads();
  }

  // dL/dy0 = a_1 + dL/dy_0
  if (tid == 0 && a.dy0) {
    if (fwd_euler) {  // lambda_0 = g_0 + (I + dt_1 j(y_0))^T a_1
      double y0v[NS], A[NS][NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) y0v[s] = yb[s];
      mdl.step_matrix(y0v, tb[0], (N >= 1 && 1 <= len) ? tb[1] - tb[0] : 0.0, A);
#pragma unroll
      for (int p = 0; p < NS; ++p) {
        double v = gb[p];
#pragma unroll
        for (int q2 = 0; q2 < NS; ++q2) v = fma((p == q2 ? 2.0 : 0.0) - A[q2][p], carry[q2], v);
        a.dy0[static_cast<size_t>(b) * NS + p] = v;
      }
    } else {
#pragma unroll
      for (int s = 0; s < NS; ++s) a.dy0[static_cast<size_t>(b) * NS + s] = carry[s] + gb[s];
    }
  }
  // deterministic block sum of the parameter gradient: warp tree, then warps in order
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    double v = acc[p];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0) s_acc[warp][p] = v;
  }
  __syncthreads();
  if (tid < NP) {
    double v = 0.0;
    for (int w = 0; w < nwarps; ++w) v += s_acc[w][tid];
    double* dst = a.per_series ? a.dparams + static_cast<size_t>(b) * NP
                               : a.partials + static_cast<size_t>(b) * NP;
    dst[tid] = v;
  }
}

}  // namespace kern
}  // namespace tvi
