// tvi_device.cuh -- device building blocks of the chunked backward-Euler solver.
//
// The block lower-bidiagonal Newton system of one chunk (Eq. batched-update),
//     A_j d_j - d_{j-1} = R_j,   j = 1..c,   d_0 = 0,
// is written as the chain of affine maps d_j = M_j d_{j-1} + v_j with
// M_j = A_j^{-1} and v_j = A_j^{-1} R_j (the sub-diagonal blocks are -I, so the
// normalised coupling is +A_j^{-1}).  Parallel cyclic reduction (Sec. 3.2,
// Alg. 3) on this normalised form is the stride-doubling update
//     v_j <- M_j v_{j-s} + v_j,   M_j <- M_j M_{j-s}   (s = 1, 2, 4, ...),
// all rows using the previous level's values: after ceil(log2 c) levels every
// v_j equals d_j.  Here that reduction runs over the lanes of a warp (register
// shuffles), then over the warps of the block (shared memory), with each
// thread first composing its own run of consecutive rows (the Sec. 3.3 hybrid:
// serial substitution inside a thread, cyclic reduction across threads).
#pragma once

#ifndef __CUDACC_RTC__  // host compile (NVRTC provides the device built-ins)
#include <cuda_runtime.h>
#include <stdint.h>
#endif

namespace tvi {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Affine map x -> M x + v on R^NS.
// ---------------------------------------------------------------------------
template <int NS, typename T>
struct Aff {
  T M[NS][NS];
  T v[NS];
};

template <int NS, typename T>
__device__ __forceinline__ void aff_identity(Aff<NS, T>& f) {
#pragma unroll
  for (int i = 0; i < NS; ++i) {
#pragma unroll
    for (int j = 0; j < NS; ++j) f.M[i][j] = (i == j) ? T(1) : T(0);
    f.v[i] = T(0);
  }
}

// out = b o a  (apply a first): M = Mb Ma, v = Mb va + vb.
template <int NS, typename T>
__device__ __forceinline__ Aff<NS, T> compose(const Aff<NS, T>& b, const Aff<NS, T>& a) {
  Aff<NS, T> o;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
#pragma unroll
    for (int j = 0; j < NS; ++j) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < NS; ++k) s = fma(b.M[i][k], a.M[k][j], s);
      o.M[i][j] = s;
    }
    T s = b.v[i];
#pragma unroll
    for (int k = 0; k < NS; ++k) s = fma(b.M[i][k], a.v[k], s);
    o.v[i] = s;
  }
  return o;
}

template <int NS, typename T>
__device__ __forceinline__ Aff<NS, T> shfl_up_aff(const Aff<NS, T>& f, int s) {
  Aff<NS, T> o;
#pragma unroll
  for (int i = 0; i < NS; ++i) {
#pragma unroll
    for (int j = 0; j < NS; ++j) o.M[i][j] = __shfl_up_sync(kFull, f.M[i][j], s);
    o.v[i] = __shfl_up_sync(kFull, f.v[i], s);
  }
  return o;
}

// 1/x for the block algebra: the division in FP64, a fast reciprocal (at most 2
// ulp from the rounded quotient) in FP32, where the blocks only steer Newton
// updates whose FP64 residual decides convergence.
template <typename T>
__device__ __forceinline__ T recip(T x) {
  if constexpr (sizeof(T) == sizeof(double)) return T(1) / x;
  else return __fdividef(1.0f, x);
}

// ---------------------------------------------------------------------------
// Block inverse: Gauss-Jordan with partial pivoting, fully in registers (row
// swaps are predicated selects, so no local memory).  NS = 2 uses the closed
// form adj(A)/det(A).
// ---------------------------------------------------------------------------
template <int NS, typename T>
__device__ __forceinline__ void block_inverse(const T (&A)[NS][NS], T (&X)[NS][NS]) {
  if constexpr (NS == 1) {
    X[0][0] = T(1) / A[0][0];
  } else if constexpr (NS == 2) {
    T det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    T r = recip<T>(det);
    X[0][0] = A[1][1] * r;
    X[0][1] = -A[0][1] * r;
    X[1][0] = -A[1][0] * r;
    X[1][1] = A[0][0] * r;
  } else {
    T W[NS][NS];
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        W[i][j] = A[i][j];
        X[i][j] = (i == j) ? T(1) : T(0);
      }
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      // pivot: largest |W[r][k]|, r >= k
      int piv = k;
      T best = fabs(W[k][k]);
#pragma unroll
      for (int r = k + 1; r < NS; ++r) {
        T a = fabs(W[r][k]);
        if (a > best) {
          best = a;
          piv = r;
        }
      }
#pragma unroll
      for (int r = k + 1; r < NS; ++r) {
        if (r == piv) {
#pragma unroll
          for (int j = 0; j < NS; ++j) {
            T t = W[k][j];
            W[k][j] = W[r][j];
            W[r][j] = t;
            t = X[k][j];
            X[k][j] = X[r][j];
            X[r][j] = t;
          }
        }
      }
      T inv = recip<T>(W[k][k]);
#pragma unroll
      for (int j = 0; j < NS; ++j) {
        W[k][j] *= inv;
        X[k][j] *= inv;
      }
#pragma unroll
      for (int r = 0; r < NS; ++r) {
        if (r == k) continue;
        T f = W[r][k];
#pragma unroll
        for (int j = 0; j < NS; ++j) {
          W[r][j] = fma(-f, W[k][j], W[r][j]);
          X[r][j] = fma(-f, X[k][j], X[r][j]);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 <-> FP32 conversions on the integer pipe.  GB300 executes FP64 at 1/64
// of the FP32 rate, so the mixed-precision path keeps format conversions off
// the FP64 unit by rebuilding the IEEE-754 fields directly:
//   binary64: sign | 11-bit exponent (bias 1023) | 52-bit fraction
//   binary32: sign |  8-bit exponent (bias  127) | 23-bit fraction
// to_f32_trunc rounds toward zero (drops the low 29 fraction bits); values
// below the normal binary32 range become signed zero, above it signed
// infinity; NaN stays NaN.  to_f64 is exact for normal floats and maps
// subnormal floats to signed zero.  Both feed only FP32 work -- the block
// algebra of an inexact Newton iteration, whose FP64 residual decides
// convergence, and the FP32 passes of the mixed-precision adjoint.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float to_f32_trunc(double x) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(x));
  const unsigned hi = static_cast<unsigned>(u >> 32), lo = static_cast<unsigned>(u);
  const unsigned sign = hi & 0x80000000u;
  const unsigned ebits = (hi >> 20) & 0x7ffu;
  const int e = static_cast<int>(ebits) - 1023 + 127;
  const unsigned frac = ((hi & 0x000fffffu) << 3) | (lo >> 29);
  unsigned bits;
  if (ebits == 0x7ffu)
    bits = sign | 0x7f800000u | (((hi & 0x000fffffu) | lo) ? 0x00400000u : 0u);  // Inf / NaN
  else if (e >= 255)
    bits = sign | 0x7f800000u;  // overflow
  else if (e <= 0)
    bits = sign;  // below the normal range
  else
    bits = sign | (static_cast<unsigned>(e) << 23) | frac;
  return __uint_as_float(bits);
}

__device__ __forceinline__ double to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xffu;
  const unsigned m = b & 0x007fffffu;
  unsigned hi, lo;
  if (e == 0u) {
    hi = sign;
    lo = 0u;
  } else if (e == 0xffu) {
    hi = sign | 0x7ff00000u | (m >> 3);
    lo = m << 29;
  } else {
    hi = sign | ((e + (1023u - 127u)) << 20) | (m >> 3);
    lo = m << 29;
  }
  return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

template <typename T>
__device__ __forceinline__ T narrow(double x) {
  if constexpr (sizeof(T) == sizeof(double)) return x;
  else return to_f32_trunc(x);
}

template <typename T>
__device__ __forceinline__ double widen(T x) {
  if constexpr (sizeof(T) == sizeof(double)) return x;
  else return to_f64(x);
}

// ---------------------------------------------------------------------------
// Infinity-norm helpers on the bit pattern: for x >= 0 the IEEE-754 ordering of
// doubles equals the unsigned ordering of their bits, and any NaN/Inf compares
// >= kNonFiniteBits, so max-reductions run on the integer pipe.
// ---------------------------------------------------------------------------
constexpr unsigned long long kNonFiniteBits = 0x7ff0000000000000ull;

__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return static_cast<unsigned long long>(__double_as_longlong(x)) & 0x7fffffffffffffffull;
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
  return a > b ? a : b;
}

// Barrier over the first `nthreads` threads of the block (whole warps).  The
// whole block uses barrier 0 (__syncthreads); a leading subset of its warps uses
// named barrier 1, so warps without work need not take part.
__device__ __forceinline__ void sync_first(int nthreads) {
  if (nthreads == static_cast<int>(blockDim.x))
    __syncthreads();
  else
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Max of a 32-bit unsigned value over the warp (one redux.sync instruction).
__device__ __forceinline__ unsigned warp_max_u32(unsigned v) {
  unsigned r;
  asm volatile("redux.sync.max.u32 %0, %1, 0xffffffff;" : "=r"(r) : "r"(v));
  return r;
}

// Exact 64-bit max over the warp: the largest high word, then the largest low
// word among the lanes that hold it.
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
  const unsigned hi = static_cast<unsigned>(v >> 32), lo = static_cast<unsigned>(v);
  const unsigned mh = warp_max_u32(hi);
  const unsigned ml = warp_max_u32(hi == mh ? lo : 0u);
  return (static_cast<unsigned long long>(mh) << 32) | ml;
}

// Max over the `nwa` warps that call it (the block's first nwa warps).  The
// caller guarantees a barrier between two consecutive calls (s_red is reused).
__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v,
                                                            unsigned long long* s_red, int lane,
                                                            int warp, int nwa) {
  v = warp_max_u64(v);
  if (nwa == 1) return v;  // one warp: no barrier needed
  if (lane == 0) s_red[warp] = v;
  sync_first(32 * nwa);
  unsigned long long r = s_red[0];
  for (int w = 1; w < nwa; ++w) r = umax64(r, s_red[w]);
  return r;
}

// The last of a thread's first `rpa` rows (1 <= rpa <= RPT), without a dynamic
// register index.
template <int RPT, int NS>
__device__ __forceinline__ void last_row(const double (&v)[RPT][NS], int rpa, double (&out)[NS]) {
#pragma unroll
  for (int s = 0; s < NS; ++s) out[s] = v[RPT - 1][s];
#pragma unroll
  for (int r = 0; r < RPT - 1; ++r)
    if (r == rpa - 1)
#pragma unroll
      for (int s = 0; s < NS; ++s) out[s] = v[r][s];
}

// ---------------------------------------------------------------------------
// Solve the chain d_j = M_j d_{j-1} + v_j over the block's rows, d_{-1} = 0.
// Called by the block's first `nwa` warps only; thread t holds its rows in
// f[0 .. rpa-1] (rpa <= RPT, the same in every thread), and rows past the
// chunk end must hold the identity map.  Lanes from `lanes` on (in every warp)
// must hold identity maps only.  On return x[r] = d of each own row r < rpa.
// Synchronisation: two barriers over those warps when nwa > 1.
// ---------------------------------------------------------------------------
template <int NS, typename T, int RPT>
__device__ __forceinline__ void solve_chain(const Aff<NS, T> (&f)[RPT], T (&x)[RPT][NS],
                                            Aff<NS, T>* s_wtot, int lane, int warp, int nwa,
                                            int rpa = RPT, int lanes = 32) {
  // (1) serial composition of the thread's own rows
  Aff<NS, T> seg = f[0];
#pragma unroll
  for (int r = 1; r < RPT; ++r)
    if (r < rpa) seg = compose(f[r], seg);
  // (2) cyclic reduction over the lanes of the warp; `lanes` (block-uniform) is
  // how many lanes of a warp hold rows, so a short chunk takes fewer levels
  for (int s = 1; s < lanes; s <<= 1) {
    Aff<NS, T> o = shfl_up_aff(seg, s);
    if (lane >= s) seg = compose(seg, o);
  }
  // (3) cyclic reduction over the warps; vin = d at the end of the previous thread
  T vin[NS];
  if (nwa > 1) {
    if (lane == 31) s_wtot[warp] = seg;
    sync_first(32 * nwa);
    if (warp == 0) {
      Aff<NS, T> w;
      if (lane < nwa)
        w = s_wtot[lane];
      else
        aff_identity(w);
      for (int s = 1; s < nwa; s <<= 1) {
        Aff<NS, T> o = shfl_up_aff(w, s);
        if (lane >= s) w = compose(w, o);
      }
      if (lane < nwa) {
#pragma unroll
        for (int i = 0; i < NS; ++i) s_wtot[lane].v[i] = w.v[i];
      }
    }
    sync_first(32 * nwa);
    T vex[NS], vfull[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) vex[i] = (warp > 0) ? s_wtot[warp - 1].v[i] : T(0);
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      T s = seg.v[i];
#pragma unroll
      for (int k = 0; k < NS; ++k) s = fma(seg.M[i][k], vex[k], s);
      vfull[i] = s;
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      T u = __shfl_up_sync(kFull, vfull[i], 1);
      vin[i] = (lane == 0) ? vex[i] : u;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      T u = __shfl_up_sync(kFull, seg.v[i], 1);
      vin[i] = (lane == 0) ? T(0) : u;
    }
  }
  // (4) fix-up: substitute forward through the own rows
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    if (r >= rpa) break;  // the same in every thread
    T xn[NS];
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      T s = f[r].v[i];
#pragma unroll
      for (int k = 0; k < NS; ++k) s = fma(f[r].M[i][k], vin[k], s);
      xn[i] = s;
    }
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      x[r][i] = xn[i];
      vin[i] = xn[i];
    }
  }
}

}  // namespace tvi
