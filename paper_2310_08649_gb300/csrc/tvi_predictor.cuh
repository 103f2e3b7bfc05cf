// tvi_predictor.cuh -- the learned Newton predictor: an MLP that maps the state
// at a chunk start, the model parameter and the chunk's step sizes to a guess of
// the whole chunk's increments dy_1..dy_c, used as Newton's starting point in
// place of dy = 0 (Sec. 2.3) when its FP64 residual is smaller.
//
// Packed FP32 layout (in = features, H = hidden width, out = outputs):
//   mean[in] std[in] scale[out] W1[H][in] b1[H] W2[H][H] b2[H] W3[out][H] b3[out]
// Features are normalised as (x - mean) / std; the network predicts the
// chunk's per-step slopes s_j / scale (dy_j = sum_{l <= j} dt_l s_l is the guess,
// formed by the caller); hidden layers use SiLU, the output layer is linear.
#pragma once

#ifndef __CUDACC_RTC__  // host compile (NVRTC provides the device built-ins)
#include <cuda_runtime.h>
#endif

namespace tvi {

struct PredDims {
  int in, hid, out;
};

struct PredOffsets {
  int mean, stdv, scale, W1, b1, W2, b2, W3, b3, total, train_begin;
};

__host__ __device__ inline PredOffsets pred_offsets(const PredDims& d) {
  PredOffsets o;
  o.mean = 0;
  o.stdv = o.mean + d.in;
  o.scale = o.stdv + d.in;
  o.W1 = o.scale + d.out;
  o.b1 = o.W1 + d.hid * d.in;
  o.W2 = o.b1 + d.hid;
  o.b2 = o.W2 + d.hid * d.hid;
  o.W3 = o.b2 + d.hid;
  o.b3 = o.W3 + d.out * d.hid;
  o.total = o.b3 + d.out;
  o.train_begin = o.W1;  // W1 .. b3 are trained; mean/std/scale are set from data
  return o;
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One dense layer for one sample, warp per output row: lanes stride the row
// (coalesced weight reads), four rows in flight per warp, the loads of up to
// 256 columns issued before their FMAs (the weights stream from L2, so the
// loop is bound by how many loads are in flight), then a butterfly sum.
// dst[u] = act(sum_k W[u][k] src[k] + bias[u]) (* mul[u] when mul != nullptr).
template <bool kSilu>
__device__ __forceinline__ void pred_layer(const float* __restrict__ W, const float* __restrict__ bias,
                                           const float* __restrict__ mul, int rows, int cols,
                                           const float* src, float* dst) {
  constexpr int kRows = 4, kSpan = 8;  // rows per pass, 32-column groups per batch of loads
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int u0 = (threadIdx.x >> 5) * kRows; u0 < rows; u0 += nw * kRows) {
    float acc[kRows];
#pragma unroll
    for (int q = 0; q < kRows; ++q) acc[q] = 0.0f;
    for (int k0 = 0; k0 < cols; k0 += 32 * kSpan) {
      float wv[kRows][kSpan];
#pragma unroll
      for (int q = 0; q < kRows; ++q)
#pragma unroll
        for (int g = 0; g < kSpan; ++g) {
          const int k = k0 + 32 * g + lane;
          wv[q][g] = (u0 + q < rows && k < cols)
                         ? __ldg(W + static_cast<size_t>(u0 + q) * cols + k)
                         : 0.0f;
        }
#pragma unroll
      for (int g = 0; g < kSpan; ++g) {
        const int k = k0 + 32 * g + lane;
        const float x = k < cols ? src[k] : 0.0f;
#pragma unroll
        for (int q = 0; q < kRows; ++q) acc[q] = fmaf(wv[q][g], x, acc[q]);
      }
    }
#pragma unroll
    for (int q = 0; q < kRows; ++q) acc[q] = warp_sum_f(acc[q]);
    if (lane < kRows && u0 + lane < rows) {
      const int u = u0 + lane;
      float z = bias[u];
#pragma unroll
      for (int q = 0; q < kRows; ++q)
        if (q == lane) z += acc[q];
      if (kSilu) z = silu_f(z);
      if (mul) z *= mul[u];
      dst[u] = z;
    }
  }
}

// Block-cooperative inference of one sample: feat[in] (raw features, shared
// memory) -> outv[out] (physical units, shared memory).  h1, h2: shared scratch
// of H floats each.  All threads of the block must call it; blockDim.x is a
// multiple of 32.
__device__ __forceinline__ void pred_infer_block(const float* __restrict__ w, const PredDims& d,
                                                 float* feat, float* h1, float* h2, float* outv) {
  const PredOffsets o = pred_offsets(d);
  for (int k = threadIdx.x; k < d.in; k += blockDim.x)
    feat[k] = (feat[k] - __ldg(w + o.mean + k)) / __ldg(w + o.stdv + k);
  __syncthreads();
  pred_layer<true>(w + o.W1, w + o.b1, nullptr, d.hid, d.in, feat, h1);
  __syncthreads();
  pred_layer<true>(w + o.W2, w + o.b2, nullptr, d.hid, d.hid, h1, h2);
  __syncthreads();
  pred_layer<false>(w + o.W3, w + o.b3, w + o.scale, d.out, d.hid, h2, outv);
  __syncthreads();
}

}  // namespace tvi
