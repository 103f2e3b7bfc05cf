// tvi_predictor.cu -- inference and training kernels of the learned Newton
// predictor (packed layout in tvi_predictor.cuh), behind the C ABI.
//
// Training step on a batch of M samples (x raw features, t targets in physical
// units), loss = mean over the batch and outputs of (o - t / scale)^2:
//   xn = (x - mean) / std
//   Z1 = xn W1^T + b1, H1 = silu(Z1); Z2 = H1 W2^T + b2, H2 = silu(Z2);
//   O  = H2 W3^T + b3
//   dO = 2 (O - t / scale) / (M out)
//   dW3 = dO^T H2, db3 = colsum dO; dH2 = dO W3, dZ2 = dH2 silu'(Z2)
//   dW2 = dZ2^T H1, db2; dZ1 = (dZ2 W2) silu'(Z1); dW1 = dZ1^T xn, db1
//   Adam (Kingma & Ba, 2015) on W1..b3 with bias-corrected moments.
// The products run in one strided, tiled FP32 GEMM kernel (64 x 64 tiles,
// 4 x 4 outputs per thread) whose operands may be transposed views.
#include <cuda_runtime.h>

#include "tvi.h"
#include "tvi_internal.h"
#include "tvi_predictor.cuh"

namespace tvi {
namespace {

// C[i][j] = sum_k A(i,k) B(k,j) (+ bias[j]); A(i,k) = A[i*sai + k*sak],
// B(k,j) = B[k*sbk + j*sbj], C row-major with leading dimension N.
// act = 1: Z = C (+bias) is stored to C and H = silu(Z) to H.
__global__ void __launch_bounds__(256) sgemm_kernel(int M, int N, int K, const float* A, int sai,
                                                    int sak, const float* B, int sbk, int sbj,
                                                    const float* bias, float* C, float* H,
                                                    int act) {
  __shared__ float sA[16][64 + 1];
  __shared__ float sB[16][64 + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int e = threadIdx.x; e < 64 * 16; e += 256) {
      const int ii = e / 16, kk = e % 16;
      const int i = i0 + ii, k = k0 + kk;
      sA[kk][ii] = (i < M && k < K) ? A[static_cast<size_t>(i) * sai + static_cast<size_t>(k) * sak]
                                    : 0.0f;
      const int jj = e % 64, kb = e / 64;
      const int j = j0 + jj, k2 = k0 + kb;
      sB[kb][jj] = (j < N && k2 < K) ? B[static_cast<size_t>(k2) * sbk + static_cast<size_t>(j) * sbj]
                                     : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = sA[kk][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = sB[kk][tx * 4 + c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty * 4 + r;
    if (i >= M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx * 4 + c;
      if (j >= N) continue;
      float z = acc[r][c] + (bias ? bias[j] : 0.0f);
      C[static_cast<size_t>(i) * N + j] = z;
      if (act) H[static_cast<size_t>(i) * N + j] = silu_f(z);
    }
  }
}

void sgemm(int M, int N, int K, const float* A, int sai, int sak, const float* B, int sbk, int sbj,
           const float* bias, float* C, float* H, int act, cudaStream_t s) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  note_launch();
  sgemm_kernel<<<grid, 256, 0, s>>>(M, N, K, A, sai, sak, B, sbk, sbj, bias, C, H, act);
}

// Batch assembly: sample m of the batch is row rows[m] (or m) of x and t.
__global__ void normalize_kernel(int M, int in, int out, const float* w, PredOffsets o,
                                 const float* x, const float* t, const int* rows, float* xn,
                                 float* tn) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < M * in) {
    const int m = e / in, k = e % in;
    const size_t src = static_cast<size_t>(rows ? rows[m] : m) * in + k;
    xn[e] = (x[src] - w[o.mean + k]) / w[o.stdv + k];
  }
  if (e < M * out) {
    const int m = e / out, u = e % out;
    const size_t src = static_cast<size_t>(rows ? rows[m] : m) * out + u;
    tn[e] = t[src] / w[o.scale + u];
  }
}

// dO = 2 (O - tn) / (M out); per-block partial of the squared error
__global__ void mse_grad_kernel(int count, const float* O, const float* tn, float* dO,
                                float* partial) {
  __shared__ float red[256];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  float sq = 0.0f;
  if (e < count) {
    const float diff = O[e] - tn[e];
    dO[e] = 2.0f * diff / static_cast<float>(count);
    sq = diff * diff;
  }
  red[threadIdx.x] = sq;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

__global__ void loss_reduce_kernel(int nb, int count, const float* partial, float* loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[b];
    *loss = static_cast<float>(s / count);
  }
}

// dZ = dH * silu'(Z), silu'(z) = s + z s (1 - s), s = sigmoid(z)
__global__ void silu_backward_kernel(int count, const float* Z, const float* dH, float* dZ) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const float z = Z[e];
  const float s = 1.0f / (1.0f + __expf(-z));
  dZ[e] = dH[e] * (s + z * s * (1.0f - s));
}

// db[j] = sum over rows of D[m][j], rows in order
__global__ void colsum_kernel(int M, int N, const float* D, float* db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.0f;
  for (int m = 0; m < M; ++m) s += D[static_cast<size_t>(m) * N + j];
  db[j] = s;
}

__global__ void adam_kernel(int count, float* p, const float* g, float* m, float* v, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const float gi = g[e];
  const float mi = b1 * m[e] + (1.0f - b1) * gi;
  const float vi = b2 * v[e] + (1.0f - b2) * gi * gi;
  m[e] = mi;
  v[e] = vi;
  p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void infer_kernel(const float* w, PredDims d, const float* x, float* y) {
  extern __shared__ float sm[];
  float* feat = sm;
  float* h1 = feat + d.in;
  float* h2 = h1 + d.hid;
  float* outv = h2 + d.hid;
  const int m = blockIdx.x;
  for (int k = threadIdx.x; k < d.in; k += blockDim.x) feat[k] = x[static_cast<size_t>(m) * d.in + k];
  __syncthreads();
  pred_infer_block(w, d, feat, h1, h2, outv);
  for (int u = threadIdx.x; u < d.out; u += blockDim.x) y[static_cast<size_t>(m) * d.out + u] = outv[u];
}

size_t al(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

struct TrainWs {
  float *xn, *tn, *Z1, *H1, *Z2, *H2, *O, *dO, *dH, *dZ, *g, *partial;
  size_t total;
};

TrainWs carve_train(char* base, const PredDims& d, int M) {
  TrainWs w{};
  size_t off = 0;
  auto take = [&](size_t n) {
    float* p = base ? reinterpret_cast<float*>(base + off) : nullptr;
    off += al(n * sizeof(float));
    return p;
  };
  const PredOffsets o = pred_offsets(d);
  w.xn = take(static_cast<size_t>(M) * d.in);
  w.tn = take(static_cast<size_t>(M) * d.out);
  w.Z1 = take(static_cast<size_t>(M) * d.hid);
  w.H1 = take(static_cast<size_t>(M) * d.hid);
  w.Z2 = take(static_cast<size_t>(M) * d.hid);
  w.H2 = take(static_cast<size_t>(M) * d.hid);
  w.O = take(static_cast<size_t>(M) * d.out);
  w.dO = take(static_cast<size_t>(M) * d.out);
  w.dH = take(static_cast<size_t>(M) * d.hid);
  w.dZ = take(static_cast<size_t>(M) * d.hid);
  w.g = take(static_cast<size_t>(o.total - o.train_begin));
  w.partial = take(static_cast<size_t>((M * d.out + 255) / 256) + 1);
  w.total = off;
  return w;
}

bool dims_ok(int in, int hid, int out) {
  return in >= 1 && out >= 1 && hid >= 2 && hid % 2 == 0 && hid <= 1024 && in <= 4096 &&
         out <= 4096;
}

}  // namespace
}  // namespace tvi

extern "C" {

int tvi_predictor_size(int in, int hidden, int out) {
  if (!tvi::dims_ok(in, hidden, out)) return -1;
  return tvi::pred_offsets(tvi::PredDims{in, hidden, out}).total;
}

size_t tvi_predictor_workspace_bytes(int in, int hidden, int out, int M) {
  if (!tvi::dims_ok(in, hidden, out) || M < 1) return 0;
  return tvi::carve_train(nullptr, tvi::PredDims{in, hidden, out}, M).total;
}

tvi_status tvi_predictor_forward(const float* packed, int in, int hidden, int out, int M,
                                 const float* x, float* y, void* stream) {
  if (!tvi::dims_ok(in, hidden, out) || M < 0 || (M > 0 && (!packed || !x || !y)))
    return TVI_EINVAL;
  if (M == 0) return TVI_OK;
  const tvi::PredDims d{in, hidden, out};
  const size_t sm = sizeof(float) * (in + 2 * hidden + out);
  if (sm > 48 * 1024) return TVI_EUNSUPPORTED;
  tvi::note_launch();
  tvi::infer_kernel<<<M, 256, sm, static_cast<cudaStream_t>(stream)>>>(packed, d, x, y);
  return cudaGetLastError() == cudaSuccess ? TVI_OK : TVI_ECUDA;
}

tvi_status tvi_predictor_train_step(float* packed, float* adam_m, float* adam_v, int in, int hidden,
                                    int out, int M, const float* x, const float* target,
                                    const int* rows, float lr, int step, float* loss,
                                    void* workspace, size_t workspace_bytes, void* stream) {
  using namespace tvi;
  if (!dims_ok(in, hidden, out) || M < 1 || step < 1 || !packed || !adam_m || !adam_v || !x ||
      !target || !loss)
    return TVI_EINVAL;
  const PredDims d{in, hidden, out};
  TrainWs w = carve_train(static_cast<char*>(workspace), d, M);
  if (!workspace || workspace_bytes < w.total) return TVI_EWORKSPACE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const PredOffsets o = pred_offsets(d);
  const int H = hidden;
  note_launch();
  normalize_kernel<<<(M * (in > out ? in : out) + 255) / 256, 256, 0, s>>>(M, in, out, packed, o, x,
                                                                          target, rows, w.xn, w.tn);
  // forward
  sgemm(M, H, in, w.xn, in, 1, packed + o.W1, 1, in, packed + o.b1, w.Z1, w.H1, 1, s);
  sgemm(M, H, H, w.H1, H, 1, packed + o.W2, 1, H, packed + o.b2, w.Z2, w.H2, 1, s);
  sgemm(M, out, H, w.H2, H, 1, packed + o.W3, 1, H, packed + o.b3, w.O, nullptr, 0, s);
  const int cnt = M * out, nb = (cnt + 255) / 256;
  note_launch();
  mse_grad_kernel<<<nb, 256, 0, s>>>(cnt, w.O, w.tn, w.dO, w.partial);
  note_launch();
  loss_reduce_kernel<<<1, 32, 0, s>>>(nb, cnt, w.partial, loss);
  // backward (gradients in the packed order W1 b1 W2 b2 W3 b3, offset by train_begin)
  float* g = w.g;
  auto G = [&](int off) { return g + (off - o.train_begin); };
  sgemm(out, H, M, w.dO, 1, out, w.H2, H, 1, nullptr, G(o.W3), nullptr, 0, s);
  note_launch();
  colsum_kernel<<<(out + 127) / 128, 128, 0, s>>>(M, out, w.dO, G(o.b3));
  sgemm(M, H, out, w.dO, out, 1, packed + o.W3, H, 1, nullptr, w.dH, nullptr, 0, s);
  note_launch();
  silu_backward_kernel<<<(M * H + 255) / 256, 256, 0, s>>>(M * H, w.Z2, w.dH, w.dZ);
  sgemm(H, H, M, w.dZ, 1, H, w.H1, H, 1, nullptr, G(o.W2), nullptr, 0, s);
  note_launch();
  colsum_kernel<<<(H + 127) / 128, 128, 0, s>>>(M, H, w.dZ, G(o.b2));
  sgemm(M, H, H, w.dZ, H, 1, packed + o.W2, H, 1, nullptr, w.dH, nullptr, 0, s);
  note_launch();
  silu_backward_kernel<<<(M * H + 255) / 256, 256, 0, s>>>(M * H, w.Z1, w.dH, w.dZ);
  sgemm(H, in, M, w.dZ, 1, H, w.xn, in, 1, nullptr, G(o.W1), nullptr, 0, s);
  note_launch();
  colsum_kernel<<<(H + 127) / 128, 128, 0, s>>>(M, H, w.dZ, G(o.b1));
  // Adam
  const int np = o.total - o.train_begin;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f - powf(b1, static_cast<float>(step));
  const float c2 = 1.0f - powf(b2, static_cast<float>(step));
  note_launch();
  adam_kernel<<<(np + 255) / 256, 256, 0, s>>>(np, packed + o.train_begin, g, adam_m, adam_v, lr, b1,
                                              b2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? TVI_OK : TVI_ECUDA;
}

}  // extern "C"
