// tvi_models.cuh -- right-hand sides h(y, t; p) of the small-state models, their
// step Jacobians A = I - dt dh/dy (Sec. 2.2, discrete Jacobian) and parameter
// vector-Jacobian products (dh/dp)^T a (App. A.1, gradient integrand).
//
// Every model provides
//   NS, NP                         state size, parameters per vector
//   load(params, b, per_series)    fetch the series' parameters into registers
//   rhs(y, t, h)                   FP64 h(y, t)                (residual: always FP64)
//   step_matrix<T>(y, t, dt, A)    A = I - dt j(y, t) in T     (block: FP32 or FP64)
//   vjp_p(y, t, a, scale, acc)     acc[NP] += scale (dh/dp)^T a at (y, t)   (FP64)
// The models here are autonomous (kUsesTime = false: the kernels then pass t =
// 0 without loading it); run-time compiled user models use it.
#pragma once

#include <cuda_runtime.h>

namespace tvi {

// van der Pol: h = [y2, mu (1 - y1^2) y2 - y1],  p = [mu].
struct ModelVdp {
  static constexpr int NS = 2;
  static constexpr int NP = 1;
  static constexpr bool kPredictable = true;  // learned Newton predictor available
  static constexpr bool kUsesTime = false;
  double mu;
  // predictor feature of the parameter
  __device__ __forceinline__ float param_feature() const { return log10f(static_cast<float>(mu)); }

  __device__ __forceinline__ void load(const double* params, int b, int per_series) {
    mu = params[per_series ? b : 0];
  }
  __device__ __forceinline__ void rhs(const double (&y)[2], double, double (&h)[2]) const {
    h[0] = y[1];
    h[1] = fma(mu * fma(-y[0], y[0], 1.0), y[1], -y[0]);
  }
  // j = [[0, 1], [-2 mu y1 y2 - 1, mu (1 - y1^2)]]
  template <typename T>
  __device__ __forceinline__ void step_matrix(const T (&y)[2], double, T dt, T (&A)[2][2]) const {
    T m = static_cast<T>(mu);
    A[0][0] = T(1);
    A[0][1] = -dt;
    A[1][0] = dt * fma(T(2) * m * y[0], y[1], T(1));
    A[1][1] = fma(-dt * m, fma(-y[0], y[0], T(1)), T(1));
  }
  // dh/dmu = [0, (1 - y1^2) y2]
  __device__ __forceinline__ void vjp_p(const double (&y)[2], double, const double (&a)[2],
                                        double scale, double (&acc)[NP]) const {
    acc[0] = fma(scale * a[1], fma(-y[0], y[0], 1.0) * y[1], acc[0]);
  }
};

// Linear: h = A y, p = A (row-major n x n).
template <int N_>
struct ModelLinear {
  static constexpr int NS = N_;
  static constexpr int NP = N_ * N_;
  static constexpr bool kPredictable = false;
  static constexpr bool kUsesTime = false;
  double A[N_][N_];
  __device__ __forceinline__ float param_feature() const { return 0.0f; }

  __device__ __forceinline__ void load(const double* params, int b, int per_series) {
    const double* p = params + (per_series ? static_cast<size_t>(b) * NP : 0);
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
      for (int j = 0; j < NS; ++j) A[i][j] = p[i * NS + j];
  }
  __device__ __forceinline__ void rhs(const double (&y)[N_], double, double (&h)[N_]) const {
#pragma unroll
    for (int i = 0; i < NS; ++i) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < NS; ++j) s = fma(A[i][j], y[j], s);
      h[i] = s;
    }
  }
  template <typename T>
  __device__ __forceinline__ void step_matrix(const T (&y)[N_], double, T dt,
                                              T (&M)[N_][N_]) const {
    (void)y;
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
      for (int j = 0; j < NS; ++j)
        M[i][j] = fma(-dt, static_cast<T>(A[i][j]), (i == j) ? T(1) : T(0));
  }
  // dh_i/dA_ij = y_j  =>  (dh/dA)^T a = a y^T
  __device__ __forceinline__ void vjp_p(const double (&y)[N_], double, const double (&a)[N_],
                                        double scale, double (&acc)[NP]) const {
#pragma unroll
    for (int i = 0; i < NS; ++i)
#pragma unroll
      for (int j = 0; j < NS; ++j) acc[i * NS + j] = fma(scale * a[i], y[j], acc[i * NS + j]);
  }
};

}  // namespace tvi
