"""Example user models: CUDA C++ device source for tvi_user_model_create
(UserModel), each defining tvi_rhs, tvi_jac and tvi_vjp_p over FP64 pointers.

    VDP          van der Pol, h = [y2, mu (1 - y1^2) y2 - y1], p = [mu]   (n 2, P 1)
                 (tvi_jac a template: FP32 Jacobians with FP32 blocks)
    VDP_FP64_JAC the same with an FP64 tvi_jac
    LINEAR       h = A y, p = A row-major                                (any n, P n^2)
    mlp_tanh()   h = tanh(W3 tanh(W2 tanh(W1 y + b1) + b2) + b3)         (any n)

    import paper_2310_08649_gb300 as tvi
    from paper_2310_08649_gb300.user_sources import VDP
    model = tvi.UserModel(2, 1, VDP).model(per_series=True)
"""

VDP = r"""
// van der Pol: h = [y2, mu (1 - y1^2) y2 - y1], p = [mu]
__device__ void tvi_rhs(const double* y, const double* p, double* h) {
  h[0] = y[1];
  h[1] = p[0] * (1.0 - y[0] * y[0]) * y[1] - y[0];
}
// the Jacobian as a template: evaluated in FP32 with FP32 blocks
template <typename T>
__device__ void tvi_jac(const T* y, const double* p, T* J) {
  const T mu = static_cast<T>(p[0]);
  J[0] = T(0);
  J[1] = T(1);
  J[2] = -T(2) * mu * y[0] * y[1] - T(1);
  J[3] = mu * (T(1) - y[0] * y[0]);
}
__device__ void tvi_vjp_p(const double* y, const double* p, const double* a, double* g) {
  g[0] = a[1] * (1.0 - y[0] * y[0]) * y[1];
}
"""

# van der Pol with a plain FP64 Jacobian (rounded to the block type after evaluation)
VDP_FP64_JAC = VDP[:VDP.index("// the Jacobian as a template")] + r"""__device__ void tvi_jac(const double* y, const double* p, double* J) {
  J[0] = 0.0;
  J[1] = 1.0;
  J[2] = -2.0 * p[0] * y[0] * y[1] - 1.0;
  J[3] = p[0] * (1.0 - y[0] * y[0]);
}
""" + VDP[VDP.index("__device__ void tvi_vjp_p"):]

LINEAR = r"""
// h = A y with A = p as a row-major TVI_N x TVI_N matrix
__device__ void tvi_rhs(const double* y, const double* p, double* h) {
  for (int i = 0; i < TVI_N; ++i) {
    double s = 0.0;
    for (int j = 0; j < TVI_N; ++j) s += p[i * TVI_N + j] * y[j];
    h[i] = s;
  }
}
__device__ void tvi_jac(const double* y, const double* p, double* J) {
  for (int k = 0; k < TVI_N * TVI_N; ++k) J[k] = p[k];
}
__device__ void tvi_vjp_p(const double* y, const double* p, const double* a, double* g) {
  for (int i = 0; i < TVI_N; ++i)
    for (int j = 0; j < TVI_N; ++j) g[i * TVI_N + j] = a[i] * y[j];
}
"""


def mlp_tanh(h1, h2):
    """h = tanh(W3 tanh(W2 tanh(W1 y + b1) + b2) + b3), parameters packed
    W1[h1][n] b1[h1] W2[h2][h1] b2[h2] W3[n][h2] b3[n]."""
    return f"#define H1 {h1}\n#define H2 {h2}\n" + r"""
struct MlpState { double a1[H1], a2[H2], h[TVI_N]; };

__device__ void mlp_eval(const double* y, const double* p, MlpState& s) {
  const double* W1 = p;
  const double* b1 = W1 + H1 * TVI_N;
  const double* W2 = b1 + H1;
  const double* b2 = W2 + H2 * H1;
  const double* W3 = b2 + H2;
  const double* b3 = W3 + TVI_N * H2;
  for (int r = 0; r < H1; ++r) {
    double z = b1[r];
    for (int c = 0; c < TVI_N; ++c) z += W1[r * TVI_N + c] * y[c];
    s.a1[r] = tanh(z);
  }
  for (int r = 0; r < H2; ++r) {
    double z = b2[r];
    for (int c = 0; c < H1; ++c) z += W2[r * H1 + c] * s.a1[c];
    s.a2[r] = tanh(z);
  }
  for (int r = 0; r < TVI_N; ++r) {
    double z = b3[r];
    for (int c = 0; c < H2; ++c) z += W3[r * H2 + c] * s.a2[c];
    s.h[r] = tanh(z);
  }
}

__device__ void tvi_rhs(const double* y, const double* p, double* h) {
  MlpState s;
  mlp_eval(y, p, s);
  for (int i = 0; i < TVI_N; ++i) h[i] = s.h[i];
}

// row i of J = d3_i W3[i,:] D2 W2 D1 W1
__device__ void tvi_jac(const double* y, const double* p, double* J) {
  const double* W1 = p;
  const double* W2 = W1 + H1 * TVI_N + H1;
  const double* W3 = W2 + H2 * H1 + H2;
  MlpState s;
  mlp_eval(y, p, s);
  for (int i = 0; i < TVI_N; ++i) {
    double u[H2], v[H1];
    for (int c = 0; c < H2; ++c)
      u[c] = (1.0 - s.h[i] * s.h[i]) * W3[i * H2 + c] * (1.0 - s.a2[c] * s.a2[c]);
    for (int c = 0; c < H1; ++c) {
      double t = 0.0;
      for (int r = 0; r < H2; ++r) t += u[r] * W2[r * H1 + c];
      v[c] = t * (1.0 - s.a1[c] * s.a1[c]);
    }
    for (int j = 0; j < TVI_N; ++j) {
      double t = 0.0;
      for (int c = 0; c < H1; ++c) t += v[c] * W1[c * TVI_N + j];
      J[i * TVI_N + j] = t;
    }
  }
}

// back-propagation of a through the three layers
__device__ void tvi_vjp_p(const double* y, const double* p, const double* a, double* g) {
  const double* W2 = p + H1 * TVI_N + H1;
  const double* W3 = W2 + H2 * H1 + H2;
  double* gW1 = g;
  double* gb1 = gW1 + H1 * TVI_N;
  double* gW2 = gb1 + H1;
  double* gb2 = gW2 + H2 * H1;
  double* gW3 = gb2 + H2;
  double* gb3 = gW3 + TVI_N * H2;
  MlpState s;
  mlp_eval(y, p, s);
  double e3[TVI_N], e2[H2], e1[H1];
  for (int i = 0; i < TVI_N; ++i) {
    e3[i] = a[i] * (1.0 - s.h[i] * s.h[i]);
    gb3[i] = e3[i];
    for (int c = 0; c < H2; ++c) gW3[i * H2 + c] = e3[i] * s.a2[c];
  }
  for (int c = 0; c < H2; ++c) {
    double t = 0.0;
    for (int i = 0; i < TVI_N; ++i) t += e3[i] * W3[i * H2 + c];
    e2[c] = t * (1.0 - s.a2[c] * s.a2[c]);
    gb2[c] = e2[c];
    for (int k = 0; k < H1; ++k) gW2[c * H1 + k] = e2[c] * s.a1[k];
  }
  for (int k = 0; k < H1; ++k) {
    double t = 0.0;
    for (int c = 0; c < H2; ++c) t += e2[c] * W2[c * H1 + k];
    e1[k] = t * (1.0 - s.a1[k] * s.a1[k]);
    gb1[k] = e1[k];
    for (int j = 0; j < TVI_N; ++j) gW1[k * TVI_N + j] = e1[k] * y[j];
  }
}
"""


def mlp_param_count(n, h1, h2):
    return h1 * n + h1 + h2 * h1 + h2 + n * h2 + n
