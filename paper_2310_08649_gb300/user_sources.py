"""Example user models: CUDA C++ device source for tvi_user_model_create
(UserModel), each defining tvi_rhs, tvi_jac and tvi_vjp_p over FP64 pointers and
the time t.

    VDP          van der Pol, h = [y2, mu (1 - y1^2) y2 - y1], p = [mu]   (n 2, P 1)
                 (tvi_jac a template: FP32 Jacobians with FP32 blocks)
    VDP_FP64_JAC the same with an FP64 tvi_jac
    LINEAR       h = A y, p = A row-major                                (any n, P n^2)
    mlp_tanh()   h = tanh(W3 tanh(W2 tanh(W1 y + b1) + b2) + b3)         (any n)
    MDS          mass-damper-spring chain of n/2 units with periodic forcing
                 (time-dependent; p = [K_1.., C_1.., M_1.., f_a, T], P = 3n/2 + 2)
    CHABOCHE     Chaboche viscoplasticity with n - 2 backstresses under a periodic
                 strain rate (p = [E, m, eta, sigma_0, K_inf, tau, C.., g.., ed_a, T])
    NEURON       n / 4 coupled neurons under a periodic current (15 parameters per
                 neuron, then the current amplitude)

    import paper_2310_08649_gb300 as tvi
    from paper_2310_08649_gb300.user_sources import VDP
    model = tvi.UserModel(2, 1, VDP).model(per_series=True)
"""

VDP = r"""
// van der Pol: h = [y2, mu (1 - y1^2) y2 - y1], p = [mu]
__device__ void tvi_rhs(const double* y, double t, const double* p, double* h) {
  h[0] = y[1];
  h[1] = p[0] * (1.0 - y[0] * y[0]) * y[1] - y[0];
}
// the Jacobian as a template: evaluated in FP32 with FP32 blocks
template <typename T>
__device__ void tvi_jac(const T* y, double t, const double* p, T* J) {
  const T mu = static_cast<T>(p[0]);
  J[0] = T(0);
  J[1] = T(1);
  J[2] = -T(2) * mu * y[0] * y[1] - T(1);
  J[3] = mu * (T(1) - y[0] * y[0]);
}
__device__ void tvi_vjp_p(const double* y, double t, const double* p, const double* a,
                          double* g) {
  g[0] = a[1] * (1.0 - y[0] * y[0]) * y[1];
}
"""

# van der Pol with a plain FP64 Jacobian (rounded to the block type after evaluation)
VDP_FP64_JAC = VDP[:VDP.index("// the Jacobian as a template")] + r"""
__device__ void tvi_jac(const double* y, double t, const double* p, double* J) {
  J[0] = 0.0;
  J[1] = 1.0;
  J[2] = -2.0 * p[0] * y[0] * y[1] - 1.0;
  J[3] = p[0] * (1.0 - y[0] * y[0]);
}
""" + VDP[VDP.index("__device__ void tvi_vjp_p"):]

LINEAR = r"""
// h = A y with A = p as a row-major TVI_N x TVI_N matrix
__device__ void tvi_rhs(const double* y, double t, const double* p, double* h) {
  for (int i = 0; i < TVI_N; ++i) {
    double s = 0.0;
    for (int j = 0; j < TVI_N; ++j) s += p[i * TVI_N + j] * y[j];
    h[i] = s;
  }
}
__device__ void tvi_jac(const double* y, double t, const double* p, double* J) {
  for (int k = 0; k < TVI_N * TVI_N; ++k) J[k] = p[k];
}
__device__ void tvi_vjp_p(const double* y, double t, const double* p, const double* a,
                          double* g) {
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

__device__ void tvi_rhs(const double* y, double t, const double* p, double* h) {
  MlpState s;
  mlp_eval(y, p, s);
  for (int i = 0; i < TVI_N; ++i) h[i] = s.h[i];
}

// row i of J = d3_i W3[i,:] D2 W2 D1 W1
__device__ void tvi_jac(const double* y, double t, const double* p, double* J) {
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
__device__ void tvi_vjp_p(const double* y, double t, const double* p, const double* a,
                          double* g) {
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


MDS = r"""
// mass-damper-spring chain of kU = TVI_N / 2 units, y = [d_1..d_u, v_1..v_u],
// p = [K_1..K_u, C_1..C_u, M_1..M_u, f_a, T]: spring and damper i join mass i
// to mass i+1 (the fixed wall for i = u); the force f_a sin(2 pi t / T) acts
// on mass 1 (the free end)
constexpr int kU = TVI_N / 2;

// F_i = K_i (d_{i+1} - d_i) + C_i (v_{i+1} - v_i), F_{-1} = 0
__device__ double mds_force(const double* y, const double* p, int i) {
  if (i < 0) return 0.0;
  const double dn = i + 1 < kU ? y[i + 1] : 0.0;
  const double vn = i + 1 < kU ? y[kU + i + 1] : 0.0;
  return p[i] * (dn - y[i]) + p[kU + i] * (vn - y[kU + i]);
}

__device__ void tvi_rhs(const double* y, double t, const double* p, double* h) {
  for (int i = 0; i < kU; ++i) {
    h[i] = y[kU + i];
    h[kU + i] = (mds_force(y, p, i) - mds_force(y, p, i - 1)) / p[2 * kU + i];
  }
  h[kU] += p[3 * kU] * sin(6.283185307179586 * t / p[3 * kU + 1]);
}

// constant in y: evaluated in the block type
template <typename T>
__device__ void tvi_jac(const T* y, double t, const double* p, T* J) {
  for (int k = 0; k < TVI_N * TVI_N; ++k) J[k] = T(0);
  for (int i = 0; i < kU; ++i) {
    J[i * TVI_N + kU + i] = T(1);
    T* row = J + (kU + i) * TVI_N;
    const T inv_m = T(1) / static_cast<T>(p[2 * kU + i]);
    const T k0 = static_cast<T>(p[i]) * inv_m, c0 = static_cast<T>(p[kU + i]) * inv_m;
    row[i] -= k0;
    row[kU + i] -= c0;
    if (i + 1 < kU) {
      row[i + 1] += k0;
      row[kU + i + 1] += c0;
    }
    if (i > 0) {
      const T k1 = static_cast<T>(p[i - 1]) * inv_m, c1 = static_cast<T>(p[kU + i - 1]) * inv_m;
      row[i] -= k1;
      row[i - 1] += k1;
      row[kU + i] -= c1;
      row[kU + i - 1] += c1;
    }
  }
}

__device__ void tvi_vjp_p(const double* y, double t, const double* p, const double* a,
                          double* g) {
  const double* av = a + kU;
  for (int i = 0; i < kU; ++i) {
    const double dn = i + 1 < kU ? y[i + 1] : 0.0;
    const double vn = i + 1 < kU ? y[kU + i + 1] : 0.0;
    // F_i enters v_i' as +F_i / M_i and v_{i+1}' as -F_i / M_{i+1}
    const double w = av[i] / p[2 * kU + i] - (i + 1 < kU ? av[i + 1] / p[2 * kU + i + 1] : 0.0);
    g[i] = w * (dn - y[i]);
    g[kU + i] = w * (vn - y[kU + i]);
    const double m = p[2 * kU + i];
    g[2 * kU + i] = -av[i] * (mds_force(y, p, i) - mds_force(y, p, i - 1)) / (m * m);
  }
  const double ph = 6.283185307179586 * t / p[3 * kU + 1];
  g[3 * kU] = av[0] * sin(ph);
  g[3 * kU + 1] = -av[0] * p[3 * kU] * cos(ph) * ph / p[3 * kU + 1];
}
"""


def mds_param_count(n_unit):
    return 3 * n_unit + 2


CHABOCHE = r"""
// Chaboche viscoplasticity with kU = TVI_N - 2 backstresses, y = [sigma, K,
// X_1..X_u], p = [E, m, eta, sigma_0, K_inf, tau, C_1..C_u, g_1..g_u, ed_a, T]:
//   s = sigma - sum X, f = (|s| - K - sigma_0) / eta, ep = max(f, 0)^m sign(s)
//   sigma' = E (ed_a sin(2 pi t / T) - ep), K' = tau (K_inf - K),
//   X_i' = 2/3 C_i ep - g_i X_i |ep|
constexpr int kU = TVI_N - 2;

// sign(s), |ep| and d = (m / eta) f^(m-1) (0 in the elastic range)
template <typename T>
__device__ void chaboche_flow(const T* y, const double* p, T& sgn, T& aep, T& d) {
  T s = y[0];
  for (int i = 0; i < kU; ++i) s -= y[2 + i];
  sgn = s > T(0) ? T(1) : (s < T(0) ? T(-1) : T(0));
  const T mexp = static_cast<T>(p[1]), eta = static_cast<T>(p[2]);
  const T f = (fabs(s) - y[1] - static_cast<T>(p[3])) / eta;
  if (f > T(0)) {
    const T fm1 = pow(f, mexp - T(1));
    aep = fm1 * f;
    d = mexp / eta * fm1;
  } else {
    aep = T(0);
    d = T(0);
  }
}

__device__ void tvi_rhs(const double* y, double t, const double* p, double* h) {
  double sgn, aep, d;
  chaboche_flow(y, p, sgn, aep, d);
  const double ep = aep * sgn;
  h[0] = p[0] * (p[6 + 2 * kU] * sin(6.283185307179586 * t / p[7 + 2 * kU]) - ep);
  h[1] = p[5] * (p[4] - y[1]);
  for (int i = 0; i < kU; ++i)
    h[2 + i] = 2.0 / 3.0 * p[6 + i] * ep - p[6 + kU + i] * y[2 + i] * aep;
}

// Jacobian in the block type: d ep = d (ds, -sgn dK), d|ep| = d (sgn ds, -dK),
// ds = dsigma - sum dX
template <typename T>
__device__ void tvi_jac(const T* y, double t, const double* p, T* J) {
  T sgn, aep, d;
  chaboche_flow(y, p, sgn, aep, d);
  const T E = static_cast<T>(p[0]);
  for (int k = 0; k < TVI_N * TVI_N; ++k) J[k] = T(0);
  J[0] = -E * d;
  J[1] = E * d * sgn;
  for (int q = 0; q < kU; ++q) J[2 + q] = E * d;
  J[TVI_N + 1] = -static_cast<T>(p[5]);
  for (int i = 0; i < kU; ++i) {
    T* row = J + (2 + i) * TVI_N;
    const T c = T(2) / T(3) * static_cast<T>(p[6 + i]);
    const T gx = static_cast<T>(p[6 + kU + i]) * y[2 + i];
    row[0] = c * d - gx * d * sgn;
    row[1] = -c * d * sgn + gx * d;
    for (int q = 0; q < kU; ++q) row[2 + q] = -c * d + gx * d * sgn;
    row[2 + i] -= static_cast<T>(p[6 + kU + i]) * aep;
  }
}

__device__ void tvi_vjp_p(const double* y, double t, const double* p, const double* a,
                          double* g) {
  double sgn, aep, d;
  chaboche_flow(y, p, sgn, aep, d);
  const double ep = aep * sgn;
  double s = y[0];
  for (int i = 0; i < kU; ++i) s -= y[2 + i];
  const double f = (fabs(s) - y[1] - p[3]) / p[2];
  // derivatives of |ep| over the flow exponent, eta and sigma_0 (0 when elastic)
  const double dm = f > 0.0 ? aep * log(f) : 0.0;
  const double deta = -d * f;
  const double ds0 = -d;
  double w = -p[0] * a[0] * sgn;  // weight of |ep| in a . h
  for (int i = 0; i < kU; ++i)
    w += a[2 + i] * (2.0 / 3.0 * p[6 + i] * sgn - p[6 + kU + i] * y[2 + i]);
  const double ph = 6.283185307179586 * t / p[7 + 2 * kU];
  g[0] = a[0] * (p[6 + 2 * kU] * sin(ph) - ep);
  g[1] = w * dm;
  g[2] = w * deta;
  g[3] = w * ds0;
  g[4] = a[1] * p[5];
  g[5] = a[1] * (p[4] - y[1]);
  for (int i = 0; i < kU; ++i) {
    g[6 + i] = a[2 + i] * 2.0 / 3.0 * ep;
    g[6 + kU + i] = -a[2 + i] * y[2 + i] * aep;
  }
  g[6 + 2 * kU] = a[0] * p[0] * sin(ph);
  g[7 + 2 * kU] = -a[0] * p[0] * p[6 + 2 * kU] * cos(ph) * ph / p[7 + 2 * kU];
}
"""


def chaboche_param_count(n_unit):
    return 2 * n_unit + 8


NEURON = r"""
// kU = TVI_N / 4 coupled neurons, y = [V_1, m_1, h_1, n_1, V_2, ...]; per neuron i
// the 15 values p[15 i ..] = [C, gNa, ENa, gK, EK, gL, EL, m_inf, tau_m, h_inf,
// tau_h, n_inf, tau_n, gC, T], then p[15 kU] = I_a:
//   V' = (-gNa m^3 h (V - ENa) - gK n^4 (V - EK) - gL (V - EL)
//         + I_a sin(2 pi t / T) + gC sum_j (V_i - V_j)) / C
//   m' = (m_inf - m) / tau_m, and h, n alike
constexpr int kU = TVI_N / 4;

__device__ void tvi_rhs(const double* y, double t, const double* p, double* h) {
  const double Ia = p[15 * kU];
  for (int i = 0; i < kU; ++i) {
    const double* q = p + 15 * i;
    const double V = y[4 * i], m = y[4 * i + 1], hh = y[4 * i + 2], n = y[4 * i + 3];
    double coup = 0.0;
    for (int j = 0; j < kU; ++j) coup += V - y[4 * j];
    const double I = -q[1] * m * m * m * hh * (V - q[2]) - q[3] * n * n * n * n * (V - q[4]) -
                     q[5] * (V - q[6]) + Ia * sin(6.283185307179586 * t / q[14]) + q[13] * coup;
    h[4 * i] = I / q[0];
    h[4 * i + 1] = (q[7] - m) / q[8];
    h[4 * i + 2] = (q[9] - hh) / q[10];
    h[4 * i + 3] = (q[11] - n) / q[12];
  }
}

template <typename T>
__device__ void tvi_jac(const T* y, double t, const double* p, T* J) {
  for (int k = 0; k < TVI_N * TVI_N; ++k) J[k] = T(0);
  for (int i = 0; i < kU; ++i) {
    const double* q = p + 15 * i;
    const T V = y[4 * i], m = y[4 * i + 1], hh = y[4 * i + 2], n = y[4 * i + 3];
    const T C = static_cast<T>(q[0]), gNa = static_cast<T>(q[1]), ENa = static_cast<T>(q[2]);
    const T gK = static_cast<T>(q[3]), EK = static_cast<T>(q[4]), gL = static_cast<T>(q[5]);
    const T gC = static_cast<T>(q[13]);
    T* row = J + 4 * i * TVI_N;
    for (int j = 0; j < kU; ++j) row[4 * j] = (j == i ? gC * T(kU - 1) : -gC) / C;
    row[4 * i] += (-gNa * m * m * m * hh - gK * n * n * n * n - gL) / C;
    row[4 * i + 1] = -T(3) * gNa * m * m * hh * (V - ENa) / C;
    row[4 * i + 2] = -gNa * m * m * m * (V - ENa) / C;
    row[4 * i + 3] = -T(4) * gK * n * n * n * (V - EK) / C;
    J[(4 * i + 1) * TVI_N + 4 * i + 1] = -T(1) / static_cast<T>(q[8]);
    J[(4 * i + 2) * TVI_N + 4 * i + 2] = -T(1) / static_cast<T>(q[10]);
    J[(4 * i + 3) * TVI_N + 4 * i + 3] = -T(1) / static_cast<T>(q[12]);
  }
}

__device__ void tvi_vjp_p(const double* y, double t, const double* p, const double* a,
                          double* g) {
  const double Ia = p[15 * kU];
  g[15 * kU] = 0.0;
  for (int i = 0; i < kU; ++i) {
    const double* q = p + 15 * i;
    double* gi = g + 15 * i;
    const double V = y[4 * i], m = y[4 * i + 1], hh = y[4 * i + 2], n = y[4 * i + 3];
    const double m3h = m * m * m * hh, n4 = n * n * n * n;
    double coup = 0.0;
    for (int j = 0; j < kU; ++j) coup += V - y[4 * j];
    const double ph = 6.283185307179586 * t / q[14];
    const double s = sin(ph);
    const double I = -q[1] * m3h * (V - q[2]) - q[3] * n4 * (V - q[4]) - q[5] * (V - q[6]) +
                     Ia * s + q[13] * coup;
    const double aV = a[4 * i] / q[0];
    gi[0] = -a[4 * i] * I / (q[0] * q[0]);
    gi[1] = -aV * m3h * (V - q[2]);
    gi[2] = aV * q[1] * m3h;
    gi[3] = -aV * n4 * (V - q[4]);
    gi[4] = aV * q[3] * n4;
    gi[5] = -aV * (V - q[6]);
    gi[6] = aV * q[5];
    gi[7] = a[4 * i + 1] / q[8];
    gi[8] = -a[4 * i + 1] * (q[7] - m) / (q[8] * q[8]);
    gi[9] = a[4 * i + 2] / q[10];
    gi[10] = -a[4 * i + 2] * (q[9] - hh) / (q[10] * q[10]);
    gi[11] = a[4 * i + 3] / q[12];
    gi[12] = -a[4 * i + 3] * (q[11] - n) / (q[12] * q[12]);
    gi[13] = aV * coup;
    gi[14] = -aV * Ia * cos(ph) * ph / q[14];
    g[15 * kU] += aV * s;
  }
}
"""


def neuron_param_count(n_unit):
    return 15 * n_unit + 1
