/*
 * tvi_oracle.c -- plain, slow, FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * Step-by-step backward-Euler Newton integration with dense LU, and the
 * discrete adjoint with dense LU of the transposed step Jacobian.  No chunks,
 * no cyclic reduction, no blocking: each series is integrated one step at a
 * time exactly as the definitions in tvi_oracle.h state.  Series are
 * independent (paper Sec. 2.1: initial conditions, parameters and times may
 * differ per series), so the loop over series runs under OpenMP.
 */
#include "tvi_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Models: h(y,t;p), j = dh/dy, (dh/dp)^T a                                  */
/* ------------------------------------------------------------------------ */

int tvo_param_count(const tvo_model* m) {
  if (!m || m->n <= 0) return -1;
  switch (m->kind) {
    case TVO_LINEAR: return m->n * m->n;
    case TVO_VDP: return m->n == 2 ? 1 : -1;
    case TVO_MDS: return m->n % 2 == 0 ? 3 * (m->n / 2) + 2 : -1;
    case TVO_CHABOCHE: return m->n >= 3 ? 2 * (m->n - 2) + 8 : -1;
    case TVO_NEURON: return m->n % 4 == 0 ? 15 * (m->n / 4) + 1 : -1;
    case TVO_MLP_TANH:
    case TVO_MLP_SILU:
      if (m->h1 <= 0 || m->h2 <= 0) return -1;
      return m->h1 * m->n + m->h1 + m->h2 * m->h1 + m->h2 + m->n * m->h2 + m->n;
    default: return -1;
  }
}

static double act(int kind, double z) {
  if (kind == TVO_MLP_TANH) return tanh(z);
  return z / (1.0 + exp(-z)); /* SiLU: z * sigmoid(z) */
}

static double act_d(int kind, double z) {
  if (kind == TVO_MLP_TANH) {
    double t = tanh(z);
    return 1.0 - t * t;
  }
  double s = 1.0 / (1.0 + exp(-z));
  return s + z * s * (1.0 - s);
}

/* Views into the flat MLP parameter vector. */
typedef struct {
  const double *W1, *b1, *W2, *b2, *W3, *b3;
} mlp_view;

static mlp_view mlp_split(const tvo_model* m, const double* p) {
  mlp_view v;
  int n = m->n, h1 = m->h1, h2 = m->h2;
  v.W1 = p;
  v.b1 = v.W1 + h1 * n;
  v.W2 = v.b1 + h1;
  v.b2 = v.W2 + h2 * h1;
  v.W3 = v.b2 + h2;
  v.b3 = v.W3 + n * h2;
  return v;
}

/* Forward pass of the MLP keeping pre-activations z1[h1], z2[h2], z3[n] and
 * activations a1[h1], a2[h2]; returns h in out[n]. */
static void mlp_forward(const tvo_model* m, const double* p, const double* y, double* z1,
                        double* a1, double* z2, double* a2, double* z3, double* out) {
  int n = m->n, h1 = m->h1, h2 = m->h2;
  mlp_view v = mlp_split(m, p);
  for (int r = 0; r < h1; ++r) {
    double s = v.b1[r];
    for (int c = 0; c < n; ++c) s += v.W1[r * n + c] * y[c];
    z1[r] = s;
    a1[r] = act(m->kind, s);
  }
  for (int r = 0; r < h2; ++r) {
    double s = v.b2[r];
    for (int c = 0; c < h1; ++c) s += v.W2[r * h1 + c] * a1[c];
    z2[r] = s;
    a2[r] = act(m->kind, s);
  }
  for (int r = 0; r < n; ++r) {
    double s = v.b3[r];
    for (int c = 0; c < h2; ++c) s += v.W3[r * h2 + c] * a2[c];
    z3[r] = s;
    out[r] = (m->kind == TVO_MLP_TANH) ? tanh(s) : s;
  }
}

static double out_d(const tvo_model* m, double z3) {
  if (m->kind == TVO_MLP_TANH) {
    double t = tanh(z3);
    return 1.0 - t * t;
  }
  return 1.0; /* SiLU network: linear output layer */
}

/* Mass-damper-spring chain: force F_i of spring and damper i (mass i to mass
 * i+1, the fixed wall for i = u), with F_0 = 0 at the free end. */
static double mds_force(int u, const double* p, const double* y, int i) {
  if (i < 0) return 0.0;
  const double* K = p;
  const double* C = p + u;
  double dn = (i + 1 < u) ? y[i + 1] : 0.0;
  double vn = (i + 1 < u) ? y[u + i + 1] : 0.0;
  return K[i] * (dn - y[i]) + C[i] * (vn - y[u + i]);
}

static const double kTwoPi = 6.283185307179586476925286766559;

/* Chaboche: the plastic strain rate ep and its derivatives.  With s = sigma -
 * sum X and f = (|s| - K - sigma_0) / eta: ep = max(f, 0)^m sign(s); for f > 0
 * d ep / d s = (m / eta) f^(m-1), d ep / d K = -(m / eta) f^(m-1) sign(s),
 * d|ep| / d s = (m / eta) f^(m-1) sign(s), d|ep| / d K = -(m / eta) f^(m-1);
 * all zero for f <= 0 (elastic). */
typedef struct {
  double s, sgn, f, ep, aep, d;  /* d = (m / eta) f^(m-1) when f > 0, else 0 */
} chab_flow;

static chab_flow chab_eval(int u, const double* p, const double* y) {
  chab_flow c;
  double sumX = 0.0;
  for (int i = 0; i < u; ++i) sumX += y[2 + i];
  c.s = y[0] - sumX;
  c.sgn = (c.s > 0.0) ? 1.0 : ((c.s < 0.0) ? -1.0 : 0.0);
  const double mexp = p[1], eta = p[2], sigma0 = p[3];
  c.f = (fabs(c.s) - y[1] - sigma0) / eta;
  if (c.f > 0.0) {
    c.aep = pow(c.f, mexp);
    c.d = mexp / eta * pow(c.f, mexp - 1.0);
  } else {
    c.aep = 0.0;
    c.d = 0.0;
  }
  c.ep = c.aep * c.sgn;
  return c;
}

/* Coupled neurons: the ionic current sum of neuron i (the bracket of V_i' without
 * the applied current), its derivatives over V_i, m_i, h_i, n_i. */
typedef struct {
  double curr, dV, dm, dh, dn;
} neuron_terms;

static neuron_terms neuron_eval(const double* q, double V, double mm, double hh, double nn) {
  /* q: the neuron's 15 parameters */
  const double gNa = q[1], ENa = q[2], gK = q[3], EK = q[4], gL = q[5], EL = q[6];
  neuron_terms r;
  const double m3 = mm * mm * mm, n4 = nn * nn * nn * nn;
  r.curr = -gNa * m3 * hh * (V - ENa) - gK * n4 * (V - EK) - gL * (V - EL);
  r.dV = -gNa * m3 * hh - gK * n4 - gL;
  r.dm = -3.0 * gNa * mm * mm * hh * (V - ENa);
  r.dh = -gNa * m3 * (V - ENa);
  r.dn = -4.0 * gK * nn * nn * nn * (V - EK);
  return r;
}

void tvo_rhs(const tvo_model* m, const double* p, const double* y, double t, double* h) {
  int n = m->n;
  if (m->kind == TVO_NEURON) {
    int u = n / 4;
    const double Ia = p[15 * u];
    for (int i = 0; i < u; ++i) {
      const double* q = p + 15 * i;
      const double* yi = y + 4 * i;
      neuron_terms r = neuron_eval(q, yi[0], yi[1], yi[2], yi[3]);
      double coup = 0.0;
      for (int j = 0; j < u; ++j) coup += yi[0] - y[4 * j];
      h[4 * i] = (r.curr + Ia * sin(kTwoPi * t / q[14]) + q[13] * coup) / q[0];
      h[4 * i + 1] = (q[7] - yi[1]) / q[8];
      h[4 * i + 2] = (q[9] - yi[2]) / q[10];
      h[4 * i + 3] = (q[11] - yi[3]) / q[12];
    }
    return;
  }
  if (m->kind == TVO_CHABOCHE) {
    int u = n - 2;
    const double *C = p + 6, *g = p + 6 + u;
    const double E = p[0], Kinf = p[4], tau = p[5], eda = p[6 + 2 * u], T = p[7 + 2 * u];
    chab_flow c = chab_eval(u, p, y);
    h[0] = E * (eda * sin(kTwoPi * t / T) - c.ep);
    h[1] = tau * (Kinf - y[1]);
    for (int i = 0; i < u; ++i) h[2 + i] = 2.0 / 3.0 * C[i] * c.ep - g[i] * y[2 + i] * c.aep;
    return;
  }
  if (m->kind == TVO_MDS) {
    int u = n / 2;
    const double* M = p + 2 * u;
    double fa = p[3 * u], T = p[3 * u + 1];
    for (int i = 0; i < u; ++i) {
      h[i] = y[u + i];
      h[u + i] = (mds_force(u, p, y, i) - mds_force(u, p, y, i - 1)) / M[i];
    }
    h[u] += fa * sin(kTwoPi * t / T);
  } else if (m->kind == TVO_LINEAR) {
    for (int r = 0; r < n; ++r) {
      double s = 0.0;
      for (int c = 0; c < n; ++c) s += p[r * n + c] * y[c];
      h[r] = s;
    }
  } else if (m->kind == TVO_VDP) {
    double mu = p[0];
    h[0] = y[1];
    h[1] = mu * (1.0 - y[0] * y[0]) * y[1] - y[0];
  } else {
    double* w = (double*)malloc(sizeof(double) * (2 * m->h1 + 2 * m->h2 + n));
    mlp_forward(m, p, y, w, w + m->h1, w + 2 * m->h1, w + 2 * m->h1 + m->h2,
                w + 2 * m->h1 + 2 * m->h2, h);
    free(w);
  }
}

void tvo_jac(const tvo_model* m, const double* p, const double* y, double t, double* j) {
  (void)t;
  int n = m->n;
  if (m->kind == TVO_NEURON) {
    int u = n / 4;
    memset(j, 0, sizeof(double) * n * n);
    for (int i = 0; i < u; ++i) {
      const double* q = p + 15 * i;
      const double* yi = y + 4 * i;
      neuron_terms r = neuron_eval(q, yi[0], yi[1], yi[2], yi[3]);
      double* rowV = j + (4 * i) * n;
      /* coupling gC sum_j (V_i - V_j): + gC (u - 1) on V_i, - gC on every other V_j */
      for (int k = 0; k < u; ++k) rowV[4 * k] = (k == i ? q[13] * (u - 1) : -q[13]) / q[0];
      rowV[4 * i] += r.dV / q[0];
      rowV[4 * i + 1] = r.dm / q[0];
      rowV[4 * i + 2] = r.dh / q[0];
      rowV[4 * i + 3] = r.dn / q[0];
      j[(4 * i + 1) * n + 4 * i + 1] = -1.0 / q[8];
      j[(4 * i + 2) * n + 4 * i + 2] = -1.0 / q[10];
      j[(4 * i + 3) * n + 4 * i + 3] = -1.0 / q[12];
    }
    return;
  }
  if (m->kind == TVO_CHABOCHE) {
    int u = n - 2;
    const double *C = p + 6, *g = p + 6 + u;
    const double E = p[0], tau = p[5];
    chab_flow c = chab_eval(u, p, y);
    /* gradients over y of ep and |ep|: s depends on sigma (+1) and X_i (-1) */
    double dep[32 + 2], daep[32 + 2];
    dep[0] = c.d;
    daep[0] = c.d * c.sgn;
    dep[1] = -c.d * c.sgn;
    daep[1] = -c.d;
    for (int i = 0; i < u; ++i) {
      dep[2 + i] = -c.d;
      daep[2 + i] = -c.d * c.sgn;
    }
    memset(j, 0, sizeof(double) * n * n);
    for (int col = 0; col < n; ++col) j[col] = -E * dep[col];
    j[n + 1] = -tau;
    for (int i = 0; i < u; ++i) {
      double* row = j + (2 + i) * n;
      for (int col = 0; col < n; ++col)
        row[col] = 2.0 / 3.0 * C[i] * dep[col] - g[i] * y[2 + i] * daep[col];
      row[2 + i] -= g[i] * c.aep;
    }
    return;
  }
  if (m->kind == TVO_MDS) {
    /* h is linear in y: column c of j is h(e_c) without the forcing */
    int u = n / 2;
    const double *K = p, *C = p + u, *M = p + 2 * u;
    memset(j, 0, sizeof(double) * n * n);
    for (int i = 0; i < u; ++i) {
      j[i * n + u + i] = 1.0;           /* d_i' = v_i */
      double* row = j + (u + i) * n;    /* v_i' */
      /* + F_i / M_i */
      row[i] -= K[i] / M[i];
      row[u + i] -= C[i] / M[i];
      if (i + 1 < u) {
        row[i + 1] += K[i] / M[i];
        row[u + i + 1] += C[i] / M[i];
      }
      /* - F_{i-1} / M_i, F_{i-1} = K_{i-1} (d_i - d_{i-1}) + C_{i-1} (v_i - v_{i-1}) */
      if (i > 0) {
        row[i] -= K[i - 1] / M[i];
        row[i - 1] += K[i - 1] / M[i];
        row[u + i] -= C[i - 1] / M[i];
        row[u + i - 1] += C[i - 1] / M[i];
      }
    }
  } else if (m->kind == TVO_LINEAR) {
    memcpy(j, p, sizeof(double) * n * n);
  } else if (m->kind == TVO_VDP) {
    double mu = p[0];
    j[0] = 0.0;
    j[1] = 1.0;
    j[2] = -2.0 * mu * y[0] * y[1] - 1.0;
    j[3] = mu * (1.0 - y[0] * y[0]);
  } else {
    /* j = D3 W3 D2 W2 D1 W1 with D_i = diag(act'(z_i)); chain rule written out
     * column by column of the input: J[:, c] = d h / d y_c. */
    int h1 = m->h1, h2 = m->h2;
    mlp_view v = mlp_split(m, p);
    double* w = (double*)malloc(sizeof(double) * (3 * h1 + 3 * h2 + 2 * n));
    double *z1 = w, *a1 = z1 + h1, *z2 = a1 + h1, *a2 = z2 + h2, *z3 = a2 + h2, *o = z3 + n;
    double *u1 = o + n, *u2 = u1 + h1;
    mlp_forward(m, p, y, z1, a1, z2, a2, z3, o);
    for (int c = 0; c < n; ++c) {
      for (int r = 0; r < h1; ++r) u1[r] = act_d(m->kind, z1[r]) * v.W1[r * n + c];
      for (int r = 0; r < h2; ++r) {
        double s = 0.0;
        for (int q = 0; q < h1; ++q) s += v.W2[r * h1 + q] * u1[q];
        u2[r] = act_d(m->kind, z2[r]) * s;
      }
      for (int r = 0; r < n; ++r) {
        double s = 0.0;
        for (int q = 0; q < h2; ++q) s += v.W3[r * h2 + q] * u2[q];
        j[r * n + c] = out_d(m, z3[r]) * s;
      }
    }
    free(w);
  }
}

void tvo_vjp_p(const tvo_model* m, const double* p, const double* y, double t, const double* a,
               double scale, double* gp) {
  int n = m->n;
  if (m->kind == TVO_NEURON) {
    int u = n / 4;
    const double Ia = p[15 * u];
    for (int i = 0; i < u; ++i) {
      const double* q = p + 15 * i;
      double* g = gp + 15 * i;
      const double* yi = y + 4 * i;
      const double V = yi[0], mm = yi[1], hh = yi[2], nn = yi[3];
      const double m3h = mm * mm * mm * hh, n4 = nn * nn * nn * nn;
      const double aV = a[4 * i] / q[0];  /* weight of the bracket of V_i' */
      neuron_terms r = neuron_eval(q, V, mm, hh, nn);
      double coup = 0.0;
      for (int k = 0; k < u; ++k) coup += V - y[4 * k];
      const double s = sin(kTwoPi * t / q[14]);
      const double bracket = r.curr + Ia * s + q[13] * coup;
      g[0] += scale * a[4 * i] * (-bracket / (q[0] * q[0]));  /* C */
      g[1] += scale * aV * (-m3h * (V - q[2]));               /* gNa */
      g[2] += scale * aV * (q[1] * m3h);                      /* ENa */
      g[3] += scale * aV * (-n4 * (V - q[4]));                /* gK */
      g[4] += scale * aV * (q[3] * n4);                       /* EK */
      g[5] += scale * aV * (-(V - q[6]));                     /* gL */
      g[6] += scale * aV * q[5];                              /* EL */
      g[7] += scale * a[4 * i + 1] / q[8];                    /* m_inf */
      g[8] += scale * a[4 * i + 1] * (-(q[7] - mm) / (q[8] * q[8]));  /* tau_m */
      g[9] += scale * a[4 * i + 2] / q[10];                   /* h_inf */
      g[10] += scale * a[4 * i + 2] * (-(q[9] - hh) / (q[10] * q[10]));  /* tau_h */
      g[11] += scale * a[4 * i + 3] / q[12];                  /* n_inf */
      g[12] += scale * a[4 * i + 3] * (-(q[11] - nn) / (q[12] * q[12]));  /* tau_n */
      g[13] += scale * aV * coup;                             /* gC */
      const double ph = kTwoPi * t / q[14];
      g[14] += scale * aV * Ia * cos(ph) * (-ph / q[14]);     /* T */
      gp[15 * u] += scale * aV * s;                           /* I_a */
    }
    return;
  }
  if (m->kind == TVO_CHABOCHE) {
    /* p = [E, m, eta, sigma0, Kinf, tau, C_1..C_u, g_1..g_u, ed_a, T] */
    int u = n - 2;
    const double *C = p + 6, *g = p + 6 + u;
    const double E = p[0], mexp = p[1], eta = p[2], Kinf = p[4], tau = p[5];
    const double eda = p[6 + 2 * u], T = p[7 + 2 * u];
    chab_flow c = chab_eval(u, p, y);
    /* derivatives of |ep| = max(f, 0)^m over m, eta, sigma0 (zero when elastic) */
    double daep_m = 0.0, daep_eta = 0.0, daep_s0 = 0.0;
    if (c.f > 0.0) {
      daep_m = c.aep * log(c.f);
      daep_eta = -c.d * c.f;  /* d f / d eta = -f / eta; times m f^(m-1) */
      daep_s0 = -c.d;         /* d f / d sigma0 = -1 / eta */
    }
    /* h depends on ep = |ep| sgn and |ep|: weight of d|ep| in a . h */
    double w = -E * a[0] * c.sgn;  /* sigma' = ... - E ep */
    for (int i = 0; i < u; ++i) w += a[2 + i] * (2.0 / 3.0 * C[i] * c.sgn - g[i] * y[2 + i]);
    const double ph = kTwoPi * t / T;
    gp[0] += scale * a[0] * (eda * sin(ph) - c.ep);        /* E */
    gp[1] += scale * w * daep_m;                            /* m */
    gp[2] += scale * w * daep_eta;                          /* eta */
    gp[3] += scale * w * daep_s0;                           /* sigma0 */
    gp[4] += scale * a[1] * tau;                            /* K_inf */
    gp[5] += scale * a[1] * (Kinf - y[1]);                  /* tau */
    for (int i = 0; i < u; ++i) {
      gp[6 + i] += scale * a[2 + i] * 2.0 / 3.0 * c.ep;     /* C_i */
      gp[6 + u + i] += scale * a[2 + i] * (-y[2 + i] * c.aep);  /* g_i */
    }
    gp[6 + 2 * u] += scale * a[0] * E * sin(ph);            /* ed_a */
    gp[7 + 2 * u] += scale * a[0] * E * eda * cos(ph) * (-ph / T);  /* T */
    return;
  }
  if (m->kind == TVO_MDS) {
    /* v_i' = (F_i - F_{i-1}) / M_i: F_i enters v_i' with +1/M_i and v_{i+1}' with
     * -1/M_{i+1}; F_i is linear in K_i and C_i. */
    int u = n / 2;
    const double* M = p + 2 * u;
    double fa = p[3 * u], T = p[3 * u + 1];
    const double* av = a + u;
    for (int i = 0; i < u; ++i) {
      double dn = (i + 1 < u) ? y[i + 1] : 0.0;
      double vn = (i + 1 < u) ? y[u + i + 1] : 0.0;
      double w = av[i] / M[i] - ((i + 1 < u) ? av[i + 1] / M[i + 1] : 0.0);
      gp[i] += scale * w * (dn - y[i]);          /* dK_i */
      gp[u + i] += scale * w * (vn - y[u + i]);  /* dC_i */
      double Fnet = mds_force(u, p, y, i) - mds_force(u, p, y, i - 1);
      gp[2 * u + i] += scale * av[i] * (-Fnet / (M[i] * M[i]));  /* dM_i */
    }
    double ph = kTwoPi * t / T;
    gp[3 * u] += scale * av[0] * sin(ph);                              /* df_a */
    gp[3 * u + 1] += scale * av[0] * fa * cos(ph) * (-ph / T);         /* dT */
  } else if (m->kind == TVO_LINEAR) {
    /* h_r = sum_c A_rc y_c  =>  dh_r/dA_rc = y_c, so (dh/dA)^T a = a y^T. */
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) gp[r * n + c] += scale * a[r] * y[c];
  } else if (m->kind == TVO_VDP) {
    /* dh/dmu = [0, (1 - y1^2) y2]. */
    gp[0] += scale * a[1] * (1.0 - y[0] * y[0]) * y[1];
  } else {
    int h1 = m->h1, h2 = m->h2;
    mlp_view v = mlp_split(m, p);
    double* w = (double*)malloc(sizeof(double) * (3 * h1 + 3 * h2 + 3 * n));
    double *z1 = w, *a1 = z1 + h1, *z2 = a1 + h1, *a2 = z2 + h2, *z3 = a2 + h2, *o = z3 + n;
    double *d3 = o + n, *d2 = d3 + n, *d1 = d2 + h2;
    mlp_forward(m, p, y, z1, a1, z2, a2, z3, o);
    /* gradient slots, same order as the flat layout */
    double* gW1 = gp;
    double* gb1 = gW1 + h1 * n;
    double* gW2 = gb1 + h1;
    double* gb2 = gW2 + h2 * h1;
    double* gW3 = gb2 + h2;
    double* gb3 = gW3 + n * h2;
    for (int r = 0; r < n; ++r) d3[r] = a[r] * out_d(m, z3[r]);
    for (int r = 0; r < n; ++r) {
      gb3[r] += scale * d3[r];
      for (int c = 0; c < h2; ++c) gW3[r * h2 + c] += scale * d3[r] * a2[c];
    }
    for (int c = 0; c < h2; ++c) {
      double s = 0.0;
      for (int r = 0; r < n; ++r) s += v.W3[r * h2 + c] * d3[r];
      d2[c] = s * act_d(m->kind, z2[c]);
    }
    for (int r = 0; r < h2; ++r) {
      gb2[r] += scale * d2[r];
      for (int c = 0; c < h1; ++c) gW2[r * h1 + c] += scale * d2[r] * a1[c];
    }
    for (int c = 0; c < h1; ++c) {
      double s = 0.0;
      for (int r = 0; r < h2; ++r) s += v.W2[r * h1 + c] * d2[r];
      d1[c] = s * act_d(m->kind, z1[c]);
    }
    for (int r = 0; r < h1; ++r) {
      gb1[r] += scale * d1[r];
      for (int c = 0; c < n; ++c) gW1[r * n + c] += scale * d1[r] * y[c];
    }
    free(w);
  }
}

/* ------------------------------------------------------------------------ */
/* Dense LU with partial pivoting: solve M x = rhs (M is n x n, row-major).  */
/* Overwrites M and rhs; returns 0, or 1 if a pivot is exactly zero.         */
/* ------------------------------------------------------------------------ */
static int lu_solve(int n, double* M, double* rhs) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = fabs(M[k * n + k]);
    for (int r = k + 1; r < n; ++r) {
      double v = fabs(M[r * n + k]);
      if (v > best) {
        best = v;
        piv = r;
      }
    }
    if (best == 0.0) return 1;
    if (piv != k) {
      for (int c = 0; c < n; ++c) {
        double t = M[k * n + c];
        M[k * n + c] = M[piv * n + c];
        M[piv * n + c] = t;
      }
      double t = rhs[k];
      rhs[k] = rhs[piv];
      rhs[piv] = t;
    }
    for (int r = k + 1; r < n; ++r) {
      double f = M[r * n + k] / M[k * n + k];
      M[r * n + k] = 0.0;
      for (int c = k + 1; c < n; ++c) M[r * n + c] -= f * M[k * n + c];
      rhs[r] -= f * rhs[k];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = rhs[r];
    for (int c = r + 1; c < n; ++c) s -= M[r * n + c] * rhs[c];
    rhs[r] = s / M[r * n + r];
  }
  return 0;
}

static double inf_norm(int n, const double* v) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    double a = fabs(v[i]);
    if (!(a <= s)) s = a; /* also propagates NaN */
  }
  return s;
}

static double step_dt(const double* tb, const int* lengths, int b, int k) {
  /* dt_k = t_k - t_{k-1} (Sec. 2.2); padded steps beyond the series length have dt = 0 */
  if (lengths && k > lengths[b]) return 0.0;
  return tb[k] - tb[k - 1];
}

int tvo_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* One backward-Euler step by Newton (Sec. 2.2): solve                        */
/*   G(y) = y - y_prev - dt h(y, t; p) = 0,   J = dG/dy = I - dt j(y),          */
/* from the previous-step guess y = y_prev, y <- y - J^{-1} G with a dense LU.  */
/* Stops when ||G||_inf <= tol_abs or <= tol_rel ||G_0||_inf, or after         */
/* max_iter updates.  w holds 2n + n^2 doubles.  Returns the status and the    */
/* number of updates in *iters.                                                 */
/* ------------------------------------------------------------------------ */
static int be_step(const tvo_model* m, const double* p, const double* yprev, double dt, double tk,
                   double tol_abs, double tol_rel, int max_iter, double* yk, int* iters,
                   double* w) {
  const int n = m->n;
  double* G = w;
  double* hv = G + n;
  double* J = hv + n;
  memcpy(yk, yprev, sizeof(double) * n); /* 0y_{k} = y_{k-1} */
  double norm0 = 0.0;
  int it = 0, st = TVO_OK;
  for (;;) {
    /* G = y_k - y_{k-1} - dt h(y_k, t_k; p) */
    tvo_rhs(m, p, yk, tk, hv);
    for (int i = 0; i < n; ++i) G[i] = yk[i] - yprev[i] - dt * hv[i];
    double nr = inf_norm(n, G);
    if (it == 0) norm0 = nr;
    if (!isfinite(nr)) {
      st = TVO_NONFINITE;
      break;
    }
    if (nr <= tol_abs || nr <= tol_rel * norm0) break;
    if (it >= max_iter) {
      st = TVO_NOT_CONVERGED;
      break;
    }
    /* J = I - dt j(y_k); y_k -= J^{-1} G */
    tvo_jac(m, p, yk, tk, J);
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) J[r * n + c] = (r == c ? 1.0 : 0.0) - dt * J[r * n + c];
    if (lu_solve(n, J, G)) {
      st = TVO_SINGULAR;
      break;
    }
    for (int i = 0; i < n; ++i) yk[i] -= G[i];
    ++it;
  }
  *iters = it;
  return st;
}

/* ------------------------------------------------------------------------ */
/* Forward: Sec. 2.2 backward Euler + Newton, previous-step starting guess.   */
/* ------------------------------------------------------------------------ */
int tvo_forward(const tvo_model* m, int B, int N, const double* y0, const double* times,
                const int* lengths, const double* params, double tol_abs, double tol_rel,
                int max_iter, int nthreads, double* y, int* iters, int* status) {
  int P = tvo_param_count(m);
  if (P < 0 || B < 0 || N < 0 || max_iter < 0) return TVO_BADARG;
  int n = m->n;
  int worst = TVO_OK;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(max : worst)
#endif
  for (int b = 0; b < B; ++b) {
    const double* p = m->per_series ? params + (size_t)b * P : params;
    const double* tb = times + (size_t)b * (N + 1);
    double* yb = y + (size_t)b * (N + 1) * n;
    double* w = (double*)malloc(sizeof(double) * (2 * n + n * n));
    int st = TVO_OK;
    memcpy(yb, y0 + (size_t)b * n, sizeof(double) * n);
    for (int k = 1; k <= N; ++k) {
      int it = 0;
      int sk = be_step(m, p, yb + (size_t)(k - 1) * n, step_dt(tb, lengths, b, k), tb[k], tol_abs,
                       tol_rel, max_iter, yb + (size_t)k * n, &it, w);
      if (sk > st) st = sk;
      if (iters) iters[(size_t)b * N + (k - 1)] = it;
      if (sk == TVO_NONFINITE || sk == TVO_SINGULAR) {
        /* leave the rest of the trajectory as NaN: nothing after this is defined */
        for (int q = k + 1; q <= N; ++q)
          for (int i = 0; i < n; ++i) yb[(size_t)q * n + i] = NAN;
        if (iters)
          for (int q = k + 1; q <= N; ++q) iters[(size_t)b * N + (q - 1)] = 0;
        break;
      }
    }
    if (status) status[b] = st;
    if (st > worst) worst = st;
    free(w);
  }
  return worst;
}

/* ------------------------------------------------------------------------ */
/* Independent step solves (Sec. 2.2): for every series and step k = 1..N,    */
/* the backward-Euler step from the GIVEN state y_prev[b][k-1], by the same    */
/* Newton as tvo_forward.  out[b][0] = y_prev[b][0].  Checks any trajectory    */
/* step by step without propagating its earlier differences.                   */
/* ------------------------------------------------------------------------ */
int tvo_step_solves(const tvo_model* m, int B, int N, const double* times, const int* lengths,
                    const double* params, const double* y_prev, double tol_abs, double tol_rel,
                    int max_iter, int nthreads, double* out, int* status) {
  int P = tvo_param_count(m);
  if (P < 0 || B < 0 || N < 0 || max_iter < 0) return TVO_BADARG;
  int n = m->n;
  int worst = TVO_OK;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(max : worst)
#endif
  for (int b = 0; b < B; ++b) {
    const double* p = m->per_series ? params + (size_t)b * P : params;
    const double* tb = times + (size_t)b * (N + 1);
    const double* yb = y_prev + (size_t)b * (N + 1) * n;
    double* ob = out + (size_t)b * (N + 1) * n;
    double* w = (double*)malloc(sizeof(double) * (2 * n + n * n));
    int st = TVO_OK;
    memcpy(ob, yb, sizeof(double) * n);
    for (int k = 1; k <= N; ++k) {
      int it = 0;
      int sk = be_step(m, p, yb + (size_t)(k - 1) * n, step_dt(tb, lengths, b, k), tb[k], tol_abs,
                       tol_rel, max_iter, ob + (size_t)k * n, &it, w);
      if (sk > st) st = sk;
    }
    if (status) status[b] = st;
    if (st > worst) worst = st;
    free(w);
  }
  return worst;
}

/* ------------------------------------------------------------------------ */
/* Adjoint: App. A.1, discrete form of the backward-Euler adjoint.           */
/* ------------------------------------------------------------------------ */
int tvo_adjoint(const tvo_model* m, int B, int N, const double* times, const int* lengths,
                const double* params, const double* y, const double* grad_out, int nthreads,
                double* dparams, double* dy0) {
  int P = tvo_param_count(m);
  if (P < 0 || B < 0 || N < 0) return TVO_BADARG;
  int n = m->n;
  size_t dp_len = m->per_series ? (size_t)B * P : (size_t)P;
  memset(dparams, 0, sizeof(double) * dp_len);
  int worst = TVO_OK;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
  nthreads = 1;
#endif
  /* shared parameters: one private accumulator per series, summed in series
   * order afterwards so the result does not depend on the thread count */
  double* acc = NULL;
  if (!m->per_series) acc = (double*)calloc((size_t)B * P, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(max : worst)
#endif
  for (int b = 0; b < B; ++b) {
    const double* p = m->per_series ? params + (size_t)b * P : params;
    double* gp = m->per_series ? dparams + (size_t)b * P : acc + (size_t)b * P;
    const double* tb = times + (size_t)b * (N + 1);
    const double* yb = y + (size_t)b * (N + 1) * n;
    const double* gb = grad_out + (size_t)b * (N + 1) * n;
    double* a = (double*)malloc(sizeof(double) * (2 * n + n * n));
    double* rhs = a + n;
    double* JT = rhs + n;
    for (int i = 0; i < n; ++i) a[i] = 0.0; /* a_{N+1} = 0 */
    for (int k = N; k >= 1; --k) {
      double dt = step_dt(tb, lengths, b, k);
      const double* yk = yb + (size_t)k * n;
      /* (I - dt j_k)^T a_k = a_{k+1} + dL/dy_k */
      for (int i = 0; i < n; ++i) rhs[i] = a[i] + gb[(size_t)k * n + i];
      double J[64 * 64];
      double* Jp = (n <= 64) ? J : (double*)malloc(sizeof(double) * n * n);
      tvo_jac(m, p, yk, tb[k], Jp);
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) JT[c * n + r] = (r == c ? 1.0 : 0.0) - dt * Jp[r * n + c];
      if (Jp != J) free(Jp);
      if (lu_solve(n, JT, rhs)) {
        if (TVO_SINGULAR > worst) worst = TVO_SINGULAR;
      }
      for (int i = 0; i < n; ++i) a[i] = rhs[i];
      /* dL/dp += dt_k (dh/dp)^T a_k */
      if (dt != 0.0) tvo_vjp_p(m, p, yk, tb[k], a, dt, gp);
    }
    if (dy0)
      for (int i = 0; i < n; ++i) dy0[(size_t)b * n + i] = a[i] + gb[i];
    free(a);
  }
  if (acc) {
    for (int b = 0; b < B; ++b)
      for (int q = 0; q < P; ++q) dparams[q] += acc[(size_t)b * P + q];
    free(acc);
  }
  return worst;
}

int tvo_forward_euler(const tvo_model* m, int B, int N, const double* y0, const double* times,
                      const int* lengths, const double* params, int nthreads, double* y,
                      int* status) {
  int P = tvo_param_count(m);
  if (P < 0 || B < 0 || N < 0) return TVO_BADARG;
  int n = m->n;
  int worst = TVO_OK;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(max : worst)
#endif
  for (int b = 0; b < B; ++b) {
    const double* p = m->per_series ? params + (size_t)b * P : params;
    const double* tb = times + (size_t)b * (N + 1);
    double* yb = y + (size_t)b * (N + 1) * n;
    double h[64];
    double* hp = (n <= 64) ? h : (double*)malloc(sizeof(double) * n);
    int st = TVO_OK;
    for (int i = 0; i < n; ++i) yb[i] = y0[(size_t)b * n + i];
    for (int k = 1; k <= N; ++k) {
      const double dt = step_dt(tb, lengths, b, k);
      const double* yp = yb + (size_t)(k - 1) * n;
      double* yk = yb + (size_t)k * n;
      tvo_rhs(m, p, yp, tb[k - 1], hp);
      for (int i = 0; i < n; ++i) {
        yk[i] = yp[i] + dt * hp[i];
        if (!isfinite(yk[i])) st = TVO_NONFINITE;
      }
    }
    if (hp != h) free(hp);
    if (status) status[b] = st;
    if (st > worst) worst = st;
  }
  return worst;
}

int tvo_adjoint_euler(const tvo_model* m, int B, int N, const double* times, const int* lengths,
                      const double* params, const double* y, const double* grad_out,
                      int nthreads, double* dparams, double* dy0) {
  int P = tvo_param_count(m);
  if (P < 0 || B < 0 || N < 0) return TVO_BADARG;
  int n = m->n;
  size_t dp_len = m->per_series ? (size_t)B * P : (size_t)P;
  memset(dparams, 0, sizeof(double) * dp_len);
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
  nthreads = 1;
#endif
  /* shared parameters: per-series accumulators summed in series order */
  double* acc = NULL;
  if (!m->per_series) acc = (double*)calloc((size_t)B * P, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
  for (int b = 0; b < B; ++b) {
    const double* p = m->per_series ? params + (size_t)b * P : params;
    double* gp = m->per_series ? dparams + (size_t)b * P : acc + (size_t)b * P;
    const double* tb = times + (size_t)b * (N + 1);
    const double* yb = y + (size_t)b * (N + 1) * n;
    const double* gb = grad_out + (size_t)b * (N + 1) * n;
    double* lam = (double*)malloc(sizeof(double) * (2 * n + n * n));
    double* nxt = lam + n;
    double* J = nxt + n;
    for (int i = 0; i < n; ++i) lam[i] = gb[(size_t)N * n + i]; /* lambda_N */
    for (int k = N; k >= 1; --k) {
      const double dt = step_dt(tb, lengths, b, k);
      const double* yp = yb + (size_t)(k - 1) * n;
      /* dL/dp += dt_k (dh/dp at y_{k-1})^T lambda_k */
      if (dt != 0.0) tvo_vjp_p(m, p, yp, tb[k - 1], lam, dt, gp);
      /* lambda_{k-1} = dL/dy_{k-1} + (I + dt_k j(y_{k-1}))^T lambda_k */
      tvo_jac(m, p, yp, tb[k - 1], J);
      for (int c = 0; c < n; ++c) {
        double s = lam[c];
        for (int r = 0; r < n; ++r) s += dt * J[r * n + c] * lam[r];
        nxt[c] = gb[(size_t)(k - 1) * n + c] + s;
      }
      for (int i = 0; i < n; ++i) lam[i] = nxt[i];
    }
    if (dy0)
      for (int i = 0; i < n; ++i) dy0[(size_t)b * n + i] = lam[i];
    free(lam);
  }
  if (acc) {
    for (int b = 0; b < B; ++b)
      for (int q = 0; q < P; ++q) dparams[q] += acc[(size_t)b * P + q];
    free(acc);
  }
  return TVO_OK;
}

int tvo_step_matrices(const tvo_model* m, int B, int N, const double* times, const int* lengths,
                      const double* params, const double* y, double* A) {
  int P = tvo_param_count(m);
  if (P < 0 || B < 0 || N < 0) return TVO_BADARG;
  int n = m->n;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int b = 0; b < B; ++b) {
    const double* p = m->per_series ? params + (size_t)b * P : params;
    const double* tb = times + (size_t)b * (N + 1);
    for (int k = 1; k <= N; ++k) {
      double dt = step_dt(tb, lengths, b, k);
      double* Ak = A + ((size_t)b * N + (k - 1)) * n * n;
      tvo_jac(m, p, y + ((size_t)b * (N + 1) + k) * n, tb[k], Ak);
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ak[r * n + c] = (r == c ? 1.0 : 0.0) - dt * Ak[r * n + c];
    }
  }
  return TVO_OK;
}
