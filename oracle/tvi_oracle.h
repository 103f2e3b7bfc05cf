/*
 * tvi_oracle.h -- CPU FP64 oracle for batched backward-Euler integration and
 * its discrete adjoint.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent checker of the
 * GPU path.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load it.  It shares no code, header, table or helper with
 * the CUDA library, and the CUDA library never calls it.
 *
 * What it computes (the plain definitions the chunked method reaches):
 *   forward  -- for every series b and every step k = 1..N, the root of the
 *               backward-Euler equation  y_k - y_{k-1} - dt_k h(y_k, t_k; p) = 0
 *               (paper Sec. 2.2, Eq. backward-euler), found by Newton's method
 *               from the previous-step guess y_{k-1} with the discrete Jacobian
 *               I - dt_k j(y_k), j = dh/dy (Sec. 2.2), each Newton system
 *               solved by dense LU with partial pivoting.
 *   adjoint  -- the exact gradient of a loss L(y_0..y_N) through those discrete
 *               equations (App. A.1, derived discrete form):
 *                 a_{N+1} = 0
 *                 (I - dt_k j(y_k))^T a_k = a_{k+1} + dL/dy_k,   k = N..1
 *                 dL/dp   = sum_k dt_k (dh/dp(y_k, t_k; p))^T a_k
 *                 dL/dy_0 = a_1 + dL/dy_0 (explicit part)
 *
 * Model right-hand sides h(y, t; p) (the ODE of Sec. 2.1, Eqs. 1-2):
 *   TVO_LINEAR    h = A y,                    p = A (n x n, row-major)
 *   TVO_VDP       h = [y2, mu (1 - y1^2) y2 - y1],   p = mu  (n = 2)
 *   TVO_MLP_TANH  h = tanh(W3 tanh(W2 tanh(W1 y + b1) + b2) + b3)
 *                 (the neural ODE of Sec. 5.1.1 without the forcing input)
 *   TVO_MLP_SILU  h = W3 silu(W2 silu(W1 y + b1) + b2) + b3
 *   TVO_MDS       mass-damper-spring chain of u = n/2 units (Sec. 5.1.1, Table
 *                 mass-params), y = [d_1..d_u, v_1..v_u],
 *                 p = [K_1..K_u, C_1..C_u, M_1..M_u, f_a, T]  (P = 3u + 2):
 *                   d_i' = v_i
 *                   v_i' = (F_i - F_{i-1}) / M_i + [i = 1] f_a sin(2 pi t / T)
 *                   F_i  = K_i (d_{i+1} - d_i) + C_i (v_{i+1} - v_i),
 *                 F_0 = 0 (free end, where the force acts) and d_{u+1} = v_{u+1} = 0
 *                 (the fixed end): spring and damper i join mass i to mass i+1.
 *   TVO_CHABOCHE  Chaboche viscoplasticity with u = n - 2 backstresses (Sec.
 *                 5.1.1, Table chaboche-params), y = [sigma, K, X_1..X_u],
 *                 p = [E, m, eta, sigma_0, K_inf, tau, C_1..C_u, g_1..g_u, ed_a, T]
 *                 (P = 2u + 8; m is the flow exponent the paper calls n):
 *                   s = sigma - sum X,  f = (|s| - K - sigma_0) / eta,
 *                   ep = max(f, 0)^m sign(s)            (plastic strain rate)
 *                   sigma' = E (ed_a sin(2 pi t / T) - ep)
 *                   K'     = tau (K_inf - K)
 *                   X_i'   = 2/3 C_i ep - g_i X_i |ep|
 *   TVO_NEURON    u = n / 4 coupled neurons (Sec. 5.1.1, Table neuron-params),
 *                 y = [V_1, m_1, h_1, n_1, V_2, ...], per neuron i the 15 values
 *                 p[15 i ..] = [C, gNa, ENa, gK, EK, gL, EL, m_inf, tau_m, h_inf,
 *                 tau_h, n_inf, tau_n, gC, T], then p[15 u] = I_a  (P = 15 u + 1):
 *                   V_i' = (-gNa m^3 h (V - ENa) - gK n^4 (V - EK) - gL (V - EL)
 *                           + I_a sin(2 pi t / T) + gC sum_j (V_i - V_j)) / C
 *                   m_i' = (m_inf - m) / tau_m   (h and n alike)
 * MLP parameter layout (flat, FP64): W1[h1][n] b1[h1] W2[h2][h1] b2[h2]
 * W3[n][h2] b3[n]; W are row-major (out x in).
 *
 * Array layouts (row-major, contiguous):
 *   y0 [B][n], times [B][N+1], lengths [B] (or NULL = all N steps real),
 *   params [B][P] when per_series else [P], y [B][N+1][n] with y[b][0] = y0[b],
 *   grad_out [B][N+1][n], dparams same shape as params, dy0 [B][n].
 * Steps k > lengths[b] are padding: their dt is taken as 0, so y_k = y_{k-1}.
 */
#ifndef TVI_ORACLE_H
#define TVI_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { TVO_LINEAR = 0, TVO_VDP = 1, TVO_MLP_TANH = 2, TVO_MLP_SILU = 3, TVO_MDS = 4,
       TVO_CHABOCHE = 5, TVO_NEURON = 6 };
enum { TVO_OK = 0, TVO_NOT_CONVERGED = 1, TVO_NONFINITE = 2, TVO_SINGULAR = 3, TVO_BADARG = -1 };

typedef struct {
  int kind;        /* TVO_LINEAR / TVO_VDP / TVO_MLP_TANH / TVO_MLP_SILU / TVO_MDS /
                      TVO_CHABOCHE / TVO_NEURON */
  int n;           /* state size */
  int h1, h2;      /* MLP hidden widths (ignored otherwise) */
  int per_series;  /* 1: params [B][P]; 0: one shared parameter vector [P] */
} tvo_model;

/* Number of parameters P of one parameter vector, or -1 on a bad model. */
int tvo_param_count(const tvo_model* m);

/* h(y, t; p) into h[n]. */
void tvo_rhs(const tvo_model* m, const double* p, const double* y, double t, double* h);
/* j = dh/dy into j[n][n] (row-major: j[r*n+c] = dh_r/dy_c). */
void tvo_jac(const tvo_model* m, const double* p, const double* y, double t, double* j);
/* gp[P] += scale * (dh/dp)^T a. */
void tvo_vjp_p(const tvo_model* m, const double* p, const double* y, double t,
               const double* a, double scale, double* gp);

/* Step-by-step backward-Euler Newton integration.  Per step, Newton stops when
 * ||G||_inf <= tol_abs or ||G||_inf <= tol_rel * ||G_0||_inf, or after
 * max_iter updates.  iters [B][N] (or NULL) receives the Newton updates taken
 * per step; status [B] (or NULL) receives TVO_OK / TVO_NOT_CONVERGED /
 * TVO_NONFINITE / TVO_SINGULAR for the series.  nthreads <= 0 uses the OpenMP
 * default.  Returns TVO_OK, TVO_BADARG, or the worst series status. */
int tvo_forward(const tvo_model* m, int B, int N, const double* y0, const double* times,
                const int* lengths, const double* params, double tol_abs, double tol_rel,
                int max_iter, int nthreads, double* y, int* iters, int* status);

/* Independent backward-Euler step solves: out[b][k] is the step k solution
 * from the given y_prev[b][k-1] (the same Newton and stopping rule as
 * tvo_forward), out[b][0] = y_prev[b][0].  status [B] (or NULL) receives the
 * worst step status of the series.  Returns TVO_OK, TVO_BADARG or the worst
 * status. */
int tvo_step_solves(const tvo_model* m, int B, int N, const double* times, const int* lengths,
                    const double* params, const double* y_prev, double tol_abs, double tol_rel,
                    int max_iter, int nthreads, double* out, int* status);

/* Discrete adjoint of tvo_forward's equations at the trajectory y.  Writes
 * dparams (zeroed first) and dy0 (may be NULL). */
int tvo_adjoint(const tvo_model* m, int B, int N, const double* times, const int* lengths,
                const double* params, const double* y, const double* grad_out, int nthreads,
                double* dparams, double* dy0);

/* Forward Euler (Sec. 2.2, explicit methods): y_k = y_{k-1} + dt_k h(y_{k-1},
 * t_{k-1}), step by step; padded steps (dt_k = 0) keep the state.  Returns
 * TVO_OK, TVO_BADARG or TVO_NONFINITE (status [B] may be NULL). */
int tvo_forward_euler(const tvo_model* m, int B, int N, const double* y0, const double* times,
                      const int* lengths, const double* params, int nthreads, double* y,
                      int* status);

/* Discrete adjoint of tvo_forward_euler's recursion at the trajectory y, written
 * out from the chain rule: lambda_N = dL/dy_N,
 *   lambda_k = dL/dy_k + (I + dt_{k+1} j(y_k))^T lambda_{k+1}   (k = N-1 .. 0),
 *   dL/dp = sum_{k=1..N} dt_k (dh/dp at y_{k-1})^T lambda_k,  dL/dy0 = lambda_0.
 * Writes dparams (zeroed first) and dy0 (may be NULL). */
int tvo_adjoint_euler(const tvo_model* m, int B, int N, const double* times, const int* lengths,
                      const double* params, const double* y, const double* grad_out,
                      int nthreads, double* dparams, double* dy0);

/* Step matrices A_k = I - dt_k j(y_k) of every series and step k = 1..N at a
 * given trajectory y, into A [B][N][n][n] (dt_k = 0 on padded steps).  Used to
 * propagate perturbations through the linearised backward-Euler recursion
 * (forward-error estimates in the tests). */
int tvo_step_matrices(const tvo_model* m, int B, int N, const double* times, const int* lengths,
                      const double* params, const double* y, double* A);

/* Threads OpenMP will use for nthreads <= 0. */
int tvo_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
