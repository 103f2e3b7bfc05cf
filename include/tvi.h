/*
 * tvi.h -- C ABI of the time-vectorized implicit integrator (sm_103a).
 *
 * Batched backward-Euler integration of dy/dt = h(y, t; p) over n_batch
 * independent series (paper Sec. 2.1, Eqs. 1-4), vectorized over a chunk of
 * sequential time steps (Sec. 2.3): each Newton iteration assembles the
 * residual of Eq. batched-backward-euler and the block lower-bidiagonal Jacobian
 * (diagonal I - dt_k j_k, sub-diagonal -I; Eq. batched-update) for every
 * (series, step) pair of the chunk and solves it by parallel cyclic reduction
 * (Sec. 3.2, Alg. 3).  The adjoint (App. A.1-A.2) solves the transposed,
 * reversed block-bidiagonal system chunk by chunk and forms dL/dparams.
 *
 * Conventions shared by every entry point:
 *   - All array pointers are DEVICE pointers unless stated otherwise, row-major
 *     and contiguous, FP64 unless stated otherwise, and 16-byte aligned (as
 *     every cudaMalloc or PyTorch allocation is; the workspace and, for the
 *     MLP models, grad_out are checked).  The caller owns every buffer; the
 *     library allocates no device memory and keeps no pointer after a call
 *     returns.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All work is
 *     enqueued on it.  A call synchronises `stream` only when it must read a
 *     result back to form its return code (see tvi_options.sync_status).
 *   - Errors are returned, never raised: no call aborts, traps or prints.  The
 *     text of the last error of the calling host thread is tvi_last_error().
 *   - rhs/jac are chosen by tvi_model.kind: a built-in model, or a user model
 *     whose rhs/jac are device source compiled at run time (tvi_user_model_create).
 */
#ifndef TVI_H
#define TVI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TVI_OK = 0,
  TVI_EINVAL = -1,        /* bad argument: sizes, NULL pointer, unsupported combination */
  TVI_EWORKSPACE = -2,    /* workspace NULL or smaller than tvi_workspace_bytes() */
  TVI_ECUDA = -3,         /* a CUDA runtime call failed (text in tvi_last_error) */
  TVI_ENOTCONV = -4,      /* some series hit the Newton iteration limit on a one-step chunk */
  TVI_ENONFINITE = -5,    /* some series produced a NaN/Inf residual on a one-step chunk */
  TVI_ETIMEOUT = -6,      /* a bounded device wait gave up (tensor-core path); results invalid.
                             Test hook: a non-negative integer in the environment variable
                             TVI_TEST_TC_FIRST_WAIT_POLLS bounds the first data wait of each
                             tensor-core block at that many polls (0: gives up at once), read
                             at every launch; unset, the full limit applies.  (A second test
                             hook, TVI_TEST_PER_PAIR_FIRST_PASS=1, makes the neural-ODE
                             forward evaluate an attempt's first residual per step instead
                             of once per series; results are the same bit for bit.) */
  TVI_EUNSUPPORTED = -7   /* model/precision/size combination not built */
} tvi_status;

/* Model right-hand sides h(y, t; p) (autonomous: t is accepted, not used).
 *   TVI_MODEL_LINEAR    h = A y; p = A [n][n] (row-major).  n in {2, 4}.
 *   TVI_MODEL_VDP       van der Pol: h = [y2, mu (1 - y1^2) y2 - y1]; p = [mu].  n = 2.
 *   TVI_MODEL_MLP_TANH  h = tanh(W3 tanh(W2 tanh(W1 y + b1) + b2) + b3)  (the neural
 *                       ODE of Sec. 5.1.1 without forcing input).
 *   TVI_MODEL_MLP_SILU  h = W3 silu(W2 silu(W1 y + b1) + b2) + b3.
 * MLP parameters are one flat FP64 vector W1[h1][n] b1[h1] W2[h2][h1] b2[h2]
 * W3[n][h2] b3[n] (W row-major, out x in), shared by all series (per_series =
 * 0); n in {4, 8, 16, 32}, hidden widths <= 128 and multiples of 4.
 *   TVI_MODEL_USER      h, dh/dy and (dh/dp)^T a given as device source
 *                       (tvi_user_model_create); n and P are the user model's,
 *                       and tvi_model.user points at it. */
typedef enum {
  TVI_MODEL_LINEAR = 0,
  TVI_MODEL_VDP = 1,
  TVI_MODEL_MLP_TANH = 2,
  TVI_MODEL_MLP_SILU = 3,
  TVI_MODEL_USER = 4
} tvi_model_kind;

/* Arithmetic of the block Jacobian, its inverse and the cyclic reduction.
 * The Newton residual, its norm, the Newton update and every output stay in
 * FP64 in all modes, so Newton acts as iterative refinement and converges to
 * the FP64 solution of the discrete equations. */
typedef enum {
  TVI_PREC_FP64 = 0,
  TVI_PREC_FP32 = 1,
  TVI_PREC_BF16 = 2       /* MLP models with n in {16, 32}: Jacobian products on the
                             tensor cores in BF16 with FP32 accumulation, block inverse
                             by a tensor-core Neumann series (Gauss-Jordan when
                             ||dt D3 J||_1 > 1/8), chain in FP32 */
} tvi_precision;

/* Time-integration scheme (Sec. 2.2).  Backward Euler: y_k - y_{k-1} -
 * dt_k h(y_k) = 0, Newton on the chunk's implicit equations.  Forward Euler:
 * y_k - y_{k-1} - dt_k h(y_{k-1}) = 0; chunked the same way, its chunk system has
 * identity diagonal blocks and sub-diagonal -(I + dt_k j(y_{k-1})), so each
 * Newton update is the same scan with no block inverse, and its adjoint is
 * a_k = dL/dy_k + (I + dt_{k+1} j(y_k))^T a_{k+1}, dL/dp = sum_k dt_k
 * (dh/dp at y_{k-1})^T a_k, dL/dy0 = dL/dy_0 + (I + dt_1 j(y_0))^T a_1. */
typedef enum { TVI_BACKWARD_EULER = 0, TVI_FORWARD_EULER = 1 } tvi_scheme;

/* A user model compiled at run time (opaque; tvi_user_model_create). */
typedef struct tvi_user_model tvi_user_model;

typedef struct {
  int kind;        /* tvi_model_kind */
  int n;           /* state size */
  int hidden1;     /* MLP hidden widths (0 otherwise) */
  int hidden2;
  int per_series;  /* 1: params [B][P] (one vector per series); 0: one shared [P] */
  const tvi_user_model* user;  /* TVI_MODEL_USER: the compiled model (n must be its n);
                                  ignored for the other kinds */
} tvi_model;

typedef struct {
  int chunk;          /* steps solved together (n_chunk, Sec. 2.3); >= 1 */
  double tol_abs;     /* Newton stops for a series when ||R||_inf <= tol_abs ... */
  double tol_rel;     /* ... or ||R||_inf <= tol_rel ||R_0||_inf (norm over the whole chunk) */
  int max_iter;       /* Newton update limit per chunk attempt */
  int precision;      /* tvi_precision */
  int retry_halving;  /* 1: a chunk whose Newton fails is re-solved by halves.  Small-state
                         engine (linear, van der Pol, user models with n <= 4): a failure
                         (limit, non-finite, or residual still > 10x its start after 4
                         updates) keeps the attempt's longest leading run of >= 8 steps
                         whose residuals are within the tolerance (those steps are solved),
                         and the rest is re-solved with half the steps, recursively down to
                         one step; after two successes in a row the chunk doubles back up
                         to `chunk`.  Large-state engines (MLP and user models with n > 4,
                         all series in lockstep): the series whose attempt hit the limit or
                         a non-finite residual re-solve the same steps as two halves,
                         recursively down to one step, while the others go on.  Every kept
                         step satisfies the same equation to the same tolerance. */
  int adjoint_refine; /* FP64-residual refinement sweeps of each adjoint chunk solve
                         (used when precision != FP64) */
  int rows_per_thread;/* solver tiling: steps held by one thread (0 = automatic) */
  int sync_status;    /* 1: synchronise `stream` and fold per-series status into the
                         return code; 0: return TVI_OK after enqueueing (status only
                         in the series_status array) */
  const float* predictor;  /* learned Newton predictor (van der Pol model only), packed
                              as tvi_predictor_* describe, device; NULL = dy = 0 guess */
  int predictor_chunk;     /* steps the predictor proposes (its output is 2 x this);
                              used for chunk attempts of exactly this length */
  int predictor_hidden;    /* hidden width of the predictor MLP (even, <= 256) */
  int scheme;              /* tvi_scheme: TVI_BACKWARD_EULER (default) or
                              TVI_FORWARD_EULER (every model with FP64 or FP32 blocks;
                              not with BF16 blocks or a predictor) */
} tvi_options;

/* Fill *opt with defaults: chunk 1, tol_abs 1e-8, tol_rel 0, max_iter 50, FP64,
 * retry_halving 1, adjoint_refine 2, rows_per_thread 0, sync_status 1, no
 * predictor, backward Euler. */
void tvi_default_options(tvi_options* opt);

/* Number of parameters P of one parameter vector, or -1 for a bad model. */
int tvi_param_count(const tvi_model* model);

/* Device workspace (bytes) that tvi_integrate / tvi_adjoint need for B series
 * of N steps.  The caller allocates it (alignment 256 B) and may reuse it for
 * any later call with the same or smaller sizes. */
size_t tvi_workspace_bytes(const tvi_model* model, const tvi_options* opt, int B, int N);

/* Steps one chunk attempt holds for this model and these options over N steps
 * (Sec. 2.3, n_chunk as actually solved), or -1 for a bad model or options.  The
 * small-state engine (linear, van der Pol, user models with n <= 4) keeps a
 * chunk on one multiprocessor and solves at most 1024 steps together: a larger
 * opt->chunk runs as 1024-step chunks, which solve the same equations to the
 * same tolerance.  Every engine also stops at N. */
int tvi_effective_chunk(const tvi_model* model, const tvi_options* opt, int N);

/*
 * Forward integration, chunked backward (or forward, opt->scheme) Euler with
 * Newton (Alg. 1).
 *   B, N        series and steps; times has N+1 entries per series.
 *   y0          [B][n]       initial states.
 *   times       [B][N+1]     per-series time points; dt_k = t_k - t_{k-1} (Sec. 2.2).
 *   lengths     [B] int32 or NULL.  Steps k > lengths[b] are padding: dt_k = 0, so
 *               y_k = y_{k-1} exactly.
 *   params      [B][P] or [P] (tvi_model.per_series).
 *   y_out       [B][N+1][n]  trajectory; y_out[b][0] = y0[b] (like scipy odeint).
 *   stats       [B][6] int32 or NULL: total Newton updates, chunks solved,
 *               chunk retries (halvings), largest Newton count of one chunk,
 *               chunks started from the predictor's guess, predictor guesses
 *               rejected because their residual was not below the dy = 0 one.
 *   series_status [B] int32 or NULL: 0 ok, 1 Newton limit, 2 non-finite residual,
 *               3 (every series) a bounded device wait of the tensor-core path gave up.
 *   workspace   >= tvi_workspace_bytes(model, opt, B, N) bytes of device memory.
 * Newton starts every chunk from dy = 0 (Sec. 2.3) and stops per series (Alg. 1,
 * converged series are frozen).  With opt->predictor, a chunk attempt of
 * predictor_chunk steps starts from the predictor's guess instead when the
 * guess's FP64 residual infinity-norm is below that of dy = 0; after k
 * rejected guesses in a row (k <= 5) the series skips the predictor on its next
 * 2^k - 1 eligible chunks, and an accepted guess resets k.  A failed chunk is
 * retried as opt->retry_halving describes; otherwise, or on a one-step chunk,
 * the series' status is set and its integration continues from the
 * unconverged iterate.
 * Returns TVI_OK, an argument error, or (sync_status = 1) TVI_ENOTCONV /
 * TVI_ENONFINITE if any series failed, TVI_ETIMEOUT if a bounded device wait of
 * the tensor-core path gave up.
 */
tvi_status tvi_integrate(const tvi_model* model, const tvi_options* opt, int B, int N,
                         const double* y0, const double* times, const int* lengths,
                         const double* params, double* y_out, int* stats, int* series_status,
                         void* workspace, size_t workspace_bytes, void* stream);

/*
 * Discrete adjoint of tvi_integrate's equations (App. A.1, chunked per App. A.2).
 *   y           [B][N+1][n]  the trajectory tvi_integrate produced (checkpoint: the
 *               Jacobians are recomputed from it, nothing else is kept).
 *   grad_out    [B][N+1][n]  dL/dy_k for every output, including k = 0.
 *   dparams     [B][P] or [P] output: dL/dp = sum_k dt_k (dh/dp(y_k))^T a_k, where
 *               a solves (I - dt_k j(y_k))^T a_k = a_{k+1} + dL/dy_k, a_{N+1} = 0
 *               (backward Euler; forward Euler: see tvi_scheme).
 *   dy0         [B][n] output or NULL: dL/dy0 = a_1 + dL/dy_0.
 * The adjoint chunk size is opt->chunk; opt->scheme must match the forward pass.
 * With FP32 / BF16 blocks the chunk solves are refined opt->adjoint_refine
 * times with FP64-assembled residuals.  Returns TVI_OK or an argument error;
 * on the tensor-core path a bounded device wait that gave up leaves NaN in
 * dparams and dy0.
 */
tvi_status tvi_adjoint(const tvi_model* model, const tvi_options* opt, int B, int N,
                       const double* times, const int* lengths, const double* params,
                       const double* y, const double* grad_out, double* dparams, double* dy0,
                       void* workspace, size_t workspace_bytes, void* stream);

/*
 * tvi_adjoint without a workspace, for callers that cannot allocate device
 * memory (code where cudaMalloc is unavailable or forbidden: a host callback or
 * real-time loop that must not enter the allocator, a plugin whose host owns
 * every allocation, a process whose allocator has reserved the whole device).
 * The paper has no counterpart: this is an interface convenience.
 *
 * Arguments and results are those of tvi_adjoint, minus the workspace.  The
 * per-series partial gradients of shared parameters live instead in a fixed
 * 4 MiB array inside the library's device image, which every GPU where it is
 * used holds until the process exits; B * P > 524,288 with shared
 * parameters (per_series = 0) is rejected with TVI_EINVAL.  Per-series
 * parameters need no scratch.  The call allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine.
 *
 * With lazy module loading (the CUDA default) the 4 MiB is committed on the first
 * call on each device rather than when the library loads: a caller whose
 * allocator will reserve the whole device should make that first call before
 * it does.  The first call in each CUDA context also looks up the array's
 * device address (cudaGetSymbolAddress, with that context's device current);
 * make it before any stream capture.  A context created after cudaDeviceReset
 * gets its own lookup.  All calls share the one array: calls whose work
 * overlaps on the GPU (other streams, other host threads) race on it and must
 * be serialised by the caller.  Every call overwrites the entries it reads, so
 * nothing from an earlier call leaks into a later result.
 */
tvi_status tvi_adjoint_noalloc(const tvi_model* model, const tvi_options* opt, int B, int N,
                               const double* times, const int* lengths, const double* params,
                               const double* y, const double* grad_out, double* dparams,
                               double* dy0, void* stream);

/*
 * Learned Newton predictor (an MLP over the chunk-start state, the model
 * parameter and the chunk's step sizes that proposes the chunk's increments
 * dy_1..dy_c as Newton's starting guess).  Newton still runs to the same
 * tolerance from that guess, so results do not change; only the iteration
 * count does.  The paper starts every chunk at dy = 0 (Sec. 2.3); it has no
 * predictor.
 *
 * Packed FP32 vector (in features, H hidden, out outputs):
 *   mean[in] std[in] scale[out] W1[H][in] b1[H] W2[H][H] b2[H] W3[out][H] b3[out]
 * network(x) = W3 silu(W2 silu(W1 (x - mean) / std + b1) + b2) + b3, and the
 * predictor's output is network(x) * scale.  For the van der Pol model with a
 * c-step predictor: in = 3 + c with x = (y1, y2, log10 mu, log10 dt_1..dt_c)
 * (dt floored at 1e-30), out = 2 c slopes s_j = (out[2(j-1)], out[2(j-1)+1]),
 * and the guess is dy_j = sum_{l <= j} dt_l s_l.
 */

/* Floats in the packed vector, or -1 for bad sizes (H even, <= 1024). */
int tvi_predictor_size(int in, int hidden, int out);

/* Batched inference: x [M][in] raw features -> y [M][out] outputs (device). */
tvi_status tvi_predictor_forward(const float* packed, int in, int hidden, int out, int M,
                                 const float* x, float* y, void* stream);

/* Device workspace for tvi_predictor_train_step with batch M. */
size_t tvi_predictor_workspace_bytes(int in, int hidden, int out, int M);

/*
 * One Adam step (Kingma & Ba 2015: beta1 0.9, beta2 0.999, eps 1e-8, bias
 * correction with step >= 1) on the trained part (W1..b3) of `packed`, for the
 * mean squared error between network(x) and target / scale over a batch of M
 * samples: sample m is row rows[m] of x [*][in] and target [*][out] (rows NULL:
 * row m).  adam_m, adam_v: moment vectors, size tvi_predictor_size - (2 in +
 * out), zeroed before step 1.  loss: device float receiving the batch loss.
 */
tvi_status tvi_predictor_train_step(float* packed, float* adam_m, float* adam_v, int in, int hidden,
                                    int out, int M, const float* x, const float* target,
                                    const int* rows, float lr, int step, float* loss,
                                    void* workspace, size_t workspace_bytes, void* stream);

/*
 * User-defined models.  The integrator of Sec. 2.2 takes the right-hand side h
 * and its Jacobian j = dh/dy as functions; here they are CUDA C++ device source,
 * compiled at run time (NVRTC, sm_103a) together with kernel templates: for
 * n <= 4 the fused small-state solver, so they run inlined in the same
 * one-block-per-series kernels as the built-in linear and van der Pol models;
 * for 5 <= n <= 40 the large-state kernels (a thread per (series, step) for the
 * residual, up to a warp per step for the Jacobian block and its inverse) around
 * the chunk solve of the MLP engine.  `source` defines, at global scope, with
 * TVI_N (= n) and TVI_P (= P) #defined before it:
 *
 *   __device__ void tvi_rhs(const double* y, double t, const double* p, double* h);
 *       h[i] = h_i(y, t; p), i < n: the ODE dy/dt = h(y, t; p) (Sec. 2.1)
 *   __device__ void tvi_jac(const double* y, double t, const double* p, double* J);
 *       J[i * n + j] = dh_i/dy_j: the step Jacobian of step k is I - dt_k J
 *   __device__ void tvi_vjp_p(const double* y, double t, const double* p,
 *                             const double* a, double* g);
 *       g[q] = sum_i a_i dh_i/dp_q, q < P: the adjoint's gradient integrand
 *       (App. A.1)
 *
 * y and p hold n and P values, a holds n, t is the time of the evaluation (t_k
 * for backward Euler's step k, t_{k-1} for forward Euler's); h, J and g must be
 * written in full.  tvi_rhs and tvi_vjp_p are evaluated in FP64.  tvi_jac may
 * instead be a template over the element type of y and J,
 *   template <typename T>
 *   __device__ void tvi_jac(const T* y, double t, const double* p, T* J);
 * and is then evaluated in the block type (FP32 with FP32 blocks, as for the
 * built-in models); a plain FP64 tvi_jac is evaluated in FP64 and rounded.
 * The library trusts them: J must be the Jacobian of h for Newton to converge
 * quadratically, and g its parameter product for the gradients to be those of
 * the discrete loss.  Sizes 1 <= n <= 40; 1 <= P <= 32 for n <= 4, 1 <= P <= 160
 * above (more than 32 are read from memory, not held in registers); FP64 or FP32
 * blocks (BF16: TVI_EUNSUPPORTED); per-series or shared parameters; no Newton
 * predictor; both schemes; retry_halving.  n <= 4 also has tvi_adjoint_noalloc;
 * n > 4 needs the workspace of tvi_workspace_bytes and rejects
 * tvi_adjoint_noalloc (TVI_EUNSUPPORTED).  Calls on one model from several host
 * threads are safe.  The paper has no counterpart to
 * run-time compilation: it is how an ABI of plain pointers accepts functions.
 */

/* Check that `source` (host string, copied) compiles against the interface
 * above and create a model.  Needs NVRTC (libnvrtc.so.13) but no GPU.
 * TVI_EINVAL: bad sizes, or source that does not compile (compiler log in
 * tvi_last_error); TVI_EUNSUPPORTED: NVRTC cannot be loaded.  *out is set only
 * on TVI_OK. */
tvi_status tvi_user_model_create(int n, int P, const char* source, tvi_user_model** out);

/* Compile the solver kernels of one block precision (TVI_PREC_FP64 or
 * TVI_PREC_FP32) now: every steps-per-thread tiling (n <= 4), or the
 * large-state kernels (n > 4).  Otherwise they are compiled (about a second
 * each) and loaded by the first tvi_integrate or tvi_adjoint that needs them;
 * do that first call, or this one, before any stream capture.  No GPU needed. */
tvi_status tvi_user_model_prepare(tvi_user_model* model, int precision);

/* Free the model and unload its kernels, after all work using it has completed.
 * NULL is ignored. */
void tvi_user_model_destroy(tvi_user_model* model);

/* Text of the last error on the calling host thread ("" if none). */
const char* tvi_last_error(void);

/* Kernels this library has enqueued since it was loaded, over every host thread
 * (a benchmark reads it before and after a region to count that region's
 * launches).  The paper has no counterpart. */
unsigned long long tvi_kernel_launches(void);

/* Library build identification, e.g. "tvi sm_103a". */
const char* tvi_version(void);

#ifdef __cplusplus
}
#endif
#endif
