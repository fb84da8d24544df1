/*
 * tdb.h - C ABI of libtdb, a GB300 (sm_103a) implementation of the in-situ
 * compressor of Zamani Ashtiani, Malik and Babaee, "Scalable in situ
 * compression of transient simulation data using time-dependent bases".
 *
 * A p-mode snapshot V(t) (p = 2..4 on the GPU) is approximated by a core T
 * (r_1 x ... x r_p) and W-orthonormal bases U_n (N_n x r_n):
 *     V ~ T x_1 U_1 x_2 ... x_p U_p                            (Eq. 2.5)
 * and streamed through the evolution equations with gauge phi = 0
 * (Eqs. 2.15, 2.16), advanced by explicit Euler with the first-order data
 * difference (Sec. 2.3), with the add/remove-mode control of Sec. 2.5.
 *
 * Conventions for every entry point
 *  - Layout: column-major, mode 1 fastest.  Element (i_1..i_p) of an N_1 x ..
 *    x N_p tensor is at offset sum_n i_n prod_{m<n} N_m; this equals a
 *    C-contiguous array of shape (N_p, ..., N_1).  U_n is N_n x r_n column-major
 *    (U[i + N_n a]); the core is r_1 x ... x r_p column-major.
 *  - Snapshot element type: double in TDB_FP64 mode, float otherwise.
 *  - Device pointers are CUDA device (or managed) memory of the current device;
 *    host pointers are ordinary host memory.  Every call is ordered on the
 *    stream given to tdb_init; calls that return host data synchronise it.
 *  - Memory: the library allocates no device memory.  The caller allocates a
 *    workspace of tdb_workspace_bytes() bytes (256-byte aligned) and owns it;
 *    it must outlive the context.  The context struct itself is host memory
 *    owned by the library (freed by tdb_destroy).
 *  - Snapshot buffers stay owned by the caller.  tdb_push_snapshot keeps a
 *    pointer to the last pushed snapshot as "previous" until the next push
 *    returns, so the caller must not modify that buffer until then (ping-pong
 *    two buffers).  tdb_init keeps V0 the same way.
 *  - Errors: every function returns a tdb_status and never throws.  A message
 *    for the last failure is in tdb_last_error().  CUDA errors are reported as
 *    TDB_ERR_CUDA; device-side conditions (non-finite data, failed Cholesky)
 *    are reported by the call that observes them.
 */
#ifndef TDB_H
#define TDB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TDB_MAX_MODES 4
#define TDB_MAX_RANK 32

typedef enum tdb_status {
  TDB_OK = 0,
  TDB_ERR_INVALID_ARG = 1,     /* null pointer, bad enum, bad threshold */
  TDB_ERR_SHAPE = 2,           /* ndim outside 2..4, >= 2^31 elements, or a mode of more than 1024
                                  points that is neither the first nor the last, or whose other
                                  modes hold more than 1024 points together */
  TDB_ERR_RANK = 3,            /* a rank outside 1..min(N_n, prod_{m!=n} r_m, TDB_MAX_RANK) */
  TDB_ERR_RANK_DEFICIENT = 4,  /* T_(n) T_(n)^T or U^T W U not positive definite */
  TDB_ERR_NONFINITE = 5,       /* NaN or Inf in a snapshot or in the state */
  TDB_ERR_CUDA = 6,            /* a CUDA runtime call failed */
  TDB_ERR_TIMEOUT = 7,         /* a bounded device-side wait ran out */
  TDB_ERR_STATE = 8,           /* call out of order (e.g. push before init) */
  TDB_WARN_RANK_CAP = 9,       /* error above eps_th with every rank at its cap */
  TDB_ERR_WORKSPACE = 10,      /* workspace null, too small or misaligned */
  TDB_ERR_UNSUPPORTED = 11     /* configuration not built (see tdb_config) */
} tdb_status;

/* Arithmetic of the projection pass (Eqs. 2.15, 2.16). */
enum tdb_precision {
  TDB_FP64 = 0,       /* double snapshots; every step in double (parity mode) */
  TDB_FP32 = 1,       /* float snapshots; unfused CUDA-core kernels, float products */
  TDB_BF16_TTM = 2    /* float snapshots; fused difference + projection on the tensor
                         cores (bf16 operands, fp32 accumulation), fp64 small algebra.
                         Where N_1 is not a multiple of 4 (TMA needs 16-byte row strides) the
                         step first copies V_{k+1} and V_k into zero-padded rows of the
                         workspace (two extra snapshot-sized buffers, an extra read and write
                         of both snapshots per projection pass). */
};

/* When the exact error of Eq. 2.20 is evaluated. */
enum tdb_error_mode {
  TDB_ERRMODE_EXACT = 0,     /* every step */
  TDB_ERRMODE_EVERY_K = 1,   /* every error_every steps */
  TDB_ERRMODE_MLP = 2,       /* when the learned estimator cannot rule out eps > eps_th */
  TDB_ERRMODE_NONE = 3       /* never (fixed rank, no control) */
};

/* Time integrator of the evolution equations (Eqs. 2.15, 2.16) with the snapshot difference
   Delta V = V_{k+1} - V_k as the data forcing (first-order forward difference, Sec. 2.3). */
enum tdb_integrator {
  TDB_EULER = 0,      /* explicit Euler: one projection pass per snapshot */
  TDB_HEUN = 1,       /* Heun's second-order Runge-Kutta scheme (Sec. 3.1 compares it with
                         Euler): the Euler increment at the state of step k gives a predicted
                         state, the increment there a second one, and the step takes their
                         mean.  Both stages use Delta V (the piecewise-linear interpolant of
                         the snapshots); the predicted state is not re-orthonormalised.  Two
                         projection passes and two fused updates per snapshot. */
  TDB_RK2_CENTRAL = 2 /* the midpoint second-order Runge-Kutta scheme with second-order
                         central differences of the data (Sec. 3.1): stage 1 takes
                         dt V'(t_k) ~ (V_{k+1} - V_{k-1}) / 2 over half a step to the midpoint
                         state, stage 2 takes dt V'(t_k + dt/2) ~ V_{k+1} - V_k at the midpoint
                         state over the whole step from the state of step k.  The first step
                         after an (re)initialisation, a state load or tdb_adapt_rank uses
                         (V_{k+1} - V_k) / 2 in stage 1.  Keeps the last TWO pushed snapshots
                         borrowed (V_{k-1} and V_k must stay unmodified until the next push
                         returns); tdb_push_snapshot only (input slots and batches refuse it
                         with TDB_ERR_UNSUPPORTED).  Two projection passes and two fused
                         updates per snapshot. */
};

typedef struct tdb_config {
  int ndim;                         /* p, 2..TDB_MAX_MODES */
  int64_t dims[TDB_MAX_MODES];      /* N_n, mode 1 fastest.  Modes of up to 1024 points; the
                                       first or the last mode may be longer when the product
                                       of the others is at most 1024 (a grouped spatial mode,
                                       Sec. 3.2): its HOSVD then comes from the short side,
                                       the Gram of the other modes' merged index, whose
                                       eigenvalues are C_n's nonzero ones and whose
                                       eigenvectors z map to C_n's as B z / sqrt(lambda). */
  int rank[TDB_MAX_MODES];          /* initial r_n; 0 = from gamma_th on the HOSVD spectrum */
  int rank_max[TDB_MAX_MODES];      /* cap on r_n (<= TDB_MAX_RANK); 0 = TDB_MAX_RANK */
  const double* weights[TDB_MAX_MODES]; /* host, length N_n: diagonal of W^(n) (Eq. 2.17);
                                       NULL = identity.  Copied by tdb_init. */
  double eps_th;                    /* epsilon_th of Sec. 2.5; <= 0 disables rank control */
  double gamma_th;                  /* gamma_th in percent (Eq. 2.21), e.g. 99.999 */
  int slope_window;                 /* K: steps of the error-slope test (Sec. 2.5); 0 = 10 */
  int precision;                    /* enum tdb_precision */
  int error_mode;                   /* enum tdb_error_mode */
  int error_every;                  /* period for TDB_ERRMODE_EVERY_K and the estimator's
                                       forced exact checks; 0 = 1 */
  int reorth;                       /* 1 = weighted Cholesky-QR of U_n after each step
                                       (recommended; the paper is silent), 0 = off */
  int integrator;                   /* enum tdb_integrator; TDB_EULER (0) unless set */
} tdb_config;

/* Per-step report (host struct filled by tdb_push_snapshot). */
typedef struct tdb_step_info {
  int64_t step;                     /* snapshots pushed since init */
  double eps;                       /* exact error after the step and any control (Eq. 2.20),
                                       or the estimate when eps_exact == 0 */
  int eps_exact;                    /* 1 = exact evaluation this step, 0 = estimate / none */
  double eps_step;                  /* exact error of the time step (Euler or Heun) before
                                       control acted */
  double gamma[TDB_MAX_MODES];      /* gamma^(n)(r_n) in percent (Eq. 2.21, second form) */
  double sigma_min[TDB_MAX_MODES];  /* smallest singular value of T_(n) (Eq. 2.18) */
  int ranks[TDB_MAX_MODES];         /* r_n after the step */
  int reinit;                       /* HOSVD re-initialisations performed this step */
  int action;                       /* 0 none, 1 reinit, 2 increase, 3 decrease, 4 revert, 5 cap */
  double cr;                        /* compression ratio CR of Sec. 2.6 at the new ranks */
  double dv_norm;                   /* ||V_{k+1} - V_k||_W */
  double ds_norm;                   /* ||dS||_F (the core increment) */
  double eps_est;                   /* the learned estimate of eps (NaN when no estimator is fitted) */
  int gate;                         /* why the exact error ran under TDB_ERRMODE_MLP: bit 0 estimate above
                                       the gate, bit 1 error_every steps without one, bit 2 a feature
                                       outside the training range; 0 = skipped */
} tdb_step_info;

typedef struct tdb_ctx tdb_ctx;

/* Bytes of device workspace needed for cfg (sized for rank_max).  0 on a bad cfg. */
size_t tdb_workspace_bytes(const tdb_config* cfg);

/* Initialise by truncated HOSVD of V0 (Sec. 2.3 last paragraph; ranks by gamma_th,
 * Sec. 2.5).  V0: device snapshot in the layout of tdb_push_snapshot, borrowed the same
 * way.  workspace: device, 256-byte aligned, >= tdb_workspace_bytes(cfg) bytes, owned by
 * the caller and outliving the context.  stream: cudaStream_t (NULL = legacy default).
 * On success *ctx owns nothing on the device but its view of workspace.  Errors:
 * TDB_ERR_INVALID_ARG / TDB_ERR_SHAPE / TDB_ERR_RANK (cfg), TDB_ERR_WORKSPACE,
 * TDB_ERR_UNSUPPORTED (a shape the tensor-core projection does not take, in
 * TDB_BF16_TTM), TDB_ERR_NONFINITE, TDB_ERR_TIMEOUT, TDB_ERR_CUDA; the message is in
 * tdb_last_error(NULL). */
tdb_status tdb_init(tdb_ctx** ctx, const tdb_config* cfg, void* workspace, size_t workspace_bytes,
                    const void* V0, void* stream);

/* Initialise from given factors instead of the HOSVD (for parity runs that start
 * from a known state).  core: host double r_1..r_p column-major; U[n]: host double
 * N_n x r_n column-major; ranks: host int[p].  V0 as for tdb_init. */
tdb_status tdb_init_from_factors(tdb_ctx** ctx, const tdb_config* cfg, void* workspace,
                                 size_t workspace_bytes, const double* core,
                                 const double* const* U, const int* ranks, const void* V0,
                                 void* stream);

/* One step of the compressor with the next snapshot (device pointer, prod N_n elements
 * of the snapshot type, storage order (N_p, ..., N_1) with mode 1 fastest):
 * difference, fused projection (Eqs. 2.15, 2.16), pseudo-inverse and complement
 * projection (Sec. 2.2), the time step of cfg.integrator (Euler, or Heun's two
 * stages), re-orthonormalisation, error (Eq. 2.20) per error_mode, and rank control
 * (Sec. 2.5).  V_next is borrowed: it becomes the previous snapshot and must stay
 * unmodified until the next push returns.  info (host, nullable) receives the report;
 * the call synchronises the stream.  A (V_next, V_k, V_{k-1}) pointer tuple pushed for
 * the second time (a ring of input buffers) has its device work recorded as a CUDA graph
 * and replayed while it recurs (six such graphs kept, least recently used dropped); the
 * results are those of the unrecorded step.  Errors: TDB_ERR_INVALID_ARG (null ctx or
 * snapshot), TDB_ERR_STATE (before init), TDB_ERR_NONFINITE (a non-finite difference),
 * TDB_ERR_RANK_DEFICIENT (a core Gram or basis Gram not positive definite),
 * TDB_ERR_TIMEOUT (a bounded device wait ran out), TDB_ERR_CUDA; TDB_WARN_RANK_CAP
 * (the step completed, but the error stays above eps_th at the rank caps). */
tdb_status tdb_push_snapshot(tdb_ctx* ctx, const void* V_next, tdb_step_info* info);

/* Write V^TDB = T x_1 U_1 ... x_p U_p (Eq. 2.5) into V_out (device, caller-owned,
 * prod N_n elements of the snapshot type).  Stream-ordered, no sync. */
tdb_status tdb_reconstruct(tdb_ctx* ctx, void* V_out);

/* Exact error (Eq. 2.20) of the current state against V_now (device, same layout and
 * type as the pushes) and one pass of the Sec. 2.5 rule on it, re-initialising by HOSVD
 * of V_now if it fires.  Afterwards the state stands for V_now: V_now becomes the
 * previous snapshot of the next push (borrowed as by tdb_push_snapshot).  ranks_out:
 * host int[p] (nullable), the ranks after the rule; eps_out: host (nullable), the error
 * after the rule.  Synchronises.  Errors as tdb_reinit; TDB_WARN_RANK_CAP when the error
 * stays above eps_th at the rank caps. */
tdb_status tdb_adapt_rank(tdb_ctx* ctx, const void* V_now, int* ranks_out, double* eps_out);

/* Re-initialise the state from V_now (device snapshot, same layout and type as the
 * pushes) by the truncated HOSVD at the current ranks (Sec. 2.3 end, Sec. 2.5): U_n =
 * W_n^{-1/2} times the leading eigenvectors of the weighted mode-n Gram, T the Eq. 2.15
 * projection of V_now.  V_now becomes the previous snapshot of the next push (it must
 * stay unmodified until then, as for tdb_push_snapshot).  Clears the slope window of the
 * rank rule.  Synchronises the stream.  Errors: TDB_ERR_INVALID_ARG (null ctx or
 * snapshot), TDB_ERR_STATE (before init), TDB_ERR_TIMEOUT / TDB_ERR_CUDA (device). */
tdb_status tdb_reinit(tdb_ctx* ctx, const void* V_now);

/* Copy the current factors to host memory: core (prod r_n doubles) and U[n]
 * (N_n x r_n doubles each); any of them may be NULL.  ranks: host int[p]
 * (nullable).  Synchronises. */
tdb_status tdb_get_factors(tdb_ctx* ctx, double* core, double* const* U, int* ranks);

/* Copy the projections of the last step to host memory (for tests): dS
 * (prod r_n doubles) and Y[n] (prod_{m<n} r_m x N_n x prod_{m>n} r_m doubles,
 * column-major, i.e. the tensor whose mode-n unfolding is Y_(n) of Eq. 2.16).
 * Any pointer may be NULL.  Synchronises. */
tdb_status tdb_get_projection(tdb_ctx* ctx, double* dS, double* const* Y);

/* Current step counter and HOSVD re-initialisation count (host outputs, nullable). */
tdb_status tdb_get_counters(tdb_ctx* ctx, int64_t* steps, int64_t* reinits, int64_t* exact_evals);

/* Serialise the state (factors, ranks, counters, controller history) into buf
 * (host).  With buf == NULL only *bytes is set.  Synchronises. */
tdb_status tdb_save_state(tdb_ctx* ctx, void* buf, size_t* bytes);
/* Restore a state saved with the same config.  The previous snapshot pointer
 * must be supplied again (device). */
tdb_status tdb_load_state(tdb_ctx* ctx, const void* buf, size_t bytes, const void* V_prev);

/* Last error message of ctx (or of the last failed tdb_init on this thread when
 * ctx is NULL).  Never NULL. */
const char* tdb_last_error(const tdb_ctx* ctx);
const char* tdb_status_string(tdb_status s);

/* Release the context (not the workspace).  NULL is accepted. */
void tdb_destroy(tdb_ctx* ctx);

/* ---- Learned error estimator --------------------------------------------------
 * Not in the paper, which evaluates the error of Eq. 2.20 by a full reconstruction.
 * A two-hidden-layer perceptron (8 -> 64 -> 64 -> 1, tanh) predicts the change of
 * log10 of that error over each step from reduced quantities: the previous step's error
 * (exact, or the estimate when skipped), ||dV||_W, the residual sqrt(||dV||_W^2 - ||dS||^2)
 * of the step and of the previous step, ||dS||, the smallest sigma_min / sigma_max of the
 * core unfoldings (Eq. 2.18), ||T|| and steps since the last re-initialisation.  Parameter vector (float,
 * tdb_mlp_param_count() entries): W1 (64 x 8, row-major), b1, W2 (64 x 64,
 * row-major), b2, w3, b3.  Training and inference run in libtdb's kernels. */
int tdb_mlp_param_count(void);
/* y[i] = MLP(X[i, :]) for n rows of 8 features (all device float). */
tdb_status tdb_mlp_forward(const float* params, const float* X, int n, float* y, void* stream);
/* Mean-squared-error loss over n rows and its gradient (device float, one per
 * parameter).  scratch: device float, >= 1024 * (tdb_mlp_param_count() + 1) entries
 * for the widest split (fewer entries use fewer partial sums).  loss may be NULL. */
tdb_status tdb_mlp_loss_grad(const float* params, const float* X, const float* t, int n, float* scratch,
                             size_t scratch_floats, float* loss, float* grad, void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8); step counts from 1; m, v device state. */
tdb_status tdb_mlp_adam_step(float* params, const float* grad, float* m, float* v, int step, float lr, void* stream);
/* Fit the context's estimator on the (features, log10 exact error) rows it has recorded
 * (every exact evaluation of an FP32/BF16 context records one): standardisation, Glorot
 * initialisation from `seed`, `iters` full-batch Adam steps at rate lr.  Afterwards, in
 * TDB_ERRMODE_MLP the exact error is evaluated only when the estimate exceeds
 * gate * eps_th, when error_every steps passed without one, or when a feature leaves
 * the training range; decisions of Sec. 2.5 are taken on exact evaluations only.
 * loss_out (host, nullable): final training loss (standardised units).  Synchronises. */
tdb_status tdb_estimator_fit(tdb_ctx* ctx, int iters, float lr, uint64_t seed, double gate, double* loss_out);
/* Copy the fitted estimator out (get_out, host, param_count + 18 floats: parameters then
 * feature means, feature scales, target mean, target scale) and / or install one
 * (set_in, same layout; gate > 0 replaces the gate factor).  Either may be NULL. */
tdb_status tdb_estimator_params(tdb_ctx* ctx, float* get_out, const float* set_in, double gate);
/* Recorded training rows, oldest first (the most recent 8192; each exact evaluation of a
 * float context adds one): on input *n is the capacity of X (n x 8) and t (n); on output
 * the number recorded (X, t may be NULL to query). */
tdb_status tdb_estimator_trace(tdb_ctx* ctx, float* X, float* t, int* n);
/* Install training rows recorded elsewhere (e.g. tdb_estimator_trace of contexts run on
 * other streams) before tdb_estimator_fit: X (host, n x 8) and t (host, n) replace the
 * context's own rows (append = 0) or are added after them (append = 1); the trace keeps
 * its most recent 8192 rows.  TDB_ERR_INVALID_ARG for null data or n < 1. */
tdb_status tdb_estimator_load_trace(tdb_ctx* ctx, const float* X, const float* t, int n, int append);

/* Accumulated device times of the phases of tdb_push_snapshot, measured with CUDA
 * events on the context's stream while profiling is enabled (tdb_set_profiling).
 * No counterpart in the paper: instrumentation for the roofline report. */
typedef struct tdb_profile {
  int64_t steps;              /* steps timed */
  double ms_project;          /* difference + projection (Eqs. 2.15, 2.16) */
  double ms_project_main;     /* the main projection kernel alone (the fused tensor-core
                                 kernel in TDB_BF16_TTM, the mode-1 product otherwise) */
  double ms_update;           /* pseudo-inverse, complement projection, Euler, Cholesky-QR,
                                 core singular values */
  double ms_error;            /* exact error (Eq. 2.20) or its estimate */
  double ms_control;          /* rank control including HOSVD re-initialisations (host clock) */
  int64_t launches_main;      /* launches of the main projection kernel */
  int64_t update_phases;      /* entries of us_update_phase in use (6 + number of modes) */
  double us_update_phase[12]; /* microseconds summed over the timed steps, per phase of the
                                 fused update kernel (device global timer at its grid barriers):
                                 rows M/X/P, P reduce, rows U'/C, Cholesky-QR factors,
                                 rows U'' with the core product of mode 1, core products of
                                 modes 2..p, Gram partials, Gram finish */
  double us_project_span;     /* TDB_BF16_TTM: microseconds summed over the timed steps from the
                                 first CTA's start to the last CTA's end of the main projection
                                 kernel (device global timer); the CUDA-event time of
                                 ms_project_main adds the launch and the event nodes to it */
  int64_t spans;              /* launches measured in us_project_span */
} tdb_profile;

/* enable != 0 starts (and zeroes) the accumulation; 0 stops it. */
tdb_status tdb_set_profiling(tdb_ctx* ctx, int enable);
tdb_status tdb_get_profile(tdb_ctx* ctx, tdb_profile* out);

/* Number of libtdb kernels launched by this process so far (all contexts). */
int64_t tdb_kernel_launches(void);

/* Allocation-free form of the fused snapshot difference + projection (the kernels
 * of the TDB_BF16_TTM step), for callers that cannot allocate device memory -
 * e.g. a simulation code that hands every byte of the GPU to its own pool
 * allocator, or runs where cudaMalloc is not allowed after start-up.  The paper
 * has no counterpart: this is a packaging of the existing computation.
 *   dims, ranks : host, ndim entries (layout of tdb_push_snapshot, mode 1 fastest)
 *   V_next, V_prev : device float snapshots (layout as above)
 *   A[n] : device float N_n x r_n, the weighted bases W_n U_n; w[n] : device double, N_n
 *   dS (prod r_n), Y[n] (the tensor with mode n of size N_n, other modes r_m) and
 *   dv2 (||V_next - V_prev||_W^2, one double): device outputs owned by the caller.
 * Refusals, all before anything is launched:
 *   TDB_ERR_INVALID_ARG  ndim outside 2..4, or a NULL pointer argument;
 *   TDB_ERR_SHAPE        some N_n < 1 or N_n > 1024;
 *   TDB_ERR_RANK         some r_n < 1, r_n > N_n or r_n > TDB_MAX_RANK (32);
 *   TDB_ERR_UNSUPPORTED  N_1 not a multiple of 4 (16-byte TMA row stride), r_1 or r_2
 *                        above 32, the bases' BF16 images too large for shared memory,
 *                        or a GPU that is not compute capability 10.x (tcgen05);
 *   TDB_ERR_WORKSPACE    the sizes need more than the 16 MiB of static scratch.
 * Scratch comes from a static device array of 16 MiB compiled into the library.  A
 * device holds it from the moment the library's projection module is loaded there
 * until process exit; CUDA loads modules lazily by default, so that is usually the
 * first call on the device that runs a tensor-core projection (this entry point, or
 * a TDB_BF16_TTM context's first step).  A caller whose pool allocator will reserve
 * the whole GPU should make its first call on each device before the pool does, or
 * the module load can fail (TDB_ERR_CUDA).  The call allocates nothing (no cudaMalloc
 * or allocating library routine).  The first call on a device also looks up the
 * array's device address once for that device; make that first call before any
 * stream capture.  All calls share the array and it keeps the last call's contents
 * (every value read is written earlier in the same call), so calls that overlap on
 * the GPU - on different streams or host threads - race.  Each call ends by
 * synchronising `stream`, and returns TDB_ERR_TIMEOUT if a bounded device wait ran
 * out. */
tdb_status tdb_project_noalloc(int ndim, const int64_t* dims, const int* ranks, const float* V_next,
                               const float* V_prev, const float* const* A, const double* const* w, float* dS,
                               float* const* Y, double* dv2, void* stream);

/* ---------------------------------------------------------------------------
 * Diagnostics.  The paper has no counterpart: these exercise the library's own device
 * arithmetic and failure handling, for tests.
 *
 * tdb_selftest_recip: the double reciprocal and reciprocal square root the small-matrix
 *   kernels use (Newton-Raphson from a float seed, see k_update.cu) over n doubles:
 *   rcp[i] = 1/x[i], rsqrt[i] = 1/sqrt(x[i]) for x[i] > 0 (0 otherwise).  x, rcp, rsqrt:
 *   device arrays of n doubles owned by the caller.  Synchronises `stream`.
 *   TDB_ERR_INVALID_ARG for a NULL pointer or n < 0.
 * tdb_selftest_timeout: makes one of the library's bounded device waits run out on
 *   purpose - which = 0: the fused update's grid barrier, launched on two co-resident
 *   CTAs and waiting for a third arrival; which = 1: the projection kernel's mbarrier
 *   wait, on a barrier nothing arrives at - with a limit of limit_cycles SM clock
 *   cycles (1 .. 4e9) instead of the usual ~2 s.  scratch: device, >= 16 bytes, owned by
 *   the caller (barrier counter and status word; cleared here).  The kernel returns
 *   after the limit with the timeout bit set; the call synchronises `stream` and
 *   returns TDB_ERR_TIMEOUT (the expected result), TDB_OK if the wait ended otherwise,
 *   TDB_ERR_INVALID_ARG for bad arguments or TDB_ERR_CUDA.  The CUDA context stays
 *   usable afterwards.
 * ------------------------------------------------------------------------- */
tdb_status tdb_selftest_recip(const double* x, double* rcp, double* rsqrt, int64_t n, void* stream);
tdb_status tdb_selftest_timeout(int which, int64_t limit_cycles, unsigned* scratch, void* stream);

/* The launch shape the tensor-core projection's tuner chose for this context (TDB_BF16_TTM
 * only; the paper has no counterpart).  The tile is fixed (128 x 128, eight strips); the
 * tuner times, on the context's first step outside stream capture, each candidate number
 * of CTAs per tile position in the persistent grid and each split target of the finishing
 * contraction, and keeps the fastest (cached per shape for the process).  Host outputs,
 * each nullable: ctas = CTAs per tile position, fin_target = the finish's split target
 * (CTAs), ncand = candidates timed (0 when the choice came from the cache), cand /
 * cand_us = up to 4 candidates and their microseconds per launch, fin_cand / fin_us = the
 * 3 split targets and theirs.  TDB_ERR_STATE before the first step or without the
 * tensor-core path.  The environment variable TDB_TC_SHAPE="ctas,target" (two positive
 * integers) replaces the tuning by that shape (ctas clamped to the tile positions' slice
 * count), e.g. to profile the shape a timed run chose. */
tdb_status tdb_tc_tuning(const tdb_ctx* ctx, int* ctas, int* fin_target, int* ncand, int* cand, float* cand_us,
                         int* fin_cand, float* fin_us);

/* Library version and build facts: "tdb <ver> sm_103a". */
/* ---------------------------------------------------------------------------
 * Input slots and recorded steps.  The paper streams one snapshot per step (Sec. 2.3);
 * these calls change only how the same step is issued, not what it computes.
 *
 * tdb_set_input_slots: two distinct device buffers, each holding one snapshot in the
 *   layout of tdb_push_snapshot, owned by the caller (who writes each new snapshot
 *   into them, e.g. straight from a simulation or a host copy).  NULL, NULL removes them.
 * tdb_push_slot: one step with V_{k+1} in slot[parity] and V_k in slot[1 - parity];
 *   the previous step (or the init) must have consumed slot[1 - parity], otherwise
 *   TDB_ERR_STATE; TDB_ERR_UNSUPPORTED under TDB_RK2_CENTRAL (its central differences
 *   need three snapshots).  The device work of the step is recorded once per slot parity and
 *   rank configuration as a CUDA graph and replayed afterwards, so a step costs one
 *   launch; the results are those of tdb_push_snapshot on the same snapshots.  Steps
 *   run unrecorded on the first step of a tensor-core context, while profiling is
 *   enabled if the runtime cannot time events inside a graph, or if the configuration
 *   cannot be recorded.
 * ------------------------------------------------------------------------- */
tdb_status tdb_set_input_slots(tdb_ctx* ctx, const void* slot0, const void* slot1);
tdb_status tdb_push_slot(tdb_ctx* ctx, int parity, tdb_step_info* info /* nullable, host */);

/* ---------------------------------------------------------------------------
 * Batches: many independent tensors (fields, species or samples of uneven sizes and
 * ranks) stepped together.  The paper compresses one tensor at a time; a batch runs
 * each member's own step, unchanged, with every member's device work recorded into one
 * CUDA graph over `nstreams` streams (member i on stream i mod nstreams) and one
 * synchronisation per batch step; the host then finishes each member in turn (error
 * control and rank adaptation, which may re-initialise a member by HOSVD on its own
 * stream and causes the graph to be recorded again at the next step).
 *
 * tdb_batch_create: members are initialised contexts with input slots set; the batch
 *   keeps pointers to them (the caller still owns and destroys them, after the batch).
 *   stream: the caller's stream on which each batch step is launched and synchronised.
 * tdb_batch_push: one step of every member, V_{k+1} in each member's slot[parity];
 *   infos (nullable) receives one record per member in member order.  Returns the most
 *   severe member status (an error over TDB_WARN_RANK_CAP); tdb_batch_last_error names
 *   the member.
 * ------------------------------------------------------------------------- */
typedef struct tdb_batch tdb_batch;
tdb_status tdb_batch_create(tdb_batch** out, tdb_ctx* const* members, int n, int nstreams, void* cuda_stream);
tdb_status tdb_batch_push(tdb_batch* batch, int parity, tdb_step_info* infos /* nullable, n records */);
const char* tdb_batch_last_error(const tdb_batch* batch);
/* How many steps of ctx (or batch steps of batch; exactly one of the two non-NULL) were
 * replayed from a recorded graph, and how many recordings were made (host, nullable). */
tdb_status tdb_get_graph_counters(const tdb_ctx* ctx, const tdb_batch* batch, int64_t* replays, int64_t* records);
void tdb_batch_destroy(tdb_batch* batch);

const char* tdb_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TDB_H */
