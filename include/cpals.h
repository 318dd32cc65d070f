/*
 * cpals.h -- C ABI of the GB300 pairwise-perturbation CP-ALS library.
 *
 * Source method: Ma & Solomonik, "Accelerating Alternating Least Squares for
 * Tensor Decomposition by Pairwise Perturbation" (arXiv 1811.10573).
 * The paper states the problem as: input a dense order-N tensor X
 * (s_1 x ... x s_N), a rank R and a PP tolerance eps; output factors
 * [[A^(1), ..., A^(N)]] (Algorithm 1 CP-ALS, Algorithm 3 PP-CP-ALS).
 * These calls expose its steps one by one.
 *
 * Conventions for every call:
 *   - Tensors are dense, row-major, last mode fastest.  Factors A^(n) are
 *     s_n x R row-major (r fastest), always exchanged as float64.
 *   - Modes are 0-based (the paper's mode n is index n-1).
 *   - Every call returns a cpals_status; nothing throws across the ABI.
 *     On failure, cpals_last_error(ctx) returns a message that stays valid
 *     until the next call on the same context.
 *   - The context owns all device memory it allocates; pointers passed in
 *     stay owned by the caller and are only read (or written, for *_out
 *     arguments) during the call.
 *   - Work runs on the context's stream (see cpals_set_stream).  Calls that
 *     return host data synchronise that stream before returning.
 *   - One context = one decomposition; a context is not thread-safe.
 */
#ifndef CPALS_H
#define CPALS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cpals_ctx cpals_ctx;

typedef enum {
  CPALS_OK = 0,
  CPALS_E_INVALID = 1,     /* bad argument: N < 3, R < 1, dims <= 0, NULL pointer, bad mode */
  CPALS_E_OOM = 2,         /* device allocation failed */
  CPALS_E_CUDA = 3,        /* CUDA runtime/driver error (text in cpals_last_error) */
  CPALS_E_STATE = 4,       /* call out of order (e.g. pp_sweep before pp_build_operators) */
  CPALS_E_SINGULAR = 5,    /* Gamma has a non-finite entry: the factor of that mode was left
                              unchanged.  A finite Gamma that is not positive definite is no
                              error: every path (float64 and double-float normal equations, the
                              fused batch) replaces its inverse by the pseudo-inverse
                              Gamma^dagger (Algorithm 1): symmetric Jacobi eigendecomposition in
                              float64, eigenvalues at or below 1e-13 of the largest dropped. */
  CPALS_E_NUMERIC = 6,     /* NaN/Inf detected in a result */
  CPALS_E_TIMEOUT = 7,     /* a bounded device wait gave up */
  CPALS_E_UNSUPPORTED = 8  /* configuration outside what this build implements */
} cpals_status;

/* Arithmetic of the contractions.  The fitness is float64 in every mode;
 * the normal-equation work (Grams, Gamma, its factorisation and the row
 * solves) follows cpals_set_normal_arith. */
typedef enum {
  CPALS_FP64 = 0,        /* tensor, contractions and operators in float64 */
  CPALS_FP32 = 1,        /* tensor, contractions and operators in float32 */
  CPALS_MIXED_BF16 = 2   /* first-level contractions and operator construction on
                            bf16 tensor cores (fp32 accumulate); lower levels,
                            operators and PP corrections in float32 */
} cpals_precision;

/* Arithmetic of the normal-equation work of Algorithm 1
 * (Grams S^(n), Gamma^(n), its Cholesky factor, the row solves, the
 * second-order terms' Z).  FP64 contexts always use IEEE float64.  FP32 and
 * MIXED_BF16 contexts default to double-float (an unevaluated sum of two
 * floats, 48-bit significand, built from error-free transformations on the
 * float32 pipes); IEEE float64 is available to them as well. */
typedef enum {
  CPALS_NE_FP64 = 0,
  CPALS_NE_DOUBLE_FLOAT = 1
} cpals_normal_arith;

/* Sweep kinds reported by cpals_run (Algorithm 3 and Table 2 of the paper). */
enum { CPALS_SWEEP_ALS = 0, CPALS_SWEEP_PP_INIT = 1, CPALS_SWEEP_PP_APPROX = 2 };

/* Create a context for an order-N tensor of size dims[0] x ... x dims[N-1]
 * and CP rank R (Sec. 2.3).  3 <= N <= 8, 1 <= R <= 128.  Allocates the
 * tensor storage and all workspaces of the dimension trees (Sec. 2.5,
 * Sec. 3.2.3).  *out receives the context; NULL on failure. */
cpals_status cpals_create(const int64_t* dims, int N, int R, int precision, cpals_ctx** out);

/* Free every device and host resource of the context.  NULL is ignored. */
void cpals_destroy(cpals_ctx* ctx);

/* Select the normal-equation arithmetic (cpals_normal_arith).  Returns
 * CPALS_E_UNSUPPORTED for CPALS_NE_DOUBLE_FLOAT on an FP64 context and
 * CPALS_E_INVALID for an unknown value.  Drops the captured sweep graphs and
 * the factors: call cpals_init_factors (again) afterwards. */
cpals_status cpals_set_normal_arith(cpals_ctx* ctx, int arith);

/* ALS variants of Sec. 5.1 (chemistry-tensor experiment), for ALS and PP
 * sweeps alike.
 *
 * Update step size: lam[n] (N host values in (0, 2]; NULL = all 1) makes
 * the update of mode n A_new = (1 - lam[n]) A^(n) + lam[n] M^(n) Gamma^(n)^-1
 * (M^(n) the exact or PP-approximated right-hand side, A^(n) the current
 * factor).  dA is then taken from A_new as usual.  Drops the captured sweep
 * graphs; the state is kept.  CPALS_E_INVALID for a value outside (0, 2].
 *
 * Symmetry constraint: modes m1 < m2 of equal size share one factor
 * (X = [[A, B, B]] is m1 = 1, m2 = 2 of an order-3 tensor, with the tensor
 * symmetric in those modes; that symmetry is the caller's to provide).  A
 * sweep solves for mode m1 and gives mode m2 its factor, Gram and change at
 * once; mode m2 is never solved for (its right-hand side is still formed
 * when it is the last mode, for the fitness).  cpals_init_factors uses
 * factors[m1] for both.  m1 = m2 = -1 removes every tie.  Drops the graphs
 * and the factors (call cpals_init_factors afterwards).  CPALS_E_INVALID
 * for modes out of range, of different sizes, or already tied. */
cpals_status cpals_set_step_size(cpals_ctx* ctx, const double* lam);
cpals_status cpals_set_symmetric(cpals_ctx* ctx, int m1, int m2);

/* Order the context's work after, and before, work already queued on a
 * caller stream (a cudaStream_t passed as void*; NULL = the legacy default
 * stream).  The library keeps its own stream and joins the caller stream at
 * the start and end of every call. */
cpals_status cpals_set_stream(cpals_ctx* ctx, void* cuda_stream);

/* Copy the input tensor X (Sec. 2.3) into the context.  data: prod(dims)
 * values, dtype 0 = float64, 1 = float32; on_device != 0 means data is a
 * device pointer, else a host pointer (pinned or pageable).  In FP32 and
 * MIXED_BF16 modes float64 input is rounded to float32; in MIXED_BF16 a bf16
 * copy for the tensor cores is also made.  ||X||_F^2 is computed in float64
 * from the stored values.  Clears any PP operators. */
cpals_status cpals_set_tensor(cpals_ctx* ctx, const void* data, int dtype, int on_device);

/* Set the factors A^(n) from N host float64 arrays of s_n x R (row-major);
 * they are the random initial guess of Algorithms 1 and 3.  Resets the
 * controller state as the start of Algorithm 3 does: dA^(n) <- A^(n), so the next
 * eps test fails, S^(n) <- A^(n)T A^(n); clears PP operators. */
cpals_status cpals_init_factors(cpals_ctx* ctx, const double* const* factors);

/* One regular ALS sweep (Algorithm 1) over modes 0..N-1 with the
 * binary dimension tree (Sec. 2.5): two first-level contractions of X per
 * sweep.  Afterwards dA^(n) = A^(n)_new - A^(n)_old (the regular sweep of Algorithm 3).
 * fitness_out (nullable): exact fitness 1 - ||X - [[A]]||/||X|| (Sec. 5). */
cpals_status cpals_als_sweep(cpals_ctx* ctx, double* fitness_out);

/* Build the PP operators M_p^(i,n), i < n, and M_p^(n) at the current
 * factors with the operator dimension tree (Sec. 3.2.3), then set
 * A_p <- A, dA <- 0 (the PP initialisation of Algorithm 3). */
cpals_status cpals_pp_build_operators(cpals_ctx* ctx);

/* One PP approximated sweep (Algorithm 3): each right-hand side
 * is Eq. 3's M~^(n); use_V != 0 adds the second-order terms V^(n,i,j).
 * dA^(n) = A^(n)_new - A_p^(n).  fitness_out (nullable): the fitness
 * estimated from the first-order part of M~^(N),
 * M_p^(N) + sum_i M_p^(i,N) x_i dA^(i), and the new factors (not exact; see
 * cpals_fitness).  CPALS_E_STATE if no operators. */
cpals_status cpals_pp_sweep(cpals_ctx* ctx, int use_V, double* fitness_out);

/* Exact fitness of the current factors: one exact MTTKRP of the last mode
 * (a full pass over X) plus float64 Grams (Sec. 5). */
cpals_status cpals_fitness(cpals_ctx* ctx, double* out);

/* Copy the factors to N caller-owned host float64 arrays of s_n x R. */
cpals_status cpals_get_factors(cpals_ctx* ctx, double* const* out);

/* out_N[n] = ||dA^(n)||_F / ||A^(n)||_F (the quantities Algorithm 3 tests). */
cpals_status cpals_get_dA_ratios(cpals_ctx* ctx, double* out_N);

/* *mask: bit n set when the last factorisation of mode n met a Gamma^(n) that
 * is not positive definite and the update went through Gamma^dagger
 * (Algorithm 1's pseudo-inverse; see CPALS_E_SINGULAR).  Waits for the
 * context's stream. */
cpals_status cpals_pinv_modes(cpals_ctx* ctx, int* mask);

/* Run Algorithm 3 for at most max_sweeps sweeps with tolerance eps (eps <= 0
 * gives plain ALS).  Each ALS sweep, PP initialisation sweep (build + one PP
 * pass) and PP approximated sweep counts as one sweep.  If target > 0 the run
 * stops after the first sweep whose exact fitness is >= target (for PP sweeps
 * the estimate is checked first, then confirmed by cpals_fitness).
 * Outputs (each nullable, length max_sweeps): fitness_trace (exact after ALS
 * sweeps, estimate after PP sweeps), kind_trace (CPALS_SWEEP_*),
 * time_trace (seconds since the start of the run at the end of each sweep).
 * *n_done receives the number of sweeps run; *reached (nullable) 1 if the
 * target was confirmed.
 * With captured graphs on, profiling off and the device loop enabled (the
 * default, cpals_set_device_loop), every decision of the algorithm is taken
 * on the GPU: one CUDA graph holds a while loop around a switch over the
 * sweep kinds and a one-thread kernel that applies the eps and target tests
 * to the device scalars, so the run synchronises with the host once, at its
 * end; time_trace then comes from the GPU's global timer.  Otherwise the
 * decisions are taken on the host after each sweep's stream
 * synchronisation (host clock).  Both take the same decisions on the same
 * values, and the sweeps run the same kernels. */
cpals_status cpals_run(cpals_ctx* ctx, int max_sweeps, double eps, int use_V, double target,
                       double* fitness_trace, int* kind_trace, double* time_trace,
                       int* n_done, int* reached);

/* Many independent decompositions at once (tensors of different shapes, one
 * context each, already given their tensor and factors): `workers` host
 * threads take the contexts one after the other from a shared counter and
 * run cpals_run(ctx, max_sweeps, eps, use_V, targets ? targets[i] : 0, ...)
 * on each, on the contexts' own streams, so up to `workers` decompositions
 * are in flight on the GPU and uneven ones balance themselves.  Every
 * context keeps its own controller (Algorithm 3) and gets the result a lone
 * cpals_run would give it.  Per instance (each output nullable, length n):
 * fitness_out = the last fitness of its trace, sweeps_out = sweeps run,
 * status_out = its cpals_status.  The contexts must all live on devices the
 * calling process can use; none may be used by another thread meanwhile.
 * Returns CPALS_E_INVALID for bad arguments, else CPALS_OK (per-instance
 * failures are in status_out). */
cpals_status cpals_run_batch(cpals_ctx* const* ctxs, int n, int workers, int max_sweeps, double eps,
                             int use_V, const double* targets, double* fitness_out,
                             int* sweeps_out, int* status_out);

/* ---- many small order-3 decompositions in one set of launches ----
 * A batch holds n independent order-3 problems of different sizes
 * (dims[3i..3i+2] <= 4096) and ranks (ranks[i] <= 64) and runs Algorithm 3
 * on all of them at once: each stage of a sweep (a first-level
 * contraction, a multi-TTV, the operator build, the PP correction of Eq. 3,
 * the factorisation of Gamma^(n), the row solves, the Grams, the fitness,
 * the decision of Algorithm 3) is one launch over every instance, and every
 * instance keeps its own controller state on the device and takes part only
 * in the stages of the sweep kind it runs.  One sweep of the batch is one
 * captured CUDA graph.  precision: CPALS_FP64 or CPALS_FP32 for the
 * contractions, operators and corrections; Gamma, its Cholesky factor, the
 * solves, the Grams and the fitness are float64 either way.
 * The batch owns its device memory and one stream; every call returns after
 * its work has finished.  Errors: CPALS_E_INVALID (bad sizes or arguments),
 * CPALS_E_UNSUPPORTED (another precision, not sm_103), CPALS_E_OOM,
 * CPALS_E_STATE (run before every instance has a tensor and factors),
 * CPALS_E_CUDA; cpals_batch_last_error describes the last failure. */
typedef struct cpals_batch cpals_batch;
cpals_status cpals_batch_create(int n, const int64_t* dims, const int* ranks, int precision,
                                cpals_batch** out);
void cpals_batch_destroy(cpals_batch* b);
/* instance i's tensor: s0 s1 s2 values row-major, dtype 0 = float64,
 * 1 = float32, host or device pointer; copied; ||X||^2 in float64 */
cpals_status cpals_batch_set_tensor(cpals_batch* b, int i, const void* data, int dtype, int on_device);
/* instance i's initial factors: three host float64 arrays s_n x R, copied */
cpals_status cpals_batch_init_factors(cpals_batch* b, int i, const double* const* factors);
/* Algorithm 3 on every instance from its initial factors for exactly
 * max_sweeps sweeps (fewer for an instance that met a non-finite value; a
 * Gamma that is not positive definite is solved through Gamma^dagger), with
 * tolerance eps, the
 * second-order terms when use_V != 0 and the stopping test inside PP runs
 * (as cpals_set_pp_stop_tol; 0 = off).  Outputs (each nullable):
 * fitness_out[n] the exact fitness of the final factors, sweeps_out[n],
 * status_out[n] (CPALS_OK, CPALS_E_SINGULAR, CPALS_E_NUMERIC), and
 * kind_trace / fitness_trace [n][max_sweeps] (CPALS_SWEEP_*; exact fitness
 * after ALS sweeps, the M~ estimate after PP sweeps). */
cpals_status cpals_batch_run(cpals_batch* b, int max_sweeps, double eps, int use_V, double pp_stop_tol,
                             double* fitness_out, int* sweeps_out, int* status_out, int* kind_trace,
                             double* fitness_trace);
/* instance i's factors into three caller-owned host float64 arrays */
cpals_status cpals_batch_get_factors(cpals_batch* b, int i, double* const* out);
/* kernels of one batch sweep graph (one launch per stage over all instances)
 * and kernels launched by the last run */
cpals_status cpals_batch_stats(const cpals_batch* b, int64_t* launches_per_sweep, int64_t* launches_last_run);
/* The tile autotuner's choice for the batch's four contraction stages
 * (M^(L), the mode-2 right-hand side, M_p^(1,2), M_p^(0,2)): tiles[4]
 * (0 = 64-row tiles with 4 outputs per thread per 16 columns, 1 = 128-row
 * tiles with 8, 2 = 32-row tiles with 2; columns are 16 ceil(R / 16) per
 * instance), ms[12] the measured launch times (stage-major, three shapes
 * per stage, -1 if not timed), *from_cache 1 when the choice came from the
 * process-wide cache of an earlier batch with the same sizes, ranks and
 * precision (nothing timed).  The tuning runs at the first cpals_batch_run.
 * Each argument nullable; CPALS_E_STATE before the first run. */
cpals_status cpals_batch_tiles(const cpals_batch* b, int* tiles, float* ms, int* from_cache);
const char* cpals_batch_last_error(const cpals_batch* b);

/* ---- Tucker-ALS and PP-Tucker-ALS (Sec. 2.4, Sec. 3.1.2, Algorithm 4) ----
 * Tensors of order 3 to 8, IEEE float64 (order 3: first-level TTMs
 * optionally on the tensor cores, cpals_tucker_set_precision), Tucker ranks
 * 1 <= R_n <= min(48, s_n), s_n <= 4096.  Factors are s_n x R_n float64
 * row-major with orthonormal columns; the core is R_1 x ... x R_N row-major.
 * Order 3 uses a tuned dimension tree; higher orders contract X twice per
 * HOOI sweep (Y^(1) and X x_1 A_1, then chains of smaller TTMs) and build
 * the C(N,2) operators from three shared contractions of X.  Each factor update takes
 * the R_n leading eigenvectors of W = Y_(n) Y_(n)^T (Y^(n) the TTMc) in
 * decreasing eigenvalue order, each column signed to a non-negative inner
 * product with the column it replaces; the eigenvectors come from subspace
 * iteration started at the current factor (at most
 * cpals_tucker_set_iterations steps, default 8; it stops once the invariance
 * residual ||W Q - Q Q^T W Q|| / ||W Q|| is below 1e-13) and a Rayleigh-Ritz
 * step, so a factor is exact once the iteration has converged (a spectral
 * gap after R_n).  Fitness: 1 - sqrt(||X||^2 - ||G||^2) / ||X||.
 * The context owns all device memory and one stream; every call returns
 * after its work has finished.  Errors as for the CP context; E_STATE for a
 * sweep before set_tensor and init_factors, or a PP sweep before
 * pp_build_operators; CPALS_E_SINGULAR if an orthonormalisation met a
 * non-positive pivot; CPALS_E_TIMEOUT if the tensor-core kernel gave up
 * waiting (mixed precision). */
typedef struct cpals_tucker cpals_tucker;
/* dims[0..N-1], ranks[0..N-1] (host, read only), 3 <= N <= 8; *out receives
 * the context or NULL.  E_INVALID for bad sizes, E_UNSUPPORTED off sm_103,
 * E_OOM if the buffers do not fit. */
cpals_status cpals_tucker_create(const int64_t* dims, int N, const int* ranks, cpals_tucker** out);
/* frees everything the context owns; NULL is a no-op */
void cpals_tucker_destroy(cpals_tucker* t);
/* maximum subspace-iteration steps per factor update, 1..1000 (E_INVALID otherwise) */
cpals_status cpals_tucker_set_iterations(cpals_tucker* t, int iters);
/* CPALS_FP64 (default) or CPALS_MIXED_BF16: the first-level TTMs (X x_3 A3,
 * X x_1 A1, and the three PP operators X x_k A_p) run on the tensor cores
 * with X rounded to bf16 and the factor as hi + lo bf16 planes, fp32
 * accumulation, converted to float64 for the rest of the sweep (relative
 * error about 1e-3 against float64).  CPALS_E_UNSUPPORTED if a contraction
 * shape is not aligned for the tensor-core kernel (s_3 and s_2 s_3 and s_3
 * multiples of 8) or the order is not 3, CPALS_E_INVALID for another value.
 * May be called before or after cpals_tucker_set_tensor. */
cpals_status cpals_tucker_set_precision(cpals_tucker* t, int precision);
/* data: row-major, last mode fastest, s_1 ... s_N values; dtype 0 = float64,
 * 1 = float32 (widened); on_device selects a device or a host pointer.  The
 * tensor is copied (the caller keeps ownership) and ||X||^2 is formed in
 * float64.  Invalidates the PP operators.  E_INVALID for a NULL pointer or
 * another dtype. */
cpals_status cpals_tucker_set_tensor(cpals_tucker* t, const void* data, int dtype, int on_device);
/* N host arrays s_n x R_n (orthonormal columns; e.g. the HOSVD), copied;
 * dA <- A, as Algorithm 4 starts.  E_INVALID for a NULL pointer. */
cpals_status cpals_tucker_init_factors(cpals_tucker* t, const double* const* factors);
/* one HOOI sweep (Algorithm 2); *fitness (nullable) exact */
cpals_status cpals_tucker_als_sweep(cpals_tucker* t, double* fitness);
/* Y_p^(i,n) and Y_p^(n) at the current factors; A_p <- A, dA <- 0 */
cpals_status cpals_tucker_pp_build_operators(cpals_tucker* t);
/* one PP approximated sweep; *fitness (nullable) the estimate from Y~^(N) */
cpals_status cpals_tucker_pp_sweep(cpals_tucker* t, double* fitness);
/* Algorithm 4 for max_sweeps sweeps (eps as in cpals_run); traces nullable,
 * length max_sweeps; kinds CPALS_SWEEP_* */
cpals_status cpals_tucker_run(cpals_tucker* t, int max_sweeps, double eps, double* fitness_trace,
                              int* kind_trace, int* n_done);
/* exact fitness at the current factors (also refreshes the core) */
cpals_status cpals_tucker_fitness(cpals_tucker* t, double* out);
/* copies the factors into N caller-owned host buffers of s_n x R_n */
cpals_status cpals_tucker_get_factors(cpals_tucker* t, double* const* out);
/* the core of the last sweep or fitness call into a caller-owned host
 * buffer of R_1 ... R_N values (in PP sweeps the estimate from Y~^(N)) */
cpals_status cpals_tucker_get_core(cpals_tucker* t, double* out);
/* message of the last failure on this context (owned by the context, valid
 * until its next call; "" if none) */
const char* cpals_tucker_last_error(const cpals_tucker* t);

/* Message describing the last failure on this context ("" if none). */
const char* cpals_last_error(const cpals_ctx* ctx);

/* ---- inspection calls used by parity tests (same kernels as the sweeps) ---- */

/* Exact MTTKRP M^(n) = X_(n) P^(n) (Sec. 2.3) at the current factors, through
 * the same first-level and multi-TTV kernels as an ALS sweep; out: s_n x R
 * float64 host buffer. */
cpals_status cpals_mttkrp(cpals_ctx* ctx, int n, double* out);

/* Copy the PP operator M_p^(i,n), i < n, (s_i x s_n x R, Sec. 3.2.1) or, for
 * i == n, M_p^(n) (s_n x R) to a float64 host buffer.  CPALS_E_STATE if the
 * operators have not been built. */
cpals_status cpals_get_operator(cpals_ctx* ctx, int i, int n, double* out);

/* Eq. 3's M~^(n) for the current A, A_p and dA, without updating anything;
 * out: s_n x R float64 host buffer. */
cpals_status cpals_pp_mttkrp(cpals_ctx* ctx, int n, int use_V, double* out);

/* Solve X Gamma^(n) = rhs (Sec. 2.3 normal equations) with the Grams the
 * context currently holds, through the same factorisation and row-solve
 * kernels as a sweep, without changing any state.  rhs, out: s_n x R float64
 * host buffers.  A Gamma^(n) that is not positive definite is solved with its
 * pseudo-inverse Gamma^dagger in every precision. */
cpals_status cpals_normal_solve(cpals_ctx* ctx, int n, const double* rhs, double* out);

/* Copy A_p^(n) (which = 0) or dA^(n) (which = 1) to a host float64 buffer. */
cpals_status cpals_get_state(cpals_ctx* ctx, int which, int n, double* out);

/* ---- learned sweep-type controller ---- */

/* The paper's Algorithm 3 chooses between PP sweeps, exact ALS sweeps and an
 * operator rebuild with one threshold test (every ||dA^(n)|| < eps
 * ||A^(n)||); its conclusion invites other switching schemes.  These calls
 * add a learned alternative: a two-layer perceptron with
 * CPALS_CTRL_FEATURES inputs, 32 ReLU hidden units and 3 outputs (0: PP
 * approximated sweep, 1: exact ALS sweep, 2: rebuild the operators, then a
 * PP sweep).  Its input, built after every sweep, holds the per-mode log10
 * ||dA||/||A|| (8 slots), the largest of the two previous sweeps, log10 of
 * the last three residual decreases, sweeps since the build, whether a PP
 * sweep is possible, the last action (one-hot), log10 eps and log10 of the
 * residual.  Parameters: W1[32][F], b1[32], W2[3][32], b2[3] as floats,
 * CPALS_CTRL_PARAMS in all. */
#define CPALS_CTRL_FEATURES 20
#define CPALS_CTRL_PARAMS (32 * CPALS_CTRL_FEATURES + 32 + 3 * 32 + 3)

/* Install (params != NULL, host array of nparams = CPALS_CTRL_PARAMS floats,
 * copied) or remove (params == NULL) the controller of a context.  A
 * decision is taken from the network only when its largest output
 * probability is >= confidence and the action is possible; otherwise the
 * eps rule decides. */
cpals_status cpals_set_controller(cpals_ctx* ctx, const float* params, int nparams, double confidence);

/* Like cpals_run, with each next sweep chosen by the installed controller
 * (the rule of cpals_run -- the eps test and, when set, the stopping test --
 * where it stands in, or everywhere when none is installed).
 * source_trace[t] (may be NULL) is 1 where the network decided, 0 where the
 * rule did.  The reported fitness follows cpals_run (a PP estimate after PP
 * sweeps, confirmed exactly when it reaches the target).  With the device
 * loop on (the default), the history, features and forward pass run in the
 * loop's decide kernel, one host synchronisation per run; otherwise one per
 * sweep. */
cpals_status cpals_run_controlled(cpals_ctx* ctx, int max_sweeps, double eps, int use_V,
                                  double target, double* fitness_trace, int* kind_trace,
                                  double* time_trace, int* source_trace, int* n_done,
                                  int* reached);

/* Training log generated by the method itself: from the current state, for
 * up to `steps` decisions, the context saves its state, tries each possible
 * action from it over four sweeps (PP sweeps against ALS sweeps when the
 * operators are valid; otherwise rebuild + PP sweep, then PP sweeps,
 * against ALS sweeps) timing them and
 * taking the exact fitness afterwards, restores the state, labels the
 * decision with the action of the larger exact-fitness gain per second, and
 * continues with that action.  Outputs (caller-owned): features
 * [steps][CPALS_CTRL_FEATURES], labels [steps], gains and costs (seconds)
 * [steps][3] (NaN for actions not tried or that broke down); *n_out = decisions logged.  The
 * saved state includes the operators when a rebuild is tried (device memory
 * of about their size is kept by the context). */
cpals_status cpals_controller_log(cpals_ctx* ctx, int steps, double eps, int use_V, float* features,
                                  int* labels, double* gains, double* costs, int* n_out);

/* The input (CPALS_CTRL_FEATURES floats) and output probabilities (3) of
 * the controller's last decision in the last cpals_run_controlled (device or
 * host loop).  Each pointer nullable; CPALS_E_STATE before any controlled
 * decision. */
cpals_status cpals_controller_last(const cpals_ctx* ctx, float* features, float* probs);

/* Labels of cpals_controller_log by the time to a target fitness instead of
 * the four-sweep gain per second: with target > 0 each candidate action is
 * followed by Algorithm 3's rule (eps test, stopping test, PP estimates at
 * the target confirmed by the exact fitness) until the fitness reaches
 * target or max_rollout sweeps have run; the label is the candidate with the
 * shorter time to the target, else (neither reached it) the one with the
 * higher exact fitness at the end of its trial.  gains/costs then hold the
 * trial's fitness gain and duration.  target = 0 restores the default
 * labels.  CPALS_E_INVALID for target < 0 or, with a target, max_rollout < 1. */
cpals_status cpals_set_controller_labels(cpals_ctx* ctx, double target, int max_rollout);

/* Full-batch Adam training of the controller on n logged samples (host
 * arrays: X [n][CPALS_CTRL_FEATURES], labels y in {0,1,2}, sample weights
 * w >= 0), minimising the weighted cross-entropy plus decay/2 ||W||^2;
 * params (CPALS_CTRL_PARAMS floats) hold the start and receive the result;
 * *loss_out (may be NULL) the final weighted mean loss.  Runs on the
 * current device; allocates and frees its own device memory. */
cpals_status cpals_mlp_train(const float* X, const int* y, const float* w, int n, float* params,
                             int nparams, int epochs, double lr, double decay, double* loss_out);

/* Controller outputs (softmax probabilities, [n][3]) for n feature vectors
 * (host arrays); runs on the current device. */
cpals_status cpals_mlp_forward(const float* params, int nparams, const float* X, int n, float* probs);

/* ---- measurement ---- */

/* enable != 0: record CUDA events around every first-level contraction on
 * the context stream (also inside captured graphs); timings accumulate per
 * kind until cpals_reset_stats. */
cpals_status cpals_set_profiling(cpals_ctx* ctx, int enable);
cpals_status cpals_reset_stats(cpals_ctx* ctx);

/* Kernel statistics since the last reset.  kind 0 = first-level
 * contraction (all launches), 1 = all kernels of the library (count only),
 * 2 = PP correction kernels (Eq. 3 first-order terms).
 * *launches: number of launches; *total_ms: summed CUDA-event time (kinds 0
 * and 2, profiling on); *bytes, *flops: algorithmic bytes moved and flops of
 * those launches (kinds 0 and 2; flops kind 0 only). */
cpals_status cpals_get_stats(cpals_ctx* ctx, int kind, int64_t* launches, double* total_ms,
                             double* bytes, double* flops);

/* Algorithm 3's stopping test inside the PP loop (its while condition on
 * Delta), in the form the paper's experiments use (Sec. 5.1: the fitness
 * difference between two neighbouring sweeps): with tol > 0, at the head of
 * every PP sweep after the first of a PP run, cpals_run goes on with the
 * run only if the last sweep raised the fitness it reports (exact after ALS
 * sweeps, the estimate after PP sweeps) by at least tol; otherwise the
 * regular ALS sweep follows, as when the eps test fails.  This ends PP runs
 * that stall at a fixed point of the approximated update.  tol = 0 (the
 * default) leaves the test out.  CPALS_E_INVALID for tol < 0 or NaN.  Used
 * by cpals_run and cpals_run_batch. */
cpals_status cpals_set_pp_stop_tol(cpals_ctx* ctx, double tol);

/* enable != 0 (default): cpals_run takes Algorithm 3's decisions on the
 * device (see cpals_run); 0: on the host after every sweep.  The device loop
 * needs captured graphs (cpals_set_graphs) and profiling off. */
cpals_status cpals_set_device_loop(cpals_ctx* ctx, int enable);

/* 1 if the next cpals_run of this context runs its decisions on the device,
 * 0 if it will use the host loop (device loop disabled, graphs off,
 * profiling on, or a driver that could not build the loop graph, whose
 * error cpals_last_error reported once). */
int cpals_device_loop_active(const cpals_ctx* ctx);

/* Bound, in SM clock cycles, of the tensor-core contraction kernel's waits
 * on its own pipeline (a stage's loads, an accumulator, the unit queue);
 * 0 restores the default (4e9 cycles, about 2 s).  When a wait runs out the
 * kernel records an error code, lets the loads and tensor-core operations it
 * already issued complete, frees its tensor memory and returns; the call
 * that ran it returns CPALS_E_TIMEOUT (as does every later call that reads
 * the context's status) until cpals_init_factors clears the status.  The
 * output of that contraction is then undefined.  A short bound exists to
 * test this path; the default never expires in normal operation.  Drops the
 * captured sweep graphs; the state is kept. */
cpals_status cpals_set_wait_limit(cpals_ctx* ctx, uint64_t cycles);

/* enable != 0 (default): capture each sweep kind in a CUDA graph on first use
 * and replay it; 0 launches kernels directly. */
cpals_status cpals_set_graphs(cpals_ctx* ctx, int enable);

/* ---- contraction without device allocation ---- */

/* The paper has no counterpart to this call.  It is the tensor-core
 * first-level contraction (the same kernel the MIXED_BF16 sweeps use) for
 * callers that cannot allocate device memory when they need it: a host
 * framework that hands out all device memory from its own pool and forbids
 * raw allocations after start-up, a latency-critical loop that cannot afford
 * cudaMalloc's implicit synchronisation, or a process whose device-memory
 * budget is already committed.  It allocates nothing; its split-K partial
 * sums live in a file-scope device array of CPALS_NOALLOC_SCRATCH_FLOATS
 * floats (16 MiB) that every GPU loading the library holds until the process
 * exits.
 *   kmajor != 0: out[m][r]    = sum_k Xb[m*K + k]         * (hi + lo)[r][k]
 *   kmajor == 0: out[b][m][r] = sum_k Xb[(b*K + k)*M + m] * (hi + lo)[r][k]
 * Xb: device bf16 tensor (row stride K if kmajor, else M; M % 8 == 0 when
 * kmajor == 0, K % 8 == 0 when kmajor != 0; batch must be 1 when kmajor).
 * Bt: device bf16, two planes [2][Rpad][Kstride], Rpad = R rounded up to 16,
 * plane 0 = bf16(b), plane 1 = bf16(b - plane 0), zero for r >= R or k >= K;
 * Kstride >= K and a multiple of 8.  out: device float32, batch*M*R values,
 * caller-owned.  splits >= 1 splits K across CTAs.  stream: cudaStream_t
 * (NULL = legacy default stream); the call waits for its own work.
 * Errors: CPALS_E_INVALID for bad arguments or when the partial sums,
 * used*batch*M*R floats, exceed CPALS_NOALLOC_SCRATCH_FLOATS (the scratch is
 * not enlarged); `used` is the number of K chunks the kernel runs, K split
 * into chunks of ceil(K/splits) rounded up to a multiple of 64, which can be
 * fewer than `splits`; used == 1 writes out directly and needs no scratch.
 * CPALS_E_UNSUPPORTED
 * for shapes the tensor-core path does not take (alignment, R > 128);
 * CPALS_E_TIMEOUT if a bounded device wait gave up; CPALS_E_CUDA otherwise.
 * The first call on a device takes the scratch array's device address
 * (cudaGetSymbolAddress) and sets the kernels' shared-memory limit, with
 * that device current; host threads making their first calls at the same
 * time do this once (it runs under a lock).  Make that first call before any
 * stream capture.  All calls share the one array and it keeps the last
 * call's contents; calls that overlap on the GPU (other streams, other host
 * threads) race on it and must be serialised by the caller. */
#define CPALS_NOALLOC_SCRATCH_FLOATS (4u << 20)
cpals_status cpals_contract_bf16_noalloc(const void* Xb, const void* Bt, float* out, int64_t batch,
                                         int64_t K, int64_t M, int R, int64_t Kstride,
                                         int kmajor, int splits, void* stream);

/* ---- host-only cost model (no GPU needed) ---- */

/* Flop counts of the kernels this library launches for one step of the
 * given kind (0 = ALS sweep, 1 = PP operator build, 2 = PP approximated
 * sweep with V, 3 = PP operator build as the paper's formula
 * 2R sum_{l=2}^{N-1} C(l+1,2) s^{N-l+2} for an equidimensional tensor)
 * for dims[0..N-1] and rank R.  Contractions only (no solve), Sec. 3.2.3 and
 * Table 1.  Returns CPALS_E_INVALID on bad sizes. */
cpals_status cpals_cost_model(const int64_t* dims, int N, int R, int kind, double* flops);

/* Flop counts of the contractions the order-3 Tucker context launches for
 * one step (0 = Tucker-ALS sweep TTMc, 1 = PP operator build, 2 = PP
 * approximated sweep, 3 = the paper's operator-construction sum
 * 2 sum_{l=2}^{N-1} C(l+1,2) s^{N-l+2} R^{l-1} for equal sizes and ranks)
 * for dims[0..2] and ranks[0..2]; eigen-updates not counted.  Sec. 3.2.2,
 * Table 1.  CPALS_E_INVALID on bad sizes or kind. */
cpals_status cpals_tucker_cost_model(const int64_t* dims, const int* ranks, int kind, double* flops);

#ifdef __cplusplus
}
#endif

#endif /* CPALS_H */
