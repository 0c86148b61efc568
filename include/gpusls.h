/*
 * gpusls.h -- C ABI of the B300 (sm_103a) GPU-SLS hot path.
 *
 * Operations follow "Safe Large-Scale Robust Nonlinear MPC in Milliseconds via
 * Reachability-Constrained System Level Synthesis on the GPU":
 *   qp_*   the ADMM solver for the LTV-QP of Sec. III-B (eq. sqp_qp), Sec. IV-A
 *   sls_*  the SLS controller / reachability solve of Sec. III-D and IV-B
 *   mlp_*  the learned warm start (no counterpart in the paper)
 *
 * Conventions (all calls):
 *   - Arrays are row-major and time-major.  Unless stated otherwise every
 *     array argument is a DEVICE pointer to float64 data.  The library copies
 *     what it keeps; the caller owns its buffers and may free them after the
 *     call returns (calls are stream-ordered on the handle's stream; results
 *     are complete when the call returns).
 *   - A "pool" is the concatenation, QP by QP, of the per-QP arrays in the
 *     order of the dims table; QP b's block starts after the blocks of QPs
 *     0..b-1 (sizes from each QP's own dims).
 *   - Every call returns an int status (GPUSLS_*).  On failure
 *     gpusls_last_error() returns a message for the calling thread.
 *   - Sizes: 1 <= nx <= 80, 1 <= nu <= 32, 0 <= nc <= 64, 0 <= nf <= 64,
 *     1 <= N <= GPUSLS_MAX_N (4096) for the qp_* calls, N <= 512 for sls_*.
 *     Larger values return GPUSLS_ERR_INVALID.  Horizons whose per-chunk
 *     vectors do not fit a CTA's shared memory (thousands of stages) keep
 *     them in a per-CTA region of the handle's device memory instead.
 */
#ifndef GPUSLS_H
#define GPUSLS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* longest horizon the qp_* calls accept */
#define GPUSLS_MAX_N 4096

/* status codes */
#define GPUSLS_OK             0   /* solved (converged to the tolerance)            */
#define GPUSLS_MAX_ITER       1   /* iteration limit reached; results are valid     */
#define GPUSLS_ERR_INVALID   -1   /* invalid argument or dimensions                 */
#define GPUSLS_ERR_NOT_SPD   -2   /* R^, Gamma^-1 or Qu not SPD, or I + C~P~ singular */
#define GPUSLS_ERR_NAN       -3   /* NaN/Inf appeared in the iterates               */
#define GPUSLS_ERR_INFEASIBLE -4  /* per-QP status (qp_info): the solve reached max_iter
                                     and a primal infeasibility certificate holds (see
                                     qp_solve); results are the last iterates       */
#define GPUSLS_ERR_CUDA      -5   /* CUDA runtime error                             */
#define GPUSLS_ERR_TIMEOUT   -6   /* a bounded device wait gave up.  Test hook: with
                                     the environment variable GPUSLS_TEST_WAIT_TIMEOUT
                                     set at launch, every solve first waits (bounded,
                                     ~1 s at most) on a copy barrier that nothing
                                     completes, gives up and returns this status; the
                                     CUDA context stays usable                       */

/* arithmetic of the solve kernels */
#define GPUSLS_FP64 0   /* all arithmetic in float64                                  */
#define GPUSLS_FP32 1   /* all arithmetic in float32 (KKT check stays float64)        */
#define GPUSLS_TF32 2   /* as GPUSLS_FP32, but the factorization's block products run
                           on the tensor cores in TF32 (one pass, FP32 accumulation):
                           faster products, ~1e-3 relative product error that the
                           FP64 KKT gate and the refinement at the eps floor absorb */
#define GPUSLS_MIXED 3  /* FP32 storage and iterations; the blocked factorization's
                           block products on the tensor cores in three TF32 passes
                           (a = a_hi + a_lo, FP32 accumulation: FP32 accuracy), its
                           per-stage nu x nu solves (Gamma_i, R^_i^-1) to FP64
                           accuracy (an FP32 inverse refined by a Newton-Schulz step
                           whose residual is formed in FP64; FP64 elimination for
                           ill-conditioned blocks), the KKT check in FP64 */

/* Dimensions of one LTV-QP (eq. sqp_qp): state nx, input nu, horizon N, stage
 * constraint rows nc (rows of C_k, D_k), terminal rows nf (rows of C_N). */
typedef struct qp_dims {
  int32_t nx, nu, N, nc, nf;
} qp_dims;

/* Solver settings.  The paper fixes none of these (Sec. IV-A.2 names an
 * OSQP-style rho update every sigma iterations); defaults via
 * qp_default_settings(). */
typedef struct qp_settings {
  double rho0;        /* initial penalty (default 0.1)                              */
  double eps;         /* in-loop tolerance on ||r_prim||_inf and ||r_dual||_inf     */
  double eps_kkt;     /* FP64 KKT tolerance gating convergence; <= 0 disables       */
  double rho_min, rho_max;
  int32_t sigma;      /* rho-update interval in iterations; 0 keeps rho fixed       */
  int32_t check_every;/* stop-test interval                                         */
  int32_t max_iter;
  int32_t precision;  /* GPUSLS_FP64, GPUSLS_FP32, GPUSLS_TF32 or GPUSLS_MIXED        */
  int32_t cluster;    /* CTAs (thread blocks) per QP, 1..16; 0 picks by N (at most
                         8).  9..16 are non-portable cluster sizes: qp_setup /
                         qp_batch_setup fail with GPUSLS_ERR_INVALID when the
                         device cannot schedule one such cluster at the
                         handle's shared memory per CTA                     */
  int32_t fixed_iters;/* > 0: run exactly this many iterations, no stop test        */
  int32_t max_refine; /* iterative-refinement rounds allowed at the eps floor (3)   */
  int32_t fallback_iters; /* > 0: a QP whose state came from a warm start
                             (qp_set_warm_start / qp_warm_start_mlp) and has not
                             converged after this many iterations restarts cold
                             (z = y = 0, setup rho) within the same solve        */
  int32_t occupancy; /* 0: as many CTAs per SM as fit; 1: one CTA per SM (the
                         shared-memory request is raised to force it)        */
  double eps_floor;   /* the KKT gate divides eps by 10 on failure, not below this
                         (0, the default: 1e-7 for GPUSLS_FP64, 1e-5 for GPUSLS_FP32);
                         at the floor a failing KKT check triggers a refinement:
                         r <- r + (FP64 u-stationarity residual).  FP32 solves
                         also run the check after 250 iterations at the floor
                         whose residuals stay above it (FP32 rounding can hold
                         them there)                                              */
  int32_t schedule;   /* launch order of the QPs of a batch: 0 (default) in index
                         order; 1 longest expected first, the expectation being
                         each QP's own previous solve on this handle (iterations +
                         180 per factorization); the first solve runs in index
                         order.  Only the order changes, never the result.     */
  int32_t factorization; /* schedule of the rho-dependent reverse scan:
                         0 (default) blocked: each CTA folds its chunk of stage
                         leaves (eq. assoc_init) into one element with combines
                         whose left operand is a leaf, the chunk elements are
                         combined across the cluster, and each chunk's Riccati
                         terms and gains follow from its right neighbour's
                         suffix; a leaf's C~ = B R^-1 B^T has rank nu, so these
                         combines invert nu x nu blocks only (Woodbury).  Falls
                         back to the tree when nu > 32 or its shared-memory
                         buffers do not fit.
                         1 tree: up-sweep and down-sweep of general combines
                         (eq. combination_rules, App. A).  Both give the same
                         P_i and K_i up to rounding.                             */
} qp_settings;

/* Per-QP result summary (host memory). */
typedef struct qp_info {
  int32_t status;     /* GPUSLS_OK, GPUSLS_MAX_ITER, GPUSLS_ERR_INFEASIBLE or a
                         negative error                                      */
  int32_t iters;      /* ADMM iterations run                                       */
  int32_t refactors;  /* rho-dependent factorizations (tree scans) performed       */
  int32_t refines;    /* iterative-refinement rounds applied                       */
  int32_t fallback;   /* 1 if a warm start was abandoned for a cold restart        */
  int32_t pad;
  double rho;         /* final penalty                                             */
  double r_prim, r_dual; /* last in-loop residuals                                 */
  double kkt;         /* FP64 KKT residual of the returned point (-1 if not evaluated) */
} qp_info;

typedef struct qp_handle qp_handle;

/* Fills s with the defaults: rho0 0.1, eps 1e-4, eps_kkt 1e-4, rho range
 * [1e-6, 1e6], sigma 25, check_every 5, max_iter 4000, FP64, cluster 0,
 * eps_floor 0 = automatic (1e-7 in FP64; 1e-5 in FP32, whose operators put a KKT
 * floor near 1e-4 on 61D problems that the refinement at the floor removes). */
void qp_default_settings(qp_settings* s);

/* Message of the last failing call on this thread ("" if none). */
const char* gpusls_last_error(void);

/* qp_setup: one LTV-QP (eq. sqp_qp), Sec. IV-A.
 *   A [N][nx][nx]  B [N][nx][nu]  c [N][nx]   (c_k is the paper's b_k)
 *   Q [N+1][nx][nx] (Q[N] = Q_N)  R [N][nu][nu]  S [N][nu][nx] or NULL (zero)
 *   (Q_k and R_k symmetric, as in the cost of eq. sqp_qp)
 *   q [N+1][nx]  r [N][nu]
 *   C [N][nc][nx]  D [N][nc][nu]  CN [nf][nx]
 *   lo, hi [N*nc + nf]: lo <= G(dx, du) <= hi, +-INFINITY allowed (the paper's
 *   one-sided z <= f is lo = -INF, hi = f)
 *   rho: initial penalty (<= 0 uses s->rho0)
 *   stream: cudaStream_t (NULL = legacy default stream)
 * The handle owns all device workspace. */
int qp_setup(qp_handle** h, qp_dims d,
             const double* A, const double* B, const double* c,
             const double* Q, const double* R, const double* S,
             const double* q, const double* r,
             const double* C, const double* D, const double* CN,
             const double* lo, const double* hi,
             double rho, const qp_settings* s, void* stream);

/* qp_batch_setup: `batch` independent QPs of possibly different dims in one
 * handle; every array argument is a pool (see conventions).  dims is a HOST
 * array [batch].  rho is a HOST array [batch] or NULL (s->rho0). */
int qp_batch_setup(qp_handle** h, int32_t batch, const qp_dims* dims,
                   const double* A, const double* B, const double* c,
                   const double* Q, const double* R, const double* S,
                   const double* q, const double* r,
                   const double* C, const double* D, const double* CN,
                   const double* lo, const double* hi,
                   const double* rho, const qp_settings* s, void* stream);

/* qp_solve: run ADMM (Sec. IV-A) from the handle's current (z, y, rho) -- a
 * cold start z = y = 0 after setup, or the state left by the previous solve
 * or by qp_set_warm_start -- until the stop test passes or `iters`
 * iterations ran (iters <= 0: s->max_iter).  tol > 0 overrides s->eps and
 * s->eps_kkt.  One persistent kernel launch solves every QP of the handle.
 *   x0 [nx] (pool for batches)   outputs: dx [N+1][nx], du [N][nu],
 *   lam [N*nc+nf] (unscaled multipliers lambda = rho * y), all pools.
 *   info: HOST array [batch] or NULL.
 * A QP that reaches the iteration limit is classified from the change w of
 * its multipliers over the last check interval (Farkas: the constraints
 * E xi = e of the dynamics and x_0, and lo <= G xi <= hi, admit no xi when
 * E^T mu + G^T w = 0 and sigma(w) + e^T mu < 0, sigma the support function
 * of the box; mu follows from the x-components, the u-components are the
 * residual): with W = ||w||_inf, a residual and a push against infinite
 * bounds of at most eps W and sigma(w) + e^T mu < -eps W, info[b].status is
 * GPUSLS_ERR_INFEASIBLE, else GPUSLS_MAX_ITER.
 * Returns GPUSLS_OK if every QP converged, GPUSLS_MAX_ITER if some did not
 * (iteration limit or infeasible: see info), or the most severe other
 * negative per-QP status. */
int qp_solve(qp_handle* h, const double* x0, int32_t iters, double tol,
             double* dx, double* du, double* lam, qp_info* info);

/* qp_set_warm_start: set the ADMM state (z, y = lambda / rho) and rho of every
 * QP (pools of [N*nc+nf]; rho a HOST array [batch]).  z or y may be NULL
 * (zero); rho may be NULL (keep).  Used by the learned warm start. */
int qp_set_warm_start(qp_handle* h, const double* z, const double* y, const double* rho);

/* qp_get_state: copy (z, y) pools and rho (HOST [batch]) out of the handle. */
int qp_get_state(qp_handle* h, double* z, double* y, double* rho);

/* qp_update: replace problem data of every QP in place (same dims; pools;
 * any argument may be NULL to keep the current array) -- a new SQP
 * linearization (A, B, c, Q, R, S, C, D, CN) and/or new linear terms and
 * bounds (q, r, lo, hi).  Allocates nothing.  Any change other than lo/hi
 * invalidates the cached factorization (the next solve refactors). */
int qp_update(qp_handle* h, const double* A, const double* B, const double* c,
              const double* Q, const double* R, const double* S,
              const double* q, const double* r,
              const double* C, const double* D, const double* CN,
              const double* lo, const double* hi);

/* qp_reset: cold start of every QP: z = y = 0, rho = the setup value, cached
 * factorization invalidated, refinement corrections of r undone. */
int qp_reset(qp_handle* h);

/* qp_kkt: FP64 KKT residual of a candidate point (dx, du, lam pools) for
 * every QP of the handle (reading of the paper's undefined "residual":
 * max of dynamics, bound violation, u-stationarity after costate recovery,
 * complementarity).  out: HOST array [batch]. */
int qp_kkt(qp_handle* h, const double* x0, const double* dx, const double* du,
           const double* lam, double* out);

/* qp_riccati: run the rho-dependent factorization (eq. augmented_matrices,
 * eq. assoc_init, the reverse scan of eq. combination_rules and eq.
 * controller_cache) at the handle's current rho and copy out
 * P [N+1][nx][nx] and K [N][nu][nx] (pools).  Exposes the refactor for
 * per-step parity checks. */
int qp_riccati(qp_handle* h, double* P, double* K);

void qp_destroy(qp_handle* h);

/* ------------------------------------------------------------------------ */
/* SLS controller synthesis and reachability margins (Sec. III-D, IV-B)     */
/* ------------------------------------------------------------------------ */
typedef struct sls_handle sls_handle;

/* sls_setup: workspace for SLS problems of dims d (nx, nu, N, nc stage rows,
 * nf terminal rows).  per_j_tau != 0 prepares one controller problem per
 * disturbance index j (costs depending on tau_{k,j}, eq.
 * sls_cost_matrices_tau); per_j_tau == 0 shares one problem (tau = 0).
 * precision: GPUSLS_FP64 or GPUSLS_FP32.  Allocates all device memory. */
int sls_setup(sls_handle** h, qp_dims d, int32_t precision, int32_t per_j_tau, void* stream);

/* sls_setup_ex: as sls_setup, with the launch shape of the controller
 * problems' factorization taken from inner (cluster: CTAs per problem, 0 =
 * by horizon; occupancy; factorization schedule); inner may be NULL. */
int sls_setup_ex(sls_handle** h, qp_dims d, int32_t precision, int32_t per_j_tau, const qp_settings* inner,
                 void* stream);

/* sls_solve: the SLS controller QP (eq. fastsls_qp) by per-j reverse scans
 * (eq. robust_combin, eq. backward_prop) and forward propagation
 * (eq. forward_prop), plus the margins of Sec. III-D.
 *   A [N][nx][nx]  B [N][nx][nu]  E [N][nx][nx] (disturbance scaling E_j)
 *   Qbar [nx][nx]  Rbar [nu][nu]  QbarN [nx][nx]   (SPD)
 *   C [N][nc][nx]  D [N][nc][nu]  CN [nf][nx]
 *   tau [N+1][N][max(nc, nf)] or NULL (zero): tau[k][j][:nc] for stage k < N,
 *       tau[N][j][:nf] terminal; requires a per_j_tau handle when non-NULL.
 * Outputs (any may be NULL):
 *   Phi_x [N*nx][N*nx]: block row k-1 (k = 1..N), block column j = Phi_x_{k,j}
 *         (zero for k <= j; Phi_x_{j+1,j} = E_j)
 *   Phi_u [N*nu][N*nx]: block row k (k = 0..N-1), block column j = Phi_u_{k,j}
 *   h [N][nc]: h_k = sum_{j<k} ||C_k Phi_x_{k,j} + D_k Phi_u_{k,j}||_{2,row}
 *   hf [nf]:   h^f = sum_{j<N} ||C_N Phi_x_{N,j}||_{2,row}
 * All arrays are device float64. */
int sls_solve(sls_handle* h, const double* A, const double* B, const double* E,
              const double* Qbar, const double* Rbar, const double* QbarN,
              const double* C, const double* D, const double* CN, const double* tau,
              double* Phi_x, double* Phi_u, double* hk, double* hf);

/* sls_tau: the FastSLS duals of App. B from the last sls_solve on h and the
 * unscaled QP multipliers lam [N*nc + nf] (device float64, the qp_solve
 * layout) of the tightened nominal QP:
 *   beta_{k,j}[c] = || row c of C_k Phi_x_{k,j} + D_k Phi_u_{k,j} ||^2  (k < N)
 *   beta_{N,j}[c] = || row c of C_N Phi_x_{N,j} ||^2
 *   tau_{k,j}[c]  = |lam_{k,c}| / sqrt(beta_{k,j}[c] + eps)  for j < k <= N,
 * zero for k <= j (where Phi_{k,j} = 0) and beyond a stage's rows.  The row
 * norms are the ones the margins of that sls_solve were summed from (solve
 * precision).  |lam|: a two-sided row lo <= g <= hi is the paper's pair of
 * one-sided rows with one row norm and at most one of them active.
 *   tau: device float64 [N+1][N][max(nc, nf)] (the sls_solve tau layout).
 * Errors: GPUSLS_ERR_INVALID before any sls_solve on h, for eps <= 0 or null
 * pointers. */
int sls_tau(sls_handle* h, const double* lam, double eps, double* tau);

void sls_destroy(sls_handle* h);

/* fastsls_solve: `iters` steps of the FastSLS alternation between the robust
 * controller and the tightened nominal trajectory (Sec. III-D, eq.
 * nmpc_problem_tightened, eq. fastsls_qp, App. B; the RTI order of Sec. IV-C):
 * each step
 *   1. sls_solve with the duals of the previous step (tau_in on the first
 *      step, NULL = zero) -> Phi_x, Phi_u, margins h_k, h^f;
 *   2. tightens the bounds: stage-k rows lo + h_k <= g <= hi - h_k, terminal
 *      rows by h^f (infinite bounds stay infinite; h_0 = 0);
 *   3. qp_update(q, bounds only: the cached factorization stays valid) and
 *      qp_solve(q) from q's current ADMM state (the previous step's solution
 *      after the first);
 *   4. sls_tau from the new multipliers and the Phi of step 1.
 * q: a qp_handle holding ONE QP whose data (A, B, C, D, CN) are the nominal
 *   linearization; s: a per-j-tau sls_handle of the same dims.
 * A, B, E, Qbar, Rbar, QbarN, C, D, CN: the sls_solve inputs (the same A, B,
 *   C, D, CN as q's data); lo, hi [N*nc+nf]: the untightened bounds; x0 [nx].
 * Outputs (device float64): tau_out (NULL: not copied) the duals of the last
 *   step, ready as the next call's tau_in; dx, du, lam the last tightened QP
 *   solution (qp_solve layouts); Phi_x, Phi_u (may be NULL), hk [N][nc],
 *   hf [nf] (NULL if nf == 0) of the last step -- the returned trajectory is
 *   feasible for the tightening of the same step.  info: HOST qp_info of the
 *   last QP solve (or NULL).
 * Returns the worst qp_solve status over the steps (GPUSLS_OK, GPUSLS_MAX_ITER)
 * or the first error. */
int fastsls_solve(qp_handle* q, sls_handle* s, const double* A, const double* B, const double* E,
                  const double* Qbar, const double* Rbar, const double* QbarN,
                  const double* C, const double* D, const double* CN,
                  const double* lo, const double* hi, const double* x0,
                  int32_t iters, double eps_tau, const double* tau_in, double* tau_out,
                  double* dx, double* du, double* lam,
                  double* Phi_x, double* Phi_u, double* hk, double* hf, qp_info* info);

/* ------------------------------------------------------------------------ */
/* Learned warm start (no counterpart in the paper)                         */
/* ------------------------------------------------------------------------ */
/* A two-hidden-layer ReLU MLP  h1 = relu(X W1^T + b1), h2 = relu(h1 W2^T + b2),
 * Y = h2 W3^T + b3, trained on the GPU with the MSE loss (1/2B) sum (Y - T)^2
 * on normalized inputs/targets and Adam (beta 0.9/0.999, eps 1e-8).  Every
 * GEMM runs on the tensor cores with BF16 operands (rounded to nearest even
 * from the FP32 values) and FP32 accumulation; weights, biases and Adam
 * moments are FP32.  All float arrays below are DEVICE float32, row-major:
 * W1 [hidden][n_in], W2 [hidden][hidden], W3 [n_out][hidden], X [B][n_in],
 * T, Y [B][n_out].  Errors: GPUSLS_ERR_INVALID for bad sizes/pointers,
 * GPUSLS_ERR_CUDA for runtime failures. */
typedef struct mlp_handle mlp_handle;

int mlp_create(mlp_handle** h, int32_t n_in, int32_t hidden, int32_t n_out, int32_t max_batch, void* stream);
/* copy parameters in (restarts Adam) / out (NULL entries skipped) */
int mlp_set_params(mlp_handle* h, const float* W1, const float* b1, const float* W2, const float* b2,
                   const float* W3, const float* b3);
int mlp_get_params(mlp_handle* h, float* W1, float* b1, float* W2, float* b2, float* W3, float* b3);
/* per-column mean / standard deviation of X [count][n_in] and T [count][n_out]
 * used to normalize inputs and targets (identity until called) */
int mlp_fit_normalization(mlp_handle* h, const float* X, const float* T, int32_t count);
/* set / get the normalization (means and standard deviations; device float32
 * [n_in], [n_in], [n_out], [n_out]; NULL outputs skipped) */
int mlp_set_normalization(mlp_handle* h, const float* xm, const float* xs, const float* ym, const float* ys);
int mlp_get_normalization(mlp_handle* h, float* xm, float* xs, float* ym, float* ys);
/* mlp_save / mlp_load: the network as a binary file (path: a HOST C string):
 * the 8-byte tag "GSLSMLP1", int32 n_in, hidden, n_out (native byte order),
 * then float32 W1, b1, W2, b2, W3, b3 (the mlp_set_params layouts) and xm,
 * xs, ym, ys.  mlp_load fills a handle of the same sizes and restarts Adam;
 * a missing, short, longer or foreign file, or other sizes, give
 * GPUSLS_ERR_INVALID and leave the handle unchanged. */
int mlp_save(mlp_handle* h, const char* path);
int mlp_load(mlp_handle* h, const char* path);
/* Y = denormalized network output for raw inputs X (B <= max_batch) */
int mlp_forward(mlp_handle* h, const float* X, int32_t B, float* Y);
/* gradients of the loss at ALREADY-normalized (Xn, Tn) into grads (device,
 * the concatenation W1, b1, W2, b2, W3, b3) and the loss (HOST float*, may be NULL) */
int mlp_gradients(mlp_handle* h, const float* Xn, const float* Tn, int32_t B, float* grads, float* loss);
/* one Adam step on a minibatch of raw (X, T); loss: HOST float* or NULL */
int mlp_train_step(mlp_handle* h, const float* X, const float* T, int32_t B, float lr, float* loss);
void mlp_destroy(mlp_handle* h);

/* qp_warm_start_mlp: evaluate the network on features [batch][n_in] (one row
 * per QP of q; n_out must be 2 m + 1 with m = N nc + nf) and set every QP's
 * ADMM state: z = clamp(Y[0:m], lo, hi), rho = clamp(exp(Y[2m]), rho_min,
 * rho_max), y = Y[m:2m] / rho (Y[m:2m] predicts the unscaled multiplier).
 * Runs on the network's stream; give both handles the same stream. */
int qp_warm_start_mlp(qp_handle* q, mlp_handle* h, const float* features, double rho_min, double rho_max);

/* Linearization features (no counterpart in the paper): what a warm-start
 * network sees of a QP, computed from the data the caller gave the handle.
 * Row of QP b: [x0 (nx), then GPUSLS_FEATURE_P values each of four fixed
 * +-1 (Rademacher) projections, scaled by 1/sqrt(inputs), of
 * mean_k (A_k - I), mean_k B_k, mean_{k<=N} q_k and the per-row mean over the
 * stages of the finite upper bounds (clamped to +-10), then N / 128]:
 * nx + 4 GPUSLS_FEATURE_P + 1 floats.  The signs come from a 32-bit hash of
 * (projection, row, input index), so no matrix is stored. */
#define GPUSLS_FEATURE_P 16

/* qp_features: features of the QPs idx[0..count) (device int32 array, or
 * NULL with count == batch for all QPs in order) for the initial states x0
 * (device pool, qp_solve layout) into out: device float32 [count][ld],
 * ld >= nx + 4 GPUSLS_FEATURE_P + 1. */
int qp_features(qp_handle* q, const double* x0, const int32_t* idx, int32_t count, int32_t ld, float* out);

/* qp_warm_start_heads: learned warm start with one network per shape family.
 * Head hh serves the QPs idx[hh][0..counts[hh]) (device int32 arrays, no QP
 * listed twice): its input is the QP's features (qp_features, so n_in = nx +
 * 4 GPUSLS_FEATURE_P + 1), its output is laid out for a horizon n_stage[hh]
 * >= every served QP's N: z of stage rows (n_stage nc), z of terminal rows
 * (nf), lambda likewise, log rho -- n_out = 2 (n_stage nc + nf) + 1.  A QP of
 * horizon N takes its first N nc stage rows and the terminal rows; z is
 * clamped to the bounds, y = lambda / rho, rho clamped to [rho_min, rho_max].
 * x0: device pool (qp_solve layout).  Runs on the QP handle's stream. */
int qp_warm_start_heads(qp_handle* q, int32_t n_heads, mlp_handle* const* heads, const int32_t* const* idx,
                        const int32_t* counts, const int32_t* n_stage, const double* x0,
                        double rho_min, double rho_max);

/* ------------------------------------------------------------------------ */
/* Serving graph: one batched serving step captured as a CUDA graph         */
/* ------------------------------------------------------------------------ */
/* qp_graph_create captures one serving step of the batch held by q into a
 * CUDA graph (on a private stream; nothing runs at creation):
 *   qp_reset -> learned warm start from features [batch][n_in] (only when
 *   m != NULL; same rules as qp_warm_start_mlp) -> x0 taken from the device
 *   pool x0 (qp_solve layout) -> the persistent solve kernel (settings of q)
 *   -> per-QP results copied to the device arrays info_i [batch][8] (status,
 *   iters, refactors, refines, fallback, 0, 0, 0) and info_d [batch][4] (rho,
 *   r_prim, r_dual, kkt); either may be NULL.
 * dx, du, lam: device outputs in the qp_solve layouts.  Every pointer given
 * here is baked into the graph: the buffers must stay valid, and be refilled
 * in place, while the graph exists.  Problem data may change between
 * launches through qp_update (same dims).  While a graph exists, calls that
 * rewrite the output pointers of q (qp_solve, qp_riccati) must not run
 * between launches.
 * qp_graph_launch replays the step on `stream` (no host synchronization, no
 * host copies).  Errors: GPUSLS_ERR_INVALID for null handles or pointers,
 * GPUSLS_ERR_CUDA if capture, instantiation or launch fails. */
typedef struct qp_graph qp_graph;
int qp_graph_create(qp_graph** g, qp_handle* q, mlp_handle* m, const float* features, const double* x0,
                    double* dx, double* du, double* lam, int32_t* info_i, double* info_d,
                    double rho_min, double rho_max);
int qp_graph_launch(qp_graph* g, void* stream);
/* qp_graph_create_heads: as qp_graph_create, with the learned warm start
 * of qp_warm_start_heads (features computed inside the graph from the
 * handle's current data and x0) in place of the single network.  The index
 * arrays, the networks and x0 must stay valid while the graph exists. */
int qp_graph_create_heads(qp_graph** g, qp_handle* q, int32_t n_heads, mlp_handle* const* heads,
                          const int32_t* const* idx, const int32_t* counts, const int32_t* n_stage,
                          const double* x0, double* dx, double* du, double* lam, int32_t* info_i, double* info_d,
                          double rho_min, double rho_max);
/* qp_graph_kernel_count: number of kernel launches one replay of the graph
 * performs (the kernel nodes of the captured graph), into *n (HOST). */
int qp_graph_kernel_count(qp_graph* g, int32_t* n);
void qp_graph_destroy(qp_graph* g);

/* ------------------------------------------------------------------------ */
/* Analytic models and the SQP / RTI outer loop (Sec. III-B, Sec. IV-C,      */
/* App. C, App. D)                                                          */
/* ------------------------------------------------------------------------ */
#define GPUSLS_MODEL_DUBINS 0   /* App. C: x = (p_x, p_y, theta), u = omega, speed v */
#define GPUSLS_MODEL_QUAD2D 1   /* App. D: x = (p_x, p_y, phi, v_x, v_y, phidot), u = thrusts;
                                   explicit Euler step of the continuous dynamics */
#define GPUSLS_MODEL_MAX_OBS 16

/* One model instance.  Cost: 1/2 |x - xref|^2_diag(Qd) + 1/2 |u - uref|^2_diag(Rd)
 * per stage, 1/2 |x_N - xref|^2_diag(QNd) terminal.  Constraints: u_lo <= u <=
 * u_hi (two-sided rows) and per obstacle (c_x, c_y, r) in obs[3 o .. 3 o + 2]:
 * r^2 - (p_x - c_x)^2 - (p_y - c_y)^2 <= 0 on every stage and on x_N
 * (eq. obstacle_constraints).  E: disturbance scaling [nx][nx] row-major.
 * Only the first nx (nu) entries of the per-state (per-input) arrays are read. */
typedef struct model_spec {
  int32_t kind, N, n_obs, pad;
  double dt, v, mass, grav, arm, inertia;
  double u_lo[2], u_hi[2];
  double xref[6], uref[2], Qd[6], Rd[2], QNd[6];
  double E[36];
  double obs[3 * GPUSLS_MODEL_MAX_OBS];
} model_spec;

/* model_dims: the LTV-QP dims of a model: nx, nu, N, nc = nu + n_obs, nf = n_obs. */
int model_dims(const model_spec* m, qp_dims* d);

/* model_linearize: the LTV-QP eq. sqp_qp around nominal trajectories, every
 * stage of every trajectory in parallel (the parallel linearization of
 * Fig. fig:schematic).  X [batch][N+1][nx], U [batch][N][nu], x0bar
 * [batch][nx] (device).  Outputs are pools in the qp_setup layouts
 * (batch QPs of identical dims): A_k, B_k the analytic Jacobians;
 * c_k = f(x_k, u_k) - x_{k+1} (the paper's b_k); Gauss-Newton Q_k =
 * diag(Qd), R_k = diag(Rd), S_k = 0, Q_N = diag(QNd); q_k, r_k, q_N the cost
 * gradients at the nominal; stage rows [input box; obstacles] with C =
 * (0; grad g_o), D = (I; 0), bounds (u_lo - u_k, u_hi - u_k) and
 * (-inf, -g_o(x_k)); terminal obstacle rows likewise; dx0 = x0bar - x_0.
 * Synchronous on `stream`. */
int model_linearize(const model_spec* m, int32_t batch, const double* X, const double* U, const double* x0bar,
                    double* A, double* B, double* c, double* Q, double* R, double* S, double* q, double* r,
                    double* C, double* D, double* CN, double* lo, double* hi, double* dx0, void* stream);

/* model_merit: l1 merit phi = J(X + a dX, U + a dU) + w (sum_k |f(x_k, u_k) -
 * x_{k+1}|_1 + |x_0 - x0bar|_1 + input-box and obstacle violations) per
 * trajectory, a = alpha[b] (device [batch]; NULL, or dX = dU = NULL: a = 0);
 * out: device [batch].  The step-size search of sqp_solve uses it. */
int model_merit(const model_spec* m, int32_t batch, const double* X, const double* U, const double* dX,
                const double* dU, const double* alpha, const double* x0bar, double w, double* out, void* stream);

/* sqp_setup: a batch of `batch` trajectories of one model, with the QP
 * settings s for the inner LTV-QP solves.  robust != 0 (batch 1, N <= 512)
 * adds the SLS controller and tightening of each RTI step (fastsls_solve with
 * E_j = E, Qbar = Rbar = QbarN = I).  Allocates all device memory. */
typedef struct sqp_handle sqp_handle;
int sqp_setup(sqp_handle** h, const model_spec* m, int32_t batch, const qp_settings* s, int32_t robust,
              void* stream);

/* sqp_solve: `iters` SQP iterations (Sec. III-B) in place on the device
 * trajectories X, U from the initial states x0bar: linearize, solve the
 * LTV-QPs (warm-started from the previous iteration's ADMM state), and step
 * x <- x + alpha dx, u <- u + alpha du with alpha in {1, 1/2, ..., 1/128}
 * chosen per trajectory as the first that lowers the l1 merit (weight
 * merit_w; line_search == 0: alpha = 1).  alpha_out: HOST [iters][batch]
 * or NULL; info: HOST qp_info [batch] of the last QP solve, or NULL.
 * Returns the worst QP status (GPUSLS_OK / GPUSLS_MAX_ITER) or an error. */
int sqp_solve(sqp_handle* h, double* X, double* U, const double* x0bar, int32_t iters, double merit_w,
              int32_t line_search, double* alpha_out, qp_info* info);

/* rti_step: one real-time iteration (Sec. IV-C) for every trajectory: one
 * linearization at the nominal (X, U) and the measured state x, one QP solve
 * (robust handles: the controller update from the previous step's duals,
 * the tightened QP and new duals, as fastsls_solve with one step), the full
 * step, the first input applied to the disturbed plant x <- f(x, u_0) + E w
 * (W [batch][nx], device, or NULL for no disturbance), and the nominal
 * shifted one stage (the last stage kept).  u_applied [batch][nu] (device or
 * NULL) receives u_0; hk [N][nc], hf [nf] (robust only, device or NULL)
 * receive the step's margins. */
int rti_step(sqp_handle* h, double* X, double* U, double* x, const double* W, double* u_applied,
             double* hk, double* hf, qp_info* info);

/* sqp_reset_duals: cold ADMM state and zero controller duals (next rti_step
 * starts the alternation from tau = 0). */
int sqp_reset_duals(sqp_handle* h);
void sqp_destroy(sqp_handle* h);

/* ------------------------------------------------------------------------ */
/* Allocation-free KKT residual (the paper has no counterpart)              */
/* ------------------------------------------------------------------------ */
/* Largest scratch (in doubles) gpusls_kkt_noalloc can use: it needs
 * (N+1)*nx + N*nu doubles, so e.g. nx = 75, nu = 21, N <= 1364. */
#define GPUSLS_NOALLOC_MAX_SCRATCH 131072

/* gpusls_kkt_noalloc: the FP64 KKT residual of qp_kkt for ONE QP, for callers
 * that cannot allocate device memory when they need it (a real-time control
 * loop where cudaMalloc may block or synchronize the device, a context that
 * forbids allocation, or a host runtime that owns all device buffers).  It
 * needs no handle and calls no allocator.
 *   Sizes accepted: 1 <= nx <= 80, 1 <= nu <= 64, 0 <= nc <= 64, 0 <= nf <= 64,
 *   N >= 1 and (N+1)*nx + N*nu <= GPUSLS_NOALLOC_MAX_SCRATCH (the residual
 *   needs no blocked buffers, so nu may exceed the solver's limit of 32).
 *   Inputs are device float64 arrays in the qp_setup layouts (S may be NULL)
 *   plus the candidate point x0 [nx], dx [N+1][nx], du [N][nu], lam [N*nc+nf];
 *   out: device float64 [5] receiving (kkt, dynamics, bound violation,
 *   u-stationarity, complementarity).  Runs asynchronously on `stream`.
 * Scratch: a fixed device array of GPUSLS_NOALLOC_MAX_SCRATCH doubles, held by
 * every GPU that loads the library until the process exits.  Sizes outside the
 * ranges above return GPUSLS_ERR_INVALID (with the sizes in
 * gpusls_last_error()).  Every call looks up the array's device address on the
 * current device (allocation-free); the first call on a device also loads the
 * library's device code there, so make that first call before any stream
 * capture.  Every call uses the same array (it is fully rewritten before it is
 * read): calls whose executions overlap on a device -- e.g. on two streams at
 * once -- race on it. */
int gpusls_kkt_noalloc(qp_dims d, const double* A, const double* B, const double* c,
                       const double* Q, const double* R, const double* S,
                       const double* q, const double* r,
                       const double* C, const double* D, const double* CN,
                       const double* lo, const double* hi,
                       const double* x0, const double* dx, const double* du, const double* lam,
                       double* out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GPUSLS_H */
