/*
 * gbosqp: ADMM solver for sparse convex QPs on one NVIDIA GB300 (sm_103a).
 *
 *     minimize    1/2 x'Px + q'x
 *     subject to  l <= Ax <= u                      (paper Section 2, eq. (qp))
 *
 * The method is Algorithm 1 (OSQP) of Schubiger, Banjac & Lygeros, "GPU
 * Acceleration of ADMM for Large-Scale Quadratic Programming", with the
 * linear-system step solved on the reduced KKT system eq. (kkt_red_sc),
 * (P + sigma I + rho A'A) x~ = sigma x - q + A'(rho z - y), by warm-started
 * Jacobi-preconditioned conjugate gradient (Algorithm 3, Section 5.3), after
 * Ruiz equilibration (Algorithm 2, Section 5.4), with R = rho I (or OSQP's
 * per-row rho vector, eq. (rho_vec), with the rho_vector setting),
 * termination checked every 5 iterations and rho adapted every 10 (Table 1),
 * and infeasibility detected at every check (Section 3.1).
 *
 * Conventions shared by every call:
 *   - Matrices are CSR with 64-bit row pointers and 32-bit column indices,
 *     zero-based, columns strictly increasing within each row (no
 *     duplicates), values double.  Internally nnz must be < 2^31 - 256 per
 *     matrix (also for the full P and for [P A'], which osqp_setup builds).
 *   - Bounds with |v| >= GBOSQP_INFINITY (or +-inf) are infinite.  l <= u.
 *   - Unless a call says otherwise, vector arguments are host pointers to
 *     double, caller-owned, of the stated length; the library copies what it
 *     needs and never keeps a caller pointer past the call.
 *   - Calls return GBOSQP_OK (0) or a negative GBOSQP_ERR_* code; they never
 *     abort the process.  gbosqp_last_error() describes the last failure of a
 *     handle.  A handle is not thread safe: one caller thread at a time.
 *   - All device work runs on the stream given in the settings (or on a
 *     stream the library creates); calls that return host data synchronise
 *     that stream.
 */
#ifndef GBOSQP_H
#define GBOSQP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes (negative) ------------------------------------------ */
#define GBOSQP_OK 0
#define GBOSQP_ERR_INVALID_ARG (-1)   /* NULL pointer, bad setting value      */
#define GBOSQP_ERR_DIMENSION (-2)     /* shapes of P, A, q, l, u disagree     */
#define GBOSQP_ERR_CSR (-3)           /* bad row pointers, unsorted or
                                         duplicate or out-of-range columns,
                                         lower entries in an upper P          */
#define GBOSQP_ERR_BOUNDS (-4)        /* l_i > u_i or NaN bound               */
#define GBOSQP_ERR_NONFINITE (-5)     /* NaN or inf in P, A or q              */
#define GBOSQP_ERR_CUDA (-6)          /* a CUDA runtime call failed           */
#define GBOSQP_ERR_OOM (-7)           /* device allocation failed             */
#define GBOSQP_ERR_DEVICE_TIMEOUT (-8)/* a bounded device wait gave up (reserved:
                                         the kernels have no spin-waits; CTAs
                                         combine results by last-arriver
                                         tickets, never by waiting)           */
#define GBOSQP_ERR_UNSUPPORTED (-9)   /* e.g. nnz >= 2^31 - 256, no sm_103a */
#define GBOSQP_ERR_POLICY (-10)       /* learned policy parameters invalid    */

/* ---- solve status (positive) ------------------------------------------ */
#define GBOSQP_SOLVED 1               /* residuals within eq. (termination)  */
#define GBOSQP_MAX_ITER 2             /* max_iter reached                     */
#define GBOSQP_NONFINITE 3            /* NaN/inf appeared in the iterates     */
#define GBOSQP_PRIMAL_INFEASIBLE 4    /* approximate certificate of eq. (prim_infeas)
                                         found (Section 3.1); y holds it       */
#define GBOSQP_DUAL_INFEASIBLE 5      /* approximate certificate of eq. (dual_infeas)
                                         found (Section 3.1); x holds it       */

/* ---- enumerations ------------------------------------------------------ */
#define GBOSQP_FP32 0                 /* matrices and vectors in FP32, PCG dot
                                         products and residual reductions in FP64 */
#define GBOSQP_FP64 1                 /* everything in FP64                   */

#define GBOSQP_RHO_RATIO 0            /* residual-ratio rule, Section 3.4     */
#define GBOSQP_RHO_LEARNED 1          /* MLP policy with ratio-rule fallback  */
#define GBOSQP_RHO_FIXED 2            /* rho never changes                    */

#define GBOSQP_HOST 0                 /* input arrays are host memory         */
#define GBOSQP_DEVICE 1               /* input arrays are device memory of the
                                         settings' device                     */

#define GBOSQP_LOOP_GRAPH 0           /* whole solve = one CUDA graph launch
                                         (conditional while nodes; no host
                                         synchronisation inside the solve)   */
#define GBOSQP_LOOP_HOST 1            /* same kernels driven by a host loop
                                         that reads the stop flags (debug)    */

#define GBOSQP_PCG_CLASSIC 0          /* Algorithm 3: a step is a direction
                                         kernel (A), a K-apply (P A') and a
                                         vector update, three grid-wide phases */
#define GBOSQP_PCG_SINGLE_REDUCTION 1 /* Algorithm 3 rearranged so that a step
                                         needs one reduction phase (Chronopoulos
                                         and Gear, 1989): the vector update rides
                                         on the direction kernel, two kernels a
                                         step, plus one K-apply of M^-1 r per
                                         PCG solve; the same iterates in exact
                                         arithmetic                          */

#define GBOSQP_INFINITY 1e20

/* Matrix selectors for the inspection calls. */
#define GBOSQP_MAT_A 0                /* scaled A, m x n                      */
#define GBOSQP_MAT_PAT 1              /* scaled [P  A'], n x (n + m): row i
                                         holds row i of the full P followed by
                                         row i of A' (columns offset by n)    */

/* Number of doubles written by gbosqp_check(). */
#define GBOSQP_CHECK_FIELDS 16

/* ---- structures -------------------------------------------------------- */
typedef struct {
    int32_t nrows, ncols;
    int64_t nnz;
    const int64_t *rowptr; /* nrows + 1 */
    const int32_t *colind; /* nnz */
    const double *val;     /* nnz */
} gbosqp_csr;

typedef struct {
    double alpha;        /* relaxation, in ]0, 2[            default 1.6  */
    double sigma;        /* > 0                              default 1e-6 */
    double rho0;         /* initial rho, > 0                 default 0.1  */
    double eps_abs;      /* >= 0                             default 1e-3 */
    double eps_rel;      /* >= 0                             default 1e-3 */
    double pcg_lambda;   /* in ]0, 1[, Section 5.3.4         default 0.15 */
    double pcg_eps_min;  /* > 0                              default 1e-7 */
    double rho_min;      /* clamp of adapted rho             default 1e-6 */
    double rho_max;      /*                                  default 1e6  */
    double eps_prim_inf; /* primal infeasibility tolerance, >= 0; 0 turns the
                            test off (Section 3.1)           default 1e-4 */
    double eps_dual_inf; /* dual infeasibility tolerance, >= 0; 0 turns the
                            test off; both 0: the detection kernels are not
                            part of the solve                default 1e-4 */
    int32_t max_iter;    /* ADMM iterations (rounded up to a multiple of
                            check_every)                     default 4000 */
    int32_t max_cg_iter; /* PCG steps per ADMM iteration     default 50   */
    int32_t check_every; /* termination check period, 1..16  default 5    */
    int32_t rho_every;   /* rho period, multiple of check_every, default 10 */
    int32_t scaling_iters; /* Ruiz passes, 0..100            default 10   */
    int32_t precision;   /* GBOSQP_FP32 | GBOSQP_FP64        default FP32 */
    int32_t rho_policy;  /* GBOSQP_RHO_*                     default RATIO */
    int32_t P_is_upper;  /* 1: P holds only its upper triangle (OSQP
                            convention); 0: P is the full symmetric matrix
                                                             default 1    */
    int32_t input_location; /* GBOSQP_HOST | GBOSQP_DEVICE   default HOST */
    int32_t loop_mode;   /* GBOSQP_LOOP_*                    default GRAPH */
    int32_t device;      /* CUDA device ordinal              default 0    */
    int32_t warm_start;  /* 1: every osqp_solve starts from the iterates
                            (and rho) the previous solve ended with, as
                            after a parametric update; 0: cold start unless
                            osqp_warm_start was called        default 0    */
    int32_t rho_vector;  /* 0: R = rho I, the paper's choice for the GPU
                            (Section 5.3); 1: R = rho diag(rs) with
                            rs_i = 1e3 on rows with l_i = u_i and 1 elsewhere,
                            OSQP's eq. (rho_vec) (fewer ADMM iterations on
                            equality-heavy problems, slower PCG)
                                                             default 0    */
    int32_t pcg_variant; /* GBOSQP_PCG_CLASSIC | GBOSQP_PCG_SINGLE_REDUCTION
                                                             default CLASSIC */
    void *cuda_stream;   /* cudaStream_t to run on; NULL: the library
                            creates and owns one.  A caller's stream must
                            stay valid until osqp_cleanup (the handle's
                            device memory, taken from the device's
                            stream-ordered pool, is returned on it)
                                                             default NULL */
    const float *policy_params; /* learned policy parameters (host, FP32,
                                   GBOSQP_POLICY_PARAMS floats) or NULL    */
} gbosqp_settings;

/* Learned-policy parameter vector (FP32): feature mean (4), feature std (4),
 * W1 (64x4, row major), b1 (64), W2 (64x64), b2 (64), W3 (2x64), b3 (2),
 * then log-multiplier clamp, lambda_min, lambda_max, use_lambda (1/0). */
#define GBOSQP_POLICY_PARAMS 4622

typedef struct {
    int32_t status;      /* GBOSQP_SOLVED ... or 0 before the first solve  */
    int32_t iters;       /* ADMM iterations                                */
    int64_t pcg_iters;   /* PCG steps summed over the solve                */
    double obj;          /* 1/2 x'Px + q'x at the returned x               */
    double r_prim;       /* ||Ax - z||_inf (unscaled, last check)          */
    double r_dual;       /* ||Px + q + A'y||_inf (unscaled, last check)    */
    double eps_prim;     /* tolerances of the last check                    */
    double eps_dual;
    double rho;          /* rho at the end of the solve                    */
    double pcg_eps;      /* PCG tolerance at the end of the solve          */
    double setup_ms;     /* wall time of osqp_setup                         */
    double solve_ms;     /* device time of the last osqp_solve             */
    int32_t rho_updates; /* number of rho changes                          */
    int32_t policy_fallbacks; /* learned policy: checks that used the ratio rule */
    int64_t nnz_P;       /* full P                                          */
    int64_t nnz_A;
    int64_t setup_launches; /* kernels launched by osqp_setup              */
    int64_t solve_launches; /* kernels executed by the last osqp_solve
                               (graph nodes included)                      */
} gbosqp_info;

typedef struct gbosqp_handle gbosqp_handle;

/* ---- core calls (paper: Algorithm 1 with Section 5 on the GPU) --------- */

/* Fill *s with the defaults above.  Returns GBOSQP_OK. */
int gbosqp_default_settings(gbosqp_settings *s);

/* Validate the problem, copy it to the device, build P (full), A' (stored
 * explicitly, Section 5.2) and the concatenated [P A'] in CSR, run Ruiz
 * equilibration (Algorithm 2) on the device, compute the Jacobi
 * preconditioner data (Section 5.3.1), and build the solve graph.
 * P: n x n (upper triangle or full, see P_is_upper), A: m x n, q: n, l, u: m,
 * with n >= 1, m >= 0 and n + m < 2^31 - 256 (GBOSQP_ERR_UNSUPPORTED otherwise,
 * as for nnz >= 2^31 - 256 in one matrix, or nnz >= 2^30 - 128 in an upper-triangular P,
 * whose full form is built with 32-bit offsets): m = 0 is a problem without constraints (A has no
 * rows; l and u must still be non-NULL but no element is read), and P may
 * have no nonzeros (a linear program).
 * Memory location of all inputs: settings->input_location.  On success *out
 * owns all device memory until osqp_cleanup.  On failure *out is NULL and
 * the code says why (no handle exists to query gbosqp_last_error; the text
 * is available from gbosqp_setup_error()). */
int osqp_setup(gbosqp_handle **out, const gbosqp_csr *P, const gbosqp_csr *A, const double *q,
               const double *l, const double *u, const gbosqp_settings *settings);

/* Run ADMM from a cold start (x = z = y = 0, rho = rho0), from the point
 * given by osqp_warm_start, or (setting warm_start = 1) from the iterates
 * and rho of the previous solve, until eq. (termination) holds, an infeasibility
 * certificate is found (Section 3.1: at every termination check the
 * differences dx = x^k - x^(k-1), dy = y^k - y^(k-1), scaled to unit
 * inf-norm, are tested against eqs. (prim_infeas) and (dual_infeas) with
 * the strict inequalities taken as < -eps), max_iter, or non-finite
 * iterates.  Returns the status (> 0) or an error (< 0).  The unscaled
 * solution stays on the device until fetched; for an infeasible problem the
 * certificate (unit inf-norm) is returned in y (primal) or x (dual), the
 * other vectors are NaN and the objective is +inf (primal) or -inf (dual). */
int osqp_solve(gbosqp_handle *h);

/* Set rho (Section 5.3.3): only the Jacobi preconditioner is recomputed;
 * no factorization exists.  The next osqp_solve starts from this rho.
 * rho must be > 0 and finite. */
int osqp_update_rho(gbosqp_handle *h, double rho);

/* Make the next osqp_solve start from x (n) and y (m) (unscaled, host);
 * z starts at the projection of Ax onto [l, u].  Either may be NULL (zero). */
int osqp_warm_start(gbosqp_handle *h, const double *x, const double *y);

/* Replace q by q_new (n doubles, on the host, or on the device when the
 * handle was set up with input_location = GBOSQP_DEVICE) without a new
 * set-up: the equilibration of osqp_setup is kept (q_bar = c D q_new) and
 * the tolerances' ||q|| are recomputed.  Matrices, bounds and iterates are
 * untouched (no counterpart in the paper: OSQP's update call for problems
 * solved in sequence, e.g. model predictive control).  A NaN or inf in
 * q_new returns GBOSQP_ERR_NONFINITE and leaves the problem unchanged. */
int osqp_update_lin_cost(gbosqp_handle *h, const double *q_new);

/* Replace l and/or u (m doubles each, same memory rule as above; NULL keeps
 * that side) without a new set-up: l_bar = E l, u_bar = E u with the
 * set-up's E; |v| >= GBOSQP_INFINITY is infinite.  NaN, l > u, l = +inf or
 * u = -inf returns GBOSQP_ERR_BOUNDS and leaves the problem unchanged. */
int osqp_update_bounds(gbosqp_handle *h, const double *l_new, const double *u_new);

/* Copy the unscaled solution of the last solve to host arrays x (n), y (m),
 * z (m); any may be NULL. */
int osqp_get_solution(const gbosqp_handle *h, double *x, double *y, double *z);

/* The same, into device arrays of the handle's device (no host copy). */
int gbosqp_get_solution_device(const gbosqp_handle *h, double *x, double *y, double *z);

/* Solver statistics of the last solve. */
int osqp_get_info(const gbosqp_handle *h, gbosqp_info *info);

/* Free everything the handle owns.  NULL is accepted. */
void osqp_cleanup(gbosqp_handle *h);

/* Text of the last error on h (never NULL). */
const char *gbosqp_last_error(const gbosqp_handle *h);

/* Text of the last osqp_setup failure in this thread (never NULL). */
const char *gbosqp_setup_error(void);

/* Static text for a return code or status. */
const char *gbosqp_error_string(int code);

/* Problem sizes of a handle (any pointer may be NULL). */
int gbosqp_dims(const gbosqp_handle *h, int32_t *n, int32_t *m, int64_t *nnz_A, int64_t *nnz_PAt);

/* ---- inspection and step-level calls (used by the parity tests) ------- *
 * These expose single steps of the method on the handle's scaled problem so
 * that each can be compared with an independent implementation.  They
 * change the handle's iterates only where stated. */

/* Ruiz scaling of Algorithm 2: D (n), E (m), c. */
int gbosqp_get_scaling(const gbosqp_handle *h, double *D, double *E, double *c);

/* Download a scaled matrix (GBOSQP_MAT_A or GBOSQP_MAT_PAT) in CSR with
 * values in double (rounded from FP32 on the FP32 path).  Sizes from
 * gbosqp_dims: rowptr nrows+1, colind and val nnz. */
int gbosqp_get_scaled_csr(const gbosqp_handle *h, int which, int64_t *rowptr, int32_t *colind,
                          double *val);

/* y = M x with the device SpMV kernel (Section 4.3.2 CSR; load-balanced row
 * blocks) for M = GBOSQP_MAT_A (x: n, y: m) or GBOSQP_MAT_PAT (x: n + m,
 * y: n).  x is rounded to the working precision; fp64_accumulate selects
 * FP64 row accumulation (as in the termination check) instead of the working
 * precision (as in PCG). */
int gbosqp_spmv(gbosqp_handle *h, int which, const double *x, double *y, int fp64_accumulate);

/* Algorithm 3 on the device for K = P + sigma I + rho A'A (scaled data) with
 * the Jacobi preconditioner for rho: start from x0 (n), stop when
 * ||K x - b||_inf <= eps or after max_iter steps.  Writes x (n), the step
 * count and the final ||r||_inf.  Does not touch the ADMM iterates. */
int gbosqp_pcg(gbosqp_handle *h, double rho, const double *b, const double *x0, double eps,
               int32_t max_iter, double *x, int32_t *iters, double *r_norm);

/* Set / get the scaled ADMM state: x (n), z (m), y (m), the PCG warm start
 * x~ (n) and rho.  set also recomputes z~ = A x~ and the preconditioner. */
int gbosqp_set_iterates(gbosqp_handle *h, const double *x, const double *z, const double *y,
                        const double *xt, double rho);
int gbosqp_get_iterates(const gbosqp_handle *h, double *x, double *z, double *y, double *xt,
                        double *rho);

/* Run k ADMM iterations from the current state with the host-driven loop
 * (same kernels as the graph), checks and rho updates included, without the
 * cold-start reset.  Writes the number of PCG steps of each iteration to
 * pcg_per_iter (k entries, may be NULL).  Returns status or error. */
int gbosqp_admm_iterations(gbosqp_handle *h, int32_t k, int32_t *pcg_per_iter);

/* Evaluate the termination check at the current state and write, in order:
 * r_prim, r_dual, eps_prim, eps_dual (unscaled, Section 3.1), the scaled
 * r_prim, r_dual, ||Ax||, ||z||, ||Px||, ||A'y||, ||q|| (used by the rho
 * rule and the PCG tolerance), the objective, the rho the residual-ratio
 * rule would set from this check, and three fields of the solve's state
 * (not of this evaluation): the PCG tolerance weight lambda, the learned
 * policy's stall count and its fallback count (decisions the ratio rule
 * took).  The evaluation itself changes no state of the solve. */
int gbosqp_check(gbosqp_handle *h, double out[GBOSQP_CHECK_FIELDS]);

/* ---- learned rho policy (not in the paper) ----------------------------- *
 * A 4-64-64-2 MLP (ReLU) proposes, at every rho decision, rho as the
 * residual-ratio rule's rho times exp(output 0) (output 0 clamped; a zero
 * output reproduces the ratio rule) and a log factor for the PCG tolerance
 * weight lambda (output 1, used when the last parameter is 1).  Its features are
 * log ||r_prim||, log ||r_dual|| (scaled problem), log rho and
 * log(1 + PCG steps since the last decision); it sees (f - mean) / std.
 * Operands are rounded to BF16 (weights, inputs, hidden activations and, in
 * training, the back-propagated signals); products accumulate in FP32.
 * These calls take host arrays, allocate device memory for the call and
 * synchronise. */

/* out (batch x 2) = network(features (batch x 4, raw)) with the device code
 * the solver uses for its decisions. */
int gbosqp_policy_forward(const float *params, const float *features, int32_t batch, float *out);

/* Gradient of loss = sum_k w_k (o_k - t_k)^2 / (2n) over the n samples
 * (features n x 4 raw, targets and weights n x 2) with respect to the
 * weights and biases; grad has GBOSQP_POLICY_PARAMS entries (zero outside
 * W1..b3).  loss may be NULL. */
int gbosqp_mlp_grad(const float *params, const float *features, const float *targets, const float *weights,
                    int32_t n, float *grad, float *loss);

/* `steps` Adam steps (lr, beta1 0.9, beta2 0.999, eps 1e-8) on the weights
 * and biases of params (updated in place), step s using the samples
 * batches[s*batch .. s*batch+batch) (indices into the n samples).  Writes the
 * loss of every step to loss_history (steps entries, may be NULL). */
int gbosqp_mlp_train(float *params, const float *features, const float *targets, const float *weights, int32_t n,
                     const int32_t *batches, int32_t steps, int32_t batch, float lr, float *loss_history);

/* Set the PCG tolerance weight lambda of Section 5.3.4 for the following
 * checks of a handle and the current PCG tolerance eps (> 0) until the next
 * check (step-level call, e.g. for policy lookahead). */
int gbosqp_set_pcg_lambda(gbosqp_handle *h, double lambda, double eps);

/* Make the next osqp_solve continue from the handle's current state: the
 * iterates (e.g. those given to gbosqp_set_iterates), rho, the PCG tolerance
 * and lambda are kept; the iteration count starts from 0, so the next rho
 * decision comes rho_every iterations later (step-level call, e.g. for
 * rollouts that score a rho choice by the rest of the solve). */
int gbosqp_resume(gbosqp_handle *h);

/* Kernel selectors for gbosqp_bench_kernel. */
#define GBOSQP_K_PCG_DIRECTION 0  /* p = -M^{-1}r + beta p, t = rho A p (SpMV A)        */
#define GBOSQP_K_PCG_KAPPLY 1     /* K p = P p + sigma p + A' t, p'Kp (SpMV [P A'])     */
#define GBOSQP_K_PCG_UPDATE 2     /* x, r, M^{-1} r updates, r'y, ||r|| (vectors, n)    */
#define GBOSQP_K_PCG_INIT 3       /* r = K x - b from [P A'] and t0 (SpMV [P A'])       */
#define GBOSQP_K_ADMM_UPDATE 4    /* z~ = A x~, projection, dual update (SpMV A)        */
#define GBOSQP_K_CHECK_A 5        /* ||Ax - z|| etc., FP64 accumulation (SpMV A); the
                                     solve runs it when infeasibility detection is off */
#define GBOSQP_K_CHECK_B 6        /* ||Px + q + A'y|| etc., FP64 (SpMV [P A'])          */
#define GBOSQP_K_INF_A 7          /* the rows of A of the check and of the detection in
                                     one pass gathering x and dx: ||Ax - z|| etc. as
                                     GBOSQP_K_CHECK_A, A dx against the bounds, dy
                                     clipping (SpMV A); the solve runs it in place of
                                     GBOSQP_K_CHECK_A when detection is on          */
#define GBOSQP_K_INF_B 8          /* ||P dx||, ||A'dy||, q'dx (SpMV [P A'])              */
#define GBOSQP_K_PCG_SR_DIRECTION 9 /* single-reduction PCG: p, s = K p, x, r, M^{-1} r
                                       updates, r'y, ||r||, t = rho A M^{-1} r (SpMV A) */
#define GBOSQP_K_PCG_SR_KAPPLY 10   /* single-reduction PCG: w = K M^{-1} r, w'y and the
                                       step coefficients (SpMV [P A'])                */

/* Time `reps` launches of one solve kernel, in the launch configuration the
 * solve uses, on the handle's current vectors, each after a write of twice
 * the L2 size (so the matrix comes from HBM, as inside a solve): the
 * sequence is captured into a CUDA graph on the handle's stream and timed
 * with CUDA events, minus the same graph without the kernel (host launch
 * cost and the flushes excluded).
 * A private copy of the scalar state is used and the iterates are restored,
 * so the next solve is unaffected.  Writes the mean duration in ms. */
int gbosqp_bench_kernel(gbosqp_handle *h, int kernel, int32_t reps, double *avg_ms);

/* y = M x, the same computation and kernel as gbosqp_spmv without FP64
 * accumulation, for callers that cannot let the library allocate device
 * memory during the call: real-time loops that must not take the
 * allocator's latency (cudaMalloc/cudaFree can take milliseconds and
 * cudaFree waits for the whole device), code recording a CUDA stream capture
 * (a device-wide synchronisation would invalidate it), and hosts whose device
 * memory is owned by another allocator.  The paper has no counterpart.
 *
 *   which  GBOSQP_MAT_A (x: n entries, y: m) or GBOSQP_MAT_PAT (x: n + m, y: n)
 *   x, y   device arrays on the handle's device, of float on an FP32 handle
 *          and double on an FP64 handle; caller-owned; may not overlap
 *
 * Allocates nothing: the scratch that combines the parts of rows cut between
 * warps is a fixed device array inside the library (1 MiB, resident on every
 * device that loads the library until the process exits), enough for the
 * launch of any GPU with up to about 20000 resident warps; a plan that needs
 * more is rejected with GBOSQP_ERR_UNSUPPORTED.  The first call on each
 * device looks up that array's device address and keeps it for the process;
 * make that first call before any stream capture, and do not use this call
 * across a device reset (cudaDeviceReset) in the same process.  Every call
 * shares the array (its tickets are cleared at the start of each call and it
 * keeps the last call's partial sums), so calls that overlap on the GPU, from
 * any thread or handle, race: serialise them.  The work is queued on the
 * handle's stream and the call returns without waiting; synchronise that
 * stream (or the device) before reading y. */
int gbosqp_spmv_noalloc(gbosqp_handle *h, int which, const void *x, void *y);

#ifdef __cplusplus
}
#endif

#endif /* GBOSQP_H */
