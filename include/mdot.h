/*
 * mdot.h -- C ABI of the GB300 (sm_103a) MDOT-PNCG library.
 *
 * Method: Kemertas, Jepson, Farahmand, "Efficient and Accurate Optimal Transport with Mirror
 * Descent and Conjugate Gradients" (arXiv 2307.08507).  The library solves the discrete optimal
 * transport problem  min_{P in U(r, c)} <P, C>  (Sec. 2.1) by MDOT (Alg. 1): a sequence of
 * entropic problems at growing inverse temperature gamma, each solved in the dual (Eq. (4)) by
 * PNCG (Alg. 2) with the approximate-Wolfe line search of App. B, warm-started by Eq. (13), and
 * finally rounded onto U(r, c) by Alg. 3.
 *
 * Conventions used throughout (the paper's):
 *   P_ij(u, v; gamma) = exp(u_i + v_j - gamma C_ij)          (Eq. (2))
 *   gamma is the INVERSE temperature; it grows from gamma_i to gamma_f.
 *   Potentials u, v are in log scale; f = u / gamma_f, g = v / gamma_f are the same potentials in
 *   cost units.  (u, v) and (u + d, v - d) describe the same plan (footnote to Prop. 1).
 *
 * Memory and ownership:
 *   - Every array argument is a DEVICE pointer (CUDA global memory on the handle's device) unless
 *     the parameter name ends in _host or the function name ends in _host.  Scalars returned
 *     through pointers (cost_out, gap_out, info) are HOST pointers.
 *   - Vectors of length n are dense and contiguous; a cost matrix is n x n, row-major, float32,
 *     leading dimension n, entries in [0, 1] (Sec. 2.1 assumes C in [0, 1]^{n x n}).
 *   - The caller owns all inputs and outputs.  The library never frees or retains caller memory
 *     past the call.  The handle owns its workspace (allocated once in mdot_create).
 *   - All work is ordered on the handle's CUDA stream; the calls return after the results are
 *     complete (they synchronise that stream) unless stated otherwise.
 *
 * Errors: every entry point returns an mdot_status.  MDOT_ERR_INVALID_ARG leaves outputs
 * untouched.  MDOT_ERR_NOT_CONVERGED still fills every output with the best iterate.
 * MDOT_ERR_CUDA means a CUDA call failed (the message is in mdot_last_error()).
 */
#ifndef MDOT_H
#define MDOT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum mdot_status {
    MDOT_OK = 0,
    MDOT_ERR_INVALID_ARG = 1,     /* bad size, null pointer, out-of-range parameter          */
    MDOT_ERR_NOT_CONVERGED = 2,   /* an iteration cap was hit; outputs hold the best iterate */
    MDOT_ERR_NUMERIC = 3,         /* a non-finite value appeared where none is allowed       */
    MDOT_ERR_TIMEOUT = 4,         /* a bounded device-side wait gave up                      */
    MDOT_ERR_OOM = 5,             /* workspace allocation failed                             */
    MDOT_ERR_CUDA = 6,            /* a CUDA runtime call failed                              */
    MDOT_NOT_READY = 7            /* asynchronous result not available yet                   */
} mdot_status;

/* Arithmetic used for the per-entry work of a dual evaluation (the O(n) work, the line-search test,
 * rounding sums and the bound are fp64 in every mode).  The `precision` argument of the
 * *_dual_eval* calls may be OR'ed with MDOT_PREC_TENSOR_CORES (see mdot_params.tensor_cores). */
#define MDOT_PREC_TENSOR_CORES 256
typedef enum mdot_precision {
    MDOT_PREC_AUTO = 0,   /* fp32 entries while its noise floor is below the stage tolerance,
                             fp64 entries for the final stage when it is not (and for n <= 512) */
    MDOT_PREC_FP32 = 1,   /* always fp32 entries (exact cost-unit difference, ex2.approx)      */
    MDOT_PREC_FP64 = 2,   /* always fp64 entries                                              */
    MDOT_PREC_FP32A = 3   /* fp32 entries with an accurately reduced exponent (the product
                             exact inside an fma) and a polynomial exp2 (about 1 ulp, unbiased);
                             AUTO uses it once a stage's tolerance is below 2e-6               */
} mdot_precision;

/* Source of the cost matrix for the *_points entry points: C_ij regenerated inside every pass
 * from coordinates x_i, y_j (n x 3 fp32 each, row-major; 2-D data uses z = 0):
 *   d_k = x_ik - y_jk,  D = (d0*d0 + d1*d1) + d2*d2 (SQEUCLID) or (|d0| + |d1|) + |d2| (L1),
 *   C_ij = D * scale,   every operation rounded to fp32 in exactly this order,
 * so C never occupies memory (the on-the-fly cost of Sec. 5.1) and equals the matrix a caller
 * would build with the same fp32 operations.  scale is normally 1 / max_ij D. */
typedef enum mdot_cost_kind {
    MDOT_COST_SQEUCLID = 1,
    MDOT_COST_L1 = 2
} mdot_cost_kind;

/* Parameters of Alg. 1 / Alg. 2 / App. B.  Fill with mdot_default_params, then override. */
typedef struct mdot_params {
    double  gamma_i;        /* first inverse temperature; Sec. 5.2 default 2^4                     */
    double  gamma_f;        /* final inverse temperature; <= 0: derived from eps_target (Prop. 2)  */
    double  p;              /* stopping exponent, eps_d = H_min / gamma^p (Alg. 1); 1.5             */
    double  q;              /* decay factor, gamma <- min(q gamma, gamma_f) (Alg. 1); 2^(1/3)        */
    double  ls_c1, ls_c2;   /* approximate Wolfe constants (App. B, Eq. (24)); 0.1 and 0.5          */
    int32_t ls_max_trials;  /* phi' evaluations per line search before the lower end is taken; 50   */
    int32_t max_iter;       /* PNCG iterations per stage; 100000                                    */
    int32_t precision;      /* mdot_precision                                                      */
    int32_t warm_start;     /* 0: Taylor step, Eq. (13); 1: eps-scaling (Sec. 3.3.1); 2: none (the   */
                            /*    previous iterate; the per-row scales are predicted from r~, which  */
                            /*    this start can miss by more than the exponent range: may fail)     */
    double  final_tol;      /* > 0: ||grad g||_1 target of the final stage instead of eps_d / 2     */
    double  fp32_floor;     /* ||grad g||_1 below which fp32 entries are not trusted; 2e-7 (the
                               spread that fp32 entries and fp32 sums leave in the marginals of a
                               converged plan, ~1.6e-7 measured): tighter stage tolerances run to it
                               in fp32 and (AUTO) finish in fp64 entries                         */
    int32_t profile;        /* non-zero: time each kernel launch with CUDA events (mdot_info t_*)    */
    int32_t smoothing;      /* 0: smoothing weight eps_d of the stage (Alg. 1); 1: fixed weight       */
                            /*    H_min / gamma_f^p in every stage (the fixed-smoothing ablation)     */
    int32_t projector;      /* 0: PNCG (Alg. 2); 1: Sinkhorn (Alg. 4) as the projection of each      */
                            /*    stage (MDOT-Sinkhorn; not in mdot_solve_batch or the server)        */
    int32_t stop_entropy;   /* entropy in eps_d = H / gamma^p (Alg. 1): 0: H = H_min(r, c); 1: H = log n, */
                            /*    the weaker bound App. C compares against (mdot_solve and             */
                            /*    mdot_solve_points only)                                               */
    int32_t precond;        /* 0: Sinkhorn direction s (Eq. (17)); 1: diagonal-Hessian direction       */
                            /*    (r~ / r(P), c~ / c(P)) - 1 (Eq. (16)) at iterations where every ratio  */
                            /*    lies in [0.01, 100], else s (mdot_solve and mdot_solve_points only)   */
    int32_t ls_init;        /* first trial step of each line search (App. B leaves it open):           */
                            /*    0: 1; 1 (default): the step accepted by the previous line search of  */
                            /*    the stage, clamped to [1/2, 2] (1 at a stage's first iteration)      */
    int32_t wait_limit_us;  /* limit of every bounded device-side wait (a CTA waiting for another CTA's
                               flag, a grid barrier), in microseconds; <= 0: 2 seconds.  A wait that
                               runs out ends the call with MDOT_ERR_TIMEOUT (outputs hold the last
                               iterate) and leaves the handle usable                                */
    int32_t tensor_cores;   /* 1: the regenerated squared-Euclidean cost of integer points
                               (|coordinate| <= 255, e.g. grid data) on the tensor cores, exact (see
                               mdot_cost_matrix); 0 (default): fp32 operations, measured faster on
                               GB300 because the pass is bound by the exponentials and sums      */
    int32_t polish_iters;   /* batched form and server only: fp64-entry PNCG iterations at most that
                               finish a problem's last stage on its own SM when its fp32 part
                               stalled above the stage's tolerance (an fp64 evaluation on one SM
                               costs ~5 ns per entry); mdot_solve_batch then finishes what is
                               left on every SM; 64; 0: neither                                   */
    int32_t reserved;
} mdot_params;

/* Diagnostics of one solve. */
typedef struct mdot_info {
    int32_t status;         /* mdot_status of the solve                                          */
    int32_t stages;         /* MDOT outer iterations run                                         */
    int64_t evals;          /* dual evaluations (one pass over C each), all stages               */
    int64_t evals_fp64;     /* of which with fp64 entries                                        */
    int64_t iters;          /* PNCG iterations, all stages                                       */
    int64_t ls_trials;      /* line-search phi' evaluations                                      */
    double  grad_l1;        /* ||grad g(gamma_f, r~, c~)||_1 at exit                             */
    double  gamma_f;        /* final inverse temperature used                                    */
    double  H_min;          /* min(H(r), H(c))                                                   */
    double  cost;           /* <G, C> of the rounded plan G                                      */
    double  lower_bound;    /* c-transform lower bound on the OT value                           */
    double  gap_cert;       /* cost - lower_bound >= true optimality gap                          */
    double  t_stage_fp32_ms;/* with profile: summed device time of the fp32-entry stage launches    */
    double  t_stage_fp64_ms;/* with profile: summed device time of the fp64-entry stage launches    */
    double  t_round_ms;     /* with profile: device time of the rounding launch                    */
    double  t_bound_ms;     /* with profile: device time of the lower-bound launch                 */
    int32_t launches;       /* kernel launches made by the call                                    */
    int32_t stage_launches_fp32; /* stage launches with fp32 entries                               */
    int32_t stalls;         /* stages ended because ||grad g||_1 stopped improving (no 1 % gain in
                               40 accepted iterations: tolerance below the arithmetic's floor)   */
    int32_t tensor_cores;   /* 1: the regenerated squared-Euclidean cost of integer points ran on the
                               tensor cores (see mdot_cost_matrix); 0 otherwise                   */
} mdot_info;

typedef struct mdot_handle mdot_handle;

/* Fill *prm with the defaults listed above (Sec. 5.2 values where the paper gives them). */
void mdot_default_params(mdot_params* prm);

/* Human-readable name of a status code (static storage). */
const char* mdot_status_string(int32_t status);

/* Message of the last CUDA error seen by this thread's calls, or "" (static thread storage). */
const char* mdot_last_error(void);

/*
 * Create a handle for problems of size up to max_n on the current CUDA device.
 * stream: a cudaStream_t (may be NULL for the legacy default stream), borrowed, not owned.
 * Allocates O(max_n) workspace plus column partials of (SM count) x max_n floats.
 * Errors: INVALID_ARG (h null, max_n < 1), OOM, CUDA.
 */
mdot_status mdot_create(mdot_handle** h, int64_t max_n, void* stream);

/* Free the handle and its workspace.  NULL is accepted. */
mdot_status mdot_destroy(mdot_handle* h);

/*
 * One dual evaluation (the two reductions of Alg. 2): one pass over C giving both log-marginals of
 * P(u, v; gamma) and, optionally, the dual objective of Eq. (4):
 *   log_rP[i] = u_i + LSE_j(v_j - gamma C_ij),   log_cP[j] = v_j + LSE_i(u_i - gamma C_ij),
 *   g(u, v; gamma, r, c) = sum_ij P_ij - <u, r> - <v, c> = sum_i r(P)_i - <u, r> - <v, c>.
 * The gradient of g is (r(P) - r, c(P) - c) (Sec. 2.1).
 * u, v: n doubles each.  C: n x n float32, row-major.  gamma > 0.
 * ref_log_rP (nullable, n doubles): an estimate of log_rP, used only to scale the row sums;
 *   when NULL an extra max pass over C computes the scales (so the call reads C twice).
 * precision: MDOT_PREC_FP32, MDOT_PREC_FP32A or MDOT_PREC_FP64 (AUTO means FP32).
 * Outputs log_rP, log_cP (device, n doubles each).  Entries of P more than 2^120 below the largest
 * row scale are flushed from the column sums.
 * g_out (HOST pointer, nullable): receives g, summed in fp64 in a fixed order inside the same
 *   launch (one more grid barrier); r, c (device, n doubles each) are then required, else they may
 *   be NULL.  INVALID_ARG if g_out is given without r or c.
 */
mdot_status mdot_dual_eval(mdot_handle* h, const double* u, const double* v, double gamma,
                           const float* C, int64_t n, const double* ref_log_rP,
                           int32_t precision, double* log_rP, double* log_cP,
                           const double* r, const double* c, double* g_out);

/*
 * Alg. 3 applied to P = exp(u 1^T + 1 v^T - gamma C) (the final plan of Alg. 1): the rounded plan
 * G = X P Y + err_r err_c^T / ||err_r||_1 lies in U(r, c).  Returns <G, C> in *cost_out (host)
 * without forming G; if G_out is non-null (device, n*n doubles, row-major) G is also written.
 * r, c: n doubles each, the ORIGINAL marginals (non-negative, each summing to 1).
 */
mdot_status mdot_round(mdot_handle* h, const double* u, const double* v, double gamma,
                       const float* C, const double* r, const double* c, int64_t n,
                       double* cost_out, double* G_out);

/*
 * Lower bound on the OT value from the potential u at inverse temperature gamma
 * (f = u / gamma): g'_j = min_i (C_ij - f_i), f'_i = min_j (C_ij - g'_j),
 * *lb_out (host) = <f', r> + <g', c>  <=  min_{P in U(r,c)} <P, C>  (weak LP duality).
 */
mdot_status mdot_lower_bound(mdot_handle* h, const double* u, double gamma, const float* C,
                             const double* r, const double* c, int64_t n, double* lb_out);

/*
 * MDOT-PNCG (Alg. 1 with Alg. 2 as the projector) followed by rounding (Alg. 3) and the lower
 * bound above.
 * r, c: n doubles each, non-negative, each summing to 1 within 1e-9 (Sec. 2: r, c in Delta_n).
 * C: n x n float32 row-major in [0, 1].
 * eps_target > 0: target optimality gap; used (when prm->gamma_f <= 0) to set
 *   gamma_f = (5 H_min / (2 eps_target))^(1/p) rounded up onto gamma_i q^k (Prop. 2).
 * prm: NULL for defaults.
 * Outputs: u_out, v_out (device, n doubles each; the last MDOT iterate at gamma_f, log scale),
 *   *cost_out = <G, C> of the rounded plan, *gap_out = certified gap (cost - lower bound),
 *   *info (nullable) diagnostics.  Host pointers for the three scalars/structs.
 */
mdot_status mdot_solve(mdot_handle* h, const double* r, const double* c, const float* C,
                       int64_t n, double eps_target, const mdot_params* prm,
                       double* u_out, double* v_out, double* cost_out, double* gap_out,
                       mdot_info* info);

/*
 * mdot_solve with the cost regenerated from coordinates (see mdot_cost_kind): x, y are device
 * arrays of n x 3 floats; no n x n buffer is read or written (memory O(n)).  Other arguments,
 * outputs and errors as mdot_solve; INVALID_ARG also for an unknown kind or scale <= 0.
 */
mdot_status mdot_solve_points(mdot_handle* h, const double* r, const double* c, const float* x,
                              const float* y, int32_t cost_kind, float scale, int64_t n,
                              double eps_target, const mdot_params* prm, double* u_out,
                              double* v_out, double* cost_out, double* gap_out, mdot_info* info);

/*
 * mdot_dual_eval with the cost regenerated from coordinates (see mdot_cost_kind); same outputs,
 * including the optional dual objective.
 */
mdot_status mdot_dual_eval_points(mdot_handle* h, const double* u, const double* v, double gamma,
                                  const float* x, const float* y, int32_t cost_kind, float scale,
                                  int64_t n, const double* ref_log_rP, int32_t precision,
                                  double* log_rP, double* log_cP,
                                  const double* r, const double* c, double* g_out);

/* One kernel launch of a profiled solve (mdot_params.profile != 0), in launch order. */
typedef struct mdot_trace_row {
    int32_t kind;       /* 0: stage with fp32 entries, 1: stage with fp64 entries, 2: rounding, 3: bound */
    int32_t reserved;
    double  ms;         /* device time of the launch (CUDA events around it on the handle's stream)    */
    int64_t evals;      /* dual evaluations the launch made (from the device state's counter)          */
} mdot_trace_row;

/*
 * Per-launch rows of the last solve on h that ran with mdot_params.profile != 0 (up to 512
 * launches): rows (host, max_rows entries) receives the first max_rows rows, *count (host) the
 * number recorded.  MDOT_NOT_READY if no profiled solve has completed on h; INVALID_ARG for NULL
 * arguments.  Diagnostic only (the paper has no counterpart): it ties a profiler's per-launch
 * figures to evaluation counts.
 */
mdot_status mdot_solve_trace(const mdot_handle* h, int32_t max_rows, mdot_trace_row* rows, int32_t* count);

/*
 * Phase timers of the fp32-entry stage kernel with dense C (diagnostic; the paper has no
 * counterpart): per CTA, the SM cycles spent in each phase of an evaluation, summed over every
 * launch since the last clear -- 0 loop top, 1 pass over C, 2 row epilogue, 3 wait for the column
 * partials, 4 merge and column epilogue, 5 CTA reduction and publication, 6 wait for the scalar
 * partials, 7 decision, 8 commit and next row constants -- then the evaluation count (10 counts per
 * CTA).  out (host): max_ctas x 10 counts; clear != 0 zeroes the counters after reading.  Only a
 * library built with -DMDOT_PHASE_TIMERS (paper_2307_08507_gb300/build.py --phases) keeps the
 * counters; any other build returns MDOT_NOT_READY.  INVALID_ARG for a null out or max_ctas < 1.
 */
mdot_status mdot_phase_timers(uint64_t* out, int32_t max_ctas, int32_t clear);

/*
 * The regenerated cost matrix written out: C_out (device, n x n float32, row-major) receives
 * C_ij for the coordinates x, y (device, n x 3 float32 each) with the arithmetic the solver's passes
 * use -- for MDOT_COST_SQEUCLID with every coordinate an integer of magnitude <= 255 (grid data),
 * the contraction |x_i|^2 + |y_j|^2 - 2 <x_i, y_j> on the tensor cores (bf16 inputs, fp32
 * accumulation, exact for such points) times scale; otherwise the fp32 operations in the order of
 * mdot_cost_kind.  Both forms give the same bits for grid data.  stream: a cudaStream_t or NULL;
 * the call synchronises it.  INVALID_ARG for bad sizes, kinds or scale; CUDA on a failed launch.
 */
mdot_status mdot_cost_matrix(const float* x, const float* y, int32_t cost_kind, float scale, int64_t n,
                             float* C_out, void* stream);

/*
 * Device time, in milliseconds, of the evaluation kernel launched by the last successful
 * mdot_dual_eval / mdot_dual_eval_points call on h (CUDA events recorded on the handle's stream
 * immediately around that launch; the copies of the results are outside it).  ms_out: host.
 * MDOT_NOT_READY if no evaluation has completed on h yet (or the last one failed);
 * INVALID_ARG for NULL arguments.
 */
mdot_status mdot_dual_eval_time(const mdot_handle* h, double* ms_out);

/* One problem of a batch.  Device pointers; either C (dense n x n fp32) or x, y (n x 3 fp32,
 * regenerated cost of kind cost_kind with the given scale). */
typedef struct mdot_problem {
    int64_t n;                /* 1 .. MDOT_BATCH_MAX_N                                           */
    const double* r;          /* n, non-negative, sums to 1                                      */
    const double* c;          /* n, non-negative, sums to 1                                      */
    const float* C;           /* dense cost or NULL                                              */
    const float* x;           /* coordinates (when C is NULL)                                    */
    const float* y;
    int32_t cost_kind;        /* mdot_cost_kind (when C is NULL)                                 */
    float scale;              /* cost scale (when C is NULL)                                     */
    double eps_target;        /* target gap (gamma_f from Prop. 2), used when gamma_f <= 0       */
    double gamma_f;           /* > 0: final inverse temperature                                  */
    double* u_out;            /* n or NULL: final potentials (log scale)                         */
    double* v_out;            /* n or NULL                                                       */
} mdot_problem;

/* Result of one problem of a batch. */
typedef struct mdot_result {
    int32_t status;           /* mdot_status of this problem                                     */
    int32_t stages;
    int64_t evals;            /* dual evaluations                                                */
    int64_t iters;            /* PNCG iterations                                                 */
    double  cost;             /* <G, C> of the rounded plan                                      */
    double  lower_bound;      /* c-transform bound (fp64, as mdot_lower_bound)                    */
    double  gap_cert;         /* cost - lower_bound                                              */
    double  grad_l1;          /* final ||grad g||_1                                              */
    double  gamma_f;
    double  H_min;
} mdot_result;

/* Largest n of a batched problem. */
#define MDOT_BATCH_MAX_N 8192

/*
 * Solve nprob independent problems (host array probs, each with device data) in one persistent
 * launch per cost form and tile variant (see mdot_batch_tuning; by default one variant): every CTA
 * takes the next problem from a work queue (largest n first) and
 * runs the whole of Alg. 1 + Alg. 3 on it (PNCG projections, line search, rounding, bound) with
 * block-level synchronisation.  Each problem gets its own gamma schedule (from its eps_target or
 * gamma_f), potentials and line-search state; a problem's result does not depend on the rest of
 * the batch (fixed-order reductions).  Entries use the fp32 tiers, and every stage's tolerance,
 * the last one's included, is floored at fp32_floor: unlike mdot_solve, which polishes the last
 * stage below fp32_floor in fp64 entries on every SM, one CTA per problem cannot afford that on
 * ill-conditioned problems (thousands of fp64 iterations); a caller who needs a tighter last
 * stage lowers fp32_floor.  With precision AUTO a last stage whose fp32 part ended by the stall
 * rule above its tolerance continues in fp64 entries on its SM for at most polish_iters
 * iterations; a problem still above it after the launch is finished by the single-problem
 * solver's fp64 stage on every SM (from its potentials; for problems that asked for none the
 * handle keeps them in scratch it allocates, 16 bytes per column; problems larger than the
 * handle's max_n are not finished) and reports MDOT_ERR_NOT_CONVERGED only if that stage
 * cannot reach the tolerance either.  polish_iters = 0 turns both off.  results: host array of
 * nprob.  prm: NULL for defaults.  Workspace (about 1.4 MiB per
 * SM) is allocated on the first call and kept by the handle.
 * Returns INVALID_ARG if any problem is malformed (nothing is solved), else MDOT_OK; per-problem
 * outcomes are in results[k].status.
 */
mdot_status mdot_solve_batch(mdot_handle* h, int32_t nprob, const mdot_problem* probs,
                             const mdot_params* prm, mdot_result* results);

/* Tile variants of the batched form, one per problem-size bucket (n < 512, < 1024, < 2048, < 4096,
 * <= MDOT_BATCH_MAX_N): 0 ("wide") 256 threads per problem, one problem per SM; 1 ("narrow") 128
 * threads per problem, two problems per SM.  The problems of each variant form one persistent
 * launch (wide first).  A new handle uses 0 for every bucket. */
typedef struct mdot_batch_tuning {
    int32_t variant[5];
    int32_t narrow_below;   /* mdot_tune_batch's pick: buckets below this index narrow, the rest wide */
    double  seconds[6];     /* mdot_tune_batch: device time of the timing batch under table k = 0..5
                               (buckets below k narrow); 0 where not timed */
} mdot_batch_tuning;

/*
 * The tile autotuner of the batched form.  It times the batch itself -- up to `sample` problems of
 * probs (host array, device data), evenly spaced in size order, solved to gamma_f = min(their
 * gamma_f, 2^12) without writing potentials, CUDA events around the launches -- under each table
 * of the form "buckets below k narrow, the others wide" (k = 0 ... 5; k = 0 is the default table),
 * and keeps the fastest in the handle for later mdot_solve_batch calls (on a tie the smaller k).
 * The measure is the batch's total device time, so it weighs what decides it: how the problems
 * pack onto the SMs, and the longest problems at the end of each launch.  *out (host) receives
 * the table and the time of every candidate.  Errors as mdot_solve_batch.
 */
mdot_status mdot_tune_batch(mdot_handle* h, int32_t nprob, const mdot_problem* probs, const mdot_params* prm,
                            int32_t sample, mdot_batch_tuning* out);

/* Install a stored tuning table (e.g. from an earlier mdot_tune_batch) in the handle: t (host) is
 * copied; only t->variant is used.  INVALID_ARG for NULL arguments or a variant outside 0 .. 1 (the
 * handle's table is then unchanged). */
mdot_status mdot_set_batch_tuning(mdot_handle* h, const mdot_batch_tuning* t);

/*
 * Serving: a request loop with continuous batching (the paper has no counterpart).  mdot_server_create starts a background worker on the current device with a
 * workspace pool of workspace_bytes (the HBM budget): a request of size n needs
 * 180 * ceil32(n) bytes of it (ceil32: n rounded up to a multiple of 32).  Requests are admitted in arrival order as soon as their workspace
 * fits; each admission round is one persistent batched launch (the solver of mdot_solve_batch,
 * one CTA per problem) on one of several streams, so work admitted while other launches run
 * overlaps with them on the device, and a problem's workspace returns to the pool as soon as that
 * problem finishes.  Requests above cfg->big_n instead go to "big lanes": cooperative solves (the
 * single-problem solver) on cfg->lane_ctas SMs each; the remaining SMs serve the batched route.  Results do not depend on what else runs (fixed-order reductions): a problem
 * gives the same result alone and in any mix.
 *   prm: NULL for defaults (entry tiers as mdot_solve_batch).  cfg: NULL for the default routing;
 *   lanes x lane_ctas must leave SMs for the batched route.
 *   submit: non-blocking; validates the problem (same rules as mdot_solve_batch, n up to
 *     MDOT_BATCH_MAX_N) and returns a ticket.  The problem's arrays (r, c, C or x/y, u_out,
 *     v_out) are used in place and must stay valid until poll/wait returns MDOT_OK for it.
 *     INVALID_ARG if malformed or larger than the whole pool; MDOT_ERR_CUDA after a device failure.
 *   poll: MDOT_OK and *out filled once the problem is solved (the ticket is then released),
 *     MDOT_NOT_READY before, INVALID_ARG for an unknown ticket.
 *   wait: poll that blocks up to timeout_s seconds.
 *   destroy: finishes every queued and admitted request, then frees everything.
 */
typedef struct mdot_server mdot_server;

/* Routing of the server (NULL in mdot_server_create: the defaults below). */
typedef struct mdot_server_config {
    int64_t big_n;            /* requests with n > big_n go to a big lane (default 2048)           */
    int32_t big_lanes;        /* concurrent cooperative solves (default 3; 0: every request batched) */
    int32_t lane_ctas;        /* CTAs (SMs) of each big lane (default: 29 % of the SMs, 44 of 152)  */
} mdot_server_config;

mdot_status mdot_server_create(mdot_server** s, uint64_t workspace_bytes, const mdot_params* prm,
                               const mdot_server_config* cfg);
mdot_status mdot_server_submit(mdot_server* s, const mdot_problem* prob, uint64_t* ticket);
mdot_status mdot_server_poll(mdot_server* s, uint64_t ticket, mdot_result* out);
mdot_status mdot_server_wait(mdot_server* s, uint64_t ticket, double timeout_s, mdot_result* out);
mdot_status mdot_server_destroy(mdot_server* s);

/*
 * mdot_solve with every array in HOST memory: copies r, c (n doubles) and C (n*n floats) to the
 * handle's device, solves, and copies u, v back (n doubles each).  The copies are part of the
 * call.  Use for callers without device buffers; same errors as mdot_solve.
 */
mdot_status mdot_solve_host(mdot_handle* h, const double* r_host, const double* c_host,
                            const float* C_host, int64_t n, double eps_target,
                            const mdot_params* prm, double* u_host, double* v_host,
                            double* cost_out, double* gap_out, mdot_info* info);


/*
 * Read-rate probe (a measurement utility; the paper has no counterpart): reads the n_floats
 * floats at buf (device, 16-byte aligned, n_floats a multiple of 4) reps times with 128-bit
 * loads on 4 CTAs per SM and adds a checksum into *out (device, cleared by the call).  The
 * caller times it with CUDA events on `stream` (a cudaStream_t or NULL); the call does not
 * synchronise.  A buffer that fits in L2 is read from L2 after the first pass, so
 * reps x n_floats x 4 bytes / time is the L2 read rate; a buffer far larger than L2 gives the HBM
 * read rate.  INVALID_ARG for a bad size, alignment or reps < 1; CUDA if the launch fails.
 */
mdot_status mdot_read_probe(const float* buf, int64_t n_floats, int32_t reps, float* out, void* stream);

/* ------------------------------------------------------------------------------------------ */
/* Dual evaluation without any allocation.                                                     */
/* ------------------------------------------------------------------------------------------ */

/* Largest n accepted by mdot_dual_eval_noalloc. */
#define MDOT_NOALLOC_MAX_N 4096

/*
 * mdot_dual_eval without a handle and without allocating device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc, e.g. plugins
 * whose host framework owns every device allocation, or pipelines that must not allocate once
 * they are running.  Its scratch (column partials, per-row/column constants, the grid barrier)
 * is a fixed static device array of about 2.6 MiB, compiled into the library: every GPU on which
 * the library is loaded holds it until the process exits.
 *
 * Semantics are those of mdot_dual_eval with precision MDOT_PREC_FP32; outputs are written
 * straight into log_rP and log_cP (device, n doubles each).  n must not exceed
 * MDOT_NOALLOC_MAX_N (larger n returns MDOT_ERR_INVALID_ARG).  stream: a cudaStream_t or NULL.
 * The call calls no cudaMalloc/cudaFree; it synchronises `stream` before returning.
 *
 * Set-up: the first call on a device looks up the device address of the static scratch with
 * cudaGetSymbolAddress (with that device current); make that first call before any stream
 * capture.  All calls share the one scratch array and leave it holding their values; the call
 * clears what must start at zero.  Calls that overlap on the GPU (other streams, other host
 * threads) race on the scratch: serialise them.
 */
mdot_status mdot_dual_eval_noalloc(const double* u, const double* v, double gamma, const float* C,
                                   int64_t n, const double* ref_log_rP, double* log_rP,
                                   double* log_cP, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MDOT_H */
