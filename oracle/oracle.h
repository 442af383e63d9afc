/*
 * CPU FP64 oracle for MDOT-PNCG (Kemertas, Jepson, Farahmand, arXiv 2307.08507).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU baseline
 * may load this library.  It shares no code, header, table or constant with the CUDA library;
 * the two agree only because both follow the paper.
 *
 * Everything is plain double precision, round-to-nearest, with libm exp/log, written for a reader
 * to check against the paper by eye: no blocking, no fusion, no reordering beyond what the
 * paper's formulas state.  Cost matrices are dense, row-major, n x n doubles (a float32 cost is
 * passed promoted to double so both sides solve the identical problem).
 *
 * Convention (the paper's): P_ij(u, v; gamma) = exp(u_i + v_j - gamma C_ij), Eq. (2);
 * gamma is the inverse temperature and grows from gamma_i to gamma_f.
 *
 * Parity status: every routine here is pinned by a CPU test (closed forms, brute-force or LP
 * optima, finite differences, invariants); none is "parity unpinned".
 */
#ifndef MDOT_ORACLE_H
#define MDOT_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double gamma_i;        /* first inverse temperature (Alg. 1 input), paper default 2^4          */
    double gamma_f;        /* final inverse temperature (Alg. 1 input)                             */
    double p;              /* stopping-rule exponent, eps_d = H_min / gamma^p (Alg. 1)             */
    double q;              /* temperature decay factor, gamma <- min(q gamma, gamma_f)             */
    double ls_c1, ls_c2;   /* approximate Wolfe constants, 0 < c1 < c2 < 1 (App. B, Eq. (24))      */
    int    ls_max_trials;  /* cap on phi' evaluations per line search                              */
    int    max_iter;       /* cap on PNCG iterations (or Sinkhorn iterations) per projection        */
    int    projector;      /* 0 = PNCG (Alg. 2), 1 = Sinkhorn (Alg. 4)                             */
    int    warm_start;     /* 0 = finite-difference Taylor step (Eq. (13)), 1 = eps-scaling, 2 = none */
    int    precond;        /* 0 = Sinkhorn direction s (Eq. (17)), 1 = diagonal Hessian (Eq. (16)) with fallback */
    int    smoothing;      /* 0 = variable weight eps_d/4 (Alg. 1), 1 = fixed weight at gamma_f */
    double final_tol;      /* if > 0: tolerance used at the final stage instead of eps_d/2         */
    int    stop_entropy;   /* entropy in eps_d (Alg. 1): 0 = H_min(r, c), 1 = log n (App. C ablation) */
    int    ls_init;        /* first trial of each line search (App. B leaves it open): 0 = 1;      */
                           /* 1 = the previous accepted step of the stage clamped to [1/2, 2]      */
} or_params;

typedef struct {
    int    stages;         /* MDOT outer iterations                                */
    long   evals;          /* full dual evaluations (row + column LSE) -- PNCG      */
    long   half_evals;     /* single LSE reductions (row or column) -- Sinkhorn     */
    long   iters;          /* PNCG or Sinkhorn iterations                           */
    long   ls_trials;      /* line-search phi' evaluations                          */
    int    status;         /* 0 ok, 1 iteration cap hit somewhere, 2 line search failed, 3 non-finite */
    double grad_l1;        /* ||grad g(gamma_f, r~, c~)||_1 at exit                 */
    double gamma_last;     /* gamma of the last stage solved                        */
    double grad_l1_init;   /* ||grad g||_1 at the first evaluation of the last projection */
} or_stats;

void   or_default_params(or_params* prm);

/* H(r) = -<r, log r>, with 0 log 0 = 0 (Sec. 2, notation). */
double or_entropy(int n, const double* r);

/* Alg. 2 (the two reductions): log r(P) = u + LSE_r(1 v^T - gamma C), log c(P) = v + LSE_c(u 1^T - gamma C),
 * each log-sum-exp stabilised by its own row / column maximum. */
void   or_dual_eval(int n, const double* C, const double* u, const double* v, double gamma,
                    double* log_rP, double* log_cP);

/* Eq. (4): g(u, v; gamma, r, c) = sum_ij P_ij - <u, r> - <v, c>. */
double or_dual_value(int n, const double* C, const double* u, const double* v, double gamma,
                     const double* r, const double* c);

/* The App. B line search on a scalar function phi (approximate Wolfe test Eq. (24), doubling
 * until bracketed, hybrid secant/bisection step Eq. (25) inside the bracket).  dphi(ctx, alpha)
 * returns phi'(alpha) (non-finite: an overshoot); keep_lo(ctx) (nullable) is called whenever the
 * trial just evaluated becomes the lower end of the bracket.  d0 = phi'(0) < 0, a0 = first trial.
 * Returns 0 with the accepted step (the last trial) in *alpha_out, 1 when the trial cap took the
 * lower end (*alpha_out = lo), 2 when no step was found. */
typedef double (*or_dphi_fn)(void* ctx, double alpha);
typedef void (*or_keep_fn)(void* ctx);
int    or_ls_search(double d0, double a0, const or_params* prm, or_dphi_fn dphi, or_keep_fn keep_lo,
                    void* ctx, double* alpha_out);

/* One PNCG projection (Alg. 2) with the App. B line search; u, v updated in place.
 * tol is the threshold on ||grad g||_1.  log_rP / log_cP (n each) receive the final marginals. */
int    or_pncg(int n, const double* C, double gamma, const double* r, const double* c, double tol,
               double* u, double* v, const or_params* prm, or_stats* st, double* log_rP, double* log_cP);

/* One Sinkhorn projection (Alg. 4); u, v updated in place; stops on the row residual. */
int    or_sinkhorn(int n, const double* C, double gamma, const double* r, const double* c, double tol,
                   double* u, double* v, const or_params* prm, or_stats* st, double* log_rP);

/* MDOT (Alg. 1) up to (not including) rounding.  u, v (n each) receive the last iterate.
 * stage_log (nullable, 6 doubles per stage: gamma, eps_d, evals so far, iters so far, final
 * grad_l1, grad_l1 at the stage's first evaluation) holds at most max_log stages. */
int    or_mdot(int n, const double* C, const double* r, const double* c, const or_params* prm,
               double* u, double* v, or_stats* st, double* stage_log, int max_log);

/* Alg. 3 (rounding onto U(r, c)) applied to P = exp(u 1^T + 1 v^T - gamma C) (the final plan of Alg. 1).
 * G (nullable, n*n) receives the rounded plan; returns <G, C>. */
double or_round(int n, const double* C, const double* u, const double* v, double gamma,
                const double* r, const double* c, double* G);

/* Lower bound on the OT cost from the potentials f = u/gamma: g'_j = min_i (C_ij - f_i), then
 * f'_i = min_j (C_ij - g'_j); returns <f', r> + <g', c> (feasible dual, weak duality). */
double or_ctransform_lb(int n, const double* C, const double* u, double gamma,
                        const double* r, const double* c);

/* gamma_f from a target gap via the Prop. 2 relation gamma_f = (5 H_min / (2 eps))^(1/p),
 * rounded up onto the schedule gamma_i q^k. */
double or_gamma_f_for_eps(double H_min, double eps, double gamma_i, double q, double p);

#ifdef __cplusplus
}
#endif
#endif
