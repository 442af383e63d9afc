/*
 * CPU FP64 oracle for MDOT-PNCG -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Written from the paper (arXiv 2307.08507): Eq. (2)-(4) (closed-form plan, dual, gradient),
 * Alg. 1 (MDOT), Eq. (13) (warm start), Alg. 2 (PNCG), Eq. (17)/(18) (Sinkhorn direction and the
 * preconditioned Hestenes-Stiefel beta), App. B (approximate-Wolfe hybrid bisection/secant line
 * search), Alg. 3 (rounding, after Altschuler et al.) and Alg. 4 (log-domain Sinkhorn).
 * Readings where the paper is silent are marked "reading:" and listed in the design notes.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j) ((size_t)(i) * (size_t)n + (size_t)(j))

void or_default_params(or_params* prm)
{
    /* Sec. 5.2: gamma_i = 2^4, q = 2^(1/3), p = 1.5.  App. B gives only 0 < c1 < c2 < 1;
     * reading: c1 = 0.1 (Hager-Zhang's delta) and c2 = 0.5, which keeps 1.5-2.5 phi'
     * evaluations per iteration (App. B) with fewer iterations than c2 = 0.9; 50-trial cap. */
    prm->gamma_i = 16.0;
    prm->gamma_f = 65536.0;
    prm->p = 1.5;
    prm->q = cbrt(2.0);
    prm->ls_c1 = 0.1;
    prm->ls_c2 = 0.5;
    prm->ls_max_trials = 50;
    prm->max_iter = 100000;
    prm->projector = 0;
    prm->warm_start = 0;
    prm->precond = 0;
    prm->smoothing = 0;
    prm->final_tol = 0.0;
    prm->stop_entropy = 0;
    /* reading: App. B fixes no first trial step; the previous accepted step (clamped to [1/2, 2])
     * needs 17-43 % fewer evaluations than 1 on grid problems (measured with this oracle) */
    prm->ls_init = 1;
}

double or_entropy(int n, const double* r)
{
    double h = 0.0;
    for (int i = 0; i < n; ++i)
        if (r[i] > 0.0) h -= r[i] * log(r[i]);
    return h;
}

/* LSE_r(1 v^T - gamma C)_i = log sum_j exp(v_j - gamma C_ij), stabilised by the row max.
 * (Rows are independent; a build with OpenMP, used only to time the CPU baseline on every host
 * core, splits them over threads without changing any row's arithmetic.) */
static void lse_rows(int n, const double* C, const double* v, double gamma, double* out)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double m = -INFINITY;
        for (int j = 0; j < n; ++j) {
            double z = v[j] - gamma * C[IDX(i, j)];
            if (z > m) m = z;
        }
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += exp(v[j] - gamma * C[IDX(i, j)] - m);
        out[i] = m + log(s);
    }
}

/* LSE_c(u 1^T - gamma C)_j = log sum_i exp(u_i - gamma C_ij), stabilised by the column max.
 * The loops run over i outside only so that C is read row by row (in strips of columns, which a
 * build with OpenMP hands to different threads); the arithmetic per column is the same
 * max-then-sum over i = 0 .. n-1 as above. */
static void lse_cols(int n, const double* C, const double* u, double gamma, double* out)
{
    enum { STRIP = 512 };
    double* m = (double*)malloc(sizeof(double) * (size_t)n);
    double* s = (double*)malloc(sizeof(double) * (size_t)n);
    const int nstrip = (n + STRIP - 1) / STRIP;
#pragma omp parallel for schedule(static)
    for (int b = 0; b < nstrip; ++b) {
        const int j0 = b * STRIP, j1 = (j0 + STRIP < n) ? j0 + STRIP : n;
        for (int j = j0; j < j1; ++j) { m[j] = -INFINITY; s[j] = 0.0; }
        for (int i = 0; i < n; ++i)
            for (int j = j0; j < j1; ++j) {
                double z = u[i] - gamma * C[IDX(i, j)];
                if (z > m[j]) m[j] = z;
            }
        for (int i = 0; i < n; ++i)
            for (int j = j0; j < j1; ++j) s[j] += exp(u[i] - gamma * C[IDX(i, j)] - m[j]);
        for (int j = j0; j < j1; ++j) out[j] = m[j] + log(s[j]);
    }
    free(m);
    free(s);
}

void or_dual_eval(int n, const double* C, const double* u, const double* v, double gamma,
                  double* log_rP, double* log_cP)
{
    /* Alg. 2, row reduction: log r(P) = u + LSE_r(1 v^T - gamma C) */
    lse_rows(n, C, v, gamma, log_rP);
    for (int i = 0; i < n; ++i) log_rP[i] += u[i];
    /* Alg. 2, column reduction: log c(P) = v + LSE_c(u 1^T - gamma C) */
    lse_cols(n, C, u, gamma, log_cP);
    for (int j = 0; j < n; ++j) log_cP[j] += v[j];
}

double or_dual_value(int n, const double* C, const double* u, const double* v, double gamma,
                     const double* r, const double* c)
{
    /* Eq. (4): g = sum_ij exp(u_i + v_j - gamma C_ij) - <u, r> - <v, c> */
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) s += exp(u[i] + v[j] - gamma * C[IDX(i, j)]);
    for (int i = 0; i < n; ++i) s -= u[i] * r[i];
    for (int j = 0; j < n; ++j) s -= v[j] * c[j];
    return s;
}

static double l1_grad(int n, const double* log_rP, const double* log_cP, const double* r, const double* c)
{
    /* ||grad g||_1 with grad g = (r(P) - r, c(P) - c), Eq. (4) */
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += fabs(exp(log_rP[i]) - r[i]);
    for (int j = 0; j < n; ++j) s += fabs(exp(log_cP[j]) - c[j]);
    return s;
}

/* phi'(alpha) = <p_u, r(P_alpha) - r> + <p_v, c(P_alpha) - c>, App. B Eq. (26) */
static double phi_prime(int n, const double* pu, const double* pv, const double* log_rP,
                        const double* log_cP, const double* r, const double* c)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += pu[i] * (exp(log_rP[i]) - r[i]);
    for (int j = 0; j < n; ++j) s += pv[j] * (exp(log_cP[j]) - c[j]);
    return s;
}

/*
 * App. B line search on a scalar function: find alpha with (2 c1 - 1) phi'(0) >= phi'(alpha) >=
 * c2 phi'(0) (approximate Wolfe, Eq. (24)).  The bracket [lo, hi] keeps phi'(lo) < 0 < phi'(hi);
 * inside a bracket the next trial is alpha_hyb = alpha_sec / 2 + (lo + hi) / 4 (Eq. (25) and the
 * text after it), alpha_sec the secant root through (lo, phi'(lo)) and (hi, phi'(hi)).
 * Readings: the first trial is a0; until an upper end is found alpha doubles; a non-finite phi'
 * counts as an upper end and the next trial bisects; after ls_max_trials the lower end is taken if
 * it is > 0.  dphi(ctx, alpha) evaluates phi'(alpha); keep_lo(ctx) is called when the trial just
 * evaluated becomes the lower end (the PNCG caller keeps its marginals).
 * Returns 0 (accepted: the last trial evaluated, *alpha_out), 1 (cap reached, lower end taken:
 * *alpha_out = lo) or 2 (no step: d0 >= 0, or the cap with lo = 0).
 */
int or_ls_search(double d0, double a0, const or_params* prm, or_dphi_fn dphi, or_keep_fn keep_lo,
                 void* ctx, double* alpha_out)
{
    const double c1 = prm->ls_c1, c2 = prm->ls_c2;
    double lo = 0.0, dlo = d0, hi = INFINITY, dhi = INFINITY;
    double a = a0;                              /* first trial step */
    if (!(d0 < 0.0)) return 2;                  /* not a descent direction */
    for (int trial = 0; trial < prm->ls_max_trials; ++trial) {
        double d = dphi(ctx, a);
        if (!isfinite(d)) {                     /* overshoot into overflow: shrink */
            hi = a;
            dhi = INFINITY;
            a = 0.5 * (lo + hi);
            continue;
        }
        if (d <= (2.0 * c1 - 1.0) * d0 && d >= c2 * d0) {   /* Eq. (24) holds */
            *alpha_out = a;
            return 0;
        }
        if (d < c2 * d0) {                      /* still descending steeply: raise lower end */
            lo = a;
            dlo = d;
            if (keep_lo) keep_lo(ctx);
        } else {                                /* overshoot: lower the upper end */
            hi = a;
            dhi = d;
        }
        if (isinf(hi)) {
            a = 2.0 * a;
        } else if (isinf(dhi)) {
            a = 0.5 * (lo + hi);
        } else {
            double a_sec = (lo * dhi - hi * dlo) / (dhi - dlo);
            a = 0.5 * a_sec + 0.5 * (0.5 * (lo + hi));
        }
    }
    if (lo > 0.0) {                             /* cap reached: take the lower end */
        *alpha_out = lo;
        return 1;
    }
    return 2;
}

/* The PNCG line search: phi'(alpha) from a full dual evaluation at (u, v) + alpha p (App. B). */
typedef struct {
    int n;
    const double *C, *r, *c, *u, *v, *pu, *pv;
    double gamma;
    double *ut, *vt, *lr, *lc, *lr_lo, *lc_lo;
    or_stats* st;
} pncg_ls_ctx;

static double pncg_dphi(void* vctx, double a)
{
    pncg_ls_ctx* x = (pncg_ls_ctx*)vctx;
    const int n = x->n;
    for (int i = 0; i < n; ++i) x->ut[i] = x->u[i] + a * x->pu[i];
    for (int j = 0; j < n; ++j) x->vt[j] = x->v[j] + a * x->pv[j];
    or_dual_eval(n, x->C, x->ut, x->vt, x->gamma, x->lr, x->lc);
    x->st->evals++;
    x->st->ls_trials++;
    return phi_prime(n, x->pu, x->pv, x->lr, x->lc, x->r, x->c);
}

static void pncg_keep_lo(void* vctx)
{
    pncg_ls_ctx* x = (pncg_ls_ctx*)vctx;
    memcpy(x->lr_lo, x->lr, sizeof(double) * (size_t)x->n);
    memcpy(x->lc_lo, x->lc, sizeof(double) * (size_t)x->n);
}

/*
 * On entry log_rP / log_cP hold the marginals at alpha = 0; on success they hold the marginals at
 * the accepted alpha (so the next PNCG iteration reuses them, App. B).  Returns as or_ls_search.
 */
static int line_search(int n, const double* C, double gamma, const double* r, const double* c,
                       const double* u, const double* v, const double* pu, const double* pv,
                       double* log_rP, double* log_cP, double a0, double* alpha_out,
                       const or_params* prm, or_stats* st)
{
    pncg_ls_ctx x;
    x.n = n; x.C = C; x.r = r; x.c = c; x.u = u; x.v = v; x.pu = pu; x.pv = pv; x.gamma = gamma;
    x.st = st;
    x.ut = (double*)malloc(sizeof(double) * (size_t)n);
    x.vt = (double*)malloc(sizeof(double) * (size_t)n);
    x.lr = (double*)malloc(sizeof(double) * (size_t)n);
    x.lc = (double*)malloc(sizeof(double) * (size_t)n);
    x.lr_lo = (double*)malloc(sizeof(double) * (size_t)n);
    x.lc_lo = (double*)malloc(sizeof(double) * (size_t)n);

    const double d0 = phi_prime(n, pu, pv, log_rP, log_cP, r, c);   /* O(n), App. B */
    int rc = or_ls_search(d0, a0, prm, pncg_dphi, pncg_keep_lo, &x, alpha_out);
    if (rc == 0) {
        memcpy(log_rP, x.lr, sizeof(double) * (size_t)n);
        memcpy(log_cP, x.lc, sizeof(double) * (size_t)n);
    } else if (rc == 1) {
        memcpy(log_rP, x.lr_lo, sizeof(double) * (size_t)n);
        memcpy(log_cP, x.lc_lo, sizeof(double) * (size_t)n);
    }
    free(x.ut); free(x.vt); free(x.lr); free(x.lc); free(x.lr_lo); free(x.lc_lo);
    return rc;
}

int or_pncg(int n, const double* C, double gamma, const double* r, const double* c, double tol,
            double* u, double* v, const or_params* prm, or_stats* st, double* log_rP, double* log_cP)
{
    const int m = 2 * n;
    double* p = (double*)calloc((size_t)m, sizeof(double));       /* p <- 0_{2n} */
    double* s = (double*)malloc(sizeof(double) * (size_t)m);
    double* gr = (double*)malloc(sizeof(double) * (size_t)m);
    double* gr_prev = (double*)malloc(sizeof(double) * (size_t)m);
    double* logr = (double*)malloc(sizeof(double) * (size_t)n);
    double* logc = (double*)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i < n; ++i) logr[i] = log(r[i]);
    for (int j = 0; j < n; ++j) logc[j] = log(c[j]);
    int status = 0;

    /* Alg. 2: marginals and gradient at the starting point */
    or_dual_eval(n, C, u, v, gamma, log_rP, log_cP);
    st->evals++;
    for (int i = 0; i < n; ++i) gr[i] = exp(log_rP[i]) - r[i];
    for (int j = 0; j < n; ++j) gr[n + j] = exp(log_cP[j]) - c[j];
    double gnorm = l1_grad(n, log_rP, log_cP, r, c);
    st->grad_l1_init = gnorm;

    int k = 0;
    double a0 = 1.0;                  /* first trial step of the next line search */
    while (gnorm > tol) {                                           /* Alg. 2: stop at ||grad g||_1 <= tol */
        if (k >= prm->max_iter) { status = 1; break; }
        ++k;
        st->iters++;
        /* Sinkhorn direction s = (log r - log r(P), log c - log c(P)), Eq. (17);
         * precond = 1: diagonal-Hessian direction (r / r(P), c / c(P)) - 1, Eq. (16), used only
         * when every ratio lies in [0.01, 100] (Sec. 4 variant), else s. */
        for (int i = 0; i < n; ++i) s[i] = logr[i] - log_rP[i];
        for (int j = 0; j < n; ++j) s[n + j] = logc[j] - log_cP[j];
        if (prm->precond == 1) {
            int ok = 1;
            for (int a = 0; a < m && ok; ++a) {
                double ratio = exp(s[a]);
                if (ratio < 0.01 || ratio > 100.0) ok = 0;
            }
            if (ok)
                for (int a = 0; a < m; ++a) s[a] = exp(s[a]) - 1.0;
        }
        /* p <- s + beta p with Eq. (18): beta_k = <g_k - g_{k-1}, -s_k> / <g_k - g_{k-1}, p_{k-1}>,
         * beta_1 = 0.  Reading: a zero or non-finite denominator gives beta = 0. */
        double beta = 0.0;
        if (k > 1) {
            double num = 0.0, den = 0.0;
            for (int a = 0; a < m; ++a) {
                double y = gr[a] - gr_prev[a];
                num += y * (-s[a]);
                den += y * p[a];
            }
            beta = (den != 0.0 && isfinite(num / den)) ? num / den : 0.0;
        }
        for (int a = 0; a < m; ++a) p[a] = s[a] + beta * p[a];
        /* reset to s if p is not a descent direction (Alg. 2) */
        double pg = 0.0;
        for (int a = 0; a < m; ++a) pg += p[a] * gr[a];
        if (pg >= 0.0)
            for (int a = 0; a < m; ++a) p[a] = s[a];
        /* line search (App. B) */
        double alpha = 0.0;
        int lrc = line_search(n, C, gamma, r, c, u, v, p, p + n, log_rP, log_cP, a0, &alpha, prm, st);
        if (lrc == 2) { status = 2; break; }
        if (lrc == 1) status = 1;
        if (prm->ls_init == 1) a0 = fmax(0.5, fmin(2.0, alpha));    /* next first trial */
        /* (u, v) <- (u, v) + alpha p */
        for (int i = 0; i < n; ++i) u[i] = u[i] + alpha * p[i];
        for (int j = 0; j < n; ++j) v[j] = v[j] + alpha * p[n + j];
        /* new gradient from the accepted trial's marginals */
        memcpy(gr_prev, gr, sizeof(double) * (size_t)m);
        for (int i = 0; i < n; ++i) gr[i] = exp(log_rP[i]) - r[i];
        for (int j = 0; j < n; ++j) gr[n + j] = exp(log_cP[j]) - c[j];
        gnorm = l1_grad(n, log_rP, log_cP, r, c);
        if (!isfinite(gnorm)) { status = 3; break; }
    }
    st->grad_l1 = gnorm;
    free(p); free(s); free(gr); free(gr_prev); free(logr); free(logc);
    return status;
}

int or_sinkhorn(int n, const double* C, double gamma, const double* r, const double* c, double tol,
                double* u, double* v, const or_params* prm, or_stats* st, double* log_rP)
{
    double* l = (double*)malloc(sizeof(double) * (size_t)n);
    int status = 0;
    /* Alg. 4: row marginal at the starting point */
    lse_rows(n, C, v, gamma, l);
    for (int i = 0; i < n; ++i) log_rP[i] = u[i] + l[i];
    st->half_evals++;
    double res = 0.0;
    for (int i = 0; i < n; ++i) res += fabs(r[i] - exp(log_rP[i]));
    st->grad_l1_init = res;
    long it = 0;
    while (res > tol) {                                             /* Alg. 4: stop on the row residual */
        if (it >= prm->max_iter) { status = 1; break; }
        ++it;
        st->iters++;
        for (int i = 0; i < n; ++i) u[i] = u[i] + log(r[i]) - log_rP[i];       /* row update */
        lse_cols(n, C, u, gamma, l);                                           /* column update */
        for (int j = 0; j < n; ++j) v[j] = log(c[j]) - l[j];
        lse_rows(n, C, v, gamma, l);                                           /* new row marginal */
        for (int i = 0; i < n; ++i) log_rP[i] = u[i] + l[i];
        st->half_evals += 2;
        res = 0.0;
        for (int i = 0; i < n; ++i) res += fabs(r[i] - exp(log_rP[i]));
        if (!isfinite(res)) { status = 3; break; }
    }
    st->grad_l1 = res;   /* the column residual is zero after the column update */
    free(l);
    return status;
}

int or_mdot(int n, const double* C, const double* r, const double* c, const or_params* prm,
            double* u, double* v, or_stats* st, double* stage_log, int max_log)
{
    /* H_min(r, c); reading: floored at 1e-12 so that a point-mass marginal (H_min = 0) still gets
     * a positive smoothing weight (Alg. 1) instead of log 0 */
    const double H = fmax(fmin(or_entropy(n, r), or_entropy(n, c)), 1e-12);
    double* rt = (double*)malloc(sizeof(double) * (size_t)n);
    double* ct = (double*)malloc(sizeof(double) * (size_t)n);
    double* u_prev = (double*)malloc(sizeof(double) * (size_t)n);
    double* v_prev = (double*)malloc(sizeof(double) * (size_t)n);
    double* lr = (double*)malloc(sizeof(double) * (size_t)n);
    double* lc = (double*)malloc(sizeof(double) * (size_t)n);
    memset(st, 0, sizeof(*st));
    int status = 0;

    double gamma = fmin(prm->gamma_i, prm->gamma_f);                /* gamma_1 = min(gamma_i, gamma_f) */
    double dgamma_prev = gamma;   /* reading: stage 0 is gamma = 0 (Prop. 1), so the first step is gamma_i */
    int t = 1;
    for (;;) {                                                      /* MDOT outer loop (Alg. 1) */
        /* stopping tolerance eps_d; App. C compares H_min with the weaker log n in its place */
        double eps_d = (prm->stop_entropy == 1 ? log((double)n) : H) / pow(gamma, prm->p);
        double w = (prm->smoothing == 1) ? H / pow(prm->gamma_f, prm->p) : eps_d;
        for (int i = 0; i < n; ++i) rt[i] = (1.0 - w / 4.0) * r[i] + w / (4.0 * n);   /* smoothing */
        for (int j = 0; j < n; ++j) ct[j] = (1.0 - w / 4.0) * c[j] + w / (4.0 * n);
        if (t == 1) {                                               /* rank-one start */
            for (int i = 0; i < n; ++i) u[i] = log(rt[i]);
            for (int j = 0; j < n; ++j) v[j] = log(ct[j]);
            /* reading: z^(0) = (log r~, log c~) is the gamma = 0 solution used by the first warm start */
            memcpy(u_prev, u, sizeof(double) * (size_t)n);
            memcpy(v_prev, v, sizeof(double) * (size_t)n);
        }
        /* projection tolerance eps_d / 2; reading: the fp64 exponent u_i + v_j - gamma C_ij cancels terms of size ~gamma,
         * so the marginals carry ~2e-16 gamma relative noise; a tolerance below
         * 1e-13 + 1e-15 gamma could never be met and is floored there (far below eps_d / 2 for
         * any gamma used in practice) */
        double tol = fmax(eps_d / 2.0, 1e-13 + 1e-15 * gamma);
        if (gamma == prm->gamma_f && prm->final_tol > 0.0) tol = prm->final_tol;
        int rc;
        if (prm->projector == 1)
            rc = or_sinkhorn(n, C, gamma, rt, ct, tol, u, v, prm, st, lr);
        else
            rc = or_pncg(n, C, gamma, rt, ct, tol, u, v, prm, st, lr, lc);
        if (rc > status) status = rc;
        st->stages = t;
        st->gamma_last = gamma;
        if (stage_log && t <= max_log) {
            double* L = stage_log + 6 * (t - 1);
            L[0] = gamma; L[1] = eps_d; L[2] = (double)st->evals + 0.5 * (double)st->half_evals;
            L[3] = (double)st->iters; L[4] = st->grad_l1; L[5] = st->grad_l1_init;
        }
        if (rc >= 2) break;
        if (gamma == prm->gamma_f) break;                           /* exit at gamma_f */
        double dgamma = (prm->q - 1.0) * gamma;                     /* gamma <- min(gamma + (q-1) gamma, gamma_f) */
        double gamma_next = fmin(gamma + dgamma, prm->gamma_f);
        dgamma = gamma_next - gamma;   /* reading: the clamped last step uses its actual size */
        /* warm start */
        if (prm->warm_start == 0) {
            /* Eq. (13): z' = z^(t) + (dgamma^(t) / dgamma^(t-1)) (z^(t) - z^(t-1)) */
            double ratio = dgamma / dgamma_prev;
            for (int i = 0; i < n; ++i) {
                double z = u[i];
                u[i] = z + ratio * (z - u_prev[i]);
                u_prev[i] = z;
            }
            for (int j = 0; j < n; ++j) {
                double z = v[j];
                v[j] = z + ratio * (z - v_prev[j]);
                v_prev[j] = z;
            }
        } else if (prm->warm_start == 1) {
            /* eps-scaling (Sec. 3.3.1): z' = (gamma^(t+1) / gamma^(t)) z^(t) */
            double ratio = gamma_next / gamma;
            for (int i = 0; i < n; ++i) u[i] *= ratio;
            for (int j = 0; j < n; ++j) v[j] *= ratio;
        }
        dgamma_prev = dgamma;
        gamma = gamma_next;
        ++t;                                                        /* next stage */
    }
    st->status = status;
    free(rt); free(ct); free(u_prev); free(v_prev); free(lr); free(lc);
    return status;
}

double or_round(int n, const double* C, const double* u, const double* v, double gamma,
                const double* r, const double* c, double* G)
{
    double* P = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double* x = (double*)malloc(sizeof(double) * (size_t)n);
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    double* rF = (double*)malloc(sizeof(double) * (size_t)n);
    double* cF = (double*)malloc(sizeof(double) * (size_t)n);
    double* er = (double*)malloc(sizeof(double) * (size_t)n);
    double* ec = (double*)malloc(sizeof(double) * (size_t)n);
    /* Alg. 1, final plan: P = exp(u 1^T + 1 v^T - gamma_f C) */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) P[IDX(i, j)] = exp(u[i] + v[j] - gamma * C[IDX(i, j)]);
    /* Alg. 3: x = r / r(P) ^ 1 (elementwise min); reading: r(P)_i = 0 gives x_i = 1 */
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += P[IDX(i, j)];
        x[i] = (s > 0.0) ? fmin(r[i] / s, 1.0) : 1.0;
    }
    /* F = X P */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) P[IDX(i, j)] *= x[i];
    /* y = c / c(F) ^ 1 */
    for (int j = 0; j < n; ++j) cF[j] = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) cF[j] += P[IDX(i, j)];
    for (int j = 0; j < n; ++j) y[j] = (cF[j] > 0.0) ? fmin(c[j] / cF[j], 1.0) : 1.0;
    /* F' = F Y */
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) P[IDX(i, j)] *= y[j];
    /* err_r = r - r(F'), err_c = c - c(F') */
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += P[IDX(i, j)];
        rF[i] = s;
        er[i] = r[i] - s;
    }
    for (int j = 0; j < n; ++j) cF[j] = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) cF[j] += P[IDX(i, j)];
    double er1 = 0.0;
    for (int i = 0; i < n; ++i) er1 += fabs(er[i]);
    for (int j = 0; j < n; ++j) ec[j] = c[j] - cF[j];
    /* G = F' + err_r err_c^T / ||err_r||_1; reading: ||err_r||_1 = 0 gives G = F' */
    double cost = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double g = P[IDX(i, j)];
            if (er1 > 0.0) g += er[i] * ec[j] / er1;
            if (G) G[IDX(i, j)] = g;
            cost += g * C[IDX(i, j)];
        }
    free(P); free(x); free(y); free(rF); free(cF); free(er); free(ec);
    return cost;
}

double or_ctransform_lb(int n, const double* C, const double* u, double gamma,
                        const double* r, const double* c)
{
    double* f = (double*)malloc(sizeof(double) * (size_t)n);
    double* g = (double*)malloc(sizeof(double) * (size_t)n);
    for (int i = 0; i < n; ++i) f[i] = u[i] / gamma;                /* cost units */
    for (int j = 0; j < n; ++j) {                                    /* g_j = min_i (C_ij - f_i) */
        double m = INFINITY;
        for (int i = 0; i < n; ++i) m = fmin(m, C[IDX(i, j)] - f[i]);
        g[j] = m;
    }
    for (int i = 0; i < n; ++i) {                                    /* f'_i = min_j (C_ij - g_j) */
        double m = INFINITY;
        for (int j = 0; j < n; ++j) m = fmin(m, C[IDX(i, j)] - g[j]);
        f[i] = m;
    }
    double lb = 0.0;
    for (int i = 0; i < n; ++i) lb += f[i] * r[i];
    for (int j = 0; j < n; ++j) lb += g[j] * c[j];
    free(f); free(g);
    return lb;
}

double or_gamma_f_for_eps(double H_min, double eps, double gamma_i, double q, double p)
{
    /* Prop. 2: gamma_f = (5 H_min / (2 eps))^(1/p); reading: rounded up onto gamma_i q^k */
    double target = pow(5.0 * H_min / (2.0 * eps), 1.0 / p);
    double g = gamma_i;
    while (g < target * (1.0 - 1e-12)) g *= q;
    return g;
}
