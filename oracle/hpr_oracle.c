/*
 * HPR-LP oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of the HPR-LP method of
 * Chen, Sun, Yuan, Zhang & Zhao, "HPR-LP: An implementation of an HPR method for
 * solving linear programming" (arXiv 2408.12179).  It exists to check the CUDA solver
 * and is loaded only by the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark.  It shares no code, header or constant table with the CUDA solver.
 *
 * Problem (Section 1, eq. (1)):  min <c,x>  s.t.  A1 x = b1,  A2 x >= b2,  l <= x <= u,
 * with A = [A1; A2] (m = m1 + m2 rows) given in CSR with sorted column indices.
 *
 * What each part follows:
 *   - preprocessing: 10 Ruiz iterations, Pock-Chambolle diagonal scaling with
 *     alpha = 1, then b / (||b||+1) and c / (||c||+1)          (Section 4.1)
 *   - T1 = lambda I - A A^*, lambda = lambda_1(A A^*) by the power method (Section 4.1)
 *   - the iteration: Algorithm 2 with the closed forms eq. (update-z), (update-x),
 *     (update-y-2) of Section 3.3, reflection and Halpern step of Algorithm 2
 *   - restart criteria eq. (restart_1)-(restart_3), merit R~ (Section 3.1)
 *   - SigmaUpdate, Algorithm 3, with eq. (sigma_T1!=0)            (Section 3.2)
 *   - termination test of Section 4.1, checked every `check_every` iterations.
 *
 * Readings where the paper is silent (all shared with the CUDA solver by
 * specification, not by code):
 *   - Ruiz scales rows and columns simultaneously from the same matrix; an empty row
 *     or column gets factor 1.  Pock-Chambolle: row i divided by sqrt(sum_j |a_ij|^(2-alpha)),
 *     column j by sqrt(sum_i |a_ij|^alpha).
 *   - the bounds are scaled like x: l_s = l / (D_c * beta_b), u_s likewise.
 *   - power method: start vector from SplitMix64(seed) mapped to U(-1,1), normalised;
 *     lambda_k = ||A^T u_k||^2; stop when |lambda_k - lambda_{k-1}| <= tol * lambda_k.
 *   - iterations are counted from k = 0; iteration k maps w^k to w^{k+1}.  A check runs
 *     in iteration k when (k+1) % check_every == 0 or k+1 == max_iter, on w_bar^{k+1}.
 *     The first iteration of every inner loop (t = 0) evaluates R~_{r,0}.
 *   - restart criteria are evaluated at checks only; criterion (restart_2) compares with
 *     the R~ of the previous evaluation in the same inner loop (R~_{r,0} at the first);
 *     criterion (restart_3) uses the counters after the iteration (t+1 >= alpha3 (k+1)).
 *   - termination is tested on the original (unscaled) problem; the back-mapped x is
 *     projected onto C again (rounding of beta_b D_c (u / (D_c beta_b)) can exceed u).
 *   - SigmaUpdate uses the scaled-space Delta_x, Delta_y and the err_p, err_d of the
 *     check that triggered the restart.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

/* ---------------------------------------------------------------- interface */

typedef struct {
    int64_t m1, m2, n, nnz;
    const int64_t *row_ptr; /* m+1 */
    const int32_t *col_idx; /* nnz, sorted within each row */
    const double *val;      /* nnz */
    const double *b;        /* m  = [b1; b2] */
    const double *c, *l, *u;/* n */
} orc_lp;

typedef struct {
    double tol;
    int64_t max_iter;
    int64_t check_every;
    double alpha1, alpha2, alpha3;
    double sigma0;
    int64_t ruiz_iters;
    double pc_alpha;
    int64_t power_max_iter;
    double power_tol;
    uint64_t seed;
    double lambda_fixed;     /* > 0: use this lambda instead of the power method */
    int64_t restart;         /* 0 disables the restart criteria */
    int64_t sigma_update;    /* 0 keeps sigma = sigma0 at restarts */
    int64_t trace_iters;     /* record the first trace_iters iterations */
    int64_t halpern;         /* 0: w = w_target instead of the Halpern step (ablation) */
    int64_t reflect;         /* 0: w_target = w_bar instead of w_hat = 2 w_bar - w (ablation) */
} orc_opts;

/* info[] layout */
enum { OI_STATUS, OI_ITERS, OI_RESTARTS, OI_SIGMA, OI_LAMBDA, OI_POWER_ITERS, OI_POBJ,
       OI_DOBJ, OI_ERRP, OI_ERRD, OI_GAP, OI_KKT, OI_BETA_B, OI_BETA_C, OI_NCHECKS,
       OI_SECONDS, OI_LEN };
/* one record per check / R~_{r,0} evaluation */
enum { OC_K, OC_R, OC_T, OC_SIGMA, OC_ERRP, OC_ERRD, OC_GAP, OC_KKT, OC_POBJ, OC_DOBJ,
       OC_RT, OC_R0, OC_CAUSE, OC_SIGMA_NEXT, OC_KIND, OC_DX, OC_DY, OC_LEN };

typedef struct {
    double *x, *y, *z;        /* final w_bar in the original space (n, m, n); may be NULL */
    double *info;             /* OI_LEN doubles */
    double *trace;            /* trace_iters records of 3n+2m: xbar, xhat, x, ybar, y */
    double *checks;           /* checks_cap records of OC_LEN */
    int64_t checks_cap;
    double *Dr, *Dc;          /* scaling (m, n); may be NULL */
    double *As_val;           /* scaled values, CSR order of A (nnz); may be NULL */
    double *bs, *cs, *ls, *us;/* scaled data; may be NULL */
} orc_out;

/* ---------------------------------------------------------------- helpers */

static double dot(int64_t n, const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static double nrm2(int64_t n, const double *a) { return sqrt(dot(n, a, a)); }

/* out = M v for an m-row CSR matrix; each row summed in index order */
static void matvec(int64_t m, const int64_t *rp, const int32_t *ci, const double *v,
                   const double *x, double *out)
{
#pragma omp parallel for schedule(static) if (m > 4096)
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += v[p] * x[ci[p]];
        out[i] = s;
    }
}

/* CSR transpose by a stable counting sort: rows of the result list the original
 * row indices in increasing order */
static void transpose(int64_t m, int64_t n, const int64_t *rp, const int32_t *ci,
                      const double *v, int64_t *rpT, int32_t *ciT, double *vT)
{
    memset(rpT, 0, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t p = 0; p < rp[m]; ++p) rpT[ci[p] + 1]++;
    for (int64_t j = 0; j < n; ++j) rpT[j + 1] += rpT[j];
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    memcpy(next, rpT, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t i = 0; i < m; ++i)
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            int64_t q = next[ci[p]]++;
            ciT[q] = (int32_t)i;
            if (v) vT[q] = v[p];
        }
    free(next);
}

/* SplitMix64 (Steele, Lea & Flood 2014), i-th output of the stream started at seed */
static uint64_t splitmix64_at(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ---------------------------------------------------------------- preprocessing */

/* Section 4.1: Ruiz (ruiz_iters), Pock-Chambolle (alpha), then b and c normalisation.
 * Writes the scaled values (CSR order of A), D_r, D_c, the scaled b, c, l, u and
 * beta = {||D_r b|| + 1, ||D_c c|| + 1}. */
int orc_scale(const orc_lp *P, int64_t ruiz_iters, double pc_alpha, double *As,
              double *Dr, double *Dc, double *bs, double *cs, double *ls, double *us,
              double *beta)
{
    const int64_t m = P->m1 + P->m2, n = P->n, nnz = P->nnz;
    const int64_t *rp = P->row_ptr;
    const int32_t *ci = P->col_idx;
    double *dr = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *dc = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    memcpy(As, P->val, sizeof(double) * (size_t)nnz);
    for (int64_t i = 0; i < m; ++i) Dr[i] = 1.0;
    for (int64_t j = 0; j < n; ++j) Dc[j] = 1.0;

    /* Ruiz equilibration: divide every row and column by the square root of its
     * infinity norm, both taken from the same matrix */
    for (int64_t it = 0; it < ruiz_iters; ++it) {
        for (int64_t i = 0; i < m; ++i) dr[i] = 0.0;
        for (int64_t j = 0; j < n; ++j) dc[j] = 0.0;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                double a = fabs(As[p]);
                if (a > dr[i]) dr[i] = a;
                if (a > dc[ci[p]]) dc[ci[p]] = a;
            }
        for (int64_t i = 0; i < m; ++i) dr[i] = dr[i] > 0.0 ? 1.0 / sqrt(dr[i]) : 1.0;
        for (int64_t j = 0; j < n; ++j) dc[j] = dc[j] > 0.0 ? 1.0 / sqrt(dc[j]) : 1.0;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) As[p] = As[p] * dr[i] * dc[ci[p]];
        for (int64_t i = 0; i < m; ++i) Dr[i] *= dr[i];
        for (int64_t j = 0; j < n; ++j) Dc[j] *= dc[j];
    }

    /* Pock-Chambolle diagonal preconditioning with parameter alpha */
    if (pc_alpha >= 0.0) {
        for (int64_t i = 0; i < m; ++i) dr[i] = 0.0;
        for (int64_t j = 0; j < n; ++j) dc[j] = 0.0;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                double a = fabs(As[p]);
                dr[i] += pc_alpha == 1.0 ? a : pow(a, 2.0 - pc_alpha);
                dc[ci[p]] += pc_alpha == 1.0 ? a : pow(a, pc_alpha);
            }
        for (int64_t i = 0; i < m; ++i) dr[i] = dr[i] > 0.0 ? 1.0 / sqrt(dr[i]) : 1.0;
        for (int64_t j = 0; j < n; ++j) dc[j] = dc[j] > 0.0 ? 1.0 / sqrt(dc[j]) : 1.0;
        for (int64_t i = 0; i < m; ++i)
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) As[p] = As[p] * dr[i] * dc[ci[p]];
        for (int64_t i = 0; i < m; ++i) Dr[i] *= dr[i];
        for (int64_t j = 0; j < n; ++j) Dc[j] *= dc[j];
    }

    /* x = D_c x~ and rows multiplied by D_r; then b / (||b||+1), c / (||c||+1) */
    for (int64_t i = 0; i < m; ++i) bs[i] = P->b[i] * Dr[i];
    for (int64_t j = 0; j < n; ++j) {
        cs[j] = P->c[j] * Dc[j];
        ls[j] = P->l[j] / Dc[j];
        us[j] = P->u[j] / Dc[j];
    }
    beta[0] = nrm2(m, bs) + 1.0;
    beta[1] = nrm2(n, cs) + 1.0;
    for (int64_t i = 0; i < m; ++i) bs[i] /= beta[0];
    for (int64_t j = 0; j < n; ++j) {
        cs[j] /= beta[1];
        ls[j] /= beta[0];
        us[j] /= beta[0];
    }
    free(dr);
    free(dc);
    return 0;
}

/* ---------------------------------------------------------------- power method */

/* lambda_1(A A^*) of an m x n CSR matrix by the power method (Section 4.1) */
double orc_power(int64_t m, int64_t n, const int64_t *rp, const int32_t *ci,
                 const double *v, uint64_t seed, int64_t max_iter, double tol,
                 int64_t *iters_out)
{
    int64_t *rpT = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *ciT = (int32_t *)malloc(sizeof(int32_t) * (size_t)(rp[m] > 0 ? rp[m] : 1));
    double *vT = (double *)malloc(sizeof(double) * (size_t)(rp[m] > 0 ? rp[m] : 1));
    double *uu = (double *)malloc(sizeof(double) * (size_t)m);
    double *s = (double *)malloc(sizeof(double) * (size_t)n);
    double *w = (double *)malloc(sizeof(double) * (size_t)m);
    transpose(m, n, rp, ci, v, rpT, ciT, vT);

    for (int64_t i = 0; i < m; ++i)
        uu[i] = 2.0 * ((double)(splitmix64_at(seed, (uint64_t)i) >> 11) * 0x1.0p-53) - 1.0;
    double nu = nrm2(m, uu);
    for (int64_t i = 0; i < m; ++i) uu[i] /= nu;

    double lam = 0.0, lam_prev = 0.0;
    int64_t k;
    for (k = 1; k <= max_iter; ++k) {
        matvec(n, rpT, ciT, vT, uu, s);          /* s = A^T u */
        lam = dot(n, s, s);                      /* Rayleigh quotient u^T A A^T u */
        if (k > 1 && fabs(lam - lam_prev) <= tol * lam) break;
        lam_prev = lam;
        matvec(m, rp, ci, v, s, w);              /* w = A A^T u */
        double nw = nrm2(m, w);
        if (!(nw > 0.0)) break;
        for (int64_t i = 0; i < m; ++i) uu[i] = w[i] / nw;
    }
    if (iters_out) *iters_out = k > max_iter ? max_iter : k;
    free(rpT); free(ciT); free(vT); free(uu); free(s); free(w);
    return lam;
}

/* ---------------------------------------------------------------- solver */

typedef struct {
    int64_t m, m1, n;
    const int64_t *rp; const int32_t *ci; const double *v;       /* scaled A */
    const int64_t *rpT; const int32_t *ciT; const double *vT;    /* scaled A^T */
} sys_t;

/* ||w - w_hat||_M = 2 ||w - w_bar||_M with M of eq. (def:M) and T1 = lambda I - A A^*:
 * ||(dy, dx)||_M^2 = sigma*lambda ||dy||^2 + 2 <dy, A dx> + ||dx||^2 / sigma */
static double merit(const sys_t *S, double sigma, double lambda, const double *x,
                    const double *xbar, const double *y, const double *ybar,
                    double *dx, double *dy, double *Adx)
{
    for (int64_t j = 0; j < S->n; ++j) dx[j] = x[j] - xbar[j];
    for (int64_t i = 0; i < S->m; ++i) dy[i] = y[i] - ybar[i];
    matvec(S->m, S->rp, S->ci, S->v, dx, Adx);
    double q = sigma * lambda * dot(S->m, dy, dy) + 2.0 * dot(S->m, dy, Adx)
             + dot(S->n, dx, dx) / sigma;
    return 2.0 * sqrt(q > 0.0 ? q : 0.0);
}

int orc_hpr(const orc_lp *P, const orc_opts *O, orc_out *out)
{
    struct timespec ts0, ts1;
    const int64_t m1 = P->m1, m = P->m1 + P->m2, n = P->n, nnz = P->nnz;
    const size_t Sm = sizeof(double) * (size_t)(m > 0 ? m : 1);
    const size_t Sn = sizeof(double) * (size_t)(n > 0 ? n : 1);
    const size_t Sz = sizeof(double) * (size_t)(nnz > 0 ? nnz : 1);

    /* ---- preprocessing (Section 4.1) */
    double *As = (double *)malloc(Sz), *Dr = (double *)malloc(Sm), *Dc = (double *)malloc(Sn);
    double *bs = (double *)malloc(Sm), *cs = (double *)malloc(Sn);
    double *ls = (double *)malloc(Sn), *us = (double *)malloc(Sn);
    double beta[2];
    orc_scale(P, O->ruiz_iters, O->pc_alpha, As, Dr, Dc, bs, cs, ls, us, beta);

    int64_t *rpT = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *ciT = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    double *AsT = (double *)malloc(Sz), *AoT = (double *)malloc(Sz);
    transpose(m, n, P->row_ptr, P->col_idx, As, rpT, ciT, AsT);
    transpose(m, n, P->row_ptr, P->col_idx, P->val, rpT, ciT, AoT); /* original A^T */
    sys_t S = { m, m1, n, P->row_ptr, P->col_idx, As, rpT, ciT, AsT };
    /* solve time excludes preprocessing and includes the power method (Section 4.1) */
    clock_gettime(CLOCK_MONOTONIC, &ts0);

    /* ---- T1 = lambda I - A A^* (Section 4.1) */
    int64_t power_iters = 0;
    double lambda = O->lambda_fixed;
    if (!(lambda > 0.0))
        lambda = orc_power(m, n, P->row_ptr, P->col_idx, As, O->seed, O->power_max_iter,
                           O->power_tol, &power_iters);

    /* norms of the original b, c for the relative residuals of Section 4.1 */
    const double nb = nrm2(m, P->b), nc = nrm2(n, P->c);

    double *x = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *x0 = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *y = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    double *y0 = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    double *s = (double *)malloc(Sn), *xhat = (double *)malloc(Sn), *q = (double *)malloc(Sm);
    double *xbar = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *zbar = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *ybar = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    double *yhat = (double *)malloc(Sm);
    double *dx = (double *)malloc(Sn), *dy = (double *)malloc(Sm), *Adx = (double *)malloc(Sm);
    double *xo = (double *)malloc(Sn), *yo = (double *)malloc(Sm), *zo = (double *)malloc(Sn);
    double *Axo = (double *)malloc(Sm), *ATyo = (double *)malloc(Sn);

    double sigma = O->sigma0;
    int64_t k = 0, t = 0, r = 0, nchecks = 0;
    int status = 1; /* max_iter unless converged */
    double R0 = 0.0, Rprev = 0.0;
    double last[6] = {0, 0, 0, 0, 0, 0}; /* pobj dobj errp errd gap kkt */

    for (k = 0; k < O->max_iter; ++k) {
        const int is_check = ((k + 1) % O->check_every == 0) || (k + 1 == O->max_iter);
        const int is_r0 = (t == 0);

        /* eq. (update-z), (update-x): v = x + sigma (A^* y - c), x_bar = Pi_C(v),
         * z_bar = (Pi_C(v) - v) / sigma; reflection x_hat = 2 x_bar - x */
        matvec(n, rpT, ciT, AsT, y, s);
        for (int64_t j = 0; j < n; ++j) {
            double v = x[j] + sigma * (s[j] - cs[j]);
            xbar[j] = fmin(fmax(v, ls[j]), us[j]);
            zbar[j] = (xbar[j] - v) / sigma;
            xhat[j] = 2.0 * xbar[j] - x[j];
        }
        /* eq. (update-y-2): y_bar = y + (b - A(2 x_bar - x)) / (lambda sigma), the m2
         * block projected onto R_+; reflection y_hat = 2 y_bar - y */
        matvec(m, P->row_ptr, P->col_idx, As, xhat, q);
        for (int64_t i = 0; i < m; ++i) {
            double yb = y[i] + (bs[i] - q[i]) / (lambda * sigma);
            if (i >= m1) yb = fmax(yb, 0.0);
            ybar[i] = yb;
            yhat[i] = 2.0 * yb - y[i];
        }

        int restart = 0, cause = 0, stop = 0;
        double sigma_next = sigma, Rt = 0.0, Dx = 0.0, Dy = 0.0;
        double rec_errp = 0, rec_errd = 0, rec_gap = 0, rec_kkt = 0, rec_pobj = 0, rec_dobj = 0;

        if (is_r0 || is_check) {
            Rt = merit(&S, sigma, lambda, x, xbar, y, ybar, dx, dy, Adx);
            if (is_r0) { R0 = Rt; Rprev = Rt; }
        }
        if (is_check) {
            /* termination test of Section 4.1 on w_bar mapped back to the original LP:
             * x = beta_b D_c x_s, y = beta_c D_r y_s, z = beta_c z_s / D_c; x is projected
             * onto C once more so that the rounding of the scaling cannot leave it */
            for (int64_t j = 0; j < n; ++j) {
                xo[j] = fmin(fmax(beta[0] * Dc[j] * xbar[j], P->l[j]), P->u[j]);
                zo[j] = beta[1] * zbar[j] / Dc[j];
            }
            for (int64_t i = 0; i < m; ++i) yo[i] = beta[1] * Dr[i] * ybar[i];
            matvec(m, P->row_ptr, P->col_idx, P->val, xo, Axo);
            matvec(n, rpT, ciT, AoT, yo, ATyo);
            double ep = 0.0, ed = 0.0, pobj = 0.0, dobj = 0.0;
            for (int64_t i = 0; i < m; ++i) {
                double ri = P->b[i] - Axo[i];          /* Pi_D(b - A x) */
                if (i >= m1) ri = fmax(ri, 0.0);
                ep += ri * ri;
            }
            for (int64_t j = 0; j < n; ++j) {
                double rj = P->c[j] - ATyo[j] - zo[j];
                ed += rj * rj;
            }
            pobj = dot(n, P->c, xo);
            dobj = dot(m, P->b, yo);                   /* <b,y> - delta_C^*(-z) */
            for (int64_t j = 0; j < n; ++j) {
                if (zo[j] > 0.0) dobj += zo[j] * P->l[j];
                else if (zo[j] < 0.0) dobj += zo[j] * P->u[j];
            }
            double errp = sqrt(ep) / (1.0 + nb), errd = sqrt(ed) / (1.0 + nc);
            double gap = fabs(dobj - pobj) / (1.0 + fabs(pobj) + fabs(dobj));
            double kkt = fmax(errp, fmax(errd, gap));
            rec_errp = errp; rec_errd = errd; rec_gap = gap; rec_kkt = kkt;
            rec_pobj = pobj; rec_dobj = dobj;
            last[0] = pobj; last[1] = dobj; last[2] = errp; last[3] = errd; last[4] = gap; last[5] = kkt;

            if (kkt <= O->tol) {
                stop = 1;
                status = 0;
                cause = -1;
            } else if (k + 1 < O->max_iter && O->restart && !is_r0) {
                /* restart criteria (restart_1)-(restart_3) */
                if (Rt <= O->alpha1 * R0) cause = 1;
                else if (Rt <= O->alpha2 * R0 && Rt > Rprev) cause = 2;
                else if ((double)(t + 1) >= O->alpha3 * (double)(k + 1)) cause = 3;
                Rprev = Rt;
                restart = cause != 0;
            }
            if (restart) {
                /* Algorithm 3 with eq. (sigma_T1!=0):
                 * Delta_x = ||x_bar - x0||, Delta_y = sqrt(lambda) ||y_bar - y0|| */
                double sx = 0.0, sy = 0.0;
                for (int64_t j = 0; j < n; ++j) sx += (xbar[j] - x0[j]) * (xbar[j] - x0[j]);
                for (int64_t i = 0; i < m; ++i) sy += (ybar[i] - y0[i]) * (ybar[i] - y0[i]);
                Dx = sqrt(sx);
                Dy = sqrt(lambda) * sqrt(sy);
                double ratio = errd / errp;
                if (O->sigma_update && Dx > 1e-16 && Dx < 1e12 && Dy > 1e-16 && Dy < 1e12 &&
                    errp > 0.0 && ratio > 1e-8 && ratio < 1e8)
                    sigma_next = Dx / Dy;
                else
                    sigma_next = O->sigma_update ? 1.0 : sigma;
            }
        }

        if (is_r0 || is_check) {
            if (out->checks && nchecks < out->checks_cap) {
                double *rec = out->checks + nchecks * OC_LEN;
                rec[OC_K] = (double)k; rec[OC_R] = (double)r; rec[OC_T] = (double)t;
                rec[OC_SIGMA] = sigma; rec[OC_ERRP] = rec_errp; rec[OC_ERRD] = rec_errd;
                rec[OC_GAP] = rec_gap; rec[OC_KKT] = rec_kkt; rec[OC_POBJ] = rec_pobj;
                rec[OC_DOBJ] = rec_dobj; rec[OC_RT] = Rt; rec[OC_R0] = R0;
                rec[OC_CAUSE] = (double)cause; rec[OC_SIGMA_NEXT] = sigma_next;
                rec[OC_KIND] = (double)(is_check ? 1 : 0) + (is_r0 ? 2 : 0);
                rec[OC_DX] = Dx; rec[OC_DY] = Dy;
            }
            nchecks++;
        }

        if (stop) {
            k++;
            break;
        }
        if (restart) {
            /* w^{r+1,0} = w_bar^{r,tau_r}; new anchor; sigma_{r+1} */
            for (int64_t j = 0; j < n; ++j) x[j] = x0[j] = xbar[j];
            for (int64_t i = 0; i < m; ++i) y[i] = y0[i] = ybar[i];
            sigma = sigma_next;
            t = 0;
            r++;
        } else {
            /* Halpern step of Algorithm 2: w = w0/(t+2) + (t+1)/(t+2) w_hat.  Ablation
             * (Section 4.2): the target is w_bar instead of w_hat without the relaxation
             * step, and w = target without the Halpern step (the DR method when both are
             * off, with restarts and sigma updates off too) */
            const double *tx = O->reflect ? xhat : xbar, *ty = O->reflect ? yhat : ybar;
            if (O->halpern) {
                const double a = 1.0 / (double)(t + 2), bcoef = (double)(t + 1) / (double)(t + 2);
                for (int64_t j = 0; j < n; ++j) x[j] = a * x0[j] + bcoef * tx[j];
                for (int64_t i = 0; i < m; ++i) y[i] = a * y0[i] + bcoef * ty[i];
            } else {
                for (int64_t j = 0; j < n; ++j) x[j] = tx[j];
                for (int64_t i = 0; i < m; ++i) y[i] = ty[i];
            }
            t++;
        }

        if (out->trace && k < O->trace_iters) {
            double *tr = out->trace + (size_t)k * (size_t)(3 * n + 2 * m);
            memcpy(tr, xbar, sizeof(double) * (size_t)n);
            memcpy(tr + n, xhat, sizeof(double) * (size_t)n);
            memcpy(tr + 2 * n, x, sizeof(double) * (size_t)n);
            memcpy(tr + 3 * n, ybar, sizeof(double) * (size_t)m);
            memcpy(tr + 3 * n + m, y, sizeof(double) * (size_t)m);
        }
    }

    /* output: the last w_bar, mapped back to the original space */
    for (int64_t j = 0; j < n; ++j) {
        if (out->x) out->x[j] = fmin(fmax(beta[0] * Dc[j] * xbar[j], P->l[j]), P->u[j]);
        if (out->z) out->z[j] = beta[1] * zbar[j] / Dc[j];
    }
    if (out->y)
        for (int64_t i = 0; i < m; ++i) out->y[i] = beta[1] * Dr[i] * ybar[i];
    if (out->Dr) memcpy(out->Dr, Dr, Sm);
    if (out->Dc) memcpy(out->Dc, Dc, Sn);
    if (out->As_val) memcpy(out->As_val, As, Sz);
    if (out->bs) memcpy(out->bs, bs, Sm);
    if (out->cs) memcpy(out->cs, cs, Sn);
    if (out->ls) memcpy(out->ls, ls, Sn);
    if (out->us) memcpy(out->us, us, Sn);

    clock_gettime(CLOCK_MONOTONIC, &ts1);
    if (out->info) {
        double *I = out->info;
        I[OI_STATUS] = status; I[OI_ITERS] = (double)k; I[OI_RESTARTS] = (double)r;
        I[OI_SIGMA] = sigma; I[OI_LAMBDA] = lambda; I[OI_POWER_ITERS] = (double)power_iters;
        I[OI_POBJ] = last[0]; I[OI_DOBJ] = last[1]; I[OI_ERRP] = last[2]; I[OI_ERRD] = last[3];
        I[OI_GAP] = last[4]; I[OI_KKT] = last[5]; I[OI_BETA_B] = beta[0]; I[OI_BETA_C] = beta[1];
        I[OI_NCHECKS] = (double)nchecks;
        I[OI_SECONDS] = (double)(ts1.tv_sec - ts0.tv_sec) + 1e-9 * (double)(ts1.tv_nsec - ts0.tv_nsec);
    }

    free(As); free(Dr); free(Dc); free(bs); free(cs); free(ls); free(us);
    free(rpT); free(ciT); free(AsT); free(AoT);
    free(x); free(x0); free(y); free(y0); free(s); free(xbar); free(zbar); free(xhat);
    free(q); free(ybar); free(yhat); free(dx); free(dy); free(Adx);
    free(xo); free(yo); free(zo); free(Axo); free(ATyo);
    return status;
}
