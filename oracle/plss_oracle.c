/*
 * plss_oracle.c -- plain, slow, single-threaded FP64 CPU PLSS.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the parity oracle for the CUDA
 * path: only the test suite, the package smoke check and the benchmark's CPU
 * baseline load it. It shares no code with the CUDA library and is compiled
 * with -ffp-contract=off so that every a*b+c is two roundings, as written.
 *
 * What it follows (Brust & Saunders, "PLSS: a projected linear systems
 * solver", arXiv 2207.07615):
 *   - plss_oracle_residual: Algorithm 1 (Sec. 5), the residual-sketch
 *     recursion of Theorem 4.1 (eq:pkShort), with the optional diagonal
 *     weight of Sec. 4.1 (eq:pkShortW), written step by step in the
 *     algorithm's order. Sums run in ascending index order.
 *   - plss_oracle_kaczmarz: the identity sketch of Sec. 7 (eq:pkKacz),
 *     with a dense history P (n x K) and Theta = diag(||p_j||^2).
 *   - plss_oracle_colweights: W = diag(1/||A_{:,j}||) of Sec. 4.1.
 *   - plss_oracle_general: a general sketch S_k = [s_1 ... s_k] (eq:genS)
 *     with random sign columns, through the update of the inverse
 *     N_k = (Y_k^T Y_k)^{-1} of Theorem 2.1 (eq:Nkrec) and the update
 *     p_k of Corollary 2.2 (eq:compute-pk-alpha1), Sec. 2.4.
 *
 * Readings where the paper is silent or inconsistent (all listed in the
 * design notes of the repository):
 *   - gamma: Algorithm 1's gamma = (theta/rho) * beta. The closed form in the
 *     statement of Theorem 4.1 differs by a factor rho.
 *   - stopping: stop when sqrt(rho)/||b|| <= tol, tested right after rho is
 *     formed (Sec. 5 suggests sqrt(rho)/||b|| < tau); maxit caps the number
 *     of updates p applied to x; the residual of the returned x is always
 *     formed (the row sweep after the last update runs).
 *   - breakdown: the initial phi must be > 0 and finite; later the factor
 *     (s/rho - 1)(s/rho + 1) must be > 0 and finite (it is <= 0 only when
 *     y is parallel to p); otherwise return the current x with status
 *     BREAKDOWN -- except when stopping on the true residual, where a
 *     breakdown after the first update (rounding has destroyed the
 *     orthogonality the recursion relies on) restarts from b - A x.
 *   - FP32 storage (prec = 1): A's values, r, p and W y are held as float,
 *     sums of products are accumulated in float, inner products and the
 *     scalar recursion in double, x in double; the residual is recomputed as
 *     b - A x in double every `refine` updates and whenever rho has fallen
 *     by inner_tol^2 since the last start (or risen above 4x its starting
 *     value) -- iterative refinement, which keeps the float recursion away
 *     from its rounding floor where it turns unstable (this extension is not
 *     in the paper). With replace = 0 the recursion restarts from the fresh
 *     residual (a new first step); with replace = 1 the fresh residual only
 *     replaces the recursive one and the recursion goes on with its p and
 *     theta (residual replacement; in exact arithmetic the two residuals are
 *     equal, so the iterates are unchanged). A stop confirmed false on
 *     b - A x refreshes the residual the same way. replace = 1 also applies
 *     the period in FP64 storage.
 *   - Kaczmarz order: rows are visited without replacement in a fresh
 *     permutation per pass (SplitMix64 stream + Fisher-Yates shuffle); the
 *     history holds at most K updates and, once full, is emptied before the
 *     next row (which then takes a plain Kaczmarz step, so every stored
 *     update lives on the union of the window's rows); a row whose projected
 *     norm delta is <= 1e-14 ||a_i||^2 is skipped; the window stores each
 *     row's direction q = p / gamma (the same projector), so a row with
 *     r_i = 0 still enters it and the window schedule does not depend on
 *     rounding in b - A x.
 *
 * Planted defects (argument `plant`, 0 in every real use): the pins of the
 * test suite must reject each of them, which shows that they can see such a
 * mistake. Residual sketch: 1 = the statement form of gamma, 2 = the drift
 * restart at 2x instead of 4x the starting rho, 3 = the inner-solve restart
 * at inner_tol instead of inner_tol^2. Identity sketch: 1 = the window is
 * emptied one row late (K + 1 directions), 2 = one row early (K - 1),
 * 3 = never (the whole history is kept). General sketch: 1 = the rank-one
 * term t t^T / delta is left out of the update of N (eq:Nkrec).
 *
 * General-sketch columns (a reading: the paper leaves the sketch open and
 * draws random normal sketches for its comparisons): s_k has entries +1 or
 * -1, entry i of the k-th column (k = 0, 1, ... counting every column drawn)
 * being the sign bit of output number k*m + i of the SplitMix64 stream
 * seeded with `seed` (output j = mix(seed + (j + 1) * golden gamma), so any
 * entry is computed directly from (seed, k, i)); bit 63 set gives -1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* The same file built with -fopenmp (oracle/__init__.py, residual_omp)
 * runs the residual sketch's row, column and vector loops on all host cores
 * (timing only: the pins use the plain build, where these expand to
 * nothing). Rows, columns and entries are independent; the dot products
 * become per-thread partial sums combined by OpenMP. */
#ifdef _OPENMP
#define PAR_FOR _Pragma("omp parallel for schedule(static)")
#define PAR_SUM(v) _Pragma(PAR_STR(omp parallel for schedule(static) reduction(+ : v)))
#define PAR_STR(x) #x
#else
#define PAR_FOR
#define PAR_SUM(v)
#endif

enum {
    ORC_CONVERGED = 0,
    ORC_NOT_CONVERGED = 1,
    ORC_BREAKDOWN = -4,
    ORC_INVALID = -1,
    ORC_NOMEM = -2
};

/* ------------------------------------------------------------------ */
/* plain sparse products                                               */
/* ------------------------------------------------------------------ */

/* out = A v, CSR, ascending nonzero order per row. */
void plss_oracle_spmv(int64_t m, const int64_t *row_ptr, const int32_t *col_idx,
                      const double *val, const double *v, double *out)
{
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            s += val[k] * v[col_idx[k]];
        out[i] = s;
    }
}

/* Builds the CSC of A (col_ptr[n+1], row_idx[nnz], cval[nnz]) with row
 * indices ascending inside each column (a stable counting sort). */
static void csr_to_csc(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                       const double *val, int64_t *col_ptr, int64_t *row_idx, double *cval)
{
    int64_t nnz = row_ptr[m];
    for (int64_t j = 0; j <= n; ++j) col_ptr[j] = 0;
    for (int64_t k = 0; k < nnz; ++k) col_ptr[col_idx[k] + 1] += 1;
    for (int64_t j = 0; j < n; ++j) col_ptr[j + 1] += col_ptr[j];
    int64_t *next = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    for (int64_t j = 0; j <= n; ++j) next[j] = col_ptr[j];
    for (int64_t i = 0; i < m; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t dst = next[col_idx[k]]++;
            row_idx[dst] = i;
            cval[dst] = val[k];
        }
    free(next);
}

/* out = A^T r, computed column by column from the CSC (ascending rows). */
static void csc_spmv(int64_t n, const int64_t *col_ptr, const int64_t *row_idx,
                     const double *cval, const double *r, double *out)
{
    PAR_FOR
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t k = col_ptr[j]; k < col_ptr[j + 1]; ++k)
            s += cval[k] * r[row_idx[k]];
        out[j] = s;
    }
}

/* out = A^T r through a freshly built CSC. */
int plss_oracle_spmvt(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                      const double *val, const double *r, double *out)
{
    int64_t nnz = row_ptr[m];
    int64_t *cp = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t *ri = (int64_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(int64_t));
    double *cv = (double *)malloc((size_t)(nnz ? nnz : 1) * sizeof(double));
    if (!cp || !ri || !cv) { free(cp); free(ri); free(cv); return ORC_NOMEM; }
    csr_to_csc(m, n, row_ptr, col_idx, val, cp, ri, cv);
    csc_spmv(n, cp, ri, cv, r, out);
    free(cp); free(ri); free(cv);
    return 0;
}

static double dot(int64_t len, const double *a, const double *b)
{
    double s = 0.0;
    PAR_SUM(s)
    for (int64_t i = 0; i < len; ++i) s += a[i] * b[i];
    return s;
}

/* W = diag(w) from the column norms of A (Sec. 4.1): mode 1 gives
 * w_j = 1/||A_{:,j}||, mode 2 gives w_j = 1/||A_{:,j}||^2; an empty
 * column gets w_j = 1. */
void plss_oracle_colweights(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                            const double *val, int mode, double *w)
{
    double *ss = (double *)calloc((size_t)(n ? n : 1), sizeof(double));
    for (int64_t i = 0; i < m; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            ss[col_idx[k]] += val[k] * val[k];
    for (int64_t j = 0; j < n; ++j) {
        if (ss[j] == 0.0) w[j] = 1.0;
        else if (mode == 2) w[j] = 1.0 / ss[j];
        else w[j] = 1.0 / sqrt(ss[j]);
    }
    free(ss);
}

/* ------------------------------------------------------------------ */
/* Residual sketch: Algorithm 1                                        */
/* ------------------------------------------------------------------ */

static inline double rf(double v, int f32) { return f32 ? (double)(float)v : v; }

/* r = b - A x, double accumulation; returns nothing. */
static void true_residual(int64_t m, const int64_t *row_ptr, const int32_t *col_idx,
                          const double *val, const double *b, const double *x, double *r)
{
    PAR_FOR
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            s += val[k] * x[col_idx[k]];
        r[i] = b[i] - s;
    }
}

/*
 * PLSS with the residual sketch S_k = [r_0 ... r_{k-1}] (Sec. 4, eq:S),
 * following Algorithm 1:
 *   r = b - A x0;  y = A^T r;  rho = r^T r;  u = W y;  phi = y^T u;
 *   p = (rho/phi) u;  theta = p^T W^{-1} p;  x = x + p;
 *   repeat: r = r - A p; y = A^T r; rho = r^T r; u = W y; phi = y^T u;
 *           beta = 1/((sqrt(theta phi)/rho - 1)(sqrt(theta phi)/rho + 1));
 *           gamma = (theta/rho) beta;  p = beta p + gamma u;
 *           theta = p^T W^{-1} p;  x = x + p.
 * W = diag(w) (w = NULL means W = I).
 *
 * Arguments: CSR A (m x n), b[m], x0[n] (NULL = 0), w[n] (NULL = I),
 * tol >= 0, maxit >= 0 (cap on updates), prec 0 = FP64, 1 = FP32 storage,
 * refine = restart period in updates for prec 1 (0 = never), inner_tol > 0:
 * restart from b - A x once rho has fallen by inner_tol^2 since the last
 * start (the inner solve of iterative refinement; 0 = never), stop_on_true:
 * the stop decision uses the residual b - A x recomputed in double,
 * plant = a planted defect (see the file header; 0 = none), replace = 1:
 * refreshes replace the residual instead of restarting (see the header).
 * Outputs: x_out[n], *iters (updates applied), *relres_rec (sqrt(rho)/||b||
 * of the last rho), *relres_true (||b - A x||/||b||), return value = status.
 * Optional history (any pointer may be NULL; hist_cap rows):
 *   hist_s[k*5 + 0..4] = rho_{k}, phi_{k+1}, beta_{k}, gamma_{k}, theta_{k+1}
 *   for update k+1 (k = 0..), i.e. the scalars that formed p_{k+1};
 *   hist_x[k*n] = x_{k+1}, hist_p[k*n] = p_{k+1}, hist_y[k*n] = y_{k+1} = A^T r_k,
 *   hist_r[k*m] = r_k (residual before update k+1; hist_cap+1 rows).
 */
int plss_oracle_residual(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                         const double *val_in, const double *b, const double *x0, const double *w,
                         double tol, int64_t maxit, int prec, int64_t refine, double inner_tol,
                         int stop_on_true, int plant, int replace, double *x_out, int64_t *iters_out,
                         double *relres_rec,
                         double *relres_true, int64_t hist_cap, double *hist_s, double *hist_x,
                         double *hist_p, double *hist_y, double *hist_r)
{
    const int f32 = (prec == 1);
    int64_t nnz = row_ptr[m];
    double *val = (double *)malloc((size_t)(nnz ? nnz : 1) * sizeof(double));
    double *r = (double *)malloc((size_t)(m ? m : 1) * sizeof(double));
    double *rt = (double *)malloc((size_t)(m ? m : 1) * sizeof(double));
    double *y = (double *)malloc((size_t)(n ? n : 1) * sizeof(double));
    double *u = (double *)malloc((size_t)(n ? n : 1) * sizeof(double));
    double *p = (double *)calloc((size_t)(n ? n : 1), sizeof(double));
    double *x = x_out;
    int64_t *cp = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t *ri = (int64_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(int64_t));
    double *cv = (double *)malloc((size_t)(nnz ? nnz : 1) * sizeof(double));
    int status = ORC_NOT_CONVERGED;
    if (!val || !r || !rt || !y || !u || !p || !cp || !ri || !cv) { status = ORC_NOMEM; goto done; }

    for (int64_t k = 0; k < nnz; ++k) val[k] = rf(val_in[k], f32);
    csr_to_csc(m, n, row_ptr, col_idx, val, cp, ri, cv);
    for (int64_t j = 0; j < n; ++j) x[j] = x0 ? x0[j] : 0.0;

    double nb = sqrt(dot(m, b, b));
    double rho = 0.0, phi = 0.0, theta = 0.0, beta = 0.0, gamma = 0.0;
    double rho_start = 0.0;   /* rho at the last (re)start */
    int64_t k = 0;          /* updates applied */
    int64_t since = 0;      /* updates since the last (re)start */
    int restart = 1;        /* next update is the initial one (p = (rho/phi) u) */
    int fresh = 0;          /* r was just recomputed as b - A x (replace = 1) */

    /* r_0 = b - A x_0 (Algorithm 1, initialization) */
    true_residual(m, row_ptr, col_idx, val, b, x, rt);
    for (int64_t i = 0; i < m; ++i) r[i] = rf(rt[i], f32);
    rho = dot(m, r, r);
    if (nb == 0.0) { status = ORC_CONVERGED; goto done; }

    for (;;) {
        if (restart || fresh) rho_start = rho;
        if (hist_r && k <= hist_cap) memcpy(hist_r + k * m, r, (size_t)m * sizeof(double));
        /* stopping rule (Sec. 5): sqrt(rho)/||b|| <= tol */
        if (sqrt(rho) / nb <= tol) {
            if (!stop_on_true || restart || fresh) { status = ORC_CONVERGED; break; }
            /* confirm on b - A x before stopping */
            true_residual(m, row_ptr, col_idx, val, b, x, rt);
            for (int64_t i = 0; i < m; ++i) r[i] = rf(rt[i], f32);
            rho = dot(m, r, r);
            if (replace) fresh = 1; else restart = 1;
            since = 0;
            continue;
        }
        if (k >= maxit) { status = ORC_NOT_CONVERGED; break; }
        if (!restart && inner_tol > 0.0 &&
            (rho <= (plant == 3 ? inner_tol : inner_tol * inner_tol) * rho_start ||
             rho > (plant == 2 ? 2.0 : 4.0) * rho_start)) {
            /* inner solve done (residual reduced by inner_tol since the last
             * start), or the float recursion has drifted above twice its
             * starting residual: refine from b - A x */
            true_residual(m, row_ptr, col_idx, val, b, x, rt);
            for (int64_t i = 0; i < m; ++i) r[i] = rf(rt[i], f32);
            rho = dot(m, r, r);
            if (replace) fresh = 1; else restart = 1;
            since = 0;
            continue;
        }

        /* y = A^T r (column sweep), u = W y, phi = y^T u */
        if (!f32) {
            csc_spmv(n, cp, ri, cv, r, y);
        } else {
            for (int64_t j = 0; j < n; ++j) {
                float s = 0.0f;
                for (int64_t q = cp[j]; q < cp[j + 1]; ++q)
                    s = s + (float)cv[q] * (float)r[ri[q]];
                y[j] = (double)s;
            }
        }
        PAR_FOR
        for (int64_t j = 0; j < n; ++j) u[j] = rf(w ? w[j] * y[j] : y[j], f32);
        phi = 0.0;
        PAR_SUM(phi)
        for (int64_t j = 0; j < n; ++j) phi += y[j] * u[j];

        if (restart) {
            /* initial update p = (rho/phi) W y */
            if (!(phi > 0.0) || !isfinite(phi)) { status = ORC_BREAKDOWN; break; }
            beta = 0.0;
            gamma = rho / phi;
            for (int64_t j = 0; j < n; ++j) p[j] = rf(gamma * u[j], f32);
        } else {
            /* Theorem 4.1 / Algorithm 1 scalars */
            double s = sqrt(theta * phi);
            double q = s / rho;
            double d = (q - 1.0) * (q + 1.0);
            if (!(d > 0.0) || !isfinite(d)) {
                if (!stop_on_true) { status = ORC_BREAKDOWN; break; }
                /* verifying on b - A x: restart from it instead */
                true_residual(m, row_ptr, col_idx, val, b, x, rt);
                for (int64_t i = 0; i < m; ++i) r[i] = rf(rt[i], f32);
                rho = dot(m, r, r);
                restart = 1; since = 0;
                continue;
            }
            beta = 1.0 / d;
            if (plant == 1)
                gamma = theta / (theta * phi - rho * rho);   /* statement form */
            else
                gamma = (theta / rho) * beta;                /* Algorithm 1 */
            PAR_FOR
            for (int64_t j = 0; j < n; ++j) p[j] = rf(beta * p[j] + gamma * u[j], f32);
        }
        /* theta = p^T W^{-1} p; x = x + p */
        theta = 0.0;
        PAR_SUM(theta)
        for (int64_t j = 0; j < n; ++j) theta += w ? (p[j] * p[j]) / w[j] : p[j] * p[j];
        PAR_FOR
        for (int64_t j = 0; j < n; ++j) x[j] += p[j];
        if (hist_s && k < hist_cap) {
            double *h = hist_s + k * 5;
            h[0] = rho; h[1] = phi; h[2] = beta; h[3] = gamma; h[4] = theta;
        }
        if (hist_x && k < hist_cap) memcpy(hist_x + k * n, x, (size_t)n * sizeof(double));
        if (hist_p && k < hist_cap) memcpy(hist_p + k * n, p, (size_t)n * sizeof(double));
        if (hist_y && k < hist_cap) memcpy(hist_y + k * n, y, (size_t)n * sizeof(double));
        k += 1;
        since += 1;
        restart = 0;
        fresh = 0;

        if ((f32 || replace) && refine > 0 && since >= refine) {
            /* FP64 refinement: recompute the residual, then restart from it
             * or let it replace the recursive one */
            true_residual(m, row_ptr, col_idx, val, b, x, rt);
            for (int64_t i = 0; i < m; ++i) r[i] = rf(rt[i], f32);
            if (replace) fresh = 1; else restart = 1;
            since = 0;
        } else if (!f32) {
            /* r = r - A p */
            PAR_FOR
            for (int64_t i = 0; i < m; ++i) {
                double s = 0.0;
                for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q)
                    s += val[q] * p[col_idx[q]];
                r[i] = r[i] - s;
            }
        } else {
            for (int64_t i = 0; i < m; ++i) {
                float s = 0.0f;
                for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q)
                    s = s + (float)val[q] * (float)p[col_idx[q]];
                r[i] = (double)((float)r[i] - s);
            }
        }
        rho = dot(m, r, r);
    }

done:
    if (status != ORC_NOMEM) {
        *iters_out = k;
        *relres_rec = nb > 0.0 ? sqrt(rho) / nb : 0.0;
        true_residual(m, row_ptr, col_idx, val, b, x, rt);
        *relres_true = nb > 0.0 ? sqrt(dot(m, rt, rt)) / nb : 0.0;
    }
    free(val); free(r); free(rt); free(y); free(u); free(p); free(cp); free(ri); free(cv);
    return status;
}

/* ------------------------------------------------------------------ */
/* Identity sketch: PLSS Kaczmarz (Sec. 7)                             */
/* ------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood, 2014): state advances by the golden
 * gamma 0x9e3779b97f4a7c15 and the output is the state passed through the
 * variant-13 mixing function. */
static uint64_t splitmix_next(uint64_t *s)
{
    uint64_t z = (*s += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Fills perm with 0..m-1 then shuffles it (Durstenfeld's Fisher-Yates:
 * for i = m-1 down to 1, swap perm[i] with perm[next() mod (i+1)]). */
void plss_oracle_permutation(uint64_t *state, int64_t m, int32_t *perm)
{
    for (int64_t i = 0; i < m; ++i) perm[i] = (int32_t)i;
    for (int64_t i = m - 1; i > 0; --i) {
        uint64_t j = splitmix_next(state) % (uint64_t)(i + 1);
        int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/*
 * PLSS Kaczmarz (eq:pkKacz): for row i = i_k,
 *   r_i = b_i - a_i^T x;  c_j = q_j^T a_i (j in the history);
 *   ||d||^2 = sum_j c_j^2 / theta_j;
 *   gamma = r_i / ((||a_i|| - ||d||)(||a_i|| + ||d||));
 *   q = a_i - sum_j (c_j/theta_j) q_j;  p = gamma q;  x = x + p;
 *   append q and theta = ||q||^2 to the history.
 * The history holds the directions q_j = p_j / gamma_j: P Theta^{-1} P^T is
 * the same projector for any column scaling, so this is eq:pkKacz, and a
 * row with r_i = 0 (p = 0) still enters the window with its direction.
 * With K = 0 (no history) this is the classical Kaczmarz step.
 * maxit caps the rows visited; after every full pass over the rows the
 * residual ||b - A x||/||b|| is tested against tol. `plant` != 0 plants a
 * wrong window reset (see the file header).
 * Outputs: x_out, *iters (rows visited), *n_skipped, *relres_true; returns status.
 */
int plss_oracle_kaczmarz(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                         const double *val, const double *b, const double *x0, double tol,
                         int64_t maxit, int64_t K, uint64_t seed, int plant, double *x_out,
                         int64_t *iters_out, int64_t *n_skipped, double *relres_true)
{
    double *x = x_out;
    /* window capacity: K, or the planted wrong one */
    int64_t cap = K;
    if (K > 0 && plant == 1) cap = K + 1;
    if (K > 1 && plant == 2) cap = K - 1;
    if (K > 0 && plant == 3) cap = maxit > 0 ? maxit : 1;
    double *P = (double *)malloc((size_t)((cap > 0 ? cap : 1) * (n ? n : 1)) * sizeof(double));
    double *th = (double *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(double));
    double *c = (double *)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(double));
    double *p = (double *)malloc((size_t)(n ? n : 1) * sizeof(double));
    double *rt = (double *)malloc((size_t)(m ? m : 1) * sizeof(double));
    int32_t *perm = (int32_t *)malloc((size_t)(m ? m : 1) * sizeof(int32_t));
    int status = ORC_NOT_CONVERGED;
    int64_t k = 0, nh = 0, skipped = 0;
    uint64_t state = seed;
    double nb;
    if (!P || !th || !c || !p || !rt || !perm) { status = ORC_NOMEM; goto kdone; }

    for (int64_t j = 0; j < n; ++j) x[j] = x0 ? x0[j] : 0.0;
    nb = sqrt(dot(m, b, b));
    if (nb == 0.0 || m == 0) { status = ORC_CONVERGED; goto kdone; }
    true_residual(m, row_ptr, col_idx, val, b, x, rt);
    if (sqrt(dot(m, rt, rt)) / nb <= tol) { status = ORC_CONVERGED; goto kdone; }

    while (k < maxit) {
        plss_oracle_permutation(&state, m, perm);
        for (int64_t t = 0; t < m && k < maxit; ++t, ++k) {
            int64_t i = perm[t];
            int64_t s0 = row_ptr[i], s1 = row_ptr[i + 1];
            if (cap > 0 && nh == cap) nh = 0;   /* window full: restart it empty */
            /* r_i = b_i - a_i^T x */
            double ax = 0.0, a2 = 0.0;
            for (int64_t q = s0; q < s1; ++q) ax += val[q] * x[col_idx[q]];
            for (int64_t q = s0; q < s1; ++q) a2 += val[q] * val[q];
            double r_i = b[i] - ax;
            /* c = P^T a_i, ||d||^2 = sum c_j^2 / theta_j */
            double d2 = 0.0;
            for (int64_t j = 0; j < nh; ++j) {
                double s = 0.0;
                for (int64_t q = s0; q < s1; ++q) s += val[q] * P[j * n + col_idx[q]];
                c[j] = s;
                d2 += (s * s) / th[j];
            }
            double na = sqrt(a2), nd = sqrt(d2);
            double delta = (na - nd) * (na + nd);
            if (!(delta > 1e-14 * a2)) { skipped += 1; continue; }
            double gamma = r_i / delta;
            /* q = a_i - sum_j (c_j/theta_j) q_j, p = gamma q, x = x + p */
            for (int64_t jj = 0; jj < n; ++jj) p[jj] = 0.0;
            for (int64_t q = s0; q < s1; ++q) p[col_idx[q]] = val[q];
            for (int64_t j = 0; j < nh; ++j) {
                double cj = c[j] / th[j];
                for (int64_t jj = 0; jj < n; ++jj) p[jj] -= cj * P[j * n + jj];
            }
            double thn = 0.0;
            for (int64_t jj = 0; jj < n; ++jj) {
                thn += p[jj] * p[jj];
                x[jj] += gamma * p[jj];
            }
            if (cap > 0 && thn > 0.0) {
                memcpy(P + nh * n, p, (size_t)n * sizeof(double));
                th[nh] = thn;
                nh += 1;
            }
        }
        /* test after each full pass */
        true_residual(m, row_ptr, col_idx, val, b, x, rt);
        if (sqrt(dot(m, rt, rt)) / nb <= tol) { status = ORC_CONVERGED; break; }
    }

kdone:
    if (status != ORC_NOMEM) {
        *iters_out = k;
        *n_skipped = skipped;
        nb = sqrt(dot(m, b, b));
        true_residual(m, row_ptr, col_idx, val, b, x, rt);
        *relres_true = nb > 0.0 ? sqrt(dot(m, rt, rt)) / nb : 0.0;
    }
    free(P); free(th); free(c); free(p); free(rt); free(perm);
    return status;
}

/* ------------------------------------------------------------------ */
/* General sketch: Theorem 2.1 / Corollary 2.2 (Sec. 2.4)              */
/* ------------------------------------------------------------------ */

/* Output number j (0-based) of the SplitMix64 stream seeded with `seed`:
 * the state after j + 1 increments by the golden gamma, mixed. */
static uint64_t splitmix_at(uint64_t seed, uint64_t j)
{
    uint64_t z = seed + (j + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Entry i of sketch column k (0-based, counting every column drawn). */
double plss_oracle_sketch_entry(uint64_t seed, int64_t m, int64_t k, int64_t i)
{
    return (splitmix_at(seed, (uint64_t)k * (uint64_t)m + (uint64_t)i) >> 63) ? -1.0 : 1.0;
}

/*
 * PLSS with a general sketch S_k = [s_1 ... s_k] (eq:genS), one random
 * sign column appended per step, computed as Sec. 2.4 does:
 *   y_k = A^T s_k (eq:yk), Y_k = [Y_{k-1} y_k];
 *   t_k = N_{k-1} Y_{k-1}^T y_k,  delta_k = y_k^T y_k - y_k^T Y_{k-1} t_k;
 *   p_k = (s_k^T r_{k-1} / delta_k) (y_k - Y_{k-1} t_k)   (Corollary 2.2);
 *   N_k = [[N_{k-1} + t t^T/delta, -t/delta], [-t^T/delta, 1/delta]]
 *                                                      (Theorem 2.1, eq:Nkrec);
 * with N_1 = 1/(y_1^T y_1) and r_k = b - A x_k formed from its definition
 * (Sec. 1: x_k = x_{k-1} + p_k). The history holds at most K columns
 * (the memory of Sec. 2.3-2.4 grows with k); a full history is emptied
 * before the next column, which then starts a new N. A column whose delta
 * is <= 1e-14 y^T y (y in the span of the history, or y = 0) is skipped
 * and not appended (its column index is still used up). maxit caps the
 * columns drawn; after each step ||r||/||b|| <= tol stops.
 * Outputs: x_out[n], *iters (columns drawn), *n_skipped, *relres_true;
 * hist_x[k*n] = x after column k (k < hist_cap) when hist_x != NULL.
 */
int plss_oracle_general(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                        const double *val, const double *b, const double *x0, double tol,
                        int64_t maxit, int64_t K, uint64_t seed, int plant, double *x_out,
                        int64_t *iters_out, int64_t *n_skipped, double *relres_true,
                        int64_t hist_cap, double *hist_x)
{
    int64_t Kc = K > 0 ? K : 1;
    double *x = x_out;
    double *Y = (double *)malloc((size_t)(Kc * (n ? n : 1)) * sizeof(double));  /* column j at Y + j*n */
    double *N = (double *)malloc((size_t)(Kc * Kc) * sizeof(double));          /* N[a*Kc + c] */
    double *N2 = (double *)malloc((size_t)(Kc * Kc) * sizeof(double));
    double *Yty = (double *)malloc((size_t)Kc * sizeof(double));
    double *t = (double *)malloc((size_t)Kc * sizeof(double));
    double *y = (double *)malloc((size_t)(n ? n : 1) * sizeof(double));
    double *p = (double *)malloc((size_t)(n ? n : 1) * sizeof(double));
    double *r = (double *)malloc((size_t)(m ? m : 1) * sizeof(double));
    int status = ORC_NOT_CONVERGED;
    int64_t k = 0, nh = 0, skipped = 0;
    double nb;
    if (!Y || !N || !N2 || !Yty || !t || !y || !p || !r) { status = ORC_NOMEM; goto gdone; }

    for (int64_t j = 0; j < n; ++j) x[j] = x0 ? x0[j] : 0.0;
    nb = sqrt(dot(m, b, b));
    true_residual(m, row_ptr, col_idx, val, b, x, r);
    if (nb == 0.0 || sqrt(dot(m, r, r)) / nb <= tol) { status = ORC_CONVERGED; goto gdone; }

    for (k = 0; k < maxit; ) {
        if (K > 0 && nh == K) nh = 0;          /* history full: start a new one */
        /* y = A^T s_k, rho = s_k^T r_{k-1} */
        double rho = 0.0;
        for (int64_t j = 0; j < n; ++j) y[j] = 0.0;
        for (int64_t i = 0; i < m; ++i) {
            double si = plss_oracle_sketch_entry(seed, m, k, i);
            rho += si * r[i];
            for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) y[col_idx[q]] += si * val[q];
        }
        double yy = dot(n, y, y);
        /* Y^T y, t = N Y^T y, delta */
        for (int64_t a = 0; a < nh; ++a) Yty[a] = dot(n, Y + a * n, y);
        for (int64_t a = 0; a < nh; ++a) {
            double sacc = 0.0;
            for (int64_t c = 0; c < nh; ++c) sacc += N[a * Kc + c] * Yty[c];
            t[a] = sacc;
        }
        double delta = yy;
        for (int64_t a = 0; a < nh; ++a) delta -= Yty[a] * t[a];
        k += 1;
        if (!(delta > 1e-14 * yy)) {
            skipped += 1;
        } else {
            /* p = (rho/delta) (y - Y t) */
            for (int64_t j = 0; j < n; ++j) {
                double v = y[j];
                for (int64_t a = 0; a < nh; ++a) v -= Y[a * n + j] * t[a];
                p[j] = (rho / delta) * v;
            }
            for (int64_t j = 0; j < n; ++j) x[j] += p[j];
            if (K > 0) {
                /* N_k from N_{k-1} (eq:Nkrec), Y_k = [Y_{k-1} y] */
                for (int64_t a = 0; a < nh; ++a)
                    for (int64_t c = 0; c < nh; ++c)
                        N2[a * Kc + c] = plant == 1 ? N[a * Kc + c]
                                                    : N[a * Kc + c] + (t[a] * t[c]) / delta;
                for (int64_t a = 0; a < nh; ++a) {
                    N2[a * Kc + nh] = -t[a] / delta;
                    N2[nh * Kc + a] = -t[a] / delta;
                }
                N2[nh * Kc + nh] = 1.0 / delta;
                for (int64_t a = 0; a <= nh; ++a)
                    for (int64_t c = 0; c <= nh; ++c) N[a * Kc + c] = N2[a * Kc + c];
                memcpy(Y + nh * n, y, (size_t)n * sizeof(double));
                nh += 1;
            }
        }
        if (hist_x && k - 1 < hist_cap) memcpy(hist_x + (k - 1) * n, x, (size_t)n * sizeof(double));
        true_residual(m, row_ptr, col_idx, val, b, x, r);
        if (sqrt(dot(m, r, r)) / nb <= tol) { status = ORC_CONVERGED; break; }
    }

gdone:
    if (status != ORC_NOMEM) {
        *iters_out = k;
        *n_skipped = skipped;
        nb = sqrt(dot(m, b, b));
        true_residual(m, row_ptr, col_idx, val, b, x, r);
        *relres_true = nb > 0.0 ? sqrt(dot(m, r, r)) / nb : 0.0;
    }
    free(Y); free(N); free(N2); free(Yty); free(t); free(y); free(p); free(r);
    return status;
}
