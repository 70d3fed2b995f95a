/*
 * FP64 CPU oracle for sparse CP tensor completion (arXiv:1910.02371).
 * TEST INFRASTRUCTURE ONLY -- see oracle.h.  Compiled with -O2
 * -ffp-contract=off so that every product and sum is rounded as written.
 *
 * The same source is compiled twice: without OpenMP (liboracle.so, the parity
 * checker) and with -fopenmp (liboracle_omp.so, the timed CPU baseline).  The
 * OpenMP pragmas only split independent loops -- nonzeros for TTTP and the
 * per-nonzero model terms, rows of the mode-sorted segments for MTTKRP and
 * Solve Factor -- and every sum keeps its order (each row sums its nonzeros in
 * input order; the objective's sum over nonzeros stays serial), so both
 * builds give bit-identical results.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Number of threads the OpenMP build uses (1 without OpenMP). */
int orc_threads(int set)
{
#ifdef _OPENMP
    if (set > 0) omp_set_num_threads(set);
    return omp_get_max_threads();
#else
    (void)set;
    return 1;
#endif
}

static int check_common(int N, const int64_t *dims, int64_t m, const int32_t *const *idx, int R)
{
    if (N < 1 || N > ORC_MAX_ORDER || m < 0 || R < 1 || !dims || (m > 0 && !idx))
        return ORC_ERR_ARG;
    for (int n = 0; n < N; ++n) {
        if (dims[n] < 1) return ORC_ERR_ARG;
        if (m > 0 && !idx[n]) return ORC_ERR_ARG;
        for (int64_t e = 0; e < m; ++e)
            if (idx[n][e] < 0 || (int64_t)idx[n][e] >= dims[n]) return ORC_ERR_RANGE;
    }
    return ORC_OK;
}

/* Sec. 3.4: counting sort keyed by the mode index (stable). */
int orc_counting_sort(int64_t m, const int32_t *key, int64_t I, int64_t *perm, int64_t *row_ptr)
{
    if (m < 0 || I < 1 || !row_ptr || (m > 0 && (!key || !perm))) return ORC_ERR_ARG;
    for (int64_t i = 0; i <= I; ++i) row_ptr[i] = 0;
    for (int64_t e = 0; e < m; ++e) {
        if (key[e] < 0 || (int64_t)key[e] >= I) return ORC_ERR_RANGE;
        row_ptr[(int64_t)key[e] + 1] += 1;                 /* histogram */
    }
    for (int64_t i = 0; i < I; ++i) row_ptr[i + 1] += row_ptr[i];   /* prefix sums */
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(I > 0 ? I : 1));
    if (!next) return ORC_ERR_ARG;
    for (int64_t i = 0; i < I; ++i) next[i] = row_ptr[i];
    for (int64_t e = 0; e < m; ++e) perm[next[key[e]]++] = e;   /* input order within a key */
    free(next);
    return ORC_OK;
}

/* Sec. 3.3, TTTP: x_e = s_e sum_r prod_{j provided} a^(j)_{i_j r}. */
int orc_tttp(int N, const int64_t *dims, int64_t m, const int32_t *const *idx,
             const double *s, int R, const double *const *A, double *x)
{
    int rc = check_common(N, dims, m, idx, R);
    if (rc) return rc;
    int provided = 0;
    for (int n = 0; n < N; ++n) provided += (A && A[n]) ? 1 : 0;
    if (!provided || (m > 0 && !x)) return ORC_ERR_ARG;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        double acc = 0.0;
        for (int r = 0; r < R; ++r) {
            double p = 1.0;
            for (int n = 0; n < N; ++n)
                if (A[n]) p = p * A[n][(int64_t)idx[n][e] * R + r];
            acc = acc + p;
        }
        x[e] = (s ? s[e] : 1.0) * acc;
    }
    return ORC_OK;
}

/* Sec. 3.2 / Appendix A: out[i,r] = sum_{e: i_mode=i} s_e prod_{n!=mode} a^(n)_{i_n r}. */
int orc_mttkrp(int N, const int64_t *dims, int64_t m, const int32_t *const *idx,
               const double *s, int R, const double *const *A, int mode, double *out)
{
    int rc = check_common(N, dims, m, idx, R);
    if (rc) return rc;
    if (mode < 0 || mode >= N || !out || !A) return ORC_ERR_ARG;
    for (int n = 0; n < N; ++n)
        if (n != mode && !A[n]) return ORC_ERR_ARG;
    const int64_t I = dims[mode];
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int64_t *row_ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(I + 1));
    if (!perm || !row_ptr) { free(perm); free(row_ptr); return ORC_ERR_ARG; }
    /* the rows' nonzeros in input order (the counting sort is stable), so
     * each out[i, r] sums its terms in input order */
    orc_counting_sort(m, m > 0 ? idx[mode] : NULL, I, perm, row_ptr);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < I; ++i) {
        double *o = out + i * R;
        for (int r = 0; r < R; ++r) o[r] = 0.0;
        for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
            const int64_t e = perm[q];
            double se = s ? s[e] : 1.0;
            for (int r = 0; r < R; ++r) {
                double p = se;
                for (int n = 0; n < N; ++n)
                    if (n != mode) p = p * A[n][(int64_t)idx[n][e] * R + r];
                o[r] = o[r] + p;
            }
        }
    }
    free(perm);
    free(row_ptr);
    return ORC_OK;
}

/* Textbook unpivoted Cholesky of the R x R matrix S (row-major, lower part
 * used) into L.  Returns 0 if a pivot is <= 0. */
static int cholesky(int R, const double *S, double *L)
{
    for (int q = 0; q < R * R; ++q) L[q] = 0.0;
    for (int j = 0; j < R; ++j) {
        double d = S[j * R + j];
        for (int k = 0; k < j; ++k) d = d - L[j * R + k] * L[j * R + k];
        if (!(d > 0.0)) return 0;
        double ljj = sqrt(d);
        L[j * R + j] = ljj;
        for (int i = j + 1; i < R; ++i) {
            double v = S[i * R + j];
            for (int k = 0; k < j; ++k) v = v - L[i * R + k] * L[j * R + k];
            L[i * R + j] = v / ljj;
        }
    }
    return 1;
}

/* Solve L L^T y = b in place (forward then backward substitution). */
static void chol_solve(int R, const double *L, double *b)
{
    for (int i = 0; i < R; ++i) {
        double v = b[i];
        for (int k = 0; k < i; ++k) v = v - L[i * R + k] * b[k];
        b[i] = v / L[i * R + i];
    }
    for (int i = R - 1; i >= 0; --i) {
        double v = b[i];
        for (int k = i + 1; k < R; ++k) v = v - L[k * R + i] * b[k];
        b[i] = v / L[i * R + i];
    }
}

/* Sec. 3.4 (Solve Factor) with the normal equations of Sec. 2.2. */
int orc_solve_factor(int N, const int64_t *dims, int64_t m, const int32_t *const *idx,
                     const double *s, int R, const double *const *A, int mode,
                     const double *rhs, double lambda, double *out, int8_t *status)
{
    int rc = check_common(N, dims, m, idx, R);
    if (rc) return rc;
    if (mode < 0 || mode >= N || !out || !rhs || !A) return ORC_ERR_ARG;
    for (int n = 0; n < N; ++n)
        if (n != mode && !A[n]) return ORC_ERR_ARG;
    const int64_t I = dims[mode];
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    int64_t *row_ptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(I + 1));
    if (!perm || !row_ptr) { free(perm); free(row_ptr); return ORC_ERR_ARG; }
    orc_counting_sort(m, m > 0 ? idx[mode] : NULL, I, perm, row_ptr);
    int bad = 0, oom = 0;
#pragma omp parallel reduction(| : bad, oom)
    {
        double *G = (double *)malloc(sizeof(double) * (size_t)R * R);
        double *L = (double *)malloc(sizeof(double) * (size_t)R * R);
        double *h = (double *)malloc(sizeof(double) * (size_t)R);
        double *a = (double *)malloc(sizeof(double) * (size_t)R);
        double *d = (double *)malloc(sizeof(double) * (size_t)R);
        const int ok = G && L && h && a && d;
        if (!ok) oom = 1;
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < I; ++i) {
            if (!ok) continue;
            /* G_i = sum_{e in row i} s_e h_e h_e^T, then + lambda I */
            for (int q = 0; q < R * R; ++q) G[q] = 0.0;
            for (int64_t q = row_ptr[i]; q < row_ptr[i + 1]; ++q) {
                int64_t e = perm[q];
                double se = s ? s[e] : 1.0;
                for (int r = 0; r < R; ++r) {
                    double p = 1.0;
                    for (int n = 0; n < N; ++n)
                        if (n != mode) p = p * A[n][(int64_t)idx[n][e] * R + r];
                    h[r] = p;
                }
                for (int r = 0; r < R; ++r)
                    for (int c = 0; c < R; ++c) G[r * R + c] = G[r * R + c] + se * h[r] * h[c];
            }
            for (int r = 0; r < R; ++r) G[r * R + r] = G[r * R + r] + lambda;
            if (!cholesky(R, G, L)) {
                bad = 1;
                if (status) status[i] = 1;
                continue;
            }
            if (status) status[i] = 0;
            for (int r = 0; r < R; ++r) a[r] = rhs[i * R + r];
            chol_solve(R, L, a);
            /* one refinement step: d = rhs - (G + lambda I) a in long double */
            for (int r = 0; r < R; ++r) {
                long double v = (long double)rhs[i * R + r];
                for (int c = 0; c < R; ++c) v -= (long double)G[r * R + c] * (long double)a[c];
                d[r] = (double)v;
            }
            chol_solve(R, L, d);
            for (int r = 0; r < R; ++r) out[i * R + r] = a[r] + d[r];
        }
        free(G); free(L); free(h); free(a); free(d);
    }
    free(perm); free(row_ptr);
    if (oom) return ORC_ERR_ARG;
    return bad ? ORC_ERR_NOT_SPD : ORC_OK;
}

/* Sec. 2.1 and Table 1: phi, phi' = d phi / d m, phi'' for each loss.
 *   least squares      phi = (t - m)^2        phi' = 2 (m - t)   phi'' = 2
 *   Poisson, log link  phi = exp(m) - t m     phi' = exp(m) - t  phi'' = exp(m)   (Sec. 5.7)
 *   Poisson, identity  phi = m - t log m      phi' = 1 - t / m   phi'' = t / m^2  (m > 0) */
int orc_loss_terms(int loss, int64_t m, const double *t, const double *model,
                   double *phi, double *d1, double *d2)
{
    if (m < 0 || (m > 0 && (!t || !model))) return ORC_ERR_ARG;
    if (loss < ORC_LOSS_LS || loss > ORC_LOSS_POISSON_ID) return ORC_ERR_ARG;
    int dom = 0;
#pragma omp parallel for schedule(static) reduction(| : dom)
    for (int64_t e = 0; e < m; ++e) {
        double te = t[e], me = model[e], p, g, hh;
        if (loss == ORC_LOSS_LS) {
            double r = te - me;
            p = r * r;
            g = 2.0 * (me - te);
            hh = 2.0;
        } else if (loss == ORC_LOSS_POISSON_LOG) {
            double ex = exp(me);
            p = ex - te * me;
            g = ex - te;
            hh = ex;
        } else {
            if (!(me > 0.0)) {
                dom = 1;
                continue;
            }
            p = me - te * log(me);
            g = 1.0 - te / me;
            hh = te / (me * me);
        }
        if (phi) phi[e] = p;
        if (d1) d1[e] = g;
        if (d2) d2[e] = hh;
    }
    return dom ? ORC_ERR_DOMAIN : ORC_OK;
}

static double frob2(int64_t rows, int R, const double *a)
{
    double v = 0.0;
    for (int64_t q = 0; q < rows * R; ++q) v = v + a[q] * a[q];
    return v;
}

/* eq. obj and Table 1 (general loss column); Appendix A for order N. */
int orc_loss_grad(int N, const int64_t *dims, int64_t m, const int32_t *const *idx,
                  const double *t, int R, const double *const *A, int loss,
                  double lambda, double *f, double *const *grad)
{
    int rc = check_common(N, dims, m, idx, R);
    if (rc) return rc;
    if (!A || (m > 0 && !t)) return ORC_ERR_ARG;
    for (int n = 0; n < N; ++n)
        if (!A[n]) return ORC_ERR_ARG;
    double *model = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *phi = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *d1 = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    if (!model || !phi || !d1) { free(model); free(phi); free(d1); return ORC_ERR_ARG; }
    rc = orc_tttp(N, dims, m, idx, NULL, R, A, model);
    if (!rc) rc = orc_loss_terms(loss, m, t, model, phi, d1, NULL);
    if (!rc && f) {
        double v = 0.0;
        for (int64_t e = 0; e < m; ++e) v = v + phi[e];
        double reg = 0.0;
        for (int n = 0; n < N; ++n) reg = reg + frob2(dims[n], R, A[n]);
        *f = v + lambda * reg;
    }
    for (int d = 0; !rc && grad && d < N; ++d) {
        if (!grad[d]) continue;
        rc = orc_mttkrp(N, dims, m, idx, d1, R, A, d, grad[d]);
        for (int64_t q = 0; !rc && q < dims[d] * R; ++q)
            grad[d][q] = grad[d][q] + 2.0 * lambda * A[d][q];
    }
    free(model); free(phi); free(d1);
    return rc;
}

/* Sec. 2.5 (Gauss-Newton: the phi' off-diagonal terms of the Hessian dropped)
 * and Appendix A; the 2 lambda I term is the Hessian of the regularizer. */
int orc_ggn_matvec(int N, const int64_t *dims, int64_t m, const int32_t *const *idx,
                   const double *t, int R, const double *const *A, int loss,
                   double lambda, const double *const *x, double *const *y)
{
    int rc = check_common(N, dims, m, idx, R);
    if (rc) return rc;
    if (!A || !x || !y || (m > 0 && !t)) return ORC_ERR_ARG;
    for (int n = 0; n < N; ++n)
        if (!A[n] || !x[n] || !y[n]) return ORC_ERR_ARG;
    double *model = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *d2 = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *w = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    if (!model || !d2 || !w) { free(model); free(d2); free(w); return ORC_ERR_ARG; }
    rc = orc_tttp(N, dims, m, idx, NULL, R, A, model);
    if (!rc) rc = orc_loss_terms(loss, m, t, model, NULL, NULL, d2);
#pragma omp parallel for schedule(static) if (!rc)
    for (int64_t e = 0; e < m; ++e) {
        if (rc) continue;
        /* z_e = sum_p sum_r x^(p)_{i_p r} prod_{n != p} a^(n)_{i_n r} */
        double z = 0.0;
        for (int p = 0; p < N; ++p)
            for (int r = 0; r < R; ++r) {
                double v = x[p][(int64_t)idx[p][e] * R + r];
                for (int n = 0; n < N; ++n)
                    if (n != p) v = v * A[n][(int64_t)idx[n][e] * R + r];
                z = z + v;
            }
        w[e] = d2[e] * z;
    }
    for (int d = 0; !rc && d < N; ++d) {
        rc = orc_mttkrp(N, dims, m, idx, w, R, A, d, y[d]);
        for (int64_t q = 0; !rc && q < dims[d] * R; ++q)
            y[d][q] = y[d][q] + 2.0 * lambda * x[d][q];
    }
    free(model); free(d2); free(w);
    return rc;
}
