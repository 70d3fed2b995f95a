/*
 * FP64 CPU oracle for sparse CP tensor completion (arXiv:1910.02371).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA library; the two only see the
 * same seeded inputs.
 *
 * Every routine is the plain definition from the paper written out as loops in
 * double precision, in a fixed order (input order of the nonzeros, then r
 * ascending), with no blocking or fusion.  Sparse tensors are coordinate lists:
 * N int32 index arrays idx[n][e] and an optional value array s[e].  Factor
 * matrices are row-major I_n x R double arrays.
 *
 * Return codes: 0 ok, 1 bad argument, 2 index out of range, 6 a row system was
 * not positive definite, 7 loss outside its domain.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_ORDER 8

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_RANGE = 2, ORC_ERR_NOT_SPD = 6,
       ORC_ERR_DOMAIN = 7 };
enum { ORC_LOSS_LS = 0, ORC_LOSS_POISSON_LOG = 1, ORC_LOSS_POISSON_ID = 2 };

/* Threads of the OpenMP build of this file (liboracle_omp.so): sets the count
 * if set > 0, returns the count in use; the plain build returns 1.  Both
 * builds give bit-identical results (see oracle.c). */
int orc_threads(int set);

/* Counting sort of the nonzeros by key (Sec. 3.4, Solve Factor: the local data
 * is sorted by the mode-n index with a counting sort).  perm[q] = input position
 * of the q-th nonzero in sorted order; equal keys keep input order.
 * row_ptr[i] = first sorted position with key i, row_ptr[I] = m. */
int orc_counting_sort(int64_t m, const int32_t *key, int64_t I, int64_t *perm,
                      int64_t *row_ptr);

/* TTTP (Sec. 3.3): x_e = s_e * sum_r prod_{n provided} A^(n)[i_n(e), r].
 * s == NULL means s_e = 1; A[n] == NULL skips mode n.  At least one factor. */
int orc_tttp(int N, const int64_t *dims, int64_t m, const int32_t *const *idx,
             const double *s, int R, const double *const *A, double *x);

/* MTTKRP restricted to the observed entries (Sec. 3.2; Appendix A gradient):
 * out[i, r] = sum_{e : i_mode(e) = i} s_e prod_{n != mode} A^(n)[i_n(e), r].
 * out is I_mode x R and is overwritten. */
int orc_mttkrp(int N, const int64_t *dims, int64_t m, const int32_t *const *idx,
               const double *s, int R, const double *const *A, int mode, double *out);

/* Solve Factor (Sec. 3.4 with Sec. 2.2): for every row i of mode `mode`,
 * G_i = sum_{e in row i} s_e h_e h_e^T with h_e = hadamard_{n != mode} A^(n)[i_n(e)],
 * then (G_i + lambda I) a_i = rhs_i by unpivoted Cholesky, followed by one step
 * of iterative refinement with the residual in long double.  A row whose
 * system has a pivot <= 0 is not written and gets status[i] = 1 (status may be
 * NULL); the call then returns ORC_ERR_NOT_SPD. */
int orc_solve_factor(int N, const int64_t *dims, int64_t m, const int32_t *const *idx,
                     const double *s, int R, const double *const *A, int mode,
                     const double *rhs, double lambda, double *out, int8_t *status);

/* Elementwise loss phi(t, m) and its first and second derivatives in m
 * (Sec. 2.1 and Table 1; the log-link Poisson loss of Sec. 5.7).  Any output
 * may be NULL. */
int orc_loss_terms(int loss, int64_t m, const double *t, const double *model,
                   double *phi, double *d1, double *d2);

/* Objective and gradient (eq. obj, Table 1, Appendix A):
 * f = sum_e phi(t_e, m_e) + lambda sum_n ||A^(n)||_F^2,
 * grad^(d) = MTTKRP(phi', d) + 2 lambda A^(d).  f or any grad[d] may be NULL. */
int orc_loss_grad(int N, const int64_t *dims, int64_t m, const int32_t *const *idx,
                  const double *t, int R, const double *const *A, int loss,
                  double lambda, double *f, double *const *grad);

/* Gauss-Newton matrix-vector product (Sec. 2.5, Appendix A, phi' terms dropped):
 * z_e = sum_p <x^(p)[i_p(e)], h^(p)_e>,
 * y^(d)[k, r] = sum_{e : i_d(e) = k} phi''_e z_e h^(d)_{e r} + 2 lambda x^(d)[k, r]. */
int orc_ggn_matvec(int N, const int64_t *dims, int64_t m, const int32_t *const *idx,
                   const double *t, int R, const double *const *A, int loss,
                   double lambda, const double *const *x, double *const *y);

#ifdef __cplusplus
}
#endif
#endif
