/*
 * tc.h -- C ABI of the GB300 (sm_103a) sparse CP tensor-completion kernels.
 *
 * The operations are the multi-tensor kernels of "Parallel Algorithms for
 * Tensor Completion in the CP Format" (arXiv:1910.02371):
 *   - the per-mode sorted pattern of the observed entries   (Sec. 3.4, counting sort)
 *   - TTTP, the sampled multilinear inner product            (Sec. 3.3)
 *   - MTTKRP restricted to the observed entries              (Sec. 3.2, Appendix A)
 *   - Solve Factor, the per-row regularized normal equations (Sec. 3.4, Sec. 2.2)
 *   - the objective and its gradient for a generalized loss  (eq. obj, Table 1)
 *   - the Gauss-Newton matrix-vector product                 (Sec. 2.5, Appendix A)
 *   - the block-diagonal preconditioner and the PCG driver   (Sec. 2.5)
 * for order-3 tensors (the order the paper develops its algorithms for).
 *
 * Conventions shared by every call
 * --------------------------------
 * Pointers.  Arrays of nonzeros, factor matrices and outputs are DEVICE
 * pointers on the pattern's device; `dims`, pointer arrays (`const void *const
 * *factors` etc.) and scalars are host values.  The caller owns every buffer it
 * passes; a tc_pattern owns the sorted copies it makes and frees them in
 * tc_pattern_destroy.  No call keeps a caller pointer after it returns, except
 * that a tc_cg object keeps the ones given at its creation (see below).
 *
 * Layout.  A factor matrix A^(n) is row-major I_n x R with row stride R, in the
 * pattern's dtype (float or double).  Index arrays are int32.  Every array of
 * length nnz that crosses the ABI is in PATTERN ORDER: the nonzeros sorted by
 * their mode-0 index, equal indices kept in input order (stable).  perm of mode
 * 0 (tc_pattern_view) maps pattern order back to input order.
 *
 * Weights.  Calls that take per-nonzero weights accept
 *   TC_W_ONE    -- s_e = 1: the pattern Omega-hat itself,
 *   TC_W_VALUES -- the values given to tc_build_pattern (the tensor T),
 *   TC_W_ARRAY  -- a caller array `s` of nnz weights in pattern order.
 *
 * Streams.  Every call is asynchronous on `stream` (a cudaStream_t; NULL is the
 * legacy default stream) and records the device work in stream order.
 * Argument errors are returned at once and launch nothing.  Errors found on
 * the device (an index out of range, a system that is not positive definite,
 * a loss evaluated outside its domain, a CG breakdown) set the pattern's device
 * status word; tc_last_error synchronizes the stream and returns and clears it.
 * No kernel traps or asserts.
 *
 * Sizes.  nnz and all offsets are int64.  R (the CP rank) is 1..64.
 * nnz == 0 is legal and gives zero outputs.
 *
 * Threading.  Calls on different patterns are independent.  Calls on one
 * pattern from several host threads must be serialized by the caller.
 *
 * Work space.  Calls that need device memory beyond their outputs (Solve
 * Factor's Gram batch, cut-row slots, refinement residuals and right-hand-side
 * copy; the work arrays of tc_newton_als_mode, tc_ccd_sweep and
 * tc_ccd_newton_sweep) take it from buffers the pattern keeps: Solve Factor
 * one set per mode, the others one set each.  A buffer is allocated the first
 * time a size is needed and kept until tc_pattern_destroy, so repeated calls
 * of the same shape allocate nothing (and may then be captured in a CUDA
 * graph); a call that needs a larger buffer synchronizes the device, frees the
 * old one and allocates anew.  Because the buffers are shared, two calls on
 * one pattern that use the same mode's Solve Factor buffers (or both the
 * Newton or coordinate-descent buffers) must be ordered on the device -- one
 * stream, or events; calls on different modes may overlap.
 */
#ifndef TC_H
#define TC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *tc_stream_t; /* the same type as cudaStream_t */

typedef enum {
    TC_OK = 0,
    TC_ERR_ARG = 1,         /* bad argument: NULL pointer, size, mode, rank, dtype */
    TC_ERR_RANGE = 2,       /* an index outside [0, I_n) */
    TC_ERR_DUPLICATE = 3,   /* a coordinate occurs twice (checked on request) */
    TC_ERR_OOM = 4,         /* device allocation failed */
    TC_ERR_CUDA = 5,        /* a CUDA runtime call failed */
    TC_ERR_NOT_SPD = 6,     /* a row system had a pivot <= 0; that row was not written */
    TC_ERR_DOMAIN = 7,      /* Poisson identity-link loss at a model entry <= 0 */
    TC_ERR_BREAKDOWN = 8,   /* CG: p^T H p <= 0; later iterations left x unchanged */
    TC_ERR_UNSUPPORTED = 9, /* a valid request this build does not implement */
    TC_ERR_TIMEOUT = 10     /* a kernel's wait for its own tensor-core work passed its time
                               limit (2 s); the kernel gave up and its outputs are incomplete.
                               Not expected in normal operation. */
} tc_status;

typedef enum { TC_F32 = 0, TC_F64 = 1 } tc_dtype;

/* phi(t, m) of eq. obj: least squares (t - m)^2 (Sec. 2.1); Poisson with the
 * log link exp(m) - t m (Sec. 5.7); Poisson with the identity link
 * m - t log m, m > 0 (Sec. 2.1). */
typedef enum { TC_LOSS_LS = 0, TC_LOSS_POISSON_LOG = 1, TC_LOSS_POISSON_ID = 2 } tc_loss;

typedef enum { TC_W_ONE = 0, TC_W_VALUES = 1, TC_W_ARRAY = 2 } tc_weights;

/* Precision forms of Solve Factor.  The Cholesky factorization and the
 * triangular solves are FP64 in every form; the forms differ in how the Gram
 * G_i is summed and in whether one step of iterative refinement follows:
 *   TC_PREC_FP32         exact products of the stored factors on the FMA
 *                        units, partial sums folded into compensated pairs:
 *                        G_i to a few ulps of the pattern dtype; no refinement.
 *   TC_PREC_TF32_REFINE  G_i on the tensor cores from TF32-rounded inputs
 *                        (FP32 accumulation), then one refinement step.
 *   TC_PREC_BF16_REFINE  the same from BF16-rounded inputs.
 *   TC_PREC_FP32_REFINE  TC_PREC_FP32, then one refinement step.
 * The refinement step: res_i = rhs_i - lambda a_i - sum_e s_e h_e (h_e^T a_i),
 * summed in FP64 over the row's nonzeros with h_e formed in FP64 from the
 * factors (exactly, for FP32 data), then a_i += (L_i L_i^T)^-1 res_i with the
 * row's Cholesky factor L_i.  It shrinks the error of a_i by about the
 * condition number of G_i + lambda I times the unit roundoff of the Gram.
 * The TF32 / BF16 forms need an FP32 pattern (TC_ERR_UNSUPPORTED otherwise). */
typedef enum {
    TC_PREC_FP32 = 0,
    TC_PREC_TF32_REFINE = 1,
    TC_PREC_BF16_REFINE = 2,
    TC_PREC_FP32_REFINE = 3,
    /* OR-ed into a *_REFINE form: factor in FP32 instead of FP64.  The
     * refinement step corrects the factorization's rounding like the Gram's
     * (its convergence factor is kappa_i times the larger unit roundoff), and
     * FP32 runs far faster than FP64 on this GPU.  Ignored without refinement. */
    TC_PREC_CHOL32 = 0x100,
    /* OR-ed into a *_REFINE form: a second refinement step (the residual with
     * the corrected a_i, then a second correction), which shrinks the error by
     * the same factor again.  Ignored without refinement. */
    TC_PREC_REFINE2 = 0x200
} tc_prec;

/* tc_build_pattern flags */
#define TC_PATTERN_CHECK_DUPLICATES 1u  /* extra sort that rejects repeated coordinates */
#define TC_PATTERN_REFILLABLE 2u        /* keep the builder's work space for tc_pattern_refill
                                           (about 24 bytes per nonzero) */
/* A lean pattern keeps no positions (no perm, no mode-d -> mode-0 maps): 12
 * bytes per nonzero per mode for FP32 values instead of 28 / 20.  Calls that
 * need the maps -- TC_W_ARRAY weights in a mode d > 0 (tc_mttkrp,
 * tc_solve_factor), and so tc_newton_als_mode on modes d > 0, tc_ccd_sweep and
 * tc_ccd_newton_sweep -- return
 * TC_ERR_UNSUPPORTED; tc_pattern_view gives perm = NULL.  The build borrows
 * its sort work space from the arrays of modes not yet built and needs 20
 * extra bytes per nonzero, 8 with TC_PATTERN_CONSUME_INPUT.  Not combinable
 * with TC_PATTERN_CHECK_DUPLICATES or TC_PATTERN_REFILLABLE (TC_ERR_ARG). */
#define TC_PATTERN_LEAN 4u
/* With TC_PATTERN_LEAN only (else TC_ERR_ARG): the build may overwrite the
 * caller's idx and vals arrays, which hold no meaningful data once the call
 * has launched its kernels (that is, unless it returns TC_ERR_ARG or
 * TC_ERR_OOM). */
#define TC_PATTERN_CONSUME_INPUT 8u

typedef struct tc_pattern tc_pattern;

/* ------------------------------------------------------------------ pattern */

/* Builds the per-mode sorted copies of a sparse tensor (Sec. 3.4: the data is
 * sorted by the mode index with a counting sort so that each row's nonzeros are
 * contiguous; Sec. 3.1: only nonempty rows are listed, as in the doubly
 * compressed formats).
 *   order   tensor order; must be 3.
 *   dims    host int64[order], I_n >= 1 and I_n <= 2^31 - 1.
 *   nnz     number of observed entries, >= 0.
 *   idx     host array of `order` device int32 pointers idx[n][e], input order.
 *   vals    device array of nnz values in input order (dtype), or NULL.
 *   dtype   TC_F32 or TC_F64: the type of vals and of every factor used later.
 * On success *out owns device copies; the call synchronizes `stream` once and
 * reports TC_ERR_RANGE / TC_ERR_DUPLICATE directly (no pattern is returned). */
tc_status tc_build_pattern(int order, const int64_t *dims, int64_t nnz,
                           const int32_t *const *idx, const void *vals, tc_dtype dtype,
                           unsigned flags, tc_stream_t stream, tc_pattern **out);

/* Rebuilds pattern p in place from a new tensor with the same order, dims,
 * nnz and dtype (a new batch of observations), reusing every device array, so
 * kernels and captured CUDA graphs that reference p see the new contents.
 * p must have been built with TC_PATTERN_REFILLABLE (else TC_ERR_ARG).  vals
 * must be given iff p was built with values.  Fully asynchronous and
 * allocation-free: out-of-range indices or duplicates (if p checks them) are
 * recorded in the status word for tc_last_error; out-of-range indices are
 * clamped into range in the sorted copies so later kernels stay in bounds. */
tc_status tc_pattern_refill(tc_pattern *p, const int32_t *const *idx, const void *vals,
                            tc_stream_t stream);

/* Frees the pattern's device memory (after synchronizing its device). */
tc_status tc_pattern_destroy(tc_pattern *p);

/* Read-only device views of mode `mode`, for tests and callers that want the
 * raw structure: row_ptr[I_mode + 1] (row i's nonzeros are sorted positions
 * row_ptr[i] .. row_ptr[i+1]-1); perm[nnz] (sorted position -> input position;
 * equal indices keep input order; NULL for a lean pattern);
 * nonempty_rows[n_nonempty] (ascending).
 * Any output pointer may be NULL.  Reading n_nonempty synchronizes the device. */
tc_status tc_pattern_view(const tc_pattern *p, int mode, const int64_t **row_ptr,
                          const int64_t **perm, const int32_t **nonempty_rows,
                          int64_t *n_nonempty);

/* Read-only device views of mode `mode`'s sorted copies: cols1[nnz] and
 * cols2[nnz] hold the indices of the other two modes in ascending mode order
 * (modes 1, 2 for mode 0; 0, 2 for mode 1; 0, 1 for mode 2), vals[nnz] the
 * values (NULL if the pattern has none), all at the sorted positions of
 * tc_pattern_view's row_ptr.  Any output pointer may be NULL. */
tc_status tc_pattern_columns(const tc_pattern *p, int mode, const int32_t **cols1,
                             const int32_t **cols2, const void **vals);

/* nnz, order, dims and dtype of a pattern (host values). */
tc_status tc_pattern_info(const tc_pattern *p, int64_t *nnz, int *order, int64_t *dims,
                          tc_dtype *dtype);

/* Synchronizes `stream`, returns the first device error recorded on pattern p
 * since the last call (TC_OK if none) and clears it. */
tc_status tc_last_error(tc_pattern *p, tc_stream_t stream);

/* ------------------------------------------------------------------ kernels */

/* TTTP (Sec. 3.3): x_e = s_e * sum_{r<R} prod_{n : factors[n] != NULL} A^(n)[i_n(e), r].
 * A NULL factor skips its mode; at least one factor must be given.
 * x: device array of nnz outputs in pattern order (overwritten). */
tc_status tc_tttp(const tc_pattern *p, tc_weights w, const void *s, int R,
                  const void *const *factors, void *x, tc_stream_t stream);

/* MTTKRP restricted to the pattern (Sec. 3.2; Appendix A, gradient as MTTKRP):
 * out[i, r] (+)= sum_{e : i_mode(e) = i} s_e prod_{n != mode} A^(n)[i_n(e), r].
 * out: device I_mode x R, overwritten (accumulate == 0) or added to.
 * factors[mode] is not read and may be NULL. */
tc_status tc_mttkrp(const tc_pattern *p, tc_weights w, const void *s, int R,
                    const void *const *factors, int mode, void *out, int accumulate,
                    tc_stream_t stream);

/* Solve Factor (Sec. 3.4 with the normal equations of Sec. 2.2): for every row
 * i of mode `mode`,
 *   G_i = sum_{e in row i} s_e h_e h_e^T,   h_e = hadamard_{n != mode} A^(n)[i_n(e)],
 *   (G_i + lambda I) a_i = rhs_i,
 * solved by an unpivoted FP64 Cholesky of each R x R system, with G_i summed
 * and refined as `prec` says (tc_prec).  Rows of any length are balanced over
 * the GPU (a row longer than a work chunk is split; see tc_solve_tuning).
 * rhs, out: device I_mode x R; out may alias rhs or factors[mode].  A row with
 * a pivot <= 0 is left unwritten, gets row_status[i] = 1 (device
 * int8[I_mode], may be NULL; other rows get 0) and records TC_ERR_NOT_SPD.
 * An empty row solves lambda a_i = rhs_i. */
tc_status tc_solve_factor(const tc_pattern *p, tc_weights w, const void *s, int R,
                          const void *const *factors, int mode, const void *rhs,
                          double lambda, tc_prec prec, void *out, int8_t *row_status,
                          tc_stream_t stream);

/* One least-squares ALS update of factor `mode` (Sec. 2.2; the MTTKRP of
 * Sec. 3.2 and Solve Factor of Sec. 3.4 in one call): for every row i,
 *   (G_i + lambda I) a_i = rhs_i,  G_i = sum_{e in row i} h_e h_e^T,
 *   rhs_i = sum_{e in row i} t_e h_e   (t: the pattern's values),
 * i.e. tc_solve_factor with unit weights on the right-hand side
 * tc_mttkrp(TC_W_VALUES) would give.  The Gram kernel forms rhs_i from the
 * same gathered rows h_e (one pass over the nonzeros instead of two), except
 * for FP64 data at R <= 16, where the MTTKRP kernel forms it first.  The right-hand side lives in the pattern's work space (I_mode x R
 * of the pattern dtype, plus one R slot of doubles per chunk boundary).
 * The pattern must have values.  out: device I_mode x R; may alias
 * factors[mode] (the usual in-place sweep).  prec, row_status and errors as
 * for tc_solve_factor. */
tc_status tc_als_update(const tc_pattern *p, int R, const void *const *factors, int mode,
                        double lambda, tc_prec prec, void *out, int8_t *row_status,
                        tc_stream_t stream);

/* Solve Factor tuning.  The Gram kernel walks a mode's sorted nonzeros in
 * chunks of `chunk_nnz` (rows longer than a chunk are split across blocks and
 * summed with FP64 atomics), and it forms the Gram triangles of at most
 * `batch_bytes` of rows before factoring them.  Neither changes what is
 * computed, only how the work is cut (FP32 sums may round differently).
 *   chunk_nnz    1 .. 2^30, or 0: automatic (about eight chunks per resident
 *                block, a power of two in [256, 16384]);
 *   batch_bytes  >= 0; 0: automatic (1 GiB).  At least one warp's rows are
 *                taken per batch whatever the value.
 *   chol_rows_per_warp  for R <= 32 one warp factors this many rows
 *                together, 32 / rows lanes sharing each row's work; fewer
 *                rows per warp spread a small mode over more warps
 *                (0: automatic, 16 for R <= 16 and 4 for R <= 32).
 *   gram_kernel  the Gram engine where two exist -- FP32 data, R = 64, the
 *                TF32 and BF16 forms: TC_GRAM_AUTO (0, the tcgen05 kernel),
 *                TC_GRAM_WARP_MMA (warp-level mma.sync, 4-warp blocks
 *                splitting the output tiles) or TC_GRAM_TCGEN05 (tcgen05.mma
 *                with the accumulator in tensor memory).  Ignored elsewhere.
 * Settings are process-wide, per dtype and rank tier (the tier of R: 1..8,
 * 9..16, 17..32, 33..64; R = 0 sets every tier).  t == NULL restores the
 * automatic choice.  Reads and writes of the setting are locked, and each
 * Solve Factor call copies the setting once when it starts, so a change made
 * on another host thread applies to later calls only. */
typedef struct {
    int64_t chunk_nnz;
    int64_t batch_bytes;
    int32_t chol_rows_per_warp;  /* R <= 32: rows one warp factors together:
                                    1, 2, 4, 8, 16 or 32; 0: automatic */
    int32_t gram_kernel;         /* TC_GRAM_*; 0: automatic */
} tc_solve_tuning;

enum { TC_GRAM_AUTO = 0, TC_GRAM_WARP_MMA = 1, TC_GRAM_TCGEN05 = 2 };

tc_status tc_set_solve_tuning(tc_dtype dtype, int R, const tc_solve_tuning *t);
tc_status tc_get_solve_tuning(tc_dtype dtype, int R, tc_solve_tuning *t);

/* Autotuner for Solve Factor (a service of the library; the paper tunes by
 * hand).  Runs tc_solve_factor on the given inputs at each candidate tuning of
 * the rank tier of R -- chunk_nnz in {automatic, 256, 1024, 4096, 16384} times
 * chol_rows_per_warp in {8, 16, 32} (R <= 16) or {4, 8, 16} (R <= 32), times
 * gram_kernel in {TC_GRAM_WARP_MMA, TC_GRAM_TCGEN05} where both engines exist
 * (FP32 data, R = 64, the TF32 and BF16 forms) -- once untimed and once timed with CUDA events on `stream`, and installs the
 * fastest for the pattern's dtype (batch_bytes is kept).  Each candidate is
 * handed to the timed calls directly: the process-wide setting that other
 * threads' calls read changes only once, to the winner, and not at all on an
 * error.  `out` is overwritten with a solution; the stream is synchronized.
 * best, ms_out (may be NULL) receive the chosen tuning and its time in
 * milliseconds. */
tc_status tc_autotune_solve(const tc_pattern *p, tc_weights w, const void *s, int R,
                            const void *const *factors, int mode, const void *rhs,
                            double lambda, tc_prec prec, void *out, tc_solve_tuning *best,
                            float *ms_out, tc_stream_t stream);

/* Objective and gradient (eq. obj; Table 1; Appendix A):
 *   f = sum_e phi(t_e, m_e) + lambda sum_n ||A^(n)||_F^2,  m_e = sum_r prod_n A^(n)[i_n(e), r]
 *   grad^(n) = MTTKRP(phi', n) + 2 lambda A^(n),
 * with t the pattern's values (tc_build_pattern needs vals).
 * loss_out: device double, written (not accumulated); may be NULL.
 * grads: host array of `order` device I_n x R outputs; the array or any entry
 * may be NULL to skip that gradient. */
tc_status tc_loss_grad(const tc_pattern *p, tc_loss loss, int R, const void *const *factors,
                       double lambda, double *loss_out, void *const *grads, tc_stream_t stream);

/* Gauss-Newton matrix-vector product (Sec. 2.5 with the phi' terms dropped;
 * Appendix A):  z_e = sum_p <x^(p)[i_p(e)], h^(p)_e>,
 *   y^(d)[k, r] = sum_{e : i_d(e) = k} phi''_e z_e h^(d)_{e r} + 2 lambda x^(d)[k, r].
 * x, y: host arrays of `order` device I_n x R blocks; y must not alias x. */
tc_status tc_ggn_matvec(const tc_pattern *p, tc_loss loss, int R, const void *const *factors,
                        const void *const *x, double lambda, void *const *y, tc_stream_t stream);

/* ------------------------------------------------------------------ general-loss ALS */

/* General-loss ALS (Sec. 2.2, last paragraph; tolerances as in Sec. 5.7):
 * Newton steps on factor `mode` with the other factors fixed.  Each step forms
 * phi', phi'' at the model entries (TTTP), the gradient
 * g = MTTKRP(phi', mode) + 2 lambda A^(mode), solves per row
 *   (sum_e phi''_e h_e h_e^T + 2 lambda I) step_i = -g_i
 * with Solve Factor (weights phi'', precision form `prec`), and sets
 * A^(mode) += step (in place in factors[mode]).  It stops after inner_iters
 * steps or as soon as ||step||_F <= tol ||A^(mode)||_F.  For least squares one
 * step is the ALS solve.  Needs the pattern's values; a domain error (identity
 * link at m <= 0) or a non-SPD row is recorded for tc_last_error.
 * steps_out (host, may be NULL) receives the number of steps taken.
 * Synchronizes `stream` once per step (the stop test reads two norms). */
tc_status tc_newton_als_mode(const tc_pattern *p, tc_loss loss, int R, void *const *factors,
                             int mode, double lambda, int inner_iters, double tol, tc_prec prec,
                             int *steps_out, tc_stream_t stream);

/* Full Newton Hessian-vector product (Sec. 2.5 before the Gauss-Newton
 * approximation; Appendix A): the product of tc_ggn_matvec plus the phi'
 * term sum_e phi'_e (d^2 m_e) x, whose block for output mode d is, for each
 * other mode q, the pattern-restricted MTTKRP of phi' with x^(q) in place of
 * A^(q) (the second derivative of m_e within one mode is zero).  The matrix
 * is symmetric but may be indefinite.  Same arguments and layout as
 * tc_ggn_matvec. */
tc_status tc_newton_matvec(const tc_pattern *p, tc_loss loss, int R, const void *const *factors,
                           const void *const *x, double lambda, void *const *y,
                           tc_stream_t stream);

/* Coordinate minimization for least squares in CCD++ order (Sec. 2.3): one
 * sweep over r = 0 .. R-1; for each r the residual takes the rank-r term back
 * (rho = t - <u, v, w> + u_r v_r w_r), column r of each factor in turn is set
 * to sum_e v_jr w_kr rho_e / (lambda + sum_e v_jr^2 w_kr^2) (updated columns
 * used at once), and the new rank-r term leaves the residual.  Factors are
 * updated in place; the residual is formed from the pattern's values at the
 * start of the sweep.  Made of rank-1 TTTP, MTTKRP and Solve Factor launches
 * (2R passes over the nonzeros plus 3R rank-1 Solve Factors). */
tc_status tc_ccd_sweep(const tc_pattern *p, int R, void *const *factors, double lambda,
                       tc_stream_t stream);

/* Coordinate minimization for a general loss (Sec. 2.3, last paragraph;
 * tolerances as in Sec. 5.7), in the same CCD++ order: for r = 0 .. R-1 and
 * each mode d in turn, Newton steps on column r of A^(d) with the rest fixed.
 * The column's elements are decoupled, so one step is, per row i,
 *   delta_i = -(sum_e phi'_e h_e + 2 lambda u_ir) / (sum_e phi''_e h_e^2 + 2 lambda),
 * h_e = prod_{n != d} A^(n)[i_n(e), r], phi', phi'' at the current model
 * entries (Table 1 scaling, as tc_loss_grad).  A column stops after
 * inner_iters steps or once ||delta||_2 <= tol ||column||_2.  For least
 * squares one step is the tc_ccd_sweep update.  Factors are updated in place;
 * needs the pattern's values and lambda >= 0; a domain error or a zero
 * denominator (lambda = 0 and an empty row) is recorded for tc_last_error.
 * steps_out: host int[R * order] (entry r * order + d: the steps taken on that
 * column) or NULL.  Synchronizes `stream` once per step. */
tc_status tc_ccd_newton_sweep(const tc_pattern *p, tc_loss loss, int R, void *const *factors,
                              double lambda, int inner_iters, double tol, int *steps_out,
                              tc_stream_t stream);

/* ------------------------------------------------------------------ GGN / PCG */

/* A preconditioned-CG solver for the Gauss-Newton system H dx = b at fixed
 * factors (Sec. 2.5).  The preconditioner is the block diagonal of H: per mode
 * d and row k, P_k = sum_{e in row k} phi''_e h_e h_e^T + 2 lambda I, factored
 * once by FP64 Cholesky (the Solve Factor systems with weights phi''), applied
 * by two triangular solves.  The iteration runs from x0 = 0 for a fixed count,
 * with FP64 inner products and step lengths kept on the device; it is captured
 * once into a CUDA graph and replayed.
 *
 * tc_cg_create keeps `p`, the factor pointers, and allocates its work vectors;
 * the factor contents may change between solves (call tc_cg_setup again). */
typedef struct tc_cg tc_cg;

tc_status tc_cg_create(const tc_pattern *p, tc_loss loss, int R, const void *const *factors,
                       double lambda, int precondition, tc_cg **out);
tc_status tc_cg_destroy(tc_cg *cg);

/* Selects the matrix the solver iterates with: 0 = the Gauss-Newton matrix
 * (the default), 1 = the full Hessian (tc_newton_matvec; Sec. 2.5, "Newton's
 * method").  The block-diagonal preconditioner is the same for both: the
 * full Hessian's phi' term has no block within a row.  The full Hessian may be
 * indefinite; PCG then stops at the first direction with p^T H p <= 0 and
 * reports TC_ERR_BREAKDOWN (the indefiniteness check).  Changing the choice
 * discards the captured graph (the next tc_cg_solve captures again); it
 * synchronizes the device. */
tc_status tc_cg_set_hessian(tc_cg *cg, int full_newton);

/* Builds (or rebuilds) the preconditioner at the current factor values. */
tc_status tc_cg_setup(tc_cg *cg, tc_stream_t stream);

/* Applies the preconditioner: z^(d) = P^-1 r^(d) for all modes (after setup). */
tc_status tc_cg_precond_apply(tc_cg *cg, const void *const *r, void *const *z,
                              tc_stream_t stream);

/* Runs `iters` PCG iterations on H dx = b from dx = 0.  b, dx: host arrays of
 * `order` device I_n x R blocks (dx overwritten).  rz_out (device double[iters+1],
 * may be NULL) receives r^T z before each iteration.  The first call with a
 * given (b, dx, iters) captures a CUDA graph; later calls replay it. */
tc_status tc_cg_solve(tc_cg *cg, const void *const *b, void *const *dx, int iters,
                      double *rz_out, tc_stream_t stream);

/* y = H x with the solver's Gauss-Newton matrix at the current factors (the
 * product tc_cg_solve iterates with: on the vector path the factor and
 * direction rows are first interleaved into the solver's own buffers).
 * x, y: host arrays of `order` device I_n x R blocks; y must not alias x. */
tc_status tc_cg_matvec(tc_cg *cg, const void *const *x, void *const *y, tc_stream_t stream);

/* One Gauss-Newton step at the current factors: gradient, preconditioner,
 * `iters` PCG iterations on H dx = -grad, then A^(n) += dx^(n) in place.
 * loss_out (device double, may be NULL) receives f before the step. */
tc_status tc_ggn_step(tc_cg *cg, int iters, double *loss_out, tc_stream_t stream);

/* The vector steps of PCG (Sec. 2.5) for drivers that run the iteration
 * themselves, e.g. over row blocks held by several processes, where the inner
 * products are summed across processes between the steps.
 *   tc_axpby: y = alpha x + beta y over n elements of dtype (device x, y; y
 *             may alias x).
 *   tc_dot:   *out = sum_i x_i y_i (accumulate = 0) or *out += it (1), summed
 *             in FP64 (device double out; the order of the partial sums is
 *             not fixed). */
tc_status tc_axpby(tc_dtype dtype, int64_t n, double alpha, const void *x, double beta, void *y,
                   tc_stream_t stream);
tc_status tc_dot(tc_dtype dtype, int64_t n, const void *x, const void *y, double *out,
                 int accumulate, tc_stream_t stream);

/* ------------------------------------------------------------------ allocation-free sort */

/* Largest nnz that tc_sort_mode_noalloc accepts. */
#define TC_SORT_NOALLOC_MAX_NNZ (1 << 20)

/* The per-mode sort of tc_build_pattern for one index array, without any
 * device allocation.  The paper has no counterpart: this is a service of the
 * library for callers that may not call cudaMalloc -- a process that handed all
 * device memory to another allocator's pool, a server that forbids new
 * allocations once it is serving so that no request can fail for lack of
 * memory, or a host thread that must not stall: a device allocation can make
 * the CUDA runtime synchronize work across streams.
 *   key      device int32[nnz]: mode indices in input order.
 *   I        the mode's dimension, 1 <= I <= 2^31 - 1.
 *   perm     device int64[nnz] output: sorted position -> input position,
 *            equal keys in input order (the same as tc_pattern_view's perm).
 *   row_ptr  device int64[I + 1] output, as tc_pattern_view's row_ptr.
 *   status   device int or NULL: set to 0, then to TC_ERR_RANGE if a key lies
 *            outside [0, I) (perm is then still a permutation, row_ptr is not
 *            meaningful).
 * Work space is one array of about 16.5 MB compiled into the library; every
 * GPU that loads the library holds it until the process exits.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  All calls share the array
 * and a call leaves its contents behind: calls whose GPU work overlaps (other
 * streams, other host threads) race and give wrong answers, so serialize them.
 * nnz > TC_SORT_NOALLOC_MAX_NNZ returns TC_ERR_UNSUPPORTED and launches
 * nothing.  Asynchronous on `stream`. */
tc_status tc_sort_mode_noalloc(int64_t nnz, const int32_t *key, int64_t I, int64_t *perm,
                               int64_t *row_ptr, int *status, tc_stream_t stream);

/* ------------------------------------------------------------------ misc */

/* Number of kernel launches this library has issued in the calling process
 * (graph replays count the kernels they contain).  For launch accounting. */
int64_t tc_launch_count(void);

/* Human-readable name of a status code. */
const char *tc_status_string(tc_status s);

#ifdef __cplusplus
}
#endif
#endif
