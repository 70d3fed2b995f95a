// Coordinate minimization for least squares in CCD++ order (Sec. 2.3): for
// each rank component r the residual gets the rank-r term back,
//   rho = t - <u, v, w> + u_r v_r w_r,
// then column r of each factor is set in turn to
//   u_ir = sum_e v_jr w_kr rho_e / (lambda + sum_e v_jr^2 w_kr^2),
// and the updated rank-r term is taken out of the residual again.  At rank 1
// the numerator is a rank-1 MTTKRP of rho and the division is exactly a rank-1
// Solve Factor, so a column update is two library kernels; the rank-1 TTTPs
// move rho.  Columns are gathered from / scattered into the row-major factors
// by two small kernels.
#include "internal.cuh"

namespace tc {

template <typename T>
__global__ void col_get_kernel(const T *__restrict__ A, int64_t I, int R, int r, T *__restrict__ c) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I;
         i += (int64_t)gridDim.x * blockDim.x)
        c[i] = A[i * R + r];
}

template <typename T>
__global__ void col_put_kernel(T *__restrict__ A, int64_t I, int R, int r, const T *__restrict__ c) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I;
         i += (int64_t)gridDim.x * blockDim.x)
        A[i * R + r] = c[i];
}

// y += alpha x  (alpha = +1 / -1: the residual moves)
template <typename T>
__global__ void resid_axpy_kernel(int64_t n, T alpha, const T *__restrict__ x, T *__restrict__ y) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        y[e] += alpha * x[e];
}

// rho = t - m
template <typename T>
__global__ void resid_init_kernel(int64_t n, const T *__restrict__ t, const T *__restrict__ m,
                                  T *__restrict__ rho) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x)
        rho[e] = t[e] - m[e];
}

static unsigned grid_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    return (unsigned)(b < 1 ? 1 : b);
}

template <typename T>
static tc_status ccd_t(const tc_pattern *p, int R, void *const *factors, double lambda,
                       cudaStream_t st) {
    const int64_t m = p->nnz;
    const int64_t I0 = p->dims[0], I1 = p->dims[1], I2 = p->dims[2];
    const int64_t Imax = I0 > I1 ? (I0 > I2 ? I0 : I2) : (I1 > I2 ? I1 : I2);
    const int64_t mm = m > 0 ? m : 1;
    // residual, rank-1 TTTP (nnz each); columns; right-hand side: the
    // pattern's work space (allocated once per size)
    T *buf = (T *)work_buffer(p, WS_CCD, sizeof(T) * (size_t)(2 * mm + I0 + I1 + I2 + Imax));
    if (!buf) return TC_ERR_OOM;
    T *rho = buf, *x = rho + mm, *c0 = x + mm, *c1 = c0 + I0, *c2 = c1 + I1, *num = c2 + I2;
    T *col[TC_ORDER] = {c0, c1, c2};
    const void *cols[TC_ORDER] = {c0, c1, c2};
    const int64_t I[TC_ORDER] = {I0, I1, I2};
    const T *t = (const T *)p->md[0].vals;
    tc_status rc = TC_OK;
    if (m > 0) {
        rc = launch_tttp(p, TC_W_ONE, nullptr, R, (const void *const *)factors, x, st);
        if (rc == TC_OK) {
            resid_init_kernel<T><<<grid_for(m), 256, 0, st>>>(m, t, x, rho);
            count_launch();
        }
    }
    for (int r = 0; r < R && rc == TC_OK; ++r) {
        for (int n = 0; n < TC_ORDER; ++n) {
            col_get_kernel<T><<<grid_for(I[n]), 256, 0, st>>>((const T *)factors[n], I[n], R, r, col[n]);
            count_launch();
        }
        if (m > 0) {   // rho += u_r v_r w_r
            rc = launch_tttp(p, TC_W_ONE, nullptr, 1, cols, x, st);
            if (rc != TC_OK) break;
            resid_axpy_kernel<T><<<grid_for(m), 256, 0, st>>>(m, T(1), x, rho);
            count_launch();
        }
        for (int d = 0; d < TC_ORDER && rc == TC_OK; ++d) {
            rc = launch_mttkrp(p, TC_W_ARRAY, rho, 1, cols, d, num, 0, st);
            if (rc != TC_OK) break;
            rc = launch_solve_factor(p, TC_W_ONE, nullptr, 1, cols, d, num, lambda, TC_PREC_FP32,
                                     col[d], nullptr, 0, TC_LOSS_LS, nullptr, st);
        }
        if (rc != TC_OK) break;
        if (m > 0) {   // rho -= (new) u_r v_r w_r
            rc = launch_tttp(p, TC_W_ONE, nullptr, 1, cols, x, st);
            if (rc != TC_OK) break;
            resid_axpy_kernel<T><<<grid_for(m), 256, 0, st>>>(m, T(-1), x, rho);
            count_launch();
        }
        for (int n = 0; n < TC_ORDER; ++n) {
            col_put_kernel<T><<<grid_for(I[n]), 256, 0, st>>>((T *)factors[n], I[n], R, r, col[n]);
            count_launch();
        }
    }
    if (rc == TC_OK && cudaGetLastError() != cudaSuccess) rc = TC_ERR_CUDA;
    return rc;
}

// Coordinate minimization for a general loss (Sec. 2.3, last paragraph), same
// order: Newton steps on column r of A^(d) with the rest fixed.  A nonzero
// involves one row of A^(d), so the column's elements are decoupled and a step
// is, per row i,
//   (sum_e phi''_e h_e^2 + 2 lambda) delta_i = -(sum_e phi'_e h_e + 2 lambda u_ir),
// h_e the product of the other columns: a rank-1 MTTKRP of phi' and a rank-1
// Solve Factor with weights phi''.  The model entries m_e (pattern order) are
// kept current by rank-1 TTTPs of (delta, other columns); phi', phi'' are
// formed from them before every step.  The stop test (Sec. 5.7 tolerances)
// reads two norms per step.
template <typename T>
static tc_status ccd_newton_t(const tc_pattern *p, tc_loss loss, int R, void *const *factors,
                              double lambda, int inner_iters, double tol, int *steps_out,
                              cudaStream_t st) {
    const int64_t m = p->nnz;
    const int64_t I[TC_ORDER] = {p->dims[0], p->dims[1], p->dims[2]};
    const int64_t Imax = I[0] > I[1] ? (I[0] > I[2] ? I[0] : I[2]) : (I[1] > I[2] ? I[1] : I[2]);
    const int64_t mm = m > 0 ? m : 1;
    // model, phi', phi'', rank-1 TTTP (nnz each); columns; g, rhs, delta (Imax
    // each): the pattern's work space (allocated once per size)
    T *buf = (T *)work_buffer(p, WS_CCD, sizeof(T) * (size_t)(4 * mm + I[0] + I[1] + I[2] + 3 * Imax));
    double *sums = (double *)work_buffer(p, WS_CCD_SUMS, 2 * sizeof(double));
    if (!buf || !sums) return TC_ERR_OOM;
    T *mv = buf, *d1 = mv + mm, *d2 = d1 + mm, *x = d2 + mm, *c0 = x + mm, *c1 = c0 + I[0],
      *c2 = c1 + I[1], *g = c2 + I[2], *rhs = g + Imax, *delta = rhs + Imax;
    T *col[TC_ORDER] = {c0, c1, c2};
    const T *t = (const T *)p->md[0].vals;
    tc_status rc = TC_OK;
    if (m > 0) rc = launch_tttp(p, TC_W_ONE, nullptr, R, (const void *const *)factors, mv, st);
    for (int r = 0; r < R && rc == TC_OK; ++r) {
        for (int n = 0; n < TC_ORDER; ++n) {
            col_get_kernel<T><<<grid_for(I[n]), 256, 0, st>>>((const T *)factors[n], I[n], R, r, col[n]);
            count_launch();
        }
        for (int d = 0; d < TC_ORDER && rc == TC_OK; ++d) {
            const void *cols[TC_ORDER] = {c0, c1, c2};
            const void *dcols[TC_ORDER] = {c0, c1, c2};
            dcols[d] = delta;
            int taken = 0;
            for (int it = 0; it < inner_iters; ++it) {
                launch_loss_derivs<T>(m, (int)loss, t, mv, d1, d2, p->status, st);
                rc = launch_mttkrp(p, TC_W_ARRAY, d1, 1, cols, d, g, 0, st);
                if (rc != TC_OK) break;
                launch_newton_rhs<T>(I[d], g, col[d], 2.0 * lambda, rhs, st);
                rc = launch_solve_factor(p, TC_W_ARRAY, d2, 1, cols, d, rhs, 2.0 * lambda,
                                         TC_PREC_FP32, delta, nullptr, 0, TC_LOSS_LS, nullptr, st);
                if (rc != TC_OK) break;
                if (m > 0) {   // m_e += delta_i h_e
                    rc = launch_tttp(p, TC_W_ONE, nullptr, 1, dcols, x, st);
                    if (rc != TC_OK) break;
                    resid_axpy_kernel<T><<<grid_for(m), 256, 0, st>>>(m, T(1), x, mv);
                    count_launch();
                }
                if (cudaMemsetAsync(sums, 0, 2 * sizeof(double), st) != cudaSuccess) {
                    rc = TC_ERR_CUDA;
                    break;
                }
                launch_newton_update<T>(I[d], col[d], delta, sums, st);
                ++taken;
                double h[2] = {0.0, 0.0};
                if (cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess) {
                    rc = TC_ERR_CUDA;
                    break;
                }
                if (sqrt(h[0]) <= tol * sqrt(h[1])) break;
            }
            if (steps_out) steps_out[r * TC_ORDER + d] = taken;
        }
        for (int n = 0; n < TC_ORDER; ++n) {
            col_put_kernel<T><<<grid_for(I[n]), 256, 0, st>>>((T *)factors[n], I[n], R, r, col[n]);
            count_launch();
        }
    }
    if (rc == TC_OK && cudaGetLastError() != cudaSuccess) rc = TC_ERR_CUDA;
    return rc;
}

}  // namespace tc

using namespace tc;

extern "C" tc_status tc_ccd_sweep(const tc_pattern *p, int R, void *const *factors, double lambda,
                                  tc_stream_t stream) {
    if (!p || R < 1 || R > TC_MAX_RANK || !factors) return TC_ERR_ARG;
    for (int n = 0; n < TC_ORDER; ++n)
        if (!factors[n]) return TC_ERR_ARG;
    if (!p->has_vals && p->nnz > 0) return TC_ERR_ARG;
    if (p->dtype == TC_F64) return ccd_t<double>(p, R, factors, lambda, (cudaStream_t)stream);
    return ccd_t<float>(p, R, factors, lambda, (cudaStream_t)stream);
}

extern "C" tc_status tc_ccd_newton_sweep(const tc_pattern *p, tc_loss loss, int R,
                                         void *const *factors, double lambda, int inner_iters,
                                         double tol, int *steps_out, tc_stream_t stream) {
    if (!p || R < 1 || R > TC_MAX_RANK || !factors) return TC_ERR_ARG;
    for (int n = 0; n < TC_ORDER; ++n)
        if (!factors[n]) return TC_ERR_ARG;
    if (loss != TC_LOSS_LS && loss != TC_LOSS_POISSON_LOG && loss != TC_LOSS_POISSON_ID)
        return TC_ERR_ARG;
    if (inner_iters < 1 || !(tol >= 0.0) || !(lambda >= 0.0)) return TC_ERR_ARG;
    if (!p->has_vals && p->nnz > 0) return TC_ERR_ARG;
    if (steps_out)
        for (int q = 0; q < R * TC_ORDER; ++q) steps_out[q] = 0;
    if (p->dtype == TC_F64)
        return ccd_newton_t<double>(p, loss, R, factors, lambda, inner_iters, tol, steps_out,
                                    (cudaStream_t)stream);
    return ccd_newton_t<float>(p, loss, R, factors, lambda, inner_iters, tol, steps_out,
                               (cudaStream_t)stream);
}
