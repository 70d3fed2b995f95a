// General-loss ALS (Sec. 2.2, last paragraph; the inner tolerances are those
// of the Poisson experiments, Sec. 5.7): Newton steps on one factor with the
// others fixed.  A step is composed of the library's kernels:
//   TTTP                m_e at every observed entry (pattern order),
//   loss_derivs_kernel  phi'(t_e, m_e), phi''(t_e, m_e),
//   MTTKRP              g = MTTKRP(phi', mode), then rhs = -(g + 2 lambda A),
//   Solve Factor        (sum_e phi''_e h_e h_e^T + 2 lambda I) step_i = rhs_i,
//   newton_update       A += step, with ||step||^2 and ||A||^2 for the stop test.
// Table 1 gives the row gradient and Hessian; the Hessian's phi' term is zero
// within a row (the model is linear in the row being updated), so this is the
// exact Newton step of each row problem.
#include "internal.cuh"

namespace tc {

template <typename T>
__global__ void loss_derivs_kernel(int64_t n, int loss, const T *__restrict__ t,
                                   const T *__restrict__ m, T *__restrict__ d1,
                                   T *__restrict__ d2, int *status) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        T phi, a, b;
        bool ok = true;
        loss_terms(loss, __ldcs(t + e), __ldcs(m + e), phi, a, b, ok);
        if (!ok) record_error(status, TC_ERR_DOMAIN);
        d1[e] = a;
        d2[e] = b;
    }
}

template <typename T>
__global__ void newton_rhs_kernel(int64_t n, const T *__restrict__ g, const T *__restrict__ A,
                                  double two_lambda, T *__restrict__ rhs) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        rhs[q] = -(g[q] + (T)two_lambda * A[q]);
}

// A += step; sums[0] += ||step||^2, sums[1] += ||A_new||^2 (FP64).
template <typename T>
__global__ void newton_update_kernel(int64_t n, T *__restrict__ A, const T *__restrict__ step,
                                     double *sums) {
    double s2 = 0.0, a2 = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const T d = step[q];
        const T a = A[q] + d;
        A[q] = a;
        s2 += (double)d * (double)d;
        a2 += (double)a * (double)a;
    }
    block_add(s2, sums);
    block_add(a2, sums + 1);
}

static unsigned newton_grid(int64_t n) {
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

template <typename T>
void launch_loss_derivs(int64_t n, int loss, const T *t, const T *m, T *d1, T *d2, int *status,
                        cudaStream_t st) {
    if (n <= 0) return;
    loss_derivs_kernel<T><<<newton_grid(n), 256, 0, st>>>(n, loss, t, m, d1, d2, status);
    count_launch();
}

template <typename T>
void launch_newton_rhs(int64_t n, const T *g, const T *A, double two_lambda, T *rhs,
                       cudaStream_t st) {
    if (n <= 0) return;
    newton_rhs_kernel<T><<<newton_grid(n), 256, 0, st>>>(n, g, A, two_lambda, rhs);
    count_launch();
}

template <typename T>
void launch_newton_update(int64_t n, T *A, const T *step, double *sums, cudaStream_t st) {
    if (n <= 0) return;
    newton_update_kernel<T><<<newton_grid(n), 256, 0, st>>>(n, A, step, sums);
    count_launch();
}

#define TC_NEWTON_LAUNCHERS(T)                                                                  \
    template void launch_loss_derivs<T>(int64_t, int, const T *, const T *, T *, T *, int *,    \
                                        cudaStream_t);                                         \
    template void launch_newton_rhs<T>(int64_t, const T *, const T *, double, T *, cudaStream_t); \
    template void launch_newton_update<T>(int64_t, T *, const T *, double *, cudaStream_t);
TC_NEWTON_LAUNCHERS(float)
TC_NEWTON_LAUNCHERS(double)
#undef TC_NEWTON_LAUNCHERS

template <typename T>
static tc_status newton_t(const tc_pattern *p, tc_loss loss, int R, void *const *factors, int mode,
                          double lambda, int inner_iters, double tol, tc_prec prec, int *steps_out,
                          cudaStream_t st) {
    const int64_t m = p->nnz, I = p->dims[mode], n = I * (int64_t)R;
    // m_e, phi', phi'' (nnz each); g, rhs, step (I x R each): the pattern's
    // work space (allocated once per size)
    const size_t elems = (size_t)3 * (size_t)(m > 0 ? m : 1) + (size_t)3 * (size_t)n;
    T *buf = (T *)work_buffer(p, WS_NEWTON, sizeof(T) * elems);
    double *sums = (double *)work_buffer(p, WS_NEWTON_SUMS, 2 * sizeof(double));
    if (!buf || !sums) return TC_ERR_OOM;
    T *mv = buf, *d1 = mv + (m > 0 ? m : 1), *d2 = d1 + (m > 0 ? m : 1);
    T *g = d2 + (m > 0 ? m : 1), *rhs = g + n, *step = rhs + n;
    T *Ad = (T *)factors[mode];
    const void *const *A = (const void *const *)factors;
    tc_status rc = TC_OK;
    int taken = 0;
    for (int it = 0; it < inner_iters && rc == TC_OK; ++it) {
        if (m > 0) {
            rc = launch_tttp(p, TC_W_ONE, nullptr, R, A, mv, st);
            if (rc != TC_OK) break;
            launch_loss_derivs<T>(m, (int)loss, (const T *)p->md[0].vals, mv, d1, d2, p->status, st);
        }
        rc = launch_mttkrp(p, TC_W_ARRAY, d1, R, A, mode, g, 0, st);
        if (rc != TC_OK) break;
        launch_newton_rhs<T>(n, g, Ad, 2.0 * lambda, rhs, st);
        rc = launch_solve_factor(p, TC_W_ARRAY, d2, R, A, mode, rhs, 2.0 * lambda, prec, step,
                                 nullptr, 0, TC_LOSS_LS, nullptr, st);
        if (rc != TC_OK) break;
        if (cudaMemsetAsync(sums, 0, 2 * sizeof(double), st) != cudaSuccess) {
            rc = TC_ERR_CUDA;
            break;
        }
        launch_newton_update<T>(n, Ad, step, sums, st);
        ++taken;
        double h[2] = {0.0, 0.0};
        if (cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = TC_ERR_CUDA;
            break;
        }
        if (sqrt(h[0]) <= tol * sqrt(h[1])) break;
    }
    if (rc == TC_OK && cudaGetLastError() != cudaSuccess) rc = TC_ERR_CUDA;
    if (steps_out) *steps_out = taken;
    return rc;
}

}  // namespace tc

using namespace tc;

extern "C" tc_status tc_newton_als_mode(const tc_pattern *p, tc_loss loss, int R,
                                        void *const *factors, int mode, double lambda,
                                        int inner_iters, double tol, tc_prec prec, int *steps_out,
                                        tc_stream_t stream) {
    if (steps_out) *steps_out = 0;
    if (!p || R < 1 || R > TC_MAX_RANK || !factors || mode < 0 || mode >= p->order) return TC_ERR_ARG;
    for (int n = 0; n < TC_ORDER; ++n)
        if (!factors[n]) return TC_ERR_ARG;
    if (loss != TC_LOSS_LS && loss != TC_LOSS_POISSON_LOG && loss != TC_LOSS_POISSON_ID)
        return TC_ERR_ARG;
    if (inner_iters < 1 || !(tol >= 0.0)) return TC_ERR_ARG;
    if (!p->has_vals && p->nnz > 0) return TC_ERR_ARG;
    const int form = prec & ~(TC_PREC_CHOL32 | TC_PREC_REFINE2);
    if (form != TC_PREC_FP32 && form != TC_PREC_TF32_REFINE && form != TC_PREC_BF16_REFINE &&
        form != TC_PREC_FP32_REFINE)
        return TC_ERR_ARG;
    if (p->dtype == TC_F64)
        return newton_t<double>(p, loss, R, factors, mode, lambda, inner_iters, tol, prec, steps_out,
                                (cudaStream_t)stream);
    return newton_t<float>(p, loss, R, factors, mode, lambda, inner_iters, tol, prec, steps_out,
                           (cudaStream_t)stream);
}
