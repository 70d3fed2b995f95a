// C ABI of libtc: argument checks and dispatch to the kernel launchers.
// Every entry point validates its arguments before launching anything and
// returns TC_ERR_ARG / TC_ERR_UNSUPPORTED without touching the device.
#include "internal.cuh"

namespace tc {
int64_t g_launches = 0;
}

using namespace tc;

static bool rank_ok(int R) { return R >= 1 && R <= TC_MAX_RANK; }

static tc_status launch_status() {
    return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

static tc_status check_weights(const tc_pattern *p, tc_weights w, const void *s) {
    if (w == TC_W_ONE) return TC_OK;
    if (w == TC_W_VALUES) return (p->has_vals || p->nnz == 0) ? TC_OK : TC_ERR_ARG;
    if (w == TC_W_ARRAY) return (s || p->nnz == 0) ? TC_OK : TC_ERR_ARG;
    return TC_ERR_ARG;
}

// All factors except `skip` must be given (skip < 0: all).
static bool factors_ok(const void *const *A, int skip) {
    if (!A) return false;
    for (int n = 0; n < TC_ORDER; ++n)
        if (n != skip && !A[n]) return false;
    return true;
}

extern "C" {

const char *tc_status_string(tc_status s) {
    switch (s) {
        case TC_OK: return "ok";
        case TC_ERR_ARG: return "invalid argument";
        case TC_ERR_RANGE: return "index out of range";
        case TC_ERR_DUPLICATE: return "duplicate coordinate";
        case TC_ERR_OOM: return "out of device memory";
        case TC_ERR_CUDA: return "CUDA error";
        case TC_ERR_NOT_SPD: return "row system not positive definite";
        case TC_ERR_DOMAIN: return "loss evaluated outside its domain";
        case TC_ERR_BREAKDOWN: return "CG breakdown";
        case TC_ERR_UNSUPPORTED: return "unsupported";
        case TC_ERR_TIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

int64_t tc_launch_count(void) { return g_launches; }

tc_status tc_build_pattern(int order, const int64_t *dims, int64_t nnz, const int32_t *const *idx,
                           const void *vals, tc_dtype dtype, unsigned flags, tc_stream_t stream,
                           tc_pattern **out) {
    if (!out) return TC_ERR_ARG;
    *out = nullptr;
    if (order != TC_ORDER) return order >= 1 ? TC_ERR_UNSUPPORTED : TC_ERR_ARG;
    if (!dims || nnz < 0 || (dtype != TC_F32 && dtype != TC_F64)) return TC_ERR_ARG;
    if (flags & ~(TC_PATTERN_CHECK_DUPLICATES | TC_PATTERN_REFILLABLE | TC_PATTERN_LEAN |
                  TC_PATTERN_CONSUME_INPUT))
        return TC_ERR_ARG;
    // a lean pattern keeps no work space and no positions; consuming the input
    // is a lean build's way to borrow its work space
    if ((flags & TC_PATTERN_LEAN) && (flags & (TC_PATTERN_CHECK_DUPLICATES | TC_PATTERN_REFILLABLE)))
        return TC_ERR_ARG;
    if ((flags & TC_PATTERN_CONSUME_INPUT) && !(flags & TC_PATTERN_LEAN)) return TC_ERR_ARG;
    for (int d = 0; d < TC_ORDER; ++d)
        if (dims[d] < 1 || dims[d] > INT32_MAX) return TC_ERR_ARG;
    if (nnz > 0) {
        if (!idx) return TC_ERR_ARG;
        for (int d = 0; d < TC_ORDER; ++d)
            if (!idx[d]) return TC_ERR_ARG;
    }
    tc_status rc = build_pattern_impl(order, dims, nnz, idx, vals, dtype, flags,
                                      (cudaStream_t)stream, out);
    if (rc == TC_OK && cudaGetLastError() != cudaSuccess) {
        free_pattern(*out);
        *out = nullptr;
        return TC_ERR_CUDA;
    }
    return rc;
}

tc_status tc_pattern_refill(tc_pattern *p, const int32_t *const *idx, const void *vals,
                            tc_stream_t stream) {
    if (!p) return TC_ERR_ARG;
    if ((vals != nullptr) != (p->has_vals != 0) && p->nnz > 0) return TC_ERR_ARG;
    if (p->nnz > 0) {
        if (!idx) return TC_ERR_ARG;
        for (int d = 0; d < TC_ORDER; ++d)
            if (!idx[d]) return TC_ERR_ARG;
    }
    tc_status rc = refill_pattern_impl(p, idx, vals, (cudaStream_t)stream);
    return rc != TC_OK ? rc : launch_status();
}

tc_status tc_pattern_destroy(tc_pattern *p) {
    if (!p) return TC_ERR_ARG;
    cudaDeviceSynchronize();
    free_pattern(p);
    return TC_OK;
}

tc_status tc_pattern_view(const tc_pattern *p, int mode, const int64_t **row_ptr,
                          const int64_t **perm, const int32_t **nonempty_rows,
                          int64_t *n_nonempty) {
    if (!p || mode < 0 || mode >= p->order) return TC_ERR_ARG;
    const ModeData &m = p->md[mode];
    if (row_ptr) *row_ptr = m.row_ptr;
    if (perm) *perm = m.perm;
    if (nonempty_rows) *nonempty_rows = m.nz_rows;
    if (n_nonempty) {
        if (cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(n_nonempty, m.n_ne_dev, sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            return TC_ERR_CUDA;
    }
    return TC_OK;
}

tc_status tc_pattern_columns(const tc_pattern *p, int mode, const int32_t **cols1,
                             const int32_t **cols2, const void **vals) {
    if (!p || mode < 0 || mode >= p->order) return TC_ERR_ARG;
    const ModeData &m = p->md[mode];
    if (cols1) *cols1 = m.cols[0];
    if (cols2) *cols2 = m.cols[1];
    if (vals) *vals = m.vals;
    return TC_OK;
}

tc_status tc_pattern_info(const tc_pattern *p, int64_t *nnz, int *order, int64_t *dims,
                          tc_dtype *dtype) {
    if (!p) return TC_ERR_ARG;
    if (nnz) *nnz = p->nnz;
    if (order) *order = p->order;
    if (dims)
        for (int d = 0; d < p->order; ++d) dims[d] = p->dims[d];
    if (dtype) *dtype = p->dtype;
    return TC_OK;
}

tc_status tc_last_error(tc_pattern *p, tc_stream_t stream) {
    if (!p) return TC_ERR_ARG;
    int h = 0;
    if (cudaMemcpyAsync(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost,
                        (cudaStream_t)stream) != cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return TC_ERR_CUDA;
    if (h) {
        if (cudaMemsetAsync(p->status, 0, sizeof(int), (cudaStream_t)stream) != cudaSuccess ||
            cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
            return TC_ERR_CUDA;
    }
    return (tc_status)h;
}

tc_status tc_tttp(const tc_pattern *p, tc_weights w, const void *s, int R,
                  const void *const *factors, void *x, tc_stream_t stream) {
    if (!p || !factors || !rank_ok(R) || (!x && p->nnz > 0)) return TC_ERR_ARG;
    if (check_weights(p, w, s) != TC_OK) return TC_ERR_ARG;
    int provided = 0;
    for (int n = 0; n < TC_ORDER; ++n) provided += factors[n] ? 1 : 0;
    if (!provided) return TC_ERR_ARG;
    tc_status rc = launch_tttp(p, w, s, R, factors, x, (cudaStream_t)stream);
    return rc != TC_OK ? rc : launch_status();
}

tc_status tc_mttkrp(const tc_pattern *p, tc_weights w, const void *s, int R,
                    const void *const *factors, int mode, void *out, int accumulate,
                    tc_stream_t stream) {
    if (!p || !rank_ok(R) || !out || mode < 0 || mode >= p->order) return TC_ERR_ARG;
    if (!factors_ok(factors, mode) || check_weights(p, w, s) != TC_OK) return TC_ERR_ARG;
    tc_status rc = launch_mttkrp(p, w, s, R, factors, mode, out, accumulate ? 1 : 0,
                                 (cudaStream_t)stream);
    return rc != TC_OK ? rc : launch_status();
}

tc_status tc_solve_factor(const tc_pattern *p, tc_weights w, const void *s, int R,
                          const void *const *factors, int mode, const void *rhs, double lambda,
                          tc_prec prec, void *out, int8_t *row_status, tc_stream_t stream) {
    if (!p || !rank_ok(R) || !out || !rhs || mode < 0 || mode >= p->order) return TC_ERR_ARG;
    if (!factors_ok(factors, mode) || check_weights(p, w, s) != TC_OK) return TC_ERR_ARG;
    const int form = prec & ~(TC_PREC_CHOL32 | TC_PREC_REFINE2);
    if (form != TC_PREC_FP32 && form != TC_PREC_TF32_REFINE && form != TC_PREC_BF16_REFINE &&
        form != TC_PREC_FP32_REFINE)
        return TC_ERR_ARG;
    tc_status rc = launch_solve_factor(p, w, s, R, factors, mode, rhs, lambda, prec, out,
                                       row_status, 0, TC_LOSS_LS, nullptr, (cudaStream_t)stream);
    return rc != TC_OK ? rc : launch_status();
}

tc_status tc_als_update(const tc_pattern *p, int R, const void *const *factors, int mode,
                        double lambda, tc_prec prec, void *out, int8_t *row_status,
                        tc_stream_t stream) {
    if (!p || !rank_ok(R) || !out || mode < 0 || mode >= p->order) return TC_ERR_ARG;
    if (!factors_ok(factors, mode)) return TC_ERR_ARG;
    if (!p->has_vals && p->nnz > 0) return TC_ERR_ARG;
    const int form = prec & ~(TC_PREC_CHOL32 | TC_PREC_REFINE2);
    if (form != TC_PREC_FP32 && form != TC_PREC_TF32_REFINE && form != TC_PREC_BF16_REFINE &&
        form != TC_PREC_FP32_REFINE)
        return TC_ERR_ARG;
    tc_status rc = launch_als_update(p, R, factors, mode, lambda, prec, out, row_status,
                                     (cudaStream_t)stream);
    return rc != TC_OK ? rc : launch_status();
}

tc_status tc_loss_grad(const tc_pattern *p, tc_loss loss, int R, const void *const *factors,
                       double lambda, double *loss_out, void *const *grads, tc_stream_t stream) {
    if (!p || !rank_ok(R) || !factors_ok(factors, -1)) return TC_ERR_ARG;
    if (loss < TC_LOSS_LS || loss > TC_LOSS_POISSON_ID) return TC_ERR_ARG;
    if (!p->has_vals && p->nnz > 0) return TC_ERR_ARG;
    tc_status rc = launch_loss_grad(p, loss, R, factors, lambda, loss_out, grads,
                                    (cudaStream_t)stream);
    return rc != TC_OK ? rc : launch_status();
}

static tc_status hessian_matvec(const tc_pattern *p, tc_loss loss, int R,
                                const void *const *factors, const void *const *x, double lambda,
                                void *const *y, int full_newton, tc_stream_t stream) {
    if (!p || !rank_ok(R) || !factors_ok(factors, -1) || !factors_ok(x, -1) || !y)
        return TC_ERR_ARG;
    if (loss < TC_LOSS_LS || loss > TC_LOSS_POISSON_ID) return TC_ERR_ARG;
    if (!p->has_vals && p->nnz > 0) return TC_ERR_ARG;
    for (int n = 0; n < TC_ORDER; ++n) {
        if (!y[n]) return TC_ERR_ARG;
        for (int m = 0; m < TC_ORDER; ++m)
            if (y[n] == x[m]) return TC_ERR_ARG;
    }
    tc_status rc = launch_ggn_matvec(p, loss, R, factors, x, lambda, y, nullptr, 1, full_newton,
                                     (cudaStream_t)stream);
    return rc != TC_OK ? rc : launch_status();
}

tc_status tc_ggn_matvec(const tc_pattern *p, tc_loss loss, int R, const void *const *factors,
                        const void *const *x, double lambda, void *const *y, tc_stream_t stream) {
    return hessian_matvec(p, loss, R, factors, x, lambda, y, 0, stream);
}

tc_status tc_newton_matvec(const tc_pattern *p, tc_loss loss, int R, const void *const *factors,
                           const void *const *x, double lambda, void *const *y,
                           tc_stream_t stream) {
    return hessian_matvec(p, loss, R, factors, x, lambda, y, 1, stream);
}

}  // extern "C"
