// Preconditioned conjugate gradients on the Gauss-Newton system (Sec. 2.5):
// implicit matrix-vector products, the block-diagonal preconditioner applied
// through the per-row Cholesky factors, FP64 inner products and step lengths
// kept on the device, and the fixed-count loop captured once in a CUDA graph.
#include "internal.cuh"

#include <new>

namespace tc {

// device scalars of one solve
enum { S_RZ = 0, S_PAP = 1, S_RZNEW = 2, S_STOP = 3, S_BETA = 4, S_COUNT = 8 };

// Offset of entry (i, e) of the direction inside the interleaved buffer (axv
// = chunk length V of the factor / direction interleave), or of a plain I x R
// array (axv = 0).
__device__ __forceinline__ int64_t dir_index(int64_t i, int e, int R, int axv) {
    if (!axv) return i * R + e;
    return i * 2 * R + (e / axv) * 2 * axv + axv + e % axv;
}

// The per-mode vectors of one solve; the rows of the three modes are numbered
// consecutively (mode d owns rows rows[d] .. rows[d+1]-1) so that one launch
// covers all modes.
template <typename T>
struct CGModes {
    const T *pinv[TC_ORDER];
    T *x[TC_ORDER], *r[TC_ORDER], *z[TC_ORDER], *p[TC_ORDER], *Ap[TC_ORDER];
    int64_t rows[TC_ORDER + 1];
    int axv;
};

__device__ __forceinline__ int mode_of(const int64_t (&rows)[TC_ORDER + 1], int64_t g) {
    return (g >= rows[1]) + (g >= rows[2]);
}

// mode == 0: z = P^-1 r and scal[acc] += r.z   (scal may be null: no dot)
// mode == 1: alpha = rz / pAp; x += alpha p; r -= alpha Ap; z = P^-1 r; scal[acc] += r.z
// P^-1 is the stored per-row inverse of the diagonal block (pinv, R x R per
// row); pinv == null means P = I.  LR lanes own one row (LR a power of two
// >= R/2, at most 32), each lane one or two of its entries; a warp takes 32/LR
// rows at a time.
template <typename T, int LR>
__global__ void __launch_bounds__(256) cg_update_kernel(int mode, int R, const CGModes<T> M,
                                                        double *scal, int acc, int *status) {
    constexpr int RPW = 32 / LR;           // rows per warp
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int l = lane % LR, slot = lane / LR, base_lane = slot * LR;
    double alpha = 0.0;
    if (mode == 1) {
        const double rz = scal[S_RZ], pap = scal[S_PAP];
        const bool stopped = scal[S_STOP] != 0.0;
        if (!stopped && rz != 0.0) {
            if (pap > 0.0 && isfinite(pap)) alpha = rz / pap;
            else if (blockIdx.x == 0 && threadIdx.x == 0) {
                record_error(status, TC_ERR_BREAKDOWN);
                scal[S_STOP] = 1.0;
            }
        }
    }
    double dot = 0.0;
    const int64_t total = M.rows[TC_ORDER];
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t groups = (total + RPW - 1) / RPW;
    for (int64_t gi = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; gi < groups; gi += nwarps) {
        const int64_t grow = gi * RPW + slot;
        const bool row_ok = grow < total;
        const int d = row_ok ? mode_of(M.rows, grow) : 0;
        const int64_t i = row_ok ? grow - M.rows[d] : 0;
        const int64_t off = i * (int64_t)R;
        T *x = M.x[d], *r = M.r[d], *z = M.z[d];
        const T *p = M.p[d], *Ap = M.Ap[d];
        // this lane's entries e0 = l and e1 = l + LR of the row
        const int e0 = l, e1 = l + LR;
        T r0 = T(0), r1 = T(0);
        if (row_ok && e0 < R) {
            r0 = r[off + e0];
            if (mode == 1) {
                x[off + e0] = (T)((double)x[off + e0] + alpha * (double)p[dir_index(i, e0, R, M.axv)]);
                r0 = (T)((double)r0 - alpha * (double)Ap[off + e0]);
                r[off + e0] = r0;
            }
        }
        if (row_ok && e1 < R) {
            r1 = r[off + e1];
            if (mode == 1) {
                x[off + e1] = (T)((double)x[off + e1] + alpha * (double)p[dir_index(i, e1, R, M.axv)]);
                r1 = (T)((double)r1 - alpha * (double)Ap[off + e1]);
                r[off + e1] = r1;
            }
        }
        T z0 = r0, z1 = r1;
        const T *pinv = M.pinv[d];
        if (pinv) {
            const T *Pi = pinv + i * (int64_t)R * R;
            z0 = T(0);
            z1 = T(0);
            for (int c = 0; c < R; ++c) {
                const T rc = __shfl_sync(0xffffffffu, c < LR ? r0 : r1, base_lane + (c % LR));
                if (row_ok && e0 < R) z0 += Pi[e0 * R + c] * rc;
                if (row_ok && e1 < R) z1 += Pi[e1 * R + c] * rc;
            }
        }
        if (row_ok && e0 < R) {
            z[off + e0] = z0;
            dot += (double)r0 * (double)z0;
        }
        if (row_ok && e1 < R) {
            z[off + e1] = z1;
            dot += (double)r1 * (double)z1;
        }
    }
    if (scal) block_add(dot, scal + acc);
}

// p = z + beta p (beta from the scalars; beta == 0 takes p = z) and the start
// of the next product: Ap = 2 lambda p, scal[S_PAP] += 2 lambda p.p
template <typename T>
__global__ void cg_dir_kernel(int R, const CGModes<T> M, T two_lambda, double *scal) {
    const double beta = scal[S_BETA];
    const int64_t n = M.rows[TC_ORDER] * R;
    double acc = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = q / R;
        const int e = (int)(q - g * R);
        const int d = mode_of(M.rows, g);
        const int64_t i = g - M.rows[d];
        const int64_t pi = dir_index(i, e, R, M.axv);
        T *p = M.p[d];
        const T zv = M.z[d][i * R + e];
        const T pn = beta != 0.0 ? (T)((double)zv + beta * (double)p[pi]) : zv;
        p[pi] = pn;
        const T y = two_lambda * pn;
        M.Ap[d][i * R + e] = y;
        acc += (double)y * (double)pn;
    }
    block_add(acc, scal + S_PAP);
}

// Between iterations: record r.z, beta = rz_new / rz, rz = rz_new, clear the sums.
__global__ void cg_scalar_kernel(double *scal, double *rz_hist, int slot, int first) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const double rz_new = scal[S_RZNEW], rz = scal[S_RZ];
        if (rz_hist) rz_hist[slot] = rz_new;
        scal[S_BETA] = (!first && rz != 0.0) ? rz_new / rz : 0.0;
        scal[S_RZ] = rz_new;
        scal[S_PAP] = 0.0;
        scal[S_RZNEW] = 0.0;
        if (first) scal[S_STOP] = 0.0;
    }
}

// y = a x + b y (elementwise)
template <typename T>
__global__ void axpby_kernel(int64_t n, T a, const T *__restrict__ x, T b, T *y) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        y[q] = a * x[q] + b * y[q];
}

// out (+)= sum x_i y_i in FP64 (one atomic per warp).
template <typename T>
__global__ void dot_kernel(int64_t n, const T *__restrict__ x, const T *__restrict__ y,
                           double *out) {
    double acc = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        acc += (double)x[q] * (double)y[q];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(out, acc);
}

// Interleaved buffer from a factor (part 0) or a direction (part 1).
template <typename T>
__global__ void ax_fill_kernel(T *__restrict__ ax, const T *__restrict__ src, int64_t I, int R,
                               int axv, int part) {
    const int64_t n = I * R;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / R;
        const int e = (int)(q - i * R);
        ax[i * 2 * R + (e / axv) * 2 * axv + part * axv + e % axv] = src[q];
    }
}

}  // namespace tc

using namespace tc;

struct tc_cg {
    const tc_pattern *p = nullptr;
    tc_loss loss = TC_LOSS_LS;
    int R = 0;
    void *A[TC_ORDER] = {nullptr, nullptr, nullptr};
    double lambda = 0.0;
    int precond = 1;
    int full_newton = 0;          // iterate with the full Hessian instead of Gauss-Newton
    void *pinv[TC_ORDER] = {nullptr, nullptr, nullptr};
    void *r[TC_ORDER] = {}, *z[TC_ORDER] = {}, *pv[TC_ORDER] = {}, *Ap[TC_ORDER] = {};
    void *grad[TC_ORDER] = {}, *dx[TC_ORDER] = {};
    void *ax[TC_ORDER] = {};      // interleaved factor / direction rows (vector path)
    int axv = 0;                  // interleave chunk length, 0 = plain direction buffers
    double *scal = nullptr;
    cudaStream_t own = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // the preconditioner's blocks are factored concurrently, one mode per stream
    cudaStream_t side[TC_ORDER] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[TC_ORDER] = {};
    // cached graph
    cudaGraphExec_t exec = nullptr;
    const void *key_b[TC_ORDER] = {}, *key_dx[TC_ORDER] = {};
    int key_iters = -1;
    double *key_rz = nullptr;
    int64_t graph_launches = 0;
};

namespace tc {

static int sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

template <typename T>
static CGModes<T> cg_modes(tc_cg *cg) {
    CGModes<T> M;
    M.rows[0] = 0;
    for (int d = 0; d < TC_ORDER; ++d) {
        M.pinv[d] = cg->precond ? (const T *)cg->pinv[d] : nullptr;
        M.x[d] = (T *)cg->dx[d];
        M.r[d] = (T *)cg->r[d];
        M.z[d] = (T *)cg->z[d];
        M.p[d] = (T *)(cg->axv ? cg->ax[d] : cg->pv[d]);
        M.Ap[d] = (T *)cg->Ap[d];
        M.rows[d + 1] = M.rows[d] + cg->p->dims[d];
    }
    M.axv = cg->axv;
    return M;
}

template <typename T, int LR>
static void launch_update_lr(int mode, int R, const CGModes<T> &M, double *scal, int acc,
                             int *status, cudaStream_t st) {
    constexpr int RPW = 32 / LR;
    const int64_t groups = (M.rows[TC_ORDER] + RPW - 1) / RPW;
    int64_t blocks = (groups + 7) / 8;
    if (blocks > 4LL * sms()) blocks = 4LL * sms();
    if (blocks < 1) blocks = 1;
    cg_update_kernel<T, LR><<<(unsigned)blocks, 256, 0, st>>>(mode, R, M, scal, acc, status);
    count_launch();
}

template <typename T>
static void launch_update(int mode, int R, const CGModes<T> &M, double *scal, int acc, int *status,
                          cudaStream_t st) {
    if (R <= 2) launch_update_lr<T, 1>(mode, R, M, scal, acc, status, st);
    else if (R <= 4) launch_update_lr<T, 2>(mode, R, M, scal, acc, status, st);
    else if (R <= 8) launch_update_lr<T, 4>(mode, R, M, scal, acc, status, st);
    else if (R <= 16) launch_update_lr<T, 8>(mode, R, M, scal, acc, status, st);
    else if (R <= 32) launch_update_lr<T, 16>(mode, R, M, scal, acc, status, st);
    else launch_update_lr<T, 32>(mode, R, M, scal, acc, status, st);
}

template <typename T>
static void launch_dir(tc_cg *cg, const CGModes<T> &M, cudaStream_t st) {
    const int64_t n = M.rows[TC_ORDER] * cg->R;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8LL * sms()) blocks = 8LL * sms();
    if (blocks < 1) blocks = 1;
    cg_dir_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(cg->R, M, (T)(2.0 * cg->lambda), cg->scal);
    count_launch();
}

template <typename T>
static void enqueue_ax_fill(tc_cg *cg, const void *const *src, int part, cudaStream_t st) {
    for (int d = 0; d < TC_ORDER; ++d) {
        const int64_t n = cg->p->dims[d] * cg->R;
        int64_t blocks = (n + 255) / 256;
        if (blocks > 8LL * sms()) blocks = 8LL * sms();
        if (blocks < 1) blocks = 1;
        ax_fill_kernel<T><<<(unsigned)blocks, 256, 0, st>>>((T *)cg->ax[d], (const T *)src[d],
                                                           cg->p->dims[d], cg->R, cg->axv, part);
        count_launch();
    }
}

// Enqueues a full solve of `iters` iterations on st (graph-capturable: no
// host synchronization, no allocation).  dx receives the solution; the
// right-hand side is in b.  Per iteration: the three mode passes of the
// product, one update launch, one scalar launch, one direction launch.
template <typename T>
static tc_status enqueue_solve(tc_cg *cg, const void *const *b, void *const *dx, int iters,
                               double *rz_out, cudaStream_t st) {
    const tc_pattern *p = cg->p;
    const size_t es = sizeof(T);
    void *save_dx[TC_ORDER];
    for (int d = 0; d < TC_ORDER; ++d) {
        save_dx[d] = cg->dx[d];
        cg->dx[d] = dx[d];
        const size_t bytes = (size_t)p->dims[d] * cg->R * es;
        TC_CUDA(cudaMemsetAsync(dx[d], 0, bytes, st));
        TC_CUDA(cudaMemcpyAsync(cg->r[d], b[d], bytes, cudaMemcpyDeviceToDevice, st));
    }
    const CGModes<T> M = cg_modes<T>(cg);
    for (int d = 0; d < TC_ORDER; ++d) cg->dx[d] = save_dx[d];
    TC_CUDA(cudaMemsetAsync(cg->scal, 0, sizeof(double) * S_COUNT, st));
    if (cg->axv) enqueue_ax_fill<T>(cg, (const void *const *)cg->A, 0, st);  // fixed during the solve
    launch_update<T>(0, cg->R, M, cg->scal, S_RZNEW, p->status, st);          // z0 = P^-1 r0, r0.z0
    cg_scalar_kernel<<<1, 32, 0, st>>>(cg->scal, rz_out, 0, 1);               // beta = 0
    count_launch();
    launch_dir<T>(cg, M, st);                                                 // p0 = z0, Ap = 2 lambda p0
    for (int it = 0; it < iters; ++it) {
        tc_status rc =
            cg->axv ? launch_ggn_matvec_ax(p, cg->loss, cg->R, (const void *const *)cg->ax, cg->lambda,
                                           cg->Ap, cg->scal + S_PAP, 0, cg->full_newton, st)
                    : launch_ggn_matvec(p, cg->loss, cg->R, (const void *const *)cg->A,
                                        (const void *const *)cg->pv, cg->lambda, cg->Ap,
                                        cg->scal + S_PAP, 0, cg->full_newton, st);
        if (rc != TC_OK) return rc;
        launch_update<T>(1, cg->R, M, cg->scal, S_RZNEW, p->status, st);
        cg_scalar_kernel<<<1, 32, 0, st>>>(cg->scal, rz_out, it + 1, 0);
        count_launch();
        if (it + 1 < iters) launch_dir<T>(cg, M, st);
    }
    return TC_OK;
}

static void free_cg(tc_cg *cg) {
    if (!cg) return;
    for (int d = 0; d < TC_ORDER; ++d) {
        cudaFree(cg->pinv[d]);
        cudaFree(cg->r[d]);
        cudaFree(cg->z[d]);
        cudaFree(cg->pv[d]);
        cudaFree(cg->Ap[d]);
        cudaFree(cg->grad[d]);
        cudaFree(cg->dx[d]);
        cudaFree(cg->ax[d]);
    }
    cudaFree(cg->scal);
    if (cg->exec) cudaGraphExecDestroy(cg->exec);
    if (cg->own) cudaStreamDestroy(cg->own);
    if (cg->ev_in) cudaEventDestroy(cg->ev_in);
    if (cg->ev_out) cudaEventDestroy(cg->ev_out);
    for (int d = 0; d < TC_ORDER; ++d) {
        if (cg->side[d]) cudaStreamDestroy(cg->side[d]);
        if (cg->ev_join[d]) cudaEventDestroy(cg->ev_join[d]);
    }
    if (cg->ev_fork) cudaEventDestroy(cg->ev_fork);
    delete cg;
}

// The preconditioner's three diagonal blocks are independent and each leaves
// most of the GPU idle (the R <= 32 factorization keeps a few warps per SM),
// so mode d is factored on side[d], forked from `st` and joined back into it;
// `work` runs on `st` meanwhile (the gradient, in a Gauss-Newton step).
// With_grad: each block's Gram pass also writes the gradient's MTTKRP(phi')
// of its mode into cg->grad and mode 0's adds sum phi into loss_acc (may be
// null); see launch_precond_grad.
template <typename F>
static tc_status setup_forked(tc_cg *cg, cudaStream_t st, F &&work, bool with_grad = false,
                              double *loss_acc = nullptr) {
    if (!cg->precond) return work();
    TC_CUDA(cudaEventRecord(cg->ev_fork, st));
    for (int d = 0; d < TC_ORDER; ++d) TC_CUDA(cudaStreamWaitEvent(cg->side[d], cg->ev_fork, 0));
    tc_status rc = TC_OK;
    for (int d = 0; d < TC_ORDER && rc == TC_OK; ++d)
        rc = with_grad
                 ? launch_precond_grad(cg->p, cg->R, (const void *const *)cg->A, d, 2.0 * cg->lambda,
                                       cg->loss, cg->pinv[d], cg->grad[d], d == 0 ? loss_acc : nullptr,
                                       cg->side[d])
                 : launch_solve_factor(cg->p, TC_W_ONE, nullptr, cg->R, (const void *const *)cg->A, d,
                                       nullptr, 2.0 * cg->lambda, TC_PREC_FP32, nullptr, nullptr, 1,
                                       cg->loss, cg->pinv[d], cg->side[d]);
    const tc_status rw = rc == TC_OK ? work() : TC_OK;
    // join every side stream, whatever happened above
    for (int d = 0; d < TC_ORDER; ++d) {
        if (cudaEventRecord(cg->ev_join[d], cg->side[d]) != cudaSuccess ||
            cudaStreamWaitEvent(st, cg->ev_join[d], 0) != cudaSuccess)
            rc = rc == TC_OK ? TC_ERR_CUDA : rc;
    }
    if (rc != TC_OK) return rc;
    if (rw != TC_OK) return rw;
    return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

}  // namespace tc

extern "C" {

tc_status tc_cg_create(const tc_pattern *p, tc_loss loss, int R, const void *const *factors,
                       double lambda, int precondition, tc_cg **out) {
    if (!p || !factors || !out || R < 1 || R > TC_MAX_RANK) return TC_ERR_ARG;
    if (loss < TC_LOSS_LS || loss > TC_LOSS_POISSON_ID) return TC_ERR_ARG;
    if (!p->has_vals && p->nnz > 0) return TC_ERR_ARG;
    for (int d = 0; d < TC_ORDER; ++d)
        if (!factors[d]) return TC_ERR_ARG;
    tc_cg *cg = new (std::nothrow) tc_cg();
    if (!cg) return TC_ERR_OOM;
    cg->p = p;
    cg->loss = loss;
    cg->R = R;
    cg->lambda = lambda;
    cg->precond = precondition ? 1 : 0;
    const size_t es = tsize(p->dtype);
    bool ok = true;
    for (int d = 0; d < TC_ORDER && ok; ++d) {
        cg->A[d] = const_cast<void *>(factors[d]);
        const size_t bytes = (size_t)p->dims[d] * R * es;
        ok = ok && cudaMalloc(&cg->r[d], bytes) == cudaSuccess;
        ok = ok && cudaMalloc(&cg->z[d], bytes) == cudaSuccess;
        ok = ok && cudaMalloc(&cg->pv[d], bytes) == cudaSuccess;
        ok = ok && cudaMalloc(&cg->Ap[d], bytes) == cudaSuccess;
        ok = ok && cudaMalloc(&cg->grad[d], bytes) == cudaSuccess;
        ok = ok && cudaMalloc(&cg->dx[d], bytes) == cudaSuccess;
        if (cg->precond)
            ok = ok && cudaMalloc(&cg->pinv[d], es * p->dims[d] * R * R) == cudaSuccess;
    }
    // interleaved factor / direction rows for the matrix-vector product
    if (vec_ok(R, rank_tier(R), es)) {
        cg->axv = (int)(16 / es);
        for (int d = 0; d < TC_ORDER && ok; ++d)
            ok = cudaMalloc(&cg->ax[d], 2 * es * p->dims[d] * R) == cudaSuccess;
    }
    ok = ok && cudaMalloc((void **)&cg->scal, sizeof(double) * S_COUNT) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&cg->own, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&cg->ev_in, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&cg->ev_out, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&cg->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    for (int d = 0; d < TC_ORDER && ok; ++d) {
        ok = cudaStreamCreateWithFlags(&cg->side[d], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&cg->ev_join[d], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        free_cg(cg);
        return TC_ERR_OOM;
    }
    prepare_ggn_matvec_ax();
    *out = cg;
    return TC_OK;
}

tc_status tc_cg_destroy(tc_cg *cg) {
    if (!cg) return TC_ERR_ARG;
    cudaDeviceSynchronize();
    free_cg(cg);
    return TC_OK;
}

tc_status tc_cg_set_hessian(tc_cg *cg, int full_newton) {
    if (!cg || (full_newton != 0 && full_newton != 1)) return TC_ERR_ARG;
    if (cg->full_newton != full_newton) {
        cudaDeviceSynchronize();
        if (cg->exec) {                 // the captured iterations change: capture again
            cudaGraphExecDestroy(cg->exec);
            cg->exec = nullptr;
        }
        cg->full_newton = full_newton;
    }
    return TC_OK;
}

tc_status tc_cg_setup(tc_cg *cg, tc_stream_t stream) {
    if (!cg) return TC_ERR_ARG;
    return setup_forked(cg, (cudaStream_t)stream, [] { return TC_OK; });
}

tc_status tc_cg_precond_apply(tc_cg *cg, const void *const *r, void *const *z,
                              tc_stream_t stream) {
    if (!cg || !r || !z) return TC_ERR_ARG;
    const tc_pattern *p = cg->p;
    for (int d = 0; d < TC_ORDER; ++d)
        if (!r[d] || !z[d]) return TC_ERR_ARG;
    if (p->dtype == TC_F64) {
        CGModes<double> M = cg_modes<double>(cg);
        for (int d = 0; d < TC_ORDER; ++d) {
            M.r[d] = (double *)const_cast<void *>(r[d]);
            M.z[d] = (double *)z[d];
        }
        launch_update<double>(0, cg->R, M, nullptr, 0, p->status, (cudaStream_t)stream);
    } else {
        CGModes<float> M = cg_modes<float>(cg);
        for (int d = 0; d < TC_ORDER; ++d) {
            M.r[d] = (float *)const_cast<void *>(r[d]);
            M.z[d] = (float *)z[d];
        }
        launch_update<float>(0, cg->R, M, nullptr, 0, p->status, (cudaStream_t)stream);
    }
    return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

tc_status tc_cg_solve(tc_cg *cg, const void *const *b, void *const *dx, int iters,
                      double *rz_out, tc_stream_t stream) {
    if (!cg || !b || !dx || iters < 0) return TC_ERR_ARG;
    for (int d = 0; d < TC_ORDER; ++d)
        if (!b[d] || !dx[d]) return TC_ERR_ARG;
    cudaStream_t caller = (cudaStream_t)stream;
    bool same = cg->exec && cg->key_iters == iters && cg->key_rz == rz_out;
    for (int d = 0; d < TC_ORDER && same; ++d) same = cg->key_b[d] == b[d] && cg->key_dx[d] == dx[d];
    if (!same) {
        if (cg->exec) {
            cudaGraphExecDestroy(cg->exec);
            cg->exec = nullptr;
        }
        const int64_t before = g_launches;
        TC_CUDA(cudaStreamBeginCapture(cg->own, cudaStreamCaptureModeThreadLocal));
        tc_status rc = cg->p->dtype == TC_F64
                           ? enqueue_solve<double>(cg, b, dx, iters, rz_out, cg->own)
                           : enqueue_solve<float>(cg, b, dx, iters, rz_out, cg->own);
        cudaGraph_t graph = nullptr;
        cudaError_t ce = cudaStreamEndCapture(cg->own, &graph);
        if (rc != TC_OK || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return rc != TC_OK ? rc : TC_ERR_CUDA;
        }
        ce = cudaGraphInstantiate(&cg->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            cg->exec = nullptr;
            return TC_ERR_CUDA;
        }
        cg->graph_launches = g_launches - before;
        g_launches = before;
        cg->key_iters = iters;
        cg->key_rz = rz_out;
        for (int d = 0; d < TC_ORDER; ++d) {
            cg->key_b[d] = b[d];
            cg->key_dx[d] = dx[d];
        }
    }
    // order the replay after the caller's prior work and the caller's later work after it
    TC_CUDA(cudaEventRecord(cg->ev_in, caller));
    TC_CUDA(cudaStreamWaitEvent(cg->own, cg->ev_in, 0));
    TC_CUDA(cudaGraphLaunch(cg->exec, cg->own));
    TC_CUDA(cudaEventRecord(cg->ev_out, cg->own));
    TC_CUDA(cudaStreamWaitEvent(caller, cg->ev_out, 0));
    count_launch((int)cg->graph_launches);
    return TC_OK;
}

tc_status tc_cg_matvec(tc_cg *cg, const void *const *x, void *const *y, tc_stream_t stream) {
    if (!cg || !x || !y) return TC_ERR_ARG;
    for (int d = 0; d < TC_ORDER; ++d) {
        if (!x[d] || !y[d]) return TC_ERR_ARG;
        for (int e = 0; e < TC_ORDER; ++e)
            if (y[d] == x[e]) return TC_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    tc_status rc;
    if (cg->axv) {
        if (cg->p->dtype == TC_F64) {
            enqueue_ax_fill<double>(cg, (const void *const *)cg->A, 0, st);
            enqueue_ax_fill<double>(cg, x, 1, st);
        } else {
            enqueue_ax_fill<float>(cg, (const void *const *)cg->A, 0, st);
            enqueue_ax_fill<float>(cg, x, 1, st);
        }
        rc = launch_ggn_matvec_ax(cg->p, cg->loss, cg->R, (const void *const *)cg->ax, cg->lambda, y,
                                  nullptr, 1, cg->full_newton, st);
    } else {
        rc = launch_ggn_matvec(cg->p, cg->loss, cg->R, (const void *const *)cg->A, x, cg->lambda, y,
                               nullptr, 1, cg->full_newton, st);
    }
    if (rc != TC_OK) return rc;
    return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

tc_status tc_ggn_step(tc_cg *cg, int iters, double *loss_out, tc_stream_t stream) {
    if (!cg || iters < 0) return TC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const tc_pattern *p = cg->p;
    tc_status rc;
    if (cg->precond && solve_fuses_rhs(p->dtype, cg->R)) {
        // The preconditioner's Gram passes (one per mode, on the side streams)
        // also form MTTKRP(phi') into grad and the loss sum phi, so the gradient
        // costs no pass of its own; the regularizer's share of the loss runs
        // on `st` meanwhile.  Then b = -(MTTKRP(phi') + 2 lambda A) in place.
        if (loss_out) TC_CUDA(cudaMemsetAsync(loss_out, 0, sizeof(double), st));
        rc = setup_forked(
            cg, st,
            [&]() -> tc_status {
                return loss_out ? launch_regularizer(p, cg->R, (const void *const *)cg->A, cg->lambda,
                                                     loss_out, st)
                                : TC_OK;
            },
            true, loss_out);
        if (rc != TC_OK) return rc;
        for (int d = 0; d < TC_ORDER; ++d) {
            const int64_t n = p->dims[d] * cg->R;
            int64_t blocks = (n + 255) / 256;
            if (blocks > 8LL * sms()) blocks = 8LL * sms();
            axpby_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(
                n, (float)(-2.0 * cg->lambda), (const float *)cg->A[d], -1.0f, (float *)cg->grad[d]);
            count_launch();
        }
    } else {
    // the gradient (and b = -grad, in place) on `st` while the preconditioner
    // blocks are factored on the side streams
    rc = setup_forked(cg, st, [&]() -> tc_status {
        const tc_status rg = launch_loss_grad(p, cg->loss, cg->R, (const void *const *)cg->A,
                                              cg->lambda, loss_out, cg->grad, st);
        if (rg != TC_OK) return rg;
        for (int d = 0; d < TC_ORDER; ++d) {
            const int64_t n = p->dims[d] * cg->R;
            int64_t blocks = (n + 255) / 256;
            if (blocks > 8LL * sms()) blocks = 8LL * sms();
            if (p->dtype == TC_F64)
                axpby_kernel<double><<<(unsigned)blocks, 256, 0, st>>>(
                    n, 0.0, (const double *)cg->grad[d], -1.0, (double *)cg->grad[d]);
            else
                axpby_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(
                    n, 0.0f, (const float *)cg->grad[d], -1.0f, (float *)cg->grad[d]);
            count_launch();
        }
        return TC_OK;
    });
    if (rc != TC_OK) return rc;
    }
    // the solution goes to the solver's own buffer dx, then A += dx
    void *dxb[TC_ORDER];
    for (int d = 0; d < TC_ORDER; ++d) dxb[d] = cg->dx[d];
    rc = tc_cg_solve(cg, (const void *const *)cg->grad, dxb, iters, nullptr, stream);
    if (rc != TC_OK) return rc;
    for (int d = 0; d < TC_ORDER; ++d) {
        const int64_t n = p->dims[d] * cg->R;
        int64_t blocks = (n + 255) / 256;
        if (blocks > 8LL * sms()) blocks = 8LL * sms();
        if (p->dtype == TC_F64)
            axpby_kernel<double><<<(unsigned)blocks, 256, 0, st>>>(n, 1.0, (const double *)cg->dx[d],
                                                                  1.0, (double *)cg->A[d]);
        else
            axpby_kernel<float><<<(unsigned)blocks, 256, 0, st>>>(n, 1.0f, (const float *)cg->dx[d],
                                                                 1.0f, (float *)cg->A[d]);
        count_launch();
    }
    return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

// ------------------------------------------------------------------ vector steps
static int64_t vec_blocks(int64_t n) {
    int64_t b = (n + 255) / 256;
    if (b > 8LL * sms()) b = 8LL * sms();
    return b < 1 ? 1 : b;
}

tc_status tc_axpby(tc_dtype dtype, int64_t n, double alpha, const void *x, double beta, void *y,
                   tc_stream_t stream) {
    if ((dtype != TC_F32 && dtype != TC_F64) || n < 0 || (n > 0 && (!x || !y))) return TC_ERR_ARG;
    if (n == 0) return TC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == TC_F64)
        axpby_kernel<double><<<(unsigned)vec_blocks(n), 256, 0, st>>>(n, alpha, (const double *)x,
                                                                     beta, (double *)y);
    else
        axpby_kernel<float><<<(unsigned)vec_blocks(n), 256, 0, st>>>(n, (float)alpha, (const float *)x,
                                                                    (float)beta, (float *)y);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

tc_status tc_dot(tc_dtype dtype, int64_t n, const void *x, const void *y, double *out,
                 int accumulate, tc_stream_t stream) {
    if ((dtype != TC_F32 && dtype != TC_F64) || n < 0 || !out || (n > 0 && (!x || !y)))
        return TC_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (!accumulate) TC_CUDA(cudaMemsetAsync(out, 0, sizeof(double), st));
    if (n == 0) return TC_OK;
    if (dtype == TC_F64)
        dot_kernel<double><<<(unsigned)vec_blocks(n), 256, 0, st>>>(n, (const double *)x,
                                                                   (const double *)y, out);
    else
        dot_kernel<float><<<(unsigned)vec_blocks(n), 256, 0, st>>>(n, (const float *)x,
                                                                  (const float *)y, out);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

}  // extern "C"
