// Solve Factor (Sec. 3.4 with the normal equations of Sec. 2.2) and the
// block-diagonal Gauss-Newton preconditioner (Sec. 2.5), which is the same
// per-row system with weights phi'' and regularization 2 lambda.
//
// One warp owns one row i of the mode.  It streams the row's nonzeros in steps
// of NG, forms h_e = hadamard of the other modes' rows with G lanes per
// nonzero, stages h_e and its weight in shared memory, and accumulates the
// R x R Gram sum_e s_e h_e h_e^T in registers (each lane owns a block of
// entries).  The Gram is then moved to shared memory in FP64, lambda is added
// to the diagonal, and an unpivoted Cholesky factorization and the two
// triangular solves run in FP64 with the lanes parallel over rows.
#include "internal.cuh"

namespace tc {

template <typename T>
struct SolveParams {
    const int64_t *row_ptr;       // I_d + 1
    int64_t I;
    const int32_t *c1, *c2;       // other modes' indices in this mode's order
    Weights<T> w;
    int use_d2;                   // weights phi''(t, <a_i, h_e>) of `loss`
    int loss;
    const T *t;                   // values in this mode's order (for use_d2)
    const T *Ad, *A1, *A2;
    const T *rhs;                 // I_d x R (solve mode)
    T *out;                       // I_d x R (solve mode)
    T *pinv;                      // I_d x R x R inverses (preconditioner mode) or null
    int8_t *row_status;
    double lambda;
    int R;
    int *status;
};

// Gram ownership: LPR lanes share one Gram row, each lane owns RPL rows and
// CPL consecutive columns.
template <int RT>
struct GramLay {
    static constexpr int LPR = RT >= 32 ? 1 : 32 / RT;
    static constexpr int RPL = RT >= 32 ? RT / 32 : 1;
    static constexpr int CPL = RT / LPR;
};

template <typename T, int RT>
struct SolveSmem {
    static constexpr int NG = Lay<T, RT>::NG;
    // per warp: h buffer, weights, FP64 system, FP64 right-hand side; the
    // preconditioner variant also holds the FP64 inverse
    static constexpr size_t h_bytes = sizeof(T) * NG * RT;
    static constexpr size_t w_bytes = sizeof(T) * NG;
    static constexpr size_t s_off = ((h_bytes + w_bytes + 15) / 16) * 16;
    static constexpr size_t per_warp = s_off + sizeof(double) * (RT * RT + RT);
    static constexpr size_t per_warp_inv = per_warp + sizeof(double) * RT * RT;
};

template <typename T, int RT, bool VEC>
__global__ void solve_kernel(const SolveParams<T> P) {
    using L = Lay<T, RT>;
    using GL = GramLay<RT>;
    using SM = SolveSmem<T, RT>;
    constexpr int V = L::V, G = L::G, NG = L::NG;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, g = lane / G, lg = lane % G;
    const int wib = threadIdx.x >> 5;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= P.I) return;
    unsigned char *wbase = smem_raw + (size_t)wib * (P.pinv ? SM::per_warp_inv : SM::per_warp);
    T *hs = reinterpret_cast<T *>(wbase);
    T *ws = hs + NG * RT;
    double *S = reinterpret_cast<double *>(wbase + SM::s_off);
    double *bv = S + RT * RT;
    const int R = P.R;

    const int r0 = (lane / GL::LPR) * GL::RPL;
    const int cb = (lane % GL::LPR) * GL::CPL;
    T acc[GL::RPL][GL::CPL];
#pragma unroll
    for (int a = 0; a < GL::RPL; ++a)
#pragma unroll
        for (int b = 0; b < GL::CPL; ++b) acc[a][b] = T(0);

    const int64_t rs = __ldg(P.row_ptr + i), re = __ldg(P.row_ptr + i + 1);
    T arow[V];
    if (P.use_d2) load_slice<T, V, VEC>(arow, P.Ad, i, R, lg);

    for (int64_t base = rs; base < re; base += NG) {
        const int64_t q = base + g;
        const bool valid = q < re;
        const int64_t qq = valid ? q : re - 1;
        T b[V], e[V];
        load_slice<T, V, VEC>(b, P.A1, __ldcs(P.c1 + qq), R, lg);
        load_slice<T, V, VEC>(e, P.A2, __ldcs(P.c2 + qq), R, lg);
        T h[V];
#pragma unroll
        for (int t = 0; t < V; ++t) h[t] = b[t] * e[t];
        T s;
        if (P.use_d2) {
            T part = T(0);
#pragma unroll
            for (int t = 0; t < V; ++t) part += arow[t] * h[t];
            const T m = group_sum<G>(part);
            T phi, d1, d2;
            bool ok = true;
            loss_terms(P.loss, __ldcs(P.t + qq), m, phi, d1, d2, ok);
            if (!ok && valid) record_error(P.status, TC_ERR_DOMAIN);
            s = d2;
        } else {
            s = weight_at(P.w, qq);
        }
        if (!valid) s = T(0);
#pragma unroll
        for (int t = 0; t < V; ++t) hs[g * RT + lg * V + t] = h[t];
        if (lg == 0) ws[g] = s;
        __syncwarp();
#pragma unroll 2
        for (int gg = 0; gg < NG; ++gg) {
            const T wgt = ws[gg];
            const T *hv = hs + gg * RT;
#pragma unroll
            for (int a = 0; a < GL::RPL; ++a) {
                const T hr = wgt * hv[r0 + a];
#pragma unroll
                for (int bb = 0; bb < GL::CPL; ++bb) acc[a][bb] += hr * hv[cb + bb];
            }
        }
        __syncwarp();
    }

    // Gram -> FP64 system in shared memory, plus lambda I
#pragma unroll
    for (int a = 0; a < GL::RPL; ++a)
#pragma unroll
        for (int bb = 0; bb < GL::CPL; ++bb) S[(r0 + a) * RT + cb + bb] = (double)acc[a][bb];
    __syncwarp();
    for (int r = lane; r < R; r += 32) {
        S[r * RT + r] += P.lambda;
        if (!P.pinv) bv[r] = (double)P.rhs[i * (int64_t)R + r];
    }
    __syncwarp();

    // unpivoted Cholesky, right-looking, lanes over rows
    bool ok = true;
    for (int j = 0; j < R; ++j) {
        const double d = S[j * RT + j];
        if (!(d > 0.0)) {
            ok = false;
            break;
        }
        const double ljj = sqrt(d);
        __syncwarp();
        for (int r = j + 1 + lane; r < R; r += 32) S[r * RT + j] /= ljj;
        if (lane == 0) S[j * RT + j] = ljj;
        __syncwarp();
        for (int r = j + 1 + lane; r < R; r += 32) {
            const double lrj = S[r * RT + j];
            for (int k = j + 1; k <= r; ++k) S[r * RT + k] -= lrj * S[k * RT + j];
        }
        __syncwarp();
    }
    ok = __all_sync(FULL, ok);
    if (!ok) {
        if (lane == 0) {
            record_error(P.status, TC_ERR_NOT_SPD);
            if (P.row_status) P.row_status[i] = 1;
        }
        if (P.pinv) {  // an identity block keeps the preconditioner defined
            T *Po = P.pinv + i * (int64_t)R * R;
            for (int q = lane; q < R * R; q += 32) Po[q] = (q / R == q % R) ? T(1) : T(0);
        }
        return;
    }
    if (lane == 0 && P.row_status) P.row_status[i] = 0;

    if (P.pinv) {
        // (L L^T)^-1 column by column in FP64: lane c solves L L^T y = e_c
        double *Y = bv + RT;
        for (int c = lane; c < R; c += 32) {
            for (int r = 0; r < R; ++r) {
                double v = (r == c) ? 1.0 : 0.0;
                for (int k = c; k < r; ++k) v -= S[r * RT + k] * Y[k * RT + c];
                Y[r * RT + c] = r < c ? 0.0 : v / S[r * RT + r];
            }
            for (int r = R - 1; r >= 0; --r) {
                double v = Y[r * RT + c];
                for (int k = r + 1; k < R; ++k) v -= S[k * RT + r] * Y[k * RT + c];
                Y[r * RT + c] = v / S[r * RT + r];
            }
        }
        __syncwarp();
        T *Po = P.pinv + i * (int64_t)R * R;
        for (int q = lane; q < R * R; q += 32) Po[q] = (T)Y[(q / R) * RT + q % R];
        return;
    }
    // L y = b, then L^T x = y
    for (int j = 0; j < R; ++j) {
        const double yj = bv[j] / S[j * RT + j];
        __syncwarp();
        for (int r = j + 1 + lane; r < R; r += 32) bv[r] -= S[r * RT + j] * yj;
        if (lane == 0) bv[j] = yj;
        __syncwarp();
    }
    for (int j = R - 1; j >= 0; --j) {
        const double xj = bv[j] / S[j * RT + j];
        __syncwarp();
        for (int r = lane; r < j; r += 32) bv[r] -= S[j * RT + r] * xj;
        if (lane == 0) bv[j] = xj;
        __syncwarp();
    }
    for (int r = lane; r < R; r += 32) P.out[i * (int64_t)R + r] = (T)bv[r];
}

template <typename T, int RT, bool VEC>
static tc_status launch_solve_rt(const SolveParams<T> &P, cudaStream_t st) {
    using SM = SolveSmem<T, RT>;
    const int warps = RT >= 64 ? 2 : 4;
    const size_t smem = (P.pinv ? SM::per_warp_inv : SM::per_warp) * warps;
    auto kern = solve_kernel<T, RT, VEC>;
    if (smem > 48 * 1024) TC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)smem));
    const int64_t blocks = (P.I + warps - 1) / warps;
    kern<<<(unsigned)blocks, warps * 32, smem, st>>>(P);
    count_launch();
    return TC_OK;
}

template <typename T>
static tc_status solve_t(const tc_pattern *p, tc_weights w, const void *s, int R,
                         const void *const *A, int mode, const void *rhs, double lambda,
                         void *out, int8_t *row_status, int use_d2, tc_loss loss, void *pinv,
                         cudaStream_t st) {
    const ModeData &md = p->md[mode];
    int o1, o2;
    other_modes(mode, o1, o2);
    SolveParams<T> P{};
    P.row_ptr = md.row_ptr;
    P.I = p->dims[mode];
    P.c1 = md.cols[0];
    P.c2 = md.cols[1];
    P.use_d2 = use_d2;
    P.loss = loss;
    P.t = (const T *)md.vals;
    P.Ad = (const T *)A[mode];
    P.A1 = (const T *)A[o1];
    P.A2 = (const T *)A[o2];
    P.rhs = (const T *)rhs;
    P.out = (T *)out;
    P.pinv = (T *)pinv;
    P.row_status = row_status;
    P.lambda = lambda;
    P.R = R;
    P.status = p->status;
    if (!use_d2) {
        P.w.kind = (int)w;
        P.w.s = nullptr;
        P.w.to0 = nullptr;
        if (w == TC_W_VALUES) P.w.s = (const T *)md.vals;
        else if (w == TC_W_ARRAY) {
            P.w.s = (const T *)s;
            if (mode != 0) P.w.to0 = md.to0;
        }
    }
    const int tier = rank_tier(R);
    const bool vec = vec_ok(R, tier, sizeof(T)) && aligned16({A[o1], A[o2]}) &&
                     (!use_d2 || aligned16({A[mode]}));
    switch (tier) {
        case 8: return vec ? launch_solve_rt<T, 8, true>(P, st) : launch_solve_rt<T, 8, false>(P, st);
        case 16: return vec ? launch_solve_rt<T, 16, true>(P, st) : launch_solve_rt<T, 16, false>(P, st);
        case 32: return vec ? launch_solve_rt<T, 32, true>(P, st) : launch_solve_rt<T, 32, false>(P, st);
        default: return vec ? launch_solve_rt<T, 64, true>(P, st) : launch_solve_rt<T, 64, false>(P, st);
    }
}

tc_status launch_solve_factor(const tc_pattern *p, tc_weights w, const void *s, int R,
                              const void *const *A, int mode, const void *rhs, double lambda,
                              void *out, int8_t *row_status, int use_loss_d2, tc_loss loss,
                              void *pinv_out, cudaStream_t st) {
    if (p->dtype == TC_F64)
        return solve_t<double>(p, w, s, R, A, mode, rhs, lambda, out, row_status, use_loss_d2,
                               loss, pinv_out, st);
    return solve_t<float>(p, w, s, R, A, mode, rhs, lambda, out, row_status, use_loss_d2, loss,
                          pinv_out, st);
}

}  // namespace tc
