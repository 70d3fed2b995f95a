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
    static constexpr int NG = Lay<T, RT, 32>::NG;
    // per warp: h buffer, weights, FP64 system, FP64 right-hand side; the
    // preconditioner variant also holds the FP64 inverse
    static constexpr size_t h_bytes = sizeof(T) * NG * RT;
    static constexpr size_t w_bytes = sizeof(T) * NG;
    static constexpr size_t s_off = ((h_bytes + w_bytes + 15) / 16) * 16;
    static constexpr size_t per_warp = s_off + sizeof(double) * (RT * RT + RT);
    static constexpr size_t per_warp_inv = per_warp + sizeof(double) * RT * RT;
};

// Accumulates row i's Gram sum_e s_e h_e h_e^T into the lane's block `acc`
// (GramLay ownership).  hs / ws: this warp's staging buffer (NG x RT values,
// NG weights).  The next step's indices are loaded one step ahead.
template <typename T, int RT, bool VEC>
__device__ __forceinline__ void gram_row(const SolveParams<T> &P, int64_t i, T *hs, T *ws,
                                         T (&acc)[GramLay<RT>::RPL][GramLay<RT>::CPL],
                                         int part = 0, int nparts = 1) {
    using L = Lay<T, RT, 32>;
    using GL = GramLay<RT>;
    constexpr int V = L::V, G = L::G, NG = L::NG;
    const int lane = threadIdx.x & 31, g = lane / G, lg = lane % G;
    const int R = P.R;
    const int r0 = (lane / GL::LPR) * GL::RPL;
    const int cb = (lane % GL::LPR) * GL::CPL;
#pragma unroll
    for (int a = 0; a < GL::RPL; ++a)
#pragma unroll
        for (int b = 0; b < GL::CPL; ++b) acc[a][b] = T(0);
    const int64_t rs = __ldg(P.row_ptr + i), re = __ldg(P.row_ptr + i + 1);
    if (rs + (int64_t)part * NG >= re) return;
    T arow[V];
    if (P.use_d2) load_slice<T, V, VEC>(arow, P.Ad, i, R, lg);
    const int64_t stride = (int64_t)nparts * NG;    // this part takes every nparts-th step
    int64_t qn = min(rs + (int64_t)part * NG + g, re - 1);
    int32_t jn = __ldcs(P.c1 + qn), kn = __ldcs(P.c2 + qn);
    for (int64_t base = rs + (int64_t)part * NG; base < re; base += stride) {
        const bool valid = base + g < re;
        const int64_t qq = valid ? base + g : re - 1;
        const int32_t j = jn, k = kn;
        if (base + stride < re) {
            qn = min(base + stride + g, re - 1);
            jn = __ldcs(P.c1 + qn);
            kn = __ldcs(P.c2 + qn);
        }
        T b[V], e[V];
        load_slice<T, V, VEC>(b, P.A1, j, R, lg);
        load_slice<T, V, VEC>(e, P.A2, k, R, lg);
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
}

template <typename T, int RT, bool VEC>
__global__ void solve_kernel(const SolveParams<T> P) {
    using L = Lay<T, RT, 32>;
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
    gram_row<T, RT, VEC>(P, i, hs, ws, acc);

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

// ------------------------------------------------------------------ tensor-core Gram (FP32)
// G_i = H^T diag(s) H on the tensor cores with mma.sync m16n8k8 (TF32 inputs,
// FP32 accumulation).  Each FP32 operand x is split into x_hi = tf32(x) and
// x_lo = tf32(x - x_hi); the product is formed as hi*hi + hi*lo + lo*hi, which
// keeps about 22 significant bits per product (the FP32 FFMA path keeps 24),
// far below the rounding of the FP32 sums themselves.  The h vectors and
// weights of KB nonzeros are staged in shared memory (row stride padded so the
// fragment loads hit distinct banks), then consumed 8 nonzeros (one K chunk)
// at a time.  Output tile (mt, nt) covers Gram rows 16 mt .. 16 mt + 15 and
// columns 8 nt .. 8 nt + 7.
template <int RT>
struct MmaGram {
    static constexpr int KB = 32;                              // staged nonzeros
    static constexpr int STRIDE = RT + (RT == 8 ? 0 : 8);      // floats per staged row
    static constexpr int MT = (RT + 15) / 16;
    static constexpr int NT = RT / 8;
    static constexpr size_t stage_floats = KB * STRIDE + KB;
};

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Accumulates row i's Gram into the warp's mma accumulators d[mt][nt][4].
template <int RT, bool VEC>
__device__ __forceinline__ void gram_row_mma(const SolveParams<float> &P, int64_t i, float *stage,
                                             float (&d)[MmaGram<RT>::MT][MmaGram<RT>::NT][4],
                                             int part = 0, int nparts = 1) {
    using L = Lay<float, RT, 32>;
    using MG = MmaGram<RT>;
    constexpr int V = L::V, G = L::G, NG = L::NG;
    constexpr int KB = MG::KB, S = MG::STRIDE;
    const int lane = threadIdx.x & 31, g = lane / G, lg = lane % G;
    const int gid = lane >> 2, tig = lane & 3;
    const int R = VEC ? RT : P.R;
    float *hs = stage;
    float *ws = stage + KB * S;
#pragma unroll
    for (int mt = 0; mt < MG::MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < MG::NT; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q) d[mt][nt][q] = 0.f;
    const int64_t rs = __ldg(P.row_ptr + i), re = __ldg(P.row_ptr + i + 1);
    if (rs + (int64_t)part * KB >= re) return;
    float arow[V];
    if (P.use_d2) load_slice<float, V, VEC>(arow, P.Ad, i, R, lg);
    // this part takes every nparts-th batch of KB nonzeros
    for (int64_t base = rs + (int64_t)part * KB; base < re; base += (int64_t)nparts * KB) {
        // stage KB nonzeros (h and weight), NG per warp step
#pragma unroll
        for (int st = 0; st < KB / NG; ++st) {
            const int slot = st * NG + g;
            const bool valid = base + slot < re;
            const int64_t qq = valid ? base + slot : re - 1;
            float b[V], e[V], h[V];
            load_slice<float, V, VEC>(b, P.A1, __ldcs(P.c1 + qq), R, lg);
            load_slice<float, V, VEC>(e, P.A2, __ldcs(P.c2 + qq), R, lg);
#pragma unroll
            for (int t = 0; t < V; ++t) h[t] = b[t] * e[t];
            float sw;
            if (P.use_d2) {
                float part = 0.f;
#pragma unroll
                for (int t = 0; t < V; ++t) part += arow[t] * h[t];
                const float m = group_sum<G>(part);
                float phi, d1, d2;
                bool ok = true;
                loss_terms(P.loss, __ldcs(P.t + qq), m, phi, d1, d2, ok);
                if (!ok && valid) record_error(P.status, TC_ERR_DOMAIN);
                sw = d2;
            } else {
                sw = weight_at(P.w, qq);
            }
            if (!valid) sw = 0.f;
#pragma unroll
            for (int t = 0; t < V; ++t) hs[slot * S + lg * V + t] = h[t];
            if (lg == 0) ws[slot] = sw;
        }
        __syncwarp();
#pragma unroll
        for (int kc = 0; kc < KB / 8; ++kc) {
            const int k0 = kc * 8 + tig, k1 = k0 + 4;
            const float w0 = ws[k0], w1 = ws[k1];
#pragma unroll
            for (int mt = 0; mt < MG::MT; ++mt) {
                const int ra = mt * 16 + gid, rb = ra + 8;
                const float x0 = hs[k0 * S + ra], x2 = hs[k1 * S + ra];
                const float x1 = rb < RT ? hs[k0 * S + rb] : 0.f;
                const float x3 = rb < RT ? hs[k1 * S + rb] : 0.f;
                uint32_t ah[4], al[4];
                split_tf32(x0, ah[0], al[0]);
                split_tf32(x1, ah[1], al[1]);
                split_tf32(x2, ah[2], al[2]);
                split_tf32(x3, ah[3], al[3]);
#pragma unroll
                for (int nt = 0; nt < MG::NT; ++nt) {
                    const int cn = nt * 8 + gid;
                    uint32_t bh0, bl0, bh1, bl1;
                    split_tf32(w0 * hs[k0 * S + cn], bh0, bl0);
                    split_tf32(w1 * hs[k1 * S + cn], bh1, bl1);
                    mma_tf32(d[mt][nt], ah, bh0, bh1);
                    mma_tf32(d[mt][nt], ah, bl0, bl1);
                    mma_tf32(d[mt][nt], al, bh0, bh1);
                }
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ two-kernel path, R <= 32
// Kernel A forms the Gram matrices: one block of W warps per row, the warps
// splitting the row's nonzeros (every W-th batch), their partial Grams summed
// in shared memory and written as packed FP64 lower triangles, plus lambda on
// the diagonal, to a scratch buffer.  Kernel B runs the FP64 part with one row
// per lane and RPW rows per warp: the unpivoted Cholesky factorization, then
// either the two triangular solves or the inverse (L L^T)^-1 = L^-T L^-1.  One
// row per lane makes every FP64 instruction do a full warp of useful work, and
// many independent warps overlap the long dependence chains.
//
// Scratch layout (shared by both kernels): row q of the batch keeps packed
// entry e = r (r + 1) / 2 + c at ((q / RPW) * TRI + e) * RPW + q % RPW.
template <typename T, int RT>
struct GramCfg {
    static constexpr int W = 4;
    static constexpr bool MMA = sizeof(T) == 4;               // FP32: tensor-core Gram
    static constexpr int NG = Lay<T, RT, 32>::NG;
    static constexpr size_t stage_elems = MMA ? MmaGram<RT>::stage_floats : (size_t)(NG * RT + NG);
    static constexpr size_t stage_per_warp = ((sizeof(T) * stage_elems + 15) / 16) * 16;
    static constexpr size_t dense_off = W * stage_per_warp;
    static constexpr size_t bytes = dense_off + (size_t)W * RT * RT * sizeof(T);
};

template <typename T, int RT, bool VEC>
__global__ void __launch_bounds__(128) gram_rows_kernel(const SolveParams<T> P, int64_t row0,
                                                        int64_t nrows, int rpw, double *gram) {
    using C = GramCfg<T, RT>;
    using GL = GramLay<RT>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T *stage = reinterpret_cast<T *>(smem_raw + w * C::stage_per_warp);
    T *dense = reinterpret_cast<T *>(smem_raw + C::dense_off);
    T *mine = dense + w * RT * RT;
    const int R = VEC ? RT : P.R;
    const int tri = R * (R + 1) / 2;
    for (int64_t q = blockIdx.x; q < nrows; q += gridDim.x) {
        const int64_t i = row0 + q;
        if constexpr (C::MMA) {
            using MG = MmaGram<RT>;
            float d[MG::MT][MG::NT][4];
            gram_row_mma<RT, VEC>(reinterpret_cast<const SolveParams<float> &>(P), i,
                                  reinterpret_cast<float *>(stage), d, w, C::W);
            const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
            for (int mt = 0; mt < MG::MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < MG::NT; ++nt)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int r = mt * 16 + gid + (e >= 2 ? 8 : 0);
                        const int c = nt * 8 + tig * 2 + (e & 1);
                        if (r < RT) mine[r * RT + c] = d[mt][nt][e];
                    }
        } else {
            T acc[GL::RPL][GL::CPL];
            gram_row<T, RT, VEC>(P, i, stage, stage + C::NG * RT, acc, w, C::W);
            const int r0 = (lane / GL::LPR) * GL::RPL, cb = (lane % GL::LPR) * GL::CPL;
#pragma unroll
            for (int a = 0; a < GL::RPL; ++a)
#pragma unroll
                for (int bb = 0; bb < GL::CPL; ++bb) mine[(r0 + a) * RT + cb + bb] = acc[a][bb];
        }
        __syncthreads();
        double *dst = gram + (q / rpw) * (int64_t)tri * rpw + q % rpw;
        for (int e = threadIdx.x; e < tri; e += blockDim.x) {
            int r = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
            while (r * (r + 1) / 2 > e) --r;
            while ((r + 1) * (r + 2) / 2 <= e) ++r;
            const int c = e - r * (r + 1) / 2;
            double v = 0.0;
#pragma unroll
            for (int ww = 0; ww < C::W; ++ww) v += (double)dense[ww * RT * RT + r * RT + c];
            if (r == c) v += P.lambda;
            dst[(int64_t)e * rpw] = v;
        }
        __syncthreads();
    }
}

template <typename T>
__global__ void __launch_bounds__(32) chol_rows_kernel(const SolveParams<T> P, int64_t row0,
                                                       int64_t nrows, int rpw, const double *gram) {
    extern __shared__ __align__(16) double sh[];
    const int lane = threadIdx.x;
    const int R = P.R, tri = R * (R + 1) / 2;
    const int64_t grp = blockIdx.x;
    double *Tri = sh;
    double *Vv = sh + (int64_t)tri * rpw;
    double *Dinv = Vv + (int64_t)R * rpw;
    const double *src = gram + grp * (int64_t)tri * rpw;
    for (int e = lane; e < tri * rpw; e += 32) Tri[e] = src[e];
    __syncwarp();
    const int slot = lane;
    if (slot >= rpw || grp * rpw + slot >= nrows) return;
    const int64_t i = row0 + grp * rpw + slot;
#define TC_TRI(r, c) Tri[((r) * ((r) + 1) / 2 + (c)) * rpw + slot]
#define TC_VEC(r) Vv[(r) * rpw + slot]
#define TC_DINV(r) Dinv[(r) * rpw + slot]
    bool ok = true;
    for (int j = 0; j < R; ++j) {
        const double dj = TC_TRI(j, j);
        if (!(dj > 0.0)) {
            ok = false;
            break;
        }
        const double ljj = sqrt(dj), inv = 1.0 / ljj;
        TC_TRI(j, j) = ljj;
        TC_DINV(j) = inv;
        for (int r = j + 1; r < R; ++r) TC_TRI(r, j) *= inv;
        for (int r = j + 1; r < R; ++r) {
            const double lrj = TC_TRI(r, j);
            for (int k = j + 1; k <= r; ++k) TC_TRI(r, k) -= lrj * TC_TRI(k, j);
        }
    }
    if (!ok) {
        record_error(P.status, TC_ERR_NOT_SPD);
        if (P.row_status) P.row_status[i] = 1;
        if (P.pinv) {  // an identity block keeps the preconditioner defined
            T *Po = P.pinv + i * (int64_t)R * R;
            for (int q = 0; q < R * R; ++q) Po[q] = (q / R == q % R) ? T(1) : T(0);
        }
        return;
    }
    if (P.row_status) P.row_status[i] = 0;
    if (!P.pinv) {
        for (int r = 0; r < R; ++r) {           // L y = b
            double v = (double)P.rhs[i * (int64_t)R + r];
            for (int k = 0; k < r; ++k) v -= TC_TRI(r, k) * TC_VEC(k);
            TC_VEC(r) = v * TC_DINV(r);
        }
        for (int r = R - 1; r >= 0; --r) {      // L^T x = y
            double v = TC_VEC(r);
            for (int k = r + 1; k < R; ++k) v -= TC_TRI(k, r) * TC_VEC(k);
            TC_VEC(r) = v * TC_DINV(r);
        }
        for (int r = 0; r < R; ++r) P.out[i * (int64_t)R + r] = (T)TC_VEC(r);
        return;
    }
    // L^-1 in place, column by column: for r > j,
    // L^-1[r][j] = -(sum_{k=j}^{r-1} L[r][k] L^-1[k][j]) / L[r][r]; columns > j still hold L.
    for (int j = 0; j < R; ++j) {
        TC_TRI(j, j) = TC_DINV(j);
        for (int r = j + 1; r < R; ++r) {
            double v = 0.0;
            for (int k = j; k < r; ++k) v += TC_TRI(r, k) * TC_TRI(k, j);
            TC_TRI(r, j) = -v * TC_DINV(r);
        }
    }
    // (L L^T)^-1 [r][c] = sum_{k >= max(r, c)} L^-1[k][r] L^-1[k][c]
    T *Po = P.pinv + i * (int64_t)R * R;
    for (int r = 0; r < R; ++r)
        for (int c = 0; c <= r; ++c) {
            double v = 0.0;
            for (int k = r; k < R; ++k) v += TC_TRI(k, r) * TC_TRI(k, c);
            Po[r * R + c] = (T)v;
            Po[c * R + r] = (T)v;
        }
#undef TC_TRI
#undef TC_VEC
#undef TC_DINV
}

template <typename T, int RT, bool VEC>
static tc_status launch_solve_two(const SolveParams<T> &P, cudaStream_t st) {
    using C = GramCfg<T, RT>;
    const int R = P.R, tri = R * (R + 1) / 2;
    const int rpw = RT <= 16 ? 32 : 16;                     // rows per warp in kernel B
    // rows per batch: scratch of at most 256 MB, a multiple of rpw
    int64_t batch = ((int64_t)256 << 20) / ((int64_t)tri * 8);
    batch = batch / rpw * rpw;
    if (batch < rpw) batch = rpw;
    if (batch > P.I) batch = (P.I + rpw - 1) / rpw * rpw;
    double *gram = nullptr;
    TC_CUDA(cudaMallocAsync((void **)&gram, sizeof(double) * tri * batch, st));
    auto ka = gram_rows_kernel<T, RT, VEC>;
    if (C::bytes > 48 * 1024)
        TC_CUDA(cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::bytes));
    const size_t smem_b = sizeof(double) * (size_t)(tri + 2 * R) * rpw;
    auto kb = chol_rows_kernel<T>;
    if (smem_b > 48 * 1024)
        TC_CUDA(cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
    for (int64_t row0 = 0; row0 < P.I; row0 += batch) {
        const int64_t n = min(batch, P.I - row0);
        ka<<<(unsigned)n, C::W * 32, C::bytes, st>>>(P, row0, n, rpw, gram);
        kb<<<(unsigned)((n + rpw - 1) / rpw), 32, smem_b, st>>>(P, row0, n, rpw, gram);
        count_launch(2);
    }
    TC_CUDA(cudaFreeAsync(gram, st));
    return TC_OK;
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
            if (mode != 0) {
                tc_status rc = ensure_to0(p, st);
                if (rc != TC_OK) return rc;
                P.w.to0 = md.to0;
            }
        }
    }
    const int tier = rank_tier(R);
    const bool vec = vec_ok(R, tier, sizeof(T)) && aligned16({A[o1], A[o2]}) &&
                     (!use_d2 || aligned16({A[mode]}));
    switch (tier) {
        case 8: return vec ? launch_solve_two<T, 8, true>(P, st) : launch_solve_two<T, 8, false>(P, st);
        case 16: return vec ? launch_solve_two<T, 16, true>(P, st) : launch_solve_two<T, 16, false>(P, st);
        case 32: return vec ? launch_solve_two<T, 32, true>(P, st) : launch_solve_two<T, 32, false>(P, st);
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
