// Segmented sweeps over one mode's sorted nonzeros: TTTP (Sec. 3.3), MTTKRP
// (Sec. 3.2), the gradient of eq. obj (Table 1, Appendix A) and the
// Gauss-Newton matrix-vector product (Sec. 2.5).
//
// Work decomposition.  Each warp owns a contiguous chunk of the sorted
// nonzeros.  A nonzero is handled by G lanes, each holding V consecutive
// entries (one 16-byte vector) of every factor row it touches, so a warp step
// covers NG = 32/G consecutive nonzeros.  Row membership is decoded from the
// compressed row offsets (nonempty rows only), so no per-nonzero row index is
// stored or read.  Row sums are formed by a segmented scan across the NG
// groups of a step plus a carry between steps; a finished row is written once
// with plain stores, and only the first and last row of a chunk, which other
// chunks may share, are added atomically.
#include "internal.cuh"

#include <atomic>
#include <mutex>
#include <unordered_map>

namespace tc {

// OP_NEWTON: the Gauss-Newton product plus the phi' term of the full Hessian
// (a separate instantiation, so the Gauss-Newton kernel is untouched by it).
enum { OP_MTTKRP = 0, OP_GRAD = 1, OP_GGN = 2, OP_NEWTON = 3 };

template <typename T>
struct SweepParams {
    const int32_t *nz_rows;
    const int64_t *nz_ptr;
    const int64_t *n_ne_dev;      // number of nonempty rows (device)
    int64_t nnz, chunk;
    const int32_t *c1, *c2;       // indices of the two other modes, this mode's order
    Weights<T> w;                 // OP_MTTKRP weights
    const T *t;                   // observed values, this mode's order (GRAD / GGN)
    const T *Ad, *A1, *A2;        // factor of this mode and of the two others
    const T *Xd, *X1, *X2;        // GGN direction blocks
    int R, loss, accumulate;
    T *out;                       // I_d x R (may be null for a loss-only pass)
    double *loss_acc;             // GRAD: += sum phi
    double *dot_acc;              // += sum_rows dot_with[row] . (flushed partial row)
    const T *dot_with;
    int *status;
};

// Per-step inputs of one nonzero group, loaded one step ahead.
template <typename T>
struct StepIn {
    int32_t j, k;
    T t, s;
};

// The warp's chunk-relative views of the nonzero streams.
template <typename T>
struct ChunkStreams {
    const int32_t *c1, *c2;
    const T *t;
    Weights<T> w;
};

template <typename T, int OP>
__device__ __forceinline__ StepIn<T> load_step(const SweepParams<T> &P, const ChunkStreams<T> &S,
                                               int off) {
    StepIn<T> in;
    in.j = __ldcs(S.c1 + off);
    in.k = __ldcs(S.c2 + off);
    if constexpr (OP == OP_MTTKRP) {
        in.s = weight_at(S.w, off);
        in.t = T(0);
    } else {
        in.s = T(0);
        in.t = (OP == OP_GGN && P.loss == TC_LOSS_LS) ? T(0) : __ldcs(S.t + off);
    }
    return in;
}

// Loads lane slices of a factor row and of the matching direction row.  AXL:
// both come from one interleaved buffer whose row holds, for each lane's
// chunk of V entries, the factor chunk followed by the direction chunk (row
// stride 2R), so one 2V-element vector load serves both.
template <typename T, int V, bool VEC, bool AXL>
__device__ __forceinline__ void load_pair(T (&a)[V], T (&x)[V], const T *A, const T *X, int64_t row,
                                          int R, int lg) {
    if constexpr (AXL) {
        T t2[2 * V];
        load_slice<T, 2 * V, VEC>(t2, A, row, 2 * R, lg);
#pragma unroll
        for (int t = 0; t < V; ++t) {
            a[t] = t2[t];
            x[t] = t2[V + t];
        }
    } else {
        load_slice<T, V, VEC>(a, A, row, R, lg);
        load_slice<T, V, VEC>(x, X, row, R, lg);
    }
}

// Contribution of one nonzero to its row of the output (one lane's V entries).
// a / xa: this mode's factor / direction rows of the nonzero's row.
template <typename T, int V, int G, bool VEC, int OP, bool AXL = false>
__device__ __forceinline__ void contribution(const SweepParams<T> &P, const StepIn<T> &in,
                                             const T (&a)[V], const T (&xa)[V], int lg, bool valid,
                                             T (&c)[V], double &lacc, bool &dom_ok) {
    constexpr int RT = V * G;
    const int R = VEC ? RT : P.R;
    T b[V], e[V];
    T xb[V], xc[V];
    if constexpr (OP == OP_GGN || OP == OP_NEWTON) {
        load_pair<T, V, VEC, AXL>(b, xb, P.A1, P.X1, in.j, R, lg);
        load_pair<T, V, VEC, AXL>(e, xc, P.A2, P.X2, in.k, R, lg);
    } else {
        load_slice<T, V, VEC>(b, P.A1, in.j, R, lg);
        load_slice<T, V, VEC>(e, P.A2, in.k, R, lg);
    }
    if constexpr (OP == OP_MTTKRP) {
#pragma unroll
        for (int t = 0; t < V; ++t) c[t] = in.s * b[t] * e[t];
    } else if constexpr (OP == OP_GRAD) {
        T part = T(0);
#pragma unroll
        for (int t = 0; t < V; ++t) part += a[t] * b[t] * e[t];
        const T m = group_sum<G>(part);
        T phi, d1, d2;
        loss_terms(P.loss, in.t, m, phi, d1, d2, dom_ok);
#pragma unroll
        for (int t = 0; t < V; ++t) c[t] = d1 * b[t] * e[t];
        if (lg == 0 && valid) lacc += (double)phi;
    } else {
        T zp = T(0), part = T(0);
#pragma unroll
        for (int t = 0; t < V; ++t) {
            const T be = b[t] * e[t];
            zp += xa[t] * be + a[t] * (xb[t] * e[t] + b[t] * xc[t]);
            part += a[t] * be;
        }
        const T z = group_sum<G>(zp);
        T d2 = T(2), d1 = T(0);
        if (OP == OP_NEWTON || P.loss != TC_LOSS_LS) {   // (m is unused for the LS Gauss-Newton product)
            const T m = group_sum<G>(part);
            T phi;
            loss_terms(P.loss, in.t, m, phi, d1, d2, dom_ok);
        }
        const T wz = d2 * z;
        if constexpr (OP == OP_NEWTON) {
            // phi' times the second derivatives of m_e: for this output mode
            // and each other mode q, the product with x^(q) in place of a^(q)
#pragma unroll
            for (int t = 0; t < V; ++t) c[t] = wz * b[t] * e[t] + d1 * (xb[t] * e[t] + b[t] * xc[t]);
        } else {
#pragma unroll
            for (int t = 0; t < V; ++t) c[t] = wz * b[t] * e[t];
        }
    }
    if (!valid) {
#pragma unroll
        for (int t = 0; t < V; ++t) c[t] = T(0);
    }
}

// Lane width per operation (bytes per lane vector), chosen by measurement.
template <int OP>
constexpr int sweep_vb() { return OP == OP_GRAD ? 32 : 16; }

template <typename T, int RT, bool VEC, int OP, bool AXL = false>
__global__ void __launch_bounds__(256) sweep_kernel(const SweepParams<T> P) {
    using L = Lay<T, RT, sweep_vb<OP>()>;
    constexpr int V = L::V, G = L::G, NG = L::NG;
    constexpr unsigned FULL = 0xffffffffu;
    constexpr bool OWN = OP != OP_MTTKRP;     // needs this mode's own factor row
    const int lane = threadIdx.x & 31, g = lane / G, lg = lane % G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t c0 = warp * P.chunk;
    const bool active = c0 < P.nnz;     // idle warps still join the block reductions
    // positions inside the chunk are 32-bit offsets from c0
    const int n = active ? (int)(min(c0 + P.chunk, P.nnz) - c0) : 0;
    const int64_t *__restrict__ nzp = P.nz_ptr;
    const int R = VEC ? RT : P.R;
    const int n_ne = active ? (int)__ldg(P.n_ne_dev) : 1;

    ChunkStreams<T> S;
    S.c1 = P.c1 + c0;
    S.c2 = P.c2 + c0;
    S.t = P.t ? P.t + c0 : nullptr;
    S.w = P.w;
    if (P.w.to0) S.w.to0 = P.w.to0 + c0;
    else if (P.w.s) S.w.s = P.w.s + c0;

    int cur = active ? search_le32(nzp, 0, n_ne - 1, c0) : 0;
    const int first_cr = cur;
    const bool first_shared = active && __ldg(nzp + cur) < c0;
    const int last_cr = active ? search_le32(nzp, cur, n_ne - 1, c0 + n - 1) : 0;
    const bool last_shared = active && __ldg(nzp + last_cr + 1) > c0 + n;
    // end of row `cur` as an offset, clamped to n (beyond the chunk)
    auto row_end_of = [&](int cr) { return (int)min(__ldg(nzp + cr + 1) - c0, (int64_t)n); };
    int row_end = active ? row_end_of(cur) : 0;

    T acc[V], a[V], xa[V];
#pragma unroll
    for (int t = 0; t < V; ++t) acc[t] = a[t] = xa[t] = T(0);
    int own_cr = -1;
    double lacc = 0.0, dacc = 0.0;
    bool dom_ok = true;

    auto flush = [&](int cr, const T(&v)[V]) {
        if (!P.out) return;
        const int64_t row = __ldg(P.nz_rows + cr);
        if ((cr == first_cr && first_shared) || (cr == last_cr && last_shared)) {
            atomic_add_slice<T, V>(P.out, row, R, lg, v);
        } else if (P.accumulate) {
            T o[V];
            T *ptr = P.out + row * (int64_t)R + lg * V;
#pragma unroll
            for (int t = 0; t < V; ++t) o[t] = (lg * V + t < R) ? ptr[t] + v[t] : T(0);
            store_slice<T, V, VEC>(P.out, row, R, lg, o);
        } else {
            store_slice<T, V, VEC>(P.out, row, R, lg, v);
        }
        if (P.dot_acc) {
            T dw[V], unused[V];
            if constexpr (AXL) load_pair<T, V, VEC, true>(unused, dw, P.dot_with, nullptr, row, R, lg);
            else load_slice<T, V, VEC>(dw, P.dot_with, row, R, lg);
#pragma unroll
            for (int t = 0; t < V; ++t) dacc += (double)dw[t] * (double)v[t];
        }
    };
    auto load_own = [&](int cr) {
        const int64_t row = __ldg(P.nz_rows + cr);
        if constexpr (OP == OP_GGN || OP == OP_NEWTON)
            load_pair<T, V, VEC, AXL>(a, xa, P.Ad, P.Xd, row, R, lg);
        else load_slice<T, V, VEC>(a, P.Ad, row, R, lg);
    };
    // A step whose row boundaries fall inside it (off: first offset; last: its
    // last valid offset; valid: this group's nonzero exists).
    auto slow_step = [&](int off, int last, bool valid, const StepIn<T> &in) {
        const int qq = valid ? off + g : last;
        // `cur` holds offset off - 1 or off, so the step spans rows cur .. cur + NG
        const int cr = search_le32(nzp, cur, min(cur + NG, n_ne - 1), c0 + qq);
        if constexpr (OWN) {
            load_own(cr);
            own_cr = cr;
        }
        T c[V];
        contribution<T, V, G, VEC, OP, AXL>(P, in, a, xa, lg, valid, c, lacc, dom_ok);
        if (cr == cur) {
#pragma unroll
            for (int t = 0; t < V; ++t) {
                acc[t] += c[t];
                c[t] = T(0);
            }
        }
        {   // row `cur` ends inside this step: reduce the private partial sums
            T tot[V];
#pragma unroll
            for (int t = 0; t < V; ++t) tot[t] = across_groups<G>(acc[t]);
            if (g == 0) flush(cur, tot);
        }
        T craw[V];
#pragma unroll
        for (int t = 0; t < V; ++t) craw[t] = c[t];
        // rows after `cur`: segmented inclusive scan over the groups
#pragma unroll
        for (int d = 1; d < NG; d <<= 1) {
            const int ocr = __shfl_up_sync(FULL, cr, d * G);
            T o[V];
#pragma unroll
            for (int t = 0; t < V; ++t) o[t] = __shfl_up_sync(FULL, c[t], d * G);
            if (g >= d && ocr == cr) {
#pragma unroll
                for (int t = 0; t < V; ++t) c[t] += o[t];
            }
        }
        const int ncr = __shfl_down_sync(FULL, cr, G);
        const int lcr = __shfl_sync(FULL, cr, (NG - 1) * G);
        const bool tail = (g == NG - 1) || (ncr != cr);
        if (tail && cr != cur && cr != lcr) flush(cr, c);       // rows wholly inside the step
#pragma unroll
        for (int t = 0; t < V; ++t) acc[t] = (cr == lcr) ? craw[t] : T(0);
        cur = lcr;
        row_end = row_end_of(cur);
        if constexpr (OWN) own_cr = (own_cr == cur) ? cur : -1;
    };

    StepIn<T> nxt;
    if (n > 0) nxt = load_step<T, OP>(P, S, min(g, n - 1));
    int off = 0;
    // full steps: every group has a nonzero
    for (; off + NG <= n; off += NG) {
        const StepIn<T> in = nxt;
        if (off + NG < n) nxt = load_step<T, OP>(P, S, min(off + NG + g, n - 1));
        if (row_end >= off + NG) {
            // the whole step lies in row `cur`: private accumulation, no shuffles
            if constexpr (OWN) {
                if (own_cr != cur) {
                    load_own(cur);
                    own_cr = cur;
                }
            }
            T c[V];
            contribution<T, V, G, VEC, OP, AXL>(P, in, a, xa, lg, true, c, lacc, dom_ok);
#pragma unroll
            for (int t = 0; t < V; ++t) acc[t] += c[t];
        } else {
            slow_step(off, off + NG - 1, true, in);
        }
    }
    // the partial last step
    if (off < n) {
        const StepIn<T> in = nxt;
        const bool valid = off + g < n;
        if (row_end >= n) {
            if constexpr (OWN) {
                if (own_cr != cur) {
                    load_own(cur);
                    own_cr = cur;
                }
            }
            T c[V];
            contribution<T, V, G, VEC, OP, AXL>(P, in, a, xa, lg, valid, c, lacc, dom_ok);
#pragma unroll
            for (int t = 0; t < V; ++t) acc[t] += c[t];
        } else {
            slow_step(off, n - 1, valid, in);
        }
    }
    if (active) {
        T tot[V];
#pragma unroll
        for (int t = 0; t < V; ++t) tot[t] = across_groups<G>(acc[t]);
        if (g == 0) flush(cur, tot);
    }

    if constexpr (OP != OP_MTTKRP) {
        if (!dom_ok) record_error(P.status, TC_ERR_DOMAIN);
    }
    if constexpr (OP == OP_GRAD) {
        if (P.loss_acc) block_add(lacc, P.loss_acc);
    }
    if (P.dot_acc) block_add(dacc, P.dot_acc);
}

// ------------------------------------------------------------------ TTTP
template <typename T>
struct TttpParams {
    const int32_t *nz_rows;
    const int64_t *nz_ptr;
    const int64_t *n_ne_dev;
    int64_t nnz, chunk;
    const int32_t *c1, *c2;
    Weights<T> w;
    const T *A0, *A1, *A2;        // any may be null (mode skipped)
    int R;
    T *x;
};

template <typename T, int RT, bool VEC>
__global__ void __launch_bounds__(256) tttp_kernel(const TttpParams<T> P) {
    using L = Lay<T, RT>;
    constexpr int V = L::V, G = L::G, NG = L::NG;
    const int lane = threadIdx.x & 31, g = lane / G, lg = lane % G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t c0 = warp * P.chunk;
    if (c0 >= P.nnz) return;
    const int n = (int)(min(c0 + P.chunk, P.nnz) - c0);
    const int64_t *__restrict__ nzp = P.nz_ptr;
    const int R = VEC ? RT : P.R;
    const int32_t *c1 = P.c1 + c0, *c2 = P.c2 + c0;
    Weights<T> W = P.w;
    if (W.to0) W.to0 += c0;
    else if (W.s) W.s += c0;
    T *x = P.x + c0;
    const int n_ne = P.A0 ? (int)__ldg(P.n_ne_dev) : 1;
    int cur = P.A0 ? search_le32(nzp, 0, n_ne - 1, c0) : 0;
    int row_end = P.A0 ? (int)min(__ldg(nzp + cur + 1) - c0, (int64_t)n) : n;
    int own_cr = -1;
    T a[V];
#pragma unroll
    for (int t = 0; t < V; ++t) a[t] = T(1);

    for (int off = 0; off < n; off += NG) {
        const bool valid = off + g < n;
        const int q = valid ? off + g : n - 1;
        const int last = min(off + NG, n) - 1;
        if (P.A0) {
            if (row_end > last) {              // the step lies in row `cur`
                if (own_cr != cur) {
                    load_slice<T, V, VEC>(a, P.A0, __ldg(P.nz_rows + cur), R, lg);
                    own_cr = cur;
                }
            } else {
                const int cr = search_le32(nzp, cur, min(cur + NG, n_ne - 1), c0 + q);
                load_slice<T, V, VEC>(a, P.A0, __ldg(P.nz_rows + cr), R, lg);
                own_cr = cr;
                const int lcr = __shfl_sync(0xffffffffu, cr, (NG - 1) * G);
                cur = lcr;
                row_end = (int)min(__ldg(nzp + cur + 1) - c0, (int64_t)n);
                own_cr = (own_cr == cur) ? cur : -1;
            }
        }
        T prod[V];
#pragma unroll
        for (int t = 0; t < V; ++t) prod[t] = a[t];
        if (P.A1) {
            T b[V];
            load_slice<T, V, VEC>(b, P.A1, __ldcs(c1 + q), R, lg);
#pragma unroll
            for (int t = 0; t < V; ++t) prod[t] *= b[t];
        }
        if (P.A2) {
            T e[V];
            load_slice<T, V, VEC>(e, P.A2, __ldcs(c2 + q), R, lg);
#pragma unroll
            for (int t = 0; t < V; ++t) prod[t] *= e[t];
        }
        const T s = weight_at(W, q);
        T part = T(0);
#pragma unroll
        for (int t = 0; t < V; ++t) part += (lg * V + t < R) ? prod[t] : T(0);
        const T m = group_sum<G>(part);
        if (valid && lg == 0) __stcs(x + q, s * m);
    }
}

// ------------------------------------------------------------------ small kernels
// y = alpha * x (n elements); optional dot += alpha * x.x (FP64).
template <typename T>
__global__ void scale_kernel(T *__restrict__ y, const T *__restrict__ x, T alpha, int64_t n,
                             double *dot) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const T v = x[i];
        y[i] = alpha * v;
        acc += (double)alpha * (double)v * (double)v;
    }
    if (dot) {
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(dot, acc);
    }
}

// acc += scale * sum x^2 (FP64)
template <typename T>
__global__ void sumsq_kernel(const T *__restrict__ x, int64_t n, double scale, double *acc) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)x[i];
        s += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc, scale * s);
}

// ------------------------------------------------------------------ launchers
// SM count, queried once (host threads may race to fill it; they store the
// same value, and the atomic makes that well defined)
static std::atomic<int> g_sm_count{0};
static int sm_count() {
    int v = g_sm_count.load(std::memory_order_relaxed);
    if (!v) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (v <= 0) v = 1;
        g_sm_count.store(v, std::memory_order_relaxed);
    }
    return v;
}

// Blocks of `kern` (256 threads, no dynamic shared memory) resident per SM,
// queried once per kernel.
static int resident_blocks(const void *kern) {
    static std::mutex mu;
    static std::unordered_map<const void *, int> cache;
    std::lock_guard<std::mutex> lock(mu);
    const auto it = cache.find(kern);
    if (it != cache.end()) return it->second;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    cache[kern] = occ;
    return occ;
}

// Nonzeros per warp: 8 to 64 warp steps, and the grid a whole number of waves
// of resident blocks, so no last partial wave leaves most SMs idle while a few
// blocks finish (every warp's chunk costs about the same on these sweeps).
template <typename K>
static int64_t pick_chunk(int64_t nnz, int NG, K kern) {
    const int64_t min_chunk = (int64_t)NG * 8, max_chunk = (int64_t)NG * 64;
    const int64_t slot_warps = (int64_t)sm_count() * resident_blocks((const void *)kern) * (256 / 32);
    int64_t waves = (nnz + slot_warps * max_chunk - 1) / (slot_warps * max_chunk);
    if (waves < 1) waves = 1;
    int64_t c = (nnz + waves * slot_warps - 1) / (waves * slot_warps);
    c = ((c + NG - 1) / NG) * NG;
    if (c < min_chunk) c = min_chunk;
    return c;
}

template <typename T>
static Weights<T> make_weights(const tc_pattern *p, int mode, tc_weights w, const void *s) {
    Weights<T> W{(int)w, nullptr, nullptr};
    if (w == TC_W_VALUES) W.s = (const T *)p->md[mode].vals;
    else if (w == TC_W_ARRAY) {
        W.s = (const T *)s;
        if (mode != 0) W.to0 = p->md[mode].to0;
    }
    return W;
}

template <typename T, int OP>
static void launch_sweep_t(const SweepParams<T> &P, int tier, bool vec, cudaStream_t st) {
    const int threads = 256;
    auto go = [&](auto kern, int NG) {
        SweepParams<T> Q = P;
        Q.chunk = pick_chunk(P.nnz, NG, kern);
        const int64_t warps = (P.nnz + Q.chunk - 1) / Q.chunk;
        const int64_t blocks = (warps * 32 + threads - 1) / threads;
        kern<<<(unsigned)blocks, threads, 0, st>>>(Q);
        count_launch();
    };
#define TC_SWEEP_CASE(RT)                                                              \
    case RT:                                                                           \
        if (vec) go(sweep_kernel<T, RT, true, OP>, Lay<T, RT, sweep_vb<OP>()>::NG);     \
        else go(sweep_kernel<T, RT, false, OP>, Lay<T, RT, sweep_vb<OP>()>::NG);        \
        break;
    switch (tier) {
        TC_SWEEP_CASE(8)
        TC_SWEEP_CASE(16)
        TC_SWEEP_CASE(32)
        TC_SWEEP_CASE(64)
    }
#undef TC_SWEEP_CASE
}

template <typename T>
static SweepParams<T> base_params(const tc_pattern *p, int mode, int R) {
    const ModeData &md = p->md[mode];
    SweepParams<T> P{};
    P.nz_rows = md.nz_rows;
    P.nz_ptr = md.nz_ptr;
    P.n_ne_dev = md.n_ne_dev;
    P.nnz = p->nnz;
    P.c1 = md.cols[0];
    P.c2 = md.cols[1];
    P.t = (const T *)md.vals;
    P.R = R;
    P.status = p->status;
    return P;
}

template <typename T>
static void launch_scale(T *y, const T *x, T alpha, int64_t n, double *dot, cudaStream_t st) {
    const int threads = 256;
    int64_t blocks = (n + threads - 1) / threads;
    if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
    if (blocks < 1) blocks = 1;
    scale_kernel<T><<<(unsigned)blocks, threads, 0, st>>>(y, x, alpha, n, dot);
    count_launch();
}

template <typename T>
static void launch_sumsq(const T *x, int64_t n, double scale, double *acc, cudaStream_t st) {
    const int threads = 256;
    int64_t blocks = (n + threads - 1) / threads;
    if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
    if (blocks < 1) blocks = 1;
    sumsq_kernel<T><<<(unsigned)blocks, threads, 0, st>>>(x, n, scale, acc);
    count_launch();
}

template <typename T>
static tc_status tttp_t(const tc_pattern *p, tc_weights w, const void *s, int R,
                        const void *const *A, void *x, cudaStream_t st) {
    if (p->nnz == 0) return TC_OK;
    const ModeData &md = p->md[0];
    TttpParams<T> P{};
    P.nz_rows = md.nz_rows;
    P.nz_ptr = md.nz_ptr;
    P.n_ne_dev = md.n_ne_dev;
    P.nnz = p->nnz;
    P.c1 = md.cols[0];
    P.c2 = md.cols[1];
    P.w = make_weights<T>(p, 0, w, s);
    P.A0 = (const T *)A[0];
    P.A1 = (const T *)A[1];
    P.A2 = (const T *)A[2];
    P.R = R;
    P.x = (T *)x;
    const int tier = rank_tier(R);
    const bool vec = vec_ok(R, tier, sizeof(T)) && aligned16({A[0], A[1], A[2]});
    const int threads = 256;
    auto go = [&](auto kern, int NG) {
        TttpParams<T> Q = P;
        Q.chunk = pick_chunk(P.nnz, NG, kern);
        const int64_t warps = (P.nnz + Q.chunk - 1) / Q.chunk;
        const int64_t blocks = (warps * 32 + threads - 1) / threads;
        kern<<<(unsigned)blocks, threads, 0, st>>>(Q);
        count_launch();
    };
#define TC_TTTP_CASE(RT)                                                     \
    case RT:                                                                 \
        if (vec) go(tttp_kernel<T, RT, true>, Lay<T, RT>::NG);               \
        else go(tttp_kernel<T, RT, false>, Lay<T, RT>::NG);                  \
        break;
    switch (tier) {
        TC_TTTP_CASE(8)
        TC_TTTP_CASE(16)
        TC_TTTP_CASE(32)
        TC_TTTP_CASE(64)
    }
#undef TC_TTTP_CASE
    return TC_OK;
}

tc_status launch_tttp(const tc_pattern *p, tc_weights w, const void *s, int R,
                      const void *const *A, void *x, cudaStream_t st) {
    return p->dtype == TC_F64 ? tttp_t<double>(p, w, s, R, A, x, st)
                              : tttp_t<float>(p, w, s, R, A, x, st);
}

template <typename T>
static tc_status mttkrp_t(const tc_pattern *p, tc_weights w, const void *s, int R,
                          const void *const *A, int mode, void *out, int accumulate,
                          cudaStream_t st) {
    const size_t bytes = (size_t)p->dims[mode] * R * sizeof(T);
    if (!accumulate) {
        TC_CUDA(cudaMemsetAsync(out, 0, bytes, st));
    }
    if (p->nnz == 0) return TC_OK;
    if (w == TC_W_ARRAY && mode != 0) {
        tc_status rc = ensure_to0(p, st);
        if (rc != TC_OK) return rc;
    }
    int o1, o2;
    other_modes(mode, o1, o2);
    SweepParams<T> P = base_params<T>(p, mode, R);
    P.w = make_weights<T>(p, mode, w, s);
    P.A1 = (const T *)A[o1];
    P.A2 = (const T *)A[o2];
    P.out = (T *)out;
    P.accumulate = accumulate;
    const int tier = rank_tier(R);
    const bool vec = vec_ok(R, tier, sizeof(T)) && aligned16({A[o1], A[o2], out});
    launch_sweep_t<T, OP_MTTKRP>(P, tier, vec, st);
    return TC_OK;
}

tc_status launch_regularizer(const tc_pattern *p, int R, const void *const *A, double lambda,
                             double *acc, cudaStream_t st) {
    for (int n = 0; n < TC_ORDER; ++n) {
        if (p->dtype == TC_F64) launch_sumsq<double>((const double *)A[n], p->dims[n] * R, lambda, acc, st);
        else launch_sumsq<float>((const float *)A[n], p->dims[n] * R, lambda, acc, st);
    }
    return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

tc_status launch_mttkrp(const tc_pattern *p, tc_weights w, const void *s, int R,
                        const void *const *A, int mode, void *out, int accumulate,
                        cudaStream_t st) {
    return p->dtype == TC_F64 ? mttkrp_t<double>(p, w, s, R, A, mode, out, accumulate, st)
                              : mttkrp_t<float>(p, w, s, R, A, mode, out, accumulate, st);
}

template <typename T>
static tc_status loss_grad_t(const tc_pattern *p, tc_loss loss, int R, const void *const *A,
                             double lambda, double *loss_out, void *const *grads,
                             cudaStream_t st) {
    const int tier = rank_tier(R);
    bool vec = vec_ok(R, tier, sizeof(T)) && aligned16({A[0], A[1], A[2]});
    if (grads) vec = vec && aligned16({grads[0], grads[1], grads[2]});
    if (loss_out) {
        TC_CUDA(cudaMemsetAsync(loss_out, 0, sizeof(double), st));
        for (int n = 0; n < TC_ORDER; ++n)
            launch_sumsq<T>((const T *)A[n], p->dims[n] * R, lambda, loss_out, st);
    }
    bool loss_done = (loss_out == nullptr) || p->nnz == 0;
    for (int d = 0; d < TC_ORDER; ++d) {
        T *g = grads ? (T *)grads[d] : nullptr;
        if (!g && (loss_done || d < TC_ORDER - 1)) continue;
        if (g) launch_scale<T>(g, (const T *)A[d], (T)(2.0 * lambda), p->dims[d] * R, nullptr, st);
        if (p->nnz == 0) continue;
        int o1, o2;
        other_modes(d, o1, o2);
        SweepParams<T> P = base_params<T>(p, d, R);
        P.Ad = (const T *)A[d];
        P.A1 = (const T *)A[o1];
        P.A2 = (const T *)A[o2];
        P.loss = loss;
        P.out = g;
        P.accumulate = 1;
        P.loss_acc = loss_done ? nullptr : loss_out;
        loss_done = true;
        launch_sweep_t<T, OP_GRAD>(P, tier, vec, st);
    }
    return TC_OK;
}

tc_status launch_loss_grad(const tc_pattern *p, tc_loss loss, int R, const void *const *A,
                           double lambda, double *loss_out, void *const *grads, cudaStream_t st) {
    return p->dtype == TC_F64 ? loss_grad_t<double>(p, loss, R, A, lambda, loss_out, grads, st)
                              : loss_grad_t<float>(p, loss, R, A, lambda, loss_out, grads, st);
}

template <typename T>
static tc_status ggn_t(const tc_pattern *p, tc_loss loss, int R, const void *const *A,
                       const void *const *x, double lambda, void *const *y, double *dot_out,
                       int init, int full_newton, cudaStream_t st) {
    const int tier = rank_tier(R);
    const bool vec = vec_ok(R, tier, sizeof(T)) && aligned16({A[0], A[1], A[2]}) &&
                     aligned16({x[0], x[1], x[2]}) && aligned16({y[0], y[1], y[2]});
    for (int d = 0; d < TC_ORDER; ++d) {
        if (init)
            launch_scale<T>((T *)y[d], (const T *)x[d], (T)(2.0 * lambda), p->dims[d] * R, dot_out,
                            st);
        if (p->nnz == 0) continue;
        int o1, o2;
        other_modes(d, o1, o2);
        SweepParams<T> P = base_params<T>(p, d, R);
        P.Ad = (const T *)A[d];
        P.A1 = (const T *)A[o1];
        P.A2 = (const T *)A[o2];
        P.Xd = (const T *)x[d];
        P.X1 = (const T *)x[o1];
        P.X2 = (const T *)x[o2];
        P.loss = loss;
        P.out = (T *)y[d];
        P.accumulate = 1;
        P.dot_acc = dot_out;
        P.dot_with = (const T *)x[d];
        if (full_newton) launch_sweep_t<T, OP_NEWTON>(P, tier, vec, st);
        else launch_sweep_t<T, OP_GGN>(P, tier, vec, st);
    }
    return TC_OK;
}

// y = alpha * (direction part of the interleaved buffer); dot += alpha x.x
template <typename T>
__global__ void scale_ax_kernel(T *__restrict__ y, const T *__restrict__ ax, T alpha, int64_t I,
                                int R, int V, double *dot) {
    double acc = 0.0;
    const int64_t n = I * R;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = q / R;
        const int e = (int)(q - i * R);
        const T v = ax[i * 2 * R + (e / V) * 2 * V + V + e % V];
        y[q] = alpha * v;
        acc += (double)alpha * (double)v * (double)v;
    }
    if (dot) block_add(acc, dot);
}

// Gauss-Newton matvec on interleaved factor / direction buffers (the PCG
// driver's layout; see load_pair).  Requires the vector path (R fills its tier).
template <typename T>
static tc_status ggn_ax_t(const tc_pattern *p, tc_loss loss, int R, const void *const *AX,
                          double lambda, void *const *y, double *dot_out, int init, int full_newton,
                          cudaStream_t st) {
    const int tier = rank_tier(R);
    constexpr int V = 16 / (int)sizeof(T);
    for (int d = 0; d < TC_ORDER; ++d) {
        const int64_t n = p->dims[d] * R;
        int64_t blocks = (n + 255) / 256;
        if (blocks > (int64_t)sm_count() * 8) blocks = (int64_t)sm_count() * 8;
        if (blocks < 1) blocks = 1;
        if (init) {
            scale_ax_kernel<T><<<(unsigned)blocks, 256, 0, st>>>((T *)y[d], (const T *)AX[d],
                                                                 (T)(2.0 * lambda), p->dims[d], R,
                                                                 V, dot_out);
            count_launch();
        }
        if (p->nnz == 0) continue;
        int o1, o2;
        other_modes(d, o1, o2);
        SweepParams<T> P = base_params<T>(p, d, R);
        P.Ad = (const T *)AX[d];
        P.A1 = (const T *)AX[o1];
        P.A2 = (const T *)AX[o2];
        P.loss = loss;
        P.out = (T *)y[d];
        P.accumulate = 1;
        P.dot_acc = dot_out;
        P.dot_with = (const T *)AX[d];
        const int threads = 256;
        auto go = [&](auto kern, int NG) {
            SweepParams<T> Q = P;
            Q.chunk = pick_chunk(P.nnz, NG, kern);
            const int64_t warps = (P.nnz + Q.chunk - 1) / Q.chunk;
            const int64_t nb = (warps * 32 + threads - 1) / threads;
            kern<<<(unsigned)nb, threads, 0, st>>>(Q);
            count_launch();
        };
        if (full_newton) {
            switch (tier) {
                case 8: go(sweep_kernel<T, 8, true, OP_NEWTON, true>, Lay<T, 8, 16>::NG); break;
                case 16: go(sweep_kernel<T, 16, true, OP_NEWTON, true>, Lay<T, 16, 16>::NG); break;
                case 32: go(sweep_kernel<T, 32, true, OP_NEWTON, true>, Lay<T, 32, 16>::NG); break;
                default: go(sweep_kernel<T, 64, true, OP_NEWTON, true>, Lay<T, 64, 16>::NG); break;
            }
        } else {
            switch (tier) {
                case 8: go(sweep_kernel<T, 8, true, OP_GGN, true>, Lay<T, 8, 16>::NG); break;
                case 16: go(sweep_kernel<T, 16, true, OP_GGN, true>, Lay<T, 16, 16>::NG); break;
                case 32: go(sweep_kernel<T, 32, true, OP_GGN, true>, Lay<T, 32, 16>::NG); break;
                default: go(sweep_kernel<T, 64, true, OP_GGN, true>, Lay<T, 64, 16>::NG); break;
            }
        }
    }
    return TC_OK;
}

tc_status prepare_ggn_matvec_ax() {
#define TC_WARM(T, RT)                                                              \
    resident_blocks((const void *)sweep_kernel<T, RT, true, OP_GGN, true>);         \
    resident_blocks((const void *)sweep_kernel<T, RT, true, OP_NEWTON, true>);
    TC_WARM(float, 8) TC_WARM(float, 16) TC_WARM(float, 32) TC_WARM(float, 64)
    TC_WARM(double, 8) TC_WARM(double, 16) TC_WARM(double, 32) TC_WARM(double, 64)
#undef TC_WARM
    return TC_OK;
}

tc_status launch_ggn_matvec_ax(const tc_pattern *p, tc_loss loss, int R, const void *const *AX,
                               double lambda, void *const *y, double *dot_out, int init,
                               int full_newton, cudaStream_t st) {
    return p->dtype == TC_F64
               ? ggn_ax_t<double>(p, loss, R, AX, lambda, y, dot_out, init, full_newton, st)
               : ggn_ax_t<float>(p, loss, R, AX, lambda, y, dot_out, init, full_newton, st);
}

tc_status launch_ggn_matvec(const tc_pattern *p, tc_loss loss, int R, const void *const *A,
                            const void *const *x, double lambda, void *const *y,
                            double *dot_out, int init, int full_newton, cudaStream_t st) {
    return p->dtype == TC_F64
               ? ggn_t<double>(p, loss, R, A, x, lambda, y, dot_out, init, full_newton, st)
               : ggn_t<float>(p, loss, R, A, x, lambda, y, dot_out, init, full_newton, st);
}

}  // namespace tc
