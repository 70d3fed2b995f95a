// Solve Factor (Sec. 3.4 with the normal equations of Sec. 2.2) and the
// block-diagonal Gauss-Newton preconditioner (Sec. 2.5), which is the same
// per-row system with weights phi'' and regularization 2 lambda.
//
// Two kernels per batch of rows.
//
// Kernel A forms the Gram matrices G_i = sum_e s_e h_e h_e^T.  It walks the
// mode's sorted nonzeros in fixed-size chunks (a persistent grid; every block
// takes every gridDim-th chunk), so the work per block is the same whatever
// the distribution of nonzeros over rows: a power-law row with millions of
// nonzeros is spread over many blocks, and a chunk may hold many short rows.
// Inside a chunk the block visits the rows it meets in turn: the block's
// threads gather h_e = (hadamard of the other modes' rows) and the weight of
// KB nonzeros into shared memory, then accumulate them with one of the Gram
// engines below (exact FP32 products on the FMA units by default; tensor-core
// forms for the refined mixed-precision solves).  At the end of a row's
// segment the packed lower triangle is written: plainly when the whole row
// lies in the chunk, otherwise added with FP64 atomics into a zeroed slot
// owned by the first chunk boundary the row crosses.  The same pass can also
// form a right-hand side from the gathered rows (RhsKind): sum_e t_e h_e for
// an ALS update, or sum_e phi'_e h_e (the gradient's MTTKRP) with the loss
// for a Gauss-Newton preconditioner block; cut rows' shares go to FP64 slots.
//
// Kernel B runs the FP64 part: lambda on the diagonal, the unpivoted Cholesky
// factorization, then the two triangular solves, or the inverse
// (L L^T)^-1 = L^-T L^-1 for the preconditioner.  For R <= 32 a warp factors
// 16 (R <= 16) or 4 (R = 32) rows together, the lanes of a row sharing each
// step's work (every FP64 instruction does a warp of useful work); for R > 32
// a warp owns one row and the trailing updates are spread evenly over the
// lanes.
#include <type_traits>

#include "internal.cuh"

#include <atomic>
#include <mutex>

namespace tc {

// What the Gram pass also forms beside G_i: nothing (the right-hand side is
// given), rhs_i = sum_e t_e h_e (the MTTKRP of the values: an ALS update), or
// rhs_i = sum_e phi'(t_e, m_e) h_e (the MTTKRP of phi': the gradient, in a
// preconditioner pass with phi'' weights).
enum RhsKind { RHS_GIVEN = 0, RHS_VALUES = 1, RHS_DPHI = 2 };

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
    int refine;                   // refinement steps after the solve (0, 1 or 2)
    int *status;
    int rhs_kind;                 // RhsKind: RHS_VALUES / RHS_DPHI form rhs_w in the Gram pass
    T *rhs_w;                     // I_d x R (rhs_kind != RHS_GIVEN)
    double *loss_acc;             // RHS_DPHI: += sum_e phi(t_e, m_e) over the pass, or null
};

// Rows [row0, row0 + nrows) of the mode and the chunks of ch nonzeros that
// cover them, starting at the batch's first nonzero nb = row_ptr[row0].
template <typename T>
struct Batch {
    int64_t row0, nrows;
    int64_t ch;
    T *light;        // nrows x TRI packed triangles of rows that lie within one chunk
                     // (with refinement: then every row's Cholesky factor)
    double *cut;     // one TRI slot per chunk boundary, for rows that cross one
    double *res;     // refinement: nrows x R residual sums (zeroed), or null
    double *cut_rhs; // rhs_kind: one R slot per chunk boundary (zeroed), or null
};

// Packed lower-triangle index of (r, c), c <= r.
__host__ __device__ __forceinline__ int tri_idx(int r, int c) { return r * (r + 1) / 2 + c; }

// (r, c) of packed index e.
__device__ __forceinline__ void tri_rc(int e, int &r, int &c) {
    r = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    while (tri_idx(r, 0) > e) --r;
    while (tri_idx(r + 1, 0) <= e) ++r;
    c = e - tri_idx(r, 0);
}

// d^(-1/2) for the Cholesky pivots: two Newton steps y <- y (3 - d y^2) / 2
// from a single-precision seed (each step doubles the correct bits: about
// 23 -> 46 -> 53), a handful of FP64 multiply-adds in place of a
// square root and a division.  Outside the single-precision range the
// correctly rounded path is taken.
__device__ __forceinline__ double rsqrt_nr(double d) {
    if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
    double y = (double)rsqrtf((float)d);
    const double h = 0.5 * d;
    y = y * (1.5 - h * y * y);
    y = y * (1.5 - h * y * y);
    return y;
}

// The same in FP32 (for the FP32 factorization of the refined forms): the
// hardware estimate and one Newton step.
__device__ __forceinline__ float rsqrt_nr(float d) {
    const float y = rsqrtf(d);
    return y * (1.5f - 0.5f * d * y * y);
}

// Exact float -> double widening with integer operations (sign, exponent
// rebias, mantissa shift), so that the cut-row flushes below keep the SM's
// FP64 pipe (about one operation per clock per SM on this GPU) free; zero,
// subnormal, infinite and NaN inputs take the ordinary conversion.
__device__ __forceinline__ double widen(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t ex = (u >> 23) & 0xffu;
    if (ex == 0u || ex == 0xffu) return (double)f;
    const uint64_t bits = ((uint64_t)(u >> 31) << 63) | ((uint64_t)(ex + 896u) << 52) |
                          ((uint64_t)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

// Adds an FP32 pair (hi + lo) or one FP32 value into an FP64 slot: the
// additions are FP64 atomics, carried out in the L2 cache.
__device__ __forceinline__ void add_cut(double *slot, float hi, float lo) {
    atomicAdd(slot, widen(hi));
    if (lo != 0.f) atomicAdd(slot, widen(lo));
}
__device__ __forceinline__ void add_cut(double *slot, float v) { atomicAdd(slot, widen(v)); }
__device__ __forceinline__ void add_cut(double *slot, double v) { atomicAdd(slot, v); }

// Slot of a nonempty row [rs, re) that crosses a chunk boundary: the first
// boundary after rs (boundary b >= 1 sits at nb + b ch; slot b - 1); -1 when
// the row lies within one chunk.
__device__ __forceinline__ int64_t cut_slot(int64_t rs, int64_t re, int64_t nb, int64_t ch) {
    const int64_t b = (rs - nb) / ch + 1;
    return nb + b * ch < re ? b - 1 : -1;
}

template <typename T>
__global__ void zero_cut_kernel(const int64_t *__restrict__ row_ptr, const Batch<T> B, int tri,
                                int R) {
    const int64_t nb = __ldg(row_ptr + B.row0), ne = __ldg(row_ptr + B.row0 + B.nrows);
    const int64_t nch = (ne - nb + B.ch - 1) / B.ch;
    const int64_t nslot = nch > 1 ? nch - 1 : 0;
    const int64_t n = nslot * (int64_t)tri, nr = B.cut_rhs ? nslot * (int64_t)R : 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n + nr;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (q < n) B.cut[q] = 0.0;
        else B.cut_rhs[q - n] = 0.0;
    }
}

// rhs_kind: the right-hand sides of the rows that cross a chunk boundary,
// summed in FP64 in the row's cut slot by every chunk that covers part of it,
// copied into rhs_w.  Slot k belongs to the row that holds position
// nb + (k + 1) ch if that row's first boundary is that one (a row longer than
// a chunk uses the slot of its first boundary only; the others stay unused).
template <typename T>
__global__ void cut_rhs_kernel(const int64_t *__restrict__ row_ptr, const Batch<T> B, int R,
                               T *__restrict__ rhs_w) {
    const int64_t nb = __ldg(row_ptr + B.row0), ne = __ldg(row_ptr + B.row0 + B.nrows);
    const int64_t nch = (ne - nb + B.ch - 1) / B.ch;
    const int64_t nslot = nch > 1 ? nch - 1 : 0;
    const int64_t last = B.row0 + B.nrows - 1;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nslot * R;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = q / R;
        const int r = (int)(q - k * R);
        const int64_t pos = nb + (k + 1) * B.ch;             // < ne
        const int64_t i = search_le(row_ptr, B.row0, last, pos);
        const int64_t rs = __ldg(row_ptr + i), re = __ldg(row_ptr + i + 1);
        if (cut_slot(rs, re, nb, B.ch) == k) rhs_w[i * (int64_t)R + r] = (T)B.cut_rhs[k * R + r];
    }
}

// ------------------------------------------------------------------ Gram engines
// How G_i = sum_e s_e h_e h_e^T is summed (the Cholesky is FP64 in every form):
//   GK_FFMA  exact FP32 (or FP64) products on the FMA units; each thread owns a
//            4 x 4 tile of the lower triangle and keeps FP32 partial sums of at
//            most 32 terms, folded into a compensated (TwoSum) FP32 pair, so
//            the Gram is accurate to a few FP32 ulps whatever the row length;
//   GK_TF32X3 tensor cores, mma.sync m16n8k8: each FP32 operand x is split
//            into x_hi = tf32(x) and x_lo = tf32(x - x_hi) and the product is
//            formed as hi*hi + hi*lo + lo*hi (about 21 significant bits per
//            product); FP32 accumulator tiles folded every 128 nonzeros into
//            compensated pairs like the FFMA form: an FP32-class Gram;
//   GK_TF32  tensor cores, mma.sync m16n8k8 with TF32 inputs (11-bit
//            significands) and FP32 accumulation;
//   GK_BF16  tensor cores, mma.sync m16n8k16 with BF16 inputs (8-bit
//            significands) and FP32 accumulation.
// TF32 / BF16 are meant to be followed by a refinement step.
enum GramKind { GK_FFMA = 0, GK_TF32 = 1, GK_BF16 = 2, GK_TF32X3 = 3 };

// s + e = a + b exactly (Knuth's TwoSum; no FMA contraction applies).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// Two floats as a bf16x2 register: `lo` in the low half (the fragment's
// element of smaller k), `hi` in the high half.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

// One K step of the tensor-core Gram on a staged block of h rows (stride S,
// weights wf): the A fragment of row tile mt (load_a), then the product into
// tile (mt, nt) (apply).  K step kc covers nonzeros 8 kc .. 8 kc + 7
// (16 kc .. 16 kc + 15 for BF16).
template <int RT, int KIND, int S>
struct MmaStep {
    uint32_t ah[4], al[4];

    __device__ __forceinline__ void load_a(const float *hf, int kc, int mt, int gid, int tig) {
        const int ra = mt * 16 + gid, rb = ra + 8;
        const bool vb = rb < RT;
        if constexpr (KIND == GK_BF16) {
            const int k0 = kc * 16 + tig * 2;
            ah[0] = pack_bf16(hf[k0 * S + ra], hf[(k0 + 1) * S + ra]);
            ah[1] = pack_bf16(vb ? hf[k0 * S + rb] : 0.f, vb ? hf[(k0 + 1) * S + rb] : 0.f);
            ah[2] = pack_bf16(hf[(k0 + 8) * S + ra], hf[(k0 + 9) * S + ra]);
            ah[3] = pack_bf16(vb ? hf[(k0 + 8) * S + rb] : 0.f, vb ? hf[(k0 + 9) * S + rb] : 0.f);
        } else {
            const int k0 = kc * 8 + tig, k1 = k0 + 4;
            const float x[4] = {hf[k0 * S + ra], vb ? hf[k0 * S + rb] : 0.f, hf[k1 * S + ra],
                                vb ? hf[k1 * S + rb] : 0.f};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if constexpr (KIND == GK_TF32X3) split_tf32(x[q], ah[q], al[q]);
                else ah[q] = to_tf32(x[q]);
            }
        }
    }
    __device__ __forceinline__ void apply(const float *hf, const float *wf, int kc, int nt, int gid,
                                          int tig, float (&d)[4]) const {
        const int cn = nt * 8 + gid;
        if constexpr (KIND == GK_BF16) {
            const int k0 = kc * 16 + tig * 2;
            const uint32_t b0 = pack_bf16(wf[k0] * hf[k0 * S + cn], wf[k0 + 1] * hf[(k0 + 1) * S + cn]);
            const uint32_t b1 = pack_bf16(wf[k0 + 8] * hf[(k0 + 8) * S + cn],
                                          wf[k0 + 9] * hf[(k0 + 9) * S + cn]);
            mma_bf16(d, ah, b0, b1);
        } else {
            const int k0 = kc * 8 + tig, k1 = k0 + 4;
            const float x0 = wf[k0] * hf[k0 * S + cn], x1 = wf[k1] * hf[k1 * S + cn];
            if constexpr (KIND == GK_TF32X3) {
                // the three split products of this K step into a zeroed tile,
                // then one round-to-nearest FP32 add into the running sum: the
                // tensor core's accumulator adds then only ever see one K
                // step's magnitude (their rounding would otherwise bias long
                // sums)
                uint32_t bh0, bl0, bh1, bl1;
                split_tf32(x0, bh0, bl0);
                split_tf32(x1, bh1, bl1);
                float t[4] = {0.f, 0.f, 0.f, 0.f};
                mma_tf32(t, al, bh0, bh1);
                mma_tf32(t, ah, bl0, bl1);
                mma_tf32(t, ah, bh0, bh1);
#pragma unroll
                for (int q = 0; q < 4; ++q) d[q] += t[q];
            } else {
                mma_tf32(d, ah, to_tf32(x0), to_tf32(x1));
            }
        }
    }
};

// Lower-triangle output tiles of the tensor-core forms: tile (mt, nt) covers
// rows 16 mt .. 16 mt + 15 and columns 8 nt .. 8 nt + 7.
template <int RT>
struct Tiles {
    static constexpr int MT = (RT + 15) / 16, NT = RT / 8;
    static constexpr int count() {
        int n = 0;
        for (int mt = 0; mt < MT; ++mt)
            for (int nt = 0; nt < NT; ++nt)
                if (16 * mt + 15 >= 8 * nt) ++n;
        return n;
    }
    static constexpr int NTL = count();
};

// (mt, nt) of lower tile t, tiles in row-major order (compile-time form).
template <int RT>
constexpr int tile_mt(int t) {
    int mt = 0;
    for (;;) {
        const int in_row = Tiles<RT>::NT < (16 * mt + 15) / 8 + 1 ? Tiles<RT>::NT : (16 * mt + 15) / 8 + 1;
        if (t < in_row) return mt;
        t -= in_row;
        ++mt;
    }
}
template <int RT>
constexpr int tile_nt(int t) {
    int mt = 0;
    for (;;) {
        const int in_row = Tiles<RT>::NT < (16 * mt + 15) / 8 + 1 ? Tiles<RT>::NT : (16 * mt + 15) / 8 + 1;
        if (t < in_row) return t;
        t -= in_row;
        ++mt;
    }
}

// (mt, nt) of lower tile t, tiles in row-major order.
template <int RT>
__device__ __forceinline__ void tile_at(int t, int &mt, int &nt) {
    mt = 0;
    for (;;) {
        const int in_row = min(Tiles<RT>::NT, (16 * mt + 15) / 8 + 1);
        if (t < in_row) break;
        t -= in_row;
        ++mt;
    }
    nt = t;
}

// Block size and reduction buffer of each form.
constexpr int pow2_floor(int x) { return x >= 32 ? 32 : x >= 16 ? 16 : x >= 8 ? 8 : x >= 4 ? 4 : x >= 2 ? 2 : 1; }

template <typename T, int RT, int KIND>
struct GramShape {
    static constexpr bool MMA = KIND != GK_FFMA;
    // FFMA: 4 x 4 thread tiles on the lower triangle; KS adjacent lanes share
    // a tile and split the nonzeros of a stage (reduced by shuffles)
    static constexpr int TR = RT / 4;
    static constexpr int NTILE = TR * (TR + 1) / 2;
    static constexpr int NTH = MMA ? 128 : (RT <= 8 ? 96 : 160);
    // tensor cores: KS warps share each tile (K split), NGRP tile groups
    static constexpr int NTL = Tiles<RT>::NTL;
    static constexpr int KS = MMA ? (RT >= 64 ? 1 : (RT >= 32 ? 2 : 4)) : pow2_floor(NTH / NTILE);
    static constexpr int NGRP = (NTH / 32) / (MMA ? KS : 1);
    static constexpr int TPW = (NTL + NGRP - 1) / NGRP;
    static constexpr int KCH = KIND == GK_BF16 ? 16 : 8;   // nonzeros per mma K step
    static constexpr bool COMP = !MMA && sizeof(T) == 4;
    // tensor cores: per-K-group partial tiles, reduced through shared memory
    static constexpr size_t red_bytes = (MMA && KS > 1) ? (size_t)KS * RT * RT * sizeof(float) : 0;
    // nonzero slices each thread gathers per stage (more for small ranks,
    // whose gathers are short and latency-bound)
    static constexpr int DEPTH = MMA ? 1 : (RT <= 16 ? 4 : 2);
    static_assert(!MMA || NGRP * TPW == NTL, "tiles divide evenly between the tile groups");
    static_assert(MMA || 32 % KS == 0, "a tile's K groups are adjacent lanes of one warp");
};

// Geometry of kernel A: per stage KB nonzeros gathered by the whole block in
// NSTEP rounds of NW * NG.
template <typename T, int RT, int KIND>
struct GramGeo {
    using SH = GramShape<T, RT, KIND>;
    static constexpr int NTH = SH::NTH, NW = NTH / 32;
    using L = Lay<T, RT, 32>;
    static constexpr int V = L::V, G = L::G, NG = L::NG;
    static constexpr int BSTEP = NW * NG;
    static constexpr int NSTEP0 = (32 + BSTEP - 1) / BSTEP;
    static constexpr int NSTEP = NSTEP0 > SH::DEPTH ? NSTEP0 : SH::DEPTH;
    static constexpr int KB = BSTEP * NSTEP;
    // staged row stride: padded so the fragment / tile loads spread over banks
    static constexpr int S = SH::MMA ? RT + (RT >= 16 ? 8 : 0) : RT + (sizeof(T) == 4 ? 4 : 0);
    static constexpr int TRI = RT * (RT + 1) / 2;
    static constexpr int EPT = (TRI + NTH - 1) / NTH;   // triangle entries per thread at a flush
    static constexpr size_t stage_bytes = ((sizeof(T) * (KB * S + KB) + 15) / 16) * 16;
    static constexpr size_t smem = stage_bytes + SH::red_bytes;
    static_assert(KB % SH::KCH == 0, "whole mma K steps per stage");
};

// FFMA form.  Thread t owns tile t / KS (if < NTILE) in K group t % KS.
template <typename T, int RT>
struct FfmaEngine {
    using SH = GramShape<T, RT, GK_FFMA>;
    static constexpr bool DIRECT = true;   // flushes by shuffles, no shared buffer
    static constexpr int FB = 32;     // FP32 terms per fold
    int r0, c0, kg, cnt;
    bool active;
    T acc[4][4];
    float hi[4][4], lo[4][4];

    __device__ __forceinline__ void init(int tid) {
        const int tile = tid / SH::KS;
        active = tile < SH::NTILE;
        int a = 0, b = 0;
        if (active) tri_rc(tile, a, b);
        r0 = 4 * a;
        c0 = 4 * b;
        kg = tid % SH::KS;
    }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                acc[i][j] = T(0);
                hi[i][j] = lo[i][j] = 0.f;
            }
        cnt = 0;
    }
    __device__ __forceinline__ void fold() {
        if constexpr (SH::COMP) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float s, e;
                    two_sum(hi[i][j], acc[i][j], s, e);
                    hi[i][j] = s;
                    lo[i][j] += e;
                    acc[i][j] = 0.f;
                }
        }
    }
    template <int S>
    __device__ __forceinline__ void accumulate(const T *hs, const T *ws, int nvalid) {
        if (!active) return;
        for (int k = kg; k < nvalid; k += SH::KS) {
            const T w = ws[k];
            const T *hk = hs + k * S;
            T a[4], c[4];
            if constexpr (sizeof(T) == 4) {
                const float4 x = *reinterpret_cast<const float4 *>(hk + r0);
                const float4 y = *reinterpret_cast<const float4 *>(hk + c0);
                a[0] = x.x; a[1] = x.y; a[2] = x.z; a[3] = x.w;
                c[0] = y.x; c[1] = y.y; c[2] = y.z; c[3] = y.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    a[q] = hk[r0 + q];
                    c[q] = hk[c0 + q];
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const T wa = w * a[i];
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += wa * c[j];
            }
            if constexpr (SH::COMP) {
                if (++cnt == FB) {
                    fold();
                    cnt = 0;
                }
            }
        }
    }
    // Sums the tile over its K groups (butterfly shuffles; every lane of the
    // warp takes part) and writes the lower entries of rows < R: plainly to
    // lrow or, for a row that crosses a chunk boundary, with FP64 atomics.
    __device__ __forceinline__ void flush(T *lrow, double *crow, bool whole, int R) {
        fold();
        cnt = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if constexpr (SH::COMP) {
                    float H = hi[i][j], Lo = lo[i][j];
#pragma unroll
                    for (int o = SH::KS / 2; o > 0; o >>= 1) {
                        const float H2 = __shfl_xor_sync(0xffffffffu, H, o);
                        const float L2 = __shfl_xor_sync(0xffffffffu, Lo, o);
                        float s, e;
                        two_sum(H, H2, s, e);
                        H = s;
                        Lo += L2 + e;
                    }
                    hi[i][j] = H;
                    lo[i][j] = Lo;
                } else {
                    T v = acc[i][j];
#pragma unroll
                    for (int o = SH::KS / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    acc[i][j] = v;
                }
            }
        if (!active || kg != 0) return;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = r0 + i, c = c0 + j;
                if (c > r || r >= R) continue;
                const int e = tri_idx(r, c);
                if constexpr (SH::COMP) {
                    if (whole) lrow[e] = hi[i][j] + lo[i][j];
                    else add_cut(crow + e, hi[i][j], lo[i][j]);
                } else {
                    if (whole) lrow[e] = acc[i][j];
                    else add_cut(crow + e, acc[i][j]);
                }
            }
    }
};

// Tensor-core forms (FP32 data only), block kernel: warp w owns tiles
// (w % NGRP) * TPW .. + TPW - 1 for K group w / NGRP.  With one K group (R =
// 64) every accumulator entry has one owner and the flush writes directly;
// otherwise the K groups are summed through shared memory.  The FP32-class
// form (TF32X3) folds its accumulators into compensated pairs every FOLDK
// K steps.
template <int RT, int KIND>
struct MmaEngine {
    using SH = GramShape<float, RT, KIND>;
    static constexpr bool DIRECT = SH::KS == 1;
    static constexpr bool COMP = KIND == GK_TF32X3;
    static constexpr int FOLDK = 16;      // K steps (128 nonzeros) between folds
    int kg, gid, tig, fc;
    int tmt[SH::TPW], tnt[SH::TPW];
    float d[SH::TPW][4];
    float hi[COMP ? SH::TPW : 1][4], lo[COMP ? SH::TPW : 1][4];

    __device__ __forceinline__ void init(int tid) {
        const int lane = tid & 31, w = tid >> 5;
        gid = lane >> 2;
        tig = lane & 3;
        kg = w / SH::NGRP;
        const int tg = w % SH::NGRP;
#pragma unroll
        for (int u = 0; u < SH::TPW; ++u) tile_at<RT>(tg * SH::TPW + u, tmt[u], tnt[u]);
    }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int u = 0; u < SH::TPW; ++u)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                d[u][q] = 0.f;
                if constexpr (COMP) hi[u][q] = lo[u][q] = 0.f;
            }
        fc = 0;
    }
    __device__ __forceinline__ void fold() {
        if constexpr (COMP) {
#pragma unroll
            for (int u = 0; u < SH::TPW; ++u)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float s, e;
                    two_sum(hi[u][q], d[u][q], s, e);
                    hi[u][q] = s;
                    lo[u][q] += e;
                    d[u][q] = 0.f;
                }
        }
    }
    template <int S>
    __device__ __forceinline__ void accumulate(const float *hf, const float *wf, int nvalid) {
        const int nkc = (nvalid + SH::KCH - 1) / SH::KCH;
        MmaStep<RT, KIND, S> step;
        for (int kc = kg; kc < nkc; kc += SH::KS) {
#pragma unroll
            for (int u = 0; u < SH::TPW; ++u) {
                if (u == 0 || tmt[u] != tmt[u - 1]) step.load_a(hf, kc, tmt[u], gid, tig);
                step.apply(hf, wf, kc, tnt[u], gid, tig, d[u]);
            }
            if constexpr (COMP) {
                if (++fc == FOLDK) {
                    fold();
                    fc = 0;
                }
            }
        }
    }
    __device__ __forceinline__ float value(int u, int q) const {
        if constexpr (COMP) return hi[u][q] + (lo[u][q] + d[u][q]);
        else return d[u][q];
    }
    // DIRECT: writes this lane's lower entries of rows < R.
    __device__ __forceinline__ void flush(float *lrow, double *crow, bool whole, int R) {
        fold();
        fc = 0;
#pragma unroll
        for (int u = 0; u < SH::TPW; ++u)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = tmt[u] * 16 + gid + (q >= 2 ? 8 : 0);
                const int c = tnt[u] * 8 + tig * 2 + (q & 1);
                if (r >= R || c > r) continue;
                const int e = tri_idx(r, c);
                if constexpr (COMP) {
                    if (whole) lrow[e] = hi[u][q] + lo[u][q];
                    else add_cut(crow + e, hi[u][q], lo[u][q]);
                } else {
                    if (whole) lrow[e] = d[u][q];
                    else add_cut(crow + e, d[u][q]);
                }
            }
    }
    __device__ __forceinline__ void to_red(unsigned char *red) {
        fold();
        fc = 0;
        float *mine = reinterpret_cast<float *>(red) + kg * RT * RT;
#pragma unroll
        for (int u = 0; u < SH::TPW; ++u)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = tmt[u] * 16 + gid + (q >= 2 ? 8 : 0);
                const int c = tnt[u] * 8 + tig * 2 + (q & 1);
                if (r < RT) mine[r * RT + c] = value(u, q);
            }
    }
    __device__ __forceinline__ void from_red(const unsigned char *red, int r, int c, double &v,
                                             float &v32) const {
        const float *x = reinterpret_cast<const float *>(red);
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < SH::KS; ++k) s += x[(k * RT + r) * RT + c];
        v = (double)s;
        v32 = s;
    }
};

template <typename T, int RT, int KIND>
struct EngineOf {
    using type = FfmaEngine<T, RT>;
};
template <int RT>
struct EngineOf<float, RT, GK_TF32> {
    using type = MmaEngine<RT, GK_TF32>;
};
template <int RT>
struct EngineOf<float, RT, GK_BF16> {
    using type = MmaEngine<RT, GK_BF16>;
};
template <int RT>
struct EngineOf<float, RT, GK_TF32X3> {
    using type = MmaEngine<RT, GK_TF32X3>;
};

template <typename T, int RT, bool VEC, int KIND>
__global__ void __launch_bounds__(GramShape<T, RT, KIND>::NTH, 2)
    gram_chunk_kernel(const SolveParams<T> P, const Batch<T> B) {
    using Q = GramGeo<T, RT, KIND>;
    using E = typename EngineOf<T, RT, KIND>::type;
    constexpr int V = Q::V, G = Q::G, NG = Q::NG, KB = Q::KB, S = Q::S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *hs = reinterpret_cast<T *>(smem_raw);
    T *ws = hs + KB * S;
    unsigned char *red = smem_raw + Q::stage_bytes;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int g = lane / G, lg = lane % G;
    const int R = VEC ? RT : P.R;
    const int tri = R * (R + 1) / 2;
    const int64_t nb = __ldg(P.row_ptr + B.row0), ne = __ldg(P.row_ptr + B.row0 + B.nrows);
    const int64_t last = B.row0 + B.nrows - 1;

    // triangle entries this thread writes at a flush
    constexpr int NE = E::DIRECT ? 1 : Q::EPT;
    int er[NE], ec[NE];
    if constexpr (!E::DIRECT) {
#pragma unroll
        for (int u = 0; u < NE; ++u) {
            const int e = tid + u * Q::NTH;
            if (e < tri) tri_rc(e, er[u], ec[u]);
            else er[u] = ec[u] = 0;
        }
    }
    E eng;
    eng.init(tid);

    // Software pipeline: the loads of stage s + 1 are issued right after stage
    // s is in shared memory, so they are in flight while the engine consumes
    // stage s -- across row boundaries too: the last stage of a row fetches
    // the next row's first stage, which is in flight during the flush.  pb /
    // pe / pw hold the fetched factor slices and raw weights (the value t for
    // phi'') of KB consecutive positions, clamped to the chunk; positions
    // past the current row are fetched but masked when staged.
    // RHS_VALUES: the values too (pt), each thread's share of sum_e t_e h_e
    // for the row (racc), folded over the block through rsm at the row's end
    const bool want_rhs = P.rhs_kind == RHS_VALUES;
    __shared__ T rsm[Q::NW][RT];
    T pb[Q::NSTEP][V], pe[Q::NSTEP][V], pw[Q::NSTEP], pt[Q::NSTEP], racc[V];
    int64_t ce = 0;
    auto fetch = [&](int64_t base) {
#pragma unroll
        for (int st = 0; st < Q::NSTEP; ++st) {
            const int slot = st * Q::BSTEP + w * NG + g;
            const int64_t qq = base + slot < ce ? base + slot : ce - 1;
            load_slice<T, V, VEC>(pb[st], P.A1, __ldcs(P.c1 + qq), R, lg);
            load_slice<T, V, VEC>(pe[st], P.A2, __ldcs(P.c2 + qq), R, lg);
            pw[st] = P.use_d2 ? __ldcs(P.t + qq) : weight_at(P.w, qq);
            pt[st] = want_rhs ? __ldcs(P.t + qq) : T(0);
        }
    };
    for (int64_t cs = nb + (int64_t)blockIdx.x * B.ch; cs < ne; cs += (int64_t)gridDim.x * B.ch) {
        ce = min(cs + B.ch, ne);
        int64_t i = search_le(P.row_ptr, B.row0, last, cs);
        bool ahead = false;
        for (;;) {
            const int64_t rs = __ldg(P.row_ptr + i), re = __ldg(P.row_ptr + i + 1);
            const int64_t ss = max(rs, cs), se = min(re, ce);
            T arow[V];
            if (P.use_d2) load_slice<T, V, VEC>(arow, P.Ad, i, R, lg);
            eng.zero();
#pragma unroll
            for (int t = 0; t < V; ++t) racc[t] = T(0);
            if (!ahead) fetch(ss);
            ahead = false;
            for (int64_t base = ss; base < se; base += KB) {
                // ---- stage KB nonzeros: h_e and weights
#pragma unroll
                for (int st = 0; st < Q::NSTEP; ++st) {
                    const int slot = st * Q::BSTEP + w * NG + g;
                    const bool valid = base + slot < se;
                    T h[V];
#pragma unroll
                    for (int t = 0; t < V; ++t) h[t] = pb[st][t] * pe[st][t];
                    T sw;
                    if (P.use_d2) {
                        T part = T(0);
#pragma unroll
                        for (int t = 0; t < V; ++t) part += arow[t] * h[t];
                        const T m = group_sum<G>(part);
                        T phi, d1, d2;
                        bool ok = true;
                        loss_terms(P.loss, pw[st], m, phi, d1, d2, ok);
                        if (!ok && valid) record_error(P.status, TC_ERR_DOMAIN);
                        sw = d2;
                    } else {
                        sw = pw[st];
                    }
                    if (!valid) {
                        sw = T(0);
#pragma unroll
                        for (int t = 0; t < V; ++t) h[t] = T(0);
                    }
                    if (want_rhs) {
#pragma unroll
                        for (int t = 0; t < V; ++t) racc[t] += pt[st] * h[t];
                    }
#pragma unroll
                    for (int t = 0; t < V; ++t) hs[slot * S + lg * V + t] = h[t];
                    if (lg == 0) ws[slot] = sw;
                }
                __syncthreads();
                if (base + KB < se) {
                    fetch(base + KB);
                } else if (se < ce) {
                    fetch(se);        // the next row's first stage (it starts at se)
                    ahead = true;
                }
                eng.template accumulate<S>(hs, ws, (int)min((int64_t)KB, se - base));
                __syncthreads();
            }
            // ---- flush the row's triangle
            const bool whole = rs >= cs && re <= ce;
            const int64_t slot = whole ? -1 : cut_slot(rs, re, nb, B.ch);
            T *lrow = B.light + (i - B.row0) * (int64_t)tri;
            double *crow = slot >= 0 ? B.cut + slot * (int64_t)tri : nullptr;
            if constexpr (E::DIRECT) {
                eng.flush(lrow, crow, whole, R);
            } else {
                // K groups reduced through `red` (the next flush writes `red`
                // only after at least one stage, whose barriers order it
                // after these reads)
                eng.to_red(red);
                __syncthreads();
#pragma unroll
                for (int u = 0; u < Q::EPT; ++u) {
                    const int e = tid + u * Q::NTH;
                    if (e < tri) {
                        double v;
                        float v32;
                        eng.from_red(red, er[u], ec[u], v, v32);
                        if (whole) lrow[e] = v32;
                        else atomicAdd(crow + e, v);
                    }
                }
            }
            if (want_rhs) {   // the row's right-hand side: groups, then warps
                T tot[V];
#pragma unroll
                for (int t = 0; t < V; ++t) tot[t] = across_groups<G>(racc[t]);
                if (g == 0) {
#pragma unroll
                    for (int t = 0; t < V; ++t)
                        if (lg * V + t < R) rsm[w][lg * V + t] = tot[t];
                }
                __syncthreads();
                for (int r = tid; r < R; r += Q::NTH) {
                    T v = T(0);
#pragma unroll
                    for (int ww = 0; ww < Q::NW; ++ww) v += rsm[ww][r];
                    if (whole) P.rhs_w[i * (int64_t)R + r] = v;
                    else add_cut(B.cut_rhs + slot * (int64_t)R + r, v);
                }
                __syncthreads();
            }
            if (re >= ce) break;
            i = search_le_near(P.row_ptr, i + 1, last, re);   // next nonempty row
        }
    }
}

// ------------------------------------------------------------------ kernel A, tcgen05, R = 64
// The TF32 and BF16 forms at R = 64 on the fifth-generation tensor cores:
// tcgen05.mma with the accumulator in tensor memory (TMEM), issued by one
// thread, the operands staged by the block in shared memory in the no-swizzle
// K-major layout (core matrices of 8 rows x 16 bytes).  One row segment at a
// time, in stages of 32 nonzeros: the block gathers h_e (rounded to the input
// type) and s_e h_e into one of two stage buffers, thread 0 issues the stage's
// MMAs -- D[m][n] += sum_k A[m][k] B[n][k] with A = h, B = s h -- and commits
// them to that buffer's mbarrier, and the block gathers the next stage into
// the other buffer meanwhile.  The MMA shape is M = 128, N = 64: rows 64..127
// of A stay zero, and D's rows 0..63 (TMEM lanes 0..63) hold G_i.  At the
// row's end warps 0 and 1 read them (tcgen05.ld) and write the packed lower
// triangle, or add it with FP64 atomics into the cut slot of a row that
// crosses a chunk boundary.  For an ALS update each thread also sums t_e h_e
// for its components (FP32, on the CUDA cores: a TF32 or BF16 right-hand side
// would not do), the warps' shares meet in shared memory and the segment's
// epilogue writes the row's right-hand side.  Every mbarrier wait has a time
// limit; past it the block records TC_ERR_TIMEOUT, lets its committed MMAs
// finish (bounded), frees its TMEM and leaves.
namespace tc05 {

constexpr int KB = 32;          // nonzeros per stage
constexpr int MM = 128;         // MMA rows (A's rows 64..127 are zero)
constexpr int NN = 64;          // MMA columns = R
constexpr int LBO = 128;        // bytes between core matrices adjacent in K
constexpr int THREADS = 128;
constexpr uint32_t TMEM_COLS = 128;    // two accumulators of 64 columns
constexpr uint64_t WAIT_NS = 2000000000ull;

template <int KIND>
struct Geo {
    static constexpr int EB = KIND == GK_BF16 ? 2 : 4;        // bytes per element
    static constexpr int EPC = 16 / EB;                       // K elements per core-matrix row
    static constexpr int SBO = (KB / EPC) * 128;              // bytes between 8-row groups
    static constexpr int A_BYTES = MM * KB * EB;
    static constexpr int B_BYTES = NN * KB * EB;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int KI = KIND == GK_BF16 ? 16 : 8;       // K per instruction
    static constexpr int NI = KB / KI;                        // instructions per stage
    static constexpr int SMEM = 2 * STAGE + 128;              // + room to align the base
    // instruction descriptor: D FP32 (bits 4-5), A and B type (bits 7-9 and
    // 10-12: 2 = TF32 for kind::tf32, 1 = BF16 for kind::f16), both K-major,
    // N >> 3 (bits 17-22), M >> 4 (bits 24-28)
    static constexpr uint32_t IDESC = (1u << 4) | ((KIND == GK_BF16 ? 1u : 2u) << 7) |
                                      ((KIND == GK_BF16 ? 1u : 2u) << 10) |
                                      ((uint32_t)(NN >> 3) << 17) | ((uint32_t)(MM >> 4) << 24);
    // byte offset of element (row, k) of an operand tile
    __device__ static __forceinline__ int off(int row, int k) {
        return (row >> 3) * SBO + (k / EPC) * LBO + (row & 7) * 16 + (k % EPC) * EB;
    }
};

// Shared-memory matrix descriptor: start address, leading (K) and stride
// (8-row group) byte offsets in 16-byte units, the fixed version bits 46-48 =
// 0b001, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, int sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((LBO >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ uint32_t smem_addr(const void *ptr) {
    return (uint32_t)__cvta_generic_to_shared(ptr);
}

// Orders this thread's generic-proxy shared-memory stores before the tensor
// core's (asynchronous-proxy) reads of them.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint16_t to_bf16(float x) {
    uint16_t r;
    asm("cvt.rn.bf16.f32 %0, %1;" : "=h"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the completion of phase `parity` of the mbarrier; false if the
// limit passed first.
__device__ __forceinline__ bool wait_phase(uint32_t bar, uint32_t parity, uint64_t limit) {
    uint32_t done = 0;
    uint64_t t0 = 0;
    for (;;) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        const uint64_t t = now_ns();
        if (t0 == 0) t0 = t;
        else if (t - t0 > limit) return false;
    }
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                    uint32_t acc, int kind_bf16) {
    if (kind_bf16)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
}

__device__ __forceinline__ void commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

}  // namespace tc05

template <int KIND>
__global__ void __launch_bounds__(tc05::THREADS) gram_tc05_kernel(const SolveParams<float> P,
                                                                 const Batch<float> B) {
    using Q = tc05::Geo<KIND>;
    constexpr int R = 64, TRI = R * (R + 1) / 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    // RHS_VALUES: each warp's partial right-hand side of the last two row
    // segments (by accumulator parity), summed by the segment's epilogue
    __shared__ float rpart[2][tc05::THREADS / 32][64];
    unsigned char *base =
        reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = tc05::smem_addr(base);
    const uint32_t bar0 = tc05::smem_addr(&mbar[0]);

    // rows 64..127 of A stay zero in both stage buffers
    for (int o = tid * 4; o < Q::A_BYTES / 2; o += tc05::THREADS * 4) {
        *reinterpret_cast<uint32_t *>(base + Q::A_BYTES / 2 + o) = 0u;
        *reinterpret_cast<uint32_t *>(base + Q::STAGE + Q::A_BYTES / 2 + o) = 0u;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc05::smem_addr(&tmem_slot)),
                     "r"(tc05::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc05::fence_before();
    __syncthreads();
    tc05::fence_after();
    const uint32_t tmem = tmem_slot;

    const int64_t nb = __ldg(P.row_ptr + B.row0), ne = __ldg(P.row_ptr + B.row0 + B.nrows);
    const int64_t last = B.row0 + B.nrows - 1;
    // gather mapping: lane i of warp w holds nonzero slots 8w + 4h + i % 4
    // (h = 0, 1) and components i / 4 + 8j (j = 0..7), so each shared store of
    // a warp fills one core matrix (or half of one for BF16) without conflicts
    const int kl = lane & 3, m0 = lane >> 2;
    const bool want_rhs = P.rhs_kind == RHS_VALUES;
    float racc[8];             // this thread's sum_e t_e h_e[m0 + 8j] over its slots
    int st_cnt = 0;            // stages committed by this block
    int row_cnt = 0;           // row segments started by this block
    bool ok = true;
    // The row segment whose Gram is still in TMEM: its epilogue runs once the
    // next segment's first MMAs are issued (into the other accumulator), so
    // its MMA latency and read-out overlap the next segment's work.
    struct Pending {
        int64_t row, slot;
        int stage, dbuf;
        bool whole, valid;
    } pend{0, -1, 0, 0, false, false};

    // waits for a segment's last stage, reads its accumulator and writes the
    // packed lower triangle (or adds it into its cut slot); block-wide
    auto epilogue = [&](const Pending &pr) -> bool {
        const bool w = tc05::wait_phase(bar0 + 8 * (pr.stage & 1), (uint32_t)((pr.stage >> 1) & 1),
                                        tc05::WAIT_NS);
        if (__syncthreads_or(!w)) return false;
        tc05::fence_after();
        if (warp < 2) {
            const int r = 32 * warp + lane;
            float *lrow = B.light + (pr.row - B.row0) * (int64_t)TRI + tri_idx(r, 0);
            double *crow = pr.slot >= 0 ? B.cut + pr.slot * (int64_t)TRI + tri_idx(r, 0) : nullptr;
#pragma unroll
            for (int c0 = 0; c0 < R; c0 += 16) {
                float v[16];
                tc05::ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(pr.dbuf * tc05::NN + c0), v);
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    if (c0 + c > r) continue;
                    if (pr.whole) lrow[c0 + c] = v[c];
                    else add_cut(crow + c0 + c, v[c]);
                }
            }
        }
        if (want_rhs && tid < R) {
            float v = 0.f;
#pragma unroll
            for (int ww = 0; ww < tc05::THREADS / 32; ++ww) v += rpart[pr.dbuf][ww][tid];
            if (pr.whole) P.rhs_w[pr.row * (int64_t)R + tid] = v;
            else add_cut(B.cut_rhs + pr.slot * (int64_t)R + tid, v);
        }
        tc05::fence_before();
        __syncthreads();              // that accumulator is free again
        return true;
    };

    for (int64_t cs = nb + (int64_t)blockIdx.x * B.ch; cs < ne && ok; cs += (int64_t)gridDim.x * B.ch) {
        const int64_t ce = min(cs + B.ch, ne);
        int64_t i = search_le(P.row_ptr, B.row0, last, cs);
        for (;;) {
            const int64_t rs = __ldg(P.row_ptr + i), re = __ldg(P.row_ptr + i + 1);
            const int64_t ss = max(rs, cs), se = min(re, ce);
            const int dbuf = row_cnt & 1;
#pragma unroll
            for (int j = 0; j < 8; ++j) racc[j] = 0.f;
            for (int64_t sb = ss; sb < se; sb += tc05::KB) {
                const int buf = st_cnt & 1;
                const uint32_t bar = bar0 + 8 * buf;
                if (st_cnt >= 2) {     // the MMAs that last read this buffer are done
                    const bool w = tc05::wait_phase(bar, (uint32_t)(((st_cnt - 2) >> 1) & 1), tc05::WAIT_NS);
                    if (__syncthreads_or(!w)) {
                        ok = false;
                        break;
                    }
                }
                unsigned char *As = base + buf * Q::STAGE, *Bs = As + Q::A_BYTES;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int k = 8 * warp + 4 * hh + kl;
                    const int64_t q = sb + k;
                    const bool valid = q < se;
                    float bv[8], ev[8], sw = 0.f, tv = 0.f;
                    if (valid) {
                        const float *br = P.A1 + (int64_t)__ldcs(P.c1 + q) * R;
                        const float *er = P.A2 + (int64_t)__ldcs(P.c2 + q) * R;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            bv[j] = __ldg(br + m0 + 8 * j);
                            ev[j] = __ldg(er + m0 + 8 * j);
                        }
                        sw = weight_at(P.w, q);
                        if (want_rhs) tv = __ldcs(P.t + q);
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int m = m0 + 8 * j;
                        const float h = valid ? bv[j] * ev[j] : 0.f;
                        const float wh = sw * h;
                        racc[j] = fmaf(tv, h, racc[j]);
                        const int o = Q::off(m, k);
                        if constexpr (KIND == GK_BF16) {
                            *reinterpret_cast<uint16_t *>(As + o) = tc05::to_bf16(h);
                            *reinterpret_cast<uint16_t *>(Bs + o) = tc05::to_bf16(wh);
                        } else {
                            *reinterpret_cast<uint32_t *>(As + o) = to_tf32(h);
                            *reinterpret_cast<uint32_t *>(Bs + o) = to_tf32(wh);
                        }
                    }
                }
                tc05::fence_proxy_async();     // the stores, before the tensor core reads them
                tc05::fence_before();
                __syncthreads();
                if (tid == 0) {
                    tc05::fence_after();
                    const uint32_t a0 = sbase + buf * Q::STAGE, b0 = a0 + Q::A_BYTES;
#pragma unroll
                    for (int ii = 0; ii < Q::NI; ++ii) {
                        const uint32_t ko = (uint32_t)(ii * (Q::KI / Q::EPC) * tc05::LBO);
                        tc05::mma(tmem + (uint32_t)(dbuf * tc05::NN), tc05::smem_desc(a0 + ko, Q::SBO),
                                  tc05::smem_desc(b0 + ko, Q::SBO), Q::IDESC,
                                  (sb > ss || ii > 0) ? 1u : 0u, KIND == GK_BF16);
                    }
                    tc05::commit(bar);
                }
                ++st_cnt;
                if (sb == ss && pend.valid) {    // the previous segment, behind this one's MMAs
                    if (!epilogue(pend)) {
                        ok = false;
                        break;
                    }
                    pend.valid = false;
                }
            }
            if (!ok) break;
            if (want_rhs) {   // this warp's share: its 8 slots per stage, lanes of equal m0 summed
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float v = racc[j];
                    v += __shfl_xor_sync(0xffffffffu, v, 1);
                    v += __shfl_xor_sync(0xffffffffu, v, 2);
                    if (kl == 0) rpart[dbuf][warp][m0 + 8 * j] = v;
                }
            }
            const bool whole = rs >= cs && re <= ce;
            pend = Pending{i, whole ? -1 : cut_slot(rs, re, nb, B.ch), st_cnt - 1, dbuf, whole, true};
            ++row_cnt;
            if (re >= ce) break;
            i = search_le_near(P.row_ptr, i + 1, last, re);   // next nonempty row
        }
    }
    if (ok && pend.valid) ok = epilogue(pend);
    if (!ok) {
        if (tid == 0) record_error(P.status, TC_ERR_TIMEOUT);
        // let the committed MMAs finish before the TMEM is released (bounded)
        for (int s = st_cnt > 2 ? st_cnt - 2 : 0; s < st_cnt; ++s)
            tc05::wait_phase(bar0 + 8 * (s & 1), (uint32_t)((s >> 1) & 1), tc05::WAIT_NS / 4);
        tc05::fence_before();
        __syncthreads();
    }
    if (warp == 0) {
        tc05::fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(tc05::TMEM_COLS)
                     : "memory");
    }
}

// ------------------------------------------------------------------ kernel A, small ranks
// For R <= 16 (FFMA form) every warp works alone: it takes every nwarps-th
// chunk of the batch's nonzeros, stages DEPTH x NG nonzeros (h_e and weight)
// in its own shared-memory region, and each lane accumulates a TR x TC block
// of the full R x R Gram in registers (the whole square is 32 lanes x TR x TC
// entries, so every entry has one owner and no reduction is needed; the
// upper half is computed and dropped, which costs less than splitting the
// triangle unevenly).  Sums are folded every 32 terms into compensated FP32
// pairs as in the block form.  No block barrier anywhere: warps stall only
// on their own gathers.
template <typename T, int RT>
struct WarpGram {
    static constexpr int NW = 4, NTH = NW * 32;
    using L = Lay<T, RT, 32>;
    static constexpr int V = L::V, G = L::G, NG = L::NG;
    static constexpr int DEPTH = 4;
    static constexpr int KBW = NG * DEPTH;                 // nonzeros per warp stage
    static constexpr int TC = RT >= 16 ? 4 : 2;            // lane block: TR rows x TC cols
    static constexpr int TR = RT * RT / 32 / TC;
    static constexpr int S = RT + (sizeof(T) == 4 ? 4 : 0);
    static constexpr size_t warp_bytes = ((sizeof(T) * (KBW * S + KBW) + 15) / 16) * 16;
    static constexpr size_t smem = NW * warp_bytes;
    static constexpr bool COMP = sizeof(T) == 4;
    static_assert(TR * TC * 32 == RT * RT, "the lanes cover the square");
};

template <typename T, int RT, bool VEC>
__global__ void __launch_bounds__(128) gram_warp_kernel(const SolveParams<T> P, const Batch<T> B) {
    using Q = WarpGram<T, RT>;
    constexpr int V = Q::V, G = Q::G, NG = Q::NG, KBW = Q::KBW, S = Q::S, TR = Q::TR, TC = Q::TC;
    constexpr int FB = 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T *hs = reinterpret_cast<T *>(smem_raw + w * Q::warp_bytes);
    T *ws = hs + KBW * S;
    const int g = lane / G, lg = lane % G;
    const int R = VEC ? RT : P.R;
    const int tri = R * (R + 1) / 2;
    const int r0 = (lane / (RT / TC)) * TR, c0 = (lane % (RT / TC)) * TC;
    const int64_t nb = __ldg(P.row_ptr + B.row0), ne = __ldg(P.row_ptr + B.row0 + B.nrows);
    const int64_t last = B.row0 + B.nrows - 1;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    T acc[TR][TC];
    float hi[TR][TC], lo[TR][TC];
    for (int64_t cs = nb + gw * B.ch; cs < ne; cs += nwarps * B.ch) {
        const int64_t ce = min(cs + B.ch, ne);
        int64_t i = search_le(P.row_ptr, B.row0, last, cs);
        for (;;) {
            const int64_t rs = __ldg(P.row_ptr + i), re = __ldg(P.row_ptr + i + 1);
            const int64_t ss = max(rs, cs), se = min(re, ce);
            T arow[V];
            if (P.use_d2) load_slice<T, V, VEC>(arow, P.Ad, i, R, lg);
#pragma unroll
            for (int a = 0; a < TR; ++a)
#pragma unroll
                for (int b = 0; b < TC; ++b) {
                    acc[a][b] = T(0);
                    hi[a][b] = lo[a][b] = 0.f;
                }
            int cnt = 0;
            for (int64_t base = ss; base < se; base += KBW) {
#pragma unroll
                for (int st = 0; st < Q::DEPTH; ++st) {
                    const int slot = st * NG + g;
                    const bool valid = base + slot < se;
                    const int64_t qq = valid ? base + slot : se - 1;
                    T b[V], e[V], h[V];
                    load_slice<T, V, VEC>(b, P.A1, __ldcs(P.c1 + qq), R, lg);
                    load_slice<T, V, VEC>(e, P.A2, __ldcs(P.c2 + qq), R, lg);
#pragma unroll
                    for (int t = 0; t < V; ++t) h[t] = b[t] * e[t];
                    T sw;
                    if (P.use_d2) {
                        T part = T(0);
#pragma unroll
                        for (int t = 0; t < V; ++t) part += arow[t] * h[t];
                        const T m = group_sum<G>(part);
                        T phi, d1, d2;
                        bool ok = true;
                        loss_terms(P.loss, __ldcs(P.t + qq), m, phi, d1, d2, ok);
                        if (!ok && valid) record_error(P.status, TC_ERR_DOMAIN);
                        sw = d2;
                    } else {
                        sw = weight_at(P.w, qq);
                    }
                    if (!valid) {
                        sw = T(0);
#pragma unroll
                        for (int t = 0; t < V; ++t) h[t] = T(0);
                    }
#pragma unroll
                    for (int t = 0; t < V; ++t) hs[slot * S + lg * V + t] = h[t];
                    if (lg == 0) ws[slot] = sw;
                }
                __syncwarp();
                const int nvalid = (int)min((int64_t)KBW, se - base);
                for (int k = 0; k < nvalid; ++k) {
                    const T wk = ws[k];
                    const T *hk = hs + k * S;
                    T a[TR], c[TC];
#pragma unroll
                    for (int q = 0; q < TR; ++q) a[q] = wk * hk[r0 + q];
#pragma unroll
                    for (int q = 0; q < TC; ++q) c[q] = hk[c0 + q];
#pragma unroll
                    for (int x = 0; x < TR; ++x)
#pragma unroll
                        for (int y = 0; y < TC; ++y) acc[x][y] += a[x] * c[y];
                    if constexpr (Q::COMP) {
                        if (++cnt == FB) {
                            cnt = 0;
#pragma unroll
                            for (int x = 0; x < TR; ++x)
#pragma unroll
                                for (int y = 0; y < TC; ++y) {
                                    float s, er;
                                    two_sum(hi[x][y], acc[x][y], s, er);
                                    hi[x][y] = s;
                                    lo[x][y] += er;
                                    acc[x][y] = 0.f;
                                }
                        }
                    }
                }
                __syncwarp();
            }
            // ---- flush: each lane writes its own lower entries
            const bool whole = rs >= cs && re <= ce;
            const int64_t slot = whole ? -1 : cut_slot(rs, re, nb, B.ch);
            T *lrow = B.light + (i - B.row0) * (int64_t)tri;
            double *crow = slot >= 0 ? B.cut + slot * (int64_t)tri : nullptr;
#pragma unroll
            for (int x = 0; x < TR; ++x)
#pragma unroll
                for (int y = 0; y < TC; ++y) {
                    const int r = r0 + x, c = c0 + y;
                    if (c > r || r >= R) continue;
                    const int e = tri_idx(r, c);
                    if constexpr (Q::COMP) {
                        float s, er;
                        two_sum(hi[x][y], acc[x][y], s, er);
                        const float l2 = lo[x][y] + er;
                        if (whole) lrow[e] = s + l2;
                        else add_cut(crow + e, s, l2);
                    } else {
                        if (whole) lrow[e] = acc[x][y];
                        else add_cut(crow + e, acc[x][y]);
                    }
                }
            if (re >= ce) break;
            i = search_le_near(P.row_ptr, i + 1, last, re);   // next nonempty row
        }
    }
}

// ------------------------------------------------------------------ kernel A, tensor cores, R <= 32
// Tensor-core forms for ranks up to 32: every warp works alone, like
// gram_warp_kernel, and holds every lower output tile of the Gram in its
// mma accumulators (R = 32: 6 tiles, 24 floats per lane; R = 16: 2 tiles),
// so each entry has one owner lane and the flush needs no reduction.  The
// FP32-class form folds the accumulators every 16 K steps into compensated
// pairs held in registers.
template <int RT, int KIND>
struct WarpMma {
    static constexpr int NW = 4, NTH = NW * 32;
    using L = Lay<float, RT, 32>;
    static constexpr int V = L::V, G = L::G, NG = L::NG;
    static constexpr int KCH = KIND == GK_BF16 ? 16 : 8;
    static constexpr int DEPTH = 4;
    static constexpr int KBW = NG * DEPTH;                 // nonzeros per warp stage
    static constexpr int S = RT + (RT >= 16 ? 8 : 0);
    static constexpr int NTL = Tiles<RT>::NTL;
    static constexpr bool COMP = KIND == GK_TF32X3;
    static constexpr int FOLDK = 16;
    // per warp: staged h rows, Gram weights, right-hand-side weights
    static constexpr size_t warp_bytes = ((sizeof(float) * (KBW * S + 2 * KBW) + 15) / 16) * 16;
    static constexpr size_t smem = NW * warp_bytes;
    // right-hand side: lane l sums component l % RP over the staged rows
    // k = l / RP, l / RP + 32 / RP, ... (RP: R rounded up to a power of two)
    static constexpr int RP = RT <= 8 ? 8 : RT <= 16 ? 16 : 32;
    static_assert(KBW % KCH == 0, "whole K steps per stage");
};

// RK (RhsKind): what the pass forms beside the Gram -- a compile-time choice,
// so that the plain Gram keeps its registers (and blocks per SM).
template <int RT, bool VEC, int KIND, int RK = RHS_GIVEN>
__global__ void __launch_bounds__(128) gram_warp_mma_kernel(const SolveParams<float> P,
                                                            const Batch<float> B) {
    using Q = WarpMma<RT, KIND>;
    constexpr int V = Q::V, G = Q::G, NG = Q::NG, KBW = Q::KBW, S = Q::S, NTL = Q::NTL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float *hs = reinterpret_cast<float *>(smem_raw + w * Q::warp_bytes);
    float *ws = hs + KBW * S;
    float *rws = ws + KBW;      // rhs_kind: the right-hand-side weight of each staged row
    const int g = lane / G, lg = lane % G;
    const int gid = lane >> 2, tig = lane & 3;
    const int R = VEC ? RT : P.R;
    const int tri = R * (R + 1) / 2;
    const int64_t nb = __ldg(P.row_ptr + B.row0), ne = __ldg(P.row_ptr + B.row0 + B.nrows);
    const int64_t last = B.row0 + B.nrows - 1;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    float d[NTL][4];
    float hi[Q::COMP ? NTL : 1][4], lo[Q::COMP ? NTL : 1][4];
    // rhs_kind: this lane's share of component lane % RP of the row's
    // right-hand side, summed from the staged rows (so the staging keeps no
    // extra registers live)
    constexpr bool want_rhs = RK != RHS_GIVEN;
    const int rcomp = lane % Q::RP, rk0 = lane / Q::RP;
    float racc = 0.f;
    double lacc = 0.0;  // loss_acc: this lane's share of sum_e phi
    for (int64_t cs = nb + gw * B.ch; cs < ne; cs += nwarps * B.ch) {
        const int64_t ce = min(cs + B.ch, ne);
        int64_t i = search_le(P.row_ptr, B.row0, last, cs);
        for (;;) {
            const int64_t rs = __ldg(P.row_ptr + i), re = __ldg(P.row_ptr + i + 1);
            const int64_t ss = max(rs, cs), se = min(re, ce);
            float arow[V];
            if (P.use_d2) load_slice<float, V, VEC>(arow, P.Ad, i, R, lg);
#pragma unroll
            for (int u = 0; u < NTL; ++u)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    d[u][q] = 0.f;
                    if constexpr (Q::COMP) hi[u][q] = lo[u][q] = 0.f;
                }
            racc = 0.f;
            int fc = 0;
            for (int64_t base = ss; base < se; base += KBW) {
#pragma unroll
                for (int st = 0; st < Q::DEPTH; ++st) {
                    const int slot = st * NG + g;
                    const bool valid = base + slot < se;
                    const int64_t qq = valid ? base + slot : se - 1;
                    float b[V], e[V], h[V];
                    load_slice<float, V, VEC>(b, P.A1, __ldcs(P.c1 + qq), R, lg);
                    load_slice<float, V, VEC>(e, P.A2, __ldcs(P.c2 + qq), R, lg);

#pragma unroll
                    for (int t = 0; t < V; ++t) h[t] = b[t] * e[t];
                    float sw, rw = 0.f;
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
                        if constexpr (RK == RHS_DPHI) {
                            rw = d1;
                            if (P.loss_acc && valid && lg == 0) lacc += (double)phi;
                        }
                    } else {
                        sw = weight_at(P.w, qq);
                        if constexpr (RK == RHS_VALUES) rw = __ldcs(P.t + qq);
                    }
                    if (!valid) {
                        sw = 0.f;
#pragma unroll
                        for (int t = 0; t < V; ++t) h[t] = 0.f;
                    }
#pragma unroll
                    for (int t = 0; t < V; ++t) hs[slot * S + lg * V + t] = h[t];
                    if (lg == 0) {
                        ws[slot] = sw;
                        if constexpr (want_rhs) rws[slot] = valid ? rw : 0.f;
                    }
                }
                __syncwarp();
                if constexpr (want_rhs) {
                    if (rcomp < R) {
                        const int nk = (int)min((int64_t)KBW, se - base);
#pragma unroll 1
                        for (int k = rk0; k < nk; k += 32 / Q::RP)
                            racc = fmaf(rws[k], hs[k * S + rcomp], racc);
                    }
                }
                const int nkc = ((int)min((int64_t)KBW, se - base) + Q::KCH - 1) / Q::KCH;
                MmaStep<RT, KIND, S> step;
                for (int kc = 0; kc < nkc; ++kc) {
#pragma unroll
                    for (int u = 0; u < NTL; ++u) {
                        if (u == 0 || tile_mt<RT>(u) != tile_mt<RT>(u - 1))
                            step.load_a(hs, kc, tile_mt<RT>(u), gid, tig);
                        step.apply(hs, ws, kc, tile_nt<RT>(u), gid, tig, d[u]);
                    }
                    if constexpr (Q::COMP) {
                        if (++fc == Q::FOLDK) {
                            fc = 0;
#pragma unroll
                            for (int u = 0; u < NTL; ++u)
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    float sm, er;
                                    two_sum(hi[u][q], d[u][q], sm, er);
                                    hi[u][q] = sm;
                                    lo[u][q] += er;
                                    d[u][q] = 0.f;
                                }
                        }
                    }
                }
                __syncwarp();
            }
            // ---- flush: each lane writes its own lower entries
            const bool whole = rs >= cs && re <= ce;
            const int64_t slot = whole ? -1 : cut_slot(rs, re, nb, B.ch);
            float *lrow = B.light + (i - B.row0) * (int64_t)tri;
            double *crow = slot >= 0 ? B.cut + slot * (int64_t)tri : nullptr;
#pragma unroll
            for (int u = 0; u < NTL; ++u)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int r = tile_mt<RT>(u) * 16 + gid + (q >= 2 ? 8 : 0);
                    const int c = tile_nt<RT>(u) * 8 + tig * 2 + (q & 1);
                    if (r >= R || c > r) continue;
                    const int e = tri_idx(r, c);
                    if constexpr (Q::COMP) {
                        float sm, er;
                        two_sum(hi[u][q], d[u][q], sm, er);
                        const float l2 = lo[u][q] + er;
                        if (whole) lrow[e] = sm + l2;
                        else add_cut(crow + e, sm, l2);
                    } else {
                        if (whole) lrow[e] = d[u][q];
                        else add_cut(crow + e, d[u][q]);
                    }
                }
            if constexpr (want_rhs) {   // the row's right-hand side: lanes of one component summed
                float v = racc;
#pragma unroll
                for (int o = Q::RP; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane < R) {
                    if (whole) P.rhs_w[i * (int64_t)R + lane] = v;
                    else add_cut(B.cut_rhs + slot * (int64_t)R + lane, v);
                }
            }
            if (re >= ce) break;
            i = search_le_near(P.row_ptr, i + 1, last, re);   // next nonempty row
        }
    }
    if constexpr (RK == RHS_DPHI) {
        if (P.loss_acc) block_add(lacc, P.loss_acc);
    }
}

// Gram entry e of batch row q (zero for an empty row).
template <typename T>
__device__ __forceinline__ double gram_entry(const T *lrow, const double *crow, int e) {
    if (crow) return crow[e];
    if (lrow) return (double)lrow[e];
    return 0.0;
}

template <typename T>
__device__ __forceinline__ void gram_source(const SolveParams<T> &P, const Batch<T> &B, int64_t nb,
                                            int64_t i, int tri, const T *&lrow,
                                            const double *&crow) {
    const int64_t rs = __ldg(P.row_ptr + i), re = __ldg(P.row_ptr + i + 1);
    lrow = nullptr;
    crow = nullptr;
    if (re == rs) return;
    const int64_t slot = cut_slot(rs, re, nb, B.ch);
    if (slot >= 0) crow = B.cut + slot * (int64_t)tri;
    else lrow = B.light + (i - B.row0) * (int64_t)tri;
}

// ------------------------------------------------------------------ kernel B, R <= 32
// rpw rows per warp, lpr = 32 / rpw lanes per row (lane = slot * lpr + sub).
// Shared layout: packed entry e of slot s at e * (rpw + 1) + s.  Every slot
// runs the same sequence of entries, so the lpr lanes of a row deal each
// step's work among themselves round-robin -- the entries of the trailing
// update, the rows of a substitution step, the columns of L^-1, the entries
// of the inverse -- and the warp meets at a barrier between steps.  FP64
// throughput on this part is charged per warp instruction, so filling all 32
// lanes (rather than one lane per row) is what keeps the pipe busy with
// useful work.  A row that is not positive definite runs on, on values that
// are discarded, so the warp keeps one instruction stream through every
// barrier.  Inverse mode keeps L^-1 in a second triangle (out of place, so
// its columns are independent).  With refinement the factor L is written
// back over the batch's Gram rows (pattern dtype; a zero first entry marks a
// row that did not factor) for the correction step.

// Moves (a, b) -- row and column of a packed lower-triangle entry -- forward
// by `step` entries.
__device__ __forceinline__ void tri_advance(int &a, int &b, int step) {
    b += step;
    while (b > a) {
        b -= a + 1;
        ++a;
    }
}

template <typename T, typename CT>
__global__ void __launch_bounds__(32) chol_rows_kernel(const SolveParams<T> P, const Batch<T> B,
                                                       int rpw) {
    extern __shared__ __align__(16) unsigned char sh_raw[];
    CT *sh = reinterpret_cast<CT *>(sh_raw);
    const int lane = threadIdx.x;
    const int R = P.R, tri = R * (R + 1) / 2, ps = rpw + 1;
    const int lpr = 32 / rpw, slot = lane / lpr, sub = lane - slot * lpr;
    const bool inv_mode = P.pinv != nullptr;
    const int64_t q0 = (int64_t)blockIdx.x * rpw;
    const int nr = (int)min((int64_t)rpw, B.nrows - q0);
    const int64_t nb = __ldg(P.row_ptr + B.row0);
    CT *Tri = sh;
    CT *Vv = sh + (int64_t)tri * ps;
    CT *Dinv = Vv + (int64_t)R * ps;
    CT *Yt = Dinv + (int64_t)R * ps;         // inverse mode: L^-1
    {
        // the first nr lanes find their rows' Gram sources (in parallel), then
        // the warp copies every slot's triangle in one flat loop, the row
        // pointers broadcast by shuffles; slots past the batch get zeros
        const T *lmine = nullptr;
        const double *cmine = nullptr;
        if (lane < nr) gram_source(P, B, nb, B.row0 + q0 + lane, tri, lmine, cmine);
        const int n = rpw * tri;
#pragma unroll 4
        for (int base = 0; base < n; base += 32) {
            const int idx = base + lane;
            const int sl = idx < n ? idx / tri : 0;
            const T *lrow = reinterpret_cast<const T *>(
                __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(lmine), sl));
            const double *crow = reinterpret_cast<const double *>(
                __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(cmine), sl));
            if (idx < n) {
                const int e = idx - sl * tri;
                Tri[e * ps + sl] = gram_entry(lrow, crow, e);
            }
        }
    }
    const bool mine = slot < nr;
    const int64_t i = B.row0 + q0 + slot;
#define TC_TRI(r, c) Tri[tri_idx(r, c) * ps + slot]
#define TC_Y(r, c) Yt[tri_idx(r, c) * ps + slot]
#define TC_VEC(r) Vv[(r) * ps + slot]
#define TC_DINV(r) Dinv[(r) * ps + slot]
    __syncwarp();
    for (int r = sub; r < R; r += lpr) TC_TRI(r, r) += (CT)P.lambda;
    __syncwarp();
    bool ok = true;
    for (int j = 0; j < R; ++j) {
        const CT dj = TC_TRI(j, j);
        ok = ok && dj > CT(0);
        const CT inv = rsqrt_nr(dj), ljj = dj * inv;
        __syncwarp();                         // every lane has read the pivot
        if (sub == 0) {
            TC_TRI(j, j) = ljj;
            TC_DINV(j) = inv;
        }
        for (int r = j + 1 + sub; r < R; r += lpr) TC_TRI(r, j) *= inv;
        __syncwarp();
        // trailing update of rows and columns j+1 .. R-1: entry (a, b) of the
        // trailing triangle is (j+1+a, j+1+b); four entries per pass, loads
        // before stores (entries of one step are distinct, column j is read only)
        const int n1 = R - 1 - j, ntr = n1 * (n1 + 1) / 2, c0 = j + 1;
        int a = 0, b = 0;
        tri_advance(a, b, sub);
        int t = sub;
        for (; t + 3 * lpr < ntr; t += 4 * lpr) {
            const int a0 = a, b0 = b;
            tri_advance(a, b, lpr);
            const int a1 = a, b1 = b;
            tri_advance(a, b, lpr);
            const int a2 = a, b2 = b;
            tri_advance(a, b, lpr);
            const int a3 = a, b3 = b;
            tri_advance(a, b, lpr);
            const CT x0 = TC_TRI(c0 + a0, c0 + b0), x1 = TC_TRI(c0 + a1, c0 + b1),
                     x2 = TC_TRI(c0 + a2, c0 + b2), x3 = TC_TRI(c0 + a3, c0 + b3);
            const CT r0 = TC_TRI(c0 + a0, j), r1 = TC_TRI(c0 + a1, j), r2 = TC_TRI(c0 + a2, j),
                     r3 = TC_TRI(c0 + a3, j);
            const CT k0 = TC_TRI(c0 + b0, j), k1 = TC_TRI(c0 + b1, j), k2 = TC_TRI(c0 + b2, j),
                     k3 = TC_TRI(c0 + b3, j);
            TC_TRI(c0 + a0, c0 + b0) = x0 - r0 * k0;
            TC_TRI(c0 + a1, c0 + b1) = x1 - r1 * k1;
            TC_TRI(c0 + a2, c0 + b2) = x2 - r2 * k2;
            TC_TRI(c0 + a3, c0 + b3) = x3 - r3 * k3;
        }
        for (; t < ntr; t += lpr) {
            TC_TRI(c0 + a, c0 + b) -= TC_TRI(c0 + a, j) * TC_TRI(c0 + b, j);
            tri_advance(a, b, lpr);
        }
        __syncwarp();
    }
    if (!inv_mode) {
        for (int r = sub; r < R; r += lpr) TC_VEC(r) = mine ? (CT)P.rhs[i * (int64_t)R + r] : CT(0);
        __syncwarp();
        for (int j = 0; j < R; ++j) {        // L y = b, by columns
            const CT yj = TC_VEC(j) * TC_DINV(j);
            __syncwarp();
            if (sub == 0) TC_VEC(j) = yj;
            for (int r = j + 1 + sub; r < R; r += lpr) TC_VEC(r) -= TC_TRI(r, j) * yj;
            __syncwarp();
        }
        for (int j = R - 1; j >= 0; --j) {   // L^T x = y, by rows of L
            const CT xj = TC_VEC(j) * TC_DINV(j);
            __syncwarp();
            if (sub == 0) TC_VEC(j) = xj;
            for (int r = sub; r < j; r += lpr) TC_VEC(r) -= TC_TRI(j, r) * xj;
            __syncwarp();
        }
        if (mine && ok)
            for (int r = sub; r < R; r += lpr) P.out[i * (int64_t)R + r] = (T)TC_VEC(r);
    } else {
        // L^-1, column c by the lane sub == the snake order of c (columns of
        // decreasing length dealt 0, 1, .., lpr-1, lpr-1, .., 0, ...): for r > c,
        // L^-1[r][c] = -(sum_{k=c}^{r-1} L[r][k] L^-1[k][c]) / L[r][r]; two
        // partial sums per dot product (the dots are short, and each extra
        // fold is one more FP64 warp instruction)
        for (int c = 0; c < R; ++c) {
            const int m = c % (2 * lpr);
            if ((m < lpr ? m : 2 * lpr - 1 - m) != sub) continue;
            TC_Y(c, c) = TC_DINV(c);
            for (int r = c + 1; r < R; ++r) {
                CT v0 = CT(0), v1 = CT(0);
                int k = c;
                for (; k + 1 < r; k += 2) {
                    v0 += TC_TRI(r, k) * TC_Y(k, c);
                    v1 += TC_TRI(r, k + 1) * TC_Y(k + 1, c);
                }
                if (k < r) v0 += TC_TRI(r, k) * TC_Y(k, c);
                TC_Y(r, c) = -(v0 + v1) * TC_DINV(r);
            }
        }
        __syncwarp();
        // (L L^T)^-1 [r][c] = sum_{k >= r} L^-1[k][r] L^-1[k][c], c <= r; the
        // packed entries dealt round-robin
        if (mine && ok) {
            T *Po = P.pinv + i * (int64_t)R * R;
            int r = 0, c = 0;
            tri_advance(r, c, sub);
            for (int t = sub; t < tri; t += lpr) {
                CT v0 = CT(0), v1 = CT(0);
                int k = r;
                for (; k + 1 < R; k += 2) {
                    v0 += TC_Y(k, r) * TC_Y(k, c);
                    v1 += TC_Y(k + 1, r) * TC_Y(k + 1, c);
                }
                if (k < R) v0 += TC_Y(k, r) * TC_Y(k, c);
                const CT v = v0 + v1;
                Po[r * R + c] = (T)v;
                Po[c * R + r] = (T)v;
                tri_advance(r, c, lpr);
            }
        }
    }
    if (mine) {
        if (!ok) {
            if (sub == 0) {
                record_error(P.status, TC_ERR_NOT_SPD);
                if (P.row_status) P.row_status[i] = 1;
                TC_TRI(0, 0) = CT(0);
            }
            if (P.pinv) {  // an identity block keeps the preconditioner defined
                T *Po = P.pinv + i * (int64_t)R * R;
                for (int q = sub; q < R * R; q += lpr) Po[q] = (q / R == q % R) ? T(1) : T(0);
            }
        } else if (sub == 0 && P.row_status) {
            P.row_status[i] = 0;
        }
    }
#undef TC_TRI
#undef TC_Y
#undef TC_VEC
#undef TC_DINV
    if (P.refine) {   // the factors, back over the Gram rows (coalesced per row)
        __syncwarp();
        for (int s = 0; s < nr; ++s) {
            T *lrow = B.light + (q0 + s) * (int64_t)tri;
            for (int e = lane; e < tri; e += 32) lrow[e] = (T)Tri[e * ps + s];
        }
    }
}

// ------------------------------------------------------------------ kernel B, R > 32
// One warp per row (grid-stride), FP64 packed triangle in shared memory.  The
// trailing update of step j touches the packed triangle of rows and columns
// j+1 .. R-1; its entries are dealt to the lanes in packed order through a
// decode table (rr, kk) shared by the block, so every lane does the same work.
constexpr int kCholWarps = 4;

template <typename T, typename CT>
__global__ void __launch_bounds__(kCholWarps * 32) chol_warp_kernel(const SolveParams<T> P,
                                                                    const Batch<T> B) {
    extern __shared__ __align__(16) unsigned char sh_raw[];
    CT *sh = reinterpret_cast<CT *>(sh_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int R = P.R, tri = R * (R + 1) / 2;
    const bool inv_mode = P.pinv != nullptr;
    const int per_warp = tri * (inv_mode ? 2 : 1) + 2 * R;
    uint32_t *tab = reinterpret_cast<uint32_t *>(sh + (size_t)kCholWarps * per_warp);
    for (int e = threadIdx.x; e < tri; e += blockDim.x) {
        int r, c;
        tri_rc(e, r, c);
        tab[e] = ((uint32_t)r << 16) | (uint32_t)c;
    }
    __syncthreads();
    CT *S = sh + (size_t)w * per_warp;
    CT *Y = S + tri;                         // L^-1 (inverse mode)
    CT *bv = S + tri * (inv_mode ? 2 : 1);
    CT *Dinv = bv + R;
    const int64_t nb = __ldg(P.row_ptr + B.row0);
    for (int64_t q = (int64_t)blockIdx.x * kCholWarps + w; q < B.nrows;
         q += (int64_t)gridDim.x * kCholWarps) {
        const int64_t i = B.row0 + q;
        const T *lrow;
        const double *crow;
        gram_source(P, B, nb, i, tri, lrow, crow);
        for (int e = lane; e < tri; e += 32) S[e] = gram_entry(lrow, crow, e);
        __syncwarp();
        for (int r = lane; r < R; r += 32) S[tri_idx(r, r)] += (CT)P.lambda;
        __syncwarp();
        bool ok = true;
        for (int j = 0; j < R; ++j) {
            const CT dj = S[tri_idx(j, j)];
            if (!(dj > CT(0))) {       // same value in every lane: a uniform exit
                ok = false;
                break;
            }
            const CT inv = rsqrt_nr(dj), ljj = dj * inv;
            __syncwarp();
            for (int r = j + 1 + lane; r < R; r += 32) S[tri_idx(r, j)] *= inv;
            if (lane == 0) {
                S[tri_idx(j, j)] = ljj;
                Dinv[j] = inv;
            }
            __syncwarp();
            const int nr = R - 1 - j, ntr = nr * (nr + 1) / 2;
            for (int e = lane; e < ntr; e += 32) {
                const uint32_t rc = tab[e];
                const int r = j + 1 + (int)(rc >> 16), k = j + 1 + (int)(rc & 0xffffu);
                S[tri_idx(r, k)] -= S[tri_idx(r, j)] * S[tri_idx(k, j)];
            }
            __syncwarp();
        }
        T *lout = B.light + q * (int64_t)tri;   // the factor, for the correction step
        if (!ok) {
            if (lane == 0) {
                record_error(P.status, TC_ERR_NOT_SPD);
                if (P.row_status) P.row_status[i] = 1;
                if (P.refine) lout[0] = T(0);
            }
            if (inv_mode) {
                T *Po = P.pinv + i * (int64_t)R * R;
                for (int e = lane; e < R * R; e += 32) Po[e] = (e / R == e % R) ? T(1) : T(0);
            }
            __syncwarp();
            continue;
        }
        if (lane == 0 && P.row_status) P.row_status[i] = 0;
        if (!inv_mode) {
            if (P.refine)
                for (int e = lane; e < tri; e += 32) lout[e] = (T)S[e];
            for (int r = lane; r < R; r += 32) bv[r] = (CT)P.rhs[i * (int64_t)R + r];
            __syncwarp();
            for (int j = 0; j < R; ++j) {        // L y = b
                const CT yj = bv[j] * Dinv[j];
                __syncwarp();
                for (int r = j + 1 + lane; r < R; r += 32) bv[r] -= S[tri_idx(r, j)] * yj;
                if (lane == 0) bv[j] = yj;
                __syncwarp();
            }
            for (int j = R - 1; j >= 0; --j) {   // L^T x = y
                const CT xj = bv[j] * Dinv[j];
                __syncwarp();
                for (int r = lane; r < j; r += 32) bv[r] -= S[tri_idx(j, r)] * xj;
                if (lane == 0) bv[j] = xj;
                __syncwarp();
            }
            for (int r = lane; r < R; r += 32) P.out[i * (int64_t)R + r] = (T)bv[r];
            __syncwarp();
            continue;
        }
        // L^-1 into Y, one column per lane (columns c and R - 1 - c pair up
        // a long and a short column): for r > c,
        // L^-1[r][c] = -(sum_{k=c}^{r-1} L[r][k] L^-1[k][c]) / L[r][r]
        for (int pass = 0; pass < 2; ++pass) {
            const int c = pass == 0 ? lane : R - 1 - lane;
            if (c < 0 || c >= R || (pass == 1 && c < 32)) continue;
            Y[tri_idx(c, c)] = Dinv[c];
            for (int r = c + 1; r < R; ++r) {
                CT v = CT(0);
                for (int k = c; k < r; ++k) v += S[tri_idx(r, k)] * Y[tri_idx(k, c)];
                Y[tri_idx(r, c)] = -v * Dinv[r];
            }
        }
        __syncwarp();
        // (L L^T)^-1 [r][c] = sum_{k >= r} L^-1[k][r] L^-1[k][c], c <= r
        T *Po = P.pinv + i * (int64_t)R * R;
        for (int e = lane; e < tri; e += 32) {
            const uint32_t rc = tab[e];
            const int r = (int)(rc >> 16), c = (int)(rc & 0xffffu);
            CT v = CT(0);
            for (int k = r; k < R; ++k) v += Y[tri_idx(k, r)] * Y[tri_idx(k, c)];
            Po[r * R + c] = (T)v;
            Po[c * R + r] = (T)v;
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ refinement (kernels C, D)
// One step of iterative refinement of the solved rows a_i (in `out`):
//   res_i = rhs_i - lambda a_i - sum_{e in row i} s_e h_e (h_e^T a_i),
//   a_i  += (L_i L_i^T)^-1 res_i,
// with L_i the row's Cholesky factor.  Kernel C accumulates the sum over the
// nonzeros with the same chunked traversal as the Gram (a warp per chunk,
// FP64 atomics into a zeroed buffer), in FP64 arithmetic for FP64 data and in
// double-float arithmetic for FP32 data: h_e = b (.) e split exactly into two
// FP32 words by a fused multiply-add, products and sums carried as FP32 pairs
// by error-free transforms (Dekker's product, Knuth's TwoSum), about 48
// significant bits at FP32 speed -- FP64 runs at about one operation per
// clock per SM on this GPU.  Kernel D forms res_i and applies
// the correction with the stored factor, one warp per row.
template <typename T, int RT, bool VEC>
__global__ void __launch_bounds__(128) refine_resid_kernel(const SolveParams<T> P, const Batch<T> B,
                                                           int64_t ch) {
    using L = Lay<T, RT, 32>;
    constexpr int V = L::V, G = L::G, NG = L::NG;
    const int lane = threadIdx.x & 31;
    const int g = lane / G, lg = lane % G;
    const int R = VEC ? RT : P.R;
    const int64_t nb = __ldg(P.row_ptr + B.row0), ne = __ldg(P.row_ptr + B.row0 + B.nrows);
    const int64_t last = B.row0 + B.nrows - 1;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t cs = nb + wid * ch; cs < ne; cs += nwarps * ch) {
        const int64_t ce = min(cs + ch, ne);
        int64_t i = search_le(P.row_ptr, B.row0, last, cs);
        for (;;) {
            const int64_t rs = __ldg(P.row_ptr + i), re = __ldg(P.row_ptr + i + 1);
            const int64_t ss = max(rs, cs), se = min(re, ce);
            T a32[V];
            load_slice<T, V, false>(a32, P.out, i, R, lg);
            if constexpr (sizeof(T) == 4) {
                // double-float (pairs of FP32 words, error-free transforms):
                // h = b e exactly as (hh, hl); z = <h, a> and the sums
                // s z h accumulated as (hi, lo) pairs, about 48 significant bits
                float ah[V], al[V];
#pragma unroll
                for (int t = 0; t < V; ++t) ah[t] = al[t] = 0.f;
                for (int64_t base = ss; base < se; base += NG) {
                    const bool valid = base + g < se;
                    const int64_t qq = valid ? base + g : se - 1;
                    T b[V], e[V];
                    load_slice<T, V, VEC>(b, P.A1, __ldcs(P.c1 + qq), R, lg);
                    load_slice<T, V, VEC>(e, P.A2, __ldcs(P.c2 + qq), R, lg);
                    float hh[V], hl[V], zh = 0.f, zl = 0.f;
#pragma unroll
                    for (int t = 0; t < V; ++t) {
                        // __fmul_rn: products that enter TwoSum must not be
                        // contracted into a fused multiply-add
                        hh[t] = __fmul_rn(b[t], e[t]);
                        hl[t] = fmaf(b[t], e[t], -hh[t]);
                        const float pr = __fmul_rn(hh[t], a32[t]);
                        const float pe = fmaf(hh[t], a32[t], -pr) + hl[t] * a32[t];
                        float sm, er;
                        two_sum(zh, pr, sm, er);
                        zh = sm;
                        zl += er + pe;
                    }
#pragma unroll
                    for (int o = G / 2; o > 0; o >>= 1) {
                        const float h2 = __shfl_xor_sync(0xffffffffu, zh, o);
                        const float l2 = __shfl_xor_sync(0xffffffffu, zl, o);
                        float sm, er;
                        two_sum(zh, h2, sm, er);
                        zh = sm;
                        zl += er + l2;
                    }
                    const float sw = valid ? (float)weight_at(P.w, qq) : 0.f;
                    const float ch = __fmul_rn(sw, zh);
                    const float cl = fmaf(sw, zh, -ch) + sw * zl;
#pragma unroll
                    for (int t = 0; t < V; ++t) {
                        const float pr = __fmul_rn(ch, hh[t]);
                        const float pe = fmaf(ch, hh[t], -pr) + (ch * hl[t] + cl * hh[t]);
                        float sm, er;
                        two_sum(ah[t], pr, sm, er);
                        ah[t] = sm;
                        al[t] += er + pe;
                    }
                }
                // sum the nonzero groups (lanes with equal lg)
#pragma unroll
                for (int t = 0; t < V; ++t) {
#pragma unroll
                    for (int o = G; o < 32; o <<= 1) {
                        const float h2 = __shfl_xor_sync(0xffffffffu, ah[t], o);
                        const float l2 = __shfl_xor_sync(0xffffffffu, al[t], o);
                        float sm, er;
                        two_sum(ah[t], h2, sm, er);
                        ah[t] = sm;
                        al[t] += er + l2;
                    }
                }
                if (g == 0) {
                    double *dst = B.res + (i - B.row0) * (int64_t)R + lg * V;
#pragma unroll
                    for (int t = 0; t < V; ++t)
                        if (lg * V + t < R) atomicAdd(dst + t, -((double)ah[t] + (double)al[t]));
                }
            } else {
                double av[V], acc[V];
#pragma unroll
                for (int t = 0; t < V; ++t) {
                    av[t] = (double)a32[t];
                    acc[t] = 0.0;
                }
                for (int64_t base = ss; base < se; base += NG) {
                    const bool valid = base + g < se;
                    const int64_t qq = valid ? base + g : se - 1;
                    T b[V], e[V];
                    load_slice<T, V, VEC>(b, P.A1, __ldcs(P.c1 + qq), R, lg);
                    load_slice<T, V, VEC>(e, P.A2, __ldcs(P.c2 + qq), R, lg);
                    double h[V], part = 0.0;
#pragma unroll
                    for (int t = 0; t < V; ++t) {
                        h[t] = (double)b[t] * (double)e[t];
                        part += h[t] * av[t];
                    }
                    const double z = group_sum<G>(part);
                    const double coef = valid ? (double)weight_at(P.w, qq) * z : 0.0;
#pragma unroll
                    for (int t = 0; t < V; ++t) acc[t] += coef * h[t];
                }
#pragma unroll
                for (int t = 0; t < V; ++t) acc[t] = across_groups<G>(acc[t]);
                if (g == 0) {
                    double *dst = B.res + (i - B.row0) * (int64_t)R + lg * V;
#pragma unroll
                    for (int t = 0; t < V; ++t)
                        if (lg * V + t < R) atomicAdd(dst + t, -acc[t]);
                }
            }
            if (re >= ce) break;
            i = search_le_near(P.row_ptr, i + 1, last, re);   // next nonempty row
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kCholWarps * 32) refine_correct_kernel(const SolveParams<T> P,
                                                                         const Batch<T> B) {
    __shared__ T rv[kCholWarps][TC_MAX_RANK];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int R = P.R, tri = R * (R + 1) / 2;
    T *v = rv[w];
    for (int64_t q = (int64_t)blockIdx.x * kCholWarps + w; q < B.nrows;
         q += (int64_t)gridDim.x * kCholWarps) {
        const int64_t i = B.row0 + q;
        const T *Lq = B.light + q * (int64_t)tri;
        if (!((double)Lq[0] > 0.0)) continue;   // the row did not factor (uniform)
        for (int r = lane; r < R; r += 32) {
            const double a = (double)P.out[i * (int64_t)R + r];
            v[r] = (T)((double)P.rhs[i * (int64_t)R + r] - P.lambda * a +
                       B.res[q * (int64_t)R + r]);
        }
        __syncwarp();
        for (int j = 0; j < R; ++j) {          // L y = res
            const T yj = v[j] / Lq[tri_idx(j, j)];
            __syncwarp();
            for (int r = j + 1 + lane; r < R; r += 32) v[r] -= Lq[tri_idx(r, j)] * yj;
            if (lane == 0) v[j] = yj;
            __syncwarp();
        }
        for (int j = R - 1; j >= 0; --j) {     // L^T d = y
            const T dj = v[j] / Lq[tri_idx(j, j)];
            __syncwarp();
            for (int r = lane; r < j; r += 32) v[r] -= Lq[tri_idx(j, r)] * dj;
            if (lane == 0) v[j] = dj;
            __syncwarp();
        }
        for (int r = lane; r < R; r += 32) {
            T *o = P.out + i * (int64_t)R + r;
            *o = (T)((double)*o + (double)v[r]);
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ host side
// SM count per device, queried once (host threads may race to fill an entry;
// they store the same value, and the atomics make that well defined)
static int device_sms() {
    static std::atomic<int> sms[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int v = sms[dev].load(std::memory_order_relaxed);
    if (!v) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
            v = 152;
        sms[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

// Process-wide tuning per dtype and rank tier (0 = automatic), read and
// written under g_tuning_mu; a call copies the setting it uses once.
static tc_solve_tuning g_tuning[2][4];
static std::mutex g_tuning_mu;

static int tier_slot(int tier) { return tier <= 8 ? 0 : tier <= 16 ? 1 : tier <= 32 ? 2 : 3; }

// Nonzeros per chunk: about eight chunks per resident block, a power of two
// in [256, 16384], unless tuned.
static int64_t chunk_nnz(int64_t m, int64_t grid, const tc_solve_tuning &t) {
    if (t.chunk_nnz > 0) return t.chunk_nnz;
    int64_t want = m / (8 * grid);
    int64_t ch = 256;
    while (ch < want && ch < 16384) ch <<= 1;
    return ch;
}

// Kernel A variant for (dtype, rank tier, form): warp-local kernels (one warp
// per chunk) for FP64 ranks <= 16 and tensor-core ranks <= 32, the block
// kernel otherwise.
// WARP_MMA = true takes the block kernel where the tcgen05 kernel would run.
template <typename T, int RT, bool VEC, int KIND, bool WARP_MMA = false>
struct GramLaunch {
    static constexpr bool HAS_TC05 =
        sizeof(T) == 4 && RT == 64 && VEC && (KIND == GK_TF32 || KIND == GK_BF16);
    static constexpr int VAR = (sizeof(T) == 8 && RT <= 16) ? 1
                               : (sizeof(T) == 4 && RT <= 32 && KIND != GK_FFMA) ? 2
                               : (HAS_TC05 && !WARP_MMA) ? 3
                                                         : 0;
    static constexpr bool PER_WARP = VAR == 1 || VAR == 2;
    // forms an ALS right-hand side (RHS_VALUES) in its own pass; and the
    // gradient's (RHS_DPHI, with phi'' weights), which solve_fuses_rhs says
    // on the host
    static constexpr bool FUSES_RHS = VAR != 1;
    static constexpr bool FUSES_DPHI = VAR == 2 && KIND == GK_TF32X3;
    static int threads() {
        if constexpr (VAR == 1) return WarpGram<T, RT>::NTH;
        else if constexpr (VAR == 2) return WarpMma<RT, KIND>::NTH;
        else if constexpr (VAR == 3) return tc05::THREADS;
        else return GramGeo<T, RT, KIND>::NTH;
    }
    static size_t smem() {
        if constexpr (VAR == 1) return WarpGram<T, RT>::smem;
        else if constexpr (VAR == 2) return WarpMma<RT, KIND>::smem;
        else if constexpr (VAR == 3) return tc05::Geo<KIND>::SMEM;
        else return GramGeo<T, RT, KIND>::smem;
    }
    static const void *fn(int rk = RHS_GIVEN) {
        if constexpr (VAR == 1) return (const void *)gram_warp_kernel<T, RT, VEC>;
        else if constexpr (VAR == 2) {
            if (rk == RHS_VALUES) return (const void *)gram_warp_mma_kernel<RT, VEC, KIND, RHS_VALUES>;
            if constexpr (KIND == GK_TF32X3)
                if (rk == RHS_DPHI) return (const void *)gram_warp_mma_kernel<RT, VEC, KIND, RHS_DPHI>;
            return (const void *)gram_warp_mma_kernel<RT, VEC, KIND>;
        }
        else if constexpr (VAR == 3) return (const void *)gram_tc05_kernel<KIND>;
        else return (const void *)gram_chunk_kernel<T, RT, VEC, KIND>;
    }
    // resident blocks per SM (queried once)
    // (per right-hand-side kind: the warp-level kernel's variants differ in
    // registers; host threads may race to fill an entry with the same value)
    static tc_status occupancy(int &occ, int rk = RHS_GIVEN) {
        static std::atomic<int> cached[3];
        const int slot = rk >= 0 && rk < 3 ? rk : 0;
        int have = cached[slot].load(std::memory_order_relaxed);
        if (!have) {
            const void *f = fn(rk);
            if (smem() > 48 * 1024) {
                TC_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem()));
                // the whole unified L1 / shared array as shared memory, so that
                // several blocks of this size fit per SM (the occupancy query
                // below assumes the carveout set here)
                TC_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                             (int)cudaSharedmemCarveoutMaxShared));
            }
            int v = 0;
            TC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, f, threads(), smem()));
            if constexpr (VAR == 3) {
                // the tcgen05 kernel: the query answers 1 block per SM (measured);
                // shared memory (with 1 KB reserved per block), at most 128
                // registers per thread and 128 of the 512 TMEM columns per block
                // allow more
                int by_smem = (int)((228 * 1024) / (smem() + 1024 + 64));
                const int by_tmem = 512 / (int)tc05::TMEM_COLS;
                if (by_smem > by_tmem) by_smem = by_tmem;
                if (by_smem > v) v = by_smem;
            }
            have = v > 0 ? v : 1;
            cached[slot].store(have, std::memory_order_relaxed);
        }
        occ = have;
        return TC_OK;
    }
    static void launch(int64_t grid, const SolveParams<T> &P, const Batch<T> &Bt, cudaStream_t st) {
        if constexpr (VAR == 1)
            gram_warp_kernel<T, RT, VEC><<<(unsigned)grid, threads(), smem(), st>>>(P, Bt);
        else if constexpr (VAR == 2) {
            if (P.rhs_kind == RHS_VALUES)
                gram_warp_mma_kernel<RT, VEC, KIND, RHS_VALUES><<<(unsigned)grid, threads(), smem(), st>>>(P, Bt);
            else if constexpr (KIND == GK_TF32X3) {
                if (P.rhs_kind == RHS_DPHI)
                    gram_warp_mma_kernel<RT, VEC, KIND, RHS_DPHI><<<(unsigned)grid, threads(), smem(), st>>>(P, Bt);
                else
                    gram_warp_mma_kernel<RT, VEC, KIND><<<(unsigned)grid, threads(), smem(), st>>>(P, Bt);
            } else {
                gram_warp_mma_kernel<RT, VEC, KIND><<<(unsigned)grid, threads(), smem(), st>>>(P, Bt);
            }
        }
        else if constexpr (VAR == 3)
            gram_tc05_kernel<KIND><<<(unsigned)grid, threads(), smem(), st>>>(P, Bt);
        else
            gram_chunk_kernel<T, RT, VEC, KIND><<<(unsigned)grid, threads(), smem(), st>>>(P, Bt);
    }
};

template <typename T, int RT, bool VEC, int KIND, bool CHOL32, bool WARP_MMA>
static tc_status launch_solve_gl(const SolveParams<T> &P0, int64_t m, const tc_solve_tuning &tun,
                                 const tc_pattern *pat, int mode, const void *const *A,
                                 cudaStream_t st) {
    using GL = GramLaunch<T, RT, VEC, KIND, WARP_MMA>;
    SolveParams<T> P = P0;
    if (P.rhs_kind == RHS_VALUES && !GL::FUSES_RHS) {
        // a Gram kernel that does not form the right-hand side: the MTTKRP of
        // the values first, then an ordinary solve on it
        const tc_status rc = launch_mttkrp(pat, TC_W_VALUES, nullptr, P.R, A, mode, P.rhs_w, 0, st);
        if (rc != TC_OK) return rc;
        P.rhs_kind = RHS_GIVEN;
    }
    if (P.rhs_kind == RHS_DPHI && !GL::FUSES_DPHI) return TC_ERR_UNSUPPORTED;   // see solve_fuses_rhs
    using CT = typename std::conditional<CHOL32, float, double>::type;   // factorization type
    const int R = P.R, tri = R * (R + 1) / 2;
    const int sms = device_sms();
    int occ = 1;
    {
        const tc_status rc = GL::occupancy(occ, P.rhs_kind);
        if (rc != TC_OK) return rc;
    }
    const int64_t grid_a = (int64_t)sms * occ;
    const int64_t ch = chunk_nnz(m, GL::PER_WARP ? grid_a * (GL::threads() / 32) : grid_a, tun);
    const int64_t ch_c = ch / 4 > 64 ? ch / 4 : 64;    // refinement: a warp per chunk

    const bool warp_b = RT > 32;
    // rows per warp of the R <= 32 factorization (32 / rpw lanes per row):
    // 16 for R <= 16, 4 for R = 32.  Each row's FP64 triangle takes
    // R(R+1)/2 * 8 bytes of shared memory (twice that in inverse mode), so at
    // R = 32 fewer rows per one-warp block fit more blocks per SM: measured on
    // GB300, 4.70 / 5.28 / 7.75 ms at 4 / 8 / 16 for a 5e4-row mode; at R = 16
    // 0.361 / 0.338 / 0.356 / 0.408 ms at 4 / 8 / 16 / 32 for a 1e4-row mode,
    // where larger modes favour fewer lanes per row (each warp computes its
    // rows' pivots once whatever its lanes per row)
    int rpw = RT <= 16 ? 16 : 4;
    if (tun.chol_rows_per_warp > 0) rpw = tun.chol_rows_per_warp < 32 ? tun.chol_rows_per_warp : 32;
    if (RT > 16 && rpw > 16) rpw = 16;
    const int align = warp_b ? kCholWarps : rpw;
    size_t smem_b;
    if (warp_b)
        smem_b = sizeof(CT) * (size_t)kCholWarps * (tri * (P.pinv ? 2 : 1) + 2 * R) +
                 sizeof(uint32_t) * tri;
    else
        smem_b = sizeof(CT) * (size_t)(tri * (P.pinv ? 2 : 1) + 2 * R) * (rpw + 1);
    if (warp_b) {
        auto kb = chol_warp_kernel<T, CT>;
        TC_CUDA(cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
    } else if (smem_b > 48 * 1024) {
        auto kb = chol_rows_kernel<T, CT>;
        TC_CUDA(cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b));
    }

    // rows per batch: Gram triangles of at most 1 GiB (or as tuned)
    const int64_t budget = tun.batch_bytes > 0 ? tun.batch_bytes : ((int64_t)1 << 30);
    int64_t batch = budget / ((int64_t)tri * (int64_t)sizeof(T));
    batch = batch / align * align;
    if (batch < align) batch = align;
    if (batch > P.I) batch = P.I;
    const int64_t slots = (m + ch - 1) / ch + 1;
    // the Gram batch, the cut-row slots and the residuals live in the
    // pattern's work space for this mode (allocated once per size)
    T *light = (T *)work_buffer(pat, WS_SOLVE_GRAM + mode, sizeof(T) * (size_t)tri * batch);
    double *cut = (double *)work_buffer(pat, WS_SOLVE_CUT + mode, sizeof(double) * (size_t)tri * slots);
    double *res = nullptr;
    if (P.refine) res = (double *)work_buffer(pat, WS_SOLVE_RES + mode, sizeof(double) * (size_t)R * batch);
    double *cut_rhs = nullptr;
    if (P.rhs_kind != RHS_GIVEN)
        cut_rhs = (double *)work_buffer(pat, WS_SOLVE_CUT_RHS + mode, sizeof(double) * (size_t)R * slots);
    if (!light || !cut || (P.refine && !res) || (P.rhs_kind != RHS_GIVEN && !cut_rhs)) return TC_ERR_OOM;
    const int64_t nblk_w0 = (int64_t)sms * 16;
    for (int64_t row0 = 0; row0 < P.I; row0 += batch) {
        Batch<T> Bt{row0, min(batch, P.I - row0), ch, light, cut, res, cut_rhs};
        int64_t zb = (slots * (tri + (cut_rhs ? R : 0)) + 255) / 256;
        if (zb > (int64_t)sms * 4) zb = (int64_t)sms * 4;
        if (zb < 1) zb = 1;
        zero_cut_kernel<T><<<(unsigned)zb, 256, 0, st>>>(P.row_ptr, Bt, tri, R);
        if (P.rhs_kind != RHS_GIVEN)   // empty rows keep a zero right-hand side
            TC_CUDA(cudaMemsetAsync(P.rhs_w + row0 * (int64_t)R, 0,
                                    sizeof(T) * (size_t)Bt.nrows * R, st));
        GL::launch(grid_a, P, Bt, st);
        if (P.rhs_kind != RHS_GIVEN) {
            int64_t fb = (slots * R + 255) / 256;
            if (fb > (int64_t)sms * 4) fb = (int64_t)sms * 4;
            if (fb < 1) fb = 1;
            cut_rhs_kernel<T><<<(unsigned)fb, 256, 0, st>>>(P.row_ptr, Bt, R, P.rhs_w);
            count_launch();
        }
        int64_t nblk_w = (Bt.nrows + kCholWarps - 1) / kCholWarps;
        if (nblk_w > nblk_w0) nblk_w = nblk_w0;
        if (warp_b)
            chol_warp_kernel<T, CT><<<(unsigned)nblk_w, kCholWarps * 32, smem_b, st>>>(P, Bt);
        else
            chol_rows_kernel<T, CT><<<(unsigned)((Bt.nrows + rpw - 1) / rpw), 32, smem_b, st>>>(P, Bt, rpw);
        count_launch(3);
        for (int step = 0; step < P.refine; ++step) {
            TC_CUDA(cudaMemsetAsync(res, 0, sizeof(double) * (size_t)R * Bt.nrows, st));
            refine_resid_kernel<T, RT, VEC><<<(unsigned)(sms * 8), 128, 0, st>>>(P, Bt, ch_c);
            refine_correct_kernel<T><<<(unsigned)nblk_w, kCholWarps * 32, 0, st>>>(P, Bt);
            count_launch(2);
        }
    }
    return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}

// The Gram engine: the tuned choice where both exist.
template <typename T, int RT, bool VEC, int KIND, bool CHOL32>
static tc_status launch_solve_rt(const SolveParams<T> &P, int64_t m, const tc_solve_tuning &tun,
                                 const tc_pattern *pat, int mode, const void *const *A,
                                 cudaStream_t st) {
    if constexpr (GramLaunch<T, RT, VEC, KIND>::HAS_TC05) {
        if (tun.gram_kernel == TC_GRAM_WARP_MMA)
            return launch_solve_gl<T, RT, VEC, KIND, CHOL32, true>(P, m, tun, pat, mode, A, st);
    }
    return launch_solve_gl<T, RT, VEC, KIND, CHOL32, false>(P, m, tun, pat, mode, A, st);
}

template <typename T, int KIND, bool C32>
static tc_status dispatch_rt(const SolveParams<T> &P, int tier, bool vec, int64_t m,
                             const tc_solve_tuning &tun, const tc_pattern *pat, int mode,
                             const void *const *A, cudaStream_t st) {
#define TC_SOLVE_RT(RT)                                                                     \
    return vec ? launch_solve_rt<T, RT, true, KIND, C32>(P, m, tun, pat, mode, A, st)       \
               : launch_solve_rt<T, RT, false, KIND, C32>(P, m, tun, pat, mode, A, st)
    switch (tier) {
        case 8: TC_SOLVE_RT(8);
        case 16: TC_SOLVE_RT(16);
        case 32: TC_SOLVE_RT(32);
        default: TC_SOLVE_RT(64);
    }
#undef TC_SOLVE_RT
}

template <typename T>
static tc_status solve_t(const tc_pattern *p, tc_weights w, const void *s, int R,
                         const void *const *A, int mode, const void *rhs, double lambda,
                         tc_prec prec, void *out, int8_t *row_status, int use_d2, tc_loss loss,
                         void *pinv, cudaStream_t st, const tc_solve_tuning &tun,
                         int rhs_kind = RHS_GIVEN, void *rhs_out = nullptr,
                         double *loss_acc = nullptr) {
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
    const tc_prec form = (tc_prec)(prec & ~(TC_PREC_CHOL32 | TC_PREC_REFINE2));
    P.refine = (!pinv && form != TC_PREC_FP32) ? ((prec & TC_PREC_REFINE2) ? 2 : 1) : 0;
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
    if (P.I == 0) return TC_OK;
    const int tier = rank_tier(R);
    const bool vec = vec_ok(R, tier, sizeof(T)) && aligned16({A[o1], A[o2]}) &&
                     (!use_d2 || aligned16({A[mode]}));
    const int64_t m = p->nnz;
    if (sizeof(T) == 8 && (form == TC_PREC_TF32_REFINE || form == TC_PREC_BF16_REFINE))
        return TC_ERR_UNSUPPORTED;
    if (rhs_kind != RHS_GIVEN) {
        // the right-hand side is formed here: into the pattern's work space
        // (an ALS update) or into the caller's buffer (a gradient)
        P.rhs_w = rhs_kind == RHS_DPHI
                      ? (T *)rhs_out
                      : (T *)work_buffer(p, WS_SOLVE_RHS + mode, sizeof(T) * (size_t)P.I * R);
        if (!P.rhs_w) return TC_ERR_OOM;
        P.rhs = P.rhs_w;
        P.rhs_kind = rhs_kind;
        P.loss_acc = loss_acc;
    } else if (P.refine && (const void *)P.out == (const void *)P.rhs) {
        // the correction step reads rhs after the solve wrote out: keep a
        // copy when they alias
        const size_t bytes = sizeof(T) * (size_t)P.I * R;
        T *rhs_copy = (T *)work_buffer(p, WS_SOLVE_RHS + mode, bytes);
        if (!rhs_copy) return TC_ERR_OOM;
        TC_CUDA(cudaMemcpyAsync(rhs_copy, P.rhs, bytes, cudaMemcpyDeviceToDevice, st));
        P.rhs = rhs_copy;
    }
    tc_status rc = TC_OK;
    const bool c32 = (prec & TC_PREC_CHOL32) != 0 && P.refine;
#define TC_SOLVE_KIND(K)                                                          \
    (c32 ? dispatch_rt<T, K, true>(P, tier, vec, m, tun, p, mode, A, st)          \
         : dispatch_rt<T, K, false>(P, tier, vec, m, tun, p, mode, A, st))
    if constexpr (sizeof(T) == 4) {
        if (form == TC_PREC_TF32_REFINE) rc = TC_SOLVE_KIND(GK_TF32);
        else if (form == TC_PREC_BF16_REFINE) rc = TC_SOLVE_KIND(GK_BF16);
        else rc = TC_SOLVE_KIND(GK_TF32X3);
    } else {
        rc = TC_SOLVE_KIND(GK_FFMA);
    }
#undef TC_SOLVE_KIND
    return rc;
}

}  // namespace tc

namespace tc {
tc_solve_tuning solve_tuning(tc_dtype dtype, int R) {
    std::lock_guard<std::mutex> lock(g_tuning_mu);
    return g_tuning[dtype == TC_F64 ? 1 : 0][tier_slot(rank_tier(R))];
}
}  // namespace tc

extern "C" tc_status tc_set_solve_tuning(tc_dtype dtype, int R, const tc_solve_tuning *t) {
    if ((dtype != TC_F32 && dtype != TC_F64) || R < 0 || R > TC_MAX_RANK) return TC_ERR_ARG;
    if (t && (t->chunk_nnz < 0 || t->chunk_nnz > ((int64_t)1 << 30) || t->batch_bytes < 0))
        return TC_ERR_ARG;
    if (t && t->chol_rows_per_warp != 0) {
        const int v = t->chol_rows_per_warp;
        if (v < 1 || v > 32 || (v & (v - 1))) return TC_ERR_ARG;
    }
    if (t && (t->gram_kernel < TC_GRAM_AUTO || t->gram_kernel > TC_GRAM_TCGEN05)) return TC_ERR_ARG;
    const tc_solve_tuning v = t ? *t : tc_solve_tuning{0, 0, 0, 0};
    std::lock_guard<std::mutex> lock(tc::g_tuning_mu);
    for (int k = 0; k < 4; ++k)
        if (R == 0 || tc::tier_slot(tc::rank_tier(R)) == k) tc::g_tuning[dtype][k] = v;
    return TC_OK;
}

extern "C" tc_status tc_get_solve_tuning(tc_dtype dtype, int R, tc_solve_tuning *t) {
    if ((dtype != TC_F32 && dtype != TC_F64) || R < 1 || R > TC_MAX_RANK || !t) return TC_ERR_ARG;
    *t = tc::solve_tuning(dtype, R);
    return TC_OK;
}

// Candidate tunings for the rank tier: chunk sizes around the automatic
// choice, the factorization's rows per warp where it applies, and the Gram
// engine where two exist.
extern "C" tc_status tc_autotune_solve(const tc_pattern *p, tc_weights w, const void *s, int R,
                                       const void *const *factors, int mode, const void *rhs,
                                       double lambda, tc_prec prec, void *out,
                                       tc_solve_tuning *best, float *ms_out, tc_stream_t stream) {
    if (!p || R < 1 || R > TC_MAX_RANK || !factors || !rhs || !out || mode < 0 || mode >= p->order)
        return TC_ERR_ARG;
    const int dt = p->dtype == TC_F64 ? 1 : 0;
    const int tier = tc::rank_tier(R), slot = tc::tier_slot(tier);
    // every candidate is passed to the solve explicitly: the process-wide
    // setting, which other threads' solves read, only changes to the winner
    const tc_solve_tuning saved = tc::solve_tuning(p->dtype, R);
    const int64_t chunks[] = {0, 256, 1024, 4096, 16384};
    int rpws[3] = {0, 0, 0};
    int nr = 1;
    if (tier <= 16) { rpws[0] = 8; rpws[1] = 16; rpws[2] = 32; nr = 3; }
    else if (tier <= 32) { rpws[0] = 4; rpws[1] = 8; rpws[2] = 16; nr = 3; }
    const tc_prec form = (tc_prec)(prec & ~(TC_PREC_CHOL32 | TC_PREC_REFINE2));
    int engines[2] = {TC_GRAM_AUTO, TC_GRAM_AUTO};
    int ne = 1;
    if (p->dtype == TC_F32 && R == 64 && (form == TC_PREC_TF32_REFINE || form == TC_PREC_BF16_REFINE)) {
        engines[0] = TC_GRAM_TCGEN05;
        engines[1] = TC_GRAM_WARP_MMA;
        ne = 2;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return TC_ERR_CUDA;
    }
    tc_solve_tuning win = saved;
    float win_ms = -1.f;
    tc_status rc = TC_OK;
    for (int64_t ch : chunks) {
        for (int k = 0; k < nr * ne && rc == TC_OK; ++k) {
            const tc_solve_tuning cand{ch, saved.batch_bytes, rpws[k % nr], engines[k / nr]};
            // one untimed call (caches, work space), then one timed
            rc = tc::launch_solve_factor(p, w, s, R, factors, mode, rhs, lambda, prec, out, nullptr,
                                         0, TC_LOSS_LS, nullptr, st, &cand);
            if (rc != TC_OK) break;
            if (cudaEventRecord(e0, st) != cudaSuccess) { rc = TC_ERR_CUDA; break; }
            rc = tc::launch_solve_factor(p, w, s, R, factors, mode, rhs, lambda, prec, out, nullptr,
                                         0, TC_LOSS_LS, nullptr, st, &cand);
            if (rc != TC_OK) break;
            float ms = 0.f;
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = TC_ERR_CUDA;
                break;
            }
            if (win_ms < 0.f || ms < win_ms) {
                win_ms = ms;
                win = cand;
            }
        }
        if (rc != TC_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != TC_OK) return rc;
    {
        std::lock_guard<std::mutex> lock(tc::g_tuning_mu);
        tc::g_tuning[dt][slot] = win;
    }
    if (best) *best = win;
    if (ms_out) *ms_out = win_ms;
    return TC_OK;
}

namespace tc {

tc_status launch_solve_factor(const tc_pattern *p, tc_weights w, const void *s, int R,
                              const void *const *A, int mode, const void *rhs, double lambda,
                              tc_prec prec, void *out, int8_t *row_status, int use_loss_d2,
                              tc_loss loss, void *pinv_out, cudaStream_t st,
                              const tc_solve_tuning *tun) {
    const tc_solve_tuning t = tun ? *tun : solve_tuning(p->dtype, R);
    if (p->dtype == TC_F64)
        return solve_t<double>(p, w, s, R, A, mode, rhs, lambda, prec, out, row_status,
                               use_loss_d2, loss, pinv_out, st, t);
    return solve_t<float>(p, w, s, R, A, mode, rhs, lambda, prec, out, row_status, use_loss_d2,
                          loss, pinv_out, st, t);
}

tc_status launch_als_update(const tc_pattern *p, int R, const void *const *A, int mode,
                            double lambda, tc_prec prec, void *out, int8_t *row_status,
                            cudaStream_t st) {
    const tc_solve_tuning t = solve_tuning(p->dtype, R);
    if (p->dtype == TC_F64)
        return solve_t<double>(p, TC_W_ONE, nullptr, R, A, mode, nullptr, lambda, prec, out,
                               row_status, 0, TC_LOSS_LS, nullptr, st, t, RHS_VALUES);
    return solve_t<float>(p, TC_W_ONE, nullptr, R, A, mode, nullptr, lambda, prec, out,
                          row_status, 0, TC_LOSS_LS, nullptr, st, t, RHS_VALUES);
}

bool solve_fuses_rhs(tc_dtype dtype, int R) {
    // GramLaunch<float, RT <= 32, *, FP32-class or tensor-core form>::FUSES_DPHI
    return dtype == TC_F32 && rank_tier(R) <= 32;
}

tc_status launch_precond_grad(const tc_pattern *p, int R, const void *const *A, int mode,
                              double lambda2, tc_loss loss, void *pinv_out, void *grad_out,
                              double *loss_acc, cudaStream_t st) {
    if (!solve_fuses_rhs(p->dtype, R)) return TC_ERR_UNSUPPORTED;
    const tc_solve_tuning t = solve_tuning(p->dtype, R);
    return solve_t<float>(p, TC_W_ONE, nullptr, R, A, mode, nullptr, lambda2, TC_PREC_FP32,
                          nullptr, nullptr, 1, loss, pinv_out, st, t, RHS_DPHI, grad_out, loss_acc);
}

}  // namespace tc
