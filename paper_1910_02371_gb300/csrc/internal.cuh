// Internal declarations and device helpers of libtc (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <initializer_list>

#include "../../include/tc.h"

#define TC_ORDER 3
#define TC_MAX_RANK 64

// ------------------------------------------------------------------ host side
struct ModeData {
    int64_t *row_ptr = nullptr;   // I_d + 1
    int64_t *perm = nullptr;      // nnz: sorted position -> input position
    int64_t *to0 = nullptr;       // nnz: mode-d position -> mode-0 position (d > 0)
    int32_t *nz_rows = nullptr;   // nonempty rows, ascending (capacity I_d)
    int64_t *nz_ptr = nullptr;    // offsets of the nonempty rows (capacity I_d + 1)
    int64_t *n_ne_dev = nullptr;  // device: number of nonempty rows
    int32_t *cols[TC_ORDER - 1] = {nullptr, nullptr};  // other modes, ascending mode order
    void *vals = nullptr;         // nnz values in this mode's order (or null)
};

// Work space of the builder, kept when the pattern may be refilled.
struct PatternScratch {
    int32_t *kbuf = nullptr, *ktmp = nullptr, *dk = nullptr, *c1tmp = nullptr, *c2tmp = nullptr;
    int64_t *vtmp = nullptr, *inv0 = nullptr, *hist = nullptr, *scan = nullptr, *flags = nullptr,
            *dp = nullptr;
    void *valtmp = nullptr;
};

// Work space of the calls that need more device memory than their outputs
// (Solve Factor's Gram batch, cut-row slots, refinement residuals, right-hand
// side copy or the right-hand side an ALS update forms, and its cut-row
// slots, per mode; the general-loss Newton and coordinate-descent buffers).  The pattern keeps
// each buffer and grows it on demand (tc::work_buffer), so a call at a size
// the pattern has served before allocates nothing.
enum WorkSlot {
    WS_SOLVE_GRAM = 0,                  // + mode
    WS_SOLVE_CUT = WS_SOLVE_GRAM + 3,   // + mode
    WS_SOLVE_RES = WS_SOLVE_CUT + 3,    // + mode
    WS_SOLVE_RHS = WS_SOLVE_RES + 3,    // + mode
    WS_SOLVE_CUT_RHS = WS_SOLVE_RHS + 3,  // + mode
    WS_NEWTON = WS_SOLVE_CUT_RHS + 3,
    WS_NEWTON_SUMS,
    WS_CCD,
    WS_CCD_SUMS,
    WS_COUNT
};

struct WorkBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct tc_pattern {
    unsigned flags = 0;
    int order = 0;
    int64_t dims[TC_ORDER] = {0, 0, 0};
    int64_t nnz = 0;
    tc_dtype dtype = TC_F32;
    int has_vals = 0;
    int device = 0;
    ModeData md[TC_ORDER];
    int *status = nullptr;        // device word: first error recorded, 0 if none
    int64_t *counts = nullptr;    // device: nonempty rows per mode
    int to0_valid = 0;            // md[d].to0 built (on first use) for the current contents
    PatternScratch work;
    WorkBuf ws[WS_COUNT];
};

namespace tc {

extern int64_t g_launches;
inline void count_launch(int n = 1) { g_launches += n; }

inline size_t tsize(tc_dtype t) { return t == TC_F64 ? 8 : 4; }

// Other modes of `mode`, ascending.
inline void other_modes(int mode, int &o1, int &o2) {
    o1 = mode == 0 ? 1 : 0;
    o2 = mode == 2 ? 1 : 2;
}

// Padded rank tier: the compile-time row width a kernel is instantiated for.
inline int rank_tier(int R) {
    if (R <= 8) return 8;
    if (R <= 16) return 16;
    if (R <= 32) return 32;
    return 64;
}

// Rows may use 32-byte vector loads when the row stride is a multiple of 32
// bytes and the rank fills the tier.
constexpr int kVecBytes = 32;
inline bool vec_ok(int R, int tier, size_t es) { return R == tier && (R * es) % kVecBytes == 0; }

// Every non-null pointer aligned for the vector loads (a caller may pass an
// offset view).
inline bool aligned16(std::initializer_list<const void *> ptrs) {
    for (const void *q : ptrs)
        if (q && (reinterpret_cast<uintptr_t>(q) & (kVecBytes - 1))) return false;
    return true;
}

#define TC_CUDA(call)                                      \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return TC_ERR_CUDA;         \
    } while (0)

// Device-side weights description.
template <typename T>
struct Weights {
    int kind;            // TC_W_ONE / TC_W_VALUES / TC_W_ARRAY
    const T *s;          // values or array in this traversal's order (mode 0 / VALUES)
    const int64_t *to0;  // for TC_W_ARRAY in a mode d > 0: index into s (pattern order)
};

// ---------------------------------------------------------------- kernel launchers
// (defined in the .cu files; each returns TC_OK or an error)
tc_status launch_tttp(const tc_pattern *p, tc_weights w, const void *s, int R,
                      const void *const *A, void *x, cudaStream_t st);
tc_status launch_mttkrp(const tc_pattern *p, tc_weights w, const void *s, int R,
                        const void *const *A, int mode, void *out, int accumulate,
                        cudaStream_t st);
tc_status launch_loss_grad(const tc_pattern *p, tc_loss loss, int R, const void *const *A,
                           double lambda, double *loss_out, void *const *grads, cudaStream_t st);
// init: first set y = 2 lambda x (and add its share to *dot_out); otherwise y
// already holds it.  full_newton: also the phi' term of the full Hessian.
tc_status launch_ggn_matvec(const tc_pattern *p, tc_loss loss, int R, const void *const *A,
                            const void *const *x, double lambda, void *const *y,
                            double *dot_out, int init, int full_newton, cudaStream_t st);
// The same on interleaved factor / direction buffers AX[n] (I_n x 2R: per lane
// chunk of 16 bytes, the factor chunk then the direction chunk); needs the
// vector path (vec_ok).
// Queries (and caches) the launch geometry of the interleaved product's
// kernels; call outside any stream capture, before the first
// launch_ggn_matvec_ax.
tc_status prepare_ggn_matvec_ax();
tc_status launch_ggn_matvec_ax(const tc_pattern *p, tc_loss loss, int R, const void *const *AX,
                               double lambda, void *const *y, double *dot_out, int init,
                               int full_newton, cudaStream_t st);
// Gram + FP64 Cholesky per row.  If pinv_out != null the inverse of each row
// system, (G_i + lambda I)^-1, is formed in FP64 from the factor and stored
// (pattern dtype, I_d x R x R) instead of solving.
// tun: the tuning to use (nullptr: the process-wide one, solve_tuning).
tc_status launch_solve_factor(const tc_pattern *p, tc_weights w, const void *s, int R,
                              const void *const *A, int mode, const void *rhs, double lambda,
                              tc_prec prec, void *out, int8_t *row_status, int use_loss_d2,
                              tc_loss loss, void *pinv_out, cudaStream_t st,
                              const tc_solve_tuning *tun = nullptr);
// One ALS update of factor `mode`: Solve Factor with unit weights and the
// right-hand side rhs_i = sum_e t_e h_e (the MTTKRP of the values) formed in
// the Gram pass where the Gram kernel supports it, else by the MTTKRP kernel
// first; the right-hand side lives in the pattern's work space.
tc_status launch_als_update(const tc_pattern *p, int R, const void *const *A, int mode,
                            double lambda, tc_prec prec, void *out, int8_t *row_status,
                            cudaStream_t st);
// True where the Gram kernel forms a right-hand side in its own pass (FP32
// data, R <= 32).
bool solve_fuses_rhs(tc_dtype dtype, int R);
// The preconditioner block of `mode` (launch_solve_factor with phi'' weights,
// inverse into pinv_out) whose Gram pass also writes the gradient's
// MTTKRP(phi', mode) into grad_out (I_mode x R, overwritten) and, if loss_acc
// is not null, adds sum_e phi(t_e, m_e) to it; TC_ERR_UNSUPPORTED unless
// solve_fuses_rhs.
tc_status launch_precond_grad(const tc_pattern *p, int R, const void *const *A, int mode,
                              double lambda2, tc_loss loss, void *pinv_out, void *grad_out,
                              double *loss_acc, cudaStream_t st);
// acc += lambda * sum_n ||A^(n)||_F^2 (the regularizer of eq. obj).
tc_status launch_regularizer(const tc_pattern *p, int R, const void *const *A, double lambda,
                             double *acc, cudaStream_t st);
tc_status build_pattern_impl(int order, const int64_t *dims, int64_t nnz,
                             const int32_t *const *idx, const void *vals, tc_dtype dtype,
                             unsigned flags, cudaStream_t st, tc_pattern **out);
tc_status refill_pattern_impl(tc_pattern *p, const int32_t *const *idx, const void *vals,
                              cudaStream_t st);
// Builds the mode-d -> mode-0 position maps (for caller weight arrays in
// pattern order) if the current contents do not have them yet.
tc_status ensure_to0(const tc_pattern *p, cudaStream_t st);

// Newton-step helpers (newton.cu), float and double:
//   loss_derivs: d1 = phi'(t, m), d2 = phi''(t, m) over n entries (domain
//                errors recorded in status);
//   newton_rhs:  rhs = -(g + two_lambda A);
//   newton_update: A += step, sums[0] += ||step||^2, sums[1] += ||A||^2 (FP64).
template <typename T>
void launch_loss_derivs(int64_t n, int loss, const T *t, const T *m, T *d1, T *d2, int *status,
                        cudaStream_t st);
template <typename T>
void launch_newton_rhs(int64_t n, const T *g, const T *A, double two_lambda, T *rhs,
                       cudaStream_t st);
template <typename T>
void launch_newton_update(int64_t n, T *A, const T *step, double *sums, cudaStream_t st);
void free_pattern(tc_pattern *p);

// A device buffer of at least `bytes` bytes held by the pattern in slot `id`.
// A slot that is too small is replaced (after synchronizing the device, since
// work in flight may still use it); returns nullptr if the allocation fails.
// Calls on one pattern that use the same slot must be ordered (one stream, or
// events): the slot is shared.
void *work_buffer(const tc_pattern *p, int id, size_t bytes);

// The Solve Factor tuning in force for (dtype, rank tier): a copy of the
// process-wide setting, read under a lock.
tc_solve_tuning solve_tuning(tc_dtype dtype, int R);

}  // namespace tc

// ------------------------------------------------------------------ device side
#ifdef __CUDACC__
namespace tc {

// Lane layout of one row of a factor: V consecutive elements per lane (one
// VB-byte vector, 16 or 32 bytes), G lanes per nonzero, NG nonzeros per warp
// step.  Kernels pick VB by measurement: 32-byte lanes halve the instructions
// per row but raise register use.
template <typename T, int RT, int VB = 16>
struct Lay {
    static constexpr int V = VB / (int)sizeof(T);
    static constexpr int G = RT / V;
    static constexpr int NG = 32 / G;
};

__device__ __forceinline__ void record_error(int *status, int code) {
    atomicCAS(status, 0, code);
}

// The vector loads carry the .L2::64B fetch-size hint: a factor row is
// gathered at a random row index, so the L2 should bring in the 64 bytes that
// are asked for and not the whole 128-byte line (with factors larger than L2,
// measured at 2^22 rows: MTTKRP reads 156 instead of 253 DRAM bytes per
// nonzero, 1-2% faster; the sweeps stay bound by the rate of random fetches).
template <typename T, int V, bool VEC>
__device__ __forceinline__ void load_slice(T (&v)[V], const T *__restrict__ A, int64_t row, int R,
                                           int lg) {
    const T *ptr = A + row * (int64_t)R + lg * V;
    if constexpr (VEC && V * sizeof(T) == 32) {
        if constexpr (sizeof(T) == 4) {
            asm("ld.global.nc.L2::64B.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]),
                  "=f"(v[6]), "=f"(v[7])
                : "l"(ptr));
        } else {
            asm("ld.global.nc.L2::64B.v4.f64 {%0,%1,%2,%3}, [%4];"
                : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
                : "l"(ptr));
        }
    } else if constexpr (VEC) {
        static_assert(V * sizeof(T) == 16, "16- or 32-byte vectors");
        if constexpr (sizeof(T) == 4) {
            asm("ld.global.nc.L2::64B.v4.f32 {%0,%1,%2,%3}, [%4];"
                : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                : "l"(ptr));
        } else {
            asm("ld.global.nc.L2::64B.v2.f64 {%0,%1}, [%2];" : "=d"(v[0]), "=d"(v[1]) : "l"(ptr));
        }
    } else {
#pragma unroll
        for (int t = 0; t < V; ++t) v[t] = (lg * V + t < R) ? __ldg(ptr + t) : T(0);
    }
}

template <typename T, int V, bool VEC>
__device__ __forceinline__ void store_slice(T *__restrict__ A, int64_t row, int R, int lg,
                                            const T (&v)[V]) {
    T *ptr = A + row * (int64_t)R + lg * V;
    if constexpr (VEC && V * sizeof(T) == 32) {
        if constexpr (sizeof(T) == 4) {
            asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(ptr), "f"(v[0]),
                         "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                         : "memory");
        } else {
            asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(ptr), "d"(v[0]), "d"(v[1]),
                         "d"(v[2]), "d"(v[3])
                         : "memory");
        }
    } else if constexpr (VEC) {
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float4 *>(ptr) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
            *reinterpret_cast<double2 *>(ptr) = make_double2(v[0], v[1]);
        }
    } else {
#pragma unroll
        for (int t = 0; t < V; ++t)
            if (lg * V + t < R) ptr[t] = v[t];
    }
}

template <typename T, int V>
__device__ __forceinline__ void atomic_add_slice(T *__restrict__ A, int64_t row, int R, int lg,
                                                 const T (&v)[V]) {
    T *ptr = A + row * (int64_t)R + lg * V;
#pragma unroll
    for (int t = 0; t < V; ++t)
        if (lg * V + t < R) atomicAdd(ptr + t, v[t]);
}

// Sum over the G lanes of one nonzero group (G is a power of two, groups are
// aligned on G lanes).
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Adds v summed over the block to *dst with one atomic; every thread of the
// block must call it (blockDim.x a multiple of 32, at most 1024).
__device__ __forceinline__ void block_add(double v, double *dst) {
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0 && v != 0.0) atomicAdd(dst, v);
    }
    __syncthreads();
}

// Largest index q in [lo, hi] with a[q] <= key (a ascending, a[lo] <= key).
__device__ __forceinline__ int64_t search_le(const int64_t *__restrict__ a, int64_t lo, int64_t hi,
                                             int64_t key) {
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (__ldg(a + mid) <= key) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The same when the answer is usually at or just after lo (the next nonempty
// row after a finished one): an exponential probe from lo, then the binary
// search inside the last interval -- one load when the next row is nonempty,
// instead of a dependent load per halving of [lo, hi].
__device__ __forceinline__ int64_t search_le_near(const int64_t *__restrict__ a, int64_t lo,
                                                  int64_t hi, int64_t key) {
    int64_t b = lo, d = 1;
    while (b + d <= hi && __ldg(a + b + d) <= key) {
        b += d;
        d <<= 1;
    }
    return search_le(a, b, min(b + d - 1, hi), key);
}

// The same with 32-bit positions in the array (row counts fit in int32).
__device__ __forceinline__ int search_le32(const int64_t *__restrict__ a, int lo, int hi,
                                          int64_t key) {
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(a + mid) <= key) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Sum of v over the NG groups of a warp (lanes with equal lane % G), every
// lane receiving the total of its own slice.
template <int G, typename T>
__device__ __forceinline__ T across_groups(T v) {
#pragma unroll
    for (int o = G; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Weight s_e of the nonzero at sorted position q of the current traversal.
template <typename T>
__device__ __forceinline__ T weight_at(const Weights<T> &w, int64_t q) {
    if (w.kind == TC_W_ONE) return T(1);
    if (w.to0) return __ldg(w.s + __ldg(w.to0 + q));
    return __ldcs(w.s + q);
}

// phi, phi' and phi'' of eq. obj / Table 1 at model entry m and value t.
template <typename T>
__device__ __forceinline__ void loss_terms(int loss, T t, T m, T &phi, T &d1, T &d2, bool &dom_ok) {
    if (loss == TC_LOSS_LS) {
        T r = t - m;
        phi = r * r;
        d1 = T(2) * (m - t);
        d2 = T(2);
    } else if (loss == TC_LOSS_POISSON_LOG) {
        T ex = exp(m);
        phi = ex - t * m;
        d1 = ex - t;
        d2 = ex;
    } else {
        if (!(m > T(0))) {
            dom_ok = false;
            phi = d1 = d2 = T(0);
            return;
        }
        phi = m - t * log(m);
        d1 = T(1) - t / m;
        d2 = t / (m * m);
    }
}

}  // namespace tc
#endif
