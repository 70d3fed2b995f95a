// Pattern builder (Sec. 3.4: the nonzeros are sorted by the mode index with a
// counting sort so that each row's nonzeros are contiguous; Sec. 3.1: only the
// nonempty rows are listed, as in the doubly compressed formats).
//
// The sort is a stable least-significant-digit radix sort with 8-bit digits
// over the mode index, carrying the input position, so equal indices keep
// input order and the result is unique (bit-exact against any stable sort).
// Each pass: per-tile digit histograms, one device-wide exclusive scan in
// digit-major order, then a scatter in which every warp ranks its elements
// with __match_any_sync in input order.  No atomics decide any position.
#include "internal.cuh"

#include <algorithm>
#include <new>
#include <type_traits>

namespace tc {

constexpr int kRadixBits = 8;
constexpr int kDigits = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kItems = 16;                       // per lane
constexpr int kTile = kSortThreads * kItems;     // 4096 elements

// ------------------------------------------------------------------ scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void scan_reduce_kernel(const int64_t *__restrict__ in, int64_t n,
                                   int64_t *__restrict__ sums) {
    __shared__ int64_t red[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t q = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (q < n) s += in[q];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
        sums[blockIdx.x] = t;
    }
}

// out = exclusive scan of in over this block's tile, offset by offs[block].
__global__ void scan_tile_kernel(const int64_t *__restrict__ in, int64_t n,
                                 const int64_t *__restrict__ offs, int64_t *__restrict__ out) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t q = base + k;
        v[k] = q < n ? in[q] : 0;
        s += v[k];
    }
    // inclusive scan of thread sums across the block
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[w] = inc;
    __syncthreads();
    int64_t woff = 0;
    for (int k = 0; k < w; ++k) woff += warp_tot[k];
    int64_t run = (offs ? offs[blockIdx.x] : 0) + woff + inc - s;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t q = base + k;
        if (q < n) out[q] = run;
        run += v[k];
    }
}

// Scratch (int64 elements) needed to scan n values: one block sum per tile
// per recursion level.
static int64_t scan_scratch_elems(int64_t n) {
    int64_t total = 0;
    while (n > kScanTile) {
        n = (n + kScanTile - 1) / kScanTile;
        total += n;
    }
    return total;
}

// Exclusive scan of n int64 values (in may equal out); block sums live in
// `scratch` (scan_scratch_elems(n) elements).  Allocates nothing.
static void scan_exclusive(const int64_t *in, int64_t *out, int64_t n, int64_t *scratch,
                           cudaStream_t st) {
    if (n <= 0) return;
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        scan_tile_kernel<<<1, kScanThreads, 0, st>>>(in, n, nullptr, out);
        count_launch();
        return;
    }
    int64_t *sums = scratch;
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, sums);
    count_launch();
    scan_exclusive(sums, sums, nb, scratch + nb, st);
    scan_tile_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, sums, out);
    count_launch();
}

// ------------------------------------------------------------------ radix sort
__global__ void radix_hist_kernel(const int32_t *__restrict__ keys, int64_t n, int shift,
                                  int64_t num_tiles, int64_t *__restrict__ hist) {
    __shared__ int h[kDigits];
    for (int d = threadIdx.x; d < kDigits; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTile;
    for (int k = 0; k < kItems; ++k) {
        const int64_t q = base + (int64_t)k * kSortThreads + threadIdx.x;
        if (q < n) atomicAdd(&h[(keys[q] >> shift) & (kDigits - 1)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kDigits; d += blockDim.x)
        hist[(int64_t)d * num_tiles + blockIdx.x] = h[d];
}

// Stable scatter: warp w of a tile owns elements [w*32*kItems, (w+1)*32*kItems)
// of the tile in input order and ranks them round by round.
__global__ void __launch_bounds__(kSortThreads)
radix_scatter_kernel(const int32_t *__restrict__ kin, const int64_t *__restrict__ vin, int64_t n,
                     int shift, int64_t num_tiles, const int64_t *__restrict__ offs,
                     int32_t *__restrict__ kout, int64_t *__restrict__ vout) {
    __shared__ int wcnt[kSortWarps][kDigits];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < kDigits; d += 32) wcnt[w][d] = 0;
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)w * 32 * kItems;
    const unsigned lt_mask = (1u << lane) - 1u;
    int32_t key[kItems];
    int64_t val[kItems];
    int pos[kItems];
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int64_t q = base + (int64_t)r * 32 + lane;
        const bool valid = q < n;
        key[r] = valid ? kin[q] : 0;
        val[r] = valid ? (vin ? vin[q] : q) : 0;
        const int dig = valid ? ((key[r] >> shift) & (kDigits - 1)) : kDigits;
        const unsigned peers = __match_any_sync(0xffffffffu, dig);
        const int rank = __popc(peers & lt_mask);
        const int cnt0 = valid ? wcnt[w][dig] : 0;
        pos[r] = cnt0 + rank;
        __syncwarp();
        if (valid && rank == 0) wcnt[w][dig] = cnt0 + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over the warps of each digit
    for (int d = threadIdx.x; d < kDigits; d += kSortThreads) {
        int s = 0;
        for (int k = 0; k < kSortWarps; ++k) {
            const int c = wcnt[k][d];
            wcnt[k][d] = s;
            s += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItems; ++r) {
        const int64_t q = base + (int64_t)r * 32 + lane;
        if (q < n) {
            const int dig = (key[r] >> shift) & (kDigits - 1);
            const int64_t dst = offs[(int64_t)dig * num_tiles + blockIdx.x] + wcnt[w][dig] + pos[r];
            kout[dst] = key[r];
            vout[dst] = val[r];
        }
    }
}

__global__ void iota_copy_kernel(const int32_t *__restrict__ kin, const int64_t *__restrict__ vin,
                                 int64_t n, int32_t *__restrict__ kout, int64_t *__restrict__ vout) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        kout[q] = kin[q];
        vout[q] = vin ? vin[q] : q;
    }
}

static unsigned grid_for(int64_t n, int threads, int64_t cap = 1 << 20) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

static int64_t sort_tiles(int64_t n) { return (n + kTile - 1) / kTile; }

// Stable sort of (key, value) pairs by key in [0, max_key]; vals_in == null
// means value = input position.  Results in kout / vout; ktmp / vtmp, hist
// (kDigits * sort_tiles(n)) and scan scratch are work space.  Allocates nothing.
static void radix_sort(const int32_t *keys_in, const int64_t *vals_in, int64_t n, int64_t max_key,
                       int32_t *kout, int64_t *vout, int32_t *ktmp, int64_t *vtmp, int64_t *hist,
                       int64_t *scan_scratch, cudaStream_t st) {
    int bits = 0;
    while (bits < 31 && (max_key >> bits) > 0) ++bits;
    const int passes = (bits + kRadixBits - 1) / kRadixBits;
    if (n == 0) return;
    if (passes == 0) {
        iota_copy_kernel<<<grid_for(n, 256), 256, 0, st>>>(keys_in, vals_in, n, kout, vout);
        count_launch();
        return;
    }
    const int64_t num_tiles = sort_tiles(n);
    const int32_t *ks = keys_in;
    const int64_t *vs = vals_in;
    for (int p = 0; p < passes; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        int32_t *kd = to_out ? kout : ktmp;
        int64_t *vd = to_out ? vout : vtmp;
        const int shift = p * kRadixBits;
        radix_hist_kernel<<<(unsigned)num_tiles, kSortThreads, 0, st>>>(ks, n, shift, num_tiles, hist);
        count_launch();
        scan_exclusive(hist, hist, kDigits * num_tiles, scan_scratch, st);
        radix_scatter_kernel<<<(unsigned)num_tiles, kSortThreads, 0, st>>>(ks, vs, n, shift, num_tiles,
                                                                          hist, kd, vd);
        count_launch();
        ks = kd;
        vs = vd;
    }
}

// ------------------------------------------------------------------ payload sort
// The pattern builder's sort carries, with each key, the input position, the
// other two modes' indices and the value, so one pass writes the final sorted
// copies (no random gathers afterwards).  Each tile of kTileP elements is
// ranked as above, staged in shared memory in its sorted order, and written
// out digit run by digit run, so consecutive threads write consecutive
// addresses.
constexpr int kTileP = 2048;
constexpr int kItemsP = kTileP / kSortThreads;
static_assert(kDigits == kSortThreads, "one thread per digit in the tile scan");

struct SortSide {
    int32_t *key;
    int64_t *perm;   // null on the first pass: the input position; a null
                     // destination perm drops the positions (lean patterns)
    int32_t *c1, *c2;
    void *val;
};

__global__ void radix_hist_p_kernel(const int32_t *__restrict__ keys, int64_t n, int shift,
                                    int64_t num_tiles, int64_t *__restrict__ hist) {
    __shared__ int h[kDigits];
    for (int d = threadIdx.x; d < kDigits; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kTileP;
    for (int k = 0; k < kItemsP; ++k) {
        const int64_t q = base + (int64_t)k * kSortThreads + threadIdx.x;
        if (q < n) atomicAdd(&h[(keys[q] >> shift) & (kDigits - 1)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kDigits; d += blockDim.x)
        hist[(int64_t)d * num_tiles + blockIdx.x] = h[d];
}

__device__ __forceinline__ int32_t clamp_index(int32_t v, int64_t I) {
    return v < 0 ? 0 : ((int64_t)v >= I ? (int32_t)(I - 1) : v);
}

// VB: value bytes (0, 4 or 8).  first: src.perm is the input position and the
// index payload is clamped into [0, I1) / [0, I2) (out-of-range indices are
// already recorded as TC_ERR_RANGE; clamping keeps later factor reads in bounds).
template <int VB>
__global__ void __launch_bounds__(kSortThreads)
radix_scatter_p_kernel(SortSide src, SortSide dst, int64_t n, int shift, int64_t num_tiles,
                       const int64_t *__restrict__ offs, int64_t I1, int64_t I2, int first) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int64_t *perm_s = reinterpret_cast<int64_t *>(smem_raw);
    int32_t *key_s = reinterpret_cast<int32_t *>(perm_s + kTileP);
    int32_t *c1_s = key_s + kTileP;
    int32_t *c2_s = c1_s + kTileP;
    unsigned char *val_s = reinterpret_cast<unsigned char *>(c2_s + kTileP);
    __shared__ int wcnt[kSortWarps][kDigits];
    __shared__ int toff[kDigits];
    __shared__ int64_t goff[kDigits];
    __shared__ int wsum[kSortWarps];
    using VT = typename std::conditional<VB == 8, double, float>::type;

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int d = lane; d < kDigits; d += 32) wcnt[w][d] = 0;
    __syncwarp();
    const int64_t tile0 = (int64_t)blockIdx.x * kTileP;
    const int64_t base = tile0 + (int64_t)w * 32 * kItemsP;
    const unsigned lt_mask = (1u << lane) - 1u;
    // only the keys and ranks stay in registers through the ranking; the
    // payload is read again (from L2) when the tile is staged, which keeps
    // the register count, and so the blocks per SM, up
    int32_t key[kItemsP];
    int pos[kItemsP];
#pragma unroll
    for (int r = 0; r < kItemsP; ++r) {
        const int64_t q = base + (int64_t)r * 32 + lane;
        const bool valid = q < n;
        key[r] = valid ? src.key[q] : 0;
        const int dig = valid ? ((key[r] >> shift) & (kDigits - 1)) : kDigits;
        const unsigned peers = __match_any_sync(0xffffffffu, dig);
        const int rank = __popc(peers & lt_mask);
        const int cnt0 = valid ? wcnt[w][dig] : 0;
        pos[r] = cnt0 + rank;
        __syncwarp();
        if (valid && rank == 0) wcnt[w][dig] = cnt0 + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {   // digit d = thread: prefix over the warps, the tile's digit offsets and the global ones
        const int d = threadIdx.x;
        int tot = 0;
        for (int k = 0; k < kSortWarps; ++k) {
            const int c = wcnt[k][d];
            wcnt[k][d] = tot;
            tot += c;
        }
        int inc = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        int wpre = 0;
        for (int k = 0; k < w; ++k) wpre += wsum[k];
        toff[d] = wpre + inc - tot;
        goff[d] = offs[(int64_t)d * num_tiles + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kItemsP; ++r) {
        const int64_t q = base + (int64_t)r * 32 + lane;
        if (q < n) {
            const int dig = (key[r] >> shift) & (kDigits - 1);
            const int l = toff[dig] + wcnt[w][dig] + pos[r];
            key_s[l] = key[r];
            if (first) {
                if (dst.perm) perm_s[l] = q;
                c1_s[l] = clamp_index(src.c1[q], I1);
                c2_s[l] = clamp_index(src.c2[q], I2);
            } else {
                if (dst.perm) perm_s[l] = src.perm[q];
                c1_s[l] = src.c1[q];
                c2_s[l] = src.c2[q];
            }
            if constexpr (VB > 0) reinterpret_cast<VT *>(val_s)[l] = reinterpret_cast<const VT *>(src.val)[q];
        }
    }
    __syncthreads();
    const int tile_n = (int)min((int64_t)kTileP, n - tile0);
    for (int j = threadIdx.x; j < tile_n; j += kSortThreads) {
        const int32_t k = key_s[j];
        const int dig = (k >> shift) & (kDigits - 1);
        const int64_t o = goff[dig] + (j - toff[dig]);
        dst.key[o] = k;
        if (dst.perm) dst.perm[o] = perm_s[j];
        dst.c1[o] = c1_s[j];
        dst.c2[o] = c2_s[j];
        if constexpr (VB > 0) reinterpret_cast<VT *>(dst.val)[o] = reinterpret_cast<const VT *>(val_s)[j];
    }
}

// A key range of one value (no sort needed): copy with the positions.
template <int VB>
__global__ void copy_p_kernel(SortSide src, SortSide dst, int64_t n, int64_t I1, int64_t I2) {
    using VT = typename std::conditional<VB == 8, double, float>::type;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        dst.key[q] = src.key[q];
        if (dst.perm) dst.perm[q] = q;
        dst.c1[q] = clamp_index(src.c1[q], I1);
        dst.c2[q] = clamp_index(src.c2[q], I2);
        if constexpr (VB > 0) reinterpret_cast<VT *>(dst.val)[q] = reinterpret_cast<const VT *>(src.val)[q];
    }
}

static int64_t sort_tiles_p(int64_t n) { return (n + kTileP - 1) / kTileP; }
static size_t scatter_p_smem(int vb) { return (size_t)kTileP * (8 + 4 + 4 + 4 + vb); }

// first_to_out: the first pass writes `out` (so `tmp` may alias `in`, whose
// contents are dead after that pass); with an even number of digit passes one
// more pass on the top digit, an identity on keys already sorted, brings the
// result back to `out`.
template <int VB>
static void radix_sort_p_t(const SortSide &in, const SortSide &out, const SortSide &tmp, int64_t n,
                           int64_t max_key, int64_t I1, int64_t I2, int64_t *hist, int64_t *scan,
                           bool first_to_out, cudaStream_t st) {
    int bits = 0;
    while (bits < 31 && (max_key >> bits) > 0) ++bits;
    const int digit_passes = (bits + kRadixBits - 1) / kRadixBits;
    const int passes = digit_passes + ((first_to_out && digit_passes % 2 == 0 && digit_passes > 0) ? 1 : 0);
    if (n == 0) return;
    if (passes == 0) {
        copy_p_kernel<VB><<<grid_for(n, 256), 256, 0, st>>>(in, out, n, I1, I2);
        count_launch();
        return;
    }
    const size_t smem = scatter_p_smem(VB);
    cudaFuncSetAttribute(radix_scatter_p_kernel<VB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    const int64_t num_tiles = sort_tiles_p(n);
    SortSide src = in;
    for (int p = 0; p < passes; ++p) {
        const SortSide &dst = ((passes - 1 - p) % 2 == 0) ? out : tmp;
        const int shift = (p < digit_passes ? p : digit_passes - 1) * kRadixBits;
        radix_hist_p_kernel<<<(unsigned)num_tiles, kSortThreads, 0, st>>>(src.key, n, shift, num_tiles,
                                                                         hist);
        count_launch();
        scan_exclusive(hist, hist, kDigits * num_tiles, scan, st);
        radix_scatter_p_kernel<VB><<<(unsigned)num_tiles, kSortThreads, smem, st>>>(
            src, dst, n, shift, num_tiles, hist, I1, I2, p == 0 ? 1 : 0);
        count_launch();
        src = dst;
    }
}

static void radix_sort_p(int vb, const SortSide &in, const SortSide &out, const SortSide &tmp,
                         int64_t n, int64_t max_key, int64_t I1, int64_t I2, int64_t *hist,
                         int64_t *scan, bool first_to_out, cudaStream_t st) {
    if (vb == 8) radix_sort_p_t<8>(in, out, tmp, n, max_key, I1, I2, hist, scan, first_to_out, st);
    else if (vb == 4) radix_sort_p_t<4>(in, out, tmp, n, max_key, I1, I2, hist, scan, first_to_out, st);
    else radix_sort_p_t<0>(in, out, tmp, n, max_key, I1, I2, hist, scan, first_to_out, st);
}

// ------------------------------------------------------------------ pattern kernels
__global__ void range_check_kernel(const int32_t *__restrict__ idx, int64_t n, int64_t I,
                                   int *status) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = idx[q];
        if (v < 0 || (int64_t)v >= I) {
            record_error(status, TC_ERR_RANGE);
            return;
        }
    }
}

// row_ptr from sorted keys: row r (0 <= r <= I) starts at the first position
// whose key is >= r, found by a binary search per row, so every row costs the
// same whatever the row lengths.  Keys outside [0, I) (already recorded as
// TC_ERR_RANGE) are clamped to [-1, I - 1]; the search result is then still
// nondecreasing in r and within [0, n], so no later kernel leaves its arrays.
__global__ void row_ptr_kernel(const int32_t *__restrict__ sk, int64_t n, int64_t I,
                               int64_t *__restrict__ row_ptr) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= I;
         r += (int64_t)gridDim.x * blockDim.x) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            const int64_t key = min(max((int64_t)__ldg(sk + mid), (int64_t)-1), I - 1);
            if (key < r) lo = mid + 1;
            else hi = mid;
        }
        row_ptr[r] = lo;
    }
}

__global__ void nonempty_flags_kernel(const int64_t *__restrict__ row_ptr, int64_t I,
                                      int64_t *__restrict__ flags) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < I;
         r += (int64_t)gridDim.x * blockDim.x)
        flags[r] = row_ptr[r + 1] > row_ptr[r] ? 1 : 0;
}

// Compacts the nonempty rows; the last row also writes their count.
__global__ void nonempty_fill_kernel(const int64_t *__restrict__ row_ptr, int64_t I,
                                     const int64_t *__restrict__ pos, int64_t n,
                                     int32_t *__restrict__ nz_rows, int64_t *__restrict__ nz_ptr,
                                     int64_t *__restrict__ n_ne) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < I;
         r += (int64_t)gridDim.x * blockDim.x) {
        const bool ne = row_ptr[r + 1] > row_ptr[r];
        if (ne) {
            nz_rows[pos[r]] = (int32_t)r;
            nz_ptr[pos[r]] = row_ptr[r];
        }
        if (r == I - 1) {
            const int64_t cnt = pos[r] + (ne ? 1 : 0);
            nz_ptr[cnt] = n;
            *n_ne = cnt;
        }
    }
}

// dst[q] = src[perm[q]], clamped to [0, I): an index outside the range is
// already recorded as TC_ERR_RANGE, and clamping keeps every later factor
// read of this pattern inside its matrix.
__global__ void gather_i32_kernel(const int32_t *__restrict__ src, const int64_t *__restrict__ perm,
                                  int64_t n, int64_t I, int32_t *__restrict__ dst) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = src[perm[q]];
        dst[q] = v < 0 ? 0 : ((int64_t)v >= I ? (int32_t)(I - 1) : v);
    }
}

template <typename T>
__global__ void gather_val_kernel(const T *__restrict__ src, const int64_t *__restrict__ perm,
                                  int64_t n, T *__restrict__ dst) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = src[perm[q]];
}

__global__ void invert_perm_kernel(const int64_t *__restrict__ perm, int64_t n,
                                   int64_t *__restrict__ inv) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        inv[perm[q]] = q;
}

__global__ void compose_kernel(const int64_t *__restrict__ inv0, const int64_t *__restrict__ perm,
                               int64_t n, int64_t *__restrict__ out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        out[q] = inv0[perm[q]];
}

// Adjacent equal coordinates in lexicographic order are duplicates.
__global__ void dup_check_kernel(const int32_t *__restrict__ i0, const int32_t *__restrict__ i1,
                                 const int32_t *__restrict__ i2, const int64_t *__restrict__ perm,
                                 int64_t n, int *status) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = perm[q - 1], b = perm[q];
        if (i0[a] == i0[b] && i1[a] == i1[b] && i2[a] == i2[b]) {
            record_error(status, TC_ERR_DUPLICATE);
            return;
        }
    }
}

// ------------------------------------------------------------------ builder
static void free_scratch(tc_pattern *p);

void free_pattern(tc_pattern *p) {
    if (!p) return;
    for (int d = 0; d < TC_ORDER; ++d) {
        ModeData &m = p->md[d];
        cudaFree(m.row_ptr);
        cudaFree(m.perm);
        cudaFree(m.to0);
        cudaFree(m.nz_rows);
        cudaFree(m.nz_ptr);
        cudaFree(m.cols[0]);
        cudaFree(m.cols[1]);
        cudaFree(m.vals);
    }
    free_scratch(p);
    for (int k = 0; k < WS_COUNT; ++k) cudaFree(p->ws[k].ptr);
    cudaFree(p->status);
    cudaFree(p->counts);
    delete p;
}

void *work_buffer(const tc_pattern *pc, int id, size_t bytes) {
    tc_pattern *p = const_cast<tc_pattern *>(pc);
    if (id < 0 || id >= WS_COUNT) return nullptr;
    WorkBuf &b = p->ws[id];
    if (bytes == 0) bytes = 16;
    if (b.ptr && b.bytes >= bytes) return b.ptr;
    if (b.ptr) {
        // work already queued may still read or write the old buffer
        if (cudaDeviceSynchronize() != cudaSuccess) return nullptr;
        cudaFree(b.ptr);
        b.ptr = nullptr;
        b.bytes = 0;
    }
    const size_t want = (bytes + 255) / 256 * 256;
    if (cudaMalloc(&b.ptr, want) != cudaSuccess) {
        cudaGetLastError();
        b.ptr = nullptr;
        return nullptr;
    }
    b.bytes = want;
    return b.ptr;
}

static bool dalloc(void **ptr, size_t bytes) {
    return cudaMalloc(ptr, bytes > 0 ? bytes : 16) == cudaSuccess;
}

static void free_scratch(tc_pattern *p) {
    PatternScratch &w = p->work;
    cudaFree(w.kbuf);
    cudaFree(w.ktmp);
    cudaFree(w.vtmp);
    cudaFree(w.inv0);
    cudaFree(w.hist);
    cudaFree(w.scan);
    cudaFree(w.flags);
    cudaFree(w.dk);
    cudaFree(w.dp);
    cudaFree(w.c1tmp);
    cudaFree(w.c2tmp);
    cudaFree(w.valtmp);
    w = PatternScratch();
}

static tc_status alloc_scratch(tc_pattern *p) {
    PatternScratch &w = p->work;
    const int64_t n = p->nnz;
    int64_t maxI = 0;
    for (int d = 0; d < TC_ORDER; ++d) maxI = p->dims[d] > maxI ? p->dims[d] : maxI;
    const int64_t hist_n = (int64_t)kDigits * std::max(sort_tiles(n), sort_tiles_p(n));
    int64_t scan_n = scan_scratch_elems(hist_n);
    const int64_t s2 = scan_scratch_elems(maxI);
    if (s2 > scan_n) scan_n = s2;
    if (p->flags & TC_PATTERN_LEAN) {
        // sorted keys and one key buffer; the payload's work space is borrowed
        // (fill_pattern) unless the input may not be overwritten
        const bool own_tmp = !(p->flags & TC_PATTERN_CONSUME_INPUT);
        const bool ok = dalloc((void **)&w.kbuf, sizeof(int32_t) * n) &&
                        dalloc((void **)&w.ktmp, sizeof(int32_t) * n) &&
                        dalloc((void **)&w.hist, sizeof(int64_t) * hist_n) &&
                        dalloc((void **)&w.scan, sizeof(int64_t) * (scan_n + 1)) &&
                        dalloc((void **)&w.flags, sizeof(int64_t) * maxI) &&
                        (!own_tmp || (dalloc((void **)&w.c1tmp, sizeof(int32_t) * n) &&
                                      dalloc((void **)&w.c2tmp, sizeof(int32_t) * n) &&
                                      (!p->has_vals || dalloc(&w.valtmp, tsize(p->dtype) * n))));
        return ok ? TC_OK : TC_ERR_OOM;
    }
    bool ok = dalloc((void **)&w.kbuf, sizeof(int32_t) * n) &&
              dalloc((void **)&w.ktmp, sizeof(int32_t) * n) &&
              dalloc((void **)&w.vtmp, sizeof(int64_t) * n) &&
              dalloc((void **)&w.inv0, sizeof(int64_t) * n) &&
              dalloc((void **)&w.hist, sizeof(int64_t) * hist_n) &&
              dalloc((void **)&w.scan, sizeof(int64_t) * (scan_n + 1)) &&
              dalloc((void **)&w.flags, sizeof(int64_t) * maxI) &&
              dalloc((void **)&w.c1tmp, sizeof(int32_t) * n) &&
              dalloc((void **)&w.c2tmp, sizeof(int32_t) * n) &&
              (!p->has_vals || dalloc(&w.valtmp, tsize(p->dtype) * n));
    if (ok && (p->flags & TC_PATTERN_CHECK_DUPLICATES))
        ok = dalloc((void **)&w.dk, sizeof(int32_t) * n) && dalloc((void **)&w.dp, sizeof(int64_t) * n);
    return ok ? TC_OK : TC_ERR_OOM;
}

// Allocates every array of a pattern (and its scratch) for the given shape.
static tc_status alloc_pattern(tc_pattern *p) {
    const int64_t n = p->nnz;
    const size_t es = tsize(p->dtype);
    const bool lean = (p->flags & TC_PATTERN_LEAN) != 0;
    bool ok = dalloc((void **)&p->status, sizeof(int)) &&
              dalloc((void **)&p->counts, sizeof(int64_t) * TC_ORDER);
    for (int d = 0; d < TC_ORDER && ok; ++d) {
        ModeData &m = p->md[d];
        const int64_t I = p->dims[d];
        ok = dalloc((void **)&m.row_ptr, sizeof(int64_t) * (I + 1)) &&
             (lean || dalloc((void **)&m.perm, sizeof(int64_t) * n)) &&
             dalloc((void **)&m.nz_rows, sizeof(int32_t) * I) &&
             dalloc((void **)&m.nz_ptr, sizeof(int64_t) * (I + 1)) &&
             dalloc((void **)&m.cols[0], sizeof(int32_t) * n) &&
             dalloc((void **)&m.cols[1], sizeof(int32_t) * n) &&
             (!p->has_vals || dalloc(&m.vals, es * n)) &&
             (d == 0 || lean || dalloc((void **)&m.to0, sizeof(int64_t) * n));
        m.n_ne_dev = p->counts ? p->counts + d : nullptr;
    }
    if (!ok) return TC_ERR_OOM;
    return alloc_scratch(p);
}

// Fills the pattern from the input coordinates; asynchronous on st, allocates
// nothing.  Range errors and duplicates are recorded in the status word.
static void fill_pattern(tc_pattern *p, const int32_t *const *idx, const void *vals,
                         cudaStream_t st) {
    const int64_t n = p->nnz;
    PatternScratch &w = p->work;
    for (int d = 0; d < TC_ORDER; ++d) {
        if (n > 0) {
            range_check_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(idx[d], n, p->dims[d],
                                                                       p->status);
            count_launch();
        }
    }
    const bool lean = (p->flags & TC_PATTERN_LEAN) != 0;
    const bool consume = (p->flags & TC_PATTERN_CONSUME_INPUT) != 0;
    for (int d = 0; d < TC_ORDER; ++d) {
        ModeData &m = p->md[d];
        const int64_t I = p->dims[d];
        // keys outside [0, I) still sort into a permutation of [0, n): digits
        // are taken from the low bits, so no write leaves the arrays
        int o1, o2;
        other_modes(d, o1, o2);
        SortSide in{const_cast<int32_t *>(idx[d]), nullptr, const_cast<int32_t *>(idx[o1]),
                    const_cast<int32_t *>(idx[o2]), const_cast<void *>(vals)};
        SortSide out{w.kbuf, m.perm, m.cols[0], m.cols[1], m.vals};
        SortSide tmp{w.ktmp, w.vtmp, w.c1tmp, w.c2tmp, w.valtmp};
        bool first_to_out = false;
        if (lean) {
            // work space of a lean build: mode 0 sorts through the arrays of
            // modes 1 and 2 (not yet built), mode 1 through those of mode 2,
            // and mode 2 through the consumed input (or its own buffers)
            const ModeData &m1 = p->md[1], &m2 = p->md[2];
            if (d == 0) {
                out.key = m1.cols[0];
                tmp = SortSide{m1.cols[1], nullptr, m2.cols[0], m2.cols[1], m2.vals};
            } else if (d == 1) {
                tmp = SortSide{w.ktmp, nullptr, m2.cols[0], m2.cols[1], m2.vals};
            } else if (consume) {
                tmp = in;
                first_to_out = true;
            }
        }
        radix_sort_p(p->has_vals ? (int)tsize(p->dtype) : 0, in, out, tmp, n, I - 1, p->dims[o1],
                     p->dims[o2], w.hist, w.scan, first_to_out, st);
        row_ptr_kernel<<<grid_for(I + 1, 256), 256, 0, st>>>(out.key, n, I, m.row_ptr);
        count_launch();
        nonempty_flags_kernel<<<grid_for(I, 256), 256, 0, st>>>(m.row_ptr, I, w.flags);
        count_launch();
        scan_exclusive(w.flags, w.flags, I, w.scan, st);
        nonempty_fill_kernel<<<grid_for(I, 256), 256, 0, st>>>(m.row_ptr, I, w.flags, n, m.nz_rows,
                                                               m.nz_ptr, m.n_ne_dev);
        count_launch();
    }
    // the mode-d -> mode-0 maps are rebuilt on first use (ensure_to0)
    p->to0_valid = 0;
    if ((p->flags & TC_PATTERN_CHECK_DUPLICATES) && n > 1) {
        // lexicographic order by (i_0, i_1, i_2): stable sorts by i_2, then i_1, then i_0
        int64_t *cur = nullptr;
        for (int d = TC_ORDER - 1; d >= 0; --d) {
            int64_t *dst = (cur == w.inv0) ? w.dp : w.inv0;
            if (cur) {
                gather_i32_kernel<<<grid_for(n, 256), 256, 0, st>>>(idx[d], cur, n, p->dims[d], w.dk);
                count_launch();
            }
            radix_sort(cur ? w.dk : idx[d], cur, n, p->dims[d] - 1, w.kbuf, dst, w.ktmp, w.vtmp,
                       w.hist, w.scan, st);
            cur = dst;
        }
        dup_check_kernel<<<grid_for(n, 256), 256, 0, st>>>(idx[0], idx[1], idx[2], cur, n, p->status);
        count_launch();
    }
}

tc_status build_pattern_impl(int order, const int64_t *dims, int64_t nnz,
                             const int32_t *const *idx, const void *vals, tc_dtype dtype,
                             unsigned flags, cudaStream_t st, tc_pattern **out) {
    tc_pattern *p = new (std::nothrow) tc_pattern();
    if (!p) return TC_ERR_OOM;
    int dev = 0;
    cudaGetDevice(&dev);
    p->device = dev;
    p->order = order;
    p->nnz = nnz;
    p->dtype = dtype;
    p->has_vals = vals != nullptr;
    p->flags = flags;
    for (int d = 0; d < TC_ORDER; ++d) p->dims[d] = dims[d];
    tc_status rc = alloc_pattern(p);
    if (rc != TC_OK) {
        free_pattern(p);
        return rc;
    }
    if (cudaMemsetAsync(p->status, 0, sizeof(int), st) != cudaSuccess) {
        free_pattern(p);
        return TC_ERR_CUDA;
    }
    fill_pattern(p, idx, vals, st);
    int h = 0;
    if (cudaMemcpyAsync(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        free_pattern(p);
        return TC_ERR_CUDA;
    }
    if (h) {
        free_pattern(p);
        return (tc_status)h;
    }
    if (!(flags & TC_PATTERN_REFILLABLE)) free_scratch(p);
    *out = p;
    return TC_OK;
}

tc_status ensure_to0(const tc_pattern *pc, cudaStream_t st) {
    tc_pattern *p = const_cast<tc_pattern *>(pc);
    if (p->to0_valid || p->nnz == 0) return TC_OK;
    if (p->flags & TC_PATTERN_LEAN) return TC_ERR_UNSUPPORTED;   // no positions kept
    const int64_t n = p->nnz;
    // the inverse permutation is needed once per pattern contents: a refillable
    // pattern keeps it in its builder work space, others borrow it for this call
    int64_t *inv0 = p->work.inv0;
    const bool temp = inv0 == nullptr;
    if (temp) TC_CUDA(cudaMallocAsync((void **)&inv0, sizeof(int64_t) * n, st));
    invert_perm_kernel<<<grid_for(n, 256), 256, 0, st>>>(p->md[0].perm, n, inv0);
    count_launch();
    for (int d = 1; d < TC_ORDER; ++d) {
        compose_kernel<<<grid_for(n, 256), 256, 0, st>>>(inv0, p->md[d].perm, n, p->md[d].to0);
        count_launch();
    }
    if (temp) TC_CUDA(cudaFreeAsync(inv0, st));
    p->to0_valid = 1;
    return TC_OK;
}

tc_status refill_pattern_impl(tc_pattern *p, const int32_t *const *idx, const void *vals,
                              cudaStream_t st) {
    if (!p->work.kbuf) return TC_ERR_ARG;     // built without TC_PATTERN_REFILLABLE
    fill_pattern(p, idx, vals, st);
    return TC_OK;
}

}  // namespace tc

// ------------------------------------------------------------------ allocation-free mode sort
// tc_sort_mode_noalloc runs the same radix-sort pipeline as the pattern
// builder, but its work space is one fixed array compiled into the library
// instead of device allocations.
#include <mutex>

namespace tc {
namespace noalloc {

constexpr int64_t kMaxNnz = TC_SORT_NOALLOC_MAX_NNZ;
constexpr int64_t kTiles = (kMaxNnz + kTile - 1) / kTile;
constexpr int64_t kHist = (int64_t)kDigits * kTiles;

constexpr int64_t scan_elems(int64_t n) {
    int64_t total = 0;
    while (n > kScanTile) {
        n = (n + kScanTile - 1) / kScanTile;
        total += n;
    }
    return total;
}

// byte offsets of the pieces (all multiples of 256)
constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kOffKtmp = 0;
constexpr size_t kOffKout = kOffKtmp + round256(sizeof(int32_t) * kMaxNnz);
constexpr size_t kOffVtmp = kOffKout + round256(sizeof(int32_t) * kMaxNnz);
constexpr size_t kOffHist = kOffVtmp + round256(sizeof(int64_t) * kMaxNnz);
constexpr size_t kOffScan = kOffHist + round256(sizeof(int64_t) * kHist);
constexpr size_t kOffStatus = kOffScan + round256(sizeof(int64_t) * (scan_elems(kHist) + 1));
constexpr size_t kBytes = kOffStatus + 256;

// The work space: each GPU that loads this library holds it (about 16.5 MB)
// until the process exits.  Only host code below needs its device address.
static __device__ __align__(256) unsigned char g_sort_scratch[kBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_mu;
static void *g_addr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device, looked up once per
// device with that device current.
static tc_status scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TC_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return TC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_sort_scratch) != cudaSuccess || !ptr) return TC_ERR_CUDA;
        g_addr[dev] = ptr;
    }
    *out = g_addr[dev];
    return TC_OK;
}

}  // namespace noalloc
}  // namespace tc

extern "C" tc_status tc_sort_mode_noalloc(int64_t nnz, const int32_t *key, int64_t I,
                                          int64_t *perm, int64_t *row_ptr, int *status,
                                          tc_stream_t stream) {
    using namespace tc;
    if (nnz < 0 || I < 1 || I > INT32_MAX || !row_ptr || (nnz > 0 && (!key || !perm)))
        return TC_ERR_ARG;
    if (nnz > noalloc::kMaxNnz) return TC_ERR_UNSUPPORTED;
    void *base = nullptr;
    tc_status rc = noalloc::scratch_address(&base);
    if (rc != TC_OK) return rc;
    unsigned char *b = static_cast<unsigned char *>(base);
    int32_t *ktmp = reinterpret_cast<int32_t *>(b + noalloc::kOffKtmp);
    int32_t *kout = reinterpret_cast<int32_t *>(b + noalloc::kOffKout);
    int64_t *vtmp = reinterpret_cast<int64_t *>(b + noalloc::kOffVtmp);
    int64_t *hist = reinterpret_cast<int64_t *>(b + noalloc::kOffHist);
    int64_t *scan = reinterpret_cast<int64_t *>(b + noalloc::kOffScan);
    int *st_word = status ? status : reinterpret_cast<int *>(b + noalloc::kOffStatus);
    cudaStream_t st = (cudaStream_t)stream;
    // Every scratch word a call reads was written earlier in the same call
    // (histograms are rewritten in full each pass), so only the status word
    // needs clearing.
    if (cudaMemsetAsync(st_word, 0, sizeof(int), st) != cudaSuccess) return TC_ERR_CUDA;
    if (nnz > 0) {
        range_check_kernel<<<grid_for(nnz, 256, 4096), 256, 0, st>>>(key, nnz, I, st_word);
        count_launch();
    }
    radix_sort(key, nullptr, nnz, I - 1, kout, perm, ktmp, vtmp, hist, scan, st);
    row_ptr_kernel<<<grid_for(I + 1, 256), 256, 0, st>>>(kout, nnz, I, row_ptr);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ERR_CUDA;
}
