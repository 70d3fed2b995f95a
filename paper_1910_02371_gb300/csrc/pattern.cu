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

// Exclusive scan of n int64 values (in may equal out).
static tc_status scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t st) {
    if (n <= 0) return TC_OK;
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        scan_tile_kernel<<<1, kScanThreads, 0, st>>>(in, n, nullptr, out);
        count_launch();
        return TC_OK;
    }
    int64_t *sums = nullptr;
    TC_CUDA(cudaMallocAsync((void **)&sums, sizeof(int64_t) * nb, st));
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, sums);
    count_launch();
    tc_status rc = scan_exclusive(sums, sums, nb, st);
    if (rc == TC_OK) {
        scan_tile_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, sums, out);
        count_launch();
    }
    cudaFreeAsync(sums, st);
    return rc;
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

// Stable sort of (key, value) pairs by key in [0, max_key]; vals_in == null
// means value = input position.  Results in kout / vout; ktmp / vtmp scratch.
static tc_status radix_sort(const int32_t *keys_in, const int64_t *vals_in, int64_t n,
                            int64_t max_key, int32_t *kout, int64_t *vout, int32_t *ktmp,
                            int64_t *vtmp, cudaStream_t st) {
    int bits = 0;
    while (bits < 31 && (max_key >> bits) > 0) ++bits;
    const int passes = (bits + kRadixBits - 1) / kRadixBits;
    if (passes == 0 || n == 0) {
        if (n > 0) {
            iota_copy_kernel<<<grid_for(n, 256), 256, 0, st>>>(keys_in, vals_in, n, kout, vout);
            count_launch();
        }
        return TC_OK;
    }
    const int64_t num_tiles = (n + kTile - 1) / kTile;
    int64_t *hist = nullptr;
    TC_CUDA(cudaMallocAsync((void **)&hist, sizeof(int64_t) * kDigits * num_tiles, st));
    const int32_t *ks = keys_in;
    const int64_t *vs = vals_in;
    tc_status rc = TC_OK;
    for (int p = 0; p < passes && rc == TC_OK; ++p) {
        const bool to_out = ((passes - 1 - p) % 2) == 0;
        int32_t *kd = to_out ? kout : ktmp;
        int64_t *vd = to_out ? vout : vtmp;
        const int shift = p * kRadixBits;
        radix_hist_kernel<<<(unsigned)num_tiles, kSortThreads, 0, st>>>(ks, n, shift, num_tiles, hist);
        count_launch();
        rc = scan_exclusive(hist, hist, kDigits * num_tiles, st);
        if (rc != TC_OK) break;
        radix_scatter_kernel<<<(unsigned)num_tiles, kSortThreads, 0, st>>>(ks, vs, n, shift, num_tiles,
                                                                          hist, kd, vd);
        count_launch();
        ks = kd;
        vs = vd;
    }
    cudaFreeAsync(hist, st);
    return rc;
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

// row_ptr from sorted keys: row r starts at the first position with key >= r.
__global__ void row_ptr_kernel(const int32_t *__restrict__ sk, int64_t n, int64_t I,
                               int64_t *__restrict__ row_ptr) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t key = sk[q];
        const int64_t prev = q > 0 ? (int64_t)sk[q - 1] : -1;
        for (int64_t r = prev + 1; r <= key; ++r) row_ptr[r] = q;
        if (q == n - 1)
            for (int64_t r = key + 1; r <= I; ++r) row_ptr[r] = n;
    }
}

__global__ void nonempty_flags_kernel(const int64_t *__restrict__ row_ptr, int64_t I,
                                      int64_t *__restrict__ flags) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < I;
         r += (int64_t)gridDim.x * blockDim.x)
        flags[r] = row_ptr[r + 1] > row_ptr[r] ? 1 : 0;
}

__global__ void nonempty_fill_kernel(const int64_t *__restrict__ row_ptr, int64_t I,
                                     const int64_t *__restrict__ pos, int64_t n,
                                     int32_t *__restrict__ nz_rows, int64_t *__restrict__ nz_ptr) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < I;
         r += (int64_t)gridDim.x * blockDim.x) {
        if (row_ptr[r + 1] > row_ptr[r]) {
            nz_rows[pos[r]] = (int32_t)r;
            nz_ptr[pos[r]] = row_ptr[r];
        }
        if (r == I - 1) nz_ptr[pos[r] + (row_ptr[r + 1] > row_ptr[r] ? 1 : 0)] = n;
    }
}

__global__ void gather_i32_kernel(const int32_t *__restrict__ src, const int64_t *__restrict__ perm,
                                  int64_t n, int32_t *__restrict__ dst) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = src[perm[q]];
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
    cudaFree(p->status);
    cudaFree(p->dscratch);
    delete p;
}

#define TC_TRY(x)                      \
    do {                               \
        tc_status r_ = (x);            \
        if (r_ != TC_OK) {             \
            rc = r_;                   \
            goto fail;                 \
        }                              \
    } while (0)
#define TC_ALLOC(ptr, bytes)                                                     \
    do {                                                                         \
        if (cudaMalloc((void **)&(ptr), (bytes) > 0 ? (bytes) : 16) != cudaSuccess) { \
            rc = TC_ERR_OOM;                                                     \
            goto fail;                                                           \
        }                                                                        \
    } while (0)

tc_status build_pattern_impl(int order, const int64_t *dims, int64_t nnz,
                             const int32_t *const *idx, const void *vals, tc_dtype dtype,
                             unsigned flags, cudaStream_t st, tc_pattern **out) {
    tc_status rc = TC_OK;
    tc_pattern *p = new (std::nothrow) tc_pattern();
    if (!p) return TC_ERR_OOM;
    int32_t *kbuf = nullptr, *ktmp = nullptr;
    int64_t *vtmp = nullptr, *inv0 = nullptr, *flags_buf = nullptr, *dp = nullptr;
    int32_t *dk = nullptr;
    const size_t es = tsize(dtype);
    const int64_t n = nnz;
    int dev = 0;
    cudaGetDevice(&dev);
    p->device = dev;
    p->order = order;
    p->nnz = nnz;
    p->dtype = dtype;
    p->has_vals = vals != nullptr;
    for (int d = 0; d < TC_ORDER; ++d) p->dims[d] = dims[d];

    TC_ALLOC(p->status, sizeof(int));
    TC_ALLOC(p->dscratch, sizeof(double) * kScratchDoubles);
    if (cudaMemsetAsync(p->status, 0, sizeof(int), st) != cudaSuccess) {
        rc = TC_ERR_CUDA;
        goto fail;
    }
    for (int d = 0; d < TC_ORDER; ++d) {
        if (n > 0) {
            range_check_kernel<<<grid_for(n, 256, 4096), 256, 0, st>>>(idx[d], n, dims[d], p->status);
            count_launch();
        }
    }
    TC_ALLOC(kbuf, sizeof(int32_t) * n);
    TC_ALLOC(ktmp, sizeof(int32_t) * n);
    TC_ALLOC(vtmp, sizeof(int64_t) * n);
    for (int d = 0; d < TC_ORDER; ++d) {
        ModeData &m = p->md[d];
        const int64_t I = dims[d];
        TC_ALLOC(m.perm, sizeof(int64_t) * n);
        TC_ALLOC(m.row_ptr, sizeof(int64_t) * (I + 1));
        // a range error would make the sort write out of bounds: stop before it
        {
            int h = 0;
            if (cudaMemcpyAsync(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess) {
                rc = TC_ERR_CUDA;
                goto fail;
            }
            if (h) {
                rc = (tc_status)h;
                goto fail;
            }
        }
        TC_TRY(radix_sort(idx[d], nullptr, n, I - 1, kbuf, m.perm, ktmp, vtmp, st));
        if (cudaMemsetAsync(m.row_ptr, 0, sizeof(int64_t) * (I + 1), st) != cudaSuccess) {
            rc = TC_ERR_CUDA;
            goto fail;
        }
        if (n > 0) {
            row_ptr_kernel<<<grid_for(n, 256), 256, 0, st>>>(kbuf, n, I, m.row_ptr);
            count_launch();
        }
        // nonempty rows
        TC_ALLOC(flags_buf, sizeof(int64_t) * I);
        nonempty_flags_kernel<<<grid_for(I, 256), 256, 0, st>>>(m.row_ptr, I, flags_buf);
        count_launch();
        int64_t last_flag = 0;
        if (cudaMemcpyAsync(&last_flag, flags_buf + (I - 1), sizeof(int64_t), cudaMemcpyDeviceToHost,
                            st) != cudaSuccess) {
            rc = TC_ERR_CUDA;
            goto fail;
        }
        TC_TRY(scan_exclusive(flags_buf, flags_buf, I, st));
        int64_t last_pos = 0;
        if (cudaMemcpyAsync(&last_pos, flags_buf + (I - 1), sizeof(int64_t), cudaMemcpyDeviceToHost,
                            st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = TC_ERR_CUDA;
            goto fail;
        }
        m.n_ne = last_pos + last_flag;
        TC_ALLOC(m.nz_rows, sizeof(int32_t) * m.n_ne);
        TC_ALLOC(m.nz_ptr, sizeof(int64_t) * (m.n_ne + 1));
        nonempty_fill_kernel<<<grid_for(I, 256), 256, 0, st>>>(m.row_ptr, I, flags_buf, n, m.nz_rows,
                                                               m.nz_ptr);
        count_launch();
        cudaStreamSynchronize(st);
        cudaFree(flags_buf);
        flags_buf = nullptr;
        // the other modes' indices and the values in this mode's order
        int o1, o2;
        other_modes(d, o1, o2);
        TC_ALLOC(m.cols[0], sizeof(int32_t) * n);
        TC_ALLOC(m.cols[1], sizeof(int32_t) * n);
        if (n > 0) {
            gather_i32_kernel<<<grid_for(n, 256), 256, 0, st>>>(idx[o1], m.perm, n, m.cols[0]);
            gather_i32_kernel<<<grid_for(n, 256), 256, 0, st>>>(idx[o2], m.perm, n, m.cols[1]);
            count_launch(2);
        }
        if (vals) {
            TC_ALLOC(m.vals, es * n);
            if (n > 0) {
                if (dtype == TC_F64)
                    gather_val_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(
                        (const double *)vals, m.perm, n, (double *)m.vals);
                else
                    gather_val_kernel<float><<<grid_for(n, 256), 256, 0, st>>>(
                        (const float *)vals, m.perm, n, (float *)m.vals);
                count_launch();
            }
        }
    }
    // mode-d position -> mode-0 position, for caller arrays in pattern order
    TC_ALLOC(inv0, sizeof(int64_t) * n);
    if (n > 0) {
        invert_perm_kernel<<<grid_for(n, 256), 256, 0, st>>>(p->md[0].perm, n, inv0);
        count_launch();
    }
    for (int d = 1; d < TC_ORDER; ++d) {
        TC_ALLOC(p->md[d].to0, sizeof(int64_t) * n);
        if (n > 0) {
            compose_kernel<<<grid_for(n, 256), 256, 0, st>>>(inv0, p->md[d].perm, n, p->md[d].to0);
            count_launch();
        }
    }
    if ((flags & TC_PATTERN_CHECK_DUPLICATES) && n > 1) {
        // lexicographic order by (i_0, i_1, i_2): stable sorts by i_2, then i_1, then i_0.
        // inv0 is free again; dk holds gathered keys, dp the next permutation.
        TC_ALLOC(dk, sizeof(int32_t) * n);
        TC_ALLOC(dp, sizeof(int64_t) * n);
        int64_t *cur = nullptr;
        for (int d = TC_ORDER - 1; d >= 0; --d) {
            int64_t *dst = (cur == inv0) ? dp : inv0;
            if (cur) {
                gather_i32_kernel<<<grid_for(n, 256), 256, 0, st>>>(idx[d], cur, n, dk);
                count_launch();
            }
            TC_TRY(radix_sort(cur ? dk : idx[d], cur, n, dims[d] - 1, kbuf, dst, ktmp, vtmp, st));
            cur = dst;
        }
        dup_check_kernel<<<grid_for(n, 256), 256, 0, st>>>(idx[0], idx[1], idx[2], cur, n, p->status);
        count_launch();
        cudaStreamSynchronize(st);
    }
    {
        int h = 0;
        if (cudaMemcpyAsync(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = TC_ERR_CUDA;
            goto fail;
        }
        if (h) {
            rc = (tc_status)h;
            goto fail;
        }
    }
    cudaFree(kbuf);
    cudaFree(ktmp);
    cudaFree(vtmp);
    cudaFree(inv0);
    cudaFree(dk);
    cudaFree(dp);
    *out = p;
    return TC_OK;
fail:
    cudaStreamSynchronize(st);
    cudaFree(kbuf);
    cudaFree(ktmp);
    cudaFree(vtmp);
    cudaFree(inv0);
    cudaFree(flags_buf);
    cudaFree(dk);
    cudaFree(dp);
    free_pattern(p);
    return rc;
}

}  // namespace tc
