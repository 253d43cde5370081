// Format conversions (Section 5.1: step 1 sorts the nonzeros into the format's order,
// step 2 populates and compresses the arrays, touching every element once).
//
//   triplets -> CRS (Section 2):  key = (row << cbits) | col, stable LSD radix sort with
//                                 the input position as payload (so equal pairs keep input
//                                 order), duplicate resolution, row_ptr by boundary fill.
//   CRS -> row-length bins        (row-split product, GPU counterpart of ParCRS)
//   CRS -> merge-path partition   (Section 3.3: split points of the row-end / nonzero path)
//   CRS -> Hilbert blocked (HB)   (Sections 3.1, 4.2): key = Hilbert index h(r, c) on the
//                                 2^K grid (or block-then-row-major), radix sort, block
//                                 segmentation where h >> 2 log2(beta) changes, packed
//                                 ((r mod beta) << 16) | (c mod beta) indices.
#include "common.cuh"
#include "convert.cuh"
#include "hilbert.cuh"
#include "df64.cuh"

#include <algorithm>

namespace spmv {

namespace {

constexpr int CB = 256;   // block size of the simple element-wise kernels
// Slack after the CRS arrays: the merge product's bulk copies read whole 16-byte units.
constexpr size_t TMA_PAD = 64;

inline unsigned grid_for(int64_t n, int per_block = CB) {
    int64_t g = (n + per_block - 1) / per_block;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 1 << 30));
}

// ---------------------------------------------------------------- validation
__global__ void k_validate(const int32_t *__restrict__ row, const int32_t *__restrict__ col, int64_t nnz, int64_t m,
                           int64_t n, uint32_t *status) {
    // four triplets per 16-byte load of each array when both are 16-byte aligned (the library's
    // own copies are)
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    auto out = [&](int32_t r, int32_t c) { return (r < 0) | ((int64_t)r >= m) | (c < 0) | ((int64_t)c >= n); };
    bool bad = false;
    const int64_t ngrp = ((reinterpret_cast<uintptr_t>(row) | reinterpret_cast<uintptr_t>(col)) & 15u) ? 0 : nnz / 4;
#pragma unroll 2
    for (int64_t g = t; g < ngrp; g += stride) {
        const int4 r4 = ((const int4 *)row)[g], c4 = ((const int4 *)col)[g];
        bad |= out(r4.x, c4.x) | out(r4.y, c4.y) | out(r4.z, c4.z) | out(r4.w, c4.w);
    }
    for (int64_t i = 4 * ngrp + t; i < nnz; i += stride) bad |= out(row[i], col[i]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_INDEX_RANGE);
}

// ---------------------------------------------------------------- COO -> CRS
__global__ void k_coo_keys(const int32_t *__restrict__ row, const int32_t *__restrict__ col, int64_t nnz, int cbits,
                           uint64_t *__restrict__ keys, uint32_t *__restrict__ perm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nnz) {
        keys[i] = ((uint64_t)(uint32_t)row[i] << cbits) | (uint32_t)col[i];
        perm[i] = (uint32_t)i;
    }
}

// head[i] = 1 where a new (row, col) starts; flags a duplicate in *status.
__global__ void k_heads(const uint64_t *__restrict__ keys, int64_t nnz, uint32_t *__restrict__ head,
                        uint32_t *status) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool dup = false;
    if (i < nnz) {
        bool h = (i == 0) || keys[i] != keys[i - 1];
        head[i] = h ? 1u : 0u;
        dup = !h;
    }
    if (__any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) atomicOr(status, ST_DUPLICATE);
}

// dst[i] = src[perm[i]]: GATHER_ILP independent random reads in flight per thread.
constexpr int GATHER_ILP = 8;

template <typename T>
__global__ void k_gather(const T *__restrict__ src, const uint32_t *__restrict__ perm, int64_t n, T *__restrict__ dst) {
    const int64_t base = (int64_t)blockIdx.x * blockDim.x * GATHER_ILP + threadIdx.x;
    uint32_t p[GATHER_ILP];
    T v[GATHER_ILP];
#pragma unroll
    for (int u = 0; u < GATHER_ILP; ++u) {
        const int64_t i = base + (int64_t)u * blockDim.x;
        p[u] = i < n ? perm[i] : 0u;
    }
#pragma unroll
    for (int u = 0; u < GATHER_ILP; ++u) {
        const int64_t i = base + (int64_t)u * blockDim.x;
        if (i < n) v[u] = __ldg(src + p[u]);
    }
#pragma unroll
    for (int u = 0; u < GATHER_ILP; ++u) {
        const int64_t i = base + (int64_t)u * blockDim.x;
        if (i < n) dst[i] = v[u];
    }
}

__device__ __forceinline__ double load_as_double(const void *v, int dt, int64_t i) {
    if (dt == SPMV_F64) return ((const double *)v)[i];
    if (dt == SPMV_F32) return (double)((const float *)v)[i];
    return (double)__bfloat162float(((const __nv_bfloat16 *)v)[i]);
}

__device__ __forceinline__ void store_from_double(void *v, int dt, int64_t i, double x) {
    if (dt == SPMV_F64) ((double *)v)[i] = x;
    else if (dt == SPMV_F32) ((float *)v)[i] = __double2float_rn(x);
    else ((__nv_bfloat16 *)v)[i] = __double2bfloat16(x);
}

// Duplicate (row, col) runs: the head writes the compacted key and column and the sum of
// the run's values in input order (double accumulation, one rounding to the stored type).
__global__ void k_dup_compact(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ perm,
                              const uint32_t *__restrict__ head, const uint32_t *__restrict__ pos, int64_t nnz,
                              int cbits, const void *__restrict__ vin, int dt, uint64_t *__restrict__ ckeys,
                              int32_t *__restrict__ col, void *__restrict__ vout) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nnz || !head[i]) return;
    int64_t o = pos[i];
    ckeys[o] = keys[i];
    col[o] = (int32_t)(keys[i] & ((1ull << cbits) - 1ull));
    if (vin) {
        double s = load_as_double(vin, dt, perm[i]);
        for (int64_t j = i + 1; j < nnz && !head[j]; ++j) s = s + load_as_double(vin, dt, perm[j]);
        store_from_double(vout, dt, o, s);
    }
}

// row_ptr by boundary fill over the sorted keys: entry i is the first of rows
// (row(i-1), row(i)]; the sentinel thread i = nnz closes rows (row(nnz-1), m].
// Gaps longer than GAP_INLINE rows are queued for k_fill_gaps.
constexpr int GAP_INLINE = 64;

// row_ptr from sorted keys: entry i (0 <= i <= nnz) gives value i to the rows between the
// row of key i-1 (exclusive) and the row of key i; runs longer than GAP_INLINE rows (empty
// rows) are recorded for k_fill_gaps.  With col != nullptr it also writes the column of
// every key and flags equal neighbouring keys (ST_DUPLICATE), the whole finish of a
// conversion without duplicates in one read of the keys.
constexpr int RPF_U = 4;   // entries per thread of k_row_ptr_fill
__global__ void k_row_ptr_fill(const uint64_t *__restrict__ keys, int64_t nnz, int cbits, int64_t m,
                               int32_t *__restrict__ row_ptr, int64_t *__restrict__ gaps,
                               unsigned long long *__restrict__ ngaps, int32_t *__restrict__ col,
                               uint32_t *__restrict__ status) {
    // entries i0 .. i0 + RPF_U - 1 (entry nnz closes the last rows); kk[u + 1] = keys[i0 + u],
    // kk[0] = keys[i0 - 1]
    const int64_t i0 = RPF_U * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    const uint64_t cmask = (1ull << cbits) - 1ull;
    bool dup = false;
    if (i0 <= nnz) {
        uint64_t kk[RPF_U + 1];
        kk[0] = i0 > 0 ? keys[i0 - 1] : 0ull;
        const bool full = i0 + RPF_U <= nnz;   // keys + i0 is 32-byte aligned (i0 a multiple of 4)
        if (full) {
            const ulonglong2 a = *(const ulonglong2 *)(keys + i0), b2 = *(const ulonglong2 *)(keys + i0 + 2);
            kk[1] = a.x;
            kk[2] = a.y;
            kk[3] = b2.x;
            kk[4] = b2.y;
        } else {
#pragma unroll
            for (int u = 0; u < RPF_U; ++u) kk[u + 1] = i0 + u < nnz ? keys[i0 + u] : 0ull;
        }
        if (col) {
            if (full) {
                *(int4 *)(col + i0) = make_int4((int32_t)(kk[1] & cmask), (int32_t)(kk[2] & cmask),
                                                (int32_t)(kk[3] & cmask), (int32_t)(kk[4] & cmask));
            } else {
#pragma unroll
                for (int u = 0; u < RPF_U; ++u)
                    if (i0 + u < nnz) col[i0 + u] = (int32_t)(kk[u + 1] & cmask);
            }
        }
#pragma unroll
        for (int u = 0; u < RPF_U; ++u) {
            const int64_t i = i0 + u;
            if (i > nnz) break;
            const uint64_t kc = kk[u + 1], kp = kk[u];
            if (col && i < nnz) dup |= i > 0 && kc == kp;
            const int64_t hi = i < nnz ? (int64_t)(kc >> cbits) : m;
            const int64_t lo = i > 0 ? (int64_t)(kp >> cbits) + 1 : 0;   // rows lo..hi get value i
            if (hi - lo + 1 <= GAP_INLINE) {
                for (int64_t r = lo; r <= hi; ++r) row_ptr[r] = (int32_t)i;
            } else {
                const unsigned long long g = atomicAdd(ngaps, 1ull);
                gaps[3 * g + 0] = lo;
                gaps[3 * g + 1] = hi;
                gaps[3 * g + 2] = i;
            }
        }
    }
    if (col && __any_sync(0xffffffffu, dup) && (threadIdx.x & 31) == 0) atomicOr(status, ST_DUPLICATE);
}

__global__ void k_fill_gaps(const int64_t *__restrict__ gaps, const unsigned long long *__restrict__ ngaps,
                            int32_t *__restrict__ row_ptr) {
    const unsigned long long ng = *ngaps;
    for (unsigned long long g = blockIdx.x; g < ng; g += gridDim.x) {
        int64_t lo = gaps[3 * g], hi = gaps[3 * g + 1];
        int32_t v = (int32_t)gaps[3 * g + 2];
        for (int64_t r = lo + threadIdx.x; r <= hi; r += blockDim.x) row_ptr[r] = v;
    }
}

// ---------------------------------------------------------------- row-length bins
// Row-length class of every row (key) with the row id (payload), the rows per class and the
// longest row.  Grid-stride with per-warp ballots and per-block totals, so that only a few
// thousand global atomics meet on the nine counters.
constexpr int ROW_CLASS_GRID = 1024;
__global__ void k_row_class(const int32_t *__restrict__ row_ptr, int64_t m, uint64_t *__restrict__ cls,
                            uint32_t *__restrict__ rows, unsigned long long *__restrict__ counts,
                            unsigned long long *__restrict__ maxlen) {
    __shared__ uint32_t sc[NUM_ROW_CLASSES];
    __shared__ unsigned long long smax;
    if (threadIdx.x < NUM_ROW_CLASSES) sc[threadIdx.x] = 0u;
    if (threadIdx.x == 0) smax = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    unsigned long long mx = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < m; i0 += stride) {   // warp-uniform trip count
        const int64_t i = i0 + threadIdx.x;
        int c = -1;
        if (i < m) {
            const unsigned long long len = (unsigned long long)(row_ptr[i + 1] - row_ptr[i]);
            c = row_class(len);
            cls[i] = (uint64_t)c;
            rows[i] = (uint32_t)i;
            mx = max(mx, len);
        }
#pragma unroll
        for (int q = 0; q < NUM_ROW_CLASSES; ++q) {
            const uint32_t bq = __ballot_sync(0xffffffffu, c == q);
            if (lane == 0 && bq) atomicAdd(&sc[q], (uint32_t)__popc(bq));
        }
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0 && mx) atomicMax(&smax, mx);
    __syncthreads();
    if (threadIdx.x < NUM_ROW_CLASSES && sc[threadIdx.x]) atomicAdd(&counts[threadIdx.x], (unsigned long long)sc[threadIdx.x]);
    if (threadIdx.x == 0 && smax) atomicMax(maxlen, smax);
}

// ---------------------------------------------------------------- merge partition
// Split point on diagonal d of the path A = row_ptr[1..m] (row ends) x B = 0..nnz-1
// (nonzero indices): the largest i <= min(d, m) such that the first i row ends are all
// consumed within the first d steps, where a tie consumes the row end (Section 3.3).
__device__ __forceinline__ int64_t merge_split(int64_t d, int64_t m, int64_t nnz, const int32_t *__restrict__ row_ptr) {
    int64_t lo = d - nnz > 0 ? d - nnz : 0;
    int64_t hi = d < m ? d : m;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)row_ptr[mid] <= d - mid) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Per-lane descriptors of the warp tiles (MERGE_WARP_ITEMS path items, MERGE_WARP_IPT per
// lane).  Row end r of a tile sits at path position r + (nonzeros of the tile before it); for
// lane l, covering positions [7l, 7l + 7): bits 0-7 the number of row ends before its range
// (its first row), bits 8-15 the number of nonzeros before it (its first nonzero), bits
// 16-22 which of its items are row ends, bits 24-26 how many items it has; bit 31 (lane 0)
// marks a tile whose first row began in an earlier tile.
__global__ void k_merge_desc(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ part_row,
                             const int32_t *__restrict__ part_nz, int64_t tiles, uint32_t *__restrict__ desc) {
    __shared__ uint32_t s_bits[8][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t t = (int64_t)blockIdx.x * 8 + w;
    if (t >= tiles) return;
    const int64_t i0 = part_row[t], j0 = part_nz[t];
    const int nrows = (int)(part_row[t + 1] - i0), nnzt = (int)(part_nz[t + 1] - j0);
    if (lane < 8) s_bits[w][lane] = 0u;
    __syncwarp();
    for (int r = lane; r < nrows; r += 32) {
        const int pos = r + (int)(row_ptr[i0 + r + 1] - j0);
        atomicOr(&s_bits[w][pos >> 5], 1u << (pos & 31));
    }
    __syncwarp();
    const int total = nrows + nnzt;
    const int d0 = min(lane * MERGE_WARP_IPT, total), d1 = min(d0 + MERGE_WARP_IPT, total);
    const int w0 = d0 >> 5, b0 = d0 & 31;
    int before = 0;
    for (int q = 0; q < w0; ++q) before += __popc(s_bits[w][q]);
    const uint32_t lo = s_bits[w][w0], hi = s_bits[w][w0 + 1];
    before += __popc(lo & ((1u << b0) - 1u));
    const uint32_t span = b0 ? (lo >> b0) | (hi << (32 - b0)) : lo;
    const uint32_t bits = span & ((1u << (d1 - d0)) - 1u);
    // bit 31 of lane 0: the tile's first row started in an earlier tile (its value is
    // completed by the carry fix-up)
    const uint32_t cont = (lane == 0 && nrows > 0 && row_ptr[i0] < j0) ? (1u << 31) : 0u;
    desc[t * 32 + lane] =
        (uint32_t)before | ((uint32_t)(d0 - before) << 8) | (bits << 16) | ((uint32_t)(d1 - d0) << 24) | cont;
}

// Lane-slotted layout of the warp tiles: one warp per tile writes the tile's header and
// lane descriptors (same fields as k_merge_desc) and, for every slot k * 32 + lane, the CRS
// index of the nonzero at path item k of the lane, or -1 for a row end or a tail slot.
// Slot values: none (pattern, or FP64 outside the double-float window), FP64 split into
// float pairs, FP32 or bfloat16 as stored.
enum SlotVals { SLOT_NONE = 0, SLOT_DF = 1, SLOT_F32 = 2, SLOT_BF16 = 3 };

__global__ void k_merge_slots(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ part_row,
                              const int32_t *__restrict__ part_nz, int64_t tiles, uint32_t *__restrict__ sdesc,
                              const int32_t *__restrict__ col, const void *__restrict__ val, int vals,
                              int32_t *__restrict__ scol, void *__restrict__ sval) {
    __shared__ uint32_t s_bits[8][8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t t = (int64_t)blockIdx.x * 8 + w;
    if (t >= tiles) return;
    const int64_t i0 = part_row[t], j0 = part_nz[t];
    const int nrows = (int)(part_row[t + 1] - i0), nnzt = (int)(part_nz[t + 1] - j0);
    if (lane < 8) s_bits[w][lane] = 0u;
    __syncwarp();
    for (int r = lane; r < nrows; r += 32) {
        const int pos = r + (int)(row_ptr[i0 + r + 1] - j0);
        atomicOr(&s_bits[w][pos >> 5], 1u << (pos & 31));
    }
    __syncwarp();
    const int total = nrows + nnzt;
    const int d0 = min(lane * MERGE_WARP_IPT, total), d1 = min(d0 + MERGE_WARP_IPT, total);
    const int w0 = d0 >> 5, b0 = d0 & 31;
    int before = 0;
    for (int q = 0; q < w0; ++q) before += __popc(s_bits[w][q]);
    const uint32_t lo = s_bits[w][w0], hi = s_bits[w][w0 + 1];
    before += __popc(lo & ((1u << b0) - 1u));
    const uint32_t span = b0 ? (lo >> b0) | (hi << (32 - b0)) : lo;
    const uint32_t bits = span & ((1u << (d1 - d0)) - 1u);
    uint32_t *hd = sdesc + t * SLOT_DESC_WORDS;
    hd[4 + lane] = (uint32_t)before | (bits << 16) | ((uint32_t)(d1 - d0) << 24);
    if (lane < 4) {
        const uint32_t cont = (nrows > 0 && row_ptr[i0] < j0) ? 1u : 0u;
        hd[lane] = lane == 0 ? (uint32_t)i0 : lane == 1 ? (uint32_t)nrows : lane == 2 ? cont : 0u;
        hd[36 + lane] = 0u;
    }
    // nonzero index of path item d0 + k: j0 + (d0 + k) - (row ends before it); a row end or a
    // tail slot holds column 0 and value 0
    int ends = before;
    const int64_t o = t * MERGE_WARP_ITEMS + lane;
#pragma unroll
    for (int k = 0; k < MERGE_WARP_IPT; ++k) {
        const bool in = k < d1 - d0;
        const bool end = in && ((bits >> k) & 1u);
        const bool nzk = in && !end;
        const int64_t j = j0 + d0 + k - ends;
        const int64_t q = o + k * 32;
        scol[q] = nzk ? col[j] : 0;
        if (vals == SLOT_DF) {
            float2 r = make_float2(0.f, 0.f);
            if (nzk) df_split(((const double *)val)[j], &r.x, &r.y);
            ((float2 *)sval)[q] = r;
        } else if (vals == SLOT_F32) {
            ((float *)sval)[q] = nzk ? ((const float *)val)[j] : 0.f;
        } else if (vals == SLOT_BF16) {
            ((__nv_bfloat16 *)sval)[q] = nzk ? ((const __nv_bfloat16 *)val)[j] : __float2bfloat16(0.f);
        }
        ends += end ? 1 : 0;
    }
}

// Static carry runs: the row in progress at the end of tile t is part_row[t + 1] (it is the
// tile's carry row), a run starts where that row changes, and its length comes from a
// bisection for the last tile ending in the same row (part_row is non-decreasing).
__global__ void k_fix_runs(const int32_t *__restrict__ part_row, int64_t tiles, int32_t *__restrict__ fix_len,
                           int32_t *__restrict__ fix_long, unsigned long long *__restrict__ nlong) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tiles) return;
    const int32_t r = part_row[t + 1];
    if (t > 0 && part_row[t] == r) {
        fix_len[t] = 0;
        return;
    }
    int64_t lo = t + 1, hi = tiles;   // largest j in [t+1, tiles] with part_row[j] == r
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (part_row[mid] <= r) lo = mid;
        else hi = mid - 1;
    }
    const int32_t len = (int32_t)(lo - t);
    fix_len[t] = len;
    if (len > FIX_SHORT) fix_long[atomicAdd(nlong, 1ull)] = (int32_t)t;
}

// Block of the first nonzero of each chunk of HB_CHUNK (largest b with blk_ptr[b] <= e);
// entry nchunks holds the last block.
__global__ void k_hb_chunks(const int32_t *__restrict__ blk_ptr, int64_t nblk, int64_t nnz, int64_t nchunks,
                            int32_t *__restrict__ chunk_blk) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > nchunks) return;
    if (c == nchunks) {
        chunk_blk[c] = (int32_t)(nblk - 1);
        return;
    }
    const int64_t e = c * HB_CHUNK;
    int64_t lo = 0, hi = nblk - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)blk_ptr[mid] <= e) lo = mid;
        else hi = mid - 1;
    }
    chunk_blk[c] = (int32_t)lo;
}

__global__ void k_merge_partition(const int32_t *__restrict__ row_ptr, int64_t m, int64_t nnz, int64_t tiles,
                                  int64_t tile_items, int32_t *__restrict__ part_row, int32_t *__restrict__ part_nz) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > tiles) return;
    int64_t d = min(t * tile_items, m + nnz);
    int64_t i = merge_split(d, m, nnz, row_ptr);
    part_row[t] = (int32_t)i;
    part_nz[t] = (int32_t)(d - i);
}

// ---------------------------------------------------------------- CRS -> HB
// Row of each CRS entry by bisection over row_ptr, bracketed per block.
constexpr int HB_KEY_TILE = 2048;

__device__ __forceinline__ int64_t row_of(const int32_t *__restrict__ row_ptr, int64_t lo, int64_t hi, int64_t k) {
    // largest r in [lo, hi] with row_ptr[r] <= k
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)row_ptr[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

constexpr int HB_KEY_ROWS = 2048;   // row_ptr slice kept in shared memory per block

// Row of the first CRS entry of every key tile (and of the last entry, at index ntiles), one
// bisection per thread, so that no key tile starts with a serial search.
__global__ void k_tile_rows(const int32_t *__restrict__ row_ptr, int64_t m, int64_t nnz, int64_t ntiles,
                            int64_t *__restrict__ tile_row) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ntiles) return;
    tile_row[c] = row_of(row_ptr, 0, m - 1, min(c * (int64_t)HB_KEY_TILE, nnz - 1));
}

// Hilbert key of every CRS entry (and its CRS position as the sort payload).  A thread takes
// HB_KEY_U consecutive entries: one bisection for the first one's row (over the tile's row_ptr
// slice in shared memory when it fits), then a forward walk for the others.
constexpr int HB_KEY_U = HB_KEY_TILE / CB;

__device__ __forceinline__ uint64_t hb_key(uint32_t r, uint32_t c, int K, int log2b, int inner, const uint16_t *fwd4) {
    if (inner == SPMV_INNER_ROWMAJOR) {
        const uint64_t blk = hilbert_key4(K - log2b, r >> log2b, c >> log2b, fwd4);
        const uint32_t mask = (1u << log2b) - 1u;
        return (blk << (2 * log2b)) | ((uint64_t)(r & mask) << log2b) | (uint64_t)(c & mask);
    }
    return hilbert_key4(K, r, c, fwd4);
}

__global__ void k_hb_keys(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int64_t m, int64_t nnz,
                          const int64_t *__restrict__ tile_row, int K, int log2b, int inner,
                          uint64_t *__restrict__ keys, uint32_t *__restrict__ perm) {
    __shared__ int32_t s_rp[HB_KEY_ROWS + 1];
    __shared__ __align__(16) uint16_t s_fwd4[1024];
    hilbert_stage(s_fwd4, g_hilbert4.fwd);
    const int64_t e0 = (int64_t)blockIdx.x * HB_KEY_TILE;
    const int64_t e1 = min(e0 + (int64_t)HB_KEY_TILE, nnz) - 1;
    const int64_t rlo = tile_row[blockIdx.x], rhi = tile_row[blockIdx.x + 1];   // rows of e0 and (at least) e1
    const bool in_smem = rhi - rlo + 1 <= HB_KEY_ROWS;
    if (in_smem)
        for (int64_t r = rlo + threadIdx.x; r <= rhi + 1 && r <= m; r += blockDim.x) s_rp[r - rlo] = row_ptr[r];
    __syncthreads();
    const int64_t k0 = e0 + (int64_t)threadIdx.x * HB_KEY_U;
    if (k0 > e1) return;
    // row of entry k0: largest r in [rlo, rhi] with row_ptr[r] <= k0
    int64_t r;
    if (in_smem) {
        int lo = 0, hi = (int)(rhi - rlo);
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((int64_t)s_rp[mid] <= k0) lo = mid;
            else hi = mid - 1;
        }
        r = rlo + lo;
    } else {
        r = row_of(row_ptr, rlo, rhi, k0);
    }
    auto next_start = [&](int64_t rr) -> int64_t {   // row_ptr[rr + 1]
        return in_smem ? (int64_t)s_rp[rr + 1 - rlo] : (int64_t)row_ptr[rr + 1];
    };
    int64_t rend = next_start(r);
    if (k0 + HB_KEY_U - 1 <= e1) {   // a full run: vector loads and stores
        const int4 cv0 = *(const int4 *)(col + k0), cv1 = *(const int4 *)(col + k0 + 4);
        const int32_t cc[HB_KEY_U] = {cv0.x, cv0.y, cv0.z, cv0.w, cv1.x, cv1.y, cv1.z, cv1.w};
        uint32_t rr[HB_KEY_U];
#pragma unroll
        for (int u = 0; u < HB_KEY_U; ++u) {
            const int64_t k = k0 + u;
            while (k >= rend) {   // entries of empty rows do not exist: walk to the row holding k
                ++r;
                rend = next_start(r);
            }
            rr[u] = (uint32_t)r;
        }
        uint64_t h[HB_KEY_U];   // the rows are known: the eight key chains run side by side
        if (inner == SPMV_INNER_ROWMAJOR) {
            const uint32_t mask = (1u << log2b) - 1u;
            uint32_t br[HB_KEY_U], bc[HB_KEY_U];
#pragma unroll
            for (int u = 0; u < HB_KEY_U; ++u) {
                br[u] = rr[u] >> log2b;
                bc[u] = (uint32_t)cc[u] >> log2b;
            }
            hilbert_key4_n<HB_KEY_U>(K - log2b, br, bc, s_fwd4, h);
#pragma unroll
            for (int u = 0; u < HB_KEY_U; ++u)
                h[u] = (h[u] << (2 * log2b)) | ((uint64_t)(rr[u] & mask) << log2b) | (uint64_t)((uint32_t)cc[u] & mask);
        } else {
            uint32_t cu[HB_KEY_U];
#pragma unroll
            for (int u = 0; u < HB_KEY_U; ++u) cu[u] = (uint32_t)cc[u];
            hilbert_key4_n<HB_KEY_U>(K, rr, cu, s_fwd4, h);
        }
        ulonglong2 *kd = (ulonglong2 *)(keys + k0);
#pragma unroll
        for (int u = 0; u < HB_KEY_U / 2; ++u) kd[u] = make_ulonglong2(h[2 * u], h[2 * u + 1]);
        const uint32_t p0 = (uint32_t)k0;
        ((uint4 *)(perm + k0))[0] = make_uint4(p0, p0 + 1, p0 + 2, p0 + 3);
        ((uint4 *)(perm + k0))[1] = make_uint4(p0 + 4, p0 + 5, p0 + 6, p0 + 7);
    } else {
        for (int64_t k = k0; k <= e1; ++k) {
            while (k >= rend) {
                ++r;
                rend = next_start(r);
            }
            keys[k] = hb_key((uint32_t)r, (uint32_t)col[k], K, log2b, inner, s_fwd4);
            perm[k] = (uint32_t)k;
        }
    }
}
static_assert(HB_KEY_U == 8, "two int4 column loads per run");

// Populate: packed in-block index, block-start flags.  Each thread decodes HB_FILL_U keys
// (elements i, i + T, ... for T threads) side by side.
constexpr int HB_FILL_U = 4;
__global__ void k_hb_fill(const uint64_t *__restrict__ keys, int64_t nnz, int K, int log2b, int inner,
                          uint32_t *__restrict__ idx, uint32_t *__restrict__ head) {
    __shared__ __align__(16) uint16_t s_inv4[1024];
    hilbert_stage(s_inv4, g_hilbert4.inv);
    __syncthreads();
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t mask = (1u << log2b) - 1u;
    uint64_t key[HB_FILL_U];
    uint32_t r[HB_FILL_U], c[HB_FILL_U];
#pragma unroll
    for (int u = 0; u < HB_FILL_U; ++u) {
        const int64_t t = t0 + u * T;
        key[u] = t < nnz ? keys[t] : 0ull;
    }
    if (inner == SPMV_INNER_ROWMAJOR) {   // block cell from the top levels, in-block cell as stored
        uint64_t bk[HB_FILL_U];
#pragma unroll
        for (int u = 0; u < HB_FILL_U; ++u) bk[u] = key[u] >> (2 * log2b);
        hilbert_cell4_n<HB_FILL_U>(K - log2b, bk, r, c, s_inv4);
#pragma unroll
        for (int u = 0; u < HB_FILL_U; ++u) {
            r[u] = (r[u] << log2b) | (uint32_t)((key[u] >> log2b) & mask);
            c[u] = (c[u] << log2b) | (uint32_t)(key[u] & mask);
        }
    } else {
        hilbert_cell4_n<HB_FILL_U>(K, key, r, c, s_inv4);
    }
#pragma unroll
    for (int u = 0; u < HB_FILL_U; ++u) {
        const int64_t t = t0 + u * T;
        if (t >= nnz) continue;
        idx[t] = ((r[u] & mask) << 16) | (c[u] & mask);
        head[t] = (t == 0 || (keys[t - 1] >> (2 * log2b)) != (key[u] >> (2 * log2b))) ? 1u : 0u;
    }
}

// Block table from the block-start entries (one per block; the cells are decoded with the
// one-level machine, no table staged).
__global__ void k_hb_blocks(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ head,
                            const uint32_t *__restrict__ bid, int64_t nnz, int K, int log2b, int inner,
                            int32_t *__restrict__ blk_ptr, int32_t *__restrict__ blk_row,
                            int32_t *__restrict__ blk_col) {
    (void)inner;
    const int64_t t0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;   // four flags per thread
    if (t0 >= nnz) return;
    uint32_t f[4];
    if (t0 + 3 < nnz) {
        const uint4 h4 = *(const uint4 *)(head + t0);
        f[0] = h4.x; f[1] = h4.y; f[2] = h4.z; f[3] = h4.w;
    } else {
        for (int u = 0; u < 4; ++u) f[u] = t0 + u < nnz ? head[t0 + u] : 0u;
    }
    for (int u = 0; u < 4; ++u) {
        if (!f[u]) continue;
        const int64_t t = t0 + u;
        // block coordinates: the top K - log2b levels of the key in either inner order (the
        // curve is hierarchical, so they are the block's own Hilbert index)
        uint32_t br, bc;
        hilbert_cell1(K - log2b, keys[t] >> (2 * log2b), &br, &bc);
        const uint32_t b = bid[t];
        blk_ptr[b] = (int32_t)t;
        blk_row[b] = (int32_t)br;
        blk_col[b] = (int32_t)bc;
    }
}

// ---------------------------------------------------------------- other block orders
// Keys of the block orders and inner orders besides the Hilbert-ordered HB above: blocks in
// row-major order (CSB and CSBH, Sections 3.1 and 4.1) or in Hilbert order with a Z-Morton
// inner order.  key = (block key << 2 lb) | in-block key, where the block key is the block's
// Hilbert index on the (K - lb)-order block grid or br * 2^(K - lb) + bc, and the in-block key
// is the Z-Morton index (row bit above the column bit at every level), the Hilbert index of
// the block's own curve of order lb, or the row-major cell index.

__device__ __forceinline__ uint32_t zm_spread(uint32_t v) {   // bits of v to the even positions
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
__device__ __forceinline__ uint32_t zm_gather(uint32_t v) {   // the even bits of v, packed
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0F0F0F0Fu;
    v = (v | (v >> 4)) & 0x00FF00FFu;
    v = (v | (v >> 8)) & 0x0000FFFFu;
    return v;
}

__device__ __forceinline__ uint64_t blk_key(uint32_t r, uint32_t c, int K, int lb, int border, int inner,
                                            const uint16_t *fwd4) {
    const uint32_t br = r >> lb, bc = c >> lb, mask = (1u << lb) - 1u, ri = r & mask, ci = c & mask;
    const uint64_t bk = border == SPMV_BLOCK_HILBERT ? hilbert_key4(K - lb, br, bc, fwd4)
                                                     : ((uint64_t)br << (K - lb)) | bc;
    uint64_t ik;
    if (inner == SPMV_INNER_ZMORTON) ik = ((uint64_t)zm_spread(ri) << 1) | zm_spread(ci);
    else if (inner == SPMV_INNER_HILBERT) ik = hilbert_key4(lb, ri, ci, fwd4);
    else ik = ((uint64_t)ri << lb) | ci;
    return (bk << (2 * lb)) | ik;
}

__device__ __forceinline__ void blk_cell(uint64_t key, int K, int lb, int border, int inner, uint32_t *br,
                                         uint32_t *bc, uint32_t *ri, uint32_t *ci) {
    const uint64_t bk = key >> (2 * lb), ik = key & ((1ull << (2 * lb)) - 1ull);
    if (border == SPMV_BLOCK_HILBERT) {
        hilbert_cell1(K - lb, bk, br, bc);
    } else {
        *br = (uint32_t)(bk >> (K - lb));
        *bc = (uint32_t)(bk & ((1ull << (K - lb)) - 1ull));
    }
    if (inner == SPMV_INNER_ZMORTON) {
        *ri = zm_gather((uint32_t)(ik >> 1));
        *ci = zm_gather((uint32_t)ik);
    } else if (inner == SPMV_INNER_HILBERT) {
        hilbert_cell1(lb, ik, ri, ci);
    } else {
        *ri = (uint32_t)(ik >> lb);
        *ci = (uint32_t)(ik & ((1ull << lb) - 1ull));
    }
}

// One thread per CRS entry; its row by bisection of row_ptr.
__global__ void k_blk_keys(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int64_t m,
                           int64_t nnz, int K, int lb, int border, int inner, uint64_t *__restrict__ keys,
                           uint32_t *__restrict__ perm) {
    __shared__ __align__(16) uint16_t s_fwd4[1024];
    hilbert_stage(s_fwd4, g_hilbert4.fwd);
    __syncthreads();
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    const int64_t r = row_of(row_ptr, 0, m - 1, k);
    keys[k] = blk_key((uint32_t)r, (uint32_t)col[k], K, lb, border, inner, s_fwd4);
    perm[k] = (uint32_t)k;
}

__global__ void k_blk_fill(const uint64_t *__restrict__ keys, int64_t nnz, int K, int lb, int border, int inner,
                           uint32_t *__restrict__ idx, uint32_t *__restrict__ head) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnz) return;
    uint32_t br, bc, ri, ci;
    blk_cell(keys[t], K, lb, border, inner, &br, &bc, &ri, &ci);
    idx[t] = (ri << 16) | ci;
    head[t] = (t == 0 || (keys[t - 1] >> (2 * lb)) != (keys[t] >> (2 * lb))) ? 1u : 0u;
}

__global__ void k_blk_blocks(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ head,
                             const uint32_t *__restrict__ bid, int64_t nnz, int K, int lb, int border, int inner,
                             int32_t *__restrict__ blk_ptr, int32_t *__restrict__ blk_row,
                             int32_t *__restrict__ blk_col) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnz || !head[t]) return;
    uint32_t br, bc, ri, ci;
    blk_cell(keys[t], K, lb, border, inner, &br, &bc, &ri, &ci);
    const uint32_t b = bid[t];
    blk_ptr[b] = (int32_t)t;
    blk_row[b] = (int32_t)br;
    blk_col[b] = (int32_t)bc;
}

__global__ void k_hilbert_keys(int K, int64_t n, const int32_t *__restrict__ rows, const int32_t *__restrict__ cols,
                               uint64_t *__restrict__ keys) {
    __shared__ __align__(16) uint16_t s_fwd4[1024], s_inv4[1024];
    hilbert_stage(s_fwd4, g_hilbert4.fwd);
    hilbert_stage(s_inv4, g_hilbert4.inv);
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const uint64_t h = hilbert_key4(K, (uint32_t)rows[i], (uint32_t)cols[i], s_fwd4);
        uint32_t r, c;
        hilbert_cell4(K, h, &r, &c, s_inv4);   // the inverse must return the cell
        keys[i] = (r == (uint32_t)rows[i] && c == (uint32_t)cols[i]) ? h : ~0ull;
    }
}

// ---------------------------------------------------------------- double-float window
__global__ void k_df_window(const double *__restrict__ v, int64_t n, uint32_t *__restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (; i < n; i += stride) {
        float h, l;
        bad |= !df_split(v[i], &h, &l);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// ---------------------------------------------------------------- helpers
spmv_status read_status(spmv_matrix *h, cudaStream_t s, uint32_t *out) {
    SPMV_CUDA_TRY(cudaMemcpyAsync(h->status_host, h->status_dev, 8, cudaMemcpyDeviceToHost, s));   // words 0 and 1
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    *out = *h->status_host;
    return SPMV_OK;
}

// Word 1 of the handle's status: set (ST_TIMEOUT) by a radix sort whose bounded waits gave
// up.  sort_begin zeroes it before a sort; sort_failed reads the host copy that the next
// synchronising read brought back.
spmv_status sort_begin(spmv_matrix *h, cudaStream_t s) {
    SPMV_CUDA_TRY(cudaMemsetAsync(h->status_dev + 1, 0, 4, s));
    return SPMV_OK;
}
spmv_status sort_fetch(spmv_matrix *h, cudaStream_t s) {
    SPMV_CUDA_TRY(cudaMemcpyAsync(h->status_host + 1, h->status_dev + 1, 4, cudaMemcpyDeviceToHost, s));
    return SPMV_OK;
}
bool sort_failed(const spmv_matrix *h) {
    if (!(h->status_host[1] & ST_TIMEOUT)) return false;
    set_error("spmv_convert: a bounded wait of the radix sort gave up");
    return true;
}

template <typename T>
void launch_gather(const void *src, const uint32_t *perm, int64_t n, void *dst, cudaStream_t s) {
    SPMV_LAUNCH("k_gather", s, (k_gather<T><<<grid_for(n, CB * GATHER_ILP), CB, 0, s>>>((const T *)src, perm, n, (T *)dst)));
}

spmv_status gather_values(const void *src, spmv_dtype dt, const uint32_t *perm, int64_t n, void *dst, cudaStream_t s) {
    switch (elem_size(dt)) {
        case 8: launch_gather<uint64_t>(src, perm, n, dst, s); break;
        case 4: launch_gather<uint32_t>(src, perm, n, dst, s); break;
        case 2: launch_gather<uint16_t>(src, perm, n, dst, s); break;
        default: return SPMV_OK;
    }
    SPMV_LAUNCH_CHECK("gather");
    return SPMV_OK;
}

spmv_status fill_row_ptr(const uint64_t *keys, int64_t nnz, int cbits, int64_t m, int32_t *row_ptr, cudaStream_t s,
                         int32_t *col = nullptr, uint32_t *status = nullptr) {
    DevBuf gaps(s), ngaps(s);
    int64_t cap = (m + 1) / GAP_INLINE + 2;
    SPMV_TRY(gaps.alloc((size_t)cap * 3 * sizeof(int64_t), "row_ptr gaps"));
    SPMV_TRY(ngaps.alloc(sizeof(unsigned long long), "row_ptr gap count"));
    SPMV_CUDA_TRY(cudaMemsetAsync(ngaps.p, 0, sizeof(unsigned long long), s));
    SPMV_LAUNCH("k_row_ptr_fill", s, (k_row_ptr_fill<<<grid_for((nnz + 1 + RPF_U - 1) / RPF_U), CB, 0, s>>>(keys, nnz, cbits, m, row_ptr, gaps.as<int64_t>(),
                                                    ngaps.as<unsigned long long>(), col, status)));
    SPMV_LAUNCH_CHECK("row_ptr fill");
    SPMV_LAUNCH("k_fill_gaps", s, (k_fill_gaps<<<1184, CB, 0, s>>>(gaps.as<int64_t>(), ngaps.as<unsigned long long>(), row_ptr)));
    SPMV_LAUNCH_CHECK("row_ptr gaps");
    return SPMV_OK;
}

}  // namespace

spmv_status launch_validate(const int32_t *row, const int32_t *col, int64_t nnz, int64_t m, int64_t n,
                            uint32_t *status, cudaStream_t s) {
    if (nnz <= 0) return SPMV_OK;
    SPMV_LAUNCH("k_validate", s, (k_validate<<<grid_for((nnz + 3) / 4, CB * 4), CB, 0, s>>>(row, col, nnz, m, n, status)));
    SPMV_LAUNCH_CHECK("validate");
    return SPMV_OK;
}

spmv_status launch_hilbert_keys(int K, int64_t n, const int32_t *rows, const int32_t *cols, uint64_t *keys,
                                cudaStream_t s) {
    if (n <= 0) return SPMV_OK;
    SPMV_LAUNCH("k_hilbert_keys", s, (k_hilbert_keys<<<grid_for(n), CB, 0, s>>>(K, n, rows, cols, keys)));
    SPMV_LAUNCH_CHECK("hilbert keys");
    return SPMV_OK;
}

spmv_status build_csr(spmv_matrix *h, cudaStream_t s) {
    const int64_t m = h->m, nnz = h->nnz_in;
    const int es = elem_size(h->dt);
    DevBuf row_ptr(s), col(s), val(s);
    SPMV_TRY(row_ptr.alloc((size_t)(m + 1) * 4 + TMA_PAD, "row_ptr"));
    int64_t nout = 0;
    if (nnz == 0) {
        SPMV_CUDA_TRY(cudaMemsetAsync(row_ptr.p, 0, (size_t)(m + 1) * 4, s));
    } else {
        const int cbits = bits_for(h->n), rbits = bits_for(h->m);
        DevBuf keys(s), keys_alt(s), perm(s), perm_alt(s), head(s), tmp(s);
        SPMV_TRY(keys.alloc((size_t)nnz * 8, "sort keys"));
        SPMV_TRY(keys_alt.alloc((size_t)nnz * 8, "sort keys"));
        SPMV_TRY(perm.alloc((size_t)nnz * 4, "sort perm"));
        SPMV_TRY(perm_alt.alloc((size_t)nnz * 4, "sort perm"));
        SPMV_TRY(tmp.alloc(std::max(radix_temp_bytes(nnz), scan_temp_bytes(nnz)), "sort temp"));
        SPMV_LAUNCH("k_coo_keys", s, (k_coo_keys<<<grid_for(nnz), CB, 0, s>>>(h->coo_row, h->coo_col, nnz, cbits, keys.as<uint64_t>(),
                                                perm.as<uint32_t>())));
        SPMV_LAUNCH_CHECK("coo keys");
        bool alt = false;
        SPMV_TRY(sort_begin(h, s));
        SPMV_TRY(radix_sort_pairs(keys.as<uint64_t>(), keys_alt.as<uint64_t>(), perm.as<uint32_t>(),
                                  perm_alt.as<uint32_t>(), nnz, 0, cbits + rbits, tmp.p, s, &alt, h->status_dev + 1));
        uint64_t *K = alt ? keys_alt.as<uint64_t>() : keys.as<uint64_t>();
        uint32_t *P = alt ? perm_alt.as<uint32_t>() : perm.as<uint32_t>();
        uint64_t *Kspare = alt ? keys.as<uint64_t>() : keys_alt.as<uint64_t>();
        uint32_t *Pspare = alt ? perm.as<uint32_t>() : perm_alt.as<uint32_t>();
        // finish assuming no duplicate keys: columns, row_ptr and the duplicate check in one pass
        SPMV_CUDA_TRY(cudaMemsetAsync(h->status_dev, 0, 4, s));
        SPMV_TRY(col.alloc((size_t)nnz * 4 + TMA_PAD, "col_ind"));
        SPMV_TRY(fill_row_ptr(K, nnz, cbits, m, row_ptr.as<int32_t>(), s, col.as<int32_t>(), h->status_dev));
        uint32_t stw = 0;
        SPMV_TRY(read_status(h, s, &stw));
        if (sort_failed(h)) return SPMV_ERR_TIMEOUT;
        if (stw & ST_DUPLICATE) {
            if (h->flags & SPMV_DUP_ERROR) {
                set_error("spmv_convert: duplicate (row, col) entries with SPMV_DUP_ERROR");
                return SPMV_ERR_DUPLICATE;
            }
            SPMV_TRY(head.alloc((size_t)nnz * 4, "heads"));
            SPMV_LAUNCH("k_heads", s, (k_heads<<<grid_for(nnz), CB, 0, s>>>(K, nnz, head.as<uint32_t>(), h->status_dev)));
            SPMV_LAUNCH_CHECK("heads");
            uint32_t *pos = Pspare;
            SPMV_TRY(exclusive_scan_u32(head.as<uint32_t>(), pos, nnz, tmp.p, s));
            uint32_t last[2] = {0, 0};
            SPMV_CUDA_TRY(cudaMemcpyAsync(&last[0], pos + nnz - 1, 4, cudaMemcpyDeviceToHost, s));
            SPMV_CUDA_TRY(cudaMemcpyAsync(&last[1], head.as<uint32_t>() + nnz - 1, 4, cudaMemcpyDeviceToHost, s));
            SPMV_CUDA_TRY(cudaStreamSynchronize(s));
            nout = (int64_t)last[0] + last[1];
            col.reset();
            SPMV_TRY(col.alloc((size_t)nout * 4 + TMA_PAD, "col_ind"));
            if (es) SPMV_TRY(val.alloc((size_t)nout * es + TMA_PAD, "values"));
            SPMV_LAUNCH("k_dup_compact", s, (k_dup_compact<<<grid_for(nnz), CB, 0, s>>>(K, P, head.as<uint32_t>(), pos, nnz, cbits,
                                                       es ? h->coo_val : nullptr, h->dt, Kspare,
                                                       col.as<int32_t>(), val.p)));
            SPMV_LAUNCH_CHECK("dup compact");
            SPMV_TRY(fill_row_ptr(Kspare, nout, cbits, m, row_ptr.as<int32_t>(), s));
        } else {
            nout = nnz;
            if (es) SPMV_TRY(val.alloc((size_t)nnz * es + TMA_PAD, "values"));
            if (es) SPMV_TRY(gather_values(h->coo_val, h->dt, P, nnz, val.p, s));
        }
    }
    h->row_ptr = (int32_t *)row_ptr.release();
    h->col = (int32_t *)col.release();
    h->val = val.release();
    h->nnz = nout;
    h->has_csr = true;
    h->bytes += (m + 1) * 4 + nout * (4 + es);
    // the triplet copy is no longer needed
    if (h->coo_row) dev_free_async(h->coo_row, s);
    if (h->coo_col) dev_free_async(h->coo_col, s);
    if (h->coo_val) dev_free_async(h->coo_val, s);
    if (nnz) h->bytes -= nnz * (8 + es);
    h->coo_row = h->coo_col = nullptr;
    h->coo_val = nullptr;
    return SPMV_OK;
}

spmv_status build_df(spmv_matrix *h, cudaStream_t s) {
    if (h->df_checked) return SPMV_OK;
    h->df_checked = true;
    h->df_ok = false;
    if (h->dt != SPMV_F64) return SPMV_OK;
    DevBuf xs(s), fl(s);
    SPMV_TRY(xs.alloc((size_t)std::max<int64_t>(h->n, 1) * sizeof(float2), "x split"));
    SPMV_TRY(fl.alloc(16, "x split flag"));
    SPMV_CUDA_TRY(cudaMemsetAsync(h->status_dev + 2, 0, 4, s));
    if (h->nnz > 0)
        SPMV_LAUNCH("k_df_window", s,
                    (k_df_window<<<grid_for(h->nnz, CB * 8), CB, 0, s>>>((const double *)h->val, h->nnz, h->status_dev + 2)));
    SPMV_LAUNCH_CHECK("df window");
    SPMV_CUDA_TRY(cudaMemcpyAsync(h->status_host + 2, h->status_dev + 2, 4, cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    h->df_ok = h->status_host[2] == 0;
    h->xsplit = (float2 *)xs.release();
    h->xsplit_flag = (uint32_t *)fl.release();
    h->bytes += std::max<int64_t>(h->n, 1) * 8 + 16;
    return SPMV_OK;
}

spmv_status build_bins(spmv_matrix *h, cudaStream_t s) {
    const int64_t m = h->m;
    for (int c = 0; c < 8; ++c) h->bin_count[c] = 0;
    h->max_row_len = 0;
    if (m == 0) {
        h->has_bins = true;
        return SPMV_OK;
    }
    DevBuf cls(s), cls_alt(s), rows(s), rows_alt(s), counts(s), tmp(s), bin_rows(s);
    SPMV_TRY(cls.alloc((size_t)m * 8, "row class"));
    SPMV_TRY(cls_alt.alloc((size_t)m * 8, "row class"));
    SPMV_TRY(rows.alloc((size_t)m * 4, "row ids"));
    SPMV_TRY(rows_alt.alloc((size_t)m * 4, "row ids"));
    SPMV_TRY(counts.alloc(16 * sizeof(unsigned long long), "class counts"));
    SPMV_TRY(tmp.alloc(radix_temp_bytes(m), "sort temp"));
    SPMV_TRY(bin_rows.alloc((size_t)m * 4, "bin rows"));
    SPMV_CUDA_TRY(cudaMemsetAsync(counts.p, 0, 16 * sizeof(unsigned long long), s));
    SPMV_LAUNCH("k_row_class", s, (k_row_class<<<(unsigned)std::min<int64_t>(grid_for(m), ROW_CLASS_GRID), CB, 0, s>>>(h->row_ptr, m, cls.as<uint64_t>(), rows.as<uint32_t>(),
                                           counts.as<unsigned long long>(), counts.as<unsigned long long>() + 8)));
    SPMV_LAUNCH_CHECK("row class");
    bool alt = false;
    SPMV_TRY(sort_begin(h, s));
    SPMV_TRY(radix_sort_pairs(cls.as<uint64_t>(), cls_alt.as<uint64_t>(), rows.as<uint32_t>(), rows_alt.as<uint32_t>(),
                              m, 0, 3, tmp.p, s, &alt, h->status_dev + 1));
    SPMV_CUDA_TRY(cudaMemcpyAsync(bin_rows.p, alt ? rows_alt.p : rows.p, (size_t)m * 4, cudaMemcpyDeviceToDevice, s));
    unsigned long long hc[16];
    SPMV_CUDA_TRY(cudaMemcpyAsync(hc, counts.p, sizeof(hc), cudaMemcpyDeviceToHost, s));
    SPMV_TRY(sort_fetch(h, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    if (sort_failed(h)) return SPMV_ERR_TIMEOUT;
    for (int c = 0; c < 8; ++c) h->bin_count[c] = (int64_t)hc[c];
    h->max_row_len = (int64_t)hc[8];
    if (h->bin_rows) dev_free_async(h->bin_rows, s);
    else h->bytes += m * 4;
    h->bin_rows = (int32_t *)bin_rows.release();
    h->has_bins = true;
    return SPMV_OK;
}

// Lane-slotted copy of the merge tiles: column indices, and the values (FP64 matrices inside
// the double-float window: split into float pairs; FP32 and bfloat16: as stored).
spmv_status build_slots(spmv_matrix *h, cudaStream_t s) {
    const int64_t tiles = h->tiles, slots = tiles * MERGE_WARP_ITEMS;
    if (h->dt == SPMV_F64) SPMV_TRY(build_df(h, s));
    const bool vals2 = h->dt == SPMV_F64 && h->df_ok;
    const size_t vbytes = h->dt == SPMV_F32 ? 4 : h->dt == SPMV_BF16 ? 2 : 0;
    const int mode = vals2 ? SLOT_DF : h->dt == SPMV_F32 ? SLOT_F32 : h->dt == SPMV_BF16 ? SLOT_BF16 : SLOT_NONE;
    DevBuf sd(s), sc(s), sv(s);
    SPMV_TRY(sd.alloc((size_t)tiles * SLOT_DESC_WORDS * 4, "slot descriptors"));
    SPMV_TRY(sc.alloc((size_t)slots * 4, "slot columns"));
    if (vals2) SPMV_TRY(sv.alloc((size_t)slots * sizeof(float2), "slot values"));
    else if (vbytes) SPMV_TRY(sv.alloc((size_t)slots * vbytes, "slot values"));
    SPMV_LAUNCH("k_merge_slots", s, (k_merge_slots<<<(unsigned)((tiles + 7) / 8), 256, 0, s>>>(
                                        h->row_ptr, h->part_row, h->part_nz, tiles, sd.as<uint32_t>(), h->col, h->val,
                                        mode, sc.as<int32_t>(), sv.p)));
    SPMV_LAUNCH_CHECK("merge slots");
    if (h->slot_desc) {
        dev_free_async(h->slot_desc, s); dev_free_async(h->slot_col, s);
        if (h->slot_val2) dev_free_async(h->slot_val2, s);
        if (h->slot_val) dev_free_async(h->slot_val, s);
    }
    h->slot_desc = (uint32_t *)sd.release();
    h->slot_col = (int32_t *)sc.release();
    h->slot_val2 = vals2 ? (float2 *)sv.release() : nullptr;
    h->slot_val = vbytes ? sv.release() : nullptr;
    h->bytes += tiles * SLOT_DESC_WORDS * 4 + slots * (4 + (vals2 ? 8 : 0) + (int64_t)vbytes);
    return SPMV_OK;
}

spmv_status build_fix_runs(spmv_matrix *h, const int32_t *part_row, int64_t tiles, int64_t old_tiles,
                           cudaStream_t s) {
    DevBuf fl(s), fg(s), cnt(s);
    SPMV_TRY(fl.alloc((size_t)tiles * 4, "carry runs"));
    SPMV_TRY(fg.alloc((size_t)tiles * 4, "long carry runs"));
    SPMV_TRY(cnt.alloc(16, "long run count"));
    SPMV_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, 8, s));
    SPMV_LAUNCH("k_fix_runs", s, (k_fix_runs<<<grid_for(tiles), CB, 0, s>>>(part_row, tiles, fl.as<int32_t>(),
                                                                           fg.as<int32_t>(),
                                                                           (unsigned long long *)cnt.p)));
    SPMV_LAUNCH_CHECK("carry runs");
    unsigned long long nlong = 0;
    SPMV_CUDA_TRY(cudaMemcpyAsync(&nlong, cnt.p, 8, cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    if (h->fix_len) {
        dev_free_async(h->fix_len, s);
        dev_free_async(h->fix_long, s);
        h->bytes -= old_tiles * 8;
    }
    h->fix_len = (int32_t *)fl.release();
    h->fix_long = (int32_t *)fg.release();
    h->fix_long_count = (int64_t)nlong;
    h->bytes += tiles * 8;
    return SPMV_OK;
}

spmv_status build_merge(spmv_matrix *h, int tile_items, cudaStream_t s) {
    const int64_t total = h->m + h->nnz;
    const int64_t tiles = std::max<int64_t>(1, (total + tile_items - 1) / tile_items);
    DevBuf pr(s), pn(s), cr(s), cv(s), ds(s);
    SPMV_TRY(ds.alloc((size_t)tiles * 32 * 4, "merge descriptors"));
    SPMV_TRY(pr.alloc((size_t)(tiles + 1) * 4, "merge partition"));
    SPMV_TRY(pn.alloc((size_t)(tiles + 1) * 4, "merge partition"));
    SPMV_TRY(cr.alloc((size_t)tiles * 4, "merge carries"));
    SPMV_TRY(cv.alloc((size_t)tiles * 16, "merge carries"));   // tile carries, then head partials
    SPMV_LAUNCH("k_merge_partition", s, (k_merge_partition<<<grid_for(tiles + 1), CB, 0, s>>>(h->row_ptr, h->m, h->nnz, tiles, tile_items,
                                                         pr.as<int32_t>(), pn.as<int32_t>())));
    SPMV_LAUNCH_CHECK("merge partition");
    SPMV_LAUNCH("k_merge_desc", s, (k_merge_desc<<<(unsigned)((tiles + 7) / 8), 256, 0, s>>>(
                                       h->row_ptr, pr.as<int32_t>(), pn.as<int32_t>(), tiles, ds.as<uint32_t>())));
    SPMV_LAUNCH_CHECK("merge descriptors");
    if (h->has_merge) {
        dev_free_async(h->part_row, s); dev_free_async(h->part_nz, s);
        dev_free_async(h->carry_row, s); dev_free_async(h->carry_val, s); dev_free_async(h->merge_desc, s);
        h->bytes -= (h->tiles + 1) * 8 + h->tiles * 20 + h->tiles * 128;
    }
    h->merge_desc = (uint32_t *)ds.release();
    h->part_row = (int32_t *)pr.release();
    h->part_nz = (int32_t *)pn.release();
    h->carry_row = (int32_t *)cr.release();
    h->carry_val = (double *)cv.release();
    const int64_t old_tiles = h->tiles;
    h->tiles = tiles;
    h->tile_items = tile_items;
    h->has_merge = true;
    h->bytes += (tiles + 1) * 8 + tiles * 20 + tiles * 128;
    const spmv_status fst = build_fix_runs(h, h->part_row, tiles, old_tiles, s);
    if (fst != SPMV_OK) {
        h->has_merge = false;
        return fst;
    }
    if (tile_items == MERGE_WARP_ITEMS) SPMV_TRY(build_slots(h, s));
    return SPMV_OK;
}

spmv_status hb_chunk_table(spmv_matrix *h, cudaStream_t s) {
    const int64_t nchunks = (h->nnz + HB_CHUNK - 1) / HB_CHUNK;
    DevBuf chk(s);
    SPMV_TRY(chk.alloc((size_t)(nchunks + 1) * 4, "hb chunk blocks"));
    if (h->nnz > 0) {
        SPMV_LAUNCH("k_hb_chunks", s, (k_hb_chunks<<<grid_for(nchunks + 1), CB, 0, s>>>(h->blk_ptr, h->nblk, h->nnz,
                                                                                     nchunks, chk.as<int32_t>())));
        SPMV_LAUNCH_CHECK("hb chunks");
    }
    if (h->hb_chunk_blk) dev_free_async(h->hb_chunk_blk, s);
    h->hb_chunk_blk = (int32_t *)chk.release();
    return SPMV_OK;
}

spmv_status build_hb(spmv_matrix *h, int log2b, int inner, cudaStream_t s, int border) {
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    const int es = elem_size(h->dt);
    const int K = bits_for(std::max<int64_t>(std::max(m, n), 2));
    if (log2b > K) log2b = K;
    DevBuf idx(s), val(s), bptr(s), brow(s), bcol(s);
    int64_t nblk = 0;
    if (nnz > 0) {
        DevBuf keys(s), keys_alt(s), perm(s), perm_alt(s), head(s), bid(s), tmp(s);
        SPMV_TRY(keys.alloc((size_t)nnz * 8, "hb keys"));
        SPMV_TRY(keys_alt.alloc((size_t)nnz * 8, "hb keys"));
        SPMV_TRY(perm.alloc((size_t)nnz * 4, "hb perm"));
        SPMV_TRY(perm_alt.alloc((size_t)nnz * 4, "hb perm"));
        SPMV_TRY(head.alloc((size_t)nnz * 4, "hb heads"));
        SPMV_TRY(bid.alloc((size_t)nnz * 4, "hb block ids"));
        SPMV_TRY(tmp.alloc(std::max(radix_temp_bytes(nnz), scan_temp_bytes(nnz)), "hb sort temp"));
        SPMV_TRY(idx.alloc((size_t)nnz * 4, "hb idx"));
        if (es) SPMV_TRY(val.alloc((size_t)nnz * es, "hb values"));
        const bool fast = border == SPMV_BLOCK_HILBERT && inner != SPMV_INNER_ZMORTON;   // the HB path
        if (fast) {
            const int64_t ktiles = (nnz + HB_KEY_TILE - 1) / HB_KEY_TILE;
            DevBuf trow(s);
            SPMV_TRY(trow.alloc((size_t)(ktiles + 1) * 8, "hb key tile rows"));
            SPMV_LAUNCH("k_tile_rows", s, (k_tile_rows<<<grid_for(ktiles + 1), CB, 0, s>>>(h->row_ptr, m, nnz, ktiles,
                                                                                         trow.as<int64_t>())));
            SPMV_LAUNCH_CHECK("hb key tile rows");
            SPMV_LAUNCH("k_hb_keys", s, (k_hb_keys<<<(unsigned)ktiles, CB, 0, s>>>(h->row_ptr, h->col, m, nnz,
                                                                                 trow.as<int64_t>(), K, log2b, inner,
                                                                                 keys.as<uint64_t>(), perm.as<uint32_t>())));
            SPMV_LAUNCH_CHECK("hb keys");
        } else {
            SPMV_LAUNCH("k_blk_keys", s, (k_blk_keys<<<grid_for(nnz), CB, 0, s>>>(h->row_ptr, h->col, m, nnz, K, log2b,
                                                                                border, inner, keys.as<uint64_t>(),
                                                                                perm.as<uint32_t>())));
            SPMV_LAUNCH_CHECK("blocked keys");
        }
        bool alt = false;
        SPMV_TRY(sort_begin(h, s));
        // A row-wise inner order is the CRS order restricted to a block, and the keys are made in
        // CRS order: a stable sort on the block key alone (bits 2 lb and up) yields the same order
        // as a sort on the whole key.
        const int begin_bit = inner == SPMV_INNER_ROWMAJOR ? 2 * log2b : 0;
        SPMV_TRY(radix_sort_pairs(keys.as<uint64_t>(), keys_alt.as<uint64_t>(), perm.as<uint32_t>(),
                                  perm_alt.as<uint32_t>(), nnz, begin_bit, 2 * K, tmp.p, s, &alt, h->status_dev + 1));
        uint64_t *Ks = alt ? keys_alt.as<uint64_t>() : keys.as<uint64_t>();
        uint32_t *Ps = alt ? perm_alt.as<uint32_t>() : perm.as<uint32_t>();
        if (fast)
            SPMV_LAUNCH("k_hb_fill", s, (k_hb_fill<<<grid_for((nnz + HB_FILL_U - 1) / HB_FILL_U), CB, 0, s>>>(Ks, nnz, K, log2b, inner, idx.as<uint32_t>(), head.as<uint32_t>())));
        else
            SPMV_LAUNCH("k_blk_fill", s, (k_blk_fill<<<grid_for(nnz), CB, 0, s>>>(Ks, nnz, K, log2b, border, inner,
                                                                                idx.as<uint32_t>(), head.as<uint32_t>())));
        SPMV_LAUNCH_CHECK("hb fill");
        if (es) SPMV_TRY(gather_values(h->val, h->dt, Ps, nnz, val.p, s));
        SPMV_TRY(exclusive_scan_u32(head.as<uint32_t>(), bid.as<uint32_t>(), nnz, tmp.p, s));
        uint32_t last[2] = {0, 0};
        SPMV_CUDA_TRY(cudaMemcpyAsync(&last[0], bid.as<uint32_t>() + nnz - 1, 4, cudaMemcpyDeviceToHost, s));
        SPMV_CUDA_TRY(cudaMemcpyAsync(&last[1], head.as<uint32_t>() + nnz - 1, 4, cudaMemcpyDeviceToHost, s));
        SPMV_TRY(sort_fetch(h, s));
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
        if (sort_failed(h)) return SPMV_ERR_TIMEOUT;
        nblk = (int64_t)last[0] + last[1];
        SPMV_TRY(bptr.alloc((size_t)(nblk + 1) * 4, "hb blk_ptr"));
        SPMV_TRY(brow.alloc((size_t)nblk * 4, "hb blk_row"));
        SPMV_TRY(bcol.alloc((size_t)nblk * 4, "hb blk_col"));
        if (fast)
            SPMV_LAUNCH("k_hb_blocks", s, (k_hb_blocks<<<grid_for((nnz + 3) / 4), CB, 0, s>>>(Ks, head.as<uint32_t>(), bid.as<uint32_t>(), nnz, K, log2b, inner,
                                                     bptr.as<int32_t>(), brow.as<int32_t>(), bcol.as<int32_t>())));
        else
            SPMV_LAUNCH("k_blk_blocks", s, (k_blk_blocks<<<grid_for(nnz), CB, 0, s>>>(Ks, head.as<uint32_t>(), bid.as<uint32_t>(), nnz, K,
                                                                                    log2b, border, inner, bptr.as<int32_t>(),
                                                                                    brow.as<int32_t>(), bcol.as<int32_t>())));
        SPMV_LAUNCH_CHECK("hb blocks");
        *h->status_host = (uint32_t)nnz;   // pinned staging slot for the tail entry
        SPMV_CUDA_TRY(cudaMemcpyAsync(bptr.as<int32_t>() + nblk, h->status_host, 4, cudaMemcpyHostToDevice, s));
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    } else {
        SPMV_TRY(bptr.alloc(4, "hb blk_ptr"));
        SPMV_CUDA_TRY(cudaMemsetAsync(bptr.p, 0, 4, s));
    }
    const int64_t nchunks = (nnz + HB_CHUNK - 1) / HB_CHUNK;
    DevBuf chk(s);
    SPMV_TRY(chk.alloc((size_t)(nchunks + 1) * 4, "hb chunk blocks"));
    if (nnz > 0) {
        SPMV_LAUNCH("k_hb_chunks", s, (k_hb_chunks<<<grid_for(nchunks + 1), CB, 0, s>>>(bptr.as<int32_t>(), nblk, nnz,
                                                                                     nchunks, chk.as<int32_t>())));
        SPMV_LAUNCH_CHECK("hb chunks");
    }
    free_mergeb(h, s);   // its tables index the blocked arrays being replaced
    if (h->has_hb) {
        dev_free_async(h->hb_idx, s); dev_free_async(h->hb_val, s); dev_free_async(h->blk_ptr, s);
        dev_free_async(h->blk_row, s); dev_free_async(h->blk_col, s); dev_free_async(h->hb_chunk_blk, s);
        h->bytes -= h->nnz * (4 + es) + h->nblk * 12 + 4 + ((h->nnz + HB_CHUNK - 1) / HB_CHUNK + 1) * 4;
    }
    h->hb_chunk_blk = (int32_t *)chk.release();
    h->hb_idx = (uint32_t *)idx.release();
    h->hb_val = val.release();
    h->blk_ptr = (int32_t *)bptr.release();
    h->blk_row = (int32_t *)brow.release();
    h->blk_col = (int32_t *)bcol.release();
    h->nblk = nblk;
    h->log2beta = log2b;
    h->grid_K = K;
    h->inner = inner;
    h->block_order = border;
    h->has_hb = true;
    h->bytes += nnz * (4 + es) + nblk * 12 + 4 + (nchunks + 1) * 4;
    return SPMV_OK;
}

}  // namespace spmv
