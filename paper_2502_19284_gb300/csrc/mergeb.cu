// Merge Blocking SpMV (Section 4.3: MergeB and MergeBH) on sm_103a.
//
// Storage.  The blocked arrays of the HB conversion in row-major block order (blk_ptr,
// blk_row, blk_col, packed in-block indices ((r mod beta) << 16 | (c mod beta)) and values;
// the entries of a block row-wise for MergeB, along the block's own Hilbert curve for
// MergeBH) plus the CRS pointer over the blocks: blk_row_ptr[i] is the first block of block
// row i (nbr + 1 entries).  Together they hold the block matrix in CRS, its nonzeros being
// the blocks, which is the storage Section 4.3 describes.
//
// Product.  Section 4.3 runs the merge-based product of Section 3.3 on the block matrix: the
// path merges the block-row ends with the blocks, consuming a block is its sparse block
// product and the temporary value becomes a temporary vector of beta rows.  A block is too
// coarse and too uneven a unit of work for a warp lane (R-MAT blocks hold from one to 10^5
// entries), so here the path merges the block-row ends with the entries of the blocks: every
// warp tile takes MB_ITEMS consecutive path items and each lane MB_IPT of them, so all lanes
// do the same amount of work whatever the sizes of the blocks.  The split points (the entry
// and the block at every lane's first item) come from the diagonal search of Section 3.3
// over (block-row ends, entries), done once at the conversion.  The temporary vector is y
// itself, kept in L2 while the warps walk a block row: a lane adds the sum of each run of its
// entries in one row to y with one reduction (y is zeroed first), so the carries between
// lanes and tiles need no fix-up pass.  Persistent warps load the next tile's entries into
// registers while they compute the current one; x is gathered from global memory.  Summation
// order across runs is not fixed (FP results within tolerance, integer results exact).
#include "common.cuh"
#include "convert.cuh"
#include "acc.cuh"

#include <algorithm>
#include <type_traits>

namespace spmv {

namespace {

constexpr int MB_IPT = 8;                        // path items per lane
constexpr int MB_ITEMS = 32 * MB_IPT;            // path items per warp tile
constexpr int MB_WARPS = 8;                      // warps (tiles) per CTA
#ifndef MB_MINB_CFG
#define MB_MINB_CFG 2
#endif
constexpr int MB_MINB = MB_MINB_CFG;             // resident CTAs per SM the registers are sized for
constexpr int MB_PAD = MB_ITEMS + MB_ITEMS / 8;  // staging slots: one spare slot per 8
constexpr int CB = 256;

inline unsigned grid_of(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + CB - 1) / CB); }

// ---------------------------------------------------------------- conversion

// ptr[i] = the first block whose block row is >= i (i = 0..nbr): the block rows after the
// previous block's row, up to block b's own row, start at block b.
__global__ void k_mb_rowptr(const int32_t *__restrict__ blk_row, int64_t nblk, int64_t nbr, int32_t *__restrict__ ptr) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nblk) return;
    const int64_t lo = b == 0 ? 0 : (int64_t)blk_row[b - 1] + 1;
    const int64_t hi = b == nblk ? nbr : (int64_t)blk_row[b];
    for (int64_t i = lo; i <= hi; ++i) ptr[i] = (int32_t)b;
}

// Split point of every lane's first path item (diagonal g * MB_IPT for lane g of the
// concatenated tiles): the diagonal search of Section 3.3 with A = the block-row ends counted
// in entries (block row i - 1 ends at blk_ptr[ptr[i]]) and B = the entries; a tie consumes
// the block-row end.  Stores the entry e reached and the block b holding it (the last block
// with blk_ptr[b] <= e; nblk once every entry is consumed).
__global__ void k_mb_desc(const int32_t *__restrict__ ptr, const int32_t *__restrict__ blk_ptr, int64_t nbr,
                          int64_t nblk, int64_t nnz, int64_t lanes, int2 *__restrict__ desc) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= lanes) return;
    const int64_t total = nbr + nnz;
    const int64_t d = min(g * MB_IPT, total);
    int64_t lo = d - nnz > 0 ? d - nnz : 0, hi = min(d, nbr);
    while (lo < hi) {   // the most block-row ends i that can precede diagonal d
        const int64_t i = lo + (hi - lo + 1) / 2;
        if ((int64_t)blk_ptr[ptr[i]] <= d - i) lo = i;
        else hi = i - 1;
    }
    const int64_t e = d - lo;
    int64_t bl = 0, bh = nblk;
    while (bl < bh) {
        const int64_t mid = bl + (bh - bl + 1) / 2;
        if ((int64_t)blk_ptr[mid] <= e) bl = mid;
        else bh = mid - 1;
    }
    desc[g] = make_int2((int)e, (int)bl);
}

// ---------------------------------------------------------------- product

// Add a run sum to y with one reduction in L2 (compensated FP32 sums are rounded first).
template <typename YT, typename Acc>
__device__ __forceinline__ void mb_red(YT *p, const Acc &a) {
    atomicAdd(p, a.template out<YT>());
}

// A warp tile's split points: this lane's (entry, block) and the entry where its items end,
// the tile's first entry and its entry count.  Loaded raw first, finished (shuffles) later.
struct MbRaw {
    int2 dc;
    int tail;   // lane 31: the first entry of the next tile (or nnz)
};
struct MbTile {
    int2 dc;
    int e1, te0, tn;
};
__device__ __forceinline__ MbRaw mb_load(const int2 *__restrict__ desc, int64_t t, int64_t ntiles, int64_t nnz,
                                         int lane) {
    MbRaw r;
    r.dc = desc[t * 32 + lane];
    r.tail = lane == 31 ? (t + 1 < ntiles ? desc[(t + 1) * 32].x : (int)nnz) : 0;
    return r;
}
__device__ __forceinline__ MbTile mb_finish(const MbRaw &r, int lane) {
    MbTile T;
    T.dc = r.dc;
    T.e1 = __shfl_down_sync(0xffffffffu, r.dc.x, 1);
    if (lane == 31) T.e1 = r.tail;
    T.te0 = __shfl_sync(0xffffffffu, r.dc.x, 0);
    // at most MB_ITEMS entries by the merge-path split (clamped, so that a damaged table can
    // never index past a staging slot)
    T.tn = max(0, min(__shfl_sync(0xffffffffu, T.e1, 31) - T.te0, MB_ITEMS));
    return T;
}

template <typename T>
__device__ __forceinline__ T ld_stream(const T *p) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        return __ushort_as_bfloat16(__ldcs(reinterpret_cast<const unsigned short *>(p)));
    } else {
        return __ldcs(p);
    }
}

// Persistent warps over the tiles w, w + W, ... (W warps in the grid).  While a tile is
// computed, the packed indices and values of the warp's next tile are already loaded into
// registers (lane-strided, streaming loads that do not displace x from L1) and the split
// points of the tile after it are on their way, so a tile's exposed latency is its x gathers;
// a warp that stays resident also never waits for its reductions to drain between tiles.  The
// tile's entries pass through the warp's shared slot (entry j at j + j / 8: a lane's 8
// consecutive entries fall on distinct banks).  VT: stored value type (Pattern: none);
// XT/YT: vector types.
template <typename Acc, typename VT, typename XT, typename YT>
__global__ __launch_bounds__(MB_WARPS * 32, MB_MINB) void k_mergeb(const int2 *__restrict__ desc,
                                                          const int32_t *__restrict__ blk_ptr,
                                                          const int32_t *__restrict__ blk_row,
                                                          const int32_t *__restrict__ blk_col,
                                                          const uint32_t *__restrict__ idx,
                                                          const VT *__restrict__ val, const XT *__restrict__ x,
                                                          YT *__restrict__ y, int64_t nblk, int64_t nnz,
                                                          int64_t ntiles, int64_t m, int64_t n, int lb,
                                                          uint32_t *__restrict__ err) {
    using Op = typename Acc::Op;
    constexpr bool PAT = std::is_same<VT, Pattern>::value;
    using VS = typename std::conditional<PAT, uint8_t, VT>::type;
    __shared__ uint32_t s_w[MB_WARPS][MB_PAD];
    __shared__ VS s_v[MB_WARPS][PAT ? 1 : MB_PAD];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * MB_WARPS;
    int64_t t = (int64_t)blockIdx.x * MB_WARPS + warp;
    if (t >= ntiles) return;   // whole warps
    uint32_t pw[MB_IPT];
    VS pv[MB_IPT];
    auto fetch = [&](const MbTile &T) {   // the tile's entries, lane-strided, into registers
#pragma unroll
        for (int k = 0; k < MB_IPT; ++k) {
            const int j = lane + 32 * k;
            if (j < T.tn) {
                pw[k] = __ldcs(idx + T.te0 + j);
                if constexpr (!PAT) pv[k] = ld_stream(val + T.te0 + j);
            }
        }
    };
    MbTile cur = mb_finish(mb_load(desc, t, ntiles, nnz, lane), lane);
    fetch(cur);
    bool more = t + W < ntiles;
    MbRaw rnext{};
    if (more) rnext = mb_load(desc, t + W, ntiles, nnz, lane);
    for (;;) {
#pragma unroll
        for (int k = 0; k < MB_IPT; ++k) {
            const int j = lane + 32 * k;
            if (j < cur.tn) {
                const int p = j + (j >> 3);
                s_w[warp][p] = pw[k];
                if constexpr (!PAT) s_v[warp][p] = pv[k];
            }
        }
        __syncwarp();
        MbTile nxt{};
        if (more) {
            nxt = mb_finish(rnext, lane);
            fetch(nxt);                                   // in flight while this tile is computed
            if (t + 2 * W < ntiles) rnext = mb_load(desc, t + 2 * W, ntiles, nnz, lane);
        }
        const int2 dc = cur.dc;
        const int ne = max(0, min(cur.e1 - dc.x, MB_IPT)), o0 = dc.x - cur.te0;
        int64_t b = dc.y, bend = 0, rbase = 0, cbase = 0;
        if (ne > 0) {
            bend = blk_ptr[b + 1];
            rbase = (int64_t)blk_row[b] << lb;
            cbase = (int64_t)blk_col[b] << lb;
        }
        int32_t row[MB_IPT];
        Op av[MB_IPT], xv[MB_IPT];
#pragma unroll
        for (int k = 0; k < MB_IPT; ++k) {
            row[k] = -1;
            av[k] = Op(0);
            xv[k] = Op(0);
            if (k < ne && o0 >= 0 && o0 + k < cur.tn) {
                if ((int64_t)dc.x + k >= bend && b + 1 < nblk) {
                    ++b;
                    bend = blk_ptr[b + 1];
                    rbase = (int64_t)blk_row[b] << lb;
                    cbase = (int64_t)blk_col[b] << lb;
                }
                const int p = o0 + k, ps = p + (p >> 3);
                const uint32_t w = s_w[warp][ps];
                const int64_t r = rbase + (w >> 16), c = cbase + (w & 0xFFFFu);
                if (r < m && c < n) {
                    row[k] = (int32_t)r;
                    xv[k] = ld_x<XT, Op>(x, c);
                    if constexpr (PAT) av[k] = Op(1);
                    else av[k] = sval<VT, Op>(s_v[warp], ps);
                } else {
                    atomicOr(err, ST_INDEX_RANGE);
                }
            }
        }
        Acc acc;
        acc.zero();
        int32_t cr = -1;
#pragma unroll
        for (int k = 0; k < MB_IPT; ++k) {
            if (row[k] < 0) continue;
            if (row[k] != cr) {
                if (cr >= 0) mb_red(y + cr, acc);
                acc.zero();
                cr = row[k];
            }
            acc.mad(av[k], xv[k]);
        }
        if (cr >= 0) mb_red(y + cr, acc);
        __syncwarp();
        if (!more) break;
        t += W;
        cur = nxt;
        more = t + W < ntiles;
    }
}

template <typename Acc, typename VT, typename XT, typename YT>
spmv_status mb_launch(const spmv_matrix *h, const void *x, void *y, cudaStream_t s) {
    constexpr size_t smem = 0;   // static slots
    int dev = 0, sms = 1, per = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mergeb<Acc, VT, XT, YT>, MB_WARPS * 32, smem) !=
            cudaSuccess)
        return cuda_status(cudaGetLastError(), "merge blocking grid");
    const int64_t tiles_ctas = (h->mb_tiles + MB_WARPS - 1) / MB_WARPS;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles_ctas, (int64_t)sms * std::max(per, 1)));
    SPMV_LAUNCH("k_mergeb", s, (k_mergeb<Acc, VT, XT, YT><<<grid, MB_WARPS * 32, smem, s>>>(
                                   h->mb_desc, h->blk_ptr, h->blk_row, h->blk_col, h->hb_idx, (const VT *)h->hb_val,
                                   (const XT *)x, (YT *)y, h->nblk, h->nnz, h->mb_tiles, h->m, h->n, h->log2beta,
                                   h->status_dev + 3)));
    SPMV_LAUNCH_CHECK("merge blocking spmv");
    return SPMV_OK;
}

template <typename Acc, typename XT, typename YT>
spmv_status mb_by_dtype(const spmv_matrix *h, const void *x, void *y, cudaStream_t s) {
    switch (h->dt) {
        case SPMV_F64: return mb_launch<Acc, double, XT, YT>(h, x, y, s);
        case SPMV_F32: return mb_launch<Acc, float, XT, YT>(h, x, y, s);
        case SPMV_BF16: return mb_launch<Acc, __nv_bfloat16, XT, YT>(h, x, y, s);
        default: return mb_launch<Acc, Pattern, XT, YT>(h, x, y, s);
    }
}

}  // namespace

void free_mergeb(spmv_matrix *h, cudaStream_t s) {
    if (!h->has_mergeb) return;
    dev_free_async(h->mb_row_ptr, s);
    dev_free_async(h->mb_desc, s);
    h->bytes -= (h->mb_nbr + 1) * 4 + h->mb_tiles * 32 * 8;
    h->mb_row_ptr = nullptr;
    h->mb_desc = nullptr;
    h->mb_nbr = 0;
    h->mb_tiles = 0;
    h->has_mergeb = false;
}

spmv_status build_mergeb(spmv_matrix *h, cudaStream_t s) {
    if (!h->has_hb || h->block_order != SPMV_BLOCK_ROWMAJOR) {
        set_error("spmv_convert: Merge Blocking needs the blocked arrays in row-major block order");
        return SPMV_ERR_INVALID_ARG;
    }
    free_mergeb(h, s);
    const int lb = h->log2beta;
    const int64_t nbr = h->m > 0 ? ((h->m - 1) >> lb) + 1 : 0;
    const int64_t ntiles = (nbr + h->nnz + MB_ITEMS - 1) / MB_ITEMS;
    DevBuf ptr(s), desc(s);
    SPMV_TRY(ptr.alloc((size_t)(nbr + 1) * 4, "merge blocking block-row pointer"));
    SPMV_LAUNCH("k_mb_rowptr", s, (k_mb_rowptr<<<grid_of(h->nblk + 1), CB, 0, s>>>(h->blk_row, h->nblk, nbr,
                                                                                  ptr.as<int32_t>())));
    SPMV_LAUNCH_CHECK("merge blocking block-row pointer");
    if (ntiles > 0) {
        SPMV_TRY(desc.alloc((size_t)ntiles * 32 * 8, "merge blocking lane split points"));
        SPMV_LAUNCH("k_mb_desc", s, (k_mb_desc<<<grid_of(ntiles * 32), CB, 0, s>>>(
                                         ptr.as<int32_t>(), h->blk_ptr, nbr, h->nblk, h->nnz, ntiles * 32,
                                         desc.as<int2>())));
        SPMV_LAUNCH_CHECK("merge blocking lane split points");
    }
    h->mb_row_ptr = (int32_t *)ptr.release();
    h->mb_desc = (int2 *)desc.release();
    h->mb_nbr = nbr;
    h->mb_tiles = ntiles;
    h->has_mergeb = true;
    h->bytes += (nbr + 1) * 4 + ntiles * 32 * 8;
    return SPMV_OK;
}

spmv_status mul_mergeb(const spmv_matrix *h, const void *x, void *y, spmv_dtype vdt, uint32_t acc, cudaStream_t s) {
    if (!h->has_mergeb) {
        set_error("spmv_mul: the Merge Blocking tables are missing (convert to MERGEB first)");
        return SPMV_ERR_NOT_CONVERTED;
    }
    const bool ok64 = vdt == SPMV_F64 && (acc == SPMV_ACC_DEFAULT || acc == SPMV_ACC_F64);
    const bool ok32 = vdt == SPMV_F32 && h->dt != SPMV_F64 &&
                      (acc == SPMV_ACC_DEFAULT || acc == SPMV_ACC_F32 || acc == SPMV_ACC_COMPENSATED);
    if (!ok64 && !ok32) {
        set_error("spmv_mul: Merge Blocking sums FP64 vectors in FP64 and FP32 vectors (FP32, bfloat16 or pattern "
                  "values) in plain or compensated FP32");
        return SPMV_ERR_UNSUPPORTED;
    }
    SPMV_CUDA_TRY(cudaMemsetAsync(y, 0, (size_t)h->m * (vdt == SPMV_F64 ? 8 : 4), s));
    if (h->mb_tiles == 0 || h->nnz == 0) return SPMV_OK;
    if (vdt == SPMV_F64) return mb_by_dtype<NativeAcc<double>, double, double>(h, x, y, s);
    if (acc == SPMV_ACC_COMPENSATED) return mb_by_dtype<CompAcc, float, float>(h, x, y, s);
    return mb_by_dtype<NativeAcc<float>, float, float>(h, x, y, s);
}

}  // namespace spmv
