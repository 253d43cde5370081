// SpMV products y := A x on sm_103a.
//
//   merge   Merge-based CRS SpMV (Section 3.3).  The path of row ends (A = row_ptr[1..m])
//           and nonzero indices (B = 0..nnz-1) is cut into equal CTA tiles by the
//           partition built at conversion.  Inside a tile: (1) products data[k]*x[col[k]]
//           are formed with coalesced loads into shared memory, row ends staged likewise;
//           (2) every thread walks an equal share of the tile's path (the same merge rule,
//           one level down), writing finished rows and keeping (row, temp) as its carry;
//           (3) thread carries are added to the row that finishes after them, in thread
//           order; the tile's trailing partial row becomes the tile carry; (4) the tile's
//           finished rows are stored coalesced.  A second kernel adds the tile carries in
//           tile order (Section 3.3 adds the per-thread carries sequentially afterwards).
//   rowsplit  CRS with rows grouped by length class (conversion), G lanes per row
//           (G = 1..32) or a whole CTA for long rows; lane-strided sums reduced by a
//           butterfly of warp shuffles.  GPU counterpart of the row-parallel ParCRS.
//   hb      Hilbert-ordered blocked format (Section 4.2): CTAs take equal ranges of the
//           Hilbert-sorted nonzeros; each entry's block is found in a shared-memory copy of
//           the range's block table, products are accumulated into y (zeroed first) with
//           global atomics.
//
// All three are memory-bound (about 0.17 flop per byte in FP64); none uses tensor cores.
#include "common.cuh"
#include "convert.cuh"
#include "df64.cuh"
#include "acc.cuh"
#include "tma.cuh"

#include <algorithm>
#include <mutex>

namespace spmv {

namespace {

inline unsigned cdivu(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// ================================================================ merge path
constexpr int MP_BLOCK = MERGE_BLOCK;

// Operand loaders: native (value converted to AT) or split into double-float pairs.
template <typename VT, typename AT>
struct NativeLoad {
    __device__ __forceinline__ static AT val(const VT *v, int64_t k) { return ld_val<VT, AT>(v, k); }
    template <typename XT> __device__ __forceinline__ static AT xg(const XT *x, int64_t j) { return ld_x<XT, AT>(x, j); }
};

// One merge-path tile (Section 3.3).  Only row ends and finished rows are staged in shared
// memory.  Each thread locates both ends of its share of the tile's path, loads the values
// and column indices of its contiguous nonzero range into registers, gathers x, and walks
// the range nonzero by nonzero (one multiply-add each), emitting every row end met on the
// way.  Carries: a run of threads ending in the same row forms one segment whose sum (in
// thread order) goes to the row finished right after the run, or becomes the tile's carry
// when the run is the tile's trailing partial row.  Runs of up to 8 threads (the common
// case) are summed sequentially by their last thread; only a tile holding a longer run (a
// row spanning many threads) uses a segmented scan.
template <typename Acc, typename Load, typename VT, typename XG, typename XT, int IPT>
__device__ __forceinline__ void merge_tile(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                           const VT *__restrict__ val, const XG *__restrict__ xg, XT *__restrict__ y,
                                           const int32_t *__restrict__ part_row, const int32_t *__restrict__ part_nz,
                                           int32_t *__restrict__ carry_row, double *__restrict__ carry_val,
                                           unsigned char *smem_raw) {
    using Op = typename Acc::Op;
    constexpr int TILE = MP_BLOCK * IPT;
    const int t = blockIdx.x;
    const int64_t i0 = part_row[t], j0 = part_nz[t];
    const int nrows = (int)(part_row[t + 1] - i0);
    const int nnzt = (int)(part_nz[t + 1] - j0);
    Acc *s_yl = (Acc *)smem_raw;                                   // TILE finished rows
    int32_t *s_rowend = (int32_t *)(s_yl + TILE);                  // TILE row ends (tile-relative)
    int32_t *s_crow = s_rowend + TILE;                             // thread carry rows + warp flags
    Acc *s_cval = (Acc *)(s_crow + MP_BLOCK + 32);                 // thread + warp sums
    for (int r = threadIdx.x; r < nrows; r += MP_BLOCK) s_rowend[r] = __ldg(row_ptr + i0 + r + 1) - (int32_t)j0;
    __syncthreads();

    const int total = nrows + nnzt;
    auto split = [&](int d) {   // row ends consumed on diagonal d of the tile's path
        int lo = max(0, d - nnzt), hi = min(d, nrows);
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (s_rowend[mid - 1] <= d - mid) lo = mid;
            else hi = mid - 1;
        }
        return lo;
    };
    const int d0 = min((int)threadIdx.x * IPT, total);
    const int d1 = min(d0 + IPT, total);
    int i = split(d0);
    const int iend = split(d1);
    const int jb = d0 - i, cnt = (d1 - iend) - jb;   // nonzeros [jb, jb + cnt) of the tile

    int32_t c[IPT];
    Op a[IPT], xv[IPT];
#pragma unroll
    for (int u = 0; u < IPT; ++u)
        if (u < cnt) {
            c[u] = __ldg(col + j0 + jb + u);
            a[u] = Load::val(val, j0 + jb + u);
        }
#pragma unroll
    for (int u = 0; u < IPT; ++u)
        if (u < cnt) xv[u] = Load::xg(xg, c[u]);
    Acc acc;
    acc.zero();
    int next_end = i < iend ? s_rowend[i] : 0x7fffffff;
#pragma unroll
    for (int u = 0; u < IPT; ++u) {
        if (u < cnt) {
            while (next_end <= jb + u) {   // row i ends before this nonzero
                s_yl[i] = acc;
                acc.zero();
                ++i;
                next_end = i < iend ? s_rowend[i] : 0x7fffffff;
            }
            acc.mad(a[u], xv[u]);
        }
    }
    while (i < iend) {   // rows ending after the last nonzero of this share
        s_yl[i] = acc;
        acc.zero();
        ++i;
    }
    s_crow[threadIdx.x] = i;
    s_cval[threadIdx.x] = acc;
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int myrow = i;
    const bool head = threadIdx.x == 0 || s_crow[threadIdx.x - 1] != myrow;
    const bool run_end = threadIdx.x == MP_BLOCK - 1 || s_crow[threadIdx.x + 1] != myrow;
    int run_start = threadIdx.x;
    if (run_end && !head) {
        int u = (int)threadIdx.x - 1;
        while (u > 0 && s_crow[u - 1] == myrow && (int)threadIdx.x - u < 8) --u;
        run_start = (u > 0 && s_crow[u - 1] == myrow) ? -1 : u;   // -1: run longer than 9
    }
    const bool long_run = __syncthreads_or(run_end && run_start < 0);
    Acc sv = acc;
    if (!long_run) {
        if (run_end && run_start < (int)threadIdx.x) {
            sv = s_cval[run_start];
            for (int u = run_start + 1; u <= (int)threadIdx.x; ++u) sv.add(s_cval[u]);
        }
    } else {
        bool f = head;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            if (__all_sync(0xffffffffu, f)) break;   // every lane has reached its segment head
            Acc ov = sv.shfl_up(o);
            const bool of = __shfl_up_sync(0xffffffffu, f, o);
            if (lane >= o) {
                if (!f) {
                    ov.add(sv);
                    sv = ov;
                }
                f = f || of;
            }
        }
        Acc *s_wsum = s_cval + MP_BLOCK;
        if (lane == 31) {
            s_wsum[warp] = sv;
            s_crow[MP_BLOCK + warp] = f ? 1 : 0;
        }
        __syncthreads();
        if (!f && warp > 0) {   // no head between this warp's start and this thread: carry-in
            Acc cin;
            cin.zero();
            for (int w = 0; w < warp; ++w) {
                if (s_crow[MP_BLOCK + w]) cin = s_wsum[w];
                else cin.add(s_wsum[w]);
            }
            cin.add(sv);
            sv = cin;
        }
    }
    if (run_end) {
        if (myrow < nrows) {
            sv.add(s_yl[myrow]);
            s_yl[myrow] = sv;
        } else {
            carry_row[t] = (int32_t)(i0 + nrows);
            carry_val[t] = sv.to_double();
        }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < nrows; r += MP_BLOCK) y[i0 + r] = s_yl[r].template out<XT>();
}

template <typename VT, typename XT, typename AT, int IPT>
__global__ __launch_bounds__(MP_BLOCK) void k_merge_spmv(const int32_t *__restrict__ row_ptr,
                                                         const int32_t *__restrict__ col, const VT *__restrict__ val,
                                                         const XT *__restrict__ x, XT *__restrict__ y,
                                                         const int32_t *__restrict__ part_row,
                                                         const int32_t *__restrict__ part_nz,
                                                         int32_t *__restrict__ carry_row, double *__restrict__ carry_val) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    merge_tile<NativeAcc<AT>, NativeLoad<VT, AT>, VT, XT, XT, IPT>(row_ptr, col, val, x, y, part_row, part_nz,
                                                                  carry_row, carry_val, smem_raw);
}

// ---------------------------------------------------------------- warp-tile merge path
// Each warp owns one tile of MW_ITEMS path items (Section 3.3's merge path cut into equal
// shares at the conversion) and runs independently of the other warps of its CTA: no block
// barrier, so one warp's memory latency never stalls another.  The tile's row ends, column
// indices and values are contiguous ranges of the CRS arrays; lane 0 brings them into the
// warp's shared-memory slot with 1-D TMA bulk copies (cp.async.bulk, completion counted on
// an mbarrier; source ranges widened to 16-byte boundaries, which the conversion's padding
// keeps inside the allocations).  Lanes then split the tile by the merge rule, gather x,
// accumulate their contiguous nonzero range, write every row they finish directly to y, and
// hold back only their first finished row, which may need the sum of the preceding lanes'
// carries (a segmented scan over lanes).  The last run of lanes becomes the tile's carry.

constexpr int MW_WARPS = 4;
constexpr int MW_IPT = MERGE_WARP_IPT;
constexpr int MW_ITEMS = 32 * MW_IPT;

// Widen the element range [e0, e1) of an array of `es`-byte elements to 16-byte boundaries:
// returns the first element copied and the byte count.
__device__ __forceinline__ void widen16(int64_t e0, int64_t e1, int es, int64_t *first, uint32_t *bytes) {
    const int64_t per = 16 / es;
    const int64_t a0 = e0 & ~(per - 1), a1 = (e1 + per - 1) & ~(per - 1);
    *first = a0;
    *bytes = e1 > e0 ? (uint32_t)((a1 - a0) * es) : 0u;
}


// Operand loaders from a tile slot (values as stored, x from the gather buffer).
template <typename VT, typename AT>
struct NativeSLoad {
    __device__ __forceinline__ static AT val(const VT *v, int k) { return sval<VT, AT>(v, k); }
    template <typename XT> __device__ __forceinline__ static AT xs(const XT *xb, int k) { return AT(xb[k]); }
};

// Shared-memory slot of one warp tile: mbarrier, lane descriptors, column indices, values,
// and the gathered x of the tile's nonzeros (reused for the finished rows once the lanes
// hold their operands in registers).
template <typename VT>
struct WarpSlot {
    static constexpr int DESC = 32;                                // uint32 per lane
    static constexpr int COL = MW_ITEMS + 8;                       // int32 column indices
    static constexpr int VAL = MW_ITEMS + 16;                      // values (VT)
    static constexpr int VAL_BYTES = std::is_same<VT, Pattern>::value ? 0 : ((VAL * (int)sizeof(VT) + 15) / 16) * 16;
    static constexpr int XB_BYTES = MW_ITEMS * 8;                  // gathered x, then finished rows
    static constexpr int OFF_DESC = 16, OFF_COL = OFF_DESC + DESC * 4, OFF_VAL = OFF_COL + COL * 4,
                         OFF_XB = OFF_VAL + VAL_BYTES;
    static constexpr int BYTES = OFF_XB + XB_BYTES;
};

__device__ __forceinline__ void cp_async_gather(void *dst, const void *src, uint64_t pol, int bytes) {
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 8, %2;" :: "r"(smem_u32(dst)), "l"(src),
                     "l"(pol) : "memory");
    else
        asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, %2;" :: "r"(smem_u32(dst)), "l"(src),
                     "l"(pol) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// Bulk copies of one warp tile into a slot (lane 0): descriptors, column indices, values.
// Completion is counted on the slot's mbarrier.
template <typename VT>
__device__ __forceinline__ void merge_warp_issue(const uint32_t *__restrict__ desc, const int32_t *__restrict__ col,
                                                 const VT *__restrict__ val, int64_t t, int64_t j0, int nnzt,
                                                 unsigned char *slot, uint64_t pol) {
    using Slot = WarpSlot<VT>;
    uint64_t *bar = (uint64_t *)slot;
    int64_t col_first, val_first = j0;
    uint32_t col_bytes, val_bytes = 0;
    widen16(j0, j0 + nnzt, 4, &col_first, &col_bytes);
    if constexpr (Slot::VAL_BYTES > 0) widen16(j0, j0 + nnzt, (int)sizeof(VT), &val_first, &val_bytes);
    const uint32_t total = 128u + col_bytes + val_bytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(total) : "memory");
    tma_load_1d(slot + Slot::OFF_DESC, desc + t * 32, 128u, bar, pol);
    if (col_bytes) tma_load_1d(slot + Slot::OFF_COL, col + col_first, col_bytes, bar, pol);
    if constexpr (Slot::VAL_BYTES > 0)
        if (val_bytes) tma_load_1d(slot + Slot::OFF_VAL, val + val_first, val_bytes, bar, pol);
}

// Lane descriptor fields (see k_merge_desc in the conversion).
__device__ __forceinline__ int desc_row(uint32_t d) { return (int)(d & 0xFFu); }
__device__ __forceinline__ int desc_nz(uint32_t d) { return (int)((d >> 8) & 0xFFu); }
__device__ __forceinline__ uint32_t desc_bits(uint32_t d) { return (d >> 16) & 0x7Fu; }
__device__ __forceinline__ int desc_items(uint32_t d) { return (int)(d >> 24); }

// Issue this lane's asynchronous gathers of x for its nonzeros of the tile in `slot`.
template <typename VT, typename XG>
__device__ __forceinline__ void merge_warp_gather(uint32_t d, int64_t j0, const XG *__restrict__ xg,
                                                  unsigned char *slot, uint64_t keep_pol) {
    using Slot = WarpSlot<VT>;
    const int32_t *s_col = (const int32_t *)(slot + Slot::OFF_COL);
    XG *xb = (XG *)(slot + Slot::OFF_XB);
    const int col_off = (int)(j0 & 3), jb = desc_nz(d), items = desc_items(d);
    const uint32_t bits = desc_bits(d);
#pragma unroll
    for (int k = 0; k < MW_IPT; ++k) {
        if (k < items && !((bits >> k) & 1u)) {
            const int jn = jb + k - __popc(bits & ((1u << k) - 1u));
            cp_async_gather(xb + jn, xg + s_col[col_off + jn], keep_pol, (int)sizeof(XG));
        }
    }
    cp_async_commit();
}

// Compute one warp tile whose operands are in `slot` (x already gathered).
template <typename Acc, typename Load, typename VT, typename XG, typename XT>
__device__ __forceinline__ void merge_warp_compute(uint32_t d, int64_t t, int64_t i0, int64_t j0, int nrows,
                                                   XT *__restrict__ y, int32_t *__restrict__ carry_row,
                                                   double *__restrict__ carry_val, double *__restrict__ head_val,
                                                   unsigned char *slot) {
    using Op = typename Acc::Op;
    using Slot = WarpSlot<VT>;
    const int lane = threadIdx.x & 31;
    const VT *s_val = (const VT *)(slot + Slot::OFF_VAL);
    const XG *xb = (const XG *)(slot + Slot::OFF_XB);
    Acc *s_rows = (Acc *)(slot + Slot::OFF_XB);
    const int perv = 16 / (int)(Slot::VAL_BYTES > 0 ? sizeof(VT) : 16);
    const int val_off = (int)(j0 & (perv - 1));
    const int istart = desc_row(d), jb = desc_nz(d), items = desc_items(d);
    const uint32_t bits = desc_bits(d);
    const int iend = istart + __popc(bits);
    Op a[MW_IPT], xv[MW_IPT];
#pragma unroll
    for (int k = 0; k < MW_IPT; ++k) {
        if (k < items && !((bits >> k) & 1u)) {
            const int jn = jb + k - __popc(bits & ((1u << k) - 1u));
            a[k] = Load::val(s_val, val_off + jn);
            xv[k] = Load::xs(xb, jn);
        }
    }
    __syncwarp();   // the x buffer becomes the finished-row buffer
    Acc acc;
    acc.zero();
    int i = istart;
#pragma unroll
    for (int k = 0; k < MW_IPT; ++k) {
        if (k < items) {
            if ((bits >> k) & 1u) {   // row i ends here: stash it
                s_rows[i] = acc;
                acc.zero();
                ++i;
            } else {
                acc.mad(a[k], xv[k]);
            }
        }
    }
    // segmented inclusive scan of the lanes' trailing partial sums (segments: equal end rows)
    const int prev_end = __shfl_up_sync(0xffffffffu, iend, 1);
    const bool head = lane == 0 || prev_end != iend;
    Acc sv = acc;
    bool f = head;
    if (!__all_sync(0xffffffffu, head)) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            if (__all_sync(0xffffffffu, f)) break;   // every lane has reached its segment head
            Acc ov = sv.shfl_up(o);
            const bool of = __shfl_up_sync(0xffffffffu, f, o);
            if (lane >= o) {
                if (!f) {
                    ov.add(sv);
                    sv = ov;
                }
                f = f || of;
            }
        }
    }
    // lane l's first finished row takes the run sum of the lanes ending in that row (the
    // run that ends at lane l-1), added before the lane's own part
    const Acc cin = sv.shfl_up(1);
    __syncwarp();
    if (lane > 0 && istart < iend) {
        Acc v = cin;
        v.add(s_rows[istart]);
        s_rows[istart] = v;
    }
    if (lane == 31) {
        carry_row[t] = (int32_t)(i0 + nrows);
        carry_val[t] = sv.to_double();
    }
    __syncwarp();
    // a first row that began in an earlier tile is completed by the fix-up: park its partial
    const bool cont = (__shfl_sync(0xffffffffu, d, 0) >> 31) != 0u;
    if (cont && lane == 0 && nrows > 0) head_val[t] = s_rows[0].to_double();
    for (int r = (cont ? 1 : 0) + lane; r < nrows; r += 32) y[i0 + r] = s_rows[r].template out<XT>();
}

// Persistent warp over tiles w, w + W, w + 2W, ... with two slots: while tile k is computed,
// the gathers of x for tile k+1 (asynchronous copies into its slot) and the bulk copies of
// tile k+2 are in flight.
template <typename Acc, typename Load, typename VT, typename XG, typename XT>
__device__ __forceinline__ void merge_warp_run(int64_t ntiles, const uint32_t *__restrict__ desc,
                                               const int32_t *__restrict__ col, const VT *__restrict__ val,
                                               const XG *__restrict__ xg, XT *__restrict__ y,
                                               const int32_t *__restrict__ part_row,
                                               const int32_t *__restrict__ part_nz, int32_t *__restrict__ carry_row,
                                               double *__restrict__ carry_val, uint32_t *__restrict__ err,
                                               unsigned char *wslots) {
    using Slot = WarpSlot<VT>;
    const int lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * MW_WARPS;
    const int64_t w = (int64_t)blockIdx.x * MW_WARPS + (threadIdx.x >> 5);
    if (w >= ntiles) return;
    auto slot = [&](int i) { return wslots + i * Slot::BYTES; };
    auto bar = [&](int i) { return (uint64_t *)(wslots + i * Slot::BYTES); };
    const uint64_t stream_pol = l2_policy_evict_first(), keep_pol = l2_policy_evict_last();
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(bar(0))) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(bar(1))) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    auto part = [&](int64_t tt, int64_t &i0, int64_t &j0, int &nr, int &nz) {
        i0 = part_row[tt];
        j0 = part_nz[tt];
        nr = (int)(part_row[tt + 1] - i0);
        nz = (int)(part_nz[tt + 1] - j0);
    };
    int64_t t = w;
    int64_t ci0, cj0, ni0 = 0, nj0 = 0;
    int cnr, cnz, nnr = 0, nnz_ = 0;
    part(t, ci0, cj0, cnr, cnz);
    if (lane == 0) merge_warp_issue<VT>(desc, col, val, t, cj0, cnz, slot(0), stream_pol);
    if (!mbar_wait(bar(0), 0u)) {
        if (lane == 0) atomicOr(err, ST_TIMEOUT);
        return;
    }
    uint32_t dcur = ((const uint32_t *)(slot(0) + Slot::OFF_DESC))[lane];
    merge_warp_gather<VT, XG>(dcur, cj0, xg, slot(0), keep_pol);
    if (t + W < ntiles) {
        part(t + W, ni0, nj0, nnr, nnz_);
        if (lane == 0) merge_warp_issue<VT>(desc, col, val, t + W, nj0, nnz_, slot(1), stream_pol);
    }
    for (int64_t k = 0; t < ntiles; ++k, t += W) {
        const int cs = (int)(k & 1), ns = cs ^ 1;
        const bool has_next = t + W < ntiles;
        uint32_t dnxt = 0;
        if (has_next) {   // the next tile's copies have landed: start its gathers
            if (!mbar_wait(bar(ns), (uint32_t)(((k + 1) >> 1) & 1))) {
                if (lane == 0) atomicOr(err, ST_TIMEOUT);
                cp_async_wait<0>();
                return;
            }
            dnxt = ((const uint32_t *)(slot(ns) + Slot::OFF_DESC))[lane];
            merge_warp_gather<VT, XG>(dnxt, nj0, xg, slot(ns), keep_pol);
            cp_async_wait<1>();   // this lane's gathers of tile t are complete
        } else {
            cp_async_wait<0>();
        }
        merge_warp_compute<Acc, Load, VT, XG, XT>(dcur, t, ci0, cj0, cnr, y, carry_row, carry_val, carry_val + ntiles,
                                                  slot(cs));
        __syncwarp();   // slot cs is free
        int64_t fi0 = 0, fj0 = 0;
        int fnr = 0, fnz = 0;
        if (t + 2 * W < ntiles) {
            part(t + 2 * W, fi0, fj0, fnr, fnz);
            if (lane == 0) merge_warp_issue<VT>(desc, col, val, t + 2 * W, fj0, fnz, slot(cs), stream_pol);
        }
        dcur = dnxt;
        ci0 = ni0; cj0 = nj0; cnr = nnr; cnz = nnz_;
        ni0 = fi0; nj0 = fj0; nnr = fnr; nnz_ = fnz;
    }
}

template <typename VT, typename XT, typename AT>
__global__ __launch_bounds__(MW_WARPS * 32) void k_merge_warp(const uint32_t *__restrict__ desc,
                                                              const int32_t *__restrict__ col,
                                                              const VT *__restrict__ val, const XT *__restrict__ x,
                                                              XT *__restrict__ y, const int32_t *__restrict__ part_row,
                                                              const int32_t *__restrict__ part_nz,
                                                              int32_t *__restrict__ carry_row,
                                                              double *__restrict__ carry_val, int64_t ntiles,
                                                              uint32_t *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    merge_warp_run<NativeAcc<AT>, NativeSLoad<VT, AT>, VT, XT, XT>(ntiles, desc, col, val, x, y, part_row, part_nz,
                                                                  carry_row, carry_val, err,
                                                                  smem_raw + (threadIdx.x >> 5) * 2 * WarpSlot<VT>::BYTES);
}

// FP32 or bfloat16 values with FP32 vectors, compensated FP32 accumulation (Acc = CompAcc
// everywhere, or SegAcc: compensated in the segmented reduction only).
template <typename VT, typename Acc>
__global__ __launch_bounds__(MW_WARPS * 32) void k_merge_warp_comp(const uint32_t *__restrict__ desc,
                                                                   const int32_t *__restrict__ col,
                                                                   const VT *__restrict__ val,
                                                                   const float *__restrict__ x, float *__restrict__ y,
                                                                   const int32_t *__restrict__ part_row,
                                                                   const int32_t *__restrict__ part_nz,
                                                                   int32_t *__restrict__ carry_row,
                                                                   double *__restrict__ carry_val, int64_t ntiles,
                                                                   uint32_t *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    merge_warp_run<Acc, NativeSLoad<VT, float>, VT, float, float>(ntiles, desc, col, val, x, y, part_row, part_nz,
                                                                     carry_row, carry_val, err,
                                                                     smem_raw + (threadIdx.x >> 5) * 2 * WarpSlot<VT>::BYTES);
}

// ---------------------------------------------------------------- lane-slotted warp tiles
// Merge-path product on the lane-slotted copy of the tiles (build_slots): path item k of
// lane l sits in slot k * 32 + l, so every operand of a lane is at a fixed offset and the
// shared memory accesses of a warp are contiguous.  A row end or tail slot holds value 0 and
// is neither gathered nor accumulated.  Stored values SV: FP64 split into float pairs at the
// conversion (float2), FP32, bfloat16, or none (pattern).  The gathers of x go straight into
// registers; once a lane holds its values in registers, the value area (grown to the row
// buffer's size where that is larger) takes the tile's finished rows.
#ifndef SLOT_CTAS_CFG
#define SLOT_CTAS_CFG 6
#endif
template <typename SV, typename Acc>
struct SlotT {
    static constexpr int OFF_HDR = 16;                                   // after the mbarrier
    static constexpr int OFF_COL = OFF_HDR + SLOT_DESC_WORDS * 4;
    static constexpr int OFF_VAL = OFF_COL + MW_ITEMS * 4;               // values, then finished rows
    static constexpr int VAL_BYTES = std::is_same<SV, Pattern>::value ? 0 : MW_ITEMS * (int)sizeof(SV);
    static constexpr int ROW_BYTES = MW_ITEMS * (int)sizeof(Acc);
    static constexpr int BYTES = OFF_VAL + ((VAL_BYTES > ROW_BYTES ? VAL_BYTES : ROW_BYTES) + 15) / 16 * 16;
    static constexpr uint32_t TX = SLOT_DESC_WORDS * 4 + MW_ITEMS * 4 + VAL_BYTES;   // bytes brought by TMA
    static_assert(OFF_VAL % 16 == 0 && OFF_COL % 16 == 0 && VAL_BYTES % 16 == 0, "16-byte bulk copies");
};

// Operand from a stored value: double-float pairs as they are, or rebuilt as an FP64 value
// (|a - hi - lo| <= 2^-48 |a|) when x is outside the double-float window; other types
// converted to the accumulator's operand type.
template <typename Acc, typename SV>
__device__ __forceinline__ typename Acc::Op slot_a(const SV *sv, int k) {
    using Op = typename Acc::Op;
    if constexpr (std::is_same<SV, float2>::value) {
        if constexpr (std::is_same<Op, float2>::value) return sv[k];
        else return (double)sv[k].x + (double)sv[k].y;
    } else if constexpr (std::is_same<Op, float2>::value) {   // pattern through double-float
        return make_float2(1.f, 0.f);
    } else {
        return sval<SV, Op>(sv, k);
    }
}

// read-only gathers with an L2 policy
__device__ __forceinline__ float ldg_hint(const float *p, uint64_t pol) {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float2 ldg_hint(const float2 *p, uint64_t pol) {
    float2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double ldg_hint(const double *p, uint64_t pol) {
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}

template <typename Slot, typename SV>
__device__ __forceinline__ void slot_issue(const uint32_t *__restrict__ sdesc, const int32_t *__restrict__ scol,
                                           const SV *__restrict__ sval, int64_t t, unsigned char *slot, uint64_t pol) {
    uint64_t *bar = (uint64_t *)slot;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(Slot::TX)
                 : "memory");
    tma_load_1d(slot + Slot::OFF_HDR, sdesc + t * SLOT_DESC_WORDS, SLOT_DESC_WORDS * 4, bar, pol);
    tma_load_1d(slot + Slot::OFF_COL, scol + t * MW_ITEMS, MW_ITEMS * 4, bar, pol);
    if constexpr (Slot::VAL_BYTES > 0) tma_load_1d(slot + Slot::OFF_VAL, sval + t * MW_ITEMS, Slot::VAL_BYTES, bar, pol);
}

// nonzero items of a lane descriptor: not a row end and inside the lane's item count
__device__ __forceinline__ uint32_t slot_nz(uint32_t d) { return ~(d >> 16) & ((1u << ((d >> 24) & 7u)) - 1u); }

template <typename Slot, typename XG>
__device__ __forceinline__ void slot_gather(const unsigned char *slot, const XG *__restrict__ xg, uint64_t pol,
                                            XG (&xr)[MW_IPT]) {
    const int lane = threadIdx.x & 31;
    const uint32_t nz = slot_nz(((const uint32_t *)(slot + Slot::OFF_HDR))[4 + lane]);
    const int32_t *sc = (const int32_t *)(slot + Slot::OFF_COL) + lane;
#pragma unroll
    for (int k = 0; k < MW_IPT; ++k) {
        xr[k] = XG{};
        if ((nz >> k) & 1u) xr[k] = ldg_hint(xg + sc[k * 32], pol);
    }
}

template <typename Slot, typename Acc, typename SV, typename XG, typename YT>
__device__ __forceinline__ void slot_compute(int64_t t, unsigned char *slot, const XG (&xr)[MW_IPT],
                                             YT *__restrict__ y, int32_t *__restrict__ carry_row,
                                             double *__restrict__ carry_val, double *__restrict__ head_val) {
    using Op = typename Acc::Op;
    const int lane = threadIdx.x & 31;
    const uint32_t *hd = (const uint32_t *)(slot + Slot::OFF_HDR);
    const uint32_t d = hd[4 + lane];
    const int64_t i0 = (int32_t)hd[0];
    const int nrows = (int)hd[1];
    const bool cont = hd[2] != 0u;
    const int istart = (int)(d & 0xFFu);
    const uint32_t bits = (d >> 16) & 0x7Fu, nz = slot_nz(d);
    const SV *sv = (const SV *)(slot + Slot::OFF_VAL) + lane;
    Op a[MW_IPT];
#pragma unroll
    for (int k = 0; k < MW_IPT; ++k) a[k] = slot_a<Acc, SV>(sv, k * 32);
    __syncwarp();   // the value area becomes the finished-row buffer
    Acc *s_rows = (Acc *)(slot + Slot::OFF_VAL);
    Acc acc;
    acc.zero();
    int i = istart;
#pragma unroll
    for (int k = 0; k < MW_IPT; ++k) {
        if ((nz >> k) & 1u) {
            acc.mad(a[k], Op(xr[k]));
        } else if ((bits >> k) & 1u) {   // row i ends here: stash it
            s_rows[i] = acc;
            acc.zero();
            ++i;
        }
    }
    // segmented inclusive scan of the lanes' trailing partial sums (segments: equal end rows)
    const int iend = istart + __popc(bits);
    const int prev_end = __shfl_up_sync(0xffffffffu, iend, 1);
    const bool head = lane == 0 || prev_end != iend;
    Acc run = acc;
    bool f = head;
    if (!__all_sync(0xffffffffu, head)) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            if (__all_sync(0xffffffffu, f)) break;   // every lane has reached its segment head
            Acc ov = run.shfl_up(o);
            const bool of = __shfl_up_sync(0xffffffffu, f, o);
            if (lane >= o) {
                if (!f) {
                    ov.add(run);
                    run = ov;
                }
                f = f || of;
            }
        }
    }
    // a lane's first finished row takes the run of the lanes before it that end in that row
    const Acc cin = run.shfl_up(1);
    __syncwarp();
    if (lane > 0 && istart < iend) {
        Acc v = cin;
        v.add(s_rows[istart]);
        s_rows[istart] = v;
    }
    __syncwarp();
    // lane 31: the tile's carry; lane 0: the partial of a first row begun in an earlier tile
    if (lane == 31 || (lane == 0 && cont && nrows > 0)) {
        const double dv = (lane == 31 ? run : s_rows[0]).to_double();
        if (lane == 31) {
            carry_row[t] = (int32_t)(i0 + nrows);
            carry_val[t] = dv;
        } else {
            head_val[t] = dv;
        }
    }
    for (int r = (cont ? 1 : 0) + lane; r < nrows; r += 32) y[i0 + r] = s_rows[r].template out<YT>();
}

// Persistent warp over tiles w, w + W, ... with two slots and two register sets: while tile
// k is computed from slot k % 2 and register set k % 2, the gathers of tile k+1 are in
// flight into the other register set and the bulk copies of tile k+2 are issued into slot
// k % 2 as soon as it is free.
constexpr int SLOT_STAGES = 2;

template <typename Slot, typename Acc, typename SV, typename XG, typename YT>
__device__ __forceinline__ bool slot_step(int64_t t, int64_t W, int64_t ntiles, int cs, uint32_t &parity,
                                          unsigned char *wslots, const uint32_t *__restrict__ sdesc,
                                          const int32_t *__restrict__ scol, const SV *__restrict__ sval,
                                          const XG *__restrict__ xg, YT *__restrict__ y,
                                          int32_t *__restrict__ carry_row, double *__restrict__ carry_val,
                                          uint32_t *__restrict__ err, const XG (&xcur)[MW_IPT], XG (&xnext)[MW_IPT],
                                          uint64_t stream_pol, uint64_t keep_pol) {
    const int lane = threadIdx.x & 31;
    const int ns = cs ^ 1;
    unsigned char *cur = wslots + cs * Slot::BYTES, *nxt = wslots + ns * Slot::BYTES;
    if (t + W < ntiles) {   // the next tile's copies have landed: start its gathers
        if (!mbar_wait((uint64_t *)nxt, (parity >> ns) & 1u)) {
            if (lane == 0) atomicOr(err, ST_TIMEOUT);
            return false;
        }
        parity ^= 1u << ns;
        slot_gather<Slot, XG>(nxt, xg, keep_pol, xnext);
    }
    slot_compute<Slot, Acc, SV, XG, YT>(t, cur, xcur, y, carry_row, carry_val, carry_val + ntiles);
    // the finished rows were written through the generic proxy: order them before the
    // bulk copy that refills the slot
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0 && t + SLOT_STAGES * W < ntiles) slot_issue<Slot, SV>(sdesc, scol, sval, t + SLOT_STAGES * W, cur, stream_pol);
    return true;
}

template <int NW, typename Acc, typename SV, typename XG, typename YT>
__device__ __forceinline__ void slot_run(int64_t ntiles, const uint32_t *__restrict__ sdesc,
                                         const int32_t *__restrict__ scol, const SV *__restrict__ sval,
                                         const XG *__restrict__ xg, YT *__restrict__ y,
                                         int32_t *__restrict__ carry_row, double *__restrict__ carry_val,
                                         uint32_t *__restrict__ err, unsigned char *wslots) {
    using Slot = SlotT<SV, Acc>;
    const int lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * NW;
    int64_t t = (int64_t)blockIdx.x * NW + (threadIdx.x >> 5);
    if (t >= ntiles) return;
    auto slot = [&](int i) { return wslots + i * Slot::BYTES; };
    auto bar = [&](int i) { return (uint64_t *)(wslots + i * Slot::BYTES); };
    const uint64_t stream_pol = l2_policy_evict_first(), keep_pol = l2_policy_evict_last();
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < SLOT_STAGES; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(bar(i))) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
#pragma unroll
        for (int i = 0; i < SLOT_STAGES; ++i)
            if (t + i * W < ntiles) slot_issue<Slot, SV>(sdesc, scol, sval, t + i * W, slot(i), stream_pol);
    }
    __syncwarp();
    uint32_t parity = 0;   // bit i: phase parity of the next completion of slot i
    if (!mbar_wait(bar(0), 0u)) {
        if (lane == 0) atomicOr(err, ST_TIMEOUT);
        return;
    }
    parity ^= 1u;
    XG xa[MW_IPT], xb[MW_IPT];
    slot_gather<Slot, XG>(slot(0), xg, keep_pol, xa);
    for (;;) {
        if (!slot_step<Slot, Acc, SV, XG, YT>(t, W, ntiles, 0, parity, wslots, sdesc, scol, sval, xg, y, carry_row,
                                              carry_val, err, xa, xb, stream_pol, keep_pol))
            return;
        t += W;
        if (t >= ntiles) return;
        if (!slot_step<Slot, Acc, SV, XG, YT>(t, W, ntiles, 1, parity, wslots, sdesc, scol, sval, xg, y, carry_row,
                                              carry_val, err, xb, xa, stream_pol, keep_pol))
            return;
        t += W;
        if (t >= ntiles) return;
    }
}

// SLOT_WARPS warps per CTA, SLOT_CTAS CTAs per SM: enough warps to cover the latencies,
// and a carveout that leaves the rest of the SM's on-chip memory to the L1 cache, which
// holds the gathers in flight and the frequently used x entries (measured on R-MAT scale
// 22: 381 us with 60-92 KB of L1 against 524 us with 28 KB).
constexpr int SLOT_WARPS = 4;
constexpr int SLOT_CTAS = SLOT_CTAS_CFG;
template <typename SV, typename Acc>
constexpr size_t slot_smem() { return (size_t)SLOT_WARPS * SLOT_STAGES * SlotT<SV, Acc>::BYTES; }

// FP64 vector through double-float: x2 holds x split per product; *xflag non-zero (some x
// outside the window) switches to native FP64 on x with the values rebuilt from their pairs.
// SV = float2 (split FP64 values) or Pattern.
template <typename SV>
__global__ __launch_bounds__(SLOT_WARPS * 32) void k_merge_slot_df(const uint32_t *__restrict__ sdesc,
                                                                   const int32_t *__restrict__ scol,
                                                                   const SV *__restrict__ sval2,
                                                                   const double *__restrict__ x,
                                                                   const float2 *__restrict__ x2,
                                                                   const uint32_t *__restrict__ xflag,
                                                                   double *__restrict__ y,
                                                                   int32_t *__restrict__ carry_row,
                                                                   double *__restrict__ carry_val, int64_t ntiles,
                                                                   uint32_t *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    static_assert(SlotT<SV, DfAcc>::BYTES == SlotT<SV, NativeAcc<double>>::BYTES, "one slot size for both forms");
    unsigned char *ws = smem_raw + (threadIdx.x >> 5) * SLOT_STAGES * SlotT<SV, DfAcc>::BYTES;
    if (*xflag == 0u)
        slot_run<SLOT_WARPS, DfAcc, SV, float2, double>(ntiles, sdesc, scol, sval2, x2, y, carry_row, carry_val, err,
                                                        ws);
    else
        slot_run<SLOT_WARPS, NativeAcc<double>, SV, double, double>(ntiles, sdesc, scol, sval2, x, y, carry_row,
                                                                    carry_val, err, ws);
}

// FP32 vectors: FP32, bfloat16 or pattern values with any accumulator (FP32, compensated,
// compensated in the segmented reduction only, or FP64).
template <typename SV, typename Acc>
__global__ __launch_bounds__(SLOT_WARPS * 32) void k_merge_slot(const uint32_t *__restrict__ sdesc,
                                                                const int32_t *__restrict__ scol,
                                                                const SV *__restrict__ sval,
                                                                const float *__restrict__ x, float *__restrict__ y,
                                                                int32_t *__restrict__ carry_row,
                                                                double *__restrict__ carry_val, int64_t ntiles,
                                                                uint32_t *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *ws = smem_raw + (threadIdx.x >> 5) * SLOT_STAGES * SlotT<SV, Acc>::BYTES;
    slot_run<SLOT_WARPS, Acc, SV, float, float>(ntiles, sdesc, scol, sval, x, y, carry_row, carry_val, err, ws);
}

// Pattern matrix (every stored value 1) with an FP64 vector through double-float: the value
// operand is the constant pair (1, 0).
struct DfPatLoad {
    __device__ __forceinline__ static float2 val(const Pattern *, int) { return make_float2(1.f, 0.f); }
    __device__ __forceinline__ static float2 xs(const float2 *xb, int k) { return xb[k]; }
};

__global__ __launch_bounds__(MW_WARPS * 32) void k_merge_warp_pat_df(const uint32_t *__restrict__ desc,
                                                                     const int32_t *__restrict__ col,
                                                                     const double *__restrict__ x,
                                                                     const float2 *__restrict__ x2,
                                                                     const uint32_t *__restrict__ xflag,
                                                                     double *__restrict__ y,
                                                                     const int32_t *__restrict__ part_row,
                                                                     const int32_t *__restrict__ part_nz,
                                                                     int32_t *__restrict__ carry_row,
                                                                     double *__restrict__ carry_val, int64_t ntiles,
                                                                     uint32_t *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *ws = smem_raw + (threadIdx.x >> 5) * 2 * WarpSlot<Pattern>::BYTES;
    if (*xflag == 0u)
        merge_warp_run<DfAcc, DfPatLoad, Pattern, float2, double>(ntiles, desc, col, nullptr, x2, y, part_row, part_nz,
                                                                  carry_row, carry_val, err, ws);
    else
        merge_warp_run<NativeAcc<double>, NativeSLoad<Pattern, double>, Pattern, double, double>(
            ntiles, desc, col, nullptr, x, y, part_row, part_nz, carry_row, carry_val, err, ws);
}

// x -> (hi, lo) float pairs; flags values outside the double-float window.
// Two entries per thread (one 16-byte load, one 16-byte store) when x is 16-byte aligned.
__global__ void k_df_split_x(const double *__restrict__ x, int64_t n, float2 *__restrict__ x2, uint32_t *flag) {
    const int64_t i = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    bool bad = false;
    if (i + 1 < n && ((reinterpret_cast<uintptr_t>(x) & 15u) == 0u)) {
        const double2 v = *reinterpret_cast<const double2 *>(x + i);
        float4 r;
        bad = !df_split(v.x, &r.x, &r.y);
        bad |= !df_split(v.y, &r.z, &r.w);
        *reinterpret_cast<float4 *>(x2 + i) = r;
    } else {
        for (int64_t j = i; j < i + 2 && j < n; ++j) {
            float2 r;
            bad |= !df_split(x[j], &r.x, &r.y);
            x2[j] = r;
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// The same split, and y := 0 over m entries, in one launch (for products that zero y first).
__global__ void k_df_split_x_zero(const double *__restrict__ x, int64_t n, float2 *__restrict__ x2, uint32_t *flag,
                                  double *__restrict__ y, int64_t m) {
    const int64_t i = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    bool bad = false;
    if (i + 1 < n && ((reinterpret_cast<uintptr_t>(x) & 15u) == 0u)) {
        const double2 v = *reinterpret_cast<const double2 *>(x + i);
        float4 r;
        bad = !df_split(v.x, &r.x, &r.y);
        bad |= !df_split(v.y, &r.z, &r.w);
        *reinterpret_cast<float4 *>(x2 + i) = r;
    } else {
        for (int64_t j = i; j < i + 2 && j < n; ++j) {
            float2 r;
            bad |= !df_split(x[j], &r.x, &r.y);
            x2[j] = r;
        }
    }
    if (i + 1 < m && ((reinterpret_cast<uintptr_t>(y) & 15u) == 0u)) {
        *reinterpret_cast<double2 *>(y + i) = make_double2(0.0, 0.0);
    } else {
        for (int64_t j = i; j < i + 2 && j < m; ++j) y[j] = 0.0;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

// Tile carries, added in tile order: the first tile of each run of equal carry rows sums
// the run and adds it to y[row] (which the finishing tile has already written).
template <typename XT>
__global__ void k_merge_fixup(int64_t tiles, int64_t m, const int32_t *__restrict__ carry_row,
                              const double *__restrict__ carry_val, XT *__restrict__ y) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tiles) return;
    const int32_t row = carry_row[t];
    if (t > 0 && carry_row[t - 1] == row) return;
    double s = carry_val[t];
    for (int64_t u = t + 1; u < tiles && carry_row[u] == row; ++u) s = s + carry_val[u];
    if (row < m) y[row] = XT((double)y[row] + s);
}

// Persistent grid: resident CTAs on every SM (occupancy from the runtime), never more
// warps than tiles.
inline unsigned persistent_grid(const void *kernel, int block, size_t smem, int64_t tiles) {
    int dev = 0, sms = 1;   // the current device's SM count (a process may drive several GPUs)
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || sms <= 0) {
        cudaGetLastError();
        sms = 1;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int64_t want = (tiles + MW_WARPS - 1) / MW_WARPS;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * per_sm));
}

// Carry fix-up of the warp tiles.  A run is a maximal sequence of tiles that end inside
// one row r (their carry row); the tile after the run finishes r.  If that tile marked r as
// begun earlier, it parked r's partial instead of writing y[r]: y[r] = run sum + partial
// (one rounding to the output type); otherwise the run's carries are all zero and y[r]
// stays as written.  The run structure is static (conversion); short runs are summed in
// tile order by one thread, long ones by a warp (lane-strided partial sums, then a fixed
// shuffle tree), so every result is the same from call to call.
struct spmv_matrix_view {   // what the fix-up kernels read of a handle
    int64_t m, tiles, fix_long_count;
    const uint32_t *desc;
    const int32_t *carry_row, *fix_len, *fix_long;
    const double *carry_val;
};
inline spmv_matrix_view view_of(const spmv_matrix *h) {
    return {h->m, h->tiles, h->fix_long_count, h->merge_desc, h->carry_row, h->fix_len, h->fix_long, h->carry_val};
}

template <typename XT>
__device__ __forceinline__ void fix_finish(const spmv_matrix_view &v, int64_t u, int32_t row, double sum, XT *y) {
    if (row >= v.m || u >= v.tiles) return;
    if (v.desc[u * 32] >> 31) y[row] = XT(sum + v.carry_val[v.tiles + u]);
    else if (sum != 0.0) y[row] = XT((double)y[row] + sum);
}

template <typename XT>
__global__ void k_fix_short(spmv_matrix_view v, XT *__restrict__ y) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= v.tiles) return;
    const int len = v.fix_len[t];
    if (len == 0 || len > FIX_SHORT) return;
    double s = v.carry_val[t];
    for (int k = 1; k < len; ++k) s = s + v.carry_val[t + k];
    fix_finish<XT>(v, t + len, v.carry_row[t], s, y);
}

template <typename XT>
__global__ void k_fix_long(spmv_matrix_view v, XT *__restrict__ y) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= v.fix_long_count) return;
    const int64_t t0 = v.fix_long[w];
    const int len = v.fix_len[t0];
    double s = 0.0;
    for (int k = lane; k < len; k += 32) s = s + v.carry_val[t0 + k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = s + __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) fix_finish<XT>(v, t0 + len, v.carry_row[t0], s, y);
}

template <typename XT>
spmv_status launch_fixup(const spmv_matrix *h, XT *y, cudaStream_t s) {
    const spmv_matrix_view v = view_of(h);
    SPMV_LAUNCH("k_merge_fixup", s, (k_fix_short<XT><<<cdivu(h->tiles, 256), 256, 0, s>>>(v, y)));
    SPMV_LAUNCH_CHECK("merge fixup");
    if (h->fix_long_count > 0) {
        SPMV_LAUNCH("k_merge_fixup_long", s, (k_fix_long<XT><<<cdivu(h->fix_long_count * 32, 256), 256, 0, s>>>(v, y)));
        SPMV_LAUNCH_CHECK("merge fixup long");
    }
    return SPMV_OK;
}

template <typename Acc>
constexpr size_t merge_smem(int ipt) {
    return (size_t)MP_BLOCK * ipt * (sizeof(Acc) + 4) + (MP_BLOCK + 32) * 4 + (MP_BLOCK + 32) * sizeof(Acc);
}

// Slotted product for FP32 vectors (values FP32, bfloat16 or pattern).
template <typename SV, typename Acc>
spmv_status launch_slot(const spmv_matrix *h, const void *x, void *y, cudaStream_t s) {
    constexpr size_t smem = slot_smem<SV, Acc>();
    static DeviceOnce attr;
    SPMV_TRY(attr([&] { return set_smem_ctas((const void *)k_merge_slot<SV, Acc>, smem, SLOT_CTAS); }));
    const unsigned grid = persistent_grid((const void *)k_merge_slot<SV, Acc>, SLOT_WARPS * 32, smem, h->tiles);
    SPMV_LAUNCH("k_merge_slot", s, (k_merge_slot<SV, Acc><<<grid, SLOT_WARPS * 32, smem, s>>>(
                                       h->slot_desc, h->slot_col, (const SV *)h->slot_val, (const float *)x, (float *)y,
                                       h->carry_row, h->carry_val, h->tiles, h->status_dev + 3)));
    SPMV_LAUNCH_CHECK("merge spmv");
    SPMV_TRY(launch_fixup<float>(h, (float *)y, s));
    return SPMV_OK;
}

// the slotted copy holds this matrix's values (or it needs none)
template <typename VT>
bool has_slot_vals(const spmv_matrix *h) {
    return h->slot_desc && (std::is_same<VT, Pattern>::value || h->slot_val);
}

template <typename VT, typename XT, typename AT, int IPT>
spmv_status launch_merge(const spmv_matrix *h, const void *x, void *y, bool allow_df, cudaStream_t s) {
    constexpr bool FP64 = std::is_same<VT, double>::value && std::is_same<XT, double>::value &&
                          std::is_same<AT, double>::value;
    constexpr size_t smem = (size_t)MW_WARPS * 2 * WarpSlot<VT>::BYTES;
    if constexpr (FP64) {
        if (allow_df && h->df_ok && h->xsplit && h->slot_val2) {
            constexpr size_t ssmem = slot_smem<float2, DfAcc>();
            static DeviceOnce attr;
            SPMV_TRY(attr([&] { return set_smem_ctas((const void *)k_merge_slot_df<float2>, ssmem, SLOT_CTAS); }));
            const unsigned grid = persistent_grid((const void *)k_merge_slot_df<float2>, SLOT_WARPS * 32, ssmem, h->tiles);
            SPMV_CUDA_TRY(cudaMemsetAsync(h->xsplit_flag, 0, 4, s));
            if (h->n > 0) {
                SPMV_LAUNCH("k_df_split_x", s,
                            (k_df_split_x<<<cdivu((h->n + 1) / 2, 256), 256, 0, s>>>((const double *)x, h->n, h->xsplit,
                                                                              h->xsplit_flag)));
                SPMV_LAUNCH_CHECK("x split");
            }
            SPMV_LAUNCH("k_merge_slot_df", s,
                        (k_merge_slot_df<float2><<<grid, SLOT_WARPS * 32, ssmem, s>>>(
                            h->slot_desc, h->slot_col, h->slot_val2, (const double *)x, h->xsplit, h->xsplit_flag,
                            (double *)y, h->carry_row, h->carry_val, h->tiles, h->status_dev + 3)));
            SPMV_LAUNCH_CHECK("merge spmv");
            SPMV_TRY(launch_fixup<double>(h, (double *)y, s));
            return SPMV_OK;
        }
    }
    if constexpr (std::is_same<XT, float>::value && !std::is_same<VT, double>::value)
        if (has_slot_vals<VT>(h)) return launch_slot<VT, NativeAcc<AT>>(h, x, y, s);
    static DeviceOnce attr;
    SPMV_TRY(attr([&] { return set_smem_ctas((const void *)k_merge_warp<VT, XT, AT>, smem, 5); }));
    const unsigned grid = persistent_grid((const void *)k_merge_warp<VT, XT, AT>, MW_WARPS * 32, smem, h->tiles);
    SPMV_LAUNCH("k_merge_warp", s, (k_merge_warp<VT, XT, AT><<<grid, MW_WARPS * 32, smem, s>>>(
                                       h->merge_desc, h->col, (const VT *)h->val, (const XT *)x, (XT *)y, h->part_row,
                                       h->part_nz, h->carry_row, h->carry_val, h->tiles, h->status_dev + 3)));
    SPMV_LAUNCH_CHECK("merge spmv");
    SPMV_TRY(launch_fixup<XT>(h, (XT *)y, s));
    return SPMV_OK;
}

// ================================================================ row split
constexpr int RS_BLOCK = 256;

struct ClassTable {
    int64_t begin[NUM_ROW_CLASSES + 1];       // offset of each class in bin_rows
    int64_t blk_begin[NUM_ROW_CLASSES + 1];   // first CTA of each class
};

// A group of G lanes per row; a warp-wide group (rows of 33..2048 nonzeros) takes
// RS_ROWS_PER_WARP rows, whose row ids and bounds are all loaded first.  Each round loads U
// column indices and values per lane before their x gathers; the last round is predicated
// instead of finished one nonzero at a time.
constexpr int RS_ROWS_PER_WARP = 4;
__host__ __device__ constexpr int rs_rows_per_group(int G) { return G == 32 ? RS_ROWS_PER_WARP : 1; }

// Row-split accumulators: RsPlain sums in AT (one fma per nonzero, butterfly of plain
// additions); RsComp keeps an FP32 sum with its compensation (the FMA error of every product
// and the TwoSum error of every addition, Neumaier style) through the lane sums and the
// butterfly, rounded once at the end.
template <typename AT>
struct RsPlain {
    AT v;
    __device__ __forceinline__ void zero() { v = AT(0); }
    __device__ __forceinline__ void mad(AT a, AT x) { v = v + a * x; }
    __device__ __forceinline__ void add(const RsPlain &o) { v = v + o.v; }
    __device__ __forceinline__ RsPlain xor_shfl(int o, int w) const {
        RsPlain r;
        r.v = __shfl_xor_sync(0xffffffffu, v, o, w);
        return r;
    }
    template <typename XT> __device__ __forceinline__ XT out() const { return XT(v); }
};
struct RsComp {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void mad(float a, float x) { df_fma(a, 0.f, x, 0.f, s, c); }
    __device__ __forceinline__ void add(const RsComp &o) { df_add(s, c, o.s, o.c); }
    __device__ __forceinline__ RsComp xor_shfl(int o, int w) const {
        RsComp r;
        r.s = __shfl_xor_sync(0xffffffffu, s, o, w);
        r.c = __shfl_xor_sync(0xffffffffu, c, o, w);
        return r;
    }
    template <typename XT> __device__ __forceinline__ XT out() const { return XT(__fadd_rn(s, c)); }
};

template <typename VT, typename XT, typename AT, typename Acc, int G>
__device__ __forceinline__ void rowsplit_group(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                               const VT *__restrict__ val, const XT *__restrict__ x,
                                               XT *__restrict__ y, const int32_t *__restrict__ rows, int64_t count,
                                               int64_t local_blk) {
    constexpr int RPG = rs_rows_per_group(G);
    constexpr int RPB = RS_BLOCK / G * RPG;   // rows per CTA
    constexpr int U = G >= 8 ? 4 : 1;         // loads in flight per lane and round
    const int g = threadIdx.x / G, lane = threadIdx.x % G;
    const int64_t r0 = local_blk * RPB + (int64_t)g * RPG;
    int32_t row[RPG], k0[RPG], k1[RPG];
#pragma unroll
    for (int i = 0; i < RPG; ++i) row[i] = r0 + i < count ? rows[r0 + i] : -1;
#pragma unroll
    for (int i = 0; i < RPG; ++i) {
        k0[i] = row[i] >= 0 ? __ldg(row_ptr + row[i]) : 0;
        k1[i] = row[i] >= 0 ? __ldg(row_ptr + row[i] + 1) : 0;
    }
#pragma unroll
    for (int i = 0; i < RPG; ++i) {
        Acc acc;
        acc.zero();
        for (int32_t kb = k0[i]; kb < k1[i]; kb += U * G) {
            int32_t c[U];
            AT a[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int32_t k = kb + u * G + lane;
                c[u] = k < k1[i] ? __ldg(col + k) : -1;
                a[u] = k < k1[i] ? ld_val<VT, AT>(val, k) : AT(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (c[u] >= 0) acc.mad(a[u], ld_x<XT, AT>(x, c[u]));
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc.add(acc.xor_shfl(o, G));
        if (row[i] >= 0 && lane == 0) y[row[i]] = acc.template out<XT>();
    }
}

template <typename VT, typename XT, typename AT, typename Acc>
__device__ __forceinline__ void rowsplit_cta(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                             const VT *__restrict__ val, const XT *__restrict__ x,
                                             XT *__restrict__ y, int32_t row) {
    constexpr int U = 8;   // independent loads in flight per thread
    __shared__ Acc red[RS_BLOCK / 32];
    const int32_t k0 = __ldg(row_ptr + row), k1 = __ldg(row_ptr + row + 1);
    Acc acc;
    acc.zero();
    for (int32_t kb = k0; kb < k1; kb += U * RS_BLOCK) {
        int32_t c[U];
        AT a[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int32_t k = kb + u * RS_BLOCK + threadIdx.x;
            if (k < k1) {
                c[u] = __ldg(col + k);
                a[u] = ld_val<VT, AT>(val, k);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int32_t k = kb + u * RS_BLOCK + threadIdx.x;
            if (k < k1) acc.mad(a[u], ld_x<XT, AT>(x, c[u]));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc.add(acc.xor_shfl(o, 32));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        Acc s = red[0];
        for (int w = 1; w < RS_BLOCK / 32; ++w) s.add(red[w]);
        y[row] = s.template out<XT>();
    }
    __syncthreads();   // red[] is free for the CTA's next row
}

template <typename VT, typename XT, typename AT, typename Acc>
__device__ __forceinline__ void rowsplit_class(int c, const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                               const VT *__restrict__ val, const XT *__restrict__ x, XT *__restrict__ y,
                                               const int32_t *__restrict__ rows, int64_t count, int64_t lb) {
    switch (c) {
        case 0: rowsplit_group<VT, XT, AT, Acc, 1>(row_ptr, col, val, x, y, rows, count, lb); break;
        case 1: rowsplit_group<VT, XT, AT, Acc, 2>(row_ptr, col, val, x, y, rows, count, lb); break;
        case 2: rowsplit_group<VT, XT, AT, Acc, 4>(row_ptr, col, val, x, y, rows, count, lb); break;
        case 3: rowsplit_group<VT, XT, AT, Acc, 8>(row_ptr, col, val, x, y, rows, count, lb); break;
        case 4: rowsplit_group<VT, XT, AT, Acc, 16>(row_ptr, col, val, x, y, rows, count, lb); break;
        case 5: rowsplit_group<VT, XT, AT, Acc, 32>(row_ptr, col, val, x, y, rows, count, lb); break;
        default: rowsplit_cta<VT, XT, AT, Acc>(row_ptr, col, val, x, y, rows[lb]); break;
    }
}

// COMP: the classes from comp_from on (rows that can be longer than the compensation
// threshold) accumulate with RsComp, the others plainly.
template <typename VT, typename XT, typename AT, bool COMP>
__global__ __launch_bounds__(RS_BLOCK) void k_rowsplit(const int32_t *__restrict__ row_ptr,
                                                       const int32_t *__restrict__ col, const VT *__restrict__ val,
                                                       const XT *__restrict__ x, XT *__restrict__ y,
                                                       const int32_t *__restrict__ bin_rows, ClassTable ct,
                                                       int comp_from) {
    const int64_t nblocks = ct.blk_begin[NUM_ROW_CLASSES];
    for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {   // persistent over the class blocks
        int c = 0;
        while (c < NUM_ROW_CLASSES - 1 && b >= ct.blk_begin[c + 1]) ++c;
        const int64_t lb = b - ct.blk_begin[c];
        const int32_t *rows = bin_rows + ct.begin[c];
        const int64_t count = ct.begin[c + 1] - ct.begin[c];
        if constexpr (COMP) {
            if (c >= comp_from) {
                rowsplit_class<VT, XT, AT, RsComp>(c, row_ptr, col, val, x, y, rows, count, lb);
                continue;
            }
        }
        rowsplit_class<VT, XT, AT, RsPlain<AT>>(c, row_ptr, col, val, x, y, rows, count, lb);
    }
}

// comp_from < 0: plain accumulation everywhere; else compensated from that length class on
// (only with FP32 accumulation).
template <typename VT, typename XT, typename AT>
spmv_status launch_rowsplit(const spmv_matrix *h, const void *x, void *y, cudaStream_t s, int comp_from = -1) {
    ClassTable ct;
    ct.begin[0] = 0;
    ct.blk_begin[0] = 0;
    for (int c = 0; c < NUM_ROW_CLASSES; ++c) {
        const int64_t cnt = h->bin_count[c];
        ct.begin[c + 1] = ct.begin[c] + cnt;
        const int64_t rpb = c < NUM_ROW_CLASSES - 1 ? RS_BLOCK / class_lanes(c) * rs_rows_per_group(class_lanes(c)) : 1;
        ct.blk_begin[c + 1] = ct.blk_begin[c] + (cnt + rpb - 1) / rpb;
    }
    const int64_t blocks = ct.blk_begin[NUM_ROW_CLASSES];
    if (blocks == 0) return SPMV_OK;
    if constexpr (std::is_same<AT, float>::value) {
        if (comp_from >= 0) {
            const unsigned grid = (unsigned)std::min<int64_t>(
                blocks, persistent_grid((const void *)k_rowsplit<VT, XT, AT, true>, RS_BLOCK, 0, blocks * MW_WARPS));
            SPMV_LAUNCH("k_rowsplit", s, (k_rowsplit<VT, XT, AT, true><<<grid, RS_BLOCK, 0, s>>>(
                                             h->row_ptr, h->col, (const VT *)h->val, (const XT *)x, (XT *)y,
                                             h->bin_rows, ct, comp_from)));
            SPMV_LAUNCH_CHECK("rowsplit spmv");
            return SPMV_OK;
        }
    }
    const unsigned grid = (unsigned)std::min<int64_t>(blocks, persistent_grid((const void *)k_rowsplit<VT, XT, AT, false>, RS_BLOCK, 0, blocks * MW_WARPS));
    SPMV_LAUNCH("k_rowsplit", s, (k_rowsplit<VT, XT, AT, false><<<grid, RS_BLOCK, 0, s>>>(h->row_ptr, h->col, (const VT *)h->val,
                                                                 (const XT *)x, (XT *)y, h->bin_rows, ct, -1)));
    SPMV_LAUNCH_CHECK("rowsplit spmv");
    return SPMV_OK;
}

// ================================================================ Hilbert blocked
constexpr int HB_BLOCK = 256;
constexpr int HB_IPT = HB_CHUNK / HB_BLOCK;

__device__ __forceinline__ void atomic_add_out(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add_out(float *p, float v) { atomicAdd(p, v); }

// Blocked product (Sections 3.1, 3.2): a CTA takes HB_CHUNK consecutive stored nonzeros (in
// the stored Hilbert order) and copies the entries of the blocks they fall in (the first
// block comes from the conversion's chunk table) into shared memory.  Thread t handles
// nonzeros e0 + j * HB_BLOCK + t (j < 8), so that each warp instruction touches 32
// consecutive nonzeros, whose rows and columns are close in Hilbert order: all index and
// value loads are issued first, then the bisections (each starting at the previous block),
// then the x gathers, then the additions to y (atomics; y is zeroed first).
template <typename VT, typename XT, typename AT>
__global__ __launch_bounds__(HB_BLOCK, 4) void k_hb_spmv(int64_t nnz, int log2b, const int32_t *__restrict__ chunk_blk,
                                                      const int32_t *__restrict__ blk_ptr,
                                                      const int32_t *__restrict__ blk_row,
                                                      const int32_t *__restrict__ blk_col,
                                                      const uint32_t *__restrict__ idx, const VT *__restrict__ val,
                                                      const XT *__restrict__ x, XT *__restrict__ y) {
    __shared__ int32_t s_ptr[HB_CHUNK + 2];
    __shared__ int32_t s_r0[HB_CHUNK + 1];
    __shared__ int32_t s_c0[HB_CHUNK + 1];
    const int64_t nchunks = (nnz + HB_CHUNK - 1) / HB_CHUNK;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {   // persistent: chunks ch, ch + grid, ...
    const int64_t e0 = ch * HB_CHUNK;
    const int64_t e1 = min(e0 + (int64_t)HB_CHUNK, nnz);   // exclusive
    const int32_t b0 = chunk_blk[ch];
    const int nb = chunk_blk[ch + 1] - b0 + 1;             // blocks touching the chunk (maybe one more)
    uint32_t p[HB_IPT];
    AT v[HB_IPT];
#pragma unroll
    for (int j = 0; j < HB_IPT; ++j) {
        const int64_t e = e0 + j * HB_BLOCK + threadIdx.x;
        p[j] = e < e1 ? __ldg(idx + e) : 0u;
        v[j] = e < e1 ? ld_val<VT, AT>(val, e) : AT(0);
    }
    for (int q = threadIdx.x; q < nb; q += HB_BLOCK) {
        s_ptr[q] = blk_ptr[b0 + q];
        s_r0[q] = blk_row[b0 + q] << log2b;
        s_c0[q] = blk_col[b0 + q] << log2b;
    }
    if (threadIdx.x == 0) s_ptr[nb] = blk_ptr[b0 + nb];
    __syncthreads();
    int64_t rr[HB_IPT], cc[HB_IPT];
    int lo = 0;
#pragma unroll
    for (int j = 0; j < HB_IPT; ++j) {
        const int64_t e = e0 + j * HB_BLOCK + threadIdx.x;
        int hi = nb - 1;   // largest b in [lo, nb) with s_ptr[b] <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((int64_t)s_ptr[mid] <= e) lo = mid;
            else hi = mid - 1;
        }
        rr[j] = (int64_t)s_r0[lo] + (p[j] >> 16);
        cc[j] = (int64_t)s_c0[lo] + (p[j] & 0xFFFFu);
    }
    AT xv[HB_IPT];
#pragma unroll
    for (int j = 0; j < HB_IPT; ++j) xv[j] = e0 + j * HB_BLOCK + threadIdx.x < e1 ? ld_x<XT, AT>(x, cc[j]) : AT(0);
    // Lanes hold consecutive nonzeros: a run of lanes with the same row is summed by a
    // segmented warp scan and added to y once, by the run's last lane.
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 0; j < HB_IPT; ++j) {
        const bool valid = e0 + j * HB_BLOCK + threadIdx.x < e1;
        const int64_t row = valid ? rr[j] : -1;
        AT p = valid ? v[j] * xv[j] : AT(0);
        const int64_t up = __shfl_up_sync(0xffffffffu, row, 1), down = __shfl_down_sync(0xffffffffu, row, 1);
        bool f = lane == 0 || up != row;   // first lane of its run
        if (!__all_sync(0xffffffffu, f)) {
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                if (__all_sync(0xffffffffu, f)) break;   // every lane has reached its segment head
                const AT pv = __shfl_up_sync(0xffffffffu, p, o);
                const bool of = __shfl_up_sync(0xffffffffu, f, o);
                if (lane >= o && !f) p += pv;
                if (lane >= o) f = f || of;
            }
        }
        if (valid && (lane == 31 || down != row)) atomic_add_out(y + row, XT(p));
    }
    __syncthreads();   // the block table of this chunk is read until here
    }
}

template <typename VT, typename XT, typename AT>
spmv_status launch_hb(const spmv_matrix *h, const void *x, void *y, cudaStream_t s) {
    SPMV_CUDA_TRY(cudaMemsetAsync(y, 0, (size_t)h->m * sizeof(XT), s));
    if (h->nnz == 0) return SPMV_OK;
    const unsigned hb_grid = std::min<unsigned>(cdivu(h->nnz, HB_CHUNK),
                                                 persistent_grid((const void *)k_hb_spmv<VT, XT, AT>, HB_BLOCK, 0, h->nnz));
    SPMV_LAUNCH("k_hb_spmv", s, (k_hb_spmv<VT, XT, AT><<<hb_grid, HB_BLOCK, 0, s>>>(
        h->nnz, h->log2beta, h->hb_chunk_blk, h->blk_ptr, h->blk_row, h->blk_col, h->hb_idx, (const VT *)h->hb_val,
        (const XT *)x, (XT *)y)));
    SPMV_LAUNCH_CHECK("hb spmv");
    return SPMV_OK;
}

// ================================================================ bounded-wait test
// One warp waits on an mbarrier that nothing arrives at, with the same bounded wait as the
// persistent kernels but `polls` polls; when it gives up it sets the timeout bit and returns,
// which leaves the context usable.
__global__ void k_test_wait(long long polls, uint32_t *__restrict__ status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (!mbar_wait(&bar, 0u, polls) && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}

spmv_status launch_test_wait(long long polls, uint32_t *status, cudaStream_t s) {
    SPMV_LAUNCH("k_test_wait", s, (k_test_wait<<<1, 32, 0, s>>>(polls, status)));
    SPMV_LAUNCH_CHECK("test wait");
    return SPMV_OK;
}

// ================================================================ dispatch
// Supported (values, vectors, accumulation): F64/F64/F64; F32/F32/F32; F32/F32/F64;
// BF16/F32/F32; BF16/F32/F64; PATTERN/F64/F64; PATTERN/F32/F32.
enum Algo { MERGE, ROWSPLIT, HB };

template <typename VT, typename Acc>
spmv_status launch_merge_comp(const spmv_matrix *h, const void *x, void *y, cudaStream_t s) {
    if (has_slot_vals<VT>(h)) return launch_slot<VT, Acc>(h, x, y, s);
    constexpr size_t smem = (size_t)MW_WARPS * 2 * WarpSlot<VT>::BYTES;
    static DeviceOnce attr;
    SPMV_TRY(attr([&] { return set_smem_ctas((const void *)k_merge_warp_comp<VT, Acc>, smem, 5); }));
    const unsigned grid = persistent_grid((const void *)k_merge_warp_comp<VT, Acc>, MW_WARPS * 32, smem, h->tiles);
    SPMV_LAUNCH("k_merge_warp_comp", s, (k_merge_warp_comp<VT, Acc><<<grid, MW_WARPS * 32, smem, s>>>(
                                       h->merge_desc, h->col, (const VT *)h->val, (const float *)x, (float *)y,
                                       h->part_row, h->part_nz, h->carry_row, h->carry_val, h->tiles,
                                       h->status_dev + 3)));
    SPMV_LAUNCH_CHECK("merge spmv");
    SPMV_TRY(launch_fixup<float>(h, (float *)y, s));
    return SPMV_OK;
}

template <typename VT, typename XT, typename AT>
spmv_status run_algo(Algo a, const spmv_matrix *h, const void *x, void *y, bool allow_df, cudaStream_t s) {
    if (a == MERGE) return launch_merge<VT, XT, AT, MERGE_IPT>(h, x, y, allow_df, s);
    if (a == ROWSPLIT) return launch_rowsplit<VT, XT, AT>(h, x, y, s);
    return launch_hb<VT, XT, AT>(h, x, y, s);
}

spmv_status dispatch(Algo a, const spmv_matrix *h, const void *x, void *y, spmv_dtype vdt, uint32_t acc,
                     cudaStream_t s) {
    const spmv_dtype dt = h->dt;
    const bool allow_df = acc == SPMV_ACC_DEFAULT;   // SPMV_ACC_F64 forces native FP64 arithmetic
    if (acc == SPMV_ACC_DEFAULT) acc = (dt == SPMV_F64 || (dt == SPMV_PATTERN && vdt == SPMV_F64)) ? SPMV_ACC_F64 : SPMV_ACC_F32;
    if (vdt == SPMV_F64) {
        if (acc != SPMV_ACC_F64) goto unsupported;
        if (dt == SPMV_F64) return run_algo<double, double, double>(a, h, x, y, allow_df, s);
        if (dt == SPMV_PATTERN) return run_algo<Pattern, double, double>(a, h, x, y, allow_df, s);
        if (dt == SPMV_F32) return run_algo<float, double, double>(a, h, x, y, allow_df, s);
        goto unsupported;
    }
    if (vdt == SPMV_F32 && a == ROWSPLIT && (acc == SPMV_ACC_COMPENSATED || acc == SPMV_ACC_SEGMENT)) {
        // compensated from the first length class whose rows can be longer than the threshold
        int from = 0;
        if (acc == SPMV_ACC_SEGMENT) {
            static const int64_t cmax[NUM_ROW_CLASSES - 1] = {2, 4, 8, 16, 32, 2048};
            while (from < NUM_ROW_CLASSES - 1 && cmax[from] <= h->comp_tau) ++from;
        }
        if (dt == SPMV_F32) return launch_rowsplit<float, float, float>(h, x, y, s, from);
        if (dt == SPMV_BF16) return launch_rowsplit<__nv_bfloat16, float, float>(h, x, y, s, from);
        if (dt == SPMV_PATTERN) return launch_rowsplit<Pattern, float, float>(h, x, y, s, from);
    }
    if (vdt == SPMV_F32 && acc == SPMV_ACC_COMPENSATED && a == MERGE) {
        if (dt == SPMV_F32) return launch_merge_comp<float, CompAcc>(h, x, y, s);
        if (dt == SPMV_BF16) return launch_merge_comp<__nv_bfloat16, CompAcc>(h, x, y, s);
        if (dt == SPMV_PATTERN) return launch_merge_comp<Pattern, CompAcc>(h, x, y, s);
    }
    if (vdt == SPMV_F32 && acc == SPMV_ACC_SEGMENT && a == MERGE) {
        if (dt == SPMV_F32) return launch_merge_comp<float, SegAcc>(h, x, y, s);
        if (dt == SPMV_BF16) return launch_merge_comp<__nv_bfloat16, SegAcc>(h, x, y, s);
        if (dt == SPMV_PATTERN) return launch_merge_comp<Pattern, SegAcc>(h, x, y, s);
    }
    if (vdt == SPMV_F32) {
        if (acc == SPMV_ACC_F32) {
            if (dt == SPMV_F32) return run_algo<float, float, float>(a, h, x, y, allow_df, s);
            if (dt == SPMV_BF16) return run_algo<__nv_bfloat16, float, float>(a, h, x, y, allow_df, s);
            if (dt == SPMV_PATTERN) return run_algo<Pattern, float, float>(a, h, x, y, allow_df, s);
        } else if (acc == SPMV_ACC_F64 && a != HB) {
            if (dt == SPMV_F32) return run_algo<float, float, double>(a, h, x, y, allow_df, s);
            if (dt == SPMV_BF16) return run_algo<__nv_bfloat16, float, double>(a, h, x, y, allow_df, s);
        }
    }
unsupported:
    set_error("spmv_mul: unsupported combination of matrix dtype, vector dtype and accumulation");
    return SPMV_ERR_UNSUPPORTED;
}

// ================================================================ allocation-free entry
// spmv_mul_csr_merge_noalloc keeps the merge-path partition and the tile carries in the
// file-scope array below instead of memory it allocates, for callers that must not
// allocate device memory.  Every call on a device shares the one array.
constexpr int64_t NOALLOC_MAX_TILES = 1 << 16;   // up to 65,536 tiles of MERGE_TILE_ITEMS path items
constexpr size_t NOALLOC_PART_BYTES = (size_t)(NOALLOC_MAX_TILES + 1) * 4;
constexpr size_t NOALLOC_BYTES = 2 * ((NOALLOC_PART_BYTES + 255) / 256 * 256) + (size_t)NOALLOC_MAX_TILES * 4 +
                                 (size_t)NOALLOC_MAX_TILES * 8;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Split points of the merge path (same rule as the conversion's partition).
__global__ void k_noalloc_partition(const int32_t *__restrict__ row_ptr, int64_t m, int64_t nnz, int64_t tiles,
                                    int64_t tile_items, int32_t *__restrict__ part_row, int32_t *__restrict__ part_nz) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > tiles) return;
    const int64_t d = min(t * tile_items, m + nnz);
    int64_t lo = d - nnz > 0 ? d - nnz : 0, hi = d < m ? d : m;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)row_ptr[mid] <= d - mid) lo = mid;
        else hi = mid - 1;
    }
    part_row[t] = (int32_t)lo;
    part_nz[t] = (int32_t)(d - lo);
}

// Device address of the scratch array, looked up once per device with that device current.
spmv_status noalloc_scratch(unsigned char **out) {
    static std::mutex mu;
    static void *addr[256] = {nullptr};
    int dev = 0;
    SPMV_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) {
        set_error("spmv_mul_csr_merge_noalloc: device ordinal out of range");
        return SPMV_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> g(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
        addr[dev] = p;
    }
    *out = (unsigned char *)addr[dev];
    return SPMV_OK;
}

spmv_status noalloc_merge(int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col,
                          const double *data, const double *x, double *y, cudaStream_t s) {
    const int64_t tiles = std::max<int64_t>(1, (m + nnz + MERGE_TILE_ITEMS - 1) / MERGE_TILE_ITEMS);
    if (tiles > NOALLOC_MAX_TILES) {
        set_error("spmv_mul_csr_merge_noalloc: m + nnz exceeds the fixed scratch (65,536 tiles of 1,792 row ends "
                  "and nonzeros, i.e. m + nnz <= 117,440,512)");
        return SPMV_ERR_UNSUPPORTED;
    }
    unsigned char *base = nullptr;
    SPMV_TRY(noalloc_scratch(&base));
    const size_t pb = (NOALLOC_PART_BYTES + 255) / 256 * 256;
    int32_t *part_row = (int32_t *)base;
    int32_t *part_nz = (int32_t *)(base + pb);
    int32_t *carry_row = (int32_t *)(base + 2 * pb);
    double *carry_val = (double *)(base + 2 * pb + (size_t)NOALLOC_MAX_TILES * 4);
    constexpr size_t smem = merge_smem<NativeAcc<double>>(MERGE_IPT);
    static_assert(smem <= 48 * 1024, "within the default dynamic shared memory limit: no attribute to set");
    k_noalloc_partition<<<cdivu(tiles + 1, 256), 256, 0, s>>>(row_ptr, m, nnz, tiles, MERGE_TILE_ITEMS, part_row, part_nz);
    SPMV_LAUNCH_CHECK("noalloc partition");
    k_merge_spmv<double, double, double, MERGE_IPT><<<(unsigned)tiles, MP_BLOCK, smem, s>>>(
        row_ptr, col, data, x, y, part_row, part_nz, carry_row, carry_val);
    SPMV_LAUNCH_CHECK("noalloc merge spmv");
    k_merge_fixup<double><<<cdivu(tiles, 256), 256, 0, s>>>(tiles, m, carry_row, carry_val, y);
    SPMV_LAUNCH_CHECK("noalloc merge fixup");
    return SPMV_OK;
}

}  // namespace

spmv_status mul_merge(const spmv_matrix *h, const void *x, void *y, spmv_dtype vdt, uint32_t acc, cudaStream_t s) {
    return dispatch(MERGE, h, x, y, vdt, acc, s);
}
spmv_status mul_rowsplit(const spmv_matrix *h, const void *x, void *y, spmv_dtype vdt, uint32_t acc, cudaStream_t s) {
    return dispatch(ROWSPLIT, h, x, y, vdt, acc, s);
}
spmv_status test_wait(long long polls, uint32_t *status, cudaStream_t s) { return launch_test_wait(polls, status, s); }
spmv_status mul_hb(const spmv_matrix *h, const void *x, void *y, spmv_dtype vdt, uint32_t acc, cudaStream_t s) {
    if (h->has_stage && !h->hb_chunked) return mul_stage(h, x, y, vdt, acc, s);
    return dispatch(HB, h, x, y, vdt, acc, s);
}

spmv_status split_x(const spmv_matrix *h, const double *x, cudaStream_t s) {
    SPMV_CUDA_TRY(cudaMemsetAsync(h->xsplit_flag, 0, 4, s));
    if (h->n > 0) {
        SPMV_LAUNCH("k_df_split_x", s,
                    (k_df_split_x<<<cdivu((h->n + 1) / 2, 256), 256, 0, s>>>(x, h->n, h->xsplit, h->xsplit_flag)));
        SPMV_LAUNCH_CHECK("x split");
    }
    return SPMV_OK;
}

spmv_status split_x_zero_y(const spmv_matrix *h, const double *x, double *y, cudaStream_t s) {
    SPMV_CUDA_TRY(cudaMemsetAsync(h->xsplit_flag, 0, 4, s));
    const int64_t e = std::max(h->n, h->m);
    if (e > 0) {
        SPMV_LAUNCH("k_df_split_x", s, (k_df_split_x_zero<<<cdivu((e + 1) / 2, 256), 256, 0, s>>>(
                                           x, h->n, h->xsplit, h->xsplit_flag, y, h->m)));
        SPMV_LAUNCH_CHECK("x split and y zero");
    }
    return SPMV_OK;
}

spmv_status mul_csr_merge_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col,
                                  const double *data, const double *x, double *y, cudaStream_t s) {
    return noalloc_merge(m, n, nnz, row_ptr, col, data, x, y, s);
}

spmv_status mul_merge_pattern_split(const spmv_matrix *h, const double *x, const float2 *x2, const uint32_t *xflag,
                                    double *y, cudaStream_t s) {
    if (h->slot_desc) {
        constexpr size_t ssmem = slot_smem<Pattern, DfAcc>();
        static DeviceOnce sattr;
        SPMV_TRY(sattr([&] { return set_smem_ctas((const void *)k_merge_slot_df<Pattern>, ssmem, SLOT_CTAS); }));
        const unsigned grid = persistent_grid((const void *)k_merge_slot_df<Pattern>, SLOT_WARPS * 32, ssmem, h->tiles);
        SPMV_LAUNCH("k_merge_slot_df", s, (k_merge_slot_df<Pattern><<<grid, SLOT_WARPS * 32, ssmem, s>>>(
                                           h->slot_desc, h->slot_col, (const Pattern *)nullptr, x, x2, xflag, y,
                                           h->carry_row, h->carry_val, h->tiles, h->status_dev + 3)));
        SPMV_LAUNCH_CHECK("pattern merge spmv");
        SPMV_TRY(launch_fixup<double>(h, y, s));
        return SPMV_OK;
    }
    constexpr size_t smem = (size_t)MW_WARPS * 2 * WarpSlot<Pattern>::BYTES;
    static DeviceOnce attr;
    SPMV_TRY(attr([&] { return set_smem_ctas((const void *)k_merge_warp_pat_df, smem, 5); }));
    const unsigned grid = persistent_grid((const void *)k_merge_warp_pat_df, MW_WARPS * 32, smem, h->tiles);
    SPMV_LAUNCH("k_merge_warp_pat_df", s, (k_merge_warp_pat_df<<<grid, MW_WARPS * 32, smem, s>>>(
                                       h->merge_desc, h->col, x, x2, xflag, y, h->part_row, h->part_nz, h->carry_row,
                                       h->carry_val, h->tiles, h->status_dev + 3)));
    SPMV_LAUNCH_CHECK("pattern merge spmv");
    SPMV_TRY(launch_fixup<double>(h, y, s));
    return SPMV_OK;
}

}  // namespace spmv
