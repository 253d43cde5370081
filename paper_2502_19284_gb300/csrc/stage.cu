// Blocked SpMV with x staged in shared memory (Sections 3.1 and 3.2: blocks of side beta,
// cache reuse of the x and y slices a block touches), laid out for sm_103a.
//
// Layout (built at the HB conversion, from the CRS arrays).  The columns are cut into
// slices of beta = 2^lb (the block columns of the HB format).  Within a slice the nonzeros
// keep the CRS order (rows ascending, columns ascending inside a row): a slice is the CRS
// of the block column, i.e. the column's beta x beta blocks taken top to bottom with
// row-major order inside each block.  The sequence of every slice is cut into warp tiles of
// ST_TILE entries; the last tile of a slice is padded.  An entry is one 32-bit word,
//     (row delta << lb) | (column - slice start),
// the row delta being the distance to the previous entry's row (a new row starts where it
// is non-zero), plus its value.  A delta too large for its 32 - lb bits is covered by
// filler entries (the all-ones delta field, which advance the row by the largest delta and
// carry no product).  Tile t holds item k of lane l (lane l owns the consecutive items
// 8l .. 8l+7) at slot t * 256 + (k mod 8) * 32 + l, so that every load of a warp is
// contiguous; a 16-byte header per tile gives the row of its first item, its slice and its
// item count.
//
// Product.  One persistent CTA per SM takes a contiguous range of tiles.  For each slice in
// its range with at least ST_STAGE_MIN tiles, the CTA copies the slice of x into shared
// memory once (beta entries) and its warps read x from there; for the few tiles of sparse
// slices x is gathered from global memory.  Each warp loads its tiles into registers with
// 16-byte loads (later tiles prefetched into L2 a few turns ahead), decodes rows from the
// deltas and the lane headers, forms the products, sums runs of equal rows inside a lane and
// across lanes (a segmented scan), and adds each run's sum to y with one reduction (red.global.add);
// y is zeroed first.  The run sums of a tile are staged in shared memory and reduced into y
// 32 at a time, so that consecutive reductions touch consecutive rows.
//
// Differences from the paper: the paper walks the blocks in Hilbert order so that a CPU's
// caches keep both slices of the blocks in flight; here the x slice is staged explicitly
// and y is summed in L2, so the blocks are visited block column by block column (one
// staging of x per slice and CTA) and the Hilbert-ordered arrays remain the exported format.
// Summation order across runs is not fixed (FP results within tolerance, integer results
// exact).
#include "common.cuh"
#include "convert.cuh"
#include "acc.cuh"
#include "tma.cuh"

#include <algorithm>
#include <type_traits>

namespace spmv {

namespace {

constexpr int ST_TILE = 256;                  // entries per warp tile
constexpr int ST_IPT = ST_TILE / 32;          // entries per lane
#ifndef ST_NW_CFG
#define ST_NW_CFG 22
#endif
#ifndef ST_PF_CFG
#define ST_PF_CFG 0
#endif
#ifndef ST_STAGE_MIN_CFG
#define ST_STAGE_MIN_CFG 16
#endif
constexpr int ST_NW = ST_NW_CFG;              // warps per CTA
constexpr int ST_STAGE_MIN = ST_STAGE_MIN_CFG;   // tiles of a slice in a CTA's range from which x is staged
constexpr int ST_X_MAX = 128 * 1024;          // largest x slice staged in shared memory (bytes)
constexpr int ST_PF = ST_PF_CFG;              // a warp prefetches into L2 the tile this many turns after its next

inline unsigned cdivu(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// ================================================================ conversion

// Rows of the CRS entries without a search: f[k] counts the rows r >= 1 that start at entry
// k (empty rows share their start), so the row of entry k is the sum of f[0..k].
__global__ void k_st_rowflags(const int32_t *__restrict__ row_ptr, int64_t m, int64_t nnz, uint32_t *__restrict__ f) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (r >= m) return;
    const int64_t k = row_ptr[r];
    if (k < nnz) atomicAdd(f + k, 1u);
}

// Sort keys: (row << 32) | column of every CRS entry, with the entry's position as the
// payload; the sort runs on the block-column bits (column >> lb), so that it keeps the CRS
// order inside a block column and every later pass reads rows and columns from the keys.
// rows[k + 1] is the row of entry k (exclusive prefix sum of the row flags).
__global__ void k_st_keys(const uint32_t *__restrict__ rows, const int32_t *__restrict__ col, int64_t nnz,
                          uint64_t *__restrict__ keys, uint32_t *__restrict__ perm) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nnz) return;
    keys[k] = ((uint64_t)rows[k + 1] << 32) | (uint32_t)col[k];
    perm[k] = (uint32_t)k;
}

__device__ __forceinline__ int64_t st_slice(uint64_t key, int lb) { return (int64_t)((uint32_t)key >> lb); }
__device__ __forceinline__ int64_t st_row(uint64_t key) { return (int64_t)(key >> 32); }

// Row delta of sorted entry e to the previous entry of its slice (0 for a slice's first).
__device__ __forceinline__ int64_t st_delta(const uint64_t *skey, int64_t e, int lb) {
    const uint64_t k = skey[e];
    if (e == 0 || st_slice(skey[e - 1], lb) != st_slice(k, lb)) return 0;
    return st_row(k) - st_row(skey[e - 1]);
}

// cnt[e] = 1 + the fillers that precede entry e; slice_start[s] = first sorted entry of
// slice s (entries of empty slices point at the next non-empty one); cnt[nnz] = 0.
__global__ void k_st_count(const uint64_t *__restrict__ skey, int64_t nnz, int64_t nsl, int lb, int64_t dmax,
                           uint32_t *__restrict__ cnt, int32_t *__restrict__ slice_start) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e > nnz) return;
    if (e == nnz) {
        cnt[nnz] = 0;
        const int64_t last = nnz ? st_slice(skey[nnz - 1], lb) : -1;
        for (int64_t q = last + 1; q <= nsl; ++q) slice_start[q] = (int32_t)nnz;
        return;
    }
    const int64_t s = st_slice(skey[e], lb);
    const int64_t sp = e ? st_slice(skey[e - 1], lb) : -1;
    if (sp != s)
        for (int64_t q = sp + 1; q <= s; ++q) slice_start[q] = (int32_t)e;
    const int64_t dr = st_delta(skey, e, lb);
    cnt[e] = 1u + (uint32_t)(dr > dmax ? (dr - 1) / dmax : 0);
}

// Tiles of every slice (its entries and fillers, rounded up to whole tiles); tiles[nsl] = 0.
__global__ void k_st_slice_tiles(const int32_t *__restrict__ slice_start, const uint32_t *__restrict__ E,
                                 int64_t nsl, uint32_t *__restrict__ tiles) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s > nsl) return;
    if (s == nsl) {
        tiles[nsl] = 0;
        return;
    }
    const uint32_t tot = E[slice_start[s + 1]] - E[slice_start[s]];
    tiles[s] = (tot + ST_TILE - 1) / ST_TILE;
}

// Position of item q (tile q / 256, lane (q mod 256) / 8, item j = q mod 8 of the lane) for
// elements of ES bytes: each lane's items are grouped by 16 bytes (VW = 16 / ES items) and
// the groups of the 32 lanes are contiguous, so that one 16-byte load per lane and group
// reads 512 contiguous bytes.
template <int ES>
__device__ __forceinline__ int64_t st_pos(int64_t q) {
    constexpr int VW = 16 / ES;
    const int k = (int)(q & (ST_TILE - 1)), l = k >> 3, j = k & (ST_IPT - 1);
    return (q & ~(int64_t)(ST_TILE - 1)) + (j / VW) * (32 * VW) + l * VW + (j % VW);
}

// Stored value of the layout from a CRS value.
template <typename SV, typename VT>
__device__ __forceinline__ SV st_value(const VT *val, int64_t p) {
    if constexpr (std::is_same<SV, float2>::value) {
        float2 r;
        df_split(val[p], &r.x, &r.y);   // every value is inside the double-float window (checked)
        return r;
    } else {
        return val[p];
    }
}

// Writes every entry (and the fillers before it) into its position; the row and slice of
// the tile headers at the positions that start a tile, and a flag in the header of every
// tile that holds a filler.  Padding and the headers stay as zeroed by the caller.
template <typename SV, typename VT>
__global__ void k_st_fill(const uint64_t *__restrict__ skey, const uint32_t *__restrict__ perm,
                          const VT *__restrict__ val, const uint32_t *__restrict__ E,
                          const int32_t *__restrict__ slice_start, const uint32_t *__restrict__ slice_tile,
                          int64_t nnz, int lb, int64_t dmax, uint32_t *__restrict__ words, SV *__restrict__ sval,
                          int4 *__restrict__ hdr) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    const uint64_t key = skey[e];
    const int64_t s = st_slice(key, lb);
    const int64_t row = st_row(key);
    const int64_t dr = st_delta(skey, e, lb);
    const int64_t f = dr > dmax ? (dr - 1) / dmax : 0;
    const int64_t base = (int64_t)slice_tile[s] * ST_TILE;
    const int64_t q0 = base + (int64_t)(E[e] - E[slice_start[s]]);
    const uint32_t filler = (uint32_t)(dmax + 1) << lb;   // all-ones delta field, column 0
    const int64_t prev = row - dr;
    for (int64_t i = 0; i < f; ++i) {
        const int64_t q = q0 + i;
        words[st_pos<4>(q)] = filler;
        atomicOr(&hdr[q / ST_TILE].w, 1);   // the tile holds a filler (no fast path)
        if ((q & (ST_TILE - 1)) == 0) {
            hdr[q / ST_TILE].x = (int)(prev + (i + 1) * dmax);
            hdr[q / ST_TILE].y = (int)s;
        }
    }
    const int64_t q = q0 + f;
    const uint32_t coff = (uint32_t)key & ((1u << lb) - 1u);
    words[st_pos<4>(q)] = ((uint32_t)(dr - f * dmax) << lb) | coff;
    if constexpr (!std::is_same<SV, Pattern>::value) sval[st_pos<(int)sizeof(SV)>(q)] = st_value<SV, VT>(val, perm[e]);
    if ((q & (ST_TILE - 1)) == 0) {
        hdr[q / ST_TILE].x = (int)row;
        hdr[q / ST_TILE].y = (int)s;
    }
}

// Item counts of the tiles (entries and fillers; the rest of a slice's last tile is padding).
__global__ void k_st_counts(const int32_t *__restrict__ slice_start, const uint32_t *__restrict__ E,
                            const uint32_t *__restrict__ slice_tile, int64_t nsl, int64_t ntiles,
                            int4 *__restrict__ hdr) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    int64_t lo = 0, hi = nsl - 1;   // the slice of tile t: largest s with slice_tile[s] <= t
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)slice_tile[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    const int64_t tot = (int64_t)(E[slice_start[lo + 1]] - E[slice_start[lo]]);
    hdr[t].z = (int)min((int64_t)ST_TILE, tot - (t - (int64_t)slice_tile[lo]) * ST_TILE);
    // bit 1 of .w: the first tile of a slice large enough to be staged (its copy costs time)
    if (t == (int64_t)slice_tile[lo] && slice_tile[lo + 1] - slice_tile[lo] >= (uint32_t)ST_STAGE_MIN) hdr[t].w |= 2;
}

// Lane headers of every tile (one warp per tile), computed from the words exactly as the
// product decodes them: the row of the lane's first item, the offset of the lane's run sums
// in the tile's output buffer (exclusive scan of the lanes' counts), the number of rows that
// end inside the lane, whether the lane's last run ends with it, whether its first run
// continues the previous lane's, and the first lane of the lane's scan segment (the last lane
// at or before it whose items start a row: a row end inside it or a first item that does not
// continue); the tile's total run count goes to bits 8..16 of header.w and the number of scan
// levels its longest segment needs (ceil log2 of its length) to bits 17..19.
__global__ void k_st_meta(const uint32_t *__restrict__ words, int4 *__restrict__ hdr, int64_t ntiles, int lb,
                          uint2 *__restrict__ lmeta) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= ntiles) return;   // whole warps
    const int4 hd = hdr[t];
    const uint32_t F = 0xFFFFFFFFu >> lb;
    uint32_t dr[ST_IPT], lsum = 0;
    int nch = 0;
#pragma unroll
    for (int j = 0; j < ST_IPT; ++j) {
        const uint32_t fld = words[st_pos<4>(t * ST_TILE + lane * ST_IPT + j)] >> lb;
        dr[j] = fld == F ? F - 1u : fld;
        if (j == 0 && lane == 0) dr[j] = 0u;
        lsum += dr[j];
        if (j > 0) nch += dr[j] != 0u ? 1 : 0;
    }
    uint32_t incl = lsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const uint32_t next_dr0 = __shfl_down_sync(0xffffffffu, dr[0], 1);
    const bool seg_end = lane == 31 || next_dr0 != 0u;
    const bool cont = lane > 0 && dr[0] == 0u;
    const int cnt = nch + (seg_end ? 1 : 0);
    int base = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, base, o);
        if (lane >= o) base += v;
    }
    const int total = __shfl_sync(0xffffffffu, base, 31);
    base -= cnt;
    const uint32_t row0 = (uint32_t)hd.x + (incl - lsum) + dr[0];
    const uint32_t heads = __ballot_sync(0xffffffffu, nch > 0 || !cont);   // lane 0 is always a head
    const int h = 31 - __clz(heads & (0xFFFFFFFFu >> (31 - lane)));
    const int longest = __reduce_max_sync(0xffffffffu, (unsigned)(lane - h + 1));
    const int levels = longest <= 1 ? 0 : 32 - __clz(longest - 1);
    lmeta[t * 32 + lane] = make_uint2(row0, (uint32_t)base | ((uint32_t)nch << 9) | ((seg_end ? 1u : 0u) << 13) |
                                                ((cont ? 1u : 0u) << 14) | ((uint32_t)h << 15));
    if (lane == 0) hdr[t].w = (hd.w & 0xFF) | (total << 8) | (levels << 17);
}

// Cost of every tile for the split between CTAs: ST_TILE_COST for the tile's 256 entries,
// ST_RUN_COST per run sum (a shared-memory round trip and a reduction in L2), plus
// ST_STAGE_COST at the first tile of a slice whose x slice gets staged.  The weights come from
// per-CTA device times of R-MAT scales 20-22: a staging costs about 70 tiles, a run about 1/350
// of a tile (a sweep around them gave the shortest kernel).  All weights are shifted right by
// `sh` (chosen by the host) so that the prefix sum of the costs fits in 32 bits; cost[ntiles] = 0.
#ifndef ST_TILE_COST_CFG
#define ST_TILE_COST_CFG 1024
#endif
#ifndef ST_RUN_COST_CFG
#define ST_RUN_COST_CFG 3
#endif
#ifndef ST_STAGE_COST_CFG
#define ST_STAGE_COST_CFG 70000
#endif
__global__ void k_st_cost(const int4 *__restrict__ hdr, int64_t ntiles, int sh, uint32_t *__restrict__ cost) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    if (t == ntiles) {
        cost[t] = 0u;
        return;
    }
    const uint32_t w = (uint32_t)hdr[t].w;
    const uint32_t c = (uint32_t)ST_TILE_COST_CFG + ((w >> 8) & 511u) * (uint32_t)ST_RUN_COST_CFG +
                       ((w & 2u) ? (uint32_t)ST_STAGE_COST_CFG : 0u);
    cost[t] = max(c >> sh, 1u);
}

// First tile of every CTA: equal shares of the prefix-summed cost.
__global__ void k_st_parts(const uint32_t *__restrict__ P, int64_t ntiles, int G, int32_t *__restrict__ part) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > G) return;
    if (c == 0 || c == G) {
        part[c] = c == 0 ? 0 : (int32_t)ntiles;
        return;
    }
    const uint64_t target = (uint64_t)P[ntiles] * (uint64_t)c / (uint64_t)G;
    int64_t lo = 0, hi = ntiles;   // first t with P[t] >= target
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((uint64_t)P[mid] >= target) hi = mid;
        else lo = mid + 1;
    }
    part[c] = (int32_t)lo;
}

}  // namespace

// ================================================================ product
namespace {

template <typename SV, typename YT>
struct StArgs {
    const int4 *hdr;
    const uint2 *lmeta;
    const int32_t *part;          // first tile of every CTA (gridDim.x + 1 entries)
    const uint32_t *words;
    const SV *vals;
    const uint32_t *slice_tile;   // first tile of every slice (nsl + 1 entries)
    int64_t nsl, ntiles, n, m;
    int lb;
    int stage_ok;                 // the x slice fits in shared memory
    int x_aligned;                // x is 16-byte aligned (vector copies into the slice)
    YT *y;
    uint32_t *err;
};

// Operand of a stored value for accumulator Acc.
template <typename Acc, typename SV>
__device__ __forceinline__ typename Acc::Op st_a(SV v) {
    using Op = typename Acc::Op;
    if constexpr (std::is_same<SV, float2>::value) {
        if constexpr (std::is_same<Op, float2>::value) return v;
        else return (double)v.x + (double)v.y;   // pair rebuilt: |a - hi - lo| <= 2^-48 |a|
    } else if constexpr (std::is_same<SV, Pattern>::value) {
        if constexpr (std::is_same<Op, float2>::value) return make_float2(1.f, 0.f);
        else return Op(1);
    } else if constexpr (std::is_same<SV, __nv_bfloat16>::value) {
        return Op(__bfloat162float(v));
    } else {
        return Op(v);
    }
}

// One tile in registers: header, 8 words and 8 values of this lane (16-byte loads).
template <typename SV>
struct StRegs {
    static constexpr int VB = std::is_same<SV, Pattern>::value ? 0 : ST_IPT * (int)sizeof(SV);   // value bytes
    static constexpr int NV = VB / 16;                                                          // value loads
    int4 hd;
    uint2 lm;   // lane header: row of item 0; output offset, run count and join flags
    uint4 w[2];
    uint4 v[NV > 0 ? NV : 1];
    template <typename YT>
    __device__ __forceinline__ void load(const StArgs<SV, YT> &a, int64_t t, int lane) {
        hd = __ldg(a.hdr + t);
        lm = __ldcs(a.lmeta + t * 32 + lane);
        const uint4 *wp = reinterpret_cast<const uint4 *>(a.words + t * ST_TILE);
        w[0] = __ldcs(wp + lane);
        w[1] = __ldcs(wp + 32 + lane);
        if constexpr (NV > 0) {
            const uint4 *vp = reinterpret_cast<const uint4 *>(a.vals + t * ST_TILE);
#pragma unroll
            for (int g = 0; g < NV; ++g) v[g] = __ldcs(vp + g * 32 + lane);
        }
    }
    // L2 prefetch of tile t (one lane): header, words and values, without waiting for them
    template <typename YT>
    static __device__ __forceinline__ void prefetch(const StArgs<SV, YT> &a, int64_t t) {
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], 16;" :: "l"(a.hdr + t) : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], 256;" :: "l"(a.lmeta + t * 32) : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(a.words + t * ST_TILE), "r"(ST_TILE * 4)
                     : "memory");
        if constexpr (NV > 0)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(a.vals + t * ST_TILE), "r"(ST_TILE * VB / ST_IPT)
                         : "memory");
    }
    __device__ __forceinline__ uint32_t word(int j) const {
        const uint4 &q = w[j >> 2];
        const int r = j & 3;
        return r == 0 ? q.x : r == 1 ? q.y : r == 2 ? q.z : q.w;
    }
    __device__ __forceinline__ SV val(int j) const {
        if constexpr (NV == 0) {
            return SV{};
        } else {
            constexpr int PER = 16 / (int)sizeof(SV);
            const SV *p = reinterpret_cast<const SV *>(&v[j / PER]);
            return p[j % PER];
        }
    }
};

// Copy x[s beta, min(n, (s+1) beta)) into the shared slice (all threads of the CTA; called
// between two barriers).  The 16-byte aligned body goes by one bulk copy (TMA) completed on
// the CTA's mbarrier, the rest by plain loads.  Returns false if the bounded wait gave up.
template <typename XS>
__device__ __forceinline__ bool st_stage(XS *xs, const XS *__restrict__ xg, int64_t s, int lb, int64_t n, int aligned,
                                         uint64_t *bar, uint32_t parity) {
    const int64_t b0 = s << lb;
    const int ne = (int)min((int64_t)1 << lb, n - b0);
    const XS *src = xg + b0;
    constexpr int PER = 16 / (int)sizeof(XS);   // elements per 16 bytes
    int done = 0;
    if (aligned && (b0 & (PER - 1)) == 0 && ne >= PER) {
        done = ne / PER * PER;
        if (threadIdx.x == 0) {
            // the slice was read through the generic proxy: order that before the async write
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            const uint32_t bytes = (uint32_t)done * (uint32_t)sizeof(XS);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(bar)), "r"(bytes)
                         : "memory");
            tma_load_1d(xs, src, bytes, bar, l2_policy_evict_last());
        }
    }
    for (int i = done + threadIdx.x; i < ne; i += blockDim.x) xs[i] = src[i];
    if (done > 0) return mbar_wait(bar, parity);
    return true;
}

// Per-warp shared buffer of a tile's run sums: rows, then sums (as the accumulator).
template <typename Acc>
struct StOut {
    static constexpr int BYTES = ST_TILE * 4 + ST_TILE * (int)sizeof(Acc);
};

// Exact float -> double by integer operations, without branches: subnormals are scaled by
// 2^24 first (exact) and the exponent corrected; zero, infinities and NaN keep their class.
__device__ __forceinline__ double st_widen(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFFu;
    const uint32_t g = e == 0u ? __float_as_uint(__fmul_rn(f, 16777216.f)) : u;   // 2^24
    const uint32_t eg = (g >> 23) & 0xFFu;
    const uint32_t de = eg == 0u ? 0u : eg == 0xFFu ? 0x7FFu : eg + 896u - (e == 0u ? 24u : 0u);
    const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) | ((unsigned long long)de << 52) |
                                 ((unsigned long long)(g & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)d);
}

// Add a run sum to y with one reduction in L2.  A double-float sum (s, c) is widened part by
// part (exact, integer operations: the short form unless a lane of the warp holds a special
// part) and joined by one FP64 addition: measured on R-MAT scale 22, one reduction per run is
// cheaper than reducing the two parts separately, which doubles the L2 atomic traffic that
// bounds the sparse slices.  FP32 sums with compensation are rounded to FP32 first.
template <typename YT, typename Acc>
__device__ __forceinline__ void st_red(YT *p, const Acc &a) {
    if constexpr (std::is_same<Acc, DfAcc>::value) {
        const bool sp = df_special(a.s) || df_special(a.c);
        double d;
        if (__any_sync(__activemask(), sp)) d = st_widen(a.s) + st_widen(a.c);   // every class, exactly
        else d = df_widen_normal(a.s) + df_widen_normal(a.c);
        atomicAdd(p, d);
    } else {
        atomicAdd(p, a.template out<YT>());
    }
}

// One tile: decode, multiply, sum runs, reduce the run sums into y.  STAGED: x from the
// shared slice, else gathered from global memory.  CLEAN: the tile holds 256 entries and no
// filler (the common case; no per-item checks).  The lane header (conversion) gives the row
// of the lane's first item, where its run sums go in the tile's output buffer and how its
// runs join the neighbouring lanes'.
template <bool STAGED, bool CLEAN, typename Acc, typename SV, typename XS, typename YT>
__device__ __forceinline__ void st_tile(const StRegs<SV> &T, const XS *xs, const XS *__restrict__ xg, int lb,
                                        int64_t n, int64_t m, unsigned char *obuf, YT *__restrict__ y,
                                        uint32_t *err) {
    using Op = typename Acc::Op;
    const int lane = threadIdx.x & 31;
    const uint32_t F = 0xFFFFFFFFu >> lb;                    // filler delta field
    const uint32_t cmask = (1u << lb) - 1u;
    const int64_t sbase = (int64_t)T.hd.y << lb;
    const uint32_t meta = T.lm.y;
    const int base = (int)(meta & 511u), nch = (int)((meta >> 9) & 15u);
    const bool seg_end = (meta >> 13) & 1u, cont = (meta >> 14) & 1u;
    const int total = (int)(((uint32_t)T.hd.w >> 8) & 511u);
    uint32_t dr[ST_IPT], co[ST_IPT];
    uint32_t valid = 0xFFu;
#pragma unroll
    for (int j = 0; j < ST_IPT; ++j) {
        const uint32_t w = T.word(j);
        dr[j] = w >> lb;
        co[j] = w & cmask;
    }
    if constexpr (!CLEAN) {
        valid = 0;
#pragma unroll
        for (int j = 0; j < ST_IPT; ++j) {
            const bool filler = dr[j] == F;
            if (filler) dr[j] = F - 1u;
            if (!filler && lane * ST_IPT + j < T.hd.z && sbase + co[j] < n) valid |= 1u << j;
        }
    }
    Op xv[ST_IPT];
#pragma unroll
    for (int j = 0; j < ST_IPT; ++j) {
        if constexpr (STAGED) xv[j] = Op(xs[co[j]]);
        else xv[j] = (valid >> j) & 1u ? Op(__ldg(xg + sbase + co[j])) : Op{};
    }
    int32_t *orow = reinterpret_cast<int32_t *>(obuf);
    Acc *oacc = reinterpret_cast<Acc *>(obuf + ST_TILE * 4);
    int64_t r = (int64_t)T.lm.x;
    Acc acc, zero;
    acc.zero();
    zero.zero();
    int q = 0;
#pragma unroll
    for (int j = 0; j < ST_IPT; ++j) {
        if (j > 0) {
            const bool c = dr[j] != 0u;   // a new row starts at item j: the run before it is done
            if (c) {
                orow[base + q] = (int32_t)r;
                oacc[base + q] = acc;
            }
            acc = c ? zero : acc;
            q += c ? 1 : 0;
            r += dr[j];
        }
        if (CLEAN || ((valid >> j) & 1u)) acc.mad(st_a<Acc, SV>(T.val(j)), xv[j]);
    }
    // segmented inclusive scan of the lanes' trailing partial sums over the levels the tile's
    // longest segment needs; a segment starts at a lane that begins a new row within itself or
    // at its first item (the segment's first lane comes with the lane header)
    const int h = (int)((meta >> 15) & 31u);
    const int levels = (int)(((uint32_t)T.hd.w >> 17) & 7u);
    Acc run = acc;
    for (int k = 0; k < levels; ++k) {
        const int o = 1 << k;
        Acc ov = run.shfl_up(o);
        if (lane - o >= h) {
            ov.add(run);
            run = ov;
        }
    }
    const Acc prev = run.shfl_up(1);
    if (seg_end) {
        orow[base + nch] = (int32_t)r;
        oacc[base + nch] = run;
    }
    __syncwarp();
    if (nch > 0 && cont) {   // the lane's first run, with what the lanes before it add to that row
        Acc v = prev;
        v.add(oacc[base]);
        oacc[base] = v;
    }
    __syncwarp();
    for (int i = lane; i < total; i += 32) {
        const int32_t row = orow[i];
        if (row >= 0 && (int64_t)row < m) st_red(y + row, oacc[i]);
        else atomicOr(err, ST_INDEX_RANGE);   // a corrupt layout: report, never write outside y
    }
    __syncwarp();   // the buffer is reused by the next tile
}

// Slice walk of a CTA: the segment [sa, sb) of the current slice within the CTA's tile range,
// and whether its x slice is staged.  advance() moves to the segment holding tile `t` (or
// past the range), staging every staged segment on the way between two block barriers, so
// that every warp passes the same barriers whatever tiles it owns.
template <typename XS>
struct StWalk {
    int64_t s, sa, sb, t0, t1;
    bool staged;
    uint32_t nstage;
    bool dead;
    template <typename SV, typename YT>
    __device__ __forceinline__ void enter(const StArgs<SV, YT> &a, XS *xs, const XS *__restrict__ xg,
                                          uint64_t *bar) {
        sa = max(t0, (int64_t)a.slice_tile[s]);
        sb = min(t1, (int64_t)a.slice_tile[s + 1]);
        staged = a.stage_ok && sb - sa >= ST_STAGE_MIN;
        if (staged) {
            __syncthreads();   // the previous slice is no longer read (and the mbarrier is set up)
            const int64_t b0 = s << a.lb;
            const bool bulk = a.x_aligned && (b0 & (16 / (int)sizeof(XS) - 1)) == 0 &&
                              min((int64_t)1 << a.lb, a.n - b0) >= 16 / (int)sizeof(XS);
            if (!st_stage<XS>(xs, xg, s, a.lb, a.n, a.x_aligned, bar, nstage & 1u) && !dead) {
                if ((threadIdx.x & 31) == 0) atomicOr(a.err, ST_TIMEOUT);
                dead = true;
            }
            nstage += bulk ? 1u : 0u;
            __syncthreads();
        }
    }
    template <typename SV, typename YT>
    __device__ __forceinline__ void advance(const StArgs<SV, YT> &a, int64_t t, XS *xs, const XS *__restrict__ xg,
                                            uint64_t *bar) {
        while (t >= sb && sb < t1) {
            ++s;
            enter(a, xs, xg, bar);
        }
    }
};

// The CTA's tile range, slice by slice.  Acc/XS: accumulator and x type of the slices.  Each
// warp takes the tiles t0 + warp, t0 + warp + ST_NW, ... in one register set, and while it
// computes one tile its next is prefetched into L2 (measured: no prefetch 0.272 ms, the next
// tile 0.251 ms, three or five tiles ahead 0.269 / 0.286 ms at R-MAT scale 22).  Two register
// sets, with the next tile's loads in flight in registers, cap the CTA at 16 warps by registers;
// one set and 22 warps is faster.
template <typename Acc, typename SV, typename XS, typename YT>
__device__ __forceinline__ void st_run(const StArgs<SV, YT> &a, const XS *__restrict__ xg, unsigned char *smem) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *obuf = smem + warp * StOut<Acc>::BYTES;
    XS *xs = reinterpret_cast<XS *>(smem + ST_NW * StOut<Acc>::BYTES);
    const int64_t t0 = a.part[blockIdx.x], t1 = a.part[blockIdx.x + 1];
    if (t0 >= t1) return;   // the same for every thread of the CTA
    int64_t lo = 0, hi = a.nsl - 1;   // slice of t0: largest s with slice_tile[s] <= t0
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if ((int64_t)a.slice_tile[mid] <= t0) lo = mid;
        else hi = mid - 1;
    }
    __shared__ __align__(8) uint64_t sbar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&sbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    StWalk<XS> wk;
    wk.s = lo;
    wk.t0 = t0;
    wk.t1 = t1;
    wk.nstage = 0;
    wk.dead = false;
    wk.enter(a, xs, xg, &sbar);
    auto tile = [&](const StRegs<SV> &T, int64_t t) {
        wk.advance(a, t, xs, xg, &sbar);
        if (wk.dead) return;
        const bool clean = T.hd.z == ST_TILE && (T.hd.w & 1) == 0;
        if (wk.staged) {
            if (clean) st_tile<true, true, Acc, SV, XS, YT>(T, xs, xg, a.lb, a.n, a.m, obuf, a.y, a.err);
            else st_tile<true, false, Acc, SV, XS, YT>(T, xs, xg, a.lb, a.n, a.m, obuf, a.y, a.err);
        } else {
            if (clean) st_tile<false, true, Acc, SV, XS, YT>(T, xs, xg, a.lb, a.n, a.m, obuf, a.y, a.err);
            else st_tile<false, false, Acc, SV, XS, YT>(T, xs, xg, a.lb, a.n, a.m, obuf, a.y, a.err);
        }
    };
    StRegs<SV> A;
    int64_t cp = t0 + warp;
    if (lane == 0)
        for (int k = 1; k < 1 + ST_PF; ++k)
            if (cp + k * ST_NW < t1) StRegs<SV>::prefetch(a, cp + k * ST_NW);
    while (cp < t1) {
        A.load(a, cp, lane);
        const int64_t tp = cp + (int64_t)(1 + ST_PF) * ST_NW;   // the next tile (ST_PF = 0) on its way into L2
        if (lane == 0 && tp < t1) StRegs<SV>::prefetch(a, tp);
        tile(A, cp);
        cp += ST_NW;
    }
    wk.advance(a, t1, xs, xg, &sbar);   // the barriers of the remaining staged segments
}

}  // namespace

// ================================================================ host side
namespace {

constexpr int ST_CB = 256;
inline unsigned st_grid(int64_t n) { return std::max(1u, cdivu(n, ST_CB)); }

// Kinds of stored values in the layout.
enum : int32_t { ST_NONE = 0, ST_F2 = 1, ST_F64 = 2, ST_F32 = 3, ST_BF16 = 4 };

template <typename SV, typename VT>
spmv_status st_fill_launch(const uint64_t *Ks, const uint32_t *Ps, const spmv_matrix *h, const uint32_t *E,
                           const int32_t *sstart, const uint32_t *stile, int lb, int64_t dmax, uint32_t *words,
                           void *vals, int4 *hdr, cudaStream_t s) {
    SPMV_LAUNCH("k_st_fill", s, (k_st_fill<SV, VT><<<st_grid(h->nnz), ST_CB, 0, s>>>(
                                     Ks, Ps, (const VT *)h->val, E, sstart, stile, h->nnz, lb, dmax, words, (SV *)vals,
                                     hdr)));
    SPMV_LAUNCH_CHECK("stage fill");
    return SPMV_OK;
}

int st_sms();

// First tile of every CTA (one CTA per SM of the current device): equal shares of the
// prefix-summed tile costs.
spmv_status st_split(const int4 *hp, int64_t ntiles, DevBuf *part, int *G, cudaStream_t s) {
    *G = st_sms();
    SPMV_TRY(part->alloc((size_t)(*G + 1) * 4, "stage CTA split"));
    DevBuf cost(s), pcost(s), ctmp(s);
    SPMV_TRY(cost.alloc((size_t)(ntiles + 1) * 4, "stage tile costs"));
    SPMV_TRY(pcost.alloc((size_t)(ntiles + 1) * 4, "stage tile costs"));
    SPMV_TRY(ctmp.alloc(scan_temp_bytes(ntiles + 1), "stage tile costs"));
    // costs at most ntiles x (tile + 256 runs) + one staging per tile: shift them into 31 bits
    const uint64_t bound = (uint64_t)ntiles * ((uint64_t)ST_TILE_COST_CFG + 256ull * ST_RUN_COST_CFG + ST_STAGE_COST_CFG);
    int sh = 0;
    while ((bound >> sh) >= (1ull << 31)) ++sh;
    SPMV_LAUNCH("k_st_cost", s, (k_st_cost<<<st_grid(ntiles + 1), ST_CB, 0, s>>>(hp, ntiles, sh,
                                                                              cost.as<uint32_t>())));
    SPMV_LAUNCH_CHECK("stage tile costs");
    SPMV_TRY(exclusive_scan_u32(cost.as<uint32_t>(), pcost.as<uint32_t>(), ntiles + 1, ctmp.p, s));
    SPMV_LAUNCH("k_st_parts", s, (k_st_parts<<<st_grid(*G + 1), ST_CB, 0, s>>>(pcost.as<uint32_t>(), ntiles, *G,
                                                                              part->as<int32_t>())));
    SPMV_LAUNCH_CHECK("stage CTA split");
    return SPMV_OK;
}

int st_sms() {
    int dev = 0, n = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || n < 1) {
        cudaGetLastError();
        return 1;
    }
    return n;
}

template <typename SV, typename YT>
StArgs<SV, YT> st_args(const spmv_matrix *h, size_t xsize, const void *xuser, void *y, bool *stage_ok) {
    StArgs<SV, YT> a;
    a.hdr = h->st_hdr;
    a.lmeta = h->st_lmeta;
    a.part = h->st_part;
    a.words = h->st_words;
    a.vals = (const SV *)h->st_vals;
    a.slice_tile = h->st_slice_tile;
    a.nsl = h->stage_nsl;
    a.ntiles = h->stage_tiles;
    a.n = h->n;
    a.m = h->m;
    a.lb = h->stage_lb;
    *stage_ok = ((size_t)1 << h->stage_lb) * xsize <= (size_t)ST_X_MAX;
    a.stage_ok = *stage_ok ? 1 : 0;
    a.x_aligned = ((uintptr_t)xuser & 15u) == 0u ? 1 : 0;
    a.y = (YT *)y;
    a.err = h->status_dev + 3;
    return a;
}

template <typename Acc>
constexpr size_t st_slots_bytes() { return (size_t)ST_NW * StOut<Acc>::BYTES; }

}  // namespace

// FP64 vectors: double-float (split x) unless x leaves the window or force_native; values
// stored as doubles or FP32 use native FP64 throughout.
template <typename SV>
__global__ __launch_bounds__(ST_NW * 32, 1) void k_hb_stage_f64(StArgs<SV, double> a, const double *__restrict__ x,
                                                             const float2 *__restrict__ x2,
                                                             const uint32_t *__restrict__ xflag, int force_native) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr bool CAN_DF = std::is_same<SV, float2>::value || std::is_same<SV, Pattern>::value;
    if constexpr (CAN_DF) {
        if (!force_native && *xflag == 0u) {
            StArgs<SV, double> b = a;
            b.x_aligned = 1;   // the split copy is the library's own, 256-byte aligned
            st_run<DfAcc, SV, float2, double>(b, x2, smem);
            return;
        }
    }
    st_run<NativeAcc<double>, SV, double, double>(a, x, smem);
}

// FP32 vectors with an FP32 accumulator (plain, compensated in the run joins, or compensated).
template <typename SV, typename Acc>
__global__ __launch_bounds__(ST_NW * 32, 1) void k_hb_stage_f32(StArgs<SV, float> a, const float *__restrict__ x) {
    extern __shared__ __align__(16) unsigned char smem[];
    st_run<Acc, SV, float, float>(a, x, smem);
}

namespace {

template <typename SV>
spmv_status st_mul_f64(const spmv_matrix *h, const double *x, double *y, bool force_native, cudaStream_t s) {
    constexpr bool CAN_DF = std::is_same<SV, float2>::value || std::is_same<SV, Pattern>::value;
    bool use_df = CAN_DF && !force_native && h->xsplit;
    if (use_df) SPMV_TRY(split_x_zero_y(h, x, y, s));   // y zeroed in the same launch
    else SPMV_CUDA_TRY(cudaMemsetAsync(y, 0, (size_t)h->m * 8, s));
    bool stage_ok = false;
    StArgs<SV, double> a = st_args<SV, double>(h, 8, x, y, &stage_ok);
    static_assert(StOut<DfAcc>::BYTES == StOut<NativeAcc<double>>::BYTES, "one buffer size for both forms");
    constexpr size_t slots = st_slots_bytes<DfAcc>();
    const size_t smem = slots + (stage_ok ? ((size_t)1 << h->stage_lb) * 8 : 0);
    static DeviceOnce attr;
    SPMV_TRY(attr([&] { return set_smem((const void *)k_hb_stage_f64<SV>, slots + ST_X_MAX); }));
    const unsigned grid = (unsigned)h->stage_parts;
    SPMV_LAUNCH("k_hb_stage", s, (k_hb_stage_f64<SV><<<grid, ST_NW * 32, smem, s>>>(
                                      a, x, h->xsplit, h->xsplit_flag, use_df ? 0 : 1)));
    SPMV_LAUNCH_CHECK("staged blocked spmv");
    return SPMV_OK;
}

template <typename SV, typename Acc>
spmv_status st_mul_f32(const spmv_matrix *h, const float *x, float *y, cudaStream_t s) {
    bool stage_ok = false;
    StArgs<SV, float> a = st_args<SV, float>(h, 4, x, y, &stage_ok);
    constexpr size_t slots = st_slots_bytes<Acc>();
    const size_t smem = slots + (stage_ok ? ((size_t)1 << h->stage_lb) * 4 : 0);
    static DeviceOnce attr;
    SPMV_TRY(attr([&] { return set_smem((const void *)k_hb_stage_f32<SV, Acc>, slots + ST_X_MAX); }));
    const unsigned grid = (unsigned)h->stage_parts;
    SPMV_LAUNCH("k_hb_stage", s, (k_hb_stage_f32<SV, Acc><<<grid, ST_NW * 32, smem, s>>>(a, x)));
    SPMV_LAUNCH_CHECK("staged blocked spmv");
    return SPMV_OK;
}

template <typename SV>
spmv_status st_mul_f32_acc(const spmv_matrix *h, const float *x, float *y, uint32_t acc, cudaStream_t s) {
    if (acc == SPMV_ACC_F32 || acc == SPMV_ACC_DEFAULT) return st_mul_f32<SV, NativeAcc<float>>(h, x, y, s);
    if (acc == SPMV_ACC_SEGMENT) return st_mul_f32<SV, SegAcc>(h, x, y, s);
    if (acc == SPMV_ACC_COMPENSATED) return st_mul_f32<SV, CompAcc>(h, x, y, s);
    set_error("spmv_mul: the blocked product sums FP32 vectors with FP32 accumulators (plain, segmented or "
              "compensated)");
    return SPMV_ERR_UNSUPPORTED;
}

}  // namespace

spmv_status mul_stage_pattern_split(const spmv_matrix *h, const double *x, const float2 *x2, const uint32_t *xflag,
                                    double *y, cudaStream_t s) {
    SPMV_CUDA_TRY(cudaMemsetAsync(y, 0, (size_t)h->m * 8, s));
    if (!h->has_stage || h->stage_tiles == 0) return SPMV_OK;
    bool stage_ok = false;
    StArgs<Pattern, double> a = st_args<Pattern, double>(h, 8, x, y, &stage_ok);
    constexpr size_t slots = st_slots_bytes<DfAcc>();
    const size_t smem = slots + (stage_ok ? ((size_t)1 << h->stage_lb) * 8 : 0);
    static DeviceOnce attr;
    SPMV_TRY(attr([&] { return set_smem((const void *)k_hb_stage_f64<Pattern>, slots + ST_X_MAX); }));
    SPMV_LAUNCH("k_hb_stage", s, (k_hb_stage_f64<Pattern><<<(unsigned)h->stage_parts, ST_NW * 32, smem, s>>>(
                                      a, x, x2, xflag, 0)));
    SPMV_LAUNCH_CHECK("staged blocked pattern spmv");
    return SPMV_OK;
}

void free_stage(spmv_matrix *h, cudaStream_t s) {
    if (!h->has_stage) return;
    pagerank_forget(h);   // a captured PageRank graph may point into the layout
    dev_free_async(h->st_hdr, s);
    dev_free_async(h->st_words, s);
    dev_free_async(h->st_vals, s);
    dev_free_async(h->st_slice_tile, s);
    dev_free_async(h->st_lmeta, s);
    dev_free_async(h->st_part, s);
    h->st_lmeta = nullptr;
    h->st_part = nullptr;
    h->bytes -= h->stage_bytes;
    h->st_hdr = nullptr;
    h->st_words = nullptr;
    h->st_vals = nullptr;
    h->st_slice_tile = nullptr;
    h->stage_bytes = 0;
    h->stage_tiles = 0;
    h->has_stage = false;
}

spmv_status build_stage(spmv_matrix *h, int lb, cudaStream_t s) {
    free_stage(h, s);
    const int64_t m = h->m, n = h->n, nnz = h->nnz;
    const int64_t nsl = n > 0 ? ((n - 1) >> lb) + 1 : 0;
    const int64_t dmax = (int64_t)(0xFFFFFFFFu >> lb) - 1;
    int32_t kind = ST_NONE;
    size_t vs = 0;
    switch (h->dt) {
        case SPMV_F64: kind = h->df_ok ? ST_F2 : ST_F64; vs = 8; break;
        case SPMV_F32: kind = ST_F32; vs = 4; break;
        case SPMV_BF16: kind = ST_BF16; vs = 2; break;
        default: break;
    }
    DevBuf stile(s), hdr(s), words(s), vals(s), lmeta(s), part(s);
    int64_t ntiles = 0;
    int G = 0;
    if (nnz > 0 && nsl > 0) {
        DevBuf keys(s), keys_alt(s), perm(s), perm_alt(s), cnt(s), E(s), sstart(s), tiles(s), tmp(s);
        SPMV_TRY(keys.alloc((size_t)nnz * 8, "stage keys"));
        SPMV_TRY(keys_alt.alloc((size_t)nnz * 8, "stage keys"));
        SPMV_TRY(perm.alloc((size_t)nnz * 4, "stage perm"));
        SPMV_TRY(perm_alt.alloc((size_t)nnz * 4, "stage perm"));
        SPMV_TRY(cnt.alloc((size_t)(nnz + 1) * 4, "stage counts"));
        SPMV_TRY(E.alloc((size_t)(nnz + 1) * 4, "stage positions"));
        SPMV_TRY(sstart.alloc((size_t)(nsl + 1) * 4, "stage slice starts"));
        SPMV_TRY(tiles.alloc((size_t)(nsl + 1) * 4, "stage slice tiles"));
        SPMV_TRY(stile.alloc((size_t)(nsl + 1) * 4, "stage slice tiles"));
        SPMV_TRY(tmp.alloc(std::max(radix_temp_bytes(nnz), scan_temp_bytes(nnz + 1)), "stage sort temp"));
        SPMV_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, (size_t)(nnz + 1) * 4, s));
        if (m > 1) {
            SPMV_LAUNCH("k_st_rowflags", s, (k_st_rowflags<<<st_grid(m - 1), ST_CB, 0, s>>>(h->row_ptr, m, nnz,
                                                                                          cnt.as<uint32_t>())));
            SPMV_LAUNCH_CHECK("stage row flags");
        }
        SPMV_TRY(exclusive_scan_u32(cnt.as<uint32_t>(), E.as<uint32_t>(), nnz + 1, tmp.p, s));
        SPMV_LAUNCH("k_st_keys", s, (k_st_keys<<<st_grid(nnz), ST_CB, 0, s>>>(E.as<uint32_t>(), h->col, nnz,
                                                                             keys.as<uint64_t>(), perm.as<uint32_t>())));
        SPMV_LAUNCH_CHECK("stage keys");
        bool alt = false;
        SPMV_CUDA_TRY(cudaMemsetAsync(h->status_dev + 1, 0, 4, s));
        SPMV_TRY(radix_sort_pairs(keys.as<uint64_t>(), keys_alt.as<uint64_t>(), perm.as<uint32_t>(),
                                  perm_alt.as<uint32_t>(), nnz, lb, lb + bits_for(std::max<int64_t>(nsl, 2)), tmp.p, s, &alt,
                                  h->status_dev + 1));
        const uint64_t *Ks = alt ? keys_alt.as<uint64_t>() : keys.as<uint64_t>();
        const uint32_t *Ps = alt ? perm_alt.as<uint32_t>() : perm.as<uint32_t>();
        SPMV_LAUNCH("k_st_count", s, (k_st_count<<<st_grid(nnz + 1), ST_CB, 0, s>>>(
                                         Ks, nnz, nsl, lb, dmax, cnt.as<uint32_t>(),
                                         sstart.as<int32_t>())));
        SPMV_LAUNCH_CHECK("stage count");
        SPMV_TRY(exclusive_scan_u32(cnt.as<uint32_t>(), E.as<uint32_t>(), nnz + 1, tmp.p, s));
        SPMV_LAUNCH("k_st_slice_tiles", s, (k_st_slice_tiles<<<st_grid(nsl + 1), ST_CB, 0, s>>>(
                                               sstart.as<int32_t>(), E.as<uint32_t>(), nsl, tiles.as<uint32_t>())));
        SPMV_LAUNCH_CHECK("stage slice tiles");
        SPMV_TRY(exclusive_scan_u32(tiles.as<uint32_t>(), stile.as<uint32_t>(), nsl + 1, tmp.p, s));
        uint32_t back[2] = {0, 0};
        SPMV_CUDA_TRY(cudaMemcpyAsync(&back[0], stile.as<uint32_t>() + nsl, 4, cudaMemcpyDeviceToHost, s));
        SPMV_CUDA_TRY(cudaMemcpyAsync(&back[1], E.as<uint32_t>() + nnz, 4, cudaMemcpyDeviceToHost, s));
        SPMV_CUDA_TRY(cudaMemcpyAsync(h->status_host + 1, h->status_dev + 1, 4, cudaMemcpyDeviceToHost, s));
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
        if (h->status_host[1] & ST_TIMEOUT) {
            set_error("spmv_convert: a bounded wait of the radix sort gave up");
            return SPMV_ERR_TIMEOUT;
        }
        if ((uint64_t)back[1] + (uint64_t)nsl * ST_TILE >= ((uint64_t)1 << 31)) {
            set_error("spmv_convert: the blocked layout needs more than 2^31 slots");
            return SPMV_ERR_UNSUPPORTED;
        }
        ntiles = back[0];
        SPMV_TRY(hdr.alloc((size_t)ntiles * 16, "stage tile headers"));
        SPMV_CUDA_TRY(cudaMemsetAsync(hdr.p, 0, (size_t)ntiles * 16, s));
        SPMV_TRY(words.alloc((size_t)ntiles * ST_TILE * 4, "stage words"));
        SPMV_CUDA_TRY(cudaMemsetAsync(words.p, 0, (size_t)ntiles * ST_TILE * 4, s));
        if (vs) {
            SPMV_TRY(vals.alloc((size_t)ntiles * ST_TILE * vs, "stage values"));
            SPMV_CUDA_TRY(cudaMemsetAsync(vals.p, 0, (size_t)ntiles * ST_TILE * vs, s));
        }
        const uint32_t *Ep = E.as<uint32_t>(), *st = stile.as<uint32_t>();
        const int32_t *ss = sstart.as<int32_t>();
        uint32_t *w = words.as<uint32_t>();
        int4 *hp = hdr.as<int4>();
        switch (kind) {
            case ST_F2: SPMV_TRY((st_fill_launch<float2, double>(Ks, Ps, h, Ep, ss, st, lb, dmax, w, vals.p, hp, s))); break;
            case ST_F64: SPMV_TRY((st_fill_launch<double, double>(Ks, Ps, h, Ep, ss, st, lb, dmax, w, vals.p, hp, s))); break;
            case ST_F32: SPMV_TRY((st_fill_launch<float, float>(Ks, Ps, h, Ep, ss, st, lb, dmax, w, vals.p, hp, s))); break;
            case ST_BF16:
                SPMV_TRY((st_fill_launch<__nv_bfloat16, __nv_bfloat16>(Ks, Ps, h, Ep, ss, st, lb, dmax, w, vals.p, hp, s)));
                break;
            default: SPMV_TRY((st_fill_launch<Pattern, Pattern>(Ks, Ps, h, Ep, ss, st, lb, dmax, w, vals.p, hp, s))); break;
        }
        SPMV_LAUNCH("k_st_counts", s, (k_st_counts<<<st_grid(ntiles), ST_CB, 0, s>>>(ss, Ep, st, nsl, ntiles, hp)));
        SPMV_LAUNCH_CHECK("stage counts");
        SPMV_TRY(lmeta.alloc((size_t)ntiles * 32 * 8, "stage lane headers"));
        SPMV_LAUNCH("k_st_meta", s, (k_st_meta<<<st_grid(ntiles * 32), ST_CB, 0, s>>>(w, hp, ntiles, lb,
                                                                                    lmeta.as<uint2>())));
        SPMV_LAUNCH_CHECK("stage lane headers");
        SPMV_TRY(st_split(hp, ntiles, &part, &G, s));
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));   // the temporaries are freed in stream order next
    }
    h->st_slice_tile = (uint32_t *)stile.release();
    h->st_hdr = (int4 *)hdr.release();
    h->st_words = (uint32_t *)words.release();
    h->st_vals = vals.release();
    h->st_lmeta = (uint2 *)lmeta.release();
    h->st_part = (int32_t *)part.release();
    h->stage_parts = G;
    h->stage_lb = lb;
    h->stage_nsl = nsl;
    h->stage_tiles = ntiles;
    h->stage_kind = kind;
    h->stage_bytes = ntiles * (16 + 256 + ST_TILE * (4 + (int64_t)vs)) + (nsl + 1) * 4 + (G + 1) * 4;
    h->bytes += h->stage_bytes;
    h->has_stage = true;
    return SPMV_OK;
}

spmv_status stage_resplit(spmv_matrix *h, cudaStream_t s) {
    if (!h->has_stage || h->stage_tiles == 0) return SPMV_OK;
    pagerank_forget(h);   // the split array is replaced
    DevBuf part(s);
    int G = 0;
    SPMV_TRY(st_split(h->st_hdr, h->stage_tiles, &part, &G, s));
    if (h->st_part) dev_free_async(h->st_part, s);
    h->bytes += (int64_t)(G - h->stage_parts) * 4;
    h->st_part = (int32_t *)part.release();
    h->stage_parts = G;
    return SPMV_OK;
}

spmv_status mul_stage(const spmv_matrix *h, const void *x, void *y, spmv_dtype vdt, uint32_t acc, cudaStream_t s) {
    if (!h->has_stage) {
        set_error("spmv_mul: the blocked layout is missing (convert to HB first)");
        return SPMV_ERR_NOT_CONVERTED;
    }
    const int k = h->stage_kind;
    const bool ok64 = vdt == SPMV_F64 && (acc == SPMV_ACC_DEFAULT || acc == SPMV_ACC_F64) && k != ST_BF16;
    const bool ok32 = vdt == SPMV_F32 && (k == ST_F32 || k == ST_BF16 || k == ST_NONE) &&
                      (acc == SPMV_ACC_DEFAULT || acc == SPMV_ACC_F32 || acc == SPMV_ACC_SEGMENT ||
                       acc == SPMV_ACC_COMPENSATED);
    if (!ok64 && !ok32) goto unsupported;
    if (h->stage_tiles == 0 || vdt == SPMV_F32) {   // FP64 products zero y themselves
        SPMV_CUDA_TRY(cudaMemsetAsync(y, 0, (size_t)h->m * (vdt == SPMV_F64 ? 8 : 4), s));
        if (h->stage_tiles == 0) return SPMV_OK;
    }
    if (vdt == SPMV_F64) {
        const bool force = acc == SPMV_ACC_F64;
        switch (h->stage_kind) {
            case ST_F2: return st_mul_f64<float2>(h, (const double *)x, (double *)y, force, s);
            case ST_F64: return st_mul_f64<double>(h, (const double *)x, (double *)y, true, s);
            case ST_F32: return st_mul_f64<float>(h, (const double *)x, (double *)y, true, s);
            case ST_NONE: return st_mul_f64<Pattern>(h, (const double *)x, (double *)y, force, s);
            default: goto unsupported;
        }
    }
    if (vdt == SPMV_F32) {
        switch (h->stage_kind) {
            case ST_F32: return st_mul_f32_acc<float>(h, (const float *)x, (float *)y, acc, s);
            case ST_BF16: return st_mul_f32_acc<__nv_bfloat16>(h, (const float *)x, (float *)y, acc, s);
            case ST_NONE: return st_mul_f32_acc<Pattern>(h, (const float *)x, (float *)y, acc, s);
            default: goto unsupported;
        }
    }
unsupported:
    set_error("spmv_mul: unsupported combination of matrix dtype, vector dtype and accumulation for the blocked product");
    return SPMV_ERR_UNSUPPORTED;
}

}  // namespace spmv
