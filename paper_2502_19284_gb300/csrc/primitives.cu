// Device primitives for the format conversions (Section 5.1: a conversion is a sort into
// the format's order followed by one populate/compress pass):
//   * exclusive prefix sum over uint32 (reduce -> scan partials -> downsweep)
//   * stable LSD radix sort of (uint64 key, uint32 value) pairs, 8-bit digits.
// Both are written for sm_103a: coalesced tile loads, warp-synchronous ranking with
// __match_any_sync, shared-memory staging so that scattered outputs leave the SM as
// contiguous digit runs.
#include "common.cuh"

#include <algorithm>

namespace spmv {

namespace {

constexpr int SCAN_BLOCK = 256;
constexpr int SCAN_IPT = 16;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_IPT;

// Block-wide exclusive scan of one value per thread; returns the block total in *total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_tot[SCAN_BLOCK / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < SCAN_BLOCK / 32 ? warp_tot[lane] : 0;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < SCAN_BLOCK / 32) warp_tot[lane] = wi - w;   // exclusive warp offsets
        if (lane == SCAN_BLOCK / 32 - 1) *total = wi;
    }
    __syncthreads();
    uint32_t r = warp_tot[warp] + incl - v;
    __syncthreads();
    return r;
}

__global__ __launch_bounds__(SCAN_BLOCK) void k_scan_reduce(const uint32_t *__restrict__ in, int64_t n,
                                                            uint32_t *__restrict__ partial) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_IPT; ++j) {
        int64_t i = base + (int64_t)j * SCAN_BLOCK + threadIdx.x;
        if (i < n) s += in[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ uint32_t ws[SCAN_BLOCK / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < SCAN_BLOCK / 32; ++w) t += ws[w];
        partial[blockIdx.x] = t;
    }
}

// Exclusive scan of one tile, plus the tile's offset from the scanned partials.  The tile is
// staged in shared memory with one padding word per 32 (thread-contiguous runs of SCAN_IPT
// words then fall on distinct banks).
__device__ __forceinline__ int scan_pad(int i) { return i + (i >> 5); }

__global__ __launch_bounds__(SCAN_BLOCK) void k_scan_down(const uint32_t *__restrict__ in, uint32_t *__restrict__ out,
                                                          int64_t n, const uint32_t *__restrict__ offsets) {
    __shared__ uint32_t tile[SCAN_TILE + SCAN_TILE / 32];
    __shared__ uint32_t tot;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
#pragma unroll
    for (int j = 0; j < SCAN_IPT; ++j) {
        int64_t i = base + (int64_t)j * SCAN_BLOCK + threadIdx.x;
        tile[scan_pad(j * SCAN_BLOCK + threadIdx.x)] = i < n ? in[i] : 0u;
    }
    __syncthreads();
    uint32_t loc[SCAN_IPT];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_IPT; ++j) {
        loc[j] = s;
        s += tile[scan_pad(threadIdx.x * SCAN_IPT + j)];
    }
    uint32_t off = block_exclusive_scan(s, &tot) + (offsets ? offsets[blockIdx.x] : 0u);
#pragma unroll
    for (int j = 0; j < SCAN_IPT; ++j) tile[scan_pad(threadIdx.x * SCAN_IPT + j)] = loc[j] + off;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < SCAN_IPT; ++j) {
        int64_t i = base + (int64_t)j * SCAN_BLOCK + threadIdx.x;
        if (i < n) out[i] = tile[scan_pad(j * SCAN_BLOCK + threadIdx.x)];
    }
}

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace

size_t scan_temp_bytes(int64_t n) {
    size_t bytes = 0;
    int64_t nb = cdiv(n, SCAN_TILE);
    while (nb > 1) {
        bytes += (size_t)cdiv(nb * 4, 256) * 256;
        nb = cdiv(nb, SCAN_TILE);
    }
    return bytes + 256;
}

spmv_status exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, void *temp, cudaStream_t s) {
    if (n <= 0) return SPMV_OK;
    int64_t nb = cdiv(n, SCAN_TILE);
    if (nb == 1) {
        SPMV_LAUNCH("k_scan_down", s, (k_scan_down<<<1, SCAN_BLOCK, 0, s>>>(in, out, n, nullptr)));
        SPMV_LAUNCH_CHECK("scan");
        return SPMV_OK;
    }
    uint32_t *partial = (uint32_t *)temp;
    void *rest = (char *)temp + (size_t)cdiv(nb * 4, 256) * 256;
    SPMV_LAUNCH("k_scan_reduce", s, (k_scan_reduce<<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(in, n, partial)));
    SPMV_LAUNCH_CHECK("scan_reduce");
    SPMV_TRY(exclusive_scan_u32(partial, partial, nb, rest, s));
    SPMV_LAUNCH("k_scan_down", s, (k_scan_down<<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(in, out, n, partial)));
    SPMV_LAUNCH_CHECK("scan_down");
    return SPMV_OK;
}

// ====================================================================== radix sort
//
// Stable LSD radix sort of (uint64 key, uint32 value) pairs, 8-bit digits, three launches
// per digit and no inter-CTA waits:
//   count   per-tile digit counts (shared-memory atomics), stored digit-major;
//   scan    exclusive prefix sum of the digit-major counts = every tile's output offsets;
//   scatter each tile ranks its keys inside each warp in input order (warp ballots), places
//           keys and values in digit order in shared memory, and writes every digit run
//           contiguously.

namespace {

constexpr int RS_BLOCK = 256;
#ifndef RS_IPT_CFG
#define RS_IPT_CFG 8
#endif
#ifndef RS_MINB_CFG
#define RS_MINB_CFG 5
#endif
constexpr int RS_IPT = RS_IPT_CFG;   // keys per thread in a radix tile
constexpr int RS_TILE = RS_BLOCK * RS_IPT;
constexpr int RS_WARPS = RS_BLOCK / 32;
constexpr int RADIX = 256;
static_assert(RS_BLOCK == RADIX, "one thread per digit in the per-tile digit work");

#ifndef RS_MATCH_ANY
#define RS_MATCH_ANY 1   // rank with __match_any_sync (else with one ballot per digit bit)
#endif
#if !RS_MATCH_ANY
// Lanes of the warp holding the same 8-bit digit as this lane (ballot per digit bit).
__device__ __forceinline__ uint32_t digit_peers(uint32_t d, bool valid) {
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const uint32_t bit = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? bit : ~bit;
    }
    return peers;
}
#endif

// hist[d * ntiles + tile] = count of digit d in tile (same tiling as k_rs_scatter)
__global__ __launch_bounds__(RS_BLOCK) void k_rs_count(const uint64_t *__restrict__ keys, int64_t n, int shift,
                                                       uint32_t mask, uint32_t *__restrict__ hist, int64_t ntiles) {
    __shared__ uint32_t sh[RS_WARPS][RADIX];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = lane; d < RADIX; d += 32) sh[warp][d] = 0;
    __syncwarp();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    uint64_t k[RS_IPT];
#pragma unroll
    for (int j = 0; j < RS_IPT; ++j) {
        const int64_t i = base + (int64_t)j * RS_BLOCK + threadIdx.x;
        k[j] = i < n ? keys[i] : 0ull;
    }
#pragma unroll
    for (int j = 0; j < RS_IPT; ++j) {
        const int64_t i = base + (int64_t)j * RS_BLOCK + threadIdx.x;
        if (i < n) atomicAdd(&sh[warp][(uint32_t)(k[j] >> shift) & mask], 1u);
    }
    __syncthreads();
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) t += sh[w][threadIdx.x];
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = t;
}

// Stable scatter of one tile at the offsets of the scanned digit-major counts.  The tile's
// payloads are brought into shared memory by one bulk copy issued at the start (they are
// not needed until the keys are ranked), the keys are loaded into registers and ranked per
// warp in input order, keys and payloads are placed in digit order in shared memory, and
// every digit run is written out contiguously.
constexpr long long RS_SPIN_LIMIT = 1ll << 22;

__device__ __forceinline__ uint32_t rs_smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__global__ __launch_bounds__(RS_BLOCK, RS_MINB_CFG) void k_rs_scatter(const uint64_t *__restrict__ keys_in,
                                                            const uint32_t *__restrict__ vals_in,
                                                            uint64_t *__restrict__ keys_out,
                                                            uint32_t *__restrict__ vals_out, int64_t n, int shift,
                                                            uint32_t mask, const uint32_t *__restrict__ offsets,
                                                            int64_t ntiles, uint32_t *__restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *s_keys = (uint64_t *)smem_raw;
    uint32_t *s_vals = (uint32_t *)(s_keys + RS_TILE);
    uint32_t *s_vin = s_vals + RS_TILE;
    uint32_t *s_wcnt = s_vin + RS_TILE;
    uint32_t *s_dstart = s_wcnt + RS_WARPS * RADIX;
    uint32_t *s_gbase = s_dstart + RADIX;
    uint64_t *s_bar = (uint64_t *)(s_gbase + RADIX);
    __shared__ uint32_t s_wt[RS_WARPS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t tile_base = (int64_t)blockIdx.x * RS_TILE;
    const int tile_n = (int)min((int64_t)RS_TILE, n - tile_base);
    const bool bulk = tile_n == RS_TILE;   // a full tile: 16 KB of payloads, 16-byte aligned
    if (threadIdx.x == 0 && bulk) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(rs_smem_u32(s_bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(rs_smem_u32(s_bar)),
                     "r"((uint32_t)RS_TILE * 4u) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"(rs_smem_u32(s_vin)), "l"(vals_in + tile_base), "r"((uint32_t)RS_TILE * 4u),
                        "r"(rs_smem_u32(s_bar)) : "memory");
    }
    const int64_t wbase = tile_base + (int64_t)warp * (32 * RS_IPT);
    for (int d = lane; d < RADIX; d += 32) s_wcnt[warp * RADIX + d] = 0;
    const uint32_t gofs = offsets[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncwarp();
    uint64_t k[RS_IPT];
#pragma unroll
    for (int j = 0; j < RS_IPT; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        k[j] = i < n ? keys_in[i] : 0ull;
    }
    uint32_t dr[RS_IPT];
#pragma unroll
    for (int j = 0; j < RS_IPT; ++j) {
        const bool valid = wbase + j * 32 + lane < n;
        const uint32_t d = (uint32_t)(k[j] >> shift) & mask;
#if RS_MATCH_ANY
        const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 0x100u + (uint32_t)lane);
#else
        const uint32_t peers = digit_peers(d, valid);
#endif
        // the first lane of each peer group reserves the group's ranks with one shared-memory
        // atomic (issued in item order, so earlier items rank first) and hands out the base
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0u;
        if (valid && lane == leader) base = atomicAdd(&s_wcnt[warp * RADIX + d], (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader < 0 ? lane : leader);
        dr[j] = (d << 16) | (base + __popc(peers & lt_mask));
    }
    __syncthreads();
    const int d = threadIdx.x;
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
        const uint32_t c = s_wcnt[w * RADIX + d];
        s_wcnt[w * RADIX + d] = cnt;
        cnt += c;
    }
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_wt[warp] = incl;
    __syncthreads();
    uint32_t woff = 0;
    for (int w = 0; w < warp; ++w) woff += s_wt[w];
    const uint32_t dstart = woff + incl - cnt;
    s_dstart[d] = dstart;
    s_gbase[d] = gofs - dstart;
    __syncthreads();
    if (bulk) {   // the payloads have landed (bounded wait)
        uint32_t done = 0;
        for (long long it = 0; it < RS_SPIN_LIMIT && !done; ++it)
            asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
                         : "=r"(done) : "r"(rs_smem_u32(s_bar)) : "memory");
        if (!__syncthreads_and(done)) {
            if (threadIdx.x == 0) atomicOr(err, 4u);
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < RS_IPT; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        if (i < n) {
            const uint32_t dj = dr[j] >> 16;
            const uint32_t p = s_dstart[dj] + s_wcnt[warp * RADIX + dj] + (dr[j] & 0xFFFFu);
            s_keys[p] = k[j];
            s_vals[p] = bulk ? s_vin[i - tile_base] : vals_in[i];
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < tile_n; q += RS_BLOCK) {
        const uint64_t kk = s_keys[q];
        const uint32_t dq = (uint32_t)(kk >> shift) & mask;
        const int64_t o = (int64_t)s_gbase[dq] + q;
        keys_out[o] = kk;
        vals_out[o] = s_vals[q];
    }
}

constexpr size_t RS_SMEM = (size_t)RS_TILE * 16 + (size_t)RS_WARPS * RADIX * 4 + 2 * RADIX * 4 + 16;

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

size_t radix_temp_bytes(int64_t n) {
    const int64_t ntiles = cdiv(std::max<int64_t>(n, 1), RS_TILE);
    return align256((size_t)ntiles * RADIX * 4) + align256(scan_temp_bytes((int64_t)ntiles * RADIX)) + 256;
}

spmv_status radix_sort_pairs(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n,
                             int begin_bit, int end_bit, void *temp, cudaStream_t s, bool *in_alt, uint32_t *err) {
    *in_alt = false;
    if (n <= 1 || end_bit <= begin_bit) return SPMV_OK;
    static DeviceOnce attr_set;
    SPMV_TRY(attr_set([&] { return set_smem((const void *)k_rs_scatter, RS_SMEM); }));
    const int64_t ntiles = cdiv(n, RS_TILE);
    uint32_t *cnt = (uint32_t *)temp;
    void *scan_tmp = (char *)temp + align256((size_t)ntiles * RADIX * 4);
    if (!err)   // no status word of the caller: the last word of the scratch takes the flag
        err = (uint32_t *)((char *)scan_tmp + align256(scan_temp_bytes((int64_t)ntiles * RADIX)));
    uint64_t *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        const uint32_t mask = (1u << std::min(8, end_bit - shift)) - 1u;
        SPMV_LAUNCH("k_rs_count", s, (k_rs_count<<<(unsigned)ntiles, RS_BLOCK, 0, s>>>(ka, n, shift, mask, cnt, ntiles)));
        SPMV_LAUNCH_CHECK("radix count");
        SPMV_TRY(exclusive_scan_u32(cnt, cnt, (int64_t)RADIX * ntiles, scan_tmp, s));
        SPMV_LAUNCH("k_rs_scatter", s,
                    (k_rs_scatter<<<(unsigned)ntiles, RS_BLOCK, RS_SMEM, s>>>(ka, va, kb, vb, n, shift, mask, cnt, ntiles,
                                                                               err)));
        SPMV_LAUNCH_CHECK("radix scatter");
        std::swap(ka, kb);
        std::swap(va, vb);
        *in_alt = !*in_alt;
    }
    return SPMV_OK;
}

}  // namespace spmv
