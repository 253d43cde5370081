// Hilbert-curve index on the 2^K x 2^K grid, as a bit-serial state machine.
//
// The curve (Section 3.2 and its figure) enters at the top-left cell and leaves at the
// top-right one; at every level the four quadrants are visited top-left, bottom-left,
// bottom-right, top-right, with the top-left sub-curve transposed and the top-right one
// anti-transposed.  Tracking the accumulated orientation as one of four symmetries of
// the square {identity, transpose, anti-transpose, half-turn} gives a 4-state automaton:
// per level, the state and the (row bit, col bit) pair select the curve digit and the
// next state.  Both tables are packed into 64-bit immediates: entry (state, input) sits
// at bit 4*(4*state + input) as (digit << 2) | next.
#pragma once
#include <stdint.h>

namespace spmv {

// forward: input = (row bit << 1) | col bit  ->  (digit << 2) | next state
//   state 0 (identity):       q0:d0>1  q1:d3>2  q2:d1>0  q3:d2>0
//   state 1 (transpose):      q0:d0>0  q1:d1>1  q2:d3>3  q3:d2>1
//   state 2 (anti-transpose): q0:d2>2  q1:d3>0  q2:d1>2  q3:d0>3
//   state 3 (half-turn):      q0:d2>3  q1:d1>3  q2:d3>1  q3:d0>2
constexpr uint64_t HILBERT_FWD =
    ((uint64_t)((0 << 2) | 1) << 0) | ((uint64_t)((3 << 2) | 2) << 4) | ((uint64_t)((1 << 2) | 0) << 8) |
    ((uint64_t)((2 << 2) | 0) << 12) |
    ((uint64_t)((0 << 2) | 0) << 16) | ((uint64_t)((1 << 2) | 1) << 20) | ((uint64_t)((3 << 2) | 3) << 24) |
    ((uint64_t)((2 << 2) | 1) << 28) |
    ((uint64_t)((2 << 2) | 2) << 32) | ((uint64_t)((3 << 2) | 0) << 36) | ((uint64_t)((1 << 2) | 2) << 40) |
    ((uint64_t)((0 << 2) | 3) << 44) |
    ((uint64_t)((2 << 2) | 3) << 48) | ((uint64_t)((1 << 2) | 3) << 52) | ((uint64_t)((3 << 2) | 1) << 56) |
    ((uint64_t)((0 << 2) | 2) << 60);

// inverse: entry (state, digit) = (input << 2) | next state
//   state 0: d0:q0>1  d1:q2>0  d2:q3>0  d3:q1>2
//   state 1: d0:q0>0  d1:q1>1  d2:q3>1  d3:q2>3
//   state 2: d0:q3>3  d1:q2>2  d2:q0>2  d3:q1>0
//   state 3: d0:q3>2  d1:q1>3  d2:q0>3  d3:q2>1
constexpr uint64_t HILBERT_INV =
    ((uint64_t)((0 << 2) | 1) << 0) | ((uint64_t)((2 << 2) | 0) << 4) | ((uint64_t)((3 << 2) | 0) << 8) |
    ((uint64_t)((1 << 2) | 2) << 12) |
    ((uint64_t)((0 << 2) | 0) << 16) | ((uint64_t)((1 << 2) | 1) << 20) | ((uint64_t)((3 << 2) | 1) << 24) |
    ((uint64_t)((2 << 2) | 3) << 28) |
    ((uint64_t)((3 << 2) | 3) << 32) | ((uint64_t)((2 << 2) | 2) << 36) | ((uint64_t)((0 << 2) | 2) << 40) |
    ((uint64_t)((1 << 2) | 0) << 44) |
    ((uint64_t)((3 << 2) | 2) << 48) | ((uint64_t)((1 << 2) | 3) << 52) | ((uint64_t)((0 << 2) | 3) << 56) |
    ((uint64_t)((2 << 2) | 1) << 60);

// One level per step, straight from the packed machine (for the few cells that do not pay
// for staging a table).
__host__ __device__ __forceinline__ void hilbert_cell1(int K, uint64_t d, uint32_t *r, uint32_t *c) {
    uint32_t rr = 0, cc = 0, st = 0;
    for (int lev = K - 1; lev >= 0; --lev) {
        const uint32_t dd = (uint32_t)(d >> (2 * lev)) & 3u;
        const uint32_t x = (uint32_t)(HILBERT_INV >> (4 * (4 * st + dd))) & 0xFu;
        rr = (rr << 1) | (x >> 3);
        cc = (cc << 1) | ((x >> 2) & 1u);
        st = x & 3u;
    }
    *r = rr;
    *c = cc;
}

// Four levels per step:
//   fwd[256 * state + (r3 r2 r1 r0) * 16 + (c3 c2 c1 c0)] = (d3 d2 d1 d0) << 2 | next
//   inv[256 * state + (d3 d2 d1 d0)] = ((r3 r2 r1 r0) * 16 + (c3 c2 c1 c0)) << 2 | next
// (four row bits, four column bits, two bits per digit; the higher level first), both
// composed from the one-level machine above at compile time.  Kernels copy the table they
// need into shared memory first (hilbert_stage).
struct Hilbert4 {
    uint16_t fwd[1024];
    uint16_t inv[1024];
    constexpr Hilbert4() : fwd(), inv() {
        for (int e = 0; e < 1024; ++e) {
            const uint32_t st0 = (uint32_t)e >> 8, r4 = ((uint32_t)e >> 4) & 15u, c4 = (uint32_t)e & 15u;
            uint32_t st = st0, dg = 0;
            for (int l = 3; l >= 0; --l) {   // forward: consume (r, c) bit pairs, highest level first
                const uint32_t q = (((r4 >> l) & 1u) << 1) | ((c4 >> l) & 1u);
                const uint32_t x = (uint32_t)(HILBERT_FWD >> (4 * (4 * st + q))) & 0xFu;
                dg = (dg << 2) | (x >> 2);
                st = x & 3u;
            }
            fwd[e] = (uint16_t)((dg << 2) | st);
            const uint32_t d8 = (uint32_t)e & 255u;
            uint32_t rr = 0, cc = 0;
            st = st0;
            for (int l = 3; l >= 0; --l) {   // inverse: consume digits, highest level first
                const uint32_t dd = (d8 >> (2 * l)) & 3u;
                const uint32_t x = (uint32_t)(HILBERT_INV >> (4 * (4 * st + dd))) & 0xFu;
                rr = (rr << 1) | (x >> 3);
                cc = (cc << 1) | ((x >> 2) & 1u);
                st = x & 3u;
            }
            inv[e] = (uint16_t)((((rr << 4) | cc) << 2) | st);
        }
    }
};
static __device__ const Hilbert4 g_hilbert4 = Hilbert4();

// Copy one 2 KB table into shared memory (16 bytes per thread); the block synchronises
// before use.
__device__ __forceinline__ void hilbert_stage(uint16_t *dst, const uint16_t *src) {
    for (int i = threadIdx.x; i < 1024 / 8; i += blockDim.x) ((uint4 *)dst)[i] = ((const uint4 *)src)[i];
}

__device__ __forceinline__ uint64_t hilbert_key4(int K, uint32_t r, uint32_t c, const uint16_t *fwd4) {
    uint64_t d = 0;
    uint32_t st = 0;
    int lev = K;
    while (lev & 3) {   // the top K mod 4 levels one at a time
        --lev;
        const uint32_t q = (((r >> lev) & 1u) << 1) | ((c >> lev) & 1u);
        const uint32_t x = (uint32_t)(HILBERT_FWD >> (4 * (4 * st + q))) & 0xFu;
        d = (d << 2) | (x >> 2);
        st = x & 3u;
    }
    while (lev > 0) {
        lev -= 4;
        const uint32_t x = fwd4[(st << 8) | (((r >> lev) & 15u) << 4) | ((c >> lev) & 15u)];
        d = (d << 8) | (x >> 2);
        st = x & 3u;
    }
    return d;
}

// U keys at once, the levels outermost: the U table lookups of a level are independent.
template <int U>
__device__ __forceinline__ void hilbert_key4_n(int K, const uint32_t *r, const uint32_t *c, const uint16_t *fwd4,
                                               uint64_t *d) {
    uint32_t st[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        d[u] = 0;
        st[u] = 0;
    }
    int lev = K;
    while (lev & 3) {
        --lev;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t q = (((r[u] >> lev) & 1u) << 1) | ((c[u] >> lev) & 1u);
            const uint32_t x = (uint32_t)(HILBERT_FWD >> (4 * (4 * st[u] + q))) & 0xFu;
            d[u] = (d[u] << 2) | (x >> 2);
            st[u] = x & 3u;
        }
    }
    while (lev > 0) {
        lev -= 4;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t x = fwd4[(st[u] << 8) | (((r[u] >> lev) & 15u) << 4) | ((c[u] >> lev) & 15u)];
            d[u] = (d[u] << 8) | (x >> 2);
            st[u] = x & 3u;
        }
    }
}

__device__ __forceinline__ void hilbert_cell4(int K, uint64_t d, uint32_t *r, uint32_t *c, const uint16_t *inv4) {
    uint32_t rr = 0, cc = 0, st = 0;
    int lev = K;
    while (lev & 3) {
        --lev;
        const uint32_t dd = (uint32_t)(d >> (2 * lev)) & 3u;
        const uint32_t x = (uint32_t)(HILBERT_INV >> (4 * (4 * st + dd))) & 0xFu;
        rr = (rr << 1) | (x >> 3);
        cc = (cc << 1) | ((x >> 2) & 1u);
        st = x & 3u;
    }
    while (lev > 0) {
        lev -= 4;
        const uint32_t x = inv4[(st << 8) | ((uint32_t)(d >> (2 * lev)) & 255u)];
        rr = (rr << 4) | (x >> 6);
        cc = (cc << 4) | ((x >> 2) & 15u);
        st = x & 3u;
    }
    *r = rr;
    *c = cc;
}

// U cells at once, the levels outermost.
template <int U>
__device__ __forceinline__ void hilbert_cell4_n(int K, const uint64_t *d, uint32_t *r, uint32_t *c,
                                                const uint16_t *inv4) {
    uint32_t st[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        r[u] = 0;
        c[u] = 0;
        st[u] = 0;
    }
    int lev = K;
    while (lev & 3) {
        --lev;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t dd = (uint32_t)(d[u] >> (2 * lev)) & 3u;
            const uint32_t x = (uint32_t)(HILBERT_INV >> (4 * (4 * st[u] + dd))) & 0xFu;
            r[u] = (r[u] << 1) | (x >> 3);
            c[u] = (c[u] << 1) | ((x >> 2) & 1u);
            st[u] = x & 3u;
        }
    }
    while (lev > 0) {
        lev -= 4;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t x = inv4[(st[u] << 8) | ((uint32_t)(d[u] >> (2 * lev)) & 255u)];
            r[u] = (r[u] << 4) | (x >> 6);
            c[u] = (c[u] << 4) | ((x >> 2) & 15u);
            st[u] = x & 3u;
        }
    }
}

}  // namespace spmv
