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

__host__ __device__ __forceinline__ uint64_t hilbert_key(int K, uint32_t r, uint32_t c) {
    uint64_t d = 0;
    uint32_t st = 0;
    for (int lev = K - 1; lev >= 0; --lev) {
        uint32_t q = (((r >> lev) & 1u) << 1) | ((c >> lev) & 1u);
        uint32_t e = (uint32_t)(HILBERT_FWD >> (4 * (4 * st + q))) & 0xFu;
        d = (d << 2) | (e >> 2);
        st = e & 3u;
    }
    return d;
}

__host__ __device__ __forceinline__ void hilbert_cell(int K, uint64_t d, uint32_t *r, uint32_t *c) {
    uint32_t rr = 0, cc = 0, st = 0;
    for (int lev = K - 1; lev >= 0; --lev) {
        uint32_t dig = (uint32_t)(d >> (2 * lev)) & 3u;
        uint32_t e = (uint32_t)(HILBERT_INV >> (4 * (4 * st + dig))) & 0xFu;
        uint32_t q = e >> 2;
        rr |= (q >> 1) << lev;
        cc |= (q & 1u) << lev;
        st = e & 3u;
    }
    *r = rr;
    *c = cc;
}

// Two levels per step.  fwd2[16 * state + (r1 c1 r0 c0)] = (d1 d0) << 2 | next and
// inv2[16 * state + (d1 d0)] = (r1 c1 r0 c0) << 2 | next (bit pairs of two consecutive
// levels, the higher level first), both derived from the one-level machine above.  Call
// hilbert_tables2 from 64 threads of a block (entry = threadIdx.x) before use.
__device__ __forceinline__ void hilbert_tables2(uint8_t *fwd2, uint8_t *inv2, int entry) {
    const uint32_t st = (uint32_t)entry >> 4, in = (uint32_t)entry & 15u;
    {   // forward: input bits r1 c1 r0 c0
        const uint32_t q1 = ((in >> 3) & 1u) << 1 | ((in >> 2) & 1u), q0 = ((in >> 1) & 1u) << 1 | (in & 1u);
        const uint32_t e1 = (uint32_t)(HILBERT_FWD >> (4 * (4 * st + q1))) & 0xFu;
        const uint32_t e0 = (uint32_t)(HILBERT_FWD >> (4 * (4 * (e1 & 3u) + q0))) & 0xFu;
        fwd2[entry] = (uint8_t)((((e1 >> 2) << 2 | (e0 >> 2)) << 2) | (e0 & 3u));
    }
    {   // inverse: input digits d1 d0
        const uint32_t d1 = in >> 2, d0 = in & 3u;
        const uint32_t e1 = (uint32_t)(HILBERT_INV >> (4 * (4 * st + d1))) & 0xFu;
        const uint32_t e0 = (uint32_t)(HILBERT_INV >> (4 * (4 * (e1 & 3u) + d0))) & 0xFu;
        const uint32_t q1 = e1 >> 2, q0 = e0 >> 2;
        const uint32_t bits = ((q1 >> 1) << 3) | ((q1 & 1u) << 2) | ((q0 >> 1) << 1) | (q0 & 1u);
        inv2[entry] = (uint8_t)((bits << 2) | (e0 & 3u));
    }
}

__device__ __forceinline__ uint64_t hilbert_key2(int K, uint32_t r, uint32_t c, const uint8_t *fwd2) {
    uint64_t d = 0;
    uint32_t st = 0;
    int lev = K;
    if (lev & 1) {   // odd order: one single level first
        --lev;
        const uint32_t q = (((r >> lev) & 1u) << 1) | ((c >> lev) & 1u);
        const uint32_t e = (uint32_t)(HILBERT_FWD >> (4 * q)) & 0xFu;   // state 0
        d = e >> 2;
        st = e & 3u;
    }
    while (lev > 0) {
        lev -= 2;
        const uint32_t rb = (r >> lev) & 3u, cb = (c >> lev) & 3u;
        const uint32_t in = ((rb >> 1) << 3) | ((cb >> 1) << 2) | ((rb & 1u) << 1) | (cb & 1u);
        const uint32_t e = fwd2[(st << 4) | in];
        d = (d << 4) | (e >> 2);
        st = e & 3u;
    }
    return d;
}

__device__ __forceinline__ void hilbert_cell2(int K, uint64_t d, uint32_t *r, uint32_t *c, const uint8_t *inv2) {
    uint32_t rr = 0, cc = 0, st = 0;
    int lev = K;
    if (lev & 1) {
        --lev;
        const uint32_t dig = (uint32_t)(d >> (2 * lev)) & 3u;
        const uint32_t e = (uint32_t)(HILBERT_INV >> (4 * dig)) & 0xFu;   // state 0
        rr = (e >> 3) & 1u;
        cc = (e >> 2) & 1u;
        st = e & 3u;
    }
    while (lev > 0) {
        lev -= 2;
        const uint32_t dd = (uint32_t)(d >> (2 * lev)) & 15u;
        const uint32_t e = inv2[(st << 4) | dd];
        const uint32_t bits = e >> 2;   // r1 c1 r0 c0
        rr = (rr << 2) | ((bits >> 3) << 1) | ((bits >> 1) & 1u);
        cc = (cc << 2) | (((bits >> 2) & 1u) << 1) | (bits & 1u);
        st = e & 3u;
    }
    *r = rr;
    *c = cc;
}

// U independent cells at once: the dependent table lookups of the U chains are
// interleaved, so one thread keeps U of them in flight.
template <int U>
__device__ __forceinline__ void hilbert_cell2_n(int K, const uint64_t *d, uint32_t *r, uint32_t *c,
                                                const uint8_t *inv2) {
    uint32_t st[U];
    int lev = K;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        r[u] = 0;
        c[u] = 0;
        st[u] = 0;
    }
    if (lev & 1) {
        --lev;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t dig = (uint32_t)(d[u] >> (2 * lev)) & 3u;
            const uint32_t e = (uint32_t)(HILBERT_INV >> (4 * dig)) & 0xFu;   // state 0
            r[u] = (e >> 3) & 1u;
            c[u] = (e >> 2) & 1u;
            st[u] = e & 3u;
        }
    }
    while (lev > 0) {
        lev -= 2;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t dd = (uint32_t)(d[u] >> (2 * lev)) & 15u;
            const uint32_t e = inv2[(st[u] << 4) | dd];
            const uint32_t bits = e >> 2;   // r1 c1 r0 c0
            r[u] = (r[u] << 2) | ((bits >> 3) << 1) | ((bits >> 1) & 1u);
            c[u] = (c[u] << 2) | (((bits >> 2) & 1u) << 1) | (bits & 1u);
            st[u] = e & 3u;
        }
    }
}

}  // namespace spmv
