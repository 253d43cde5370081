/*
 * GPU twin of synth.c's R-MAT edge and value draws, for inputs too large to generate on the
 * host in benchmark time (thousands of millions of edges).  INPUT GENERATION ONLY: no format
 * conversion, no product.  Every draw is the same counter-based SplitMix64 output as in synth.c
 * (Steele, Lea and Flood, OOPSLA 2014: the 64-bit finaliser applied to key + (ctr + 1) * gamma,
 * stream keys derived from (seed, stream id) the same way), so an edge list or value array
 * drawn here equals the host's bit for bit (checked by the tests on a sample).
 *
 * Raw edges: duplicates are not removed here; a caller that needs a set removes them (or
 * ingests the triplets with duplicates summed, as the library's default does).
 */
#include <cuda_runtime.h>
#include <stdint.h>

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

__device__ __forceinline__ uint64_t g_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t g_draw(uint64_t key, uint64_t ctr) { return g_mix64(key + (ctr + 1) * GOLDEN_GAMMA); }
__device__ __forceinline__ double g_u01(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

static uint64_t h_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static uint64_t h_stream_key(uint64_t seed, uint64_t stream) {
    return h_mix64(h_mix64(seed ^ 0x5851F42D4C957F2DULL) + stream * GOLDEN_GAMMA);
}

enum { STREAM_EDGES = 1, STREAM_VALUES = 2, STREAM_VECTOR = 3 };

__global__ void k_rmat(int K, int64_t edges, uint64_t key, double a, double ab, double abc, int32_t *rows,
                       int32_t *cols) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= edges) return;
    uint32_t r = 0, c = 0;
    for (int lev = K - 1; lev >= 0; --lev) {
        const double u = g_u01(g_draw(key, (uint64_t)e * (uint64_t)K + (uint64_t)(K - 1 - lev)));
        uint32_t rb, cb;
        if (u < a) { rb = 0; cb = 0; }
        else if (u < ab) { rb = 0; cb = 1; }
        else if (u < abc) { rb = 1; cb = 0; }
        else { rb = 1; cb = 1; }
        r |= rb << lev;
        c |= cb << lev;
    }
    rows[e] = (int32_t)r;
    cols[e] = (int32_t)c;
}

__device__ __forceinline__ double g_value(uint64_t r, int kind) {
    const double u = g_u01(r);
    return kind == 0 ? 2.0 * u - 1.0 : floor(17.0 * u) - 8.0;
}

__global__ void k_values(int64_t n, const int32_t *rows, const int32_t *cols, uint64_t key, int kind, int f32,
                         void *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t rc = ((uint64_t)(uint32_t)rows[i] << 32) | (uint32_t)cols[i];
    const double v = g_value(g_draw(key, rc), kind);
    if (f32) ((float *)out)[i] = __double2float_rn(v);
    else ((double *)out)[i] = v;
}

static unsigned blocks(int64_t n) { return (unsigned)((n + 255) / 256); }

extern "C" {

/* Raw R-MAT edges (no deduplication) into device arrays rows/cols of `edges` entries, on
 * `stream`.  Edge e equals edge e of synth_rmat before its duplicate removal. */
int synth_gpu_rmat(int scale, int64_t edges, double a, double b, double c, uint64_t seed, int32_t *rows,
                   int32_t *cols, void *stream) {
    if (edges <= 0) return 0;
    k_rmat<<<blocks(edges), 256, 0, (cudaStream_t)stream>>>(scale, edges, h_stream_key(seed, STREAM_EDGES), a, a + b,
                                                           a + b + c, rows, cols);
    return (int)cudaGetLastError();
}

/* Values v(seed, r, c) (kind 0: U[-1,1); 1: integers in [-8,8]) as doubles or, with f32 != 0,
 * rounded to float (nearest even); device arrays, on `stream`. */
int synth_gpu_values(int64_t n, const int32_t *rows, const int32_t *cols, uint64_t seed, int kind, int f32, void *out,
                     void *stream) {
    if (n <= 0) return 0;
    k_values<<<blocks(n), 256, 0, (cudaStream_t)stream>>>(n, rows, cols, h_stream_key(seed, STREAM_VALUES), kind, f32,
                                                          out);
    return (int)cudaGetLastError();
}

}
