/*
 * Seeded synthetic input generators for the SpMV library's tests and benchmark.
 *
 * This file produces INPUTS only (sparse patterns, matrix values, dense vectors).
 * It holds none of the SpMV method's arithmetic: no format conversion, no product.
 * Both the oracle tests and the CUDA path draw their inputs from here.
 *
 * Random numbers: counter-based SplitMix64 (G. L. Steele, D. Lea, C. H. Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014): the 64-bit
 * finaliser applied to  key + (counter + 1) * 0x9E3779B97F4A7C15.
 * Every draw is a pure function of (seed, stream, counter), so the output is
 * independent of thread count and of generation order.
 *
 * Generators (inputs standing in for the paper's test set of power-law and
 * random unstructured matrices, Section 5.2):
 *   - R-MAT (Graph500 parameters a/b/c/d), duplicate edges removed, first
 *     occurrence kept, output in edge order;
 *   - Erdos-Renyi with exactly `per_row` distinct uniform columns per row;
 *   - power-law rows: Zipf(alpha) row lengths capped, a fraction of empty rows,
 *     distinct uniform columns.
 * Values are a function of (seed, row, col) so they do not depend on edge order
 * or on deduplication; dense vectors are a function of (seed, index).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* One SplitMix64 output for position `ctr` of the stream keyed by `key`. */
uint64_t synth_draw(uint64_t key, uint64_t ctr) { return mix64(key + (ctr + 1) * GOLDEN_GAMMA); }

/* Stream key for (seed, stream id). */
uint64_t synth_stream_key(uint64_t seed, uint64_t stream) {
    return mix64(mix64(seed ^ 0x5851F42D4C957F2DULL) + stream * GOLDEN_GAMMA);
}

/* Uniform double in [0,1) from the top 53 bits. */
static inline double u01(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* Uniform integer in [0, n) (multiply-high, no modulo bias beyond 2^-64). */
static inline uint64_t below(uint64_t r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)r * (unsigned __int128)n) >> 64);
}

enum { STREAM_EDGES = 1, STREAM_VALUES = 2, STREAM_VECTOR = 3, STREAM_ER = 4,
       STREAM_ZLEN = 5, STREAM_ZEMPTY = 6, STREAM_ZCOL = 7 };

/* ------------------------------------------------------------------ threads */
typedef struct {
    void (*fn)(void *, int64_t, int64_t);
    void *arg;
    int64_t lo, hi;
} job_t;

static void *job_run(void *p) {
    job_t *j = (job_t *)p;
    j->fn(j->arg, j->lo, j->hi);
    return NULL;
}

static int g_threads = 0;
void synth_set_threads(int t) { g_threads = t; }

static int n_threads(void) {
    if (g_threads > 0) return g_threads;
    const char *e = getenv("SYNTH_THREADS");
    if (e && atoi(e) > 0) return atoi(e);
    return 8;
}

/* Run fn over [0, n) split into contiguous ranges; results are independent of
 * the split because every draw is counter-based. */
static void parallel_for(int64_t n, void (*fn)(void *, int64_t, int64_t), void *arg) {
    int t = n_threads();
    if (t > 64) t = 64;
    if (n < 65536 || t <= 1) { fn(arg, 0, n); return; }
    pthread_t th[64];
    job_t jobs[64];
    for (int i = 0; i < t; ++i) {
        jobs[i].fn = fn; jobs[i].arg = arg;
        jobs[i].lo = n * i / t; jobs[i].hi = n * (i + 1) / t;
        if (pthread_create(&th[i], NULL, job_run, &jobs[i]) != 0) {
            /* fall back to running inline */
            job_run(&jobs[i]);
            th[i] = 0;
        }
    }
    for (int i = 0; i < t; ++i) if (th[i]) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------------- R-MAT */
typedef struct {
    int scale; uint64_t key; double a, ab, abc;
    int32_t *rows, *cols;
} rmat_arg;

static void rmat_body(void *p, int64_t lo, int64_t hi) {
    rmat_arg *g = (rmat_arg *)p;
    const int K = g->scale;
    for (int64_t e = lo; e < hi; ++e) {
        uint32_t r = 0, c = 0;
        for (int lev = K - 1; lev >= 0; --lev) {
            double u = u01(synth_draw(g->key, (uint64_t)e * (uint64_t)K + (uint64_t)(K - 1 - lev)));
            uint32_t rb, cb;
            if (u < g->a) { rb = 0; cb = 0; }
            else if (u < g->ab) { rb = 0; cb = 1; }
            else if (u < g->abc) { rb = 1; cb = 0; }
            else { rb = 1; cb = 1; }
            r |= rb << lev; c |= cb << lev;
        }
        g->rows[e] = (int32_t)r; g->cols[e] = (int32_t)c;
    }
}

/* LSD radix sort of (key, idx) pairs, 16-bit digits, over the low `bits` bits. */
static int sort_pairs(uint64_t *key, uint32_t *idx, int64_t n, int bits) {
    uint64_t *k2 = (uint64_t *)malloc((size_t)n * 8);
    uint32_t *i2 = (uint32_t *)malloc((size_t)n * 4);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * 65536);
    if (!k2 || !i2 || !cnt) { free(k2); free(i2); free(cnt); return -1; }
    uint64_t *ka = key, *kb = k2; uint32_t *ia = idx, *ib = i2;
    for (int sh = 0; sh < bits; sh += 16) {
        memset(cnt, 0, sizeof(int64_t) * 65536);
        for (int64_t i = 0; i < n; ++i) cnt[(ka[i] >> sh) & 0xFFFF]++;
        int64_t s = 0;
        for (int d = 0; d < 65536; ++d) { int64_t c = cnt[d]; cnt[d] = s; s += c; }
        for (int64_t i = 0; i < n; ++i) {
            int64_t p = cnt[(ka[i] >> sh) & 0xFFFF]++;
            kb[p] = ka[i]; ib[p] = ia[i];
        }
        uint64_t *tk = ka; ka = kb; kb = tk;
        uint32_t *ti = ia; ia = ib; ib = ti;
    }
    if (ka != key) { memcpy(key, ka, (size_t)n * 8); memcpy(idx, ia, (size_t)n * 4); }
    free(k2); free(i2); free(cnt);
    return 0;
}

/*
 * R-MAT edge list with 2^scale vertices and `edges` draws.  For each edge and each
 * level (most significant first) one uniform draw picks the quadrant:
 * u < a -> (0,0), < a+b -> (0,1), < a+b+c -> (1,0), else (1,1).
 * No noise, no vertex permutation; self loops kept.  Duplicates are removed,
 * keeping the first occurrence, and the survivors stay in edge order.
 * rows/cols must hold `edges` entries.  Returns the number kept, or -1 on OOM.
 */
int64_t synth_rmat(int scale, int64_t edges, double a, double b, double c, uint64_t seed,
                   int32_t *rows, int32_t *cols) {
    rmat_arg g = {scale, synth_stream_key(seed, STREAM_EDGES), a, a + b, a + b + c, rows, cols};
    parallel_for(edges, rmat_body, &g);
    uint64_t *key = (uint64_t *)malloc((size_t)edges * 8);
    uint32_t *idx = (uint32_t *)malloc((size_t)edges * 4);
    uint8_t *keep = (uint8_t *)calloc((size_t)edges, 1);
    if (!key || !idx || !keep) { free(key); free(idx); free(keep); return -1; }
    for (int64_t e = 0; e < edges; ++e) {
        key[e] = ((uint64_t)(uint32_t)rows[e] << scale) | (uint64_t)(uint32_t)cols[e];
        idx[e] = (uint32_t)e;
    }
    if (sort_pairs(key, idx, edges, 2 * scale) != 0) { free(key); free(idx); free(keep); return -1; }
    /* stable sort: the first of each run of equal keys is the earliest edge */
    for (int64_t i = 0; i < edges; ++i)
        if (i == 0 || key[i] != key[i - 1]) keep[idx[i]] = 1;
    int64_t w = 0;
    for (int64_t e = 0; e < edges; ++e)
        if (keep[e]) { rows[w] = rows[e]; cols[w] = cols[e]; ++w; }
    free(key); free(idx); free(keep);
    return w;
}

/* R-MAT edges exactly as drawn, duplicates kept (the first step of synth_rmat). */
void synth_rmat_raw(int scale, int64_t edges, double a, double b, double c, uint64_t seed, int32_t *rows,
                    int32_t *cols) {
    rmat_arg g = {scale, synth_stream_key(seed, STREAM_EDGES), a, a + b, a + b + c, rows, cols};
    parallel_for(edges, rmat_body, &g);
}

/* ------------------------------------------------------------------ values */
typedef struct { uint64_t key; int kind; const int32_t *rows, *cols; double *out; } val_arg;

static inline double value_of(uint64_t r, int kind) {
    double u = u01(r);
    if (kind == 0) return 2.0 * u - 1.0;           /* uniform [-1, 1)        */
    return floor(17.0 * u) - 8.0;                  /* integer in [-8, 8]     */
}

static void val_body(void *p, int64_t lo, int64_t hi) {
    val_arg *g = (val_arg *)p;
    for (int64_t i = lo; i < hi; ++i) {
        uint64_t rc = ((uint64_t)(uint32_t)g->rows[i] << 32) | (uint32_t)g->cols[i];
        g->out[i] = value_of(synth_draw(g->key, rc), g->kind);
    }
}

/* Matrix values as a function of (seed, row, col).  kind 0: U[-1,1); 1: integer [-8,8]. */
void synth_values(int64_t nnz, const int32_t *rows, const int32_t *cols, uint64_t seed, int kind,
                  double *out) {
    val_arg g = {synth_stream_key(seed, STREAM_VALUES), kind, rows, cols, out};
    parallel_for(nnz, val_body, &g);
}

typedef struct { uint64_t key; int kind; double *out; } vec_arg;
static void vec_body(void *p, int64_t lo, int64_t hi) {
    vec_arg *g = (vec_arg *)p;
    for (int64_t i = lo; i < hi; ++i) g->out[i] = value_of(synth_draw(g->key, (uint64_t)i), g->kind);
}

/* Dense vector x_j as a function of (seed, j); same kinds as synth_values. */
void synth_vector(int64_t n, uint64_t seed, int kind, double *out) {
    vec_arg g = {synth_stream_key(seed, STREAM_VECTOR), kind, out};
    parallel_for(n, vec_body, &g);
}

/* -------------------------------------------------------------- Erdos-Renyi */
typedef struct { uint64_t key; int64_t n; int per_row; int32_t *rows, *cols; } er_arg;

static void er_body(void *p, int64_t lo, int64_t hi) {
    er_arg *g = (er_arg *)p;
    for (int64_t r = lo; r < hi; ++r) {
        int32_t *cr = g->cols + r * g->per_row;
        uint64_t ctr = (uint64_t)r << 20;
        for (int t = 0; t < g->per_row;) {
            int32_t cnd = (int32_t)below(synth_draw(g->key, ctr++), (uint64_t)g->n);
            int dup = 0;
            for (int u = 0; u < t; ++u) dup |= (cr[u] == cnd);
            if (!dup) { cr[t] = cnd; g->rows[r * g->per_row + t] = (int32_t)r; ++t; }
        }
    }
}

/* n x n matrix with exactly per_row distinct uniform columns in every row
 * (per_row <= n).  rows/cols hold n*per_row entries, emitted row by row. */
int64_t synth_er(int64_t n, int per_row, uint64_t seed, int32_t *rows, int32_t *cols) {
    if (per_row > n) return -1;
    er_arg g = {synth_stream_key(seed, STREAM_ER), n, per_row, rows, cols};
    parallel_for(n, er_body, &g);
    return n * (int64_t)per_row;
}

/* ------------------------------------------------------------- power-law rows */
/*
 * Row lengths: P(L = k) proportional to k^-alpha for 1 <= k <= cap, then a
 * fraction `empty_frac` of rows (chosen by hash) set to zero.  Writes lengths
 * to len[n] and returns the total.
 */
int64_t synth_zipf_lengths(int64_t n, double alpha, int64_t cap, double empty_frac, uint64_t seed,
                           int64_t *len) {
    double *cdf = (double *)malloc(sizeof(double) * (size_t)cap);
    if (!cdf) return -1;
    double s = 0.0;
    for (int64_t k = 1; k <= cap; ++k) { s += pow((double)k, -alpha); cdf[k - 1] = s; }
    uint64_t kl = synth_stream_key(seed, STREAM_ZLEN), ke = synth_stream_key(seed, STREAM_ZEMPTY);
    int64_t total = 0;
    for (int64_t r = 0; r < n; ++r) {
        if (u01(synth_draw(ke, (uint64_t)r)) < empty_frac) { len[r] = 0; continue; }
        double u = u01(synth_draw(kl, (uint64_t)r)) * s;
        int64_t lo = 0, hi = cap - 1;          /* first k with cdf >= u */
        while (lo < hi) { int64_t mid = (lo + hi) / 2; if (cdf[mid] < u) lo = mid + 1; else hi = mid; }
        if (lo + 1 > n) lo = n - 1;
        len[r] = lo + 1;
        total += len[r];
    }
    free(cdf);
    return total;
}

typedef struct { uint64_t key; int64_t n; const int64_t *off, *len; int32_t *rows, *cols; } zc_arg;

static void zc_body(void *p, int64_t lo, int64_t hi) {
    zc_arg *g = (zc_arg *)p;
    uint64_t words = ((uint64_t)g->n + 63) / 64;
    uint64_t *bits = (uint64_t *)calloc(words, 8);
    for (int64_t r = lo; r < hi; ++r) {
        int64_t L = g->len[r], o = g->off[r];
        uint64_t ctr = (uint64_t)r << 24;
        int32_t *cr = g->cols + o;
        for (int64_t t = 0; t < L;) {
            uint64_t cnd = below(synth_draw(g->key, ctr++), (uint64_t)g->n);
            if (bits && (bits[cnd >> 6] >> (cnd & 63)) & 1) continue;
            if (!bits) { /* no scratch: quadratic duplicate check */
                int dup = 0;
                for (int64_t u = 0; u < t; ++u) dup |= (cr[u] == (int32_t)cnd);
                if (dup) continue;
            } else bits[cnd >> 6] |= 1ULL << (cnd & 63);
            cr[t] = (int32_t)cnd; g->rows[o + t] = (int32_t)r; ++t;
        }
        if (bits) for (int64_t t = 0; t < L; ++t) bits[(uint64_t)cr[t] >> 6] = 0;
    }
    free(bits);
}

/* Fill distinct uniform columns for the lengths produced above.  off is the
 * exclusive prefix sum of len (n+1 entries). */
void synth_zipf_fill(int64_t n, uint64_t seed, const int64_t *off, const int64_t *len,
                     int32_t *rows, int32_t *cols) {
    zc_arg g = {synth_stream_key(seed, STREAM_ZCOL), n, off, len, rows, cols};
    parallel_for(n, zc_body, &g);
}
