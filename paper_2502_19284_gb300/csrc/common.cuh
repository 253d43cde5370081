// Internal declarations shared by the CUDA translation units of libspmv.
// Nothing here is part of the public ABI (see include/spmv.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>

#include "../../include/spmv.h"

namespace spmv {

// ------------------------------------------------------------------ errors
void set_error(const std::string &msg);
spmv_status cuda_status(cudaError_t e, const char *what);   // records text, maps OOM

#define SPMV_CUDA_TRY(call)                                               \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return ::spmv::cuda_status(e_, #call);     \
    } while (0)

#define SPMV_TRY(call)                                                    \
    do {                                                                  \
        spmv_status s_ = (call);                                          \
        if (s_ != SPMV_OK) return s_;                                     \
    } while (0)

// Launch error check (kernel launches report configuration errors lazily).
#define SPMV_LAUNCH_CHECK(what) SPMV_CUDA_TRY(cudaPeekAtLastError())

// Kernel attributes (cudaFuncSetAttribute) belong to the current device: a DeviceOnce runs
// its set-up once per device, under a lock, so that a process that drives several GPUs, from
// one thread or several, launches every kernel with its attributes on each of them.  A
// failed set-up is retried on the next call.
class DeviceOnce {
public:
    template <typename F>
    spmv_status operator()(F &&setup) {
        int dev = 0;
        SPMV_CUDA_TRY(cudaGetDevice(&dev));
        const uint64_t bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0ull;   // beyond 64: every call
        if (bit && (done_.load(std::memory_order_acquire) & bit)) return SPMV_OK;
        std::lock_guard<std::mutex> g(mu_);
        if (bit && (done_.load(std::memory_order_relaxed) & bit)) return SPMV_OK;
        const spmv_status st = setup();
        if (st == SPMV_OK && bit) done_.fetch_or(bit, std::memory_order_release);
        return st;
    }

private:
    std::mutex mu_;
    std::atomic<uint64_t> done_{0};
};

// ------------------------------------------------------------------ tracing
// When tracing is on (spmv_trace_enable), every kernel launch is bracketed by two CUDA
// events on its stream; spmv_trace_read() turns them into per-kernel launch counts and
// device time.  Off by default: then a TraceScope costs one relaxed load.
bool trace_on();
struct TraceScope {
    const char *name;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    TraceScope(const char *n, cudaStream_t st);
    ~TraceScope();
};
#define SPMV_LAUNCH(name, stream, launch)             \
    do {                                              \
        ::spmv::TraceScope trace_scope_(name, stream); \
        launch;                                       \
    } while (0)

// ------------------------------------------------------------------ memory
// Stream-ordered device allocation from the device's default memory pool (kept
// cached between calls).  A host-side hook (spmv_test_fail_alloc) makes the n-th
// allocation fail for tests.  dev_free releases synchronously (safe after any work);
// dev_free_async releases in the order of stream s.
spmv_status dev_alloc(void **p, size_t bytes, const char *what, cudaStream_t s);
// Dynamic shared memory limit of a kernel, with the carveout at its maximum so that the
// residency the occupancy calculator reports is the one the launch gets (a persistent grid
// sized for more CTAs than fit would run a second, late wave).
spmv_status set_smem(const void *kernel, size_t bytes);
// The same with the smallest carveout that holds `ctas` CTAs per SM: the rest of the SM's
// on-chip memory stays L1 cache (which the x gathers of the products hit).
spmv_status set_smem_ctas(const void *kernel, size_t bytes, int ctas);
void dev_free(void *p);
void dev_free_async(void *p, cudaStream_t s);

// Owns one device buffer until released; frees it in stream order otherwise.
struct DevBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    explicit DevBuf(cudaStream_t st) : s(st) {}
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { if (p) dev_free_async(p, s); }
    spmv_status alloc(size_t bytes, const char *what) { return dev_alloc(&p, bytes < 16 ? 16 : bytes, what, s); }
    template <typename T> T *as() const { return (T *)p; }
    void *release() { void *q = p; p = nullptr; return q; }
    void reset() {
        if (p) dev_free_async(p, s);
        p = nullptr;
    }
};

// Device status word bits (written by kernels with atomicOr).
enum : uint32_t {
    ST_INDEX_RANGE = 1u,
    ST_DUPLICATE = 2u,
    ST_TIMEOUT = 4u,
};

inline int elem_size(spmv_dtype d) {
    switch (d) {
        case SPMV_F64: return 8;
        case SPMV_F32: return 4;
        case SPMV_BF16: return 2;
        default: return 0;
    }
}

inline int bits_for(int64_t v) {   // smallest b with 2^b >= v (v >= 1), at least 1
    int b = 1;
    while (((int64_t)1 << b) < v) ++b;
    return b;
}

// ------------------------------------------------------------------ primitives
// Exclusive prefix sum of n uint32 values (in place allowed).  temp: scan_temp_bytes(n).
size_t scan_temp_bytes(int64_t n);
spmv_status exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, void *temp, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs on key bits [begin_bit, end_bit).
// Double-buffered: keys/vals hold the input; keys_alt/vals_alt are scratch of the
// same size.  On return *in_alt tells which buffer pair holds the sorted result.
size_t radix_temp_bytes(int64_t n);
spmv_status radix_sort_pairs(uint64_t *keys, uint64_t *keys_alt, uint32_t *vals, uint32_t *vals_alt, int64_t n,
                             int begin_bit, int end_bit, void *temp, cudaStream_t s, bool *in_alt,
                             uint32_t *err = nullptr);   // err: a zeroed status word; a timed-out wait
                                                         // sets ST_TIMEOUT in it

// Hilbert index of (r, c) on the 2^K grid (device function lives in hilbert.cuh).
spmv_status launch_hilbert_keys(int K, int64_t n, const int32_t *rows, const int32_t *cols, uint64_t *keys,
                                cudaStream_t s);

}  // namespace spmv

// ------------------------------------------------------------------ handle
struct spmv_matrix {
    int64_t m = 0, n = 0;
    int64_t nnz_in = 0;        // triplets given
    int64_t nnz = 0;           // distinct nonzeros (valid once has_csr)
    spmv_dtype dt = SPMV_F64;
    uint32_t flags = 0;
    int32_t format = -1;       // active spmv_format
    int device = 0;

    // triplets (library copy; freed once the CRS arrays exist)
    int32_t *coo_row = nullptr, *coo_col = nullptr;
    void *coo_val = nullptr;

    // CRS
    bool has_csr = false;
    int32_t *row_ptr = nullptr, *col = nullptr;
    void *val = nullptr;

    // row-split bins (rows grouped by length class, ascending inside a class)
    bool has_bins = false;
    int32_t *bin_rows = nullptr;
    int64_t bin_count[8] = {0};
    int64_t max_row_len = 0;
    // compensation threshold of the row-split product under SPMV_ACC_SEGMENT: rows whose length
    // class reaches beyond comp_tau entries are summed with compensation
    int64_t comp_tau = SPMV_COMP_TAU_DEFAULT;

    // merge-path partition and carries
    bool has_merge = false;
    int32_t tile_items = 0;
    int64_t tiles = 0;
    int32_t *part_row = nullptr, *part_nz = nullptr;
    int32_t *carry_row = nullptr;
    // static run structure of the carries (a run: consecutive tiles ending inside one row):
    // fix_len[t] = run length at a run's first tile, else 0; fix_long lists the runs longer
    // than FIX_SHORT tiles (fix_long_count of them), which a whole warp sums
    int32_t *fix_len = nullptr, *fix_long = nullptr;
    int64_t fix_long_count = 0;
    double *carry_val = nullptr;      // tiles carries, then tiles head partials (a tile's first
                                      // row when it began in an earlier tile)
    uint32_t *merge_desc = nullptr;   // per-lane descriptors of the warp tiles (32 words per tile)
    // lane-slotted copy of the warp tiles: path item k of lane l of tile t sits in slot
    // t * 224 + k * 32 + l (a row end or a tail slot holds column 0 and value 0), so a lane
    // finds its operands at fixed offsets; 40 words of header and lane descriptors per tile
    uint32_t *slot_desc = nullptr;
    int32_t *slot_col = nullptr;
    float2 *slot_val2 = nullptr;      // FP64 values split into float pairs (when df_ok)
    void *slot_val = nullptr;         // FP32 or bfloat16 values as stored

    // Hilbert-ordered blocked format
    bool has_hb = false;
    int32_t log2beta = 0, grid_K = 0, inner = 0, block_order = 0;
    int64_t nblk = 0;
    uint32_t *hb_idx = nullptr;
    void *hb_val = nullptr;
    int32_t *blk_ptr = nullptr, *blk_row = nullptr, *blk_col = nullptr;
    int32_t *hb_chunk_blk = nullptr;  // block of the first nonzero of every HB_CHUNK chunk (+ last block)

    // blocked layout of the staged-x product (stage.cu): the block columns (slices of 2^stage_lb
    // columns) in CRS order, cut into warp tiles of 256 entries (32-bit row delta | column
    // word plus the value), with a 16-byte header per tile and the first tile of every slice
    bool has_stage = false;
    int32_t stage_lb = 0, stage_kind = 0;
    int64_t stage_nsl = 0, stage_tiles = 0, stage_bytes = 0;
    int4 *st_hdr = nullptr;
    uint32_t *st_words = nullptr;
    void *st_vals = nullptr;
    uint32_t *st_slice_tile = nullptr;
    uint2 *st_lmeta = nullptr;        // per tile and lane: row of the lane's first item, output offset and flags
    int32_t *st_part = nullptr;       // first tile of every CTA of the product (cost-balanced)
    int32_t stage_parts = 0;
    bool hb_chunked = false;          // the HB product walks the Hilbert-ordered chunks instead

    // Merge Blocking (mergeb.cu), over the blocked arrays in row-major block order: the CRS
    // pointer over the blocks (first block of every block row) and the merge-path split point
    // (entry, block) of every lane's first item of the warp tiles
    bool has_mergeb = false;
    int32_t *mb_row_ptr = nullptr;
    int2 *mb_desc = nullptr;
    int64_t mb_nbr = 0, mb_tiles = 0;

    // FP64 through double-float arithmetic (df64.cuh): set when every stored value lies in
    // the double-float window; x is split into float pairs per product (scratch below)
    bool df_checked = false, df_ok = false;
    float2 *xsplit = nullptr;
    uint32_t *xsplit_flag = nullptr;

    // PageRank buffers and the captured iteration graph
    double *pr_inv = nullptr, *pr_z = nullptr, *pr_y = nullptr, *pr_part = nullptr;
    float2 *pr_z2 = nullptr;
    void *pr_graph = nullptr;         // cudaGraphExec_t
    const double *pr_graph_x = nullptr;
    int pr_graph_iters = 0;
    double pr_graph_damping = 0.0;
    bool pr_graph_staged = false;     // the graph runs the staged blocked product

    uint32_t *status_dev = nullptr;   // device status word
    uint32_t *status_host = nullptr;  // pinned read-back slot
    int64_t bytes = 0;
};
