// Declarations shared between the conversion and product translation units.
#pragma once
#include "common.cuh"

namespace spmv {

// Row-length classes of the row-split product.  Class c < 6 serves rows with
// length <= CLASS_MAX_LEN[c] using CLASS_LANES[c] lanes per row (several rows per
// warp); class 6 serves longer rows with a whole CTA per row.
constexpr int NUM_ROW_CLASSES = 7;

// Merge-path product: a CTA of MERGE_BLOCK threads walks MERGE_TILE_ITEMS path items
// (row ends + nonzeros), MERGE_IPT per thread.  MERGE_IPT is odd so that consecutive
// threads' shared-memory walks start in different banks.
constexpr int MERGE_BLOCK = 256;
constexpr int MERGE_IPT = 7;
constexpr int MERGE_TILE_ITEMS = MERGE_BLOCK * MERGE_IPT;   // CTA tile (allocation-free entry)
// The library's merge product cuts the path into warp tiles of MERGE_WARP_ITEMS items.
constexpr int MERGE_WARP_IPT = 7;
constexpr int MERGE_WARP_ITEMS = 32 * MERGE_WARP_IPT;
// Lane-slotted tile header: words 0..3 = first row, row count, continuation flag, 0;
// words 4..35 = the 32 lane descriptors; words 36..39 = 0 (a tile's block is 160 bytes).
constexpr int SLOT_DESC_WORDS = 40;
// Blocked product: a CTA takes HB_CHUNK consecutive stored nonzeros; the conversion records
// the block holding each chunk's first nonzero.
constexpr int HB_CHUNK = 2048;
// Carry runs up to FIX_SHORT tiles are summed by one thread, longer ones by a warp.
constexpr int FIX_SHORT = 16;

__host__ __device__ __forceinline__ int class_lanes(int c) {
    return c == 0 ? 1 : c == 1 ? 2 : c == 2 ? 4 : c == 3 ? 8 : c == 4 ? 16 : 32;
}

__host__ __device__ __forceinline__ int row_class(unsigned long long len) {
    if (len <= 2) return 0;
    if (len <= 4) return 1;
    if (len <= 8) return 2;
    if (len <= 16) return 3;
    if (len <= 32) return 4;
    if (len <= 2048) return 5;
    return 6;
}

spmv_status launch_validate(const int32_t *row, const int32_t *col, int64_t nnz, int64_t m, int64_t n,
                            uint32_t *status, cudaStream_t s);
spmv_status build_csr(spmv_matrix *h, cudaStream_t s);
spmv_status build_bins(spmv_matrix *h, cudaStream_t s);
spmv_status build_merge(spmv_matrix *h, int tile_items, cudaStream_t s);
spmv_status build_hb(spmv_matrix *h, int log2b, int inner, cudaStream_t s, int border = SPMV_BLOCK_HILBERT);
// FP64 matrices: check the double-float window of the stored values and allocate the
// x-split scratch (n float pairs + a flag word).
spmv_status build_df(spmv_matrix *h, cudaStream_t s);

// products (spmv.cu)
spmv_status mul_merge(const spmv_matrix *h, const void *x, void *y, spmv_dtype vdt, uint32_t acc, cudaStream_t s);
// (the FP64 products use double-float arithmetic when acc == SPMV_ACC_DEFAULT and h->df_ok)
spmv_status mul_rowsplit(const spmv_matrix *h, const void *x, void *y, spmv_dtype vdt, uint32_t acc, cudaStream_t s);
spmv_status mul_hb(const spmv_matrix *h, const void *x, void *y, spmv_dtype vdt, uint32_t acc, cudaStream_t s);
// Staged-x blocked layout and product (stage.cu), built from the CRS arrays with slices of
// 2^lb columns; free_stage releases it in stream order.
spmv_status build_stage(spmv_matrix *h, int lb, cudaStream_t s);
// Recompute the CTA split of the staged layout for the current device (after a load).
spmv_status stage_resplit(spmv_matrix *h, cudaStream_t s);
// (Re)build the HB chunk table from blk_ptr (after a load).
spmv_status hb_chunk_table(spmv_matrix *h, cudaStream_t s);
void free_stage(spmv_matrix *h, cudaStream_t s);
spmv_status mul_stage(const spmv_matrix *h, const void *x, void *y, spmv_dtype vdt, uint32_t acc, cudaStream_t s);
// Merge Blocking (mergeb.cu): block-row pointer and lane split points over the blocked arrays
// (which must be in row-major block order); free_mergeb releases them in stream order.
spmv_status build_mergeb(spmv_matrix *h, cudaStream_t s);
void free_mergeb(spmv_matrix *h, cudaStream_t s);
spmv_status mul_mergeb(const spmv_matrix *h, const void *x, void *y, spmv_dtype vdt, uint32_t acc, cudaStream_t s);
// x -> float pairs in h->xsplit, with the window flag h->xsplit_flag reset and set (spmv.cu).
spmv_status split_x(const spmv_matrix *h, const double *x, cudaStream_t s);
// The same, and y := 0 (m doubles) in the same launch.
spmv_status split_x_zero_y(const spmv_matrix *h, const double *x, double *y, cudaStream_t s);
// Bounded-wait check: one warp waits `polls` polls on an mbarrier nothing arrives at and sets
// ST_TIMEOUT in *status (device word) when it gives up.
spmv_status test_wait(long long polls, uint32_t *status, cudaStream_t s);
// Pattern product (values taken as 1) y = A x through the merge warp tiles, with x already
// split into float pairs in x2 (*xflag non-zero: use native FP64 on x).
spmv_status mul_merge_pattern_split(const spmv_matrix *h, const double *x, const float2 *x2, const uint32_t *xflag,
                                    double *y, cudaStream_t s);
spmv_status pagerank(spmv_matrix *h, double damping, int iters, double *x, cudaStream_t s);
// Drop the captured PageRank graph (its kernels hold pointers into tables being replaced).
void pagerank_forget(spmv_matrix *h);
// Pattern product (values taken as 1) y = A x through the staged blocked layout, with x split
// into float pairs in x2 (*xflag non-zero: native FP64 on x); y is zeroed first (stage.cu).
spmv_status mul_stage_pattern_split(const spmv_matrix *h, const double *x, const float2 *x2, const uint32_t *xflag,
                                    double *y, cudaStream_t s);
spmv_status mul_csr_merge_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr, const int32_t *col,
                                  const double *data, const double *x, double *y, cudaStream_t s);
// Batched multi-RHS merge-path products (batch.cu); plans that name a handle are dropped
// when it is converted again or destroyed.
spmv_status mul_batch(int count, spmv_matrix *const *hs, int k, const void *const *X, void *const *Y,
                      spmv_dtype vdt, uint32_t acc, cudaStream_t s);
void forget_batch_plans(const spmv_matrix *h);
// Uncaptured batch on caller-owned scratch (one BatchSlot per concurrent stream).
struct BatchSlot;
BatchSlot *batch_slot_new();
void batch_slot_free(BatchSlot *b);
int64_t batch_scratch_bytes(int count, spmv_matrix *const *hs, int k);
spmv_status batch_direct(BatchSlot *b, int count, spmv_matrix *const *hs, int k, const void *const *X,
                         void *const *Y, spmv_dtype vdt, uint32_t acc, cudaStream_t s);

}  // namespace spmv
