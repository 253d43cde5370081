/*
 * spmv.h -- C ABI of the GB300 (sm_103a) sparse matrix-vector library.
 *
 * Computes y = A x for a sparse A in R^{m x n} with nnz nonzeros and dense x, y
 * (Bergmans, Meerbergen, Vandebril, "Algorithms for Parallel Shared-Memory Sparse
 * Matrix-Vector Multiplication on Unstructured Matrices", Section 1), together with
 * the storage-format conversions the products need (Section 5.1: a conversion sorts
 * the nonzeros into the format's order, then populates and compresses the arrays).
 *
 * Conventions shared by every call:
 *   - Indices are 0-based int32; nnz < 2^31, m, n < 2^31 (SPMV_ERR_UNSUPPORTED otherwise).
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Work is enqueued on it in stream order.
 *   - Device pointers are plain CUDA device addresses; the library never frees a
 *     caller's buffer and never keeps a caller pointer after a call returns.
 *   - Every call returns a status and never aborts, traps or exits.  On error,
 *     spmv_last_error() describes the failure (thread-local text).
 *   - A handle is not thread-safe: calls on one handle must not run concurrently
 *     from several host threads.  Different handles are independent.
 */
#ifndef GB300_SPMV_H
#define GB300_SPMV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spmv_matrix *spmv_handle;   /* opaque; owns all of its device storage */

typedef enum {
    SPMV_OK = 0,
    SPMV_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, unknown enum, handle misuse   */
    SPMV_ERR_INDEX_RANGE = 2,   /* a triplet index outside [0,m) x [0,n)                 */
    SPMV_ERR_DUPLICATE = 3,     /* duplicate (row, col) with SPMV_DUP_ERROR              */
    SPMV_ERR_OOM = 4,           /* device allocation failed (nothing leaked)             */
    SPMV_ERR_UNSUPPORTED = 5,   /* size/format/dtype combination not provided            */
    SPMV_ERR_CUDA = 6,          /* a CUDA runtime call failed; see spmv_last_error()     */
    SPMV_ERR_TIMEOUT = 7,       /* a bounded device wait gave up                         */
    SPMV_ERR_NOT_CONVERTED = 8, /* spmv_mul before any spmv_convert                      */
    SPMV_ERR_IO = 9             /* a file could not be opened, written or read back whole */
} spmv_status;

/* Element types.  SPMV_PATTERN: no stored values, every nonzero is 1 (data == NULL). */
typedef enum { SPMV_F64 = 0, SPMV_F32 = 1, SPMV_BF16 = 2, SPMV_PATTERN = 3 } spmv_dtype;

/* Storage formats / product algorithms.
 *   CSR_ROWSPLIT  CRS (Section 2, Algorithm 1) with rows split over warps by length
 *                 bins -- the GPU counterpart of ParCRS (Section 5.1).
 *   CSR_MERGE     CRS with the merge-path partition of Section 3.3: equal shares of
 *                 (row ends + nonzeros) per tile, carries added in tile order.
 *   HB            Hilbert-ordered blocked format (Sections 3.1, 4.2: BCOHC/BCOHCH
 *                 storage -- beta x beta blocks, packed 16+16-bit in-block indices,
 *                 nonzeros and blocks in Hilbert-curve order).
 *   AUTO          the library picks one from the matrix's row-length statistics.
 *   MERGEB        Merge Blocking (Section 4.3): beta x beta blocks in row-major block
 *                 order held as a CRS over the blocks, packed 16+16-bit in-block indices,
 *                 entries row-wise inside a block (MergeB, inner_order =
 *                 SPMV_INNER_ROWMAJOR) or along the block's Hilbert curve (MergeBH,
 *                 SPMV_INNER_HILBERT); merge-path product over (block-row ends, entries). */
typedef enum {
    SPMV_FMT_CSR_ROWSPLIT = 0,
    SPMV_FMT_CSR_MERGE = 1,
    SPMV_FMT_HB = 2,
    SPMV_FMT_AUTO = 3,
    SPMV_FMT_MERGEB = 4
} spmv_format;

/* spmv_create_coo flags */
#define SPMV_DEVICE_PTRS 0x1u   /* row_ind/col_ind/data are device pointers (else host) */
#define SPMV_DUP_SUM 0x0u       /* duplicates are added, in input order (default)       */
#define SPMV_DUP_ERROR 0x2u     /* duplicates are rejected with SPMV_ERR_DUPLICATE       */

/* Order of nonzeros inside a block of the blocked format. */
#define SPMV_INNER_HILBERT 0    /* Hilbert order (BCOHCH, Section 4.2; CSBH, Section 4.1) */
#define SPMV_INNER_ROWMAJOR 1   /* row-wise (BCOHC, Section 4.2)                        */
#define SPMV_INNER_ZMORTON 2    /* Z-Morton order (CSB, Section 3.1)                     */

/* Order of the blocks of the blocked format. */
#define SPMV_BLOCK_HILBERT 0    /* Hilbert order of the blocks (BCOHC/BCOHCH, Section 4.2) */
#define SPMV_BLOCK_ROWMAJOR 1   /* block rows in turn (CSB/CSBH, Sections 3.1 and 4.1)     */

/* Product of the HB format. */
#define SPMV_HB_STAGED 0        /* block column by block column, x slice staged on chip   */
#define SPMV_HB_CHUNKED 1       /* Hilbert-ordered chunks, x gathered per nonzero          */

typedef struct {
    int32_t log2_beta;    /* HB block side 2^log2_beta; 0 = Eq. 2 rule (Section 3.1)     */
    int32_t inner_order;  /* SPMV_INNER_*                                                */
    int32_t tile;         /* CSR_MERGE: path items per CTA tile; 0 = library default     */
    int32_t hb_product;   /* HB: SPMV_HB_STAGED (default) or SPMV_HB_CHUNKED             */
    int32_t block_order;  /* HB: SPMV_BLOCK_HILBERT (default) or SPMV_BLOCK_ROWMAJOR       */
} spmv_convert_opts;

/*
 * Accumulation precision of spmv_mul (values are always converted on load).
 *   SPMV_ACC_DEFAULT  F64 data: double precision results; when every stored value and
 *                     every x lies in [2^-50, 2^45] (or is 0) the products and sums are
 *                     evaluated with compensated FP32 arithmetic (double-float: 48-bit
 *                     operands, error-free products, TwoSum accumulation; error below
 *                     4e-14 * (|A||x|)_i), otherwise with native FP64.  Other data: F32.
 *   SPMV_ACC_F64      native FP64 arithmetic throughout.
 *   SPMV_ACC_F32      FP32 accumulation.
 *   SPMV_ACC_COMPENSATED  FP32 vectors and values: FP32 products and sums whose rounding
 *                     errors are collected in a second FP32 term (FMA product errors,
 *                     TwoSum addition errors); CSR_MERGE only.  The compensation runs on
 *                     every row and every product.
 *   SPMV_ACC_SEGMENT  FP32 vectors and values, CSR_MERGE only: FP32 products and sums
 *                     inside each lane's share of a warp tile (at most 7 path items), the
 *                     compensated (TwoSum) reduction only where partial sums of a row are
 *                     joined across lanes and tiles -- i.e. only for rows longer than the
 *                     in-lane threshold.  Error about 8u (|A||x|)_i + u |y_i| (u = 2^-24),
 *                     independent of the row length, at close to plain FP32 cost.
 */
#define SPMV_ACC_DEFAULT 0u
#define SPMV_ACC_F32 1u
#define SPMV_ACC_F64 2u
#define SPMV_ACC_COMPENSATED 3u
#define SPMV_ACC_SEGMENT 4u

/*
 * spmv_create_coo -- ingest a matrix in triplet (coordinate) form (Section 2, Eq. 1).
 *   m, n        matrix shape, 0 <= m, n < 2^31.
 *   nnz         number of triplets, 0 <= nnz < 2^31 (nnz = 0 is a valid empty matrix).
 *   row_ind     nnz int32 row indices; col_ind: nnz int32 column indices; any order.
 *   data        nnz values of type dt, or NULL when dt == SPMV_PATTERN.
 *   flags       SPMV_DEVICE_PTRS if the three arrays live on the device, plus one of
 *               SPMV_DUP_SUM / SPMV_DUP_ERROR (applied when a format is built).
 *   stream      stream for the copy and validation.
 *   out         receives the handle on success, NULL on failure.
 * The library copies the triplets into its own device memory; the caller may free or
 * reuse the arrays as soon as the call returns.  Indices are range-checked on the
 * device; the call synchronises `stream` once to return SPMV_ERR_INDEX_RANGE.
 */
spmv_status spmv_create_coo(int64_t m, int64_t n, int64_t nnz, const int32_t *row_ind,
                            const int32_t *col_ind, const void *data, spmv_dtype dt, uint32_t flags,
                            void *stream, spmv_handle *out);

/*
 * spmv_convert -- build format `f` from the handle's triplets (Section 5.1).
 *   CSR_ROWSPLIT / CSR_MERGE: stable LSD radix sort on the key (row, col), duplicate
 *   resolution, row_ptr by boundary fill, plus the algorithm's partition tables.
 *   HB: Hilbert key h(r, c) on the 2^K grid (K = ceil(log2 max(m, n))), radix sort on h
 *   (or on (h >> 2 log2_beta, r, c) for SPMV_INNER_ROWMAJOR), block segmentation,
 *   packed indices ((r mod beta) << 16 | (c mod beta)).  Requires beta <= 2^16.  With
 *   block_order = SPMV_BLOCK_ROWMAJOR the blocks follow each other block row by block row
 *   (CSB, Section 3.1, with SPMV_INNER_ZMORTON; CSBH, Section 4.1, with SPMV_INNER_HILBERT,
 *   the block's own curve), sorted on (br * 2^(K - log2_beta) + bc, in-block key).  With
 *   hb_product = SPMV_HB_STAGED (the default) the conversion also lays the blocks out for
 *   the staged product (Sections 3.1, 3.2: the x slice of a block column held on chip):
 *   the entries of every block column (a slice of beta columns) in CRS order, in warp tiles
 *   of 256 entries of one 32-bit (row delta, column offset) word and the value each (one
 *   stable radix pass on the block column from the CRS arrays).  Its product visits the
 *   block columns in turn, copies each column's x slice into shared memory once per CTA and
 *   adds row sums into y with reductions (y is zeroed first; the order of the additions
 *   across runs is not fixed).  SPMV_HB_CHUNKED keeps the Hilbert-ordered product that
 *   gathers x per nonzero.
 *   MERGEB: the blocked arrays in row-major block order (as HB with block_order =
 *   SPMV_BLOCK_ROWMAJOR; log2_beta and inner_order as for HB, inner_order ROWMAJOR = MergeB,
 *   HILBERT = MergeBH, ZMORTON accepted), the CRS pointer over the blocks and the merge-path
 *   split point of every warp lane: the path of Section 3.3 over A = the block-row ends and
 *   B = the entries of the blocks, cut into warp tiles of 256 items, 8 per lane.  With a
 *   row-wise inner order the sort runs on the block key only (the CRS order already orders
 *   a block's entries row-wise), the conversion the paper finds cheapest (Section 6.2).  The
 *   product adds each lane's run sums of one row into y with reductions (y is zeroed first;
 *   the order of the additions across runs is not fixed); FP64 vectors accumulate in FP64,
 *   FP32 vectors in plain or compensated FP32.  The blocked arrays are shared with HB: a
 *   later HB conversion with another block order rebuilds them (and drops the MERGEB tables).
 * opt may be NULL (defaults).  The CRS arrays are kept once built, so a later
 * conversion to another CSR algorithm or to HB reuses them.  The converted format
 * becomes the one spmv_mul uses.  Synchronises `stream` (status read-backs).  Errors:
 * SPMV_ERR_DUPLICATE (duplicates with SPMV_DUP_ERROR), SPMV_ERR_TIMEOUT (a bounded wait of
 * a radix sort gave up; the handle keeps its previous formats), SPMV_ERR_OOM, SPMV_ERR_CUDA.
 */
spmv_status spmv_convert(spmv_handle h, spmv_format f, const spmv_convert_opts *opt, void *stream);

/*
 * spmv_mul -- y := A x (overwrites y; Algorithm 1 starts from y = 0).
 *   x           device array of n elements of vec_dt; y: device array of m elements.
 *   vec_dt      SPMV_F64 or SPMV_F32 (type of both x and y).
 *   accum       SPMV_ACC_* (SPMV_ACC_DEFAULT is always valid).
 * Asynchronous: enqueues kernels on `stream` and returns.  Uses the format of the
 * last successful spmv_convert.  The handle's internal scratch is shared by its
 * calls, so two spmv_mul calls on one handle must be ordered (same stream or
 * events); calls on different handles may overlap freely.  A bounded device wait that
 * gives up is reported by spmv_wait.
 */
spmv_status spmv_mul(spmv_handle h, const void *x, void *y, spmv_dtype vec_dt, uint32_t accum, void *stream);

/*
 * spmv_wait -- synchronise `stream` and report whether a product on this handle (spmv_mul,
 * spmv_mul_batch, spmv_pagerank) enqueued on it gave up a bounded device wait since the last
 * spmv_wait: SPMV_ERR_TIMEOUT (its results are not valid; the flag is cleared) or SPMV_OK.
 * SPMV_ERR_CUDA if the synchronisation fails.
 */
spmv_status spmv_wait(spmv_handle h, void *stream);

/*
 * spmv_mul_batch -- Y_i := A_i X_i for `count` handles and k right-hand sides each
 * (the multiple-vector product of Section 3; the batch over many matrices has no
 * counterpart in the paper).
 *   hs          count converted handles of one matrix dtype (any format: the merge-path
 *               tiles of Section 3.3 are built on first use for handles that lack them).
 *   k           right-hand sides per product, 1 <= k <= 16.
 *   X, Y        count device pointers; X[i] is n_i x k row-major (the k values of
 *               x_j contiguous), Y[i] is m_i x k row-major (overwritten).
 *   vec_dt, accum  as spmv_mul's merge path: F64 vectors accumulate in native FP64;
 *               F32 vectors in FP32, compensated FP32, or (F32/BF16 matrices) FP64.
 * Every product runs in one persistent launch over the concatenated tiles of all
 * matrices, followed by one carry fix-up launch.  Both are captured into a CUDA graph
 * the first time a batch shape (the handles, k, dtypes, accumulation and 16-byte
 * alignment of X/Y) is seen, and replayed after that; only the table of X/Y pointers is
 * copied per call.  Per column, the result is bitwise the one spmv_mul gives for the
 * same accumulation on the merge path (FP64 vectors accumulate in native FP64 here, so
 * SPMV_ACC_DEFAULT matches spmv_mul with SPMV_ACC_F64).  With k = 1, a handle whose active
 * format is row-split, HB or MERGEB (spmv_convert, or chosen by spmv_tune) runs that format's
 * product after the persistent launch instead, with spmv_mul's result.  Calls with the same batch shape share scratch
 * and must be ordered.  Not capturable into a caller's graph (the pointer table is
 * uploaded from pageable memory).  A handle's plans are dropped when it is converted
 * again or destroyed.
 */
spmv_status spmv_mul_batch(int count, const spmv_handle *hs, int k, const void *const *X, void *const *Y,
                           spmv_dtype vec_dt, uint32_t accum, void *stream);

/* spmv_destroy -- free every device buffer of the handle (synchronises with its stream). */
spmv_status spmv_destroy(spmv_handle h);

/*
 * spmv_tune -- autotuner: time one product y = A x in each candidate storage format of the
 * handle (Section 6.1 finds that the best method depends on the matrix; here it is
 * measured), and make the fastest the active format.  Candidates: row-split CRS and
 * merge-path CRS (built if missing, both cheap), the Hilbert-blocked format with both of
 * its products (staged block columns and Hilbert-ordered chunks) if it is already built or
 * flags has SPMV_TUNE_HB (its conversion costs far more than a product), and Merge Blocking
 * (MERGEB, row-wise inside the blocks) if its tables are built or flags has SPMV_TUNE_MERGEB
 * (which rebuilds the blocked arrays in row-major block order when they are in another order;
 * the HB products then run on those).
 *   vec_dt, accum   the product to time (as in spmv_mul).
 *   out             may be NULL; receives the chosen format (and HB product) and the median
 *                   time of one product per candidate in milliseconds (-1 where not tried).
 * Allocates scratch x and y of the handle's size, runs 2 + 2*reps products per candidate
 * on `stream` and synchronises it.  spmv_mul then uses the chosen format; spmv_mul_batch
 * with k = 1 runs a handle whose active format is row-split or blocked with that product,
 * after the persistent launch of the merge-path matrices of the batch.
 */
enum { SPMV_TUNE_HB = 0x1, SPMV_TUNE_MERGEB = 0x2 };
typedef struct {
    int32_t chosen;     /* SPMV_FMT_CSR_ROWSPLIT, SPMV_FMT_CSR_MERGE, SPMV_FMT_HB or SPMV_FMT_MERGEB */
    int32_t reps;       /* timed products per candidate */
    float ms[5];        /* median ms per product: [ROWSPLIT, MERGE, HB staged, HB chunked, MERGEB],
                           -1 if not tried */
    int32_t hb_product; /* SPMV_HB_STAGED or SPMV_HB_CHUNKED when chosen is SPMV_FMT_HB */
    int32_t pad_;
} spmv_tune_result;
spmv_status spmv_tune(spmv_handle h, spmv_dtype vec_dt, uint32_t accum, uint32_t flags, spmv_tune_result *out,
                      void *stream);

/*
 * spmv_set_compensation_threshold -- the threshold tau of SPMV_ACC_SEGMENT for the row-split
 * product (FP32 vectors): rows are summed in plain FP32 where their length class (<= 2, 4, 8,
 * 16, 32, 2048 entries, or longer) lies within tau entries, and with compensated FP32 (the FMA
 * error of every product and the TwoSum error of every addition, through the lane sums and
 * the butterfly that joins them) where it can reach beyond tau.  tau = 0 compensates every
 * row (as SPMV_ACC_COMPENSATED); a tau at or beyond the longest row compensates none.  The
 * paper has no counterpart (it does not discuss precision).  The merge-path product's
 * SPMV_ACC_SEGMENT keeps its structural threshold: rows longer than one lane's seven items,
 * whose partial sums it joins across lanes and tiles.  Default SPMV_COMP_TAU_DEFAULT = 0, from a
 * sweep over tau on Erdos-Renyi (8 per row) and Zipf(1.8) rows on GB300: the row-split product is
 * memory-bound, so compensating every row costs no measurable time (within 0.5%), while plain
 * FP32 sums of rows of 8 entries already double the error.  SPMV_ERR_INVALID_ARG for tau < 0.
 */
#define SPMV_COMP_TAU_DEFAULT 0
spmv_status spmv_set_compensation_threshold(spmv_handle h, int64_t tau);

/* ---------------------------------------------------------------- iterative use */

/*
 * spmv_cg -- conjugate gradients (Hestenes and Stiefel) for A x = b with a symmetric positive
 * definite A: the repeated products on one converted matrix over which the paper's
 * break-even count amortises a conversion (Sections 6.2 and 7).
 *   h           converted handle (square; FP64, FP32 or pattern values); every iteration runs one
 *               spmv_mul with FP64 vectors in the handle's active format (SPMV_ACC_DEFAULT).
 *   b           device, n doubles; x: device, n doubles (overwritten; x0 = 0).
 *   tol         stop when the recursive residual ||r|| <= tol ||b||; max_iters: iteration cap.
 *   iters_out, resid_out   may be NULL: iterations run and the final ||r||.
 * Dot products are deterministic (fixed partial sums and order); the scalars stay on the
 * device and the residual is read back every 8 iterations, so up to 7 iterations may run past
 * the threshold.  Allocates scratch (3 n doubles), synchronises `stream` at those read-backs.
 * SPMV_ERR_INVALID_ARG (NULL, non-square, tol < 0), SPMV_ERR_NOT_CONVERTED, SPMV_ERR_UNSUPPORTED
 * (bfloat16 values).
 */
spmv_status spmv_cg(spmv_handle h, const double *b, double *x, double tol, int max_iters, void *stream,
                    int *iters_out, double *resid_out);

/* ---------------------------------------------------------------- storage */

/*
 * spmv_save / spmv_load -- keep converted formats on disk so that a later run skips the
 * conversion (the paper's future work: storing several formats of a matrix, Section 8).
 * spmv_save writes the handle's CRS arrays and, when built, its Hilbert-ordered blocked arrays
 * and staged blocked layout, with its active format and a checksum of every array; it copies
 * through a pinned host buffer on `stream` and synchronises it.  spmv_load reads such a file
 * into a new handle (*out), verifies the checksum before any kernel reads the arrays, rebuilds
 * the cheap derived tables (the HB chunk table, the staged layout's split between the loading
 * device's SMs) and makes the saved format active again (its other tables, e.g. the merge-path
 * partition, come from the CRS arrays as a conversion would build them).  The file format is
 * this library's own (host byte order; see csrc/store.cu).  Errors: SPMV_ERR_INVALID_ARG (NULL
 * argument, not a file of this library or one written by a build with another file format
 * version), SPMV_ERR_NOT_CONVERTED (save before any conversion),
 * SPMV_ERR_IO (open, write or read failed, truncated or damaged file), SPMV_ERR_OOM.
 */
spmv_status spmv_save(spmv_handle h, const char *path, void *stream);
spmv_status spmv_load(const char *path, void *stream, spmv_handle *out);

/* ---------------------------------------------------------------- inspection */

typedef struct {
    int64_t m, n;
    int64_t nnz;            /* distinct nonzeros once converted, else the triplet count */
    int32_t format;         /* active spmv_format, or -1 before conversion               */
    int32_t dtype;          /* spmv_dtype of the stored values                           */
    int32_t log2_beta;      /* HB block side (0 if no HB)                                */
    int32_t grid_order;     /* K of the Hilbert grid                                     */
    int64_t nblk;           /* non-empty HB blocks                                       */
    int64_t merge_tiles;    /* CSR_MERGE tiles                                           */
    int32_t merge_tile_items;
    int32_t hb_orders;      /* 16 x block order + inner order of the blocked arrays      */
    int64_t device_bytes;   /* device memory held by the handle                          */
    int64_t block_rows;     /* MERGEB: block rows nbr = ceil(m / beta) (0 if not built)  */
    int64_t mergeb_tiles;   /* MERGEB: warp tiles of 256 path items                      */
} spmv_info_t;

spmv_status spmv_info(spmv_handle h, spmv_info_t *out);

/*
 * spmv_export_csr -- copy the CRS arrays to host buffers (row_ptr: m+1, col_ind and
 * data: nnz; data may be NULL; it receives values in the stored dtype).
 */
spmv_status spmv_export_csr(spmv_handle h, int32_t *row_ptr, int32_t *col_ind, void *data);

/*
 * spmv_export_hb -- copy the HB arrays to host buffers: idx and data (nnz),
 * blk_ptr (nblk+1), blk_row and blk_col (nblk).  Any pointer may be NULL.
 */
spmv_status spmv_export_hb(spmv_handle h, uint32_t *idx, void *data, int32_t *blk_ptr, int32_t *blk_row,
                           int32_t *blk_col);

/*
 * spmv_export_merge_partition -- copy the merge-path split points of the CSR_MERGE
 * partition (Section 3.3): for tile t = 0..tiles, row_start[t] row ends and
 * nz_start[t] nonzeros are consumed before the tile (tiles+1 entries each).
 */
spmv_status spmv_export_merge_partition(spmv_handle h, int32_t *row_start, int32_t *nz_start);

/*
 * spmv_export_mergeb -- copy the MERGEB tables to host buffers: blk_row_ptr (block_rows + 1
 * entries: the first block of every block row), and for every lane g = 0 .. 32 *
 * mergeb_tiles - 1 of the warp tiles the merge-path split point of its first item (path
 * diagonal 8 g, clamped to the path length): lane_entry[g] entries and, implicitly,
 * 8 g - lane_entry[g] block-row ends consumed before it; lane_block[g] the block holding
 * entry lane_entry[g] (nblk when every entry is consumed).  Sizes from spmv_info; any
 * pointer may be NULL.  SPMV_ERR_NOT_CONVERTED if the tables are not built.
 */
spmv_status spmv_export_mergeb(spmv_handle h, int32_t *blk_row_ptr, int32_t *lane_entry, int32_t *lane_block);

/* Text of the last error raised on the calling host thread ("" if none). */
const char *spmv_last_error(void);

/* Name of a status code. */
const char *spmv_status_string(spmv_status s);

/* Hilbert index of (r, c) on the 2^K grid, computed by the device kernel for n
 * points (device arrays rows, cols -> keys).  Exposed for testing the key kernel. */
spmv_status spmv_hilbert_keys(int K, int64_t n, const int32_t *rows, const int32_t *cols, uint64_t *keys,
                              void *stream);

/* ---------------------------------------------------------------- PageRank */

/*
 * spmv_pagerank -- PageRank by power iteration on the square matrix of h (Section 1 names
 * PageRank among the applications built on SpMV; the paper does not define it, so the
 * iteration is stated here).  Stored values are ignored: a stored entry (i, j) is an edge
 * j -> i, and the out-degree of j is the number of stored entries in column j.
 *   x0 = 1/n;  for each iteration:  dangling = sum of x_j over columns of out-degree 0,
 *   x_i <- damping * ( sum_j A_ij x_j / outdeg_j + dangling / n ) + (1 - damping) / n.
 *   damping     in [0, 1] (0.85 is customary);  iters: number of iterations, 0..10000.
 *   x           device array of n doubles; receives the final vector (it is also the
 *               working vector of the iteration).
 * Builds the CRS arrays and the merge-path partition if needed.  The product of every
 * iteration is the pattern merge-path product, or, when the handle's active format is HB
 * with the staged product, the staged blocked pattern product (x read in slices, which pays
 * once x no longer fits in L2; its summation order is not fixed, so its results agree within
 * FP64 rounding but are not bitwise reproducible).  The iterations are captured into a CUDA
 * graph on the first call for a given (x, iters, damping, product) and the graph is replayed
 * on `stream` (asynchronously) by this and later calls; a conversion that replaces the staged
 * layout drops the graph.
 */
spmv_status spmv_pagerank(spmv_handle h, double damping, int iters, double *x, void *stream);

/* ---------------------------------------------------------------- serving */

/*
 * A request loop over a resident set of converted matrices (the paper has no counterpart;
 * its introduction names PageRank as an application built on SpMV).  A worker thread admits
 * queued requests in arrival order as launch slots and the memory budget allow: the first
 * request that fits opens a group; a SpMV group then takes every later queued SpMV request
 * with the same vector type and accumulation (up to max_batch) that still fits and runs
 * them as one batched launch (the product of spmv_mul_batch, without capture); a PageRank
 * request runs alone, at most one per matrix at a time.  Slots run concurrently on their
 * own CUDA streams, so requests arriving while others run start as soon as a slot and
 * memory free up.  Every SpMV result is bitwise the spmv_mul result with the same
 * accumulation on the merge path (FP64 vectors accumulate in native FP64, as with
 * SPMV_ACC_F64), and every PageRank result the spmv_pagerank result, whatever else is in
 * flight (bitwise for matrices whose active format is not HB; HB matrices run PageRank on the
 * staged product, whose summation order is not fixed).
 *
 * Memory: the budget covers the resident matrices (their spmv_info bytes at spmv_server_add,
 * plus the PageRank scratch of a matrix from its first PageRank request on) and, per admitted
 * SpMV request, its device x and y and batch scratch.  A request that cannot fit even with
 * nothing else in flight completes with SPMV_ERR_OOM.
 * Host buffers: x and y may be device pointers, pinned host memory (copied by DMA), or
 * pageable host memory (staged through pinned buffers of the slot).  The caller keeps them
 * valid until the request completes.  Latency = completion - arrival on the host's steady
 * clock; completion is the moment the worker sees the request's work (including the copy of
 * y) finished.
 */
typedef struct spmv_server *spmv_server_t;

typedef struct {
    int64_t budget_bytes;   /* device memory for resident matrices and admitted requests */
    int32_t slots;          /* concurrent launches, one CUDA stream each: 1..64 */
    int32_t max_batch;      /* SpMV requests grouped into one launch: 1..1024 */
} spmv_server_opts;

enum { SPMV_REQ_SPMV = 0, SPMV_REQ_PAGERANK = 1 };

typedef struct {
    int32_t kind;        /* SPMV_REQ_SPMV or SPMV_REQ_PAGERANK */
    int32_t matrix;      /* id returned by spmv_server_add */
    int32_t vec_dt;      /* SpMV: SPMV_F64 or SPMV_F32 (type of x and y) */
    uint32_t accum;      /* SpMV: SPMV_ACC_* as in spmv_mul (merge path) */
    int32_t iters;       /* PageRank: iterations (0..10000) */
    int32_t pad_;        /* 0 */
    double damping;      /* PageRank: in [0, 1] */
    const void *x;       /* SpMV: n elements of vec_dt; unused for PageRank */
    void *y;             /* SpMV: m elements of vec_dt; PageRank: n doubles */
} spmv_request;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t launches;            /* batched SpMV launches */
    int64_t batched_requests;    /* SpMV requests those launches carried */
    int64_t resident_bytes;      /* resident set */
    int64_t peak_bytes;          /* peak of resident set + admitted requests */
    int64_t deferred;            /* admissions postponed because memory was short */
} spmv_server_stats_t;

/* Start the worker thread on the current device.  Errors: SPMV_ERR_INVALID_ARG (limits
 * above), SPMV_ERR_CUDA. */
spmv_status spmv_server_create(const spmv_server_opts *opts, spmv_server_t *out);
/* Add a converted handle (any format; its merge-path tiles are built if missing) to the
 * resident set.  The caller keeps ownership and destroys it after spmv_server_destroy.
 * SPMV_ERR_OOM if the resident set would exceed the budget. */
spmv_status spmv_server_add(spmv_server_t srv, spmv_handle h, int32_t *matrix_id);
/* Queue a request (arrival = now); *ticket identifies it for spmv_server_wait. */
spmv_status spmv_server_submit(spmv_server_t srv, const spmv_request *req, int64_t *ticket);
/* Block until the request completes; returns its status and (if latency_s) its latency in
 * seconds.  A ticket can be waited for once. */
spmv_status spmv_server_wait(spmv_server_t srv, int64_t ticket, double *latency_s);
/* Open-loop replay: submit reqs[i] at arrival_s[i] seconds (non-decreasing) after the call
 * starts, from the calling thread, then wait for all; latency_s[i] receives each latency
 * (-1 for requests not submitted after an error).  Returns the first error. */
spmv_status spmv_server_replay(spmv_server_t srv, int64_t n, const spmv_request *reqs, const double *arrival_s,
                               double *latency_s);
spmv_status spmv_server_stats(spmv_server_t srv, spmv_server_stats_t *out);
/* Finish queued and running requests, stop the worker, free the server's memory. */
spmv_status spmv_server_destroy(spmv_server_t srv);

/* ---------------------------------------------------------------- no allocation */

/*
 * spmv_mul_csr_merge_noalloc -- y := A x for a CRS matrix the caller already holds on the
 * device, with the merge-path product, without allocating any device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot allocate,
 * for example callers that reserved all device memory up front for their own allocator,
 * code that runs under a memory budget enforced by someone else, or serving loops that
 * cannot afford the device synchronisation that cudaMalloc and cudaFree imply.  The library's other calls keep
 * their scratch in memory they allocate; this one keeps the merge-path partition and the
 * tile carries in a fixed array that is part of the library itself (about 1.3 MB, held on
 * every GPU that loads the library until the process exits).
 *
 *   m, n, nnz   shape and nonzero count; nnz must equal row_ptr[m].
 *   row_ptr     device, m+1 int32 (non-decreasing, row_ptr[0] = 0); col_ind: device, nnz
 *               int32 in [0, n); data: device, nnz doubles; x: device, n doubles;
 *               y: device, m doubles (overwritten).  All are the caller's and are only read
 *               (y written) by the kernels enqueued on `stream`.
 * Limit: m + nnz <= 117,440,512 (65,536 tiles of 1,792 row ends and nonzeros); larger
 * inputs are rejected with SPMV_ERR_UNSUPPORTED before anything is enqueued.
 * Arithmetic is native FP64 (as spmv_mul with SPMV_ACC_F64).
 * The first call on each device looks up the array's device address with that device
 * current; make that first call before capturing a stream into a graph.  All calls on a
 * device share the one array and overwrite it (every entry they read is written by the
 * same call first), so calls whose kernels may overlap on the GPU -- on different streams
 * without ordering -- race and must not be issued.
 */
spmv_status spmv_mul_csr_merge_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr,
                                       const int32_t *col_ind, const double *data, const double *x, double *y,
                                       void *stream);

/* ---------------------------------------------------------------- tracing */

/*
 * spmv_trace_enable -- turn kernel tracing on (1) or off (0).  While on, every kernel
 * the library launches is bracketed by two CUDA events on its stream (a few
 * microseconds of host overhead per launch, no change to the kernels).  Turning it on
 * clears the table.  Synchronises the device.
 */
spmv_status spmv_trace_enable(int on);

/*
 * spmv_trace_read -- synchronise the device and return the number of distinct traced
 * kernels; the first max_entries of them are written as (name, launches, total device
 * milliseconds).  Names are static strings owned by the library.  Returns -1 if the
 * synchronisation fails.
 */
int spmv_trace_read(int max_entries, const char **names, long long *counts, double *total_ms);

/* Test hook: the allocation after `n` further successful ones fails with
 * SPMV_ERR_OOM, without touching the device (n < 0 turns the hook off). */
void spmv_test_fail_alloc(long long n);

/* Test hook for the bounded device waits (every mbarrier wait of the persistent kernels
 * gives up after a fixed number of polls, sets a timeout bit in a status word and returns):
 * one warp waits `polls` polls (1 <= polls <= 2^22) on an mbarrier that nothing arrives at.
 * On return *status_out (host memory, owned by the caller) holds the status word the
 * kernel wrote: bit 2 (value 4) set when the wait gave up, as it always should.  The device
 * stays usable.  Returns SPMV_ERR_INVALID_ARG for a bad argument, SPMV_ERR_OOM or
 * SPMV_ERR_CUDA if the status word cannot be allocated or read. */
spmv_status spmv_test_wait_timeout(long long polls, uint32_t *status_out);

#ifdef __cplusplus
}
#endif

#endif /* GB300_SPMV_H */
