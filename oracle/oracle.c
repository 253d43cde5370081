/*
 * CPU oracle for the GB300 SpMV library -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, sequential, obviously correct restatements of what the method computes,
 * in double precision with floating-point contraction disabled (built with
 * -ffp-contract=off), so that each function can be checked against the paper by
 * eye.  Only the tests, the package's smoke check and the benchmark's CPU
 * baseline may load this file.  It shares no code with the CUDA library.
 *
 * Paper: K. Bergmans, K. Meerbergen, R. Vandebril, "Algorithms for Parallel
 * Shared-Memory Sparse Matrix-Vector Multiplication on Unstructured Matrices"
 * (arXiv 2502.19284).  Notation: A in R^{m x n} with nnz nonzeros, y = A x (Section 1).
 *
 * Functions and the passages they follow:
 *   oracle_coo_to_csr      Section 2 (triplet format, CRS format) + Section 5.1 (conversion
 *                          = sort into the format's order, then populate/compress)
 *   oracle_csr_spmv        Algorithm 1 (CRS SpMV): rows in order, entries in storage order, FP64
 *   oracle_coo_spmv        Eq. 1 (triplet SpMV) -- used only as a cross-check
 *   oracle_hilbert_index   Section 3.2 and the Hilbert recursion figure: quadrant order
 *                          TL, BL, BR, TR; TL sub-curve transposed, TR anti-transposed
 *   oracle_log2_beta       Eq. 2 (CSB block size bound) + Section 3.1 constraints
 *   oracle_csr_to_hb       Section 4.2 (BCOHC / BCOHCH): nonzeros sorted on the Hilbert
 *                          curve, stored per beta x beta block as packed 16+16-bit triplets
 *   oracle_csr_to_csb      Sections 3.1 and 4.1 (CSB / CSBH): row-major block order, Z-Morton
 *                          (or the block's own Hilbert curve) inside every block
 *   oracle_hb_spmv         block-by-block product over the structures above
 *   oracle_merge_path_search, oracle_merge_spmv
 *                          Section 3.3 and the merge-path figure: diagonal split of the
 *                          (row ends x nonzero indices) path; ties consume a row end first;
 *                          per-part carries added afterwards in order
 *   oracle_block_row_ptr, oracle_mergeb_spmv
 *                          Section 4.3 (Merge Blocking, MergeB / MergeBH): the block matrix in
 *                          CRS over blocks in row-major order (oracle_csr_to_csb with a
 *                          row-wise or Hilbert inner order), merge path over (block-row ends x
 *                          blocks), a temporary vector in place of the temporary value
 *   oracle_csr_transpose  plain transpose (for the adjoint identity test)
 *   oracle_csr_spmv_neumaier  Neumaier (1974) compensated row sums, an accuracy reference
 *   oracle_round_f32, oracle_round_bf16  storage rounding to nearest-even, directly from double
 *   oracle_pagerank        Section 1 names PageRank as an SpMV application; the iteration
 *                          written out: x <- d (P x + dangling/n) + (1-d)/n, P = A D^{-1}
 *   oracle_cg              conjugate gradients (Hestenes and Stiefel, 1952) on repeated
 *                          Algorithm 1 products, the iterative use of Sections 6.2 and 7
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OK 0
#define ERR_INVALID_ARG 1
#define ERR_INDEX_RANGE 2
#define ERR_DUPLICATE 3
#define ERR_OOM 4
#define ERR_UNSUPPORTED 5

/* ------------------------------------------------------------ COO -> CRS */

typedef struct { int32_t col; int64_t pos; } colpos_t;

static int cmp_colpos(const void *a, const void *b) {
    const colpos_t *x = (const colpos_t *)a, *y = (const colpos_t *)b;
    if (x->col != y->col) return x->col < y->col ? -1 : 1;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    return 0;
}

/*
 * Triplet (row_ind, col_ind, data) -> CRS (row_ptr, col_ind, data), Section 2.
 * Step 1 (Section 5.1): order the nonzeros row-wise; within a row by column; equal
 * (row, col) pairs keep their input order.  Step 2: compress the row indices into
 * row_ptr (m+1 entries).  Duplicate (row, col) pairs: dup_mode 0 adds them in input
 * order (left to right); dup_mode 1 rejects them with ERR_DUPLICATE.
 * vals may be NULL (pattern matrix); then val_out is not written.
 * Output arrays must hold nnz entries (row_ptr: m+1).  *nnz_out receives the
 * number of distinct entries.
 */
int oracle_coo_to_csr(int64_t m, int64_t n, int64_t nnz, const int32_t *row, const int32_t *col,
                      const double *vals, int dup_mode, int32_t *row_ptr, int32_t *col_out,
                      double *val_out, int64_t *nnz_out) {
    if (m < 0 || n < 0 || nnz < 0) return ERR_INVALID_ARG;
    if (nnz >= ((int64_t)1 << 31) || m >= ((int64_t)1 << 31) || n >= ((int64_t)1 << 31)) return ERR_UNSUPPORTED;
    for (int64_t i = 0; i < nnz; ++i)
        if (row[i] < 0 || row[i] >= m || col[i] < 0 || col[i] >= n) return ERR_INDEX_RANGE;
    /* counting sort by row: count, prefix, stable placement */
    int64_t *cnt = (int64_t *)calloc((size_t)m + 1, sizeof(int64_t));
    colpos_t *tmp = (colpos_t *)malloc(sizeof(colpos_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!cnt || !tmp) { free(cnt); free(tmp); return ERR_OOM; }
    for (int64_t i = 0; i < nnz; ++i) cnt[row[i] + 1]++;
    for (int64_t r = 0; r < m; ++r) cnt[r + 1] += cnt[r];
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    if (!next) { free(cnt); free(tmp); return ERR_OOM; }
    for (int64_t r = 0; r < m; ++r) next[r] = cnt[r];
    for (int64_t i = 0; i < nnz; ++i) {
        int64_t p = next[row[i]]++;
        tmp[p].col = col[i];
        tmp[p].pos = i;
    }
    free(next);
    /* within each row: by column, then by input position */
    for (int64_t r = 0; r < m; ++r)
        if (cnt[r + 1] - cnt[r] > 1) qsort(tmp + cnt[r], (size_t)(cnt[r + 1] - cnt[r]), sizeof(colpos_t), cmp_colpos);
    /* populate, merging duplicates */
    int64_t w = 0;
    row_ptr[0] = 0;
    for (int64_t r = 0; r < m; ++r) {
        for (int64_t k = cnt[r]; k < cnt[r + 1]; ++k) {
            if (k > cnt[r] && tmp[k].col == tmp[k - 1].col) {
                if (dup_mode == 1) { free(cnt); free(tmp); return ERR_DUPLICATE; }
                if (vals) val_out[w - 1] = val_out[w - 1] + vals[tmp[k].pos];
                continue;
            }
            col_out[w] = tmp[k].col;
            if (vals) val_out[w] = vals[tmp[k].pos];
            ++w;
        }
        row_ptr[r + 1] = (int32_t)w;
    }
    *nnz_out = w;
    free(cnt); free(tmp);
    return OK;
}

/* ---------------------------------------------------------------- Algorithm 1 */

/*
 * The CRS product of Algorithm 1 (Section 2).  Contract: y is overwritten; every
 * row is summed on its own, its stored entries taken in storage order, each product
 * rounded to FP64 and then added to the running FP64 row sum (no fused multiply-add,
 * the file is built with -ffp-contract=off).  data == NULL means a pattern matrix
 * (every stored value is 1).
 */
void oracle_csr_spmv(int64_t m, const int32_t *row_ptr, const int32_t *col_ind, const double *data,
                     const double *x, double *y) {
    for (int64_t i = 0; i < m; ++i) y[i] = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t j = col_ind[k];
            double a = data ? data[k] : 1.0;
            double prod = a * x[j];
            y[i] = y[i] + prod;
        }
    }
}

/* Same as Algorithm 1 but with k right-hand sides: X is n x k row-major, Y is m x k. */
void oracle_csr_spmm(int64_t m, int64_t k, const int32_t *row_ptr, const int32_t *col_ind,
                     const double *data, const double *X, double *Y) {
    for (int64_t i = 0; i < m * k; ++i) Y[i] = 0.0;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            double a = data ? data[p] : 1.0;
            for (int64_t t = 0; t < k; ++t) {
                double prod = a * X[(int64_t)col_ind[p] * k + t];
                Y[i * k + t] = Y[i * k + t] + prod;
            }
        }
}

/* Eq. 1: triplet SpMV, y[row_ind[i]] += data[i] * x[col_ind[i]] in input order. */
void oracle_coo_spmv(int64_t m, int64_t nnz, const int32_t *row, const int32_t *col, const double *data,
                     const double *x, double *y) {
    for (int64_t i = 0; i < m; ++i) y[i] = 0.0;
    for (int64_t i = 0; i < nnz; ++i) {
        double a = data ? data[i] : 1.0;
        double prod = a * x[col[i]];
        y[row[i]] = y[row[i]] + prod;
    }
}

/* Row-wise Neumaier compensated sum of data[k]*x[j] (each product rounded once);
 * an accuracy reference beside Algorithm 1. */
void oracle_csr_spmv_neumaier(int64_t m, const int32_t *row_ptr, const int32_t *col_ind,
                              const double *data, const double *x, double *y) {
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0, c = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            double a = data ? data[k] : 1.0;
            double p = a * x[col_ind[k]];
            double t = s + p;
            if (fabs(s) >= fabs(p)) c = c + ((s - t) + p);
            else c = c + ((p - t) + s);
            s = t;
        }
        y[i] = s + c;
    }
}

/* Row sums of |data[k]| * |x[j]|: the scale (|A| |x|)_i used by the tolerance. */
void oracle_csr_absmul(int64_t m, const int32_t *row_ptr, const int32_t *col_ind, const double *data,
                       const double *x, double *y) {
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            double a = data ? fabs(data[k]) : 1.0;
            s = s + a * fabs(x[col_ind[k]]);
        }
        y[i] = s;
    }
}

/* Plain CRS transpose: A^T as CRS (n rows).  Entries of each output row keep the
 * order of increasing source row. */
int oracle_csr_transpose(int64_t m, int64_t n, const int32_t *row_ptr, const int32_t *col_ind,
                         const double *data, int32_t *t_row_ptr, int32_t *t_col, double *t_val) {
    int64_t nnz = row_ptr[m];
    int64_t *next = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!next) return ERR_OOM;
    for (int64_t k = 0; k < nnz; ++k) next[col_ind[k] + 1]++;
    for (int64_t j = 0; j < n; ++j) next[j + 1] += next[j];
    for (int64_t j = 0; j <= n; ++j) t_row_ptr[j] = (int32_t)next[j];
    for (int64_t i = 0; i < m; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t p = next[col_ind[k]]++;
            t_col[p] = (int32_t)i;
            if (data && t_val) t_val[p] = data[k];
        }
    free(next);
    return OK;
}

/* -------------------------------------------------------------- Hilbert curve */

/*
 * Index of cell (r, c) on the Hilbert curve over the 2^K x 2^K grid, as drawn in
 * the paper's Hilbert figure (Section 3.2): the curve enters at the top-left cell
 * and leaves at the top-right cell.  Recursively, the order-K curve visits the
 * four quadrants top-left, bottom-left, bottom-right, top-right; the bottom two
 * hold the order-(K-1) curve as is, the top-left one holds it transposed
 * (r, c) -> (c, r), and the top-right one holds it anti-transposed
 * (r, c) -> (S-1-c, S-1-r), with S = 2^(K-1) the quadrant side.
 */
uint64_t oracle_hilbert_index(int K, int64_t r, int64_t c) {
    if (K == 0) return 0;
    int64_t S = (int64_t)1 << (K - 1);
    uint64_t Q = (uint64_t)1 << (2 * (K - 1));
    int top = r < S, left = c < S;
    if (top && left) return 0 * Q + oracle_hilbert_index(K - 1, c, r);
    if (!top && left) return 1 * Q + oracle_hilbert_index(K - 1, r - S, c);
    if (!top && !left) return 2 * Q + oracle_hilbert_index(K - 1, r - S, c - S);
    /* top right */
    int64_t lr = r, lc = c - S;
    return 3 * Q + oracle_hilbert_index(K - 1, S - 1 - lc, S - 1 - lr);
}

/* Z-Morton index (Section 3.1 and the Z-Morton figure): quadrants TL, TR, BL, BR
 * recursively, i.e. the row bit above the column bit at every level. */
uint64_t oracle_zmorton_index(int K, int64_t r, int64_t c) {
    if (K == 0) return 0;
    int64_t S = (int64_t)1 << (K - 1);
    uint64_t Q = (uint64_t)1 << (2 * (K - 1));
    int q = (r >= S ? 2 : 0) + (c >= S ? 1 : 0);
    return (uint64_t)q * Q + oracle_zmorton_index(K - 1, r % S, c % S);
}

/* Smallest K >= 1 with 2^K >= max(m, n): the grid the curve is drawn on. */
int oracle_grid_order(int64_t m, int64_t n) {
    int64_t d = m > n ? m : n;
    int K = 1;
    while (((int64_t)1 << K) < d) ++K;
    return K;
}

/*
 * Block size rule of Section 3.1 (Eq. 2): ceil(log2 sqrt(n)) <= log2 beta <=
 * 3 + ceil(log2 sqrt(n)).  Start at the upper bound and lower log2 beta by one
 * until the constraints hold: beta <= 2^16 (16-bit packed in-block indices) and
 * the slice of x a block needs (beta * x_bytes) fits the on-chip budget
 * `slice_budget_bytes`.  log2 beta is never taken below 4.
 */
int oracle_log2_beta(int64_t n, int64_t x_bytes, int64_t slice_budget_bytes) {
    /* ceil(log2(sqrt(n))) = ceil(log2(n) / 2), computed on integers */
    int lg = 0;
    while (((int64_t)1 << lg) < n) ++lg;       /* lg = ceil(log2 n) */
    int c = (lg + 1) / 2;                      /* ceil(ceil(log2 n)/2) = ceil(log2 sqrt n) */
    int b = 3 + c;
    while (b > 4 && (b > 16 || (((int64_t)1 << b) * x_bytes) > slice_budget_bytes)) --b;
    return b;
}

/* ----------------------------------------------------------- CRS -> blocked */

typedef struct { uint64_t key; int32_t row, col; int64_t src; } hb_ent;

static int cmp_hb(const void *a, const void *b) {
    const hb_ent *x = (const hb_ent *)a, *y = (const hb_ent *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->src != y->src) return x->src < y->src ? -1 : 1;
    return 0;
}

/*
 * CRS -> Hilbert-ordered blocked format (Section 4.2, BCOHC/BCOHCH storage with
 * one global ordering).  K = grid order; every nonzero gets the Hilbert index
 * h(r, c) on the 2^K grid; with inner_order 0 (Hilbert) nonzeros are sorted by h,
 * with inner_order 1 (row-wise inside blocks, BCOHC) by (h >> 2 log2beta, r, c).
 * Because every aligned beta x beta square is one contiguous range of the curve
 * (the recursive definition), each block is one run of the sorted sequence and the
 * blocks follow the Hilbert order.  Output: packed in-block indices
 * ((r mod beta) << 16) | (c mod beta) (row in the high half, Section 3.1),
 * values, blk_ptr (nblk+1), blk_row and blk_col (block coordinates).
 * Arrays idx/val_out hold nnz entries; blk_* hold up to nnz (+1) entries.
 */
int oracle_csr_to_hb(int64_t m, int64_t n, const int32_t *row_ptr, const int32_t *col_ind,
                     const double *data, int log2beta, int inner_order, uint32_t *idx,
                     double *val_out, int32_t *blk_ptr, int32_t *blk_row, int32_t *blk_col,
                     int64_t *nblk_out) {
    if (log2beta < 1 || log2beta > 16) return ERR_INVALID_ARG;
    int K = oracle_grid_order(m, n);
    if (log2beta > K) log2beta = K;
    int64_t nnz = row_ptr[m];
    hb_ent *e = (hb_ent *)malloc(sizeof(hb_ent) * (size_t)(nnz > 0 ? nnz : 1));
    if (!e) return ERR_OOM;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t j = col_ind[k];
            uint64_t h = oracle_hilbert_index(K, i, j);
            if (inner_order == 1) {
                uint64_t blk = h >> (2 * log2beta);
                uint64_t mask = ((uint64_t)1 << log2beta) - 1;
                h = (blk << (2 * log2beta)) | (((uint64_t)i & mask) << log2beta) | ((uint64_t)j & mask);
            }
            e[k].key = h; e[k].row = (int32_t)i; e[k].col = (int32_t)j; e[k].src = k;
        }
    qsort(e, (size_t)nnz, sizeof(hb_ent), cmp_hb);
    int64_t nb = 0;
    uint64_t mask = ((uint64_t)1 << log2beta) - 1;
    for (int64_t t = 0; t < nnz; ++t) {
        uint64_t blk = e[t].key >> (2 * log2beta);
        if (t == 0 || blk != (e[t - 1].key >> (2 * log2beta))) {
            blk_ptr[nb] = (int32_t)t;
            blk_row[nb] = (int32_t)(e[t].row >> log2beta);
            blk_col[nb] = (int32_t)(e[t].col >> log2beta);
            ++nb;
        }
        idx[t] = (uint32_t)((((uint64_t)e[t].row & mask) << 16) | ((uint64_t)e[t].col & mask));
        if (data && val_out) val_out[t] = data[e[t].src];
    }
    blk_ptr[nb] = (int32_t)nnz;
    *nblk_out = nb;
    free(e);
    return OK;
}

/*
 * CRS -> compressed sparse blocks (Section 3.1, CSB, and Section 4.1, CSBH): the beta x beta
 * blocks in row-major block order (block rows top to bottom, left to right inside a block
 * row) and, inside every block, the nonzeros in Z-Morton order (inner_order 2: the row bit
 * above the column bit at every level, the Z-Morton figure), in the Hilbert order of the
 * block's own curve (inner_order 0, CSBH) or row by row (inner_order 1).  Same output arrays
 * as oracle_csr_to_hb.
 */
int oracle_csr_to_csb(int64_t m, int64_t n, const int32_t *row_ptr, const int32_t *col_ind, const double *data,
                      int log2beta, int inner_order, uint32_t *idx, double *val_out, int32_t *blk_ptr,
                      int32_t *blk_row, int32_t *blk_col, int64_t *nblk_out) {
    if (log2beta < 1 || log2beta > 16 || inner_order < 0 || inner_order > 2) return ERR_INVALID_ARG;
    int K = oracle_grid_order(m, n);
    if (log2beta > K) log2beta = K;
    int64_t nnz = row_ptr[m];
    hb_ent *e = (hb_ent *)malloc(sizeof(hb_ent) * (size_t)(nnz > 0 ? nnz : 1));
    if (!e) return ERR_OOM;
    const int64_t bcols = (int64_t)1 << (K - log2beta);   /* blocks per block row */
    const uint64_t mask = ((uint64_t)1 << log2beta) - 1;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t j = col_ind[k];
            uint64_t blk = (uint64_t)((i >> log2beta) * bcols + (j >> log2beta));
            int64_t ri = i & (int64_t)mask, cj = j & (int64_t)mask;
            uint64_t inner;
            if (inner_order == 2) inner = oracle_zmorton_index(log2beta, ri, cj);
            else if (inner_order == 0) inner = oracle_hilbert_index(log2beta, ri, cj);
            else inner = ((uint64_t)ri << log2beta) | (uint64_t)cj;
            e[k].key = (blk << (2 * log2beta)) | inner;
            e[k].row = (int32_t)i; e[k].col = (int32_t)j; e[k].src = k;
        }
    qsort(e, (size_t)nnz, sizeof(hb_ent), cmp_hb);
    int64_t nb = 0;
    for (int64_t t = 0; t < nnz; ++t) {
        uint64_t blk = e[t].key >> (2 * log2beta);
        if (t == 0 || blk != (e[t - 1].key >> (2 * log2beta))) {
            blk_ptr[nb] = (int32_t)t;
            blk_row[nb] = (int32_t)(e[t].row >> log2beta);
            blk_col[nb] = (int32_t)(e[t].col >> log2beta);
            ++nb;
        }
        idx[t] = (uint32_t)((((uint64_t)e[t].row & mask) << 16) | ((uint64_t)e[t].col & mask));
        if (data && val_out) val_out[t] = data[e[t].src];
    }
    blk_ptr[nb] = (int32_t)nnz;
    *nblk_out = nb;
    free(e);
    return OK;
}

/* Product over the blocked structure: y = 0, then blocks in stored order, entries
 * in stored order, y[r] = y[r] + v * x[c]. */
void oracle_hb_spmv(int64_t m, int64_t nblk, int log2beta, const int32_t *blk_ptr, const int32_t *blk_row,
                    const int32_t *blk_col, const uint32_t *idx, const double *data, const double *x,
                    double *y) {
    for (int64_t i = 0; i < m; ++i) y[i] = 0.0;
    for (int64_t b = 0; b < nblk; ++b) {
        int64_t r0 = (int64_t)blk_row[b] << log2beta, c0 = (int64_t)blk_col[b] << log2beta;
        for (int64_t t = blk_ptr[b]; t < blk_ptr[b + 1]; ++t) {
            int64_t r = r0 + (idx[t] >> 16), c = c0 + (idx[t] & 0xFFFF);
            double a = data ? data[t] : 1.0;
            double prod = a * x[c];
            y[r] = y[r] + prod;
        }
    }
}

/* -------------------------------------------------------------- merge path */

/*
 * Merge-path split on diagonal `diag` (Section 3.3 and the merge-path figure):
 * list A (length alen, sorted) against list B (length blen, sorted); returns the
 * number of A items (ai) and B items (bi = diag - ai) consumed by the first
 * `diag` steps of the merge, where a step consumes the smaller head and a tie
 * consumes the A item.  Written as the plain merge walk, O(diag).
 */
void oracle_merge_path_walk(int64_t diag, const int64_t *A, int64_t alen, const int64_t *B, int64_t blen,
                            int64_t *ai, int64_t *bi) {
    int64_t i = 0, j = 0;
    for (int64_t s = 0; s < diag; ++s) {
        if (i < alen && (j >= blen || A[i] <= B[j])) ++i;
        else ++j;
    }
    *ai = i; *bi = j;
}

/*
 * The same split for the SpMV lists of Section 3.3: A = row_ptr[1..m] (row ends),
 * B = 0, 1, ..., nnz-1 (nonzero indices).  Found by bisection on the diagonal:
 * the split takes the largest i such that the first i row ends all come before
 * the nonzero index they are compared with (A[i-1] <= B[diag-i]).
 */
void oracle_merge_path_search(int64_t diag, int64_t m, const int32_t *row_ptr, int64_t nnz, int64_t *ai,
                              int64_t *bi) {
    int64_t lo = diag - nnz > 0 ? diag - nnz : 0;
    int64_t hi = diag < m ? diag : m;
    while (lo < hi) {
        int64_t i = lo + (hi - lo + 1) / 2;   /* candidate: i row ends consumed */
        /* consuming i row ends and diag-i nonzeros is on the path iff row end i-1
           does not come after nonzero diag-i, i.e. row_ptr[i] <= diag - i */
        if ((int64_t)row_ptr[i] <= diag - i) lo = i; else hi = i - 1;
    }
    *ai = lo; *bi = diag - lo;
}

/*
 * Merge-based CRS SpMV (Section 3.3), `parts` parts executed one after another:
 * the path of length m + nnz is cut into `parts` equal diagonal bands (the last
 * may be shorter: part p covers diagonals [p*L, min((p+1)*L, m+nnz)) with
 * L = ceil((m+nnz)/parts)).  Each part walks its band with temp = 0: consuming
 * nonzero k does temp = temp + data[k]*x[col[k]]; consuming row end i writes
 * y[i] = temp and resets temp.  At the end of its band a part keeps (row, temp)
 * as its carry.  After all parts, carries are added into y in part order.
 * carry_row/carry_val (parts entries) may be NULL.
 */
void oracle_merge_spmv(int64_t m, const int32_t *row_ptr, const int32_t *col_ind, const double *data,
                       const double *x, double *y, int64_t parts, int64_t *carry_row, double *carry_val) {
    int64_t nnz = row_ptr[m];
    int64_t total = m + nnz;
    if (parts < 1) parts = 1;
    int64_t L = (total + parts - 1) / parts;
    for (int64_t i = 0; i < m; ++i) y[i] = 0.0;
    int64_t *cr = (int64_t *)malloc(sizeof(int64_t) * (size_t)parts);
    double *cv = (double *)malloc(sizeof(double) * (size_t)parts);
    for (int64_t p = 0; p < parts; ++p) {
        int64_t d0 = p * L < total ? p * L : total, d1 = (p + 1) * L < total ? (p + 1) * L : total;
        int64_t i, k, i1, k1;
        oracle_merge_path_search(d0, m, row_ptr, nnz, &i, &k);
        oracle_merge_path_search(d1, m, row_ptr, nnz, &i1, &k1);
        double temp = 0.0;
        while (i < i1 || k < k1) {
            if (i < i1 && (int64_t)row_ptr[i + 1] <= k) {   /* row end i comes first */
                y[i] = temp; temp = 0.0; ++i;
            } else {
                double a = data ? data[k] : 1.0;
                double prod = a * x[col_ind[k]];
                temp = temp + prod; ++k;
            }
        }
        cr[p] = i; cv[p] = temp;
    }
    for (int64_t p = 0; p < parts; ++p) {
        if (cr[p] < m) y[cr[p]] = y[cr[p]] + cv[p];
        if (carry_row) carry_row[p] = cr[p];
        if (carry_val) carry_val[p] = cv[p];
    }
    free(cr); free(cv);
}

/* --------------------------------------------------------- merge blocking */

/*
 * Block-row pointer of blocks stored in row-major block order (Section 4.3, Merge Blocking:
 * the block matrix is kept in CRS, its "nonzeros" being the non-empty blocks):
 * ptr[i] = the number of blocks whose block row is below i, for i = 0..nbr, so that the
 * blocks of block row i are ptr[i] .. ptr[i+1]-1 and ptr[nbr] = nblk.
 */
void oracle_block_row_ptr(int64_t nblk, const int32_t *blk_row, int64_t nbr, int32_t *ptr) {
    int64_t b = 0;
    for (int64_t i = 0; i <= nbr; ++i) {
        while (b < nblk && (int64_t)blk_row[b] < i) ++b;
        ptr[i] = (int32_t)b;
    }
}

/*
 * Merge Blocking SpMV (Section 4.3, MergeB; MergeBH has the same product over blocks whose
 * entries follow the block's Hilbert curve): the merge-based product of Section 3.3 applied
 * to the block matrix.  Its path merges A = the block-row ends (blk_row_ptr[1..nbr]) with
 * B = the block indices 0..nblk-1 and is cut into `parts` equal diagonal bands as in
 * oracle_merge_spmv.  Each part walks its band with a temporary vector temp[0..beta) = 0:
 * consuming block b is the sparse block product, temp[r mod beta] += v * x[c] over the
 * block's entries in storage order (r = blk_row*beta + (idx >> 16), c = blk_col[b]*beta +
 * (idx & 0xFFFF)); consuming the end of block row i copies temp into rows i*beta .. of y
 * (those below m) and resets it.  At the end of its band a part keeps (block row, temp) as
 * its carry; after all parts the carries are added into y in part order.  A tie between a
 * block-row end and a block consumes the block-row end (the rule of Section 3.3).
 * data == NULL: pattern matrix.  Returns ERR_OOM if the carry vectors cannot be allocated.
 */
int oracle_mergeb_spmv(int64_t m, int64_t nbr, int log2beta, const int32_t *blk_row_ptr, const int32_t *blk_ptr,
                       const int32_t *blk_col, const uint32_t *idx, const double *data, const double *x,
                       double *y, int64_t parts) {
    const int64_t beta = (int64_t)1 << log2beta;
    const int64_t nblk = blk_row_ptr[nbr];
    const int64_t total = nbr + nblk;
    if (parts < 1) parts = 1;
    const int64_t L = (total + parts - 1) / parts;
    double *temp = (double *)calloc((size_t)beta, sizeof(double));
    double *cv = (double *)calloc((size_t)(parts * beta), sizeof(double));
    int64_t *cr = (int64_t *)malloc(sizeof(int64_t) * (size_t)parts);
    if (!temp || !cv || !cr) { free(temp); free(cv); free(cr); return ERR_OOM; }
    for (int64_t i = 0; i < m; ++i) y[i] = 0.0;
    for (int64_t p = 0; p < parts; ++p) {
        int64_t d0 = p * L < total ? p * L : total, d1 = (p + 1) * L < total ? (p + 1) * L : total;
        int64_t i, b, i1, b1;
        /* blk_row_ptr plays row_ptr's part: block-row ends against block indices */
        oracle_merge_path_search(d0, nbr, blk_row_ptr, nblk, &i, &b);
        oracle_merge_path_search(d1, nbr, blk_row_ptr, nblk, &i1, &b1);
        for (int64_t r = 0; r < beta; ++r) temp[r] = 0.0;
        while (i < i1 || b < b1) {
            if (i < i1 && (int64_t)blk_row_ptr[i + 1] <= b) {   /* end of block row i comes first */
                for (int64_t r = 0; r < beta && i * beta + r < m; ++r) y[i * beta + r] = temp[r];
                for (int64_t r = 0; r < beta; ++r) temp[r] = 0.0;
                ++i;
            } else {   /* block b: the sparse block multiplication into temp */
                const int64_t c0 = (int64_t)blk_col[b] << log2beta;
                for (int64_t t = blk_ptr[b]; t < blk_ptr[b + 1]; ++t) {
                    const int64_t r = idx[t] >> 16, c = c0 + (idx[t] & 0xFFFF);
                    double a = data ? data[t] : 1.0;
                    double prod = a * x[c];
                    temp[r] = temp[r] + prod;
                }
                ++b;
            }
        }
        cr[p] = i;
        for (int64_t r = 0; r < beta; ++r) cv[p * beta + r] = temp[r];
    }
    for (int64_t p = 0; p < parts; ++p)
        if (cr[p] < nbr)
            for (int64_t r = 0; r < beta && cr[p] * beta + r < m; ++r)
                y[cr[p] * beta + r] = y[cr[p] * beta + r] + cv[p * beta + r];
    free(temp); free(cv); free(cr);
    return OK;
}

/* ------------------------------------------------------------ precision */

/* Round a double to the nearest float, ties to even (C conversion under the
 * default rounding mode). */
float oracle_round_f32(double v) { return (float)v; }

/*
 * Round a double to bfloat16 (1 sign, 8 exponent, 7 fraction bits), to nearest
 * with ties to even, directly from the double (no intermediate float, so no
 * double rounding).  Returns the 16-bit pattern.  Values beyond the bfloat16
 * range round to infinity; NaN maps to a quiet NaN.
 */
uint16_t oracle_round_bf16(double v) {
    if (isnan(v)) return 0x7FC0;
    uint16_t sign = signbit(v) ? 0x8000 : 0;
    double a = fabs(v);
    if (a == 0.0) return sign;
    /* bfloat16 grid: normal numbers have 8 significant bits; the smallest normal
       is 2^-126 and the subnormal spacing is 2^-133 */
    int e;
    frexp(a, &e);                   /* a = f * 2^e, f in [0.5, 1) */
    int exp_unbiased = e - 1;       /* a in [2^exp, 2^(exp+1)) */
    int q = exp_unbiased < -126 ? -133 : exp_unbiased - 7;   /* spacing exponent */
    double scaled = ldexp(a, -q);   /* exact: a / 2^q */
    double fl = floor(scaled);
    double rem = scaled - fl;
    double rq;
    if (rem > 0.5) rq = fl + 1.0;
    else if (rem < 0.5) rq = fl;
    else rq = (fmod(fl, 2.0) == 0.0) ? fl : fl + 1.0;
    double r = ldexp(rq, q);
    if (r > 3.3895313892515355e38) return sign | 0x7F80;   /* above the largest finite bfloat16 */
    /* encode r exactly as bfloat16 */
    float f = (float)r;             /* exact: r has at most 8 significant bits */
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)(sign | ((u >> 16) & 0x7FFF));
}

double oracle_bf16_to_double(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* ---------------------------------------------------------------- PageRank */

/*
 * PageRank power iteration on a pattern matrix (Section 1 names PageRank as an
 * SpMV application; the paper does not define the iteration, so it is written
 * out here).  A_ij = 1 for an edge j -> i; out-degree of j = column sum;
 * P = A D^{-1}.  x0 = 1/n; for each iteration:
 *   dangling = sum of x_j over columns with zero out-degree,
 *   x_i <- d * ( (A (x / outdeg))_i + dangling / n ) + (1 - d) / n.
 * The product uses Algorithm 1 on the vector z_j = x_j / outdeg_j (0 for
 * dangling j).  Square matrices only.
 */
int oracle_pagerank(int64_t n, const int32_t *row_ptr, const int32_t *col_ind, double damping, int iters,
                    double *x) {
    int64_t nnz = row_ptr[n];
    double *deg = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *z = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!deg || !z || !y) { free(deg); free(z); free(y); return ERR_OOM; }
    for (int64_t k = 0; k < nnz; ++k) deg[col_ind[k]] = deg[col_ind[k]] + 1.0;
    for (int64_t j = 0; j < n; ++j) x[j] = 1.0 / (double)n;
    for (int it = 0; it < iters; ++it) {
        double dangling = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (deg[j] == 0.0) { dangling = dangling + x[j]; z[j] = 0.0; }
            else z[j] = x[j] / deg[j];
        }
        oracle_csr_spmv(n, row_ptr, col_ind, NULL, z, y);
        double tele = (1.0 - damping) / (double)n;
        double dshare = dangling / (double)n;
        for (int64_t i = 0; i < n; ++i) x[i] = damping * (y[i] + dshare) + tele;
    }
    free(deg); free(z); free(y);
    return OK;
}

/* ---------------------------------------------------------------- conjugate gradients */

/*
 * Conjugate gradients (Hestenes and Stiefel, 1952) for a symmetric positive definite A in
 * CRS form, x0 = 0, every product by Algorithm 1 (oracle_csr_spmv), every dot product a
 * left-to-right FP64 sum.  Iterates while the recursive residual norm exceeds tol * ||b|| and
 * fewer than max_iters iterations ran.  Returns the iteration count; *resid = ||r||.
 */
int oracle_cg(int64_t n, const int32_t *row_ptr, const int32_t *col_ind, const double *data, const double *b,
              double tol, int max_iters, double *x, double *resid) {
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *p = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *q = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!r || !p || !q) { free(r); free(p); free(q); return -1; }
    double rho = 0.0;
    for (int64_t i = 0; i < n; ++i) { x[i] = 0.0; r[i] = b[i]; p[i] = b[i]; rho = rho + r[i] * r[i]; }
    const double stop = tol * sqrt(rho);
    int it = 0;
    while (it < max_iters && sqrt(rho) > stop) {
        oracle_csr_spmv(n, row_ptr, col_ind, data, p, q);
        double pq = 0.0;
        for (int64_t i = 0; i < n; ++i) pq = pq + p[i] * q[i];
        const double alpha = pq != 0.0 ? rho / pq : 0.0;
        double rho1 = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            x[i] = x[i] + alpha * p[i];
            r[i] = r[i] - alpha * q[i];
            rho1 = rho1 + r[i] * r[i];
        }
        const double beta = rho != 0.0 ? rho1 / rho : 0.0;
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rho = rho1;
        ++it;
    }
    if (resid) *resid = sqrt(rho);
    free(r); free(p); free(q);
    return it;
}
