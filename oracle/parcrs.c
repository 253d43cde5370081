/*
 * ParCRS -- the paper's row-parallel CRS product as a CPU BASELINE (not the oracle).
 *
 * TEST / BENCHMARK INFRASTRUCTURE ONLY: the benchmark times it on the host cores next to the
 * GPU products; nothing in the library loads it.  Section 5.1 describes the implementation
 * this restates: OpenMP parallelism over the rows of Algorithm 1 with a dynamic schedule in
 * chunks of 512 rows, threads bound to cores (OMP_PROC_BIND=true, which the caller sets in
 * the environment before this library is loaded).  Each thread forms whole row sums in FP64,
 * so the result equals the sequential oracle row for row (same order inside a row).
 */
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void parcrs_spmv(int64_t m, const int32_t *row_ptr, const int32_t *col_ind, const double *data, const double *x,
                 double *y) {
    int64_t i;
#pragma omp parallel for schedule(dynamic, 512)
    for (i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) s = s + data[k] * x[col_ind[k]];
        y[i] = s;
    }
}

/* Threads the parallel loop uses (1 when built without OpenMP). */
int parcrs_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
