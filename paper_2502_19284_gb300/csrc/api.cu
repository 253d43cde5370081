// C ABI of libspmv (declared in include/spmv.h): argument checking, handle life cycle,
// format dispatch.  Every entry point returns a status; none aborts.
#include "common.cuh"
#include "convert.cuh"

#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <vector>

namespace spmv {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

spmv_status cuda_status(cudaError_t e, const char *what) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    g_err = buf;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();   // clear the sticky-free allocation error
        return SPMV_ERR_OOM;
    }
    return SPMV_ERR_CUDA;
}

// ---------------------------------------------------------------- memory
static std::atomic<long long> g_fail_after{-1};   // allocations left before an injected failure
static std::once_flag g_pool_once;

static void configure_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;   // keep freed blocks cached in the pool
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
}

spmv_status set_smem_ctas(const void *kernel, size_t bytes, int ctas) {
    int dev = 0, per_sm = 0, reserved = 0;
    SPMV_CUDA_TRY(cudaGetDevice(&dev));
    SPMV_CUDA_TRY(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    SPMV_CUDA_TRY(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
    const size_t need = (size_t)ctas * (bytes + (size_t)reserved);
    const int pct = per_sm > 0 ? (int)std::min<size_t>(100, (need * 100 + per_sm - 1) / per_sm) : 100;
    SPMV_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    SPMV_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    return SPMV_OK;
}

spmv_status set_smem(const void *kernel, size_t bytes) {
    SPMV_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    SPMV_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared));
    return SPMV_OK;
}

spmv_status dev_alloc(void **p, size_t bytes, const char *what, cudaStream_t s) {
    *p = nullptr;
    long long left = g_fail_after.load();
    if (left >= 0) {
        if (left == 0) {
            g_err = std::string(what) + ": injected allocation failure";
            return SPMV_ERR_OOM;
        }
        g_fail_after.fetch_sub(1);
    }
    std::call_once(g_pool_once, configure_pool);
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_status(e, what);
    }
    return SPMV_OK;
}

void dev_free(void *p) {
    if (p) cudaFree(p);
}

void dev_free_async(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

// ---------------------------------------------------------------- tracing
namespace {
struct TraceRec {
    const char *name;
    cudaEvent_t a, b;
};
struct TraceAgg {
    const char *name;
    long long count;
    double ms;
};
std::atomic<bool> g_trace{false};
std::mutex g_trace_mu;
std::vector<TraceRec> g_trace_pending;
std::vector<TraceAgg> g_trace_table;
}  // namespace

bool trace_on() { return g_trace.load(std::memory_order_relaxed); }

TraceScope::TraceScope(const char *n, cudaStream_t st) : name(n), s(st) {
    if (!trace_on()) return;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventRecord(a, s) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        a = nullptr;
    }
}

TraceScope::~TraceScope() {
    if (!a) return;
    cudaEvent_t b = nullptr;
    if (cudaEventCreate(&b) != cudaSuccess || cudaEventRecord(b, s) != cudaSuccess) {
        cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        return;
    }
    std::lock_guard<std::mutex> g(g_trace_mu);
    g_trace_pending.push_back({name, a, b});
}

static void trace_drain() {   // caller holds g_trace_mu; device already synchronised
    for (auto &r : g_trace_pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
        bool found = false;
        for (auto &t : g_trace_table)
            if (strcmp(t.name, r.name) == 0) {
                t.count += 1;
                t.ms += ms;
                found = true;
                break;
            }
        if (!found) g_trace_table.push_back({r.name, 1, (double)ms});
    }
    g_trace_pending.clear();
}

}  // namespace spmv

using namespace spmv;

namespace {


spmv_status check_handle(spmv_handle h) {
    if (!h) {
        set_error("NULL handle");
        return SPMV_ERR_INVALID_ARG;
    }
    return SPMV_OK;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Pinned 16-byte status slots, carved from 4 KB pinned pages that are kept for the life of
// the process: a handle takes one instead of a page-locking allocation of its own.
std::mutex g_pin_mu;
std::vector<uint32_t *> g_pin_free;

uint32_t *pinned_slot() {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        void *page = nullptr;
        if (cudaMallocHost(&page, 4096) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (int i = 4096 / 16 - 1; i >= 0; --i) g_pin_free.push_back((uint32_t *)((char *)page + 16 * i));
    }
    uint32_t *p = g_pin_free.back();
    g_pin_free.pop_back();
    return p;
}

void release_slot(uint32_t *p) {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}

void free_all(spmv_matrix *h) {
    void *ptrs[] = {h->coo_row, h->coo_col, h->coo_val, h->row_ptr, h->col, h->val, h->bin_rows,
                    h->part_row, h->part_nz, h->carry_row, h->carry_val, h->merge_desc, h->hb_idx, h->hb_val,
                    h->blk_ptr, h->blk_row, h->blk_col, h->hb_chunk_blk, h->st_hdr, h->st_words, h->st_vals, h->st_slice_tile, h->st_lmeta, h->st_part, h->xsplit, h->xsplit_flag, h->slot_desc, h->slot_col, h->slot_val2, h->slot_val, h->fix_len, h->fix_long, h->mb_row_ptr, h->mb_desc,
                    h->pr_inv, h->pr_z, h->pr_z2, h->pr_y, h->pr_part, h->status_dev};
    if (h->pr_graph) cudaGraphExecDestroy((cudaGraphExec_t)h->pr_graph);
    for (void *p : ptrs) dev_free(p);
    if (h->status_host) release_slot(h->status_host);
}

// Eq. 2 rule (Section 3.1) for the block side: start at 3 + ceil(log2 sqrt(n)) and
// lower it until beta <= 2^16 and the x slice of one block fits the on-chip budget.
int default_log2_beta(int64_t n, int x_bytes) {
    int lg = 0;
    while (((int64_t)1 << lg) < n) ++lg;
    int b = 3 + (lg + 1) / 2;
    const int64_t budget = 200 * 1024;
    while (b > 4 && (b > 16 || (((int64_t)1 << b) * x_bytes) > budget)) --b;
    return b;
}

}  // namespace

extern "C" {

const char *spmv_last_error(void) { return g_err.c_str(); }

const char *spmv_status_string(spmv_status s) {
    switch (s) {
        case SPMV_OK: return "SPMV_OK";
        case SPMV_ERR_INVALID_ARG: return "SPMV_ERR_INVALID_ARG";
        case SPMV_ERR_INDEX_RANGE: return "SPMV_ERR_INDEX_RANGE";
        case SPMV_ERR_DUPLICATE: return "SPMV_ERR_DUPLICATE";
        case SPMV_ERR_OOM: return "SPMV_ERR_OOM";
        case SPMV_ERR_UNSUPPORTED: return "SPMV_ERR_UNSUPPORTED";
        case SPMV_ERR_CUDA: return "SPMV_ERR_CUDA";
        case SPMV_ERR_TIMEOUT: return "SPMV_ERR_TIMEOUT";
        case SPMV_ERR_NOT_CONVERTED: return "SPMV_ERR_NOT_CONVERTED";
        case SPMV_ERR_IO: return "SPMV_ERR_IO";
    }
    return "SPMV_ERR_UNKNOWN";
}

// Host-side fault injection for tests: the allocation after `n` more successful ones
// fails with SPMV_ERR_OOM (n < 0 disables).
void spmv_test_fail_alloc(long long n) { g_fail_after.store(n); }

// Device-side check of the bounded waits: a kernel waits on an mbarrier that nothing arrives
// at, gives up after `polls` polls and reports ST_TIMEOUT through a status word.
spmv_status spmv_test_wait_timeout(long long polls, uint32_t *status_out) {
    g_err.clear();
    if (polls < 1 || polls > (1ll << 22) || !status_out) {
        set_error("spmv_test_wait_timeout: polls outside [1, 2^22] or NULL output");
        return SPMV_ERR_INVALID_ARG;
    }
    uint32_t *word = nullptr;
    cudaStream_t s = nullptr;
    SPMV_TRY(dev_alloc((void **)&word, 16, "test status word", s));
    spmv_status st = SPMV_OK;
    cudaError_t e = cudaMemsetAsync(word, 0, 4, s);
    if (e != cudaSuccess) st = cuda_status(e, "memset");
    if (st == SPMV_OK) st = test_wait(polls, word, s);
    if (st == SPMV_OK && (e = cudaMemcpy(status_out, word, 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
        st = cuda_status(e, "status read");
    dev_free(word);
    return st;
}

spmv_status spmv_trace_enable(int on) {
    cudaError_t e = cudaDeviceSynchronize();
    {
        std::lock_guard<std::mutex> g(g_trace_mu);
        trace_drain();
        g_trace_table.clear();
        g_trace.store(on != 0);
    }
    if (e != cudaSuccess) return cuda_status(e, "spmv_trace_enable");
    return SPMV_OK;
}

int spmv_trace_read(int max_entries, const char **names, long long *counts, double *total_ms) {
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    std::lock_guard<std::mutex> g(g_trace_mu);
    trace_drain();
    int n = (int)g_trace_table.size();
    for (int i = 0; i < n && i < max_entries; ++i) {
        if (names) names[i] = g_trace_table[i].name;
        if (counts) counts[i] = g_trace_table[i].count;
        if (total_ms) total_ms[i] = g_trace_table[i].ms;
    }
    return n;
}

spmv_status spmv_create_coo(int64_t m, int64_t n, int64_t nnz, const int32_t *row_ind, const int32_t *col_ind,
                            const void *data, spmv_dtype dt, uint32_t flags, void *stream, spmv_handle *out) {
    g_err.clear();
    if (!out) {
        set_error("spmv_create_coo: out is NULL");
        return SPMV_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (m < 0 || n < 0 || nnz < 0) {
        set_error("spmv_create_coo: negative size");
        return SPMV_ERR_INVALID_ARG;
    }
    if (m >= ((int64_t)1 << 31) || n >= ((int64_t)1 << 31) || nnz >= ((int64_t)1 << 31)) {
        set_error("spmv_create_coo: m, n and nnz must be below 2^31 (int32 indices)");
        return SPMV_ERR_UNSUPPORTED;
    }
    if ((int)dt < 0 || (int)dt > 3 || (flags & ~0x3u)) {
        set_error("spmv_create_coo: unknown dtype or flag");
        return SPMV_ERR_INVALID_ARG;
    }
    if (nnz > 0 && (!row_ind || !col_ind || (dt != SPMV_PATTERN && !data))) {
        set_error("spmv_create_coo: NULL triplet array");
        return SPMV_ERR_INVALID_ARG;
    }
    const bool dev = (flags & SPMV_DEVICE_PTRS) != 0;
    if (nnz > 0 && dev && (!is_device_ptr(row_ind) || !is_device_ptr(col_ind) ||
                           (dt != SPMV_PATTERN && !is_device_ptr(data)))) {
        set_error("spmv_create_coo: SPMV_DEVICE_PTRS given but an array is not device memory");
        return SPMV_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    spmv_matrix *h = new (std::nothrow) spmv_matrix();
    if (!h) {
        set_error("spmv_create_coo: host allocation failed");
        return SPMV_ERR_OOM;
    }
    h->m = m;
    h->n = n;
    h->nnz_in = nnz;
    h->dt = dt;
    h->flags = flags;
    cudaGetDevice(&h->device);
    const int es = elem_size(dt);
    spmv_status st = SPMV_OK;
    auto fail = [&](spmv_status e) {
        cudaStreamSynchronize(s);
        free_all(h);
        delete h;
        return e;
    };
    if ((st = dev_alloc((void **)&h->status_dev, 16, "status word", s)) != SPMV_OK) return fail(st);
    if (!(h->status_host = pinned_slot())) return fail(cuda_status(cudaErrorMemoryAllocation, "pinned status slot"));
    if (cudaMemsetAsync(h->status_dev, 0, 16, s) != cudaSuccess) return fail(cuda_status(cudaGetLastError(), "memset"));
    if (nnz > 0) {
        if ((st = dev_alloc((void **)&h->coo_row, (size_t)nnz * 4, "triplet rows", s)) != SPMV_OK ||
            (st = dev_alloc((void **)&h->coo_col, (size_t)nnz * 4, "triplet cols", s)) != SPMV_OK ||
            (es && (st = dev_alloc(&h->coo_val, (size_t)nnz * es, "triplet values", s)) != SPMV_OK))
            return fail(st);
        cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        cudaError_t e = cudaMemcpyAsync(h->coo_row, row_ind, (size_t)nnz * 4, kind, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->coo_col, col_ind, (size_t)nnz * 4, kind, s);
        if (e == cudaSuccess && es) e = cudaMemcpyAsync(h->coo_val, data, (size_t)nnz * es, kind, s);
        if (e != cudaSuccess) return fail(cuda_status(e, "spmv_create_coo copy"));
        if ((st = launch_validate(h->coo_row, h->coo_col, nnz, m, n, h->status_dev, s)) != SPMV_OK) return fail(st);
        h->bytes = nnz * (8 + es);
    }
    cudaError_t e = cudaMemcpyAsync(h->status_host, h->status_dev, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_status(e, "spmv_create_coo sync"));
    if (*h->status_host & ST_INDEX_RANGE) {
        set_error("spmv_create_coo: a triplet index lies outside [0,m) x [0,n)");
        return fail(SPMV_ERR_INDEX_RANGE);
    }
    *out = h;
    return SPMV_OK;
}

spmv_status spmv_convert(spmv_handle h, spmv_format f, const spmv_convert_opts *opt, void *stream) {
    g_err.clear();
    SPMV_TRY(check_handle(h));
    forget_batch_plans(h);
    cudaStream_t s = (cudaStream_t)stream;
    spmv_convert_opts o = {0, SPMV_INNER_HILBERT, 0, SPMV_HB_STAGED, SPMV_BLOCK_HILBERT};
    if (opt) o = *opt;
    if (f == SPMV_FMT_AUTO) {
        // Row-length statistics decide: very long rows favour the merge path (it splits
        // rows across tiles); otherwise the row-split product.
        if (!h->has_csr) SPMV_TRY(build_csr(h, s));
        if (!h->has_bins) SPMV_TRY(build_bins(h, s));
        f = (h->max_row_len > 4096 || h->nnz > ((int64_t)1 << 20)) ? SPMV_FMT_CSR_MERGE : SPMV_FMT_CSR_ROWSPLIT;
    }
    if ((int)f < 0 || ((int)f > 2 && f != SPMV_FMT_MERGEB)) {
        set_error("spmv_convert: unknown format");
        return SPMV_ERR_INVALID_ARG;
    }
    if (o.inner_order != SPMV_INNER_HILBERT && o.inner_order != SPMV_INNER_ROWMAJOR &&
        o.inner_order != SPMV_INNER_ZMORTON) {
        set_error("spmv_convert: unknown inner order");
        return SPMV_ERR_INVALID_ARG;
    }
    if (o.block_order != SPMV_BLOCK_HILBERT && o.block_order != SPMV_BLOCK_ROWMAJOR) {
        set_error("spmv_convert: unknown block order");
        return SPMV_ERR_INVALID_ARG;
    }
    if (o.log2_beta < 0 || o.log2_beta > 16) {
        set_error("spmv_convert: log2_beta must be in [1, 16] (0 = Eq. 2 rule)");
        return SPMV_ERR_INVALID_ARG;
    }
    if (o.hb_product != SPMV_HB_STAGED && o.hb_product != SPMV_HB_CHUNKED) {
        set_error("spmv_convert: unknown HB product");
        return SPMV_ERR_INVALID_ARG;
    }
    if (o.tile != 0 && o.tile != MERGE_WARP_ITEMS) {
        set_error("spmv_convert: only the default merge tile (224 path items per warp) is built in");
        return SPMV_ERR_UNSUPPORTED;
    }
    if (!h->has_csr) SPMV_TRY(build_csr(h, s));
    if (f == SPMV_FMT_CSR_ROWSPLIT && !h->has_bins) SPMV_TRY(build_bins(h, s));
    if (f == SPMV_FMT_CSR_MERGE && !h->has_merge) SPMV_TRY(build_merge(h, MERGE_WARP_ITEMS, s));
    SPMV_TRY(build_df(h, s));
    if (f == SPMV_FMT_HB) {
        int lb = o.log2_beta ? o.log2_beta : default_log2_beta(h->n, h->dt == SPMV_F64 ? 8 : 4);
        const int K = bits_for(std::max<int64_t>(std::max(h->m, h->n), 2));
        if (lb > K) lb = K;
        if (!h->has_hb || h->log2beta != lb || h->inner != o.inner_order || h->block_order != o.block_order)
            SPMV_TRY(build_hb(h, lb, o.inner_order, s, o.block_order));
        if (o.hb_product == SPMV_HB_STAGED && (!h->has_stage || h->stage_lb != lb)) SPMV_TRY(build_stage(h, lb, s));
        h->hb_chunked = o.hb_product == SPMV_HB_CHUNKED;
    }
    if (f == SPMV_FMT_MERGEB) {
        int lb = o.log2_beta ? o.log2_beta : default_log2_beta(h->n, h->dt == SPMV_F64 ? 8 : 4);
        const int K = bits_for(std::max<int64_t>(std::max(h->m, h->n), 2));
        if (lb > K) lb = K;
        if (!h->has_hb || h->log2beta != lb || h->inner != o.inner_order || h->block_order != SPMV_BLOCK_ROWMAJOR)
            SPMV_TRY(build_hb(h, lb, o.inner_order, s, SPMV_BLOCK_ROWMAJOR));
        if (!h->has_mergeb) SPMV_TRY(build_mergeb(h, s));
    }
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    h->format = (int32_t)f;
    return SPMV_OK;
}

spmv_status spmv_mul(spmv_handle h, const void *x, void *y, spmv_dtype vec_dt, uint32_t accum, void *stream) {
    SPMV_TRY(check_handle(h));
    if (h->format < 0) {
        set_error("spmv_mul: call spmv_convert first");
        return SPMV_ERR_NOT_CONVERTED;
    }
    if ((h->n > 0 && !x) || (h->m > 0 && !y)) {
        set_error("spmv_mul: NULL vector");
        return SPMV_ERR_INVALID_ARG;
    }
    if (accum > SPMV_ACC_SEGMENT || (vec_dt != SPMV_F64 && vec_dt != SPMV_F32)) {
        set_error("spmv_mul: unknown vector dtype or accumulation mode");
        return SPMV_ERR_INVALID_ARG;
    }
    if (h->m == 0) return SPMV_OK;
    cudaStream_t s = (cudaStream_t)stream;
    switch (h->format) {
        case SPMV_FMT_CSR_MERGE: return mul_merge(h, x, y, vec_dt, accum, s);
        case SPMV_FMT_CSR_ROWSPLIT: return mul_rowsplit(h, x, y, vec_dt, accum, s);
        case SPMV_FMT_HB: return mul_hb(h, x, y, vec_dt, accum, s);
        case SPMV_FMT_MERGEB: return mul_mergeb(h, x, y, vec_dt, accum, s);
    }
    set_error("spmv_mul: bad format");
    return SPMV_ERR_INVALID_ARG;
}

spmv_status spmv_wait(spmv_handle h, void *stream) {
    g_err.clear();
    SPMV_TRY(check_handle(h));
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(h->status_host + 3, h->status_dev + 3, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e, "spmv_wait");
    if (h->status_host[3] & ST_TIMEOUT) {
        if ((e = cudaMemsetAsync(h->status_dev + 3, 0, 4, s)) != cudaSuccess) return cuda_status(e, "spmv_wait");
        set_error("spmv_wait: a bounded device wait of a product gave up");
        return SPMV_ERR_TIMEOUT;
    }
    return SPMV_OK;
}

spmv_status spmv_tune(spmv_handle h, spmv_dtype vec_dt, uint32_t accum, uint32_t flags, spmv_tune_result *out,
                      void *stream) {
    g_err.clear();
    SPMV_TRY(check_handle(h));
    if ((vec_dt != SPMV_F64 && vec_dt != SPMV_F32) || accum > SPMV_ACC_SEGMENT ||
        (flags & ~(uint32_t)(SPMV_TUNE_HB | SPMV_TUNE_MERGEB))) {
        set_error("spmv_tune: bad vector dtype, accumulation or flags");
        return SPMV_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    forget_batch_plans(h);
    if (!h->has_csr) SPMV_TRY(build_csr(h, s));
    if (!h->has_bins) SPMV_TRY(build_bins(h, s));
    if (!h->has_merge) SPMV_TRY(build_merge(h, MERGE_WARP_ITEMS, s));
    if (h->dt == SPMV_F64) SPMV_TRY(build_df(h, s));
    if ((flags & SPMV_TUNE_MERGEB) && !h->has_mergeb) {
        const int K = bits_for(std::max<int64_t>(std::max(h->m, h->n), 2));
        const int lb = std::min(default_log2_beta(h->n, h->dt == SPMV_F64 ? 8 : 4), K);
        if (!h->has_hb || h->block_order != SPMV_BLOCK_ROWMAJOR || h->log2beta != lb)
            SPMV_TRY(build_hb(h, lb, SPMV_INNER_ROWMAJOR, s, SPMV_BLOCK_ROWMAJOR));
        SPMV_TRY(build_mergeb(h, s));
    }
    if ((flags & SPMV_TUNE_HB) && !h->has_hb)
        SPMV_TRY(build_hb(h, default_log2_beta(h->n, h->dt == SPMV_F64 ? 8 : 4), SPMV_INNER_HILBERT, s));
    if ((flags & SPMV_TUNE_HB) && h->has_hb && !h->has_stage) SPMV_TRY(build_stage(h, h->log2beta, s));
    spmv_tune_result r;
    r.reps = 5;
    r.pad_ = 0;
    r.hb_product = SPMV_HB_STAGED;
    for (float &v : r.ms) v = -1.f;
    const int es = vec_dt == SPMV_F64 ? 8 : 4;
    DevBuf x(s), y(s);
    SPMV_TRY(x.alloc((size_t)std::max<int64_t>(h->n, 1) * es, "tune x"));
    SPMV_TRY(y.alloc((size_t)std::max<int64_t>(h->m, 1) * es, "tune y"));
    SPMV_CUDA_TRY(cudaMemsetAsync(x.p, 0, (size_t)std::max<int64_t>(h->n, 1) * es, s));
    const int32_t fmts[5] = {SPMV_FMT_CSR_ROWSPLIT, SPMV_FMT_CSR_MERGE, SPMV_FMT_HB, SPMV_FMT_HB, SPMV_FMT_MERGEB};
    const bool chunked[5] = {false, false, false, true, false};
    cudaEvent_t e0, e1;
    SPMV_CUDA_TRY(cudaEventCreate(&e0));
    SPMV_CUDA_TRY(cudaEventCreate(&e1));
    const int32_t keep = h->format;
    const bool keep_chunked = h->hb_chunked;
    spmv_status st = SPMV_OK;
    int best = -1;
    for (int f = 0; f < 5 && st == SPMV_OK; ++f) {
        if (fmts[f] == SPMV_FMT_HB && (!h->has_hb || (!chunked[f] && !h->has_stage))) continue;
        if (fmts[f] == SPMV_FMT_MERGEB && !h->has_mergeb) continue;
        h->format = fmts[f];
        h->hb_chunked = chunked[f];
        std::vector<float> t;
        for (int rep = 0; rep < 2 + 2 * r.reps && st == SPMV_OK; ++rep) {
            cudaEventRecord(e0, s);
            st = spmv_mul(h, x.p, y.p, vec_dt, accum, s);
            cudaEventRecord(e1, s);
            if (st == SPMV_ERR_UNSUPPORTED) break;   // this format lacks the product: skip it
            if (cudaEventSynchronize(e1) != cudaSuccess) st = cuda_status(cudaGetLastError(), "spmv_tune");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep >= 2) t.push_back(ms);
        }
        if (st == SPMV_ERR_UNSUPPORTED) {
            st = SPMV_OK;
            g_err.clear();
            continue;
        }
        if (st != SPMV_OK || t.empty()) break;
        std::sort(t.begin(), t.end());
        r.ms[f] = t[t.size() / 2];
        if (best < 0 || r.ms[f] < r.ms[best]) best = f;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SPMV_OK || best < 0) {
        h->format = keep;
        h->hb_chunked = keep_chunked;
        if (st == SPMV_OK) {
            set_error("spmv_tune: no format supports this product");
            st = SPMV_ERR_UNSUPPORTED;
        }
        return st;
    }
    h->format = fmts[best];
    h->hb_chunked = chunked[best];
    r.chosen = fmts[best];
    r.hb_product = chunked[best] ? SPMV_HB_CHUNKED : SPMV_HB_STAGED;
    if (out) *out = r;
    return SPMV_OK;
}

spmv_status spmv_mul_batch(int count, const spmv_handle *hs, int k, const void *const *X, void *const *Y,
                           spmv_dtype vec_dt, uint32_t accum, void *stream) {
    if (count < 0 || (count > 0 && (!hs || !X || !Y)) || k < 1 || k > 16) {
        set_error("spmv_mul_batch: bad arguments");
        return SPMV_ERR_INVALID_ARG;
    }
    if (vec_dt != SPMV_F64 && vec_dt != SPMV_F32) {
        set_error("spmv_mul_batch: vectors are SPMV_F64 or SPMV_F32");
        return SPMV_ERR_INVALID_ARG;
    }
    for (int i = 0; i < count; ++i) {
        SPMV_TRY(check_handle(hs[i]));
        if (!X[i] || !Y[i]) {
            set_error("spmv_mul_batch: null vector pointer");
            return SPMV_ERR_INVALID_ARG;
        }
        if (!hs[i]->has_csr) {
            set_error("spmv_mul_batch: handle not converted (call spmv_convert first)");
            return SPMV_ERR_NOT_CONVERTED;
        }
        // the batch runs on the merge-path tiles; build them for handles converted to
        // another format
        if (!hs[i]->has_merge) SPMV_TRY(build_merge(hs[i], MERGE_WARP_ITEMS, (cudaStream_t)stream));
    }
    // k = 1: a handle whose active format (spmv_convert or spmv_tune) is row-split or blocked
    // runs its own product; the others share the persistent merge-path launch
    if (k == 1) {
        std::vector<spmv_matrix *> mh;
        std::vector<const void *> mx;
        std::vector<void *> my;
        std::vector<int> own;
        for (int i = 0; i < count; ++i) {
            if (hs[i]->format == SPMV_FMT_CSR_ROWSPLIT || hs[i]->format == SPMV_FMT_HB ||
                hs[i]->format == SPMV_FMT_MERGEB) {
                own.push_back(i);
            } else {
                mh.push_back(hs[i]);
                mx.push_back(X[i]);
                my.push_back(Y[i]);
            }
        }
        if (!own.empty()) {
            cudaStream_t s = (cudaStream_t)stream;
            if (!mh.empty()) SPMV_TRY(mul_batch((int)mh.size(), mh.data(), 1, mx.data(), my.data(), vec_dt, accum, s));
            for (int i : own) {
                if (hs[i]->m == 0) continue;
                if (hs[i]->format == SPMV_FMT_HB) SPMV_TRY(mul_hb(hs[i], X[i], Y[i], vec_dt, accum, s));
                else if (hs[i]->format == SPMV_FMT_MERGEB) SPMV_TRY(mul_mergeb(hs[i], X[i], Y[i], vec_dt, accum, s));
                else SPMV_TRY(mul_rowsplit(hs[i], X[i], Y[i], vec_dt, accum, s));
            }
            return SPMV_OK;
        }
    }
    return mul_batch(count, (spmv_matrix *const *)hs, k, X, Y, vec_dt, accum, (cudaStream_t)stream);
}

spmv_status spmv_set_compensation_threshold(spmv_handle h, int64_t tau) {
    g_err.clear();
    SPMV_TRY(check_handle(h));
    if (tau < 0) {
        set_error("spmv_set_compensation_threshold: tau must be >= 0");
        return SPMV_ERR_INVALID_ARG;
    }
    h->comp_tau = tau;
    return SPMV_OK;
}

spmv_status spmv_destroy(spmv_handle h) {
    if (!h) return SPMV_OK;
    cudaError_t e = cudaDeviceSynchronize();
    forget_batch_plans(h);
    free_all(h);
    delete h;
    if (e != cudaSuccess) return cuda_status(e, "spmv_destroy");
    return SPMV_OK;
}

spmv_status spmv_info(spmv_handle h, spmv_info_t *out) {
    SPMV_TRY(check_handle(h));
    if (!out) return SPMV_ERR_INVALID_ARG;
    memset(out, 0, sizeof *out);
    out->m = h->m;
    out->n = h->n;
    out->nnz = h->has_csr ? h->nnz : h->nnz_in;
    out->format = h->format;
    out->dtype = h->dt;
    out->log2_beta = h->has_hb ? h->log2beta : 0;
    out->grid_order = h->has_hb ? h->grid_K : 0;
    out->nblk = h->nblk;
    out->merge_tiles = h->tiles;
    out->merge_tile_items = h->tile_items;
    out->hb_orders = h->has_hb ? 16 * h->block_order + h->inner : 0;
    out->device_bytes = h->bytes;
    out->block_rows = h->mb_nbr;
    out->mergeb_tiles = h->mb_tiles;
    return SPMV_OK;
}

spmv_status spmv_export_csr(spmv_handle h, int32_t *row_ptr, int32_t *col_ind, void *data) {
    SPMV_TRY(check_handle(h));
    if (!h->has_csr) {
        set_error("spmv_export_csr: no CRS arrays (convert first)");
        return SPMV_ERR_NOT_CONVERTED;
    }
    SPMV_CUDA_TRY(cudaDeviceSynchronize());
    if (row_ptr) SPMV_CUDA_TRY(cudaMemcpy(row_ptr, h->row_ptr, (size_t)(h->m + 1) * 4, cudaMemcpyDeviceToHost));
    if (col_ind && h->nnz) SPMV_CUDA_TRY(cudaMemcpy(col_ind, h->col, (size_t)h->nnz * 4, cudaMemcpyDeviceToHost));
    if (data && h->nnz && elem_size(h->dt))
        SPMV_CUDA_TRY(cudaMemcpy(data, h->val, (size_t)h->nnz * elem_size(h->dt), cudaMemcpyDeviceToHost));
    return SPMV_OK;
}

spmv_status spmv_export_hb(spmv_handle h, uint32_t *idx, void *data, int32_t *blk_ptr, int32_t *blk_row,
                           int32_t *blk_col) {
    SPMV_TRY(check_handle(h));
    if (!h->has_hb) {
        set_error("spmv_export_hb: no HB arrays (convert first)");
        return SPMV_ERR_NOT_CONVERTED;
    }
    SPMV_CUDA_TRY(cudaDeviceSynchronize());
    if (idx && h->nnz) SPMV_CUDA_TRY(cudaMemcpy(idx, h->hb_idx, (size_t)h->nnz * 4, cudaMemcpyDeviceToHost));
    if (data && h->nnz && elem_size(h->dt))
        SPMV_CUDA_TRY(cudaMemcpy(data, h->hb_val, (size_t)h->nnz * elem_size(h->dt), cudaMemcpyDeviceToHost));
    if (blk_ptr) SPMV_CUDA_TRY(cudaMemcpy(blk_ptr, h->blk_ptr, (size_t)(h->nblk + 1) * 4, cudaMemcpyDeviceToHost));
    if (blk_row && h->nblk) SPMV_CUDA_TRY(cudaMemcpy(blk_row, h->blk_row, (size_t)h->nblk * 4, cudaMemcpyDeviceToHost));
    if (blk_col && h->nblk) SPMV_CUDA_TRY(cudaMemcpy(blk_col, h->blk_col, (size_t)h->nblk * 4, cudaMemcpyDeviceToHost));
    return SPMV_OK;
}

spmv_status spmv_export_mergeb(spmv_handle h, int32_t *blk_row_ptr, int32_t *lane_entry, int32_t *lane_block) {
    SPMV_TRY(check_handle(h));
    if (!h->has_mergeb) {
        set_error("spmv_export_mergeb: no Merge Blocking tables (convert to MERGEB first)");
        return SPMV_ERR_NOT_CONVERTED;
    }
    SPMV_CUDA_TRY(cudaDeviceSynchronize());
    if (blk_row_ptr)
        SPMV_CUDA_TRY(cudaMemcpy(blk_row_ptr, h->mb_row_ptr, (size_t)(h->mb_nbr + 1) * 4, cudaMemcpyDeviceToHost));
    if ((lane_entry || lane_block) && h->mb_tiles > 0) {
        std::vector<int2> d((size_t)h->mb_tiles * 32);
        SPMV_CUDA_TRY(cudaMemcpy(d.data(), h->mb_desc, d.size() * sizeof(int2), cudaMemcpyDeviceToHost));
        for (size_t g = 0; g < d.size(); ++g) {
            if (lane_entry) lane_entry[g] = d[g].x;
            if (lane_block) lane_block[g] = d[g].y;
        }
    }
    return SPMV_OK;
}

spmv_status spmv_export_merge_partition(spmv_handle h, int32_t *row_start, int32_t *nz_start) {
    SPMV_TRY(check_handle(h));
    if (!h->has_merge) {
        set_error("spmv_export_merge_partition: no merge partition (convert to CSR_MERGE first)");
        return SPMV_ERR_NOT_CONVERTED;
    }
    SPMV_CUDA_TRY(cudaDeviceSynchronize());
    if (row_start) SPMV_CUDA_TRY(cudaMemcpy(row_start, h->part_row, (size_t)(h->tiles + 1) * 4, cudaMemcpyDeviceToHost));
    if (nz_start) SPMV_CUDA_TRY(cudaMemcpy(nz_start, h->part_nz, (size_t)(h->tiles + 1) * 4, cudaMemcpyDeviceToHost));
    return SPMV_OK;
}

spmv_status spmv_mul_csr_merge_noalloc(int64_t m, int64_t n, int64_t nnz, const int32_t *row_ptr,
                                       const int32_t *col_ind, const double *data, const double *x, double *y,
                                       void *stream) {
    g_err.clear();
    if (m < 0 || n < 0 || nnz < 0 || m >= ((int64_t)1 << 31) || n >= ((int64_t)1 << 31) ||
        nnz >= ((int64_t)1 << 31)) {
        set_error("spmv_mul_csr_merge_noalloc: sizes must lie in [0, 2^31)");
        return SPMV_ERR_INVALID_ARG;
    }
    if (!row_ptr || (nnz > 0 && (!col_ind || !data)) || (n > 0 && !x) || (m > 0 && !y)) {
        set_error("spmv_mul_csr_merge_noalloc: NULL array");
        return SPMV_ERR_INVALID_ARG;
    }
    if (m == 0) return SPMV_OK;
    return mul_csr_merge_noalloc(m, n, nnz, row_ptr, col_ind, data, x, y, (cudaStream_t)stream);
}

spmv_status spmv_pagerank(spmv_handle h, double damping, int iters, double *x, void *stream) {
    g_err.clear();
    SPMV_TRY(check_handle(h));
    if (h->m != h->n || !(damping >= 0.0 && damping <= 1.0) || iters < 0 || iters > 10000 || (h->n > 0 && !x)) {
        set_error("spmv_pagerank: needs a square matrix, damping in [0, 1], 0 <= iters <= 10000 and x");
        return SPMV_ERR_INVALID_ARG;
    }
    if (h->n == 0) return SPMV_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (!h->has_csr) SPMV_TRY(build_csr(h, s));
    if (!h->has_merge) SPMV_TRY(build_merge(h, MERGE_WARP_ITEMS, s));
    return pagerank(h, damping, iters, x, s);
}

spmv_status spmv_hilbert_keys(int K, int64_t n, const int32_t *rows, const int32_t *cols, uint64_t *keys,
                              void *stream) {
    if (K < 1 || K > 31 || n < 0 || (n > 0 && (!rows || !cols || !keys))) {
        set_error("spmv_hilbert_keys: bad arguments");
        return SPMV_ERR_INVALID_ARG;
    }
    return launch_hilbert_keys(K, n, rows, cols, keys, (cudaStream_t)stream);
}

}  // extern "C"
