// PageRank power iteration on the GPU.  The paper names PageRank as an application built on
// SpMV (Section 1) without defining it; the iteration computed here is
//   out-degree of column j = number of stored entries in column j (values ignored),
//   x0 = 1/n, and per iteration, with dangling = sum of x_j over columns of out-degree 0,
//   x_i <- d * ( (A z)_i + dangling / n ) + (1 - d) / n,   z_j = x_j / outdeg_j (0 if dangling).
// Each iteration is three fused kernels around the pattern product -- the merge-path product,
// or, when the handle's active format is HB with the staged product, the staged blocked
// product (x slices read once per CTA by bulk copies instead of gathered per nonzero, which
// matters once the split x no longer fits in L2; its summation order is not fixed):
//   prep    z = x * (1/outdeg), split into float pairs for the double-float product, and
//           per-block partial sums of the dangling mass (fixed order: deterministic);
//   dsum    one block adds the partials in a fixed tree order;
//   update  x = d (y + dangling/n) + (1 - d)/n.
// The whole iteration count is captured once into a CUDA graph per (handle, x, iterations,
// damping) and replayed.
#include "common.cuh"
#include "convert.cuh"
#include "df64.cuh"

namespace spmv {

namespace {

constexpr int PR_BLOCK = 256;
constexpr int PR_PARTS = 1024;   // blocks of the prep kernel (grid-stride), one partial each

__global__ void k_pr_degree(const int32_t *__restrict__ col, int64_t nnz, int32_t *__restrict__ deg) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&deg[col[k]], 1);
}

__global__ void k_pr_invdeg(const int32_t *__restrict__ deg, int64_t n, double *__restrict__ inv) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) inv[j] = deg[j] > 0 ? 1.0 / (double)deg[j] : 0.0;
}

__global__ void k_pr_init(double *__restrict__ x, int64_t n) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) x[j] = 1.0 / (double)n;
}

__global__ __launch_bounds__(PR_BLOCK) void k_pr_prep(const double *__restrict__ x, const double *__restrict__ inv,
                                                      int64_t n, double *__restrict__ z, float2 *__restrict__ z2,
                                                      uint32_t *__restrict__ flag, double *__restrict__ part) {
    double dang = 0.0;
    bool bad = false;
    for (int64_t j = (int64_t)blockIdx.x * PR_BLOCK + threadIdx.x; j < n; j += (int64_t)gridDim.x * PR_BLOCK) {
        const double xj = x[j], w = inv[j];
        const double zj = xj * w;
        if (w == 0.0) dang = dang + xj;
        z[j] = zj;
        float2 r;
        bad |= !df_split(zj, &r.x, &r.y);
        z2[j] = r;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
    __shared__ double ws[PR_BLOCK / 32];
    for (int o = 16; o > 0; o >>= 1) dang = dang + __shfl_down_sync(0xffffffffu, dang, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = dang;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < PR_BLOCK / 32; ++w) t = t + ws[w];
        part[blockIdx.x] = t;
    }
}

__global__ __launch_bounds__(PR_PARTS) void k_pr_dsum(const double *__restrict__ part, double *__restrict__ total) {
    __shared__ double s[PR_PARTS];
    s[threadIdx.x] = part[threadIdx.x];
    __syncthreads();
    for (int h = PR_PARTS / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) s[threadIdx.x] = s[threadIdx.x] + s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = s[0];
}

__global__ void k_pr_update(const double *__restrict__ y, const double *__restrict__ total, double damping,
                            int64_t n, double *__restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double share = *total / (double)n, tele = (1.0 - damping) / (double)n;
        x[i] = damping * (y[i] + share) + tele;
    }
}

inline unsigned blocks_for(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + 255) / 256); }

spmv_status pr_buffers(spmv_matrix *h, cudaStream_t s) {
    if (h->pr_inv) return SPMV_OK;
    const int64_t n = h->n;
    DevBuf deg(s), inv(s), z(s), z2(s), y(s), part(s);
    SPMV_TRY(deg.alloc((size_t)n * 4, "pagerank degrees"));
    SPMV_TRY(inv.alloc((size_t)n * 8, "pagerank 1/degree"));
    SPMV_TRY(z.alloc((size_t)n * 8, "pagerank z"));
    SPMV_TRY(z2.alloc((size_t)n * 8, "pagerank z split"));
    SPMV_TRY(y.alloc((size_t)n * 8, "pagerank y"));
    SPMV_TRY(part.alloc((size_t)(PR_PARTS + 2) * 8 + 16, "pagerank partials"));
    SPMV_CUDA_TRY(cudaMemsetAsync(deg.p, 0, (size_t)n * 4, s));
    if (h->nnz > 0)
        SPMV_LAUNCH("k_pr_degree", s, (k_pr_degree<<<1184, 256, 0, s>>>(h->col, h->nnz, deg.as<int32_t>())));
    SPMV_LAUNCH_CHECK("pagerank degree");
    SPMV_LAUNCH("k_pr_invdeg", s, (k_pr_invdeg<<<blocks_for(n), 256, 0, s>>>(deg.as<int32_t>(), n, inv.as<double>())));
    SPMV_LAUNCH_CHECK("pagerank inverse degree");
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));   // deg is scratch
    h->pr_inv = inv.as<double>();
    inv.release();
    h->pr_z = (double *)z.release();
    h->pr_z2 = (float2 *)z2.release();
    h->pr_y = (double *)y.release();
    h->pr_part = (double *)part.release();
    h->bytes += n * 32 + (PR_PARTS + 2) * 8 + 16;
    return SPMV_OK;
}

bool pr_staged(const spmv_matrix *h) {
    return h->format == SPMV_FMT_HB && h->has_stage && !h->hb_chunked && h->stage_tiles > 0;
}

spmv_status pr_enqueue(spmv_matrix *h, double damping, int iters, double *x, cudaStream_t s) {
    const bool staged = pr_staged(h);
    const int64_t n = h->n;
    double *total = h->pr_part + PR_PARTS;
    uint32_t *flag = (uint32_t *)(h->pr_part + PR_PARTS + 1);
    SPMV_LAUNCH("k_pr_init", s, (k_pr_init<<<blocks_for(n), 256, 0, s>>>(x, n)));
    SPMV_LAUNCH_CHECK("pagerank init");
    for (int it = 0; it < iters; ++it) {
        SPMV_CUDA_TRY(cudaMemsetAsync(flag, 0, 4, s));
        SPMV_LAUNCH("k_pr_prep", s, (k_pr_prep<<<PR_PARTS, PR_BLOCK, 0, s>>>(x, h->pr_inv, n, h->pr_z, h->pr_z2, flag,
                                                                          h->pr_part)));
        SPMV_LAUNCH_CHECK("pagerank prep");
        SPMV_LAUNCH("k_pr_dsum", s, (k_pr_dsum<<<1, PR_PARTS, 0, s>>>(h->pr_part, total)));
        SPMV_LAUNCH_CHECK("pagerank dangling sum");
        if (staged) SPMV_TRY(mul_stage_pattern_split(h, h->pr_z, h->pr_z2, flag, h->pr_y, s));
        else SPMV_TRY(mul_merge_pattern_split(h, h->pr_z, h->pr_z2, flag, h->pr_y, s));
        SPMV_LAUNCH("k_pr_update", s, (k_pr_update<<<blocks_for(n), 256, 0, s>>>(h->pr_y, total, damping, n, x)));
        SPMV_LAUNCH_CHECK("pagerank update");
    }
    return SPMV_OK;
}

}  // namespace

spmv_status pagerank(spmv_matrix *h, double damping, int iters, double *x, cudaStream_t s) {
    SPMV_TRY(pr_buffers(h, s));
    // one graph per (x, iterations, damping, product); re-captured when any of them changes
    if (!h->pr_graph || h->pr_graph_x != x || h->pr_graph_iters != iters || h->pr_graph_damping != damping ||
        h->pr_graph_staged != pr_staged(h)) {
        if (h->pr_graph) {
            cudaGraphExecDestroy((cudaGraphExec_t)h->pr_graph);
            h->pr_graph = nullptr;
        }
        cudaStream_t cs;
        SPMV_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        spmv_status st = SPMV_OK;
        if (e == cudaSuccess) {
            st = pr_enqueue(h, damping, iters, x, cs);
            e = cudaStreamEndCapture(cs, &g);
        }
        cudaGraphExec_t ge = nullptr;
        if (e == cudaSuccess && st == SPMV_OK) e = cudaGraphInstantiate(&ge, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (st != SPMV_OK) return st;
        if (e != cudaSuccess) return cuda_status(e, "pagerank graph capture");
        h->pr_graph = ge;
        h->pr_graph_x = x;
        h->pr_graph_iters = iters;
        h->pr_graph_damping = damping;
        h->pr_graph_staged = pr_staged(h);
    }
    SPMV_CUDA_TRY(cudaGraphLaunch((cudaGraphExec_t)h->pr_graph, s));
    return SPMV_OK;
}

void pagerank_forget(spmv_matrix *h) {
    if (!h->pr_graph) return;
    cudaGraphExecDestroy((cudaGraphExec_t)h->pr_graph);
    h->pr_graph = nullptr;
}

}  // namespace spmv
