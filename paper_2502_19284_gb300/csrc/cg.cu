// Conjugate gradients on one resident matrix: repeated y = A x (the use that amortises a
// conversion over many products, Sections 6.2 and 7) for a symmetric positive definite A.
//
// Hestenes-Stiefel iteration in FP64, x0 = 0: r = b, p = r, rho = r.r; per iteration
//   q = A p (the handle's active product), alpha = rho / (p.q), x += alpha p, r -= alpha q,
//   rho' = r.r, stop when sqrt(rho') <= tol ||b||, p = r + (rho'/rho) p.
// The dot products are deterministic (fixed per-CTA partial sums reduced in a fixed order by
// one CTA); alpha and beta stay on the device and the vector updates read them there, so an
// iteration costs no host round trip; the residual is read back every CG_CHECK iterations.
#include "common.cuh"
#include "convert.cuh"

#include <cmath>

namespace spmv {
namespace {

constexpr int CG_BLOCK = 256;
constexpr int CG_PARTS = 1024;   // CTAs of a dot product (partials reduced by one CTA)
constexpr int CG_CHECK = 8;      // iterations between residual read-backs

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[CG_BLOCK / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < CG_BLOCK / 32; ++w) s += sh[w];
    __syncthreads();
    return s;   // valid in thread 0
}

// partial[b] = sum over the grid-strided elements of CTA b of a_i * c_i
__global__ void k_dot_part(const double *__restrict__ a, const double *__restrict__ c, int64_t n,
                           double *__restrict__ partial) {
    double v = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * CG_BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * CG_BLOCK)
        v += a[i] * c[i];
    v = block_sum(v);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

// The partials summed in a fixed order; mode 0: out[0] = sum (rho);
// mode 1: alpha = rho / sum -> out[1]; mode 2: rho' = sum, beta = rho' / rho -> out[2], rho = rho'.
// Scalars: s[0] rho, s[1] alpha, s[2] beta.
__global__ void k_dot_final(const double *__restrict__ partial, int parts, int mode, double *__restrict__ s) {
    double v = 0.0;
    for (int i = threadIdx.x; i < parts; i += CG_BLOCK) v += partial[i];
    v = block_sum(v);
    if (threadIdx.x != 0) return;
    if (mode == 0) {
        s[0] = v;
    } else if (mode == 1) {
        s[1] = v != 0.0 ? s[0] / v : 0.0;
    } else {
        s[2] = s[0] != 0.0 ? v / s[0] : 0.0;
        s[0] = v;
    }
}

// x += alpha p; r -= alpha q
__global__ void k_cg_update(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                            const double *__restrict__ q, int64_t n, const double *__restrict__ s) {
    const double alpha = s[1];
    for (int64_t i = (int64_t)blockIdx.x * CG_BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * CG_BLOCK) {
        x[i] += alpha * p[i];
        r[i] -= alpha * q[i];
    }
}

// p = r + beta p
__global__ void k_cg_dir(double *__restrict__ p, const double *__restrict__ r, int64_t n, const double *__restrict__ s) {
    const double beta = s[2];
    for (int64_t i = (int64_t)blockIdx.x * CG_BLOCK + threadIdx.x; i < n; i += (int64_t)gridDim.x * CG_BLOCK)
        p[i] = r[i] + beta * p[i];
}

unsigned grid(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>(CG_PARTS, (n + CG_BLOCK - 1) / CG_BLOCK)); }

spmv_status dot(const double *a, const double *c, int64_t n, double *partial, int mode, double *s, cudaStream_t st) {
    const unsigned g = grid(n);
    SPMV_LAUNCH("k_dot_part", st, (k_dot_part<<<g, CG_BLOCK, 0, st>>>(a, c, n, partial)));
    SPMV_LAUNCH("k_dot_final", st, (k_dot_final<<<1, CG_BLOCK, 0, st>>>(partial, (int)g, mode, s)));
    SPMV_LAUNCH_CHECK("cg dot");
    return SPMV_OK;
}

}  // namespace
}  // namespace spmv

using namespace spmv;

extern "C" spmv_status spmv_cg(spmv_handle h, const double *b, double *x, double tol, int max_iters, void *stream,
                               int *iters_out, double *resid_out) {
    if (!h || !b || !x || max_iters < 0 || !(tol >= 0.0)) {
        set_error("spmv_cg: NULL handle or vector, max_iters < 0 or tol < 0");
        return SPMV_ERR_INVALID_ARG;
    }
    if (h->format < 0) {
        set_error("spmv_cg: call spmv_convert first");
        return SPMV_ERR_NOT_CONVERTED;
    }
    if (h->m != h->n) {
        set_error("spmv_cg: the matrix must be square (and symmetric positive definite)");
        return SPMV_ERR_INVALID_ARG;
    }
    if (h->dt == SPMV_BF16) {
        set_error("spmv_cg: FP64 vectors need FP64, FP32 or pattern values");
        return SPMV_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = h->n;
    DevBuf r(s), p(s), q(s), part(s), sc(s);
    SPMV_TRY(r.alloc((size_t)std::max<int64_t>(n, 1) * 8, "cg r"));
    SPMV_TRY(p.alloc((size_t)std::max<int64_t>(n, 1) * 8, "cg p"));
    SPMV_TRY(q.alloc((size_t)std::max<int64_t>(n, 1) * 8, "cg q"));
    SPMV_TRY(part.alloc(CG_PARTS * 8, "cg partials"));
    SPMV_TRY(sc.alloc(4 * 8, "cg scalars"));
    double *R = r.as<double>(), *P = p.as<double>(), *Q = q.as<double>(), *S = sc.as<double>();
    double *pt = part.as<double>();
    SPMV_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)n * 8, s));
    SPMV_CUDA_TRY(cudaMemcpyAsync(R, b, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    SPMV_CUDA_TRY(cudaMemcpyAsync(P, b, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
    SPMV_TRY(dot(R, R, n, pt, 0, S, s));
    double rho = 0.0;
    SPMV_CUDA_TRY(cudaMemcpyAsync(&rho, S, 8, cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    const double bnorm = std::sqrt(rho), stop = tol * bnorm;
    int it = 0;
    double res = bnorm;
    const unsigned g = grid(n);
    while (it < max_iters && res > stop) {
        SPMV_TRY(spmv_mul(h, P, Q, SPMV_F64, SPMV_ACC_DEFAULT, s));
        SPMV_TRY(dot(P, Q, n, pt, 1, S, s));
        SPMV_LAUNCH("k_cg_update", s, (k_cg_update<<<g, CG_BLOCK, 0, s>>>(x, R, P, Q, n, S)));
        SPMV_TRY(dot(R, R, n, pt, 2, S, s));
        SPMV_LAUNCH("k_cg_dir", s, (k_cg_dir<<<g, CG_BLOCK, 0, s>>>(P, R, n, S)));
        SPMV_LAUNCH_CHECK("cg update");
        ++it;
        if (it % CG_CHECK == 0 || it == max_iters) {
            SPMV_CUDA_TRY(cudaMemcpyAsync(&rho, S, 8, cudaMemcpyDeviceToHost, s));
            SPMV_CUDA_TRY(cudaStreamSynchronize(s));
            res = std::sqrt(std::fabs(rho));
            if (!std::isfinite(res)) break;
        }
    }
    SPMV_CUDA_TRY(cudaMemcpyAsync(&rho, S, 8, cudaMemcpyDeviceToHost, s));
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    if (iters_out) *iters_out = it;
    if (resid_out) *resid_out = std::sqrt(std::fabs(rho));
    return SPMV_OK;
}
