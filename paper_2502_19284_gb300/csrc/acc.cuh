// Element access and accumulators shared by the product kernels (spmv.cu, stage.cu).
#pragma once
#include "common.cuh"
#include "df64.cuh"

#include <type_traits>

namespace spmv {

// ---------------------------------------------------------------- element access
struct Pattern {};   // value type tag of a pattern matrix (every stored value is 1)

template <typename VT, typename AT>
__device__ __forceinline__ AT ld_val(const VT *__restrict__ v, int64_t k) {
    if constexpr (std::is_same<VT, Pattern>::value) {
        return AT(1);
    } else if constexpr (std::is_same<VT, __nv_bfloat16>::value) {
        return AT(__bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16 *>(v) + k)));
    } else {
        return AT(__ldg(v + k));
    }
}

template <typename XT, typename AT>
__device__ __forceinline__ AT ld_x(const XT *__restrict__ x, int64_t j) {
    return AT(__ldg(x + j));
}

// Value of a stored element held in shared memory (a pattern matrix stores none).
template <typename VT, typename AT>
__device__ __forceinline__ AT sval(const VT *v, int k) {
    if constexpr (std::is_same<VT, Pattern>::value) return AT(1);
    else if constexpr (std::is_same<VT, __nv_bfloat16>::value) return AT(__bfloat162float(v[k]));
    else return AT(v[k]);
}

// Accumulators.  NativeAcc<AT> sums in AT with one fma per nonzero.  DfAcc keeps an FP64
// sum as a float pair (double-float, df64.cuh) so that the FP64 path runs on the FP32
// pipes; its operands arrive already split into (hi, lo) floats.
template <typename AT>
struct NativeAcc {
    using Op = AT;   // operand type of one side of a product
    AT v;
    __device__ __forceinline__ void zero() { v = AT(0); }
    __device__ __forceinline__ void mad(Op a, Op x) { v = fma(a, x, v); }
    __device__ __forceinline__ void add(const NativeAcc &o) { v = v + o.v; }
    __device__ __forceinline__ NativeAcc shfl_up(int o) const { NativeAcc r; r.v = __shfl_up_sync(0xffffffffu, v, o); return r; }
    __device__ __forceinline__ double to_double() const { return (double)v; }
    template <typename XT> __device__ __forceinline__ XT out() const { return XT(v); }
};

struct DfAcc {
    using Op = float2;
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void mad(float2 a, float2 x) { df_fma(a.x, a.y, x.x, x.y, s, c); }
    __device__ __forceinline__ void add(const DfAcc &o) { df_add(s, c, o.s, o.c); }
    __device__ __forceinline__ DfAcc shfl_up(int o) const {
        DfAcc r;
        r.s = __shfl_up_sync(0xffffffffu, s, o);
        r.c = __shfl_up_sync(0xffffffffu, c, o);
        return r;
    }
    __device__ __forceinline__ double to_double() const { return df_to_double(s, c); }
    template <typename XT> __device__ __forceinline__ XT out() const { return XT(df_to_double(s, c)); }
};

// FP32 sum with compensation (SPMV_ACC_COMPENSATED): the rounding error of every product
// (FMA) and of every addition (TwoSum, Knuth) is collected in a second float, as in
// Neumaier's compensated summation; the result carries ~2^-46 relative error in the sum of
// |terms| instead of FP32's L * 2^-24.
struct CompAcc {
    using Op = float;
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void mad(float a, float x) { df_fma(a, 0.f, x, 0.f, s, c); }
    __device__ __forceinline__ void add(const CompAcc &o) { df_add(s, c, o.s, o.c); }
    __device__ __forceinline__ CompAcc shfl_up(int o) const {
        CompAcc r;
        r.s = __shfl_up_sync(0xffffffffu, s, o);
        r.c = __shfl_up_sync(0xffffffffu, c, o);
        return r;
    }
    __device__ __forceinline__ double to_double() const { return df_to_double(s, c); }
    template <typename XT> __device__ __forceinline__ XT out() const { return XT(__fadd_rn(s, c)); }
};

// FP32 products and sums inside a lane (at most MERGE_WARP_IPT terms), compensated only in
// the segmented reduction that joins lanes and tiles (SPMV_ACC_SEGMENT): a row contained in
// one lane costs plain FP32; a longer row's lane partials are combined with TwoSum, so its
// error stays at the short in-lane sums' ~7u instead of growing with the row length.
struct SegAcc : CompAcc {
    __device__ __forceinline__ void mad(float a, float x) { s = __fmaf_rn(a, x, s); }
    __device__ __forceinline__ SegAcc shfl_up(int o) const {
        SegAcc r;
        r.s = __shfl_up_sync(0xffffffffu, s, o);
        r.c = __shfl_up_sync(0xffffffffu, c, o);
        return r;
    }
    __device__ __forceinline__ void add(const SegAcc &o) { df_add(s, c, o.s, o.c); }
};


}  // namespace spmv
