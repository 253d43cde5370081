// Batched multi-RHS products Y_i = A_i X_i (spmv_mul_batch) in one persistent launch.
//
// Every matrix of the batch keeps its own merge-path warp tiles (the CSR_MERGE partition and
// lane descriptors built at conversion).  The batch plan concatenates them into one global
// tile space: a prefix of tile counts and a device table of per-matrix pointers.  A
// persistent warp takes global tiles w, w + W, ..., finds the matrix by bisection over the
// prefix, brings the tile's descriptors, column indices and values into shared memory with
// a 1-D TMA bulk copy, and then, for each block of KB right-hand sides, gathers KB
// consecutive values of the row-major X per nonzero (one vector load), walks its path items
// exactly as the single-vector product does, and writes finished rows of Y.  Carries and the
// partials of rows begun in earlier tiles are kept per (tile, right-hand side); one fix-up
// kernel over the global tile space completes them.  The plan (tables, scratch, and the
// CUDA graph of the two launches) is built once per batch shape and replayed; only the X/Y
// pointer table is refreshed per call.
#include "common.cuh"
#include "convert.cuh"
#include "df64.cuh"

#include <map>
#include <mutex>
#include <vector>

namespace spmv {

namespace {

constexpr int BW = 4;                 // warps per CTA
constexpr int BIPT = MERGE_WARP_IPT;  // path items per lane
constexpr int BITEMS = MERGE_WARP_ITEMS;
constexpr long long B_SPIN_LIMIT = 1ll << 22;

struct MatEntry {   // device table, one per matrix
    const uint32_t *desc;
    const int32_t *col;
    const void *val;
    const int32_t *part_row, *part_nz;
    const void *x;
    void *y;
    double *carry;    // tiles * k carries, then tiles * k head partials
    int32_t *carry_row;
    const int32_t *fix_len, *fix_long;   // static carry runs of the handle (see build_fix_runs)
    uint32_t *err;    // the handle's status word for a timed-out wait
    int64_t m, tiles;
};

__device__ __forceinline__ uint32_t smem_u32b(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

struct FAcc {   // FP32 accumulation
    float v;
    __device__ __forceinline__ void zero() { v = 0.f; }
    __device__ __forceinline__ void mad(float a, float x) { v = fmaf(a, x, v); }
    __device__ __forceinline__ void add(const FAcc &o) { v = v + o.v; }
    __device__ __forceinline__ FAcc shfl_up(int o) const { FAcc r; r.v = __shfl_up_sync(0xffffffffu, v, o); return r; }
    __device__ __forceinline__ double dbl() const { return (double)v; }
    template <typename XT> __device__ __forceinline__ XT out() const { return XT(v); }
};
struct CAcc {   // compensated FP32 (see SPMV_ACC_COMPENSATED)
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void mad(float a, float x) { df_fma(a, 0.f, x, 0.f, s, c); }
    __device__ __forceinline__ void add(const CAcc &o) { df_add(s, c, o.s, o.c); }
    __device__ __forceinline__ CAcc shfl_up(int o) const {
        CAcc r;
        r.s = __shfl_up_sync(0xffffffffu, s, o);
        r.c = __shfl_up_sync(0xffffffffu, c, o);
        return r;
    }
    __device__ __forceinline__ double dbl() const { return df_to_double(s, c); }
    template <typename XT> __device__ __forceinline__ XT out() const { return XT(__fadd_rn(s, c)); }
};
struct SAcc {   // FP32 inside a lane, compensated across lanes and tiles (SPMV_ACC_SEGMENT)
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void mad(float a, float x) { s = __fmaf_rn(a, x, s); }
    __device__ __forceinline__ void add(const SAcc &o) { df_add(s, c, o.s, o.c); }
    __device__ __forceinline__ SAcc shfl_up(int o) const {
        SAcc r;
        r.s = __shfl_up_sync(0xffffffffu, s, o);
        r.c = __shfl_up_sync(0xffffffffu, c, o);
        return r;
    }
    __device__ __forceinline__ double dbl() const { return df_to_double(s, c); }
    template <typename XT> __device__ __forceinline__ XT out() const { return XT(__fadd_rn(s, c)); }
};
struct DAcc {   // native FP64
    double v;
    __device__ __forceinline__ void zero() { v = 0.0; }
    __device__ __forceinline__ void mad(double a, double x) { v = fma(a, x, v); }
    __device__ __forceinline__ void add(const DAcc &o) { v = v + o.v; }
    __device__ __forceinline__ DAcc shfl_up(int o) const { DAcc r; r.v = __shfl_up_sync(0xffffffffu, v, o); return r; }
    __device__ __forceinline__ double dbl() const { return v; }
    template <typename XT> __device__ __forceinline__ XT out() const { return XT(v); }
};

struct PatternB {};

template <typename VT, typename T>
__device__ __forceinline__ T bval(const VT *v, int k) {
    if constexpr (std::is_same<VT, PatternB>::value) return T(1);
    else if constexpr (std::is_same<VT, __nv_bfloat16>::value) return T(__bfloat162float(v[k]));
    else return T(v[k]);
}

template <typename VT, typename Acc, int KB>
struct BSlot {
    static constexpr int VAL = BITEMS + 16;
    static constexpr int VAL_BYTES = std::is_same<VT, PatternB>::value ? 0 : ((VAL * (int)sizeof(VT) + 15) / 16) * 16;
    static constexpr int OFF_DESC = 16, OFF_COL = OFF_DESC + 128, OFF_VAL = OFF_COL + (BITEMS + 8) * 4,
                         OFF_ROWS = OFF_VAL + VAL_BYTES;
    static constexpr int BYTES = OFF_ROWS + ((BITEMS * KB * (int)sizeof(Acc) + 15) / 16) * 16;
};

__device__ __forceinline__ void widen16b(int64_t e0, int64_t e1, int es, int64_t *first, uint32_t *bytes) {
    const int64_t per = 16 / es;
    const int64_t a0 = e0 & ~(per - 1), a1 = (e1 + per - 1) & ~(per - 1);
    *first = a0;
    *bytes = e1 > e0 ? (uint32_t)((a1 - a0) * es) : 0u;
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(smem_u32b(dst)), "l"(src), "r"(bytes), "r"(smem_u32b(bar)) : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done = 0;
    for (long long it = 0; it < B_SPIN_LIMIT && !done; ++it)
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done) : "r"(smem_u32b(bar)), "r"(parity) : "memory");
    return __all_sync(0xffffffffu, done);
}

// KB consecutive values of X row `c` starting at right-hand side r0, as T.
template <typename XT, typename T, int KB>
__device__ __forceinline__ void gather_x(const XT *X, int64_t c, int k, int r0, T *out) {
    const XT *p = X + c * k + r0;
    if constexpr (KB == 4 && std::is_same<XT, float>::value) {
        const float4 v = __ldg((const float4 *)p);
        out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
    } else if constexpr (KB == 4 && std::is_same<XT, double>::value) {
        const double2 a = __ldg((const double2 *)p), b = __ldg((const double2 *)p + 1);
        out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
    } else {
#pragma unroll
        for (int q = 0; q < KB; ++q) out[q] = T(__ldg(p + q));
    }
}

template <typename VT, typename XT, typename T, typename Acc, int KB>
__global__ __launch_bounds__(BW * 32) void k_batch(const MatEntry *__restrict__ mats, const int64_t *__restrict__ prefix,
                                                   int count, int64_t total_tiles, int k) {
    using Slot = BSlot<VT, Acc, KB>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    unsigned char *slot = smem_raw + (threadIdx.x >> 5) * Slot::BYTES;
    uint64_t *bar = (uint64_t *)slot;
    const uint32_t *s_desc = (const uint32_t *)(slot + Slot::OFF_DESC);
    const int32_t *s_col = (const int32_t *)(slot + Slot::OFF_COL);
    const VT *s_val = (const VT *)(slot + Slot::OFF_VAL);
    Acc *s_rows = (Acc *)(slot + Slot::OFF_ROWS);
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32b(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const int64_t W = (int64_t)gridDim.x * BW;
    uint32_t phase = 0;
    for (int64_t g = (int64_t)blockIdx.x * BW + (threadIdx.x >> 5); g < total_tiles; g += W, phase ^= 1u) {
        int lo = 0, hi = count - 1;   // matrix of global tile g: largest i with prefix[i] <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= g) lo = mid;
            else hi = mid - 1;
        }
        const MatEntry me = mats[lo];
        const int64_t t = g - prefix[lo];
        const int64_t i0 = me.part_row[t], j0 = me.part_nz[t];
        const int nrows = (int)(me.part_row[t + 1] - i0), nnzt = (int)(me.part_nz[t + 1] - j0);
        if (lane == 0) {
            int64_t cf, vf = j0;
            uint32_t cb, vb = 0;
            widen16b(j0, j0 + nnzt, 4, &cf, &cb);
            if constexpr (Slot::VAL_BYTES > 0) widen16b(j0, j0 + nnzt, (int)sizeof(VT), &vf, &vb);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32b(bar)),
                         "r"(128u + cb + vb) : "memory");
            bulk_load(slot + Slot::OFF_DESC, me.desc + t * 32, 128u, bar);
            if (cb) bulk_load(slot + Slot::OFF_COL, me.col + cf, cb, bar);
            if constexpr (Slot::VAL_BYTES > 0)
                if (vb) bulk_load(slot + Slot::OFF_VAL, (const VT *)me.val + vf, vb, bar);
        }
        if (!bar_wait(bar, phase)) {
            if (lane == 0) atomicOr(me.err, ST_TIMEOUT);
            return;
        }
        const uint32_t d = s_desc[lane];
        const int col_off = (int)(j0 & 3);
        const int perv = 16 / (int)(Slot::VAL_BYTES > 0 ? sizeof(VT) : 16);
        const int val_off = (int)(j0 & (perv - 1));
        const int istart = (int)(d & 0xFFu), jb = (int)((d >> 8) & 0xFFu), items = (int)((d >> 24) & 0x7Fu);
        const uint32_t bits = (d >> 16) & 0x7Fu;
        const int iend = istart + __popc(bits);
        const bool cont = (__shfl_sync(0xffffffffu, d, 0) >> 31) != 0u;
        T a[BIPT];
        int cidx[BIPT];
#pragma unroll
        for (int q = 0; q < BIPT; ++q)
            if (q < items && !((bits >> q) & 1u)) {
                const int jn = jb + q - __popc(bits & ((1u << q) - 1u));
                a[q] = bval<VT, T>(s_val, val_off + jn);
                cidx[q] = s_col[col_off + jn];
            }
        const XT *X = (const XT *)me.x;
        XT *Y = (XT *)me.y;
        for (int r0 = 0; r0 < k; r0 += KB) {
            T xv[BIPT][KB];
#pragma unroll
            for (int q = 0; q < BIPT; ++q)
                if (q < items && !((bits >> q) & 1u)) gather_x<XT, T, KB>(X, cidx[q], k, r0, xv[q]);
            Acc acc[KB];
#pragma unroll
            for (int b = 0; b < KB; ++b) acc[b].zero();
            int i = istart;
#pragma unroll
            for (int q = 0; q < BIPT; ++q) {
                if (q < items) {
                    if ((bits >> q) & 1u) {
#pragma unroll
                        for (int b = 0; b < KB; ++b) {
                            s_rows[i * KB + b] = acc[b];
                            acc[b].zero();
                        }
                        ++i;
                    } else {
#pragma unroll
                        for (int b = 0; b < KB; ++b) acc[b].mad(a[q], xv[q][b]);
                    }
                }
            }
            const int prev_end = __shfl_up_sync(0xffffffffu, iend, 1);
            const bool head = lane == 0 || prev_end != iend;
            const bool all_heads = __all_sync(0xffffffffu, head);
#pragma unroll
            for (int b = 0; b < KB; ++b) {
                Acc sv = acc[b];
                bool f = head;
                if (!all_heads) {
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        if (__all_sync(0xffffffffu, f)) break;   // every lane has reached its segment head
                        Acc ov = sv.shfl_up(o);
                        const bool of = __shfl_up_sync(0xffffffffu, f, o);
                        if (lane >= o) {
                            if (!f) {
                                ov.add(sv);
                                sv = ov;
                            }
                            f = f || of;
                        }
                    }
                }
                const Acc cin = sv.shfl_up(1);
                __syncwarp();
                if (lane > 0 && istart < iend) {
                    Acc v = cin;
                    v.add(s_rows[istart * KB + b]);
                    s_rows[istart * KB + b] = v;
                }
                if (lane == 31) {
                    me.carry[t * k + r0 + b] = sv.dbl();
                    if (r0 + b == 0) me.carry_row[t] = (int32_t)(i0 + nrows);
                }
            }
            __syncwarp();
            if (cont && lane == 0 && nrows > 0)
                for (int b = 0; b < KB; ++b) me.carry[(me.tiles + t) * k + r0 + b] = s_rows[b].dbl();
            for (int e = (cont ? KB : 0) + lane; e < nrows * KB; e += 32) {
                const int r = e / KB, b = e % KB;
                Y[(i0 + r) * k + r0 + b] = s_rows[e].template out<XT>();
            }
            __syncwarp();
        }
        __syncwarp();
    }
}

// Carry fix-up over the global tile space, as the single-vector product's (same run
// structure, same summation order, so each column equals spmv_mul's result bitwise): one
// thread per (tile, right-hand side) sums a short run in tile order; one warp per (long run,
// right-hand side) sums a long one with lane-strided partials and a fixed shuffle tree.
template <typename XT>
__device__ __forceinline__ void batch_finish(const MatEntry &me, int64_t u, int32_t row, int k, int r, double sum) {
    if (row >= me.m || u >= me.tiles) return;
    XT *Y = (XT *)me.y;
    if (me.desc[u * 32] >> 31) Y[(int64_t)row * k + r] = XT(sum + me.carry[(me.tiles + u) * k + r]);
    else if (sum != 0.0) Y[(int64_t)row * k + r] = XT((double)Y[(int64_t)row * k + r] + sum);
}

__device__ __forceinline__ int find_entry(const int64_t *__restrict__ prefix, int count, int64_t g) {
    int lo = 0, hi = count - 1;   // largest i with prefix[i] <= g
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename XT>
__global__ void k_batch_fixup(const MatEntry *__restrict__ mats, const int64_t *__restrict__ prefix, int count,
                              int64_t total_tiles, int k) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= total_tiles * k) return;
    const int64_t g = gid / k;
    const int r = (int)(gid % k);
    const int i = find_entry(prefix, count, g);
    const MatEntry &me = mats[i];
    const int64_t t = g - prefix[i];
    const int len = me.fix_len[t];
    if (len == 0 || len > FIX_SHORT) return;
    double s = me.carry[t * k + r];
    for (int q = 1; q < len; ++q) s = s + me.carry[(t + q) * k + r];
    batch_finish<XT>(me, t + len, me.carry_row[t], k, r, s);
}

template <typename XT>
__global__ void k_batch_fixup_long(const MatEntry *__restrict__ mats, const int64_t *__restrict__ lprefix, int count,
                                   int64_t total_long, int k) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= total_long * k) return;
    const int64_t g = w / k;
    const int r = (int)(w % k);
    const int i = find_entry(lprefix, count, g);
    const MatEntry &me = mats[i];
    const int64_t t0 = me.fix_long[g - lprefix[i]];
    const int len = me.fix_len[t0];
    double s = 0.0;
    for (int q = lane; q < len; q += 32) s = s + me.carry[(t0 + q) * k + r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = s + __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) batch_finish<XT>(me, t0 + len, me.carry_row[t0], k, r, s);
}

// ---------------------------------------------------------------- plans
struct Plan {
    std::vector<spmv_matrix *> hs;
    int k = 0, vdt = 0, dt = 0;
    uint32_t acc = 0;
    bool vec4 = false;
    MatEntry *d_mats = nullptr;
    int64_t *d_prefix = nullptr;
    int64_t *d_lprefix = nullptr;   // prefix of the matrices' long carry runs
    int64_t total_long = 0;
    double *d_carry = nullptr;
    int32_t *d_crow = nullptr;
    std::vector<MatEntry> h_mats;
    int64_t total_tiles = 0;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t graph_stream = nullptr;
};

std::mutex g_plan_mu;
std::vector<Plan *> g_plans;

void free_plan(Plan *p) {
    if (p->graph) cudaGraphExecDestroy(p->graph);
    dev_free(p->d_mats);
    dev_free(p->d_prefix);
    dev_free(p->d_lprefix);
    dev_free(p->d_carry);
    dev_free(p->d_crow);
    delete p;
}

template <typename VT, typename XT, typename T, typename Acc, int KB>
spmv_status enqueue_batch(Plan *p, cudaStream_t s) {
    using Slot = BSlot<VT, Acc, KB>;
    const size_t smem = (size_t)BW * Slot::BYTES;
    static DeviceOnce attr;
    SPMV_TRY(attr([&] { return set_smem_ctas((const void *)k_batch<VT, XT, T, Acc, KB>, smem, 5); }));
    int dev = 0, sms = 1, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<VT, XT, T, Acc, KB>, BW * 32, smem) !=
            cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int64_t want = (p->total_tiles + BW - 1) / BW;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * per_sm));
    SPMV_LAUNCH("k_batch", s, (k_batch<VT, XT, T, Acc, KB><<<grid, BW * 32, smem, s>>>(
                                  p->d_mats, p->d_prefix, (int)p->hs.size(), p->total_tiles, p->k)));
    SPMV_LAUNCH_CHECK("batch");
    const int64_t nfix = p->total_tiles * p->k;
    SPMV_LAUNCH("k_batch_fixup", s, (k_batch_fixup<XT><<<(unsigned)((nfix + 255) / 256), 256, 0, s>>>(
                                        p->d_mats, p->d_prefix, (int)p->hs.size(), p->total_tiles, p->k)));
    SPMV_LAUNCH_CHECK("batch fixup");
    if (p->total_long > 0) {
        const int64_t threads = p->total_long * p->k * 32;
        SPMV_LAUNCH("k_batch_fixup_long", s, (k_batch_fixup_long<XT><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
                                                 p->d_mats, p->d_lprefix, (int)p->hs.size(), p->total_long, p->k)));
        SPMV_LAUNCH_CHECK("batch fixup long");
    }
    return SPMV_OK;
}

template <typename VT, typename XT, typename T, typename Acc>
spmv_status enqueue_kb(Plan *p, bool vec4, cudaStream_t s) {
    if (vec4) return enqueue_batch<VT, XT, T, Acc, 4>(p, s);
    return enqueue_batch<VT, XT, T, Acc, 1>(p, s);
}

// The combinations of spmv_mul's merge path: F64 vectors accumulate in FP64; F32 vectors in
// FP32, compensated FP32, or (F32/BF16 matrices) FP64.
spmv_status enqueue_plan(Plan *p, cudaStream_t s) {
    const int dt = p->dt;
    const bool v4 = p->vec4;
    if (p->vdt == SPMV_F64 && p->acc == SPMV_ACC_F64) {
        if (dt == SPMV_F64) return enqueue_kb<double, double, double, DAcc>(p, v4, s);
        if (dt == SPMV_PATTERN) return enqueue_kb<PatternB, double, double, DAcc>(p, v4, s);
        if (dt == SPMV_F32) return enqueue_kb<float, double, double, DAcc>(p, v4, s);
    } else if (p->vdt == SPMV_F32 && p->acc == SPMV_ACC_F32) {
        if (dt == SPMV_F32) return enqueue_kb<float, float, float, FAcc>(p, v4, s);
        if (dt == SPMV_BF16) return enqueue_kb<__nv_bfloat16, float, float, FAcc>(p, v4, s);
        if (dt == SPMV_PATTERN) return enqueue_kb<PatternB, float, float, FAcc>(p, v4, s);
    } else if (p->vdt == SPMV_F32 && p->acc == SPMV_ACC_COMPENSATED) {
        if (dt == SPMV_F32) return enqueue_kb<float, float, float, CAcc>(p, v4, s);
        if (dt == SPMV_BF16) return enqueue_kb<__nv_bfloat16, float, float, CAcc>(p, v4, s);
        if (dt == SPMV_PATTERN) return enqueue_kb<PatternB, float, float, CAcc>(p, v4, s);
    } else if (p->vdt == SPMV_F32 && p->acc == SPMV_ACC_SEGMENT) {
        if (dt == SPMV_F32) return enqueue_kb<float, float, float, SAcc>(p, v4, s);
        if (dt == SPMV_BF16) return enqueue_kb<__nv_bfloat16, float, float, SAcc>(p, v4, s);
        if (dt == SPMV_PATTERN) return enqueue_kb<PatternB, float, float, SAcc>(p, v4, s);
    } else if (p->vdt == SPMV_F32 && p->acc == SPMV_ACC_F64) {
        if (dt == SPMV_F32) return enqueue_kb<float, float, double, DAcc>(p, v4, s);
        if (dt == SPMV_BF16) return enqueue_kb<__nv_bfloat16, float, double, DAcc>(p, v4, s);
    }
    set_error("spmv_mul_batch: unsupported combination of matrix dtype, vector dtype and accumulation");
    return SPMV_ERR_UNSUPPORTED;
}

}  // namespace

// ---------------------------------------------------------------- direct batches
// A batch launched without capture, on caller-owned scratch (one per concurrent stream): the
// serving loop groups whatever requests are admitted together, so shapes rarely repeat.
struct BatchSlot {
    Plan plan;
    int64_t cap_mats = 0, cap_tiles = 0, cap_carry = 0;   // device capacities (entries)
};

BatchSlot *batch_slot_new() { return new BatchSlot(); }

void batch_slot_free(BatchSlot *b) {
    if (!b) return;
    dev_free(b->plan.d_mats);
    dev_free(b->plan.d_prefix);
    dev_free(b->plan.d_lprefix);
    dev_free(b->plan.d_carry);
    dev_free(b->plan.d_crow);
    b->plan.d_mats = nullptr;
    delete b;
}

int64_t batch_scratch_bytes(int count, spmv_matrix *const *hs, int k) {
    int64_t tiles = 0;
    for (int i = 0; i < count; ++i) tiles += hs[i]->tiles;
    return (int64_t)count * (int64_t)sizeof(MatEntry) + (count + 1) * 8 + tiles * (16 * k + 4);
}

spmv_status batch_direct(BatchSlot *b, int count, spmv_matrix *const *hs, int k, const void *const *X,
                         void *const *Y, spmv_dtype vdt, uint32_t acc, cudaStream_t s) {
    if (count == 0) return SPMV_OK;
    const int dt = hs[0]->dt;
    for (int i = 0; i < count; ++i)
        if (!hs[i]->has_merge || hs[i]->dt != dt) {
            set_error("batch: every matrix needs merge tiles and one dtype");
            return SPMV_ERR_UNSUPPORTED;
        }
    if (acc == SPMV_ACC_DEFAULT)
        acc = (dt == SPMV_F64 || (dt == SPMV_PATTERN && vdt == SPMV_F64)) ? SPMV_ACC_F64 : SPMV_ACC_F32;
    const int es = vdt == SPMV_F64 ? 8 : 4;
    bool vec4 = (k % 4) == 0;
    for (int i = 0; i < count && vec4; ++i)
        vec4 = ((uintptr_t)X[i] % (size_t)(4 * es)) == 0 && ((uintptr_t)Y[i] % (size_t)es) == 0;
    Plan *p = &b->plan;
    p->hs.assign(hs, hs + count);
    p->k = k;
    p->vdt = vdt;
    p->acc = acc;
    p->dt = dt;
    p->vec4 = vec4;
    std::vector<int64_t> prefix(count + 1, 0), lprefix(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        prefix[i + 1] = prefix[i] + hs[i]->tiles;
        lprefix[i + 1] = lprefix[i] + hs[i]->fix_long_count;
    }
    p->total_tiles = prefix[count];
    p->total_long = lprefix[count];
    if (p->total_tiles == 0) return SPMV_OK;
    auto grow = [&](void **ptr, int64_t &cap, int64_t need, size_t unit, const char *what) -> spmv_status {
        if (need <= cap) return SPMV_OK;
        if (*ptr) dev_free_async(*ptr, s);
        *ptr = nullptr;
        cap = 0;
        SPMV_TRY(dev_alloc(ptr, (size_t)need * unit, what, s));
        cap = need;
        return SPMV_OK;
    };
    int64_t cap_prefix = b->cap_mats ? b->cap_mats + 1 : 0, cap_lprefix = cap_prefix;
    SPMV_TRY(grow((void **)&p->d_mats, b->cap_mats, count, sizeof(MatEntry), "batch table"));
    SPMV_TRY(grow((void **)&p->d_prefix, cap_prefix, count + 1, 8, "batch prefix"));
    SPMV_TRY(grow((void **)&p->d_lprefix, cap_lprefix, count + 1, 8, "batch long-run prefix"));
    SPMV_TRY(grow((void **)&p->d_carry, b->cap_carry, 2 * p->total_tiles * k, 8, "batch carries"));
    SPMV_TRY(grow((void **)&p->d_crow, b->cap_tiles, p->total_tiles, 4, "batch carry rows"));
    p->h_mats.resize(count);
    for (int i = 0; i < count; ++i) {
        MatEntry &e = p->h_mats[i];
        spmv_matrix *h = hs[i];
        e.desc = h->merge_desc;
        e.col = h->col;
        e.val = h->val;
        e.part_row = h->part_row;
        e.part_nz = h->part_nz;
        e.x = X[i];
        e.y = Y[i];
        e.carry = p->d_carry + 2 * prefix[i] * k;
        e.carry_row = p->d_crow + prefix[i];
        e.fix_len = h->fix_len;
        e.fix_long = h->fix_long;
        e.err = h->status_dev + 3;
        e.m = h->m;
        e.tiles = h->tiles;
    }
    // pageable sources are staged before the calls return
    SPMV_CUDA_TRY(cudaMemcpyAsync(p->d_prefix, prefix.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
    SPMV_CUDA_TRY(cudaMemcpyAsync(p->d_lprefix, lprefix.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
    SPMV_CUDA_TRY(cudaMemcpyAsync(p->d_mats, p->h_mats.data(), sizeof(MatEntry) * count, cudaMemcpyHostToDevice, s));
    return enqueue_plan(p, s);
}

spmv_status mul_batch(int count, spmv_matrix *const *hs, int k, const void *const *X, void *const *Y,
                      spmv_dtype vdt, uint32_t acc, cudaStream_t s) {
    if (count == 0) return SPMV_OK;
    const int dt = hs[0]->dt;
    for (int i = 0; i < count; ++i) {
        if (!hs[i]->has_merge) {
            set_error("spmv_mul_batch: every handle must be converted to CSR_MERGE (or AUTO) first");
            return SPMV_ERR_NOT_CONVERTED;
        }
        if (hs[i]->dt != dt) {
            set_error("spmv_mul_batch: all matrices of a batch must have the same dtype");
            return SPMV_ERR_UNSUPPORTED;
        }
    }
    if (acc == SPMV_ACC_DEFAULT)
        acc = (dt == SPMV_F64 || (dt == SPMV_PATTERN && vdt == SPMV_F64)) ? SPMV_ACC_F64 : SPMV_ACC_F32;
    const int es = vdt == SPMV_F64 ? 8 : 4;
    bool vec4 = (k % 4) == 0;
    for (int i = 0; i < count && vec4; ++i)
        vec4 = ((uintptr_t)X[i] % (size_t)(4 * es)) == 0 && ((uintptr_t)Y[i] % (size_t)es) == 0;
    std::lock_guard<std::mutex> g(g_plan_mu);
    Plan *plan = nullptr;
    for (Plan *p : g_plans)
        if (p->k == k && p->vdt == vdt && p->acc == acc && p->dt == dt && p->vec4 == vec4 &&
            (int)p->hs.size() == count &&
            std::equal(p->hs.begin(), p->hs.end(), hs))
            plan = p;
    if (!plan) {
        plan = new Plan();
        plan->hs.assign(hs, hs + count);
        plan->k = k;
        plan->vdt = vdt;
        plan->acc = acc;
        plan->dt = dt;
        plan->vec4 = vec4;
        std::vector<int64_t> prefix(count + 1, 0), lprefix(count + 1, 0);
        for (int i = 0; i < count; ++i) {
            prefix[i + 1] = prefix[i] + hs[i]->tiles;
            lprefix[i + 1] = lprefix[i] + hs[i]->fix_long_count;
        }
        plan->total_tiles = prefix[count];
        plan->total_long = lprefix[count];
        auto fail = [&](spmv_status st) { free_plan(plan); return st; };
        spmv_status st;
        if ((st = dev_alloc((void **)&plan->d_mats, sizeof(MatEntry) * count, "batch table", s)) != SPMV_OK ||
            (st = dev_alloc((void **)&plan->d_prefix, sizeof(int64_t) * (count + 1), "batch prefix", s)) != SPMV_OK ||
            (st = dev_alloc((void **)&plan->d_lprefix, sizeof(int64_t) * (count + 1), "batch long-run prefix", s)) !=
                SPMV_OK ||
            (st = dev_alloc((void **)&plan->d_carry, sizeof(double) * 2 * plan->total_tiles * k, "batch carries", s)) !=
                SPMV_OK ||
            (st = dev_alloc((void **)&plan->d_crow, sizeof(int32_t) * plan->total_tiles, "batch carry rows", s)) !=
                SPMV_OK)
            return fail(st);
        plan->h_mats.resize(count);
        for (int i = 0; i < count; ++i) {
            MatEntry &e = plan->h_mats[i];
            spmv_matrix *h = hs[i];
            e.desc = h->merge_desc;
            e.col = h->col;
            e.val = h->val;
            e.part_row = h->part_row;
            e.part_nz = h->part_nz;
            e.carry = plan->d_carry + 2 * prefix[i] * k;
            e.carry_row = plan->d_crow + prefix[i];
            e.fix_len = h->fix_len;
            e.fix_long = h->fix_long;
            e.err = h->status_dev + 3;
            e.m = h->m;
            e.tiles = h->tiles;
        }
        cudaError_t e = cudaMemcpyAsync(plan->d_prefix, prefix.data(), sizeof(int64_t) * (count + 1),
                                        cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(plan->d_lprefix, lprefix.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return fail(cuda_status(e, "batch plan upload"));
        if (plan->total_tiles > 0) {   // capture the two launches once per batch shape
            cudaStream_t cs;
            e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            if (e != cudaSuccess) return fail(cuda_status(e, "batch capture stream"));
            cudaGraph_t gr = nullptr;
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            st = SPMV_OK;
            if (e == cudaSuccess) {
                st = enqueue_plan(plan, cs);
                const cudaError_t e2 = cudaStreamEndCapture(cs, &gr);
                if (e == cudaSuccess) e = e2;
            }
            if (e == cudaSuccess && st == SPMV_OK) e = cudaGraphInstantiate(&plan->graph, gr, 0);
            if (gr) cudaGraphDestroy(gr);
            cudaStreamDestroy(cs);
            if (st != SPMV_OK) return fail(st);
            if (e != cudaSuccess) return fail(cuda_status(e, "batch graph capture"));
        }
        g_plans.push_back(plan);
    }
    if (plan->total_tiles == 0) return SPMV_OK;
    for (int i = 0; i < count; ++i) {
        plan->h_mats[i].x = X[i];
        plan->h_mats[i].y = Y[i];
    }
    // pageable source: the copy is staged before the call returns, so the host table can
    // change for the next call
    SPMV_CUDA_TRY(cudaMemcpyAsync(plan->d_mats, plan->h_mats.data(), sizeof(MatEntry) * count,
                                  cudaMemcpyHostToDevice, s));
    SPMV_CUDA_TRY(cudaGraphLaunch(plan->graph, s));
    return SPMV_OK;
}

void forget_batch_plans(const spmv_matrix *h) {
    std::lock_guard<std::mutex> g(g_plan_mu);
    for (size_t i = 0; i < g_plans.size();) {
        Plan *p = g_plans[i];
        if (std::find(p->hs.begin(), p->hs.end(), h) != p->hs.end()) {
            free_plan(p);
            g_plans.erase(g_plans.begin() + i);
        } else {
            ++i;
        }
    }
}

}  // namespace spmv
