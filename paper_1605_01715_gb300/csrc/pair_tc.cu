// Host side of the tcgen05 translation GEMM (see pair_tc.cuh): scaling and FP16
// hi/lo splitting of the operator tables, their TMA tensor maps, the per-box scaling and
// splitting of the input vectors, and the launcher.
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "pair_tc.cuh"

namespace kifmm {

namespace {

// max |x| of a non-negative-compared float array (bit pattern of |x| orders like the value)
__global__ void k_absmax(const float* __restrict__ x, size_t n, unsigned int* __restrict__ out) {
    __shared__ unsigned int red[256];
    unsigned int m = 0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fabsf(x[i])));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(out, red[0]);
}

// hi = nearest FP16 of x * scale, lo = nearest FP16 of the remainder.
__global__ void k_split_table(const float* __restrict__ x, __half* __restrict__ hi, __half* __restrict__ lo,
                              size_t n, float scale) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float v = x[i] * scale;
    __half h = __float2half_rn(v);
    hi[i] = h;
    lo[i] = __float2half_rn(v - __half2float(h));
}

// Box b of [b0, b1), one warp per box: e[b] = kScaleTop - floor(log2 max_k |v[b][k]|),
// the power of two bringing its vector into [2^14, 2^15) (0 for an all-zero vector), and
// hi[b][k] + lo[b][k] = v[b][k] * 2^e[b] as two nearest FP16 values; columns past Q zero.
constexpr int kSplitWarps = 8;
__global__ void __launch_bounds__(32 * kSplitWarps) k_box_split(const float* __restrict__ v, int Q, int Qp, int b0,
                                                                int b1, __half* __restrict__ hi,
                                                                __half* __restrict__ lo, int* __restrict__ e) {
    const int lane = threadIdx.x & 31;
    const int b = b0 + (int)blockIdx.x * kSplitWarps + (int)(threadIdx.x >> 5);
    if (b >= b1) return;                      // whole warp; no block-wide barrier below
    const float* vb = v + (size_t)b * Qp;
    float m = 0.f;
    for (int k = lane; k < Q; k += 32) m = fmaxf(m, fabsf(vb[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    int ex = 0;
    if (m > 0.f) ex = tc::kScaleTop - ilogbf(m);
    ex = max(-100, min(100, ex));
    if (lane == 0) e[b] = ex;
    const float sc = tc::pow2f(ex);
    for (int k = lane; k < Qp; k += 32) {
        const float x = k < Q ? vb[k] * sc : 0.f;
        const __half h = __float2half_rn(x);
        hi[(size_t)b * Qp + k] = h;
        lo[(size_t)b * Qp + k] = __float2half_rn(x - __half2float(h));
    }
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

int get_encoder(EncodeTiled* fn) {
    static std::mutex mu;
    static EncodeTiled cached = nullptr;
    std::lock_guard<std::mutex> g(mu);
    if (!cached) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
            set_error("cuTensorMapEncodeTiled unavailable: %s", cudaGetErrorString(e));
            return KIFMM_ERR_CUDA;
        }
        cached = reinterpret_cast<EncodeTiled>(p);
    }
    *fn = cached;
    return KIFMM_OK;
}

}  // namespace

// Operator rows per work item and pairs per tile for operators of Mr (padded) rows.
int tc_rows(int Mr) { return Mr <= 128 ? 128 : 256; }
int tc_tile_pairs(int Mr) { return Mr <= 128 ? 256 : 128; }

// Scale an FP32 operator table by 2^texp (largest entry into [2^14, 2^15)) and split it
// into FP16 hi and lo tables.  Synchronizes the stream (texp is needed on the host).
int tc_split_table(const float* table, __half* hi, __half* lo, size_t n, int* texp, cudaStream_t s) {
    *texp = 0;
    if (!n) return KIFMM_OK;
    DBuf<unsigned int> mx;
    KF_TRY(mx.alloc(1));
    KF_CHECK_CUDA(cudaMemsetAsync(mx.p, 0, sizeof(unsigned int), s));
    k_absmax<<<1024, 256, 0, s>>>(table, n, mx.p);
    KF_CHECK_LAUNCH();
    unsigned int hm = 0;
    KF_CHECK_CUDA(cudaMemcpyAsync(&hm, mx.p, sizeof(hm), cudaMemcpyDeviceToHost, s));
    KF_CHECK_CUDA(cudaStreamSynchronize(s));
    float m;
    memcpy(&m, &hm, sizeof(m));
    if (m > 0.f) *texp = tc::kScaleTop - std::ilogb(m);
    k_split_table<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(table, hi, lo, n, std::ldexp(1.0f, *texp));
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

// Per-box scales and FP16 hi/lo splits of boxes [b0, b1) of a check-potential buffer.
int tc_box_split(const float* v, int Q, int Qp, int b0, int b1, __half* hi, __half* lo, int* e, cudaStream_t s) {
    if (b1 <= b0) return KIFMM_OK;
    k_box_split<<<(b1 - b0 + kSplitWarps - 1) / kSplitWarps, 32 * kSplitWarps, 0, s>>>(v, Q, Qp, b0, b1, hi, lo, e);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

// 2-D tiled map over rows (op * Mr + row) x columns (Kp) of an FP16 table, box kKS
// columns x tc_rows(Mr) rows, 64-byte swizzle, zero fill outside.
int tc_make_map(CUtensorMap* map, const __half* table, int nops, int Mr, int Kp) {
    EncodeTiled enc;
    KF_TRY(get_encoder(&enc));
    cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)nops * (cuuint64_t)Mr};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * sizeof(__half)};
    cuuint32_t box[2] = {(cuuint32_t)tc::kKS, (cuuint32_t)tc_rows(Mr)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half*>(table), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for a %d x %d table", (int)r, nops * Mr, Kp);
        return KIFMM_ERR_CUDA;
    }
    return KIFMM_OK;
}

template <int SLABS, int N>
static int launch_shape(int which, const CUtensorMap& hi, const CUtensorMap& lo, int texp, int M, int Mr, int Kp,
                        int ostride, const int4* tiles, int ntiles, const int* pin, const int* pout,
                        const int* bexp, const __half* in_hi, const __half* in_lo, float* out, int* err,
                        const int* kcount, cudaStream_t s) {
    using S = tc::Shape<SLABS, N>;
    auto kern = which == 0   ? tc::k_u2u_tc<SLABS, N>
                : which == 1 ? tc::k_m2l_tc<SLABS, N>
                : which == 2 ? tc::k_l2l_tc<SLABS, N>
                             : tc::k_proj_tc<SLABS, N>;
    // set on every launch: the attribute belongs to the current device's context
    KF_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kSmemBytes));
    const int mgroups = (Mr + S::kRows - 1) / S::kRows;
    const int nitems = ntiles * mgroups;
    // persistent: one CTA per SM (one fits by shared memory), each walking its share of
    // the work items
    int dev = 0, nsm = 0;
    KF_CHECK_CUDA(cudaGetDevice(&dev));
    KF_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = nitems < nsm ? nitems : nsm;
    kern<<<grid, tc::kThreads, S::kSmemBytes, s>>>(hi, lo, M, Kp, ostride, Mr, mgroups, nitems, tiles, pin, pout,
                                                    bexp, texp, in_hi, in_lo, out, err, kcount);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

// which: 0 = U2U, 1 = M2L, 2 = L2L, 3 = projection onto a check-space basis.  The
// operators are Mr x Kp (M valid rows); in_hi / in_lo: the split input vectors
// (tc_box_split, Kp per box) of every box a pair reads; out: ostride per box.
int launch_pair_tc(int which, const CUtensorMap& hi, const CUtensorMap& lo, int texp, int M, int Mr, int Kp,
                   int ostride, const int4* tiles, int ntiles, const int* pin, const int* pout, const int* bexp,
                   const __half* in_hi, const __half* in_lo, float* out, int* err, cudaStream_t s,
                   const int* kcount) {
    if (ntiles <= 0) return KIFMM_OK;
    if (Mr <= 128)
        return launch_shape<1, 256>(which, hi, lo, texp, M, Mr, Kp, ostride, tiles, ntiles, pin, pout, bexp, in_hi,
                                    in_lo, out, err, kcount, s);
    return launch_shape<2, 128>(which, hi, lo, texp, M, Mr, Kp, ostride, tiles, ntiles, pin, pout, bexp, in_hi,
                                in_lo, out, err, kcount, s);
}

}  // namespace kifmm
