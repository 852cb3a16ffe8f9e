// Host side of the tcgen05 translation GEMM (see pair_tc.cuh): TF32 splitting of the
// operator tables, their TMA tensor maps, and the launcher.
#include <mutex>

#include "common.cuh"
#include "pair_tc.cuh"

namespace kifmm {

namespace {

// hi = nearest TF32 of x (written over x), lo = nearest TF32 of x - hi.
__global__ void k_split_table(float* __restrict__ hi, float* __restrict__ lo, size_t n) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x = hi[i];
    float h = tc::tf32_rna(x);
    hi[i] = h;
    lo[i] = tc::tf32_rna(x - h);
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

// Rows of operator per CTA and pairs per tile for a padded order.
int tc_rows(int Qp) { return Qp <= 128 ? 128 : 256; }
int tc_tile_pairs(int Qp) { return Qp <= 128 ? 256 : 128; }

// Split an operator table (nops x Qp x Qp FP32) into TF32 hi (in place) and lo parts.
int tc_split_table(float* table, float* lo, size_t n, cudaStream_t s) {
    if (!n) return KIFMM_OK;
    k_split_table<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(table, lo, n);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

// 2-D tiled map over rows (op * Qp + row) x columns (Qp), box 32 columns x tc_rows(Qp)
// rows, 128-byte swizzle, zero fill outside.
int tc_make_map(CUtensorMap* map, const float* table, int nops, int Qp) {
    EncodeTiled enc;
    KF_TRY(get_encoder(&enc));
    cuuint64_t dims[2] = {(cuuint64_t)Qp, (cuuint64_t)nops * (cuuint64_t)Qp};
    cuuint64_t strides[1] = {(cuuint64_t)Qp * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)tc::kKC, (cuuint32_t)tc_rows(Qp)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(table), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for a %d x %d table", (int)r, nops * Qp, Qp);
        return KIFMM_ERR_CUDA;
    }
    return KIFMM_OK;
}

template <int SLABS, int N>
static int launch_shape(int which, const CUtensorMap& hi, const CUtensorMap& lo, int Q, int Qp, const int4* tiles,
                        int ntiles, const int* pin, const int* pout, const float* in, float* out, int* err,
                        cudaStream_t s) {
    using S = tc::Shape<SLABS, N>;
    auto kern = which == 0 ? tc::k_u2u_tc<SLABS, N> : which == 1 ? tc::k_m2l_tc<SLABS, N> : tc::k_l2l_tc<SLABS, N>;
    // set on every launch: the attribute belongs to the current device's context
    KF_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kSmemBytes));
    const int mgroups = (Qp + S::kRows - 1) / S::kRows;
    kern<<<ntiles * mgroups, tc::kThreads, S::kSmemBytes, s>>>(hi, lo, Q, Qp, mgroups, tiles, pin, pout, in, out, err);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

// which: 0 = U2U (M2M'), 1 = M2L', 2 = L2L'.
int launch_pair_tc(int which, const CUtensorMap& hi, const CUtensorMap& lo, int Q, int Qp, const int4* tiles,
                   int ntiles, const int* pin, const int* pout, const float* in, float* out, int* err, cudaStream_t s) {
    if (ntiles <= 0) return KIFMM_OK;
    if (Qp <= 128) return launch_shape<1, 256>(which, hi, lo, Q, Qp, tiles, ntiles, pin, pout, in, out, err, s);
    return launch_shape<2, 128>(which, hi, lo, Q, Qp, tiles, ntiles, pin, pout, in, out, err, s);
}

}  // namespace kifmm
