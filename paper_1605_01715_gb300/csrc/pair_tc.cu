// Host launcher of the tcgen05 translation GEMM (see pair_tc.cuh).
#include "common.cuh"
#include "pair_tc.cuh"

namespace kifmm {

// Pairs per tile for a given padded order: the tile's N (TMEM columns per slab).
int tc_tile_pairs(int Qp) { return Qp <= 128 ? 256 : 128; }

template <int SLABS, int N>
static int launch_shape(const float* ops, int Q, int Qp, const int4* tiles, int ntiles, const int* pin,
                        const int* pout, const float* in, float* out, int* err, cudaStream_t s) {
    using S = tc::Shape<SLABS, N>;
    // set on every launch: the attribute belongs to the current device's context
    KF_CHECK_CUDA(cudaFuncSetAttribute(tc::k_pair_tc<SLABS, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       S::kSmemBytes));
    const int mgroups = (Qp + S::kRows - 1) / S::kRows;
    tc::k_pair_tc<SLABS, N><<<ntiles * mgroups, tc::kThreads, S::kSmemBytes, s>>>(ops, Q, Qp, mgroups, tiles, pin,
                                                                                   pout, in, out, err);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

int launch_pair_tc(const float* ops, int Q, int Qp, const int4* tiles, int ntiles, const int* pin, const int* pout,
                   const float* in, float* out, int* err, cudaStream_t s) {
    if (ntiles <= 0) return KIFMM_OK;
    if (Qp <= 128) return launch_shape<1, 256>(ops, Q, Qp, tiles, ntiles, pin, pout, in, out, err, s);
    return launch_shape<2, 128>(ops, Q, Qp, tiles, ntiles, pin, pout, in, out, err, s);
}

}  // namespace kifmm
