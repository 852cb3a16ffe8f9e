// Peak-rate microbenchmarks: the denominators of the near-field and FP64 rooflines.
//
// Each kernel issues one kind of arithmetic instruction from every resident thread
// of every SM, on eight independent dependency chains per thread, with nothing else
// in its loop but the loop counter.  The rate is the instruction count over the
// CUDA-event time of the launch: what this GPU sustains for that instruction at the
// clock it runs during the measurement.
//   unit 0  FP32 FMA, scalar (fmaf)                     2 flops per lane-op
//   unit 1  FP32 FMA, packed pairs (__ffma2_rn)         4 flops per lane-op
//   unit 2  FP32 reciprocal square root                 1 op per lane-op
//           (rsqrt.approx.ftz.f32, the near field's instruction)
//   unit 3  FP64 FMA (fma)                              2 flops per lane-op
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"

namespace kifmm {
namespace {

constexpr int kPeakThreads = 512;
constexpr int kChains = 8;
constexpr int kUnroll = 8;

template <int UNIT>
__global__ void __launch_bounds__(kPeakThreads) k_peak(int iters, float seed, float* __restrict__ sink) {
    const float s = seed + 1e-7f * (float)(threadIdx.x & 7);
    if constexpr (UNIT == 0) {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = s + (float)k;
        const float b = 0.9999f, c = 1e-4f;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
        }
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) t += a[k];
        if (t == 12345.678f) sink[threadIdx.x] = t;
    } else if constexpr (UNIT == 1) {
        float2 a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = make_float2(s + (float)k, s - (float)k);
        const float2 b = make_float2(0.9999f, 0.9998f), c = make_float2(1e-4f, 2e-4f);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = __ffma2_rn(a[k], b, c);
        }
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) t += a[k].x + a[k].y;
        if (t == 12345.678f) sink[threadIdx.x] = t;
    } else if constexpr (UNIT == 2) {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = 1.5f + s + (float)k;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int k = 0; k < kChains; ++k)                        // x -> x^(-1/2): stays near 1
                    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(a[k]) : "f"(a[k]));
        }
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) t += a[k];
        if (t == 12345.678f) sink[threadIdx.x] = t;
    } else {
        double a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = (double)s + k;
        const double b = 0.9999, c = 1e-4;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
#pragma unroll
                for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
        }
        double t = 0.0;
#pragma unroll
        for (int k = 0; k < kChains; ++k) t += a[k];
        if (t == 12345.678) sink[threadIdx.x] = (float)t;
    }
}

template <int UNIT>
int time_peak(int iters, cudaStream_t s, float* sink, unsigned grid, float* ms) {
    cudaEvent_t e0, e1;
    KF_CHECK_CUDA(cudaEventCreate(&e0));
    KF_CHECK_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, s);
    k_peak<UNIT><<<grid, kPeakThreads, 0, s>>>(iters, 1.0f, sink);
    cudaError_t le = cudaGetLastError();
    cudaEventRecord(e1, s);
    cudaError_t se = cudaEventSynchronize(e1);
    float t = 0.f;
    if (le == cudaSuccess && se == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (le != cudaSuccess || se != cudaSuccess) {
        set_error("peak kernel: %s", cudaGetErrorString(le != cudaSuccess ? le : se));
        return KIFMM_ERR_CUDA;
    }
    *ms = t;
    return KIFMM_OK;
}

template <int UNIT>
int run_peak(int reps, cudaStream_t s, double* rate, double* ms_out) {
    int dev = 0, nsm = 0, per_sm = 0;
    KF_CHECK_CUDA(cudaGetDevice(&dev));
    KF_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    KF_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peak<UNIT>, kPeakThreads, 0));
    per_sm = std::max(per_sm, 1);
    const unsigned grid = (unsigned)(nsm * per_sm);
    DBuf<float> sink;
    KF_TRY(sink.alloc(kPeakThreads));
    // size the launch to about 10 ms from a short calibration launch
    int iters = 256;
    float ms = 0.f;
    KF_TRY(time_peak<UNIT>(iters, s, sink.p, grid, &ms));
    for (int k = 0; k < 3 && ms < 2.0f; ++k) {
        const double scale = ms > 0.01f ? 10.0 / ms : 16.0;
        iters = (int)std::min(1.0e8, std::max(256.0, iters * std::min(scale, 64.0)));
        KF_TRY(time_peak<UNIT>(iters, s, sink.p, grid, &ms));
    }
    float best = 1e30f;
    for (int r = 0; r < std::max(reps, 1); ++r) {
        KF_TRY(time_peak<UNIT>(iters, s, sink.p, grid, &ms));
        best = std::min(best, ms);
    }
    const double lane_ops = (double)grid * kPeakThreads * (double)iters * kUnroll * kChains;
    const double per_op = (UNIT == 0 || UNIT == 3) ? 2.0 : (UNIT == 1 ? 4.0 : 1.0);
    *rate = lane_ops * per_op / (best * 1e-3);
    if (ms_out) *ms_out = best;
    return KIFMM_OK;
}

}  // namespace
}  // namespace kifmm

using namespace kifmm;

extern "C" int kifmm_peak_rate(int unit, int reps, double* rate, double* ms, void* stream) {
    clear_error();
    KF_ARG(rate != nullptr, "rate is NULL");
    KF_ARG(unit >= 0 && unit <= 3, "unit must be 0..3");
    KF_ARG(reps >= 1 && reps <= 100, "reps must be in [1, 100]");
    cudaStream_t s = (cudaStream_t)stream;
    switch (unit) {
    case 0: return run_peak<0>(reps, s, rate, ms);
    case 1: return run_peak<1>(reps, s, rate, ms);
    case 2: return run_peak<2>(reps, s, rate, ms);
    default: return run_peak<3>(reps, s, rate, ms);
    }
}
