// Grouped translation GEMM on the 5th-generation tensor cores (tcgen05), 3xTF32.
//
// Every tile of the work list shares one Qp x Qp operator Op (M2M', M2L' or L2L') and
// holds up to kTcN (input box, output box) pairs; the CTA computes one 128-row slab of
//   out[pout[j]][row] += sum_k Op[row][k] * in[pin[j]][k]
// for all pairs j of the tile as D(128 x N) = A(128 x K) B(N x K)^T with A = the
// operator rows and B = the gathered input vectors, accumulated in TMEM (FP32).
//
// Two-term FP16: every operand is scaled by a power of two into [2^14, 2^15) at its
// largest entry and written as x = x_hi + x_lo with x_hi, x_lo the nearest FP16 values
// (22 significant bits); D += A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped A_lo B_lo
// term is ~2^-22 relative) with kind::f16 MMAs, and the epilogue undoes both scales.
// Operator tables have one scale each (texp); input vectors one per box (bexp).
//
// Accumulation: the tensor core adds into its FP32 accumulator with truncation, so a
// long K loop into one accumulator drifts by ~1 ulp of the running sum per MMA.  Each
// K-chunk of 32 therefore starts a fresh accumulator (correction products first, then
// the hi*hi products) in one of two TMEM buffers, and the threads fold every chunk's
// partial into FP32 registers (round-to-nearest) while the next chunk multiplies.
//
// Operands: the operator rows come pre-split (FP16 hi and lo tables) by TMA, one
// 64-column box per table and chunk, into the canonical K-major 128-byte-swizzled
// layout (rows of 128 B, 16-byte chunks XOR-permuted by row within 1024-byte atoms);
// the gathered input vectors are scaled and split by the threads into the same layout.  Every
// mbarrier wait is bounded; on a timeout the CTA records an error, waits (bounded)
// once more for work in flight, frees its TMEM and returns without writing.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace kifmm {
namespace tc {

constexpr int kKC = 64;             // K elements (FP16) per pipeline stage (4 MMA k-steps of 16)
constexpr int kThreads = 256;
constexpr uint32_t kRowBytes = kKC * 2;          // 128 B: one swizzle row
constexpr uint32_t kSBO = 8 * kRowBytes;         // 1024 B between 8-row groups
constexpr int kSlabBytes = 128 * kRowBytes;      // one 128-row operand slab of one chunk: 16 KB
constexpr int kScaleTop = 14;                    // operands scaled into [2^14, 2^15)
static_assert(kRowBytes == 128, "the 128-byte swizzle needs 64 FP16 per row");
constexpr long long kSpinLimit = 1LL << 26;

// Tile shape: SLABS x 128 operator rows by N pairs; two accumulator buffers fill the
// 512 TMEM columns (2 * SLABS * N = 512).  Each warp owns one lane quarter and 128
// accumulator columns, held as FP32 registers.
template <int SLABS, int N>
struct Shape {
    static constexpr int kRows = SLABS * 128;
    static constexpr int kTmemCols = 512;
    static constexpr int kBufCols = SLABS * N;                 // one accumulator buffer
    static constexpr int kABytes = SLABS * kSlabBytes;        // per hi or lo copy
    static constexpr int kBBytes = (N / 128) * kSlabBytes;     // per hi or lo copy (N multiple of 128)
    static constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes;
    static constexpr int kStages = 2;
    static constexpr int kSmemBytes = kStages * kStageBytes + 1024;
    static constexpr int kBVec = N * (kKC / 8) / kThreads;       // 8-element groups of B per thread per chunk
    static_assert(2 * SLABS * N == 512, "two accumulator buffers fill TMEM");
    static_assert(N % 128 == 0 && N <= 256, "N must be 128 or 256");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major, 128-byte swizzle: 8-row groups kSBO apart, leading offset unused (1),
// descriptor version 1, layout type 2 (SWIZZLE_128B).  Tiles are 1024-byte aligned;
// a K step inside the 128-byte row advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((kSBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 2-D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// kind::f16 instruction descriptor: D FP32, A/B FP16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (long long i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (i > 64) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 2^e as a float (e in [-126, 127]).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// Eight scaled values -> FP16 hi and lo parts, packed (x * scale = hi + lo to ~2^-22).
__device__ __forceinline__ void split_f16x8(float4 a, float4 b, float scale, uint4& hi, uint4& lo) {
    float x[8] = {a.x * scale, a.y * scale, a.z * scale, a.w * scale,
                  b.x * scale, b.y * scale, b.z * scale, b.w * scale};
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __half h0 = __float2half_rn(x[2 * i]), h1 = __float2half_rn(x[2 * i + 1]);
        __half l0 = __float2half_rn(x[2 * i] - __half2float(h0));
        __half l1 = __float2half_rn(x[2 * i + 1] - __half2float(h1));
        h[i] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
        l[i] = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Byte offset of (row r, 16-byte chunk c) in a K-major 128-byte-swizzled tile.
__device__ __forceinline__ uint32_t sw128_off(int r, int c) {
    return (uint32_t)(r * kRowBytes + ((c ^ (r & 7)) << 4));
}

// Element e of a chunk's grid of 16-byte (8 x FP16) groups -> (row r, chunk c).  Eight
// consecutive threads take eight consecutive rows of one chunk: after the swizzle
// their 16-byte stores hit eight different bank groups; a warp reads 128 contiguous
// bytes (FP32 source) from each of 8 rows in global memory.
__device__ __forceinline__ void chunk_coord(int e, int& r, int& c) {
    constexpr int KQ = kKC / 8;
    const int w = e % (8 * KQ);
    r = (e / (8 * KQ)) * 8 + (w & 7);
    c = w >> 3;
}

// grid.x = ntiles * mgroups (row group fastest).  tiles[t] = (op, first pair, count, 0).
// map_hi / map_lo: 2-D tensor maps of the split FP16 operator tables (scaled by 2^texp),
// rows = op * Qp + row, box = 64 columns x kRows rows, 128-byte swizzle.  bexp[box]:
// the power of two that brings the input vector of a box into FP16 range.
template <int SLABS, int N>
__device__ __forceinline__ void pair_tc_body(const CUtensorMap& map_hi, const CUtensorMap& map_lo, int texp, int Q,
                                             int Qp, int mgroups, const int4* __restrict__ tiles,
                                             const int* __restrict__ pin, const int* __restrict__ pout,
                                             const int* __restrict__ bexp, const float* __restrict__ in,
                                             float* __restrict__ out, int* __restrict__ err) {
    using S = Shape<SLABS, N>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    __shared__ uint64_t full_bar[2];      // TMA of stage s landed
    __shared__ uint64_t mma_bar[2];       // MMAs of accumulator buffer b (and stage b) done
    __shared__ uint32_t tmem_base;
    __shared__ int s_in[N], s_out[N];
    __shared__ float s_bscale[N], s_oscale[N];   // input scale, output unscale per pair
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile_id = blockIdx.x / mgroups, mg = blockIdx.x % mgroups;
    const int4 t = tiles[tile_id];
    const int cnt = t.z;
    const int m0 = mg * S::kRows;
    const int arow = t.x * Qp + m0;       // first operator row of this CTA in the table
    const int nchunks = (Qp + kKC - 1) / kKC;  // Qp is a multiple of 16; the tail is zero-filled

    for (int j = tid; j < N; j += kThreads) {
        const int bi = j < cnt ? pin[t.y + j] : -1;
        s_in[j] = bi;
        s_out[j] = j < cnt ? pout[t.y + j] : -1;
        const int e = bi >= 0 ? bexp[bi] : 0;
        s_bscale[j] = pow2f(e);
        s_oscale[j] = pow2f(-(e + texp));
    }
    auto stage_base = [&](int st) -> unsigned char* { return base + st * S::kStageBytes; };
    auto issue_tma = [&](int c) {
        unsigned char* sb = stage_base(c & 1);
        mbar_expect_tx(&full_bar[c & 1], 2u * S::kABytes);
        tma_load_2d(smem_u32(sb), &map_hi, c * kKC, arow, &full_bar[c & 1]);
        tma_load_2d(smem_u32(sb + S::kABytes), &map_lo, c * kKC, arow, &full_bar[c & 1]);
    };
    if (tid == 0) {
        s_abort = 0;
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full_bar[i], 1);
            mbar_init(&mma_bar[i], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        issue_tma(0);
        if (nchunks > 1) issue_tma(1);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(S::kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = idesc_f16(128, N);

    // this warp's accumulator columns: lane quarter q, slab my_slab, columns [my_col0, +128)
    const int quarter = warp & 3, half = warp >> 2;
    const int my_slab = (half * 128) / N, my_col0 = (half * 128) % N;
    float acc[128];
#pragma unroll
    for (int j = 0; j < 128; ++j) acc[j] = 0.f;

    // staged B: scaled, split and packed at load time (8 FP16 per 16-byte group)
    uint4 rhi[S::kBVec], rlo[S::kBVec];
    auto load_b = [&](int c) {
        const int k0 = c * kKC;
#pragma unroll
        for (int i = 0; i < S::kBVec; ++i) {
            int r, ch;
            chunk_coord(tid + i * kThreads, r, ch);
            int bi = s_in[r], k = k0 + 8 * ch;   // an 8-group lies wholly inside or outside Qp
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (bi >= 0 && k < Qp) {
                const float4* src = reinterpret_cast<const float4*>(in + (size_t)bi * Qp + k);
                a = src[0];
                b = src[1];
            }
            split_f16x8(a, b, s_bscale[r], rhi[i], rlo[i]);
        }
    };
    auto store_b = [&](unsigned char* sb) {
        unsigned char* bh = sb + 2 * S::kABytes;
#pragma unroll
        for (int i = 0; i < S::kBVec; ++i) {
            int r, ch;
            chunk_coord(tid + i * kThreads, r, ch);
            uint32_t o = (uint32_t)((r >> 7) * kSlabBytes) + sw128_off(r & 127, ch);
            *reinterpret_cast<uint4*>(bh + o) = rhi[i];
            *reinterpret_cast<uint4*>(bh + S::kBBytes + o) = rlo[i];
        }
    };
    auto fold = [&](int b) {
        const uint32_t col = (uint32_t)(b * S::kBufCols + my_slab * N + my_col0);
#pragma unroll
        for (int j0 = 0; j0 < 128; j0 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + col + (uint32_t)j0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j0 + j] += v[j];
        }
    };

    // thread 0 bookkeeping: last chunk whose MMAs were committed, last chunk whose TMA
    // was issued / waited for, and whether a wait gave up
    int issued = -1, tma_issued = nchunks > 1 ? 1 : 0, tma_waited = -1;
    bool dead = false;
    load_b(0);
    for (int c = 0; c < nchunks; ++c) {
        const int b = c & 1;
        unsigned char* sb = stage_base(b);
        // stage b / accumulator buffer b were last used by chunk c - 2: waited for and
        // folded in the previous iteration
        store_b(sb);
        if (c + 1 < nchunks) load_b(c + 1);       // in flight while this chunk multiplies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_fence_before();
        __syncthreads();
        if (tid == 0 && !dead) {
            if (!mbar_wait(&full_bar[b], (uint32_t)((c >> 1) & 1))) {
                dead = true;
                s_abort = 1;
            } else {
                tma_waited = c;
                tc_fence_after();
                const uint32_t a_hi = smem_u32(sb), a_lo = a_hi + S::kABytes;
                const uint32_t b_hi = a_hi + 2 * S::kABytes, b_lo = b_hi + S::kBBytes;
#pragma unroll
                for (int sl = 0; sl < SLABS; ++sl) {
                    const uint32_t d = tmem + (uint32_t)(b * S::kBufCols + sl * N);
                    const uint32_t ao = (uint32_t)(sl * kSlabBytes);
                    // small correction products first, then the hi*hi products
#pragma unroll
                    for (int ks = 0; ks < kKC / 16; ++ks) {
                        const uint32_t koff = ks * 32;  // 16 FP16 along K inside the swizzled row
                        mma_f16(d, smem_desc(a_hi + ao + koff), smem_desc(b_lo + koff), idesc, ks > 0 ? 1u : 0u);
                        mma_f16(d, smem_desc(a_lo + ao + koff), smem_desc(b_hi + koff), idesc, 1u);
                    }
#pragma unroll
                    for (int ks = 0; ks < kKC / 16; ++ks) {
                        const uint32_t koff = ks * 32;
                        mma_f16(d, smem_desc(a_hi + ao + koff), smem_desc(b_hi + koff), idesc, 1u);
                    }
                }
                mma_commit(&mma_bar[b]);
                issued = c;
            }
        }
        if (c >= 1) {
            const int pc = c - 1;
            if (tid == 0 && !dead) {
                if (!mbar_wait(&mma_bar[pc & 1], (uint32_t)((pc >> 1) & 1))) {
                    dead = true;
                    s_abort = 1;
                } else if (c + 1 < nchunks) {
                    issue_tma(c + 1);              // its stage was read by chunk c - 1, now done
                    tma_issued = c + 1;
                }
            }
            __syncthreads();
            if (s_abort) break;
            tc_fence_after();
            fold(pc & 1);
            tc_fence_before();
        }
    }
    // the last chunk
    if (tid == 0 && !dead) {
        if (issued != nchunks - 1 || !mbar_wait(&mma_bar[issued & 1], (uint32_t)((issued >> 1) & 1))) {
            dead = true;
            s_abort = 2;
        }
    }
    __syncthreads();
    if (!s_abort) {
        tc_fence_after();
        fold((nchunks - 1) & 1);          // uniform: every thread folds the last chunk's buffer
        const int row = m0 + my_slab * 128 + quarter * 32 + lane;
        if (row < Q) {
#pragma unroll
            for (int j = 0; j < 128; ++j) {
                int ob = s_out[my_col0 + j];
                if (ob >= 0) atomicAdd(out + (size_t)ob * Qp + row, acc[j] * s_oscale[my_col0 + j]);
            }
        }
    } else if (tid == 0) {
        // a wait gave up: one more bounded wait for the work in flight, then report
        if (issued >= 0) mbar_wait(&mma_bar[issued & 1], (uint32_t)((issued >> 1) & 1));
        for (int ch = tma_waited + 1; ch <= tma_issued; ++ch)
            mbar_wait(&full_bar[ch & 1], (uint32_t)((ch >> 1) & 1));
        atomicOr(err, s_abort);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::kTmemCols)
                     : "memory");
    }
}

// One kernel name per translation so profiles tell them apart.
#define KF_TC_KERNEL(NAME)                                                                                    \
    template <int SLABS, int N>                                                                               \
    __global__ void __launch_bounds__(kThreads, 1)                                                            \
        NAME(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo, int Q,   \
             int Qp, int mgroups, const int4* __restrict__ tiles, const int* __restrict__ pin,                \
             const int* __restrict__ pout, const int* __restrict__ bexp, int texp, const float* __restrict__ in, \
             float* __restrict__ out, int* __restrict__ err) {                                                 \
        pair_tc_body<SLABS, N>(map_hi, map_lo, texp, Q, Qp, mgroups, tiles, pin, pout, bexp, in, out, err);    \
    }
KF_TC_KERNEL(k_u2u_tc)
KF_TC_KERNEL(k_m2l_tc)
KF_TC_KERNEL(k_l2l_tc)
#undef KF_TC_KERNEL

}  // namespace tc
}  // namespace kifmm
