// Grouped translation GEMM on the 5th-generation tensor cores (tcgen05), two-term FP16.
//
// A work item is one tile of up to N (input box, output box) pairs that share one
// operator Op (Mr x Kp rows and columns of a table of such operators: a translation,
// or a projection onto a check-space basis) and one group of 128 * SLABS rows:
//   out[pout[j]][row] += sum_k Op[row][k] * in[pin[j]][k]
// computed as D(128 x N) = A(128 x K) B(N x K)^T per 128-row slab, with A = operator
// rows and B = the gathered input vectors, accumulated in TMEM.
//
// Two-term FP16: every operand is scaled by a power of two into [2^14, 2^15) at its
// largest entry and written as x = x_hi + x_lo with x_hi, x_lo the nearest FP16 values
// (22 significant bits); D += A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped A_lo B_lo
// term is ~2^-22 relative) with kind::f16 MMAs, and the epilogue undoes both scales.
// Operator tables have one scale each (texp); input vectors one per box (bexp), and
// both come pre-split: the operators once at setup, the box vectors right before the
// launch (one pass over the input buffer).
//
// Accumulation: the tensor core adds into its FP32 accumulator with truncation, so a
// long K loop into one accumulator drifts by ~1 ulp of the running sum per MMA.  Every
// FOLD * 32 columns of K therefore start a fresh accumulator (correction products
// first, then the hi*hi products) in one of two TMEM buffers, and the fold warps add
// each partial into FP32 registers (round-to-nearest) while the other buffer fills.
// The truncation dominates the rounding error of the whole mixed-precision matvec:
// folding every 32 columns instead of every 64 halved it (1M-point cube at p = 10,
// sampled rel-L2 8.9e-7 -> 4.4e-7) for 7 % more M2L time.
//
// Schedule: persistent, one CTA per SM walking the items blockIdx.x + k * gridDim.x,
// with the warps split into roles joined only by mbarriers:
//   warp 0      TMA of the operator rows (hi and lo tables, one 32-column box each)
//   warp 1      MMA issue (one thread); its commits free ring stages and fill accumulators
//   warps 2-3   cp.async of the input rows (16-byte copies, straight into the layout)
//   warps 4-11  fold of each accumulator into registers, then the scatter epilogue
// over a ring of kStages K-stages of 32 columns in the canonical K-major 64-byte-swizzled
// layout (rows of 64 B, 16-byte chunks XOR-permuted by row within 512-byte atoms).  The
// MMAs of the next item run while the fold warps scatter the previous one.
// Every wait is bounded; a wait that runs out raises an abort flag that stops the other
// roles, each of which then waits (bounded) for its own copies or MMAs in flight; the CTA
// records the error, frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace kifmm {
namespace tc {

constexpr int kKS = 32;                 // K elements (FP16) per ring stage: 2 MMA k-steps of 16
constexpr int kFoldStages = 1;          // ring stages per accumulator (32 columns of K)
constexpr int kStages = 4;              // ring depth
constexpr int kBLag = 2;                // stages of input copies a producer thread keeps in flight
// An accumulator holds its stages until its last one arrives; the producers must then
// still be able to fill that stage without waiting on the accumulator itself.
static_assert(kFoldStages + kBLag <= kStages, "ring too shallow for the fold group and the copy lag");
constexpr int kWarps = 12;
constexpr int kThreads = kWarps * 32;
constexpr int kProdWarp0 = 2, kProdThreads = 64;     // input-row producers
constexpr int kFoldWarp0 = 4, kFoldThreads = 256;    // fold / epilogue
constexpr int kFoldBar = 1;                          // named barrier of the fold warps
constexpr uint32_t kRowBytes = kKS * 2;              // 64 B: one swizzle row
constexpr uint32_t kSBO = 8 * kRowBytes;             // 512 B between 8-row groups
constexpr int kSlabBytes = 128 * kRowBytes;          // one 128-row slab of one stage: 8 KB
constexpr int kScaleTop = 14;                        // operands scaled into [2^14, 2^15)
static_assert(kRowBytes == 64, "the 64-byte swizzle needs 32 FP16 per row");
static_assert(kFoldThreads == (kWarps - kFoldWarp0) * 32 && kProdThreads == (kFoldWarp0 - kProdWarp0) * 32,
              "role split");
constexpr long long kSpinLimit = 1LL << 26;

// Tile shape: SLABS x 128 operator rows by N pairs; two accumulator buffers fill the
// 512 TMEM columns (2 * SLABS * N = 512).  Each fold warp owns one lane quarter and 128
// accumulator columns, held as FP32 registers.
template <int SLABS, int N>
struct Shape {
    static constexpr int kRows = SLABS * 128;
    static constexpr int kTmemCols = 512;
    static constexpr int kBufCols = SLABS * N;                 // one accumulator buffer
    static constexpr int kABytes = SLABS * kSlabBytes;        // per hi or lo table, one stage
    static constexpr int kBBytes = N * (int)kRowBytes;         // per hi or lo table, one stage
    static constexpr int kStageBytes = 2 * kABytes + 2 * kBBytes;
    static constexpr int kSmemBytes = kStages * kStageBytes + 1024;
    static constexpr int kBRows = N / 16;                      // input rows per producer thread
    static_assert(2 * SLABS * N == 512, "two accumulator buffers fill TMEM");
    static_assert(N % 128 == 0 && N <= 256, "N must be 128 or 256");
    static_assert(kStageBytes % 1024 == 0, "stages stay 1024-byte aligned");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major, 64-byte swizzle: 8-row groups kSBO apart, leading offset unused (1),
// descriptor version 1, layout type 4 (SWIZZLE_64B).  Tiles are 1024-byte aligned; a K
// step of 16 inside the 64-byte row advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((kSBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
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

// Bounded wait that also gives up once another role has raised *abort; a timeout
// raises it.  Returns false if it gave up.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* bar, uint32_t parity, volatile int* abort) {
    for (long long i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (i > 64) __nanosleep(32);
    }
    *abort = 1;
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Named barrier over the n threads of one role (id 0 is __syncthreads); the second
// form also returns whether pred held in any of them.
__device__ __forceinline__ void bar_named(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ bool bar_named_or(int id, int n, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %2, 0;\n\t"
        "bar.red.or.pred q, %1, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(id), "r"((uint32_t)pred), "r"(n)
        : "memory");
    return r != 0;
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

// 2^e as a float (e in [-126, 127]).
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// 16-byte asynchronous copy global -> shared; src_bytes = 0 writes zeros and reads nothing.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// Byte offset of (row r, 16-byte chunk c) in a K-major 64-byte-swizzled tile: the chunk
// index is XORed with bits 7-8 of the row's byte offset.
__device__ __forceinline__ uint32_t sw64_off(int r, int c) {
    return (uint32_t)(r * kRowBytes + ((c ^ ((r >> 1) & 3)) << 4));
}

// tiles[t] = (op, first pair, count, chain); work item w = (tile w / mgroups, row group
// w % mgroups).  chain = 1 (only with mgroups = 1): item w + gridDim.x, this CTA's next,
// has the same output box in every column and its products are added to this item's
// before they are written.  kcount (null: all items c + k G) holds each CTA's item count.  map_hi / map_lo: 2-D tensor maps of the split FP16 operator tables
// (scaled by 2^texp), rows = op * Mr + row (Mr rows per operator), columns Kp, box = 32
// columns x kRows rows, 64-byte swizzle.  in_hi / in_lo: the input vectors of all boxes
// scaled by 2^bexp[box] and split, Kp FP16 per box.  out: ostride floats per box, of
// which rows < M are written.
template <int SLABS, int N, int FOLD>
__device__ __forceinline__ void pair_tc_body(const CUtensorMap& map_hi, const CUtensorMap& map_lo, int texp, int M,
                                             int Kp, int ostride, int Mr, int mgroups, int nitems,
                                             const int4* __restrict__ tiles,
                                             const int* __restrict__ pin, const int* __restrict__ pout,
                                             const int* __restrict__ bexp, const __half* __restrict__ in_hi,
                                             const __half* __restrict__ in_lo, float* __restrict__ out,
                                             int* __restrict__ err, const int* __restrict__ kcount) {
    using S = Shape<SLABS, N>;
    const int G = gridDim.x;
    // items of this CTA: every G-th from blockIdx.x, or the first kcount[blockIdx.x] of them
    const int K = kcount ? kcount[blockIdx.x]
                         : (nitems > (int)blockIdx.x ? (nitems - (int)blockIdx.x + G - 1) / G : 0);
    if (K == 0) return;                   // uniform: nothing allocated yet
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
    __shared__ uint64_t tma_full[kStages];    // operator rows of a stage landed (TMA bytes)
    __shared__ uint64_t b_full[kStages];      // input rows of a stage landed (producer arrivals)
    __shared__ uint64_t empty[kStages];       // MMAs reading a stage done
    __shared__ uint64_t acc_full[2];          // accumulator buffer complete
    __shared__ uint64_t acc_empty[2];         // accumulator buffer folded
    __shared__ uint64_t drain_bar;            // all MMAs of the CTA done
    __shared__ uint32_t tmem_base;
    __shared__ int s_out[N];
    __shared__ __align__(16) float s_oscale[N];   // output unscale per pair
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nst = (Kp + kKS - 1) / kKS;                     // stages per item (tail zero-filled)
    const int nfg = (nst + FOLD - 1) / FOLD;   // accumulators per item
    volatile int* abort = &s_abort;
    auto stage_u32 = [&](int s) -> uint32_t { return smem_u32(base) + (uint32_t)(s * S::kStageBytes); };

    if (tid == 0) {
        s_abort = 0;
        for (int i = 0; i < kStages; ++i) {
            mbar_init(&tma_full[i], 1);
            mbar_init(&b_full[i], kProdThreads);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc_full[i], 1);
            mbar_init(&acc_empty[i], kFoldThreads);
        }
        mbar_init(&drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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

    if (warp == 0) {
        // ---- operator rows by TMA ----
        if (lane == 0) {
            int g = 0;
            bool ok = true;
            for (int k = 0; k < K && ok; ++k) {
                const int w = (int)blockIdx.x + k * G;
                const int arow = tiles[w / mgroups].x * Mr + (w % mgroups) * S::kRows;
                for (int i = 0; i < nst; ++i, ++g) {
                    const int s = g % kStages;
                    if (g >= kStages && !mbar_wait_ab(&empty[s], (uint32_t)(((g / kStages) - 1) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&tma_full[s], 2u * S::kABytes);
                    tma_load_2d(stage_u32(s), &map_hi, i * kKS, arow, &tma_full[s]);
                    tma_load_2d(stage_u32(s) + S::kABytes, &map_lo, i * kKS, arow, &tma_full[s]);
                }
            }
            // every issued load has landed before the CTA can end (not cut short by an abort)
            for (int s = 0; s < kStages && s < g; ++s) {
                const int last = s + ((g - 1 - s) / kStages) * kStages;
                if (!mbar_wait(&tma_full[s], (uint32_t)((last / kStages) & 1))) *abort = 1;
            }
        }
    } else if (warp == 1) {
        // ---- MMA issue ----
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_f16(128, N);
            bool ok = true, any = false;
            int g = 0;
            for (int k = 0; k < K && ok; ++k) {
                for (int i = 0; i < nst; ++i, ++g) {
                    const int s = g % kStages;
                    const int f = k * nfg + i / FOLD, b = f & 1;
                    const bool first = i % FOLD == 0;
                    const bool last = i % FOLD == FOLD - 1 || i == nst - 1;
                    if (first && f >= 2 && !mbar_wait_ab(&acc_empty[b], (uint32_t)(((f >> 1) - 1) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    const uint32_t ph = (uint32_t)((g / kStages) & 1);
                    if (!mbar_wait_ab(&tma_full[s], ph, abort) || !mbar_wait_ab(&b_full[s], ph, abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // the small correction products of this stage now; the hi*hi products of
                    // every stage of the accumulator last, once all its stages are resident
                    // (the same order as one K step of the accumulator: fewer truncating adds at the
                    // accumulator's full magnitude)
                    const uint32_t a_hi = stage_u32(s), a_lo = a_hi + S::kABytes;
                    const uint32_t b_hi = a_hi + 2 * S::kABytes, b_lo = b_hi + S::kBBytes;
#pragma unroll
                    for (int sl = 0; sl < SLABS; ++sl) {
                        const uint32_t d = tmem + (uint32_t)(b * S::kBufCols + sl * N);
                        const uint32_t ao = (uint32_t)(sl * kSlabBytes);
#pragma unroll
                        for (int ks = 0; ks < kKS / 16; ++ks) {
                            const uint32_t koff = ks * 32;  // 16 FP16 along K inside the swizzled row
                            mma_f16(d, smem_desc(a_hi + ao + koff), smem_desc(b_lo + koff), idesc,
                                    (first && ks == 0) ? 0u : 1u);
                            mma_f16(d, smem_desc(a_lo + ao + koff), smem_desc(b_hi + koff), idesc, 1u);
                        }
                    }
                    any = true;
                    if (last) {
                        const int g0 = g - i % FOLD;   // first stage of this accumulator
                        for (int gg = g0; gg <= g; ++gg) {
                            const uint32_t ah = stage_u32(gg % kStages), bh = ah + 2 * S::kABytes;
#pragma unroll
                            for (int sl = 0; sl < SLABS; ++sl) {
                                const uint32_t d = tmem + (uint32_t)(b * S::kBufCols + sl * N);
                                const uint32_t ao = (uint32_t)(sl * kSlabBytes);
#pragma unroll
                                for (int ks = 0; ks < kKS / 16; ++ks) {
                                    const uint32_t koff = ks * 32;
                                    mma_f16(d, smem_desc(ah + ao + koff), smem_desc(bh + koff), idesc, 1u);
                                }
                            }
                        }
                        for (int gg = g0; gg <= g; ++gg) mma_commit(&empty[gg % kStages]);
                        mma_commit(&acc_full[b]);
                    }
                }
            }
            // every MMA (and the arrivals it owes) is done before the CTA can end
            if (any) {
                mma_commit(&drain_bar);
                if (!mbar_wait(&drain_bar, 0)) *abort = 1;
            }
        }
    } else if (warp < kFoldWarp0) {
        // ---- input rows by cp.async: thread pt copies 16-byte chunk pt % 4 of rows
        // pt / 4 + 16 j, so four neighbouring threads read one 64-byte row slice ----
        const int pt = tid - kProdWarp0 * 32, rr = pt >> 2, c = pt & 3;
        int bi[S::kBRows];
        int g = 0;
        bool ok = true;
        for (int k = 0; k < K && ok; ++k) {
            const int w = (int)blockIdx.x + k * G;
            const int4 t = tiles[w / mgroups];
#pragma unroll
            for (int j = 0; j < S::kBRows; ++j) {
                const int r = j * 16 + rr;
                bi[j] = r < t.z ? pin[t.y + r] : -1;
            }
            for (int i = 0; i < nst; ++i, ++g) {
                const int s = g % kStages;
                if (g >= kStages && !mbar_wait_ab(&empty[s], (uint32_t)(((g / kStages) - 1) & 1), abort)) {
                    ok = false;
                    break;
                }
                const uint32_t bh = stage_u32(s) + 2 * S::kABytes;
                const int kk = i * kKS + 8 * c;          // an 8-group lies wholly inside or outside Kp
#pragma unroll
                for (int j = 0; j < S::kBRows; ++j) {
                    const bool v = bi[j] >= 0 && kk < Kp;
                    const size_t off = v ? (size_t)bi[j] * Kp + kk : 0;
                    const uint32_t o = sw64_off(j * 16 + rr, c);
                    cp_async16(bh + o, in_hi + off, v ? 16u : 0u);
                    cp_async16(bh + S::kBBytes + o, in_lo + off, v ? 16u : 0u);
                }
                cp_async_commit();
                if (g >= kBLag) {
                    // stage g - kBLag: this thread's copies have landed; hand them to the
                    // tensor core's (async) proxy and arrive
                    cp_async_wait<kBLag>();
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive(&b_full[(g - kBLag) % kStages]);
                }
            }
        }
        cp_async_wait<0>();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (ok)
            for (int gg = g > kBLag ? g - kBLag : 0; gg < g; ++gg) mbar_arrive(&b_full[gg % kStages]);
    } else {
        // ---- fold and epilogue: lane quarter warp % 4 (the TMEM lanes this warp may
        // read), slab my_slab, accumulator columns [my_col0, +128) ----
        const int fw = warp - kFoldWarp0, ft = tid - kFoldWarp0 * 32;
        const int quarter = warp & 3, half = fw >> 2;
        const int my_slab = (half * 128) / N, my_col0 = (half * 128) % N;
        float2 acc[64];                       // columns 2j and 2j+1 of this thread's row
        auto load_meta = [&](int k) {
            const int w = (int)blockIdx.x + k * G;
            const int4 t = tiles[w / mgroups];
            for (int j = ft; j < N; j += kFoldThreads) {
                const int bi = j < t.z ? pin[t.y + j] : -1;
                s_out[j] = j < t.z ? pout[t.y + j] : -1;
                s_oscale[j] = pow2f(-((bi >= 0 ? bexp[bi] : 0) + texp));
            }
        };
        load_meta(0);
        bar_named(kFoldBar, kFoldThreads);
        // A chain: consecutive items of this CTA with the same output box in every column
        // (tile.w = 1: the next item of this CTA continues it).  Its sums stay in acc
        // across its items and are written once, after the last.  Each fold adds its
        // columns already unscaled (by powers of two, so the sums round as if unscaled
        // at the end).
        bool cont_prev = false;
        const float4* osc4 = reinterpret_cast<const float4*>(s_oscale + my_col0);
        for (int k = 0; k < K; ++k) {
            const int w = (int)blockIdx.x + k * G;
            const bool cont = mgroups == 1 && tiles[w / mgroups].w != 0;
            if (!cont_prev) {
#pragma unroll
                for (int j = 0; j < 64; ++j) acc[j] = make_float2(0.f, 0.f);
            }
            bool ok = true;
            for (int j = 0; j < nfg; ++j) {
                const int f = k * nfg + j, b = f & 1;
                if (!mbar_wait_ab(&acc_full[b], (uint32_t)((f >> 1) & 1), abort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t col = (uint32_t)(b * S::kBufCols + my_slab * N + my_col0);
#pragma unroll
                for (int j0 = 0; j0 < 128; j0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + col + (uint32_t)j0, v);
#pragma unroll
                    for (int jj = 0; jj < 16; jj += 4) {
                        // packed FP32x2: the same roundings as two scalar FMAs
                        const float4 sc = osc4[(j0 + jj) >> 2];
                        const int a = (j0 + jj) >> 1;
                        acc[a] = __ffma2_rn(make_float2(v[jj], v[jj + 1]), make_float2(sc.x, sc.y), acc[a]);
                        acc[a + 1] = __ffma2_rn(make_float2(v[jj + 2], v[jj + 3]), make_float2(sc.z, sc.w), acc[a + 1]);
                    }
                }
                tc_fence_before();
                mbar_arrive(&acc_empty[b]);
            }
            if (bar_named_or(kFoldBar, kFoldThreads, !ok)) break;   // uniform across the fold warps
            const int row = (w % mgroups) * S::kRows + my_slab * 128 + quarter * 32 + lane;
            if (!cont && row < M) {
#pragma unroll
                for (int j = 0; j < 128; ++j) {
                    const int ob = s_out[my_col0 + j];
                    if (ob >= 0) atomicAdd(out + (size_t)ob * ostride + row, (j & 1) ? acc[j >> 1].y : acc[j >> 1].x);
                }
            }
            cont_prev = cont;
            if (k + 1 < K) {
                bar_named(kFoldBar, kFoldThreads);   // every fold thread is done with item k's table
                load_meta(k + 1);
                bar_named(kFoldBar, kFoldThreads);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && s_abort) atomicOr(err, 1);
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::kTmemCols)
                     : "memory");
    }
}

// One kernel name per translation so profiles tell them apart.
#define KF_TC_KERNEL(NAME, FOLD)                                                                                \
    template <int SLABS, int N>                                                                                 \
    __global__ void __launch_bounds__(kThreads, 1)                                                              \
        NAME(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo, int M,     \
             int Kp, int ostride, int Mr, int mgroups, int nitems, const int4* __restrict__ tiles,               \
             const int* __restrict__ pin, const int* __restrict__ pout, const int* __restrict__ bexp, int texp,  \
             const __half* __restrict__ in_hi, const __half* __restrict__ in_lo, float* __restrict__ out,        \
             int* __restrict__ err, const int* __restrict__ kcount) {                                            \
        pair_tc_body<SLABS, N, FOLD>(map_hi, map_lo, texp, M, Kp, ostride, Mr, mgroups, nitems, tiles, pin, pout,     \
                               bexp, in_hi, in_lo, out, err, kcount);                                            \
    }
KF_TC_KERNEL(k_u2u_tc, kFoldStages)
KF_TC_KERNEL(k_m2l_tc, kFoldStages)
KF_TC_KERNEL(k_l2l_tc, kFoldStages)
KF_TC_KERNEL(k_proj_tc, kFoldStages)
#undef KF_TC_KERNEL

}  // namespace tc
}  // namespace kifmm
