// KIFMM plan set-up and the matvec f = K q (Sec. II.A, Eq. sum_fmm) on the device.
//
// One matvec, all in check-potential space (see operators.cu):
//   gather  q into Morton order (DL: q n_j, the source normal applied at the
//           source-to-check step, Sec. III.A.1 Eq. p2m -- the paper's second method)
//   S2U     leaf up-check potentials from the leaf's sources
//   U2U     parent up-check += M2M'_oct child up-check, level by level upward
//   X       down-check potentials from the sources of X-list leaves (non-leaf targets;
//           a target leaf takes its X-list sources directly in P2P)
//   M2L     down-check += M2L'_offset up-check of each V-list box
//   L2L     child down-check += L2L'_oct parent down-check, level by level downward
//   D2T     far-field value at each target = its precomputed row . leaf down-check
//   P2P     near field over U-, W- (and for leaves X-) list sources, added, scattered to
//           input order
// Near-singular pairs (|r_i - r_j| < 1e-5) contribute nothing (Sec. III.A.1).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <queue>
#include <type_traits>
#include <unordered_map>

#include "cheb.cuh"
#include "common.cuh"
#include "operators.cuh"
#include "plan.cuh"

namespace kifmm {

int tc_tile_pairs(int Qp);
int tc_split_table(const float* table, __half* hi, __half* lo, size_t n, int* texp, cudaStream_t s);
int tc_box_split(const float* v, int Q, int Qp, int b0, int b1, __half* hi, __half* lo, int* e, cudaStream_t s);
int tc_make_map(CUtensorMap* map, const __half* table, int nops, int Mr, int Kp);
int launch_pair_tc(int which, const CUtensorMap& hi, const CUtensorMap& lo, int texp, int M, int Mr, int Kp,
                   int ostride, const int4* tiles, int ntiles, const int* pin, const int* pout, const int* bexp,
                   const __half* in_hi, const __half* in_lo, float* out, int* err, cudaStream_t s,
                   const int* kcount = nullptr);

namespace {

// Largest pseudo-inverse rank of the mixed form: the operator rows one tensor-core work
// item covers (two 128-row slabs).
constexpr int kMixedMaxRank = 256;

// 1/sqrt(x) by the hardware approximation with subnormal inputs and results flushed to
// zero (PTX rsqrt.approx.ftz.f32), without the rescaling of subnormal inputs that
// rsqrtf adds around it.  Every r^2 that reaches it is a normal float, or 0 for a pair
// within the tolerance radius, whose term a select then drops.
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <typename Real> struct RT;
template <> struct RT<float> {
    static __device__ __forceinline__ float rsq(float x) { return rsqrt_ftz(x); }
};
template <> struct RT<double> {
    static __device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
};

// Kernels whose target side is a gradient (ADL: along the target normal; the field: all
// three components).  Only the variation of a down-check potential reaches them.
inline bool gradient_kernel(int kernel) { return kernel == KIFMM_KERNEL_ADL || kernel == KIFMM_KERNEL_FIELD; }

// ---------------------------------------------------------------- gather
// lo: also write the rounding remainders of the dipoles (3 more rows, read by the
// mixed near field's exact products)
template <typename Real>
__global__ void k_gather_q(const double* __restrict__ q, const int64_t* __restrict__ perm, int64_t n,
                           const double* __restrict__ snrm, Real* __restrict__ qs, bool lo) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = q[perm[i]];
    if (snrm) {  // dipole strengths q n_j, SoA
        for (int d = 0; d < 3; ++d) {
            const double pd = v * snrm[d * n + i];
            qs[d * n + i] = (Real)pd;
            if (lo) qs[(3 + d) * n + i] = (Real)(pd - (double)(Real)pd);
        }
    } else {
        qs[i] = (Real)v;
    }
}

// The same from q in input order (a host buffer: each element read once, in order)
// scattered to the sorted positions iperm[i].
template <typename Real>
__global__ void k_scatter_q(const double* __restrict__ q, const int64_t* __restrict__ iperm, int64_t n,
                            const double* __restrict__ snrm, Real* __restrict__ qs, bool lo) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = q[i];
    const int64_t j = iperm[i];
    if (snrm) {
        for (int d = 0; d < 3; ++d) {
            const double pd = v * snrm[d * n + j];
            qs[d * n + j] = (Real)pd;
            if (lo) qs[(3 + d) * n + j] = (Real)(pd - (double)(Real)pd);
        }
    } else {
        qs[j] = (Real)v;
    }
}

// iperm[perm[j]] = j
__global__ void k_invert_perm(const int64_t* __restrict__ perm, int64_t n, int64_t* __restrict__ iperm) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < n) iperm[perm[j]] = j;
}

// ---------------------------------------------------------------- sources -> surface (S2U, X list)
// One block per box; threads own surface points; sources of the CSR boxes staged in
// shared memory relative to the box centre.  DIPOLE: n_j.(x - y)/|x - y|^3 q_j, else q_j/|x - y|.
constexpr int kSurfThreads = 128;
constexpr int kSurfPer = 8;  // Q <= 1024
constexpr double kSkelTol = 1e-9;   // pivots of the S2U skeleton: |R_ii| above this x |R_00|

template <typename Real, bool DIPOLE>
__global__ void __launch_bounds__(kSurfThreads)
k_src2surf(const int* __restrict__ boxes, const int* __restrict__ off, const int* __restrict__ idx,
           double radius, const int* __restrict__ lvl, const double* __restrict__ ctr, double root_h,
           const int64_t* __restrict__ rng, const double* __restrict__ sxyz, int64_t ns,
           const Real* __restrict__ qs, const Real* __restrict__ surf, int Q, int Qp,
           Real* __restrict__ outbuf) {
    __shared__ Real sy[4][kSurfThreads];
    __shared__ Real sq[3][kSurfThreads];
    int b = boxes[blockIdx.x];
    double cx = ctr[3 * b], cy = ctr[3 * b + 1], cz = ctr[3 * b + 2];
    Real rf = (Real)(radius * ldexp(root_h, -lvl[b]));
    Real px[kSurfPer], py[kSurfPer], pz[kSurfPer], acc[kSurfPer];
#pragma unroll
    for (int i = 0; i < kSurfPer; ++i) {
        int k = threadIdx.x + i * kSurfThreads;
        int kk = k < Q ? k : 0;
        px[i] = rf * surf[3 * kk];
        py[i] = rf * surf[3 * kk + 1];
        pz[i] = rf * surf[3 * kk + 2];
        acc[i] = 0;
    }
    const Real d2 = (Real)(kDelta * kDelta);
    for (int e = off[blockIdx.x]; e < off[blockIdx.x + 1]; ++e) {
        int a = idx[e];
        int64_t sb = rng[4 * a], se = rng[4 * a + 1];
        for (int64_t j0 = sb; j0 < se; j0 += kSurfThreads) {
            int64_t j = j0 + threadIdx.x;
            if (j < se) {
                sy[0][threadIdx.x] = (Real)(sxyz[j] - cx);
                sy[1][threadIdx.x] = (Real)(sxyz[ns + j] - cy);
                sy[2][threadIdx.x] = (Real)(sxyz[2 * ns + j] - cz);
                if (DIPOLE) {
                    sq[0][threadIdx.x] = qs[j];
                    sq[1][threadIdx.x] = qs[ns + j];
                    sq[2][threadIdx.x] = qs[2 * ns + j];
                } else {
                    sq[0][threadIdx.x] = qs[j];
                }
            }
            __syncthreads();
            int cnt = (int)((se - j0) < (int64_t)kSurfThreads ? (se - j0) : (int64_t)kSurfThreads);
            for (int jj = 0; jj < cnt; ++jj) {
                Real yx = sy[0][jj], yy = sy[1][jj], yz = sy[2][jj];
#pragma unroll
                for (int i = 0; i < kSurfPer; ++i) {
                    if (i * kSurfThreads >= Q) break;
                    Real dx = px[i] - yx, dy = py[i] - yy, dz = pz[i] - yz;
                    Real r2 = dx * dx + dy * dy + dz * dz;
                    Real inv = RT<Real>::rsq(r2);
                    Real v;
                    if (DIPOLE) v = (sq[0][jj] * dx + sq[1][jj] * dy + sq[2][jj] * dz) * inv * inv * inv;
                    else v = sq[0][jj] * inv;
                    acc[i] += (r2 >= d2) ? v : (Real)0;
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < kSurfPer; ++i) {
        int k = threadIdx.x + i * kSurfThreads;
        if (k < Q) outbuf[(size_t)b * Qp + k] += acc[i];
    }
}

// FP32 form.  Each of NT threads owns 2 NP surface points (points threadIdx.x + i NT)
// as NP packed pairs: every step is one FP32x2 instruction for two points (the same
// round-to-nearest operations as the scalar form).  Staged sources are float4 --
// (x, y, z, q), and (q n_j) over two float4 for dipoles -- built from FP32 hi/lo
// coordinates relative to the box centre, so one broadcast load feeds 2 NP
// evaluations.  Box centres (hi/lo), half-widths and check radii come as FP32 from a
// per-box table (bcf: 3 float4 per box).  The tolerance-radius test is dropped for a
// source box whose cube is provably farther than 2 delta from the check surface in
// the max-norm (outside the surface's cube, or inside it).
// DIFF (monopoles only): q (1/|p - y| - 1/|y|), the potential less its value at the box
// centre, as q (2 p.y - |p|^2) / (|p - y| |y| (|p - y| + |y|)) -- exact for the variation
// across the check surface, which is all a gradient kernel's far field keeps (sd holds
// 1/|y| and |y| per source; pp the |p|^2 of each packed check point pair).
// AX (dipoles): 0..2 when every source's dipole lies along that axis -- one term of
// n . (p - y), the same value as the three-term sum, whose other products are exact zeros.
template <bool NEAR, bool DIPOLE, int NP, bool DIFF = false, int AX = 3>
__device__ __forceinline__ void surf_pairs(const float4* __restrict__ sp, const float4* __restrict__ sd, int cnt,
                                           const float2* px, const float2* py, const float2* pz, float2* acc,
                                           const float2* pp = nullptr) {
    const float d2 = (float)(kDelta * kDelta);
#pragma unroll 2
    for (int jj = 0; jj < cnt; ++jj) {
        const float4 y = sp[jj];
        const float2 nx = make_float2(-y.x, -y.x), ny = make_float2(-y.y, -y.y), nz = make_float2(-y.z, -y.z);
        float2 qa = make_float2(y.w, y.w), qb, qc;
        if (DIPOLE || DIFF) {
            const float4 dq = sd[jj];
            qb = make_float2(dq.x, dq.x);
            qc = make_float2(dq.y, dq.y);
        }
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const float2 dx = __fadd2_rn(px[m], nx), dy = __fadd2_rn(py[m], ny), dz = __fadd2_rn(pz[m], nz);
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            const float2 inv = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
            float2 f, w;                                                     // the pair's value f w
            if (DIFF) {
                // |y|^2 - |p - y|^2 = 2 p.y - |p|^2; |p - y| = r2 inv
                const float2 dot = __ffma2_rn(pz[m], make_float2(y.z, y.z),
                                   __ffma2_rn(py[m], make_float2(y.y, y.y), __fmul2_rn(px[m], make_float2(y.x, y.x))));
                const float2 dp = __ffma2_rn(make_float2(2.f, 2.f), dot, make_float2(-pp[m].x, -pp[m].y));
                const float2 a = __fmul2_rn(r2, inv);
                const float2 sum = __fadd2_rn(a, qc);                        // |p - y| + |y|
                const float2 rs = make_float2(__fdividef(1.f, sum.x), __fdividef(1.f, sum.y));
                f = __fmul2_rn(__fmul2_rn(qa, dp), __fmul2_rn(inv, qb));
                w = rs;
            } else if (DIPOLE) {
                if (AX == 0) f = __fmul2_rn(qa, dx);
                else if (AX == 1) f = __fmul2_rn(qb, dy);
                else if (AX == 2) f = __fmul2_rn(qc, dz);
                else f = __ffma2_rn(qc, dz, __ffma2_rn(qb, dy, __fmul2_rn(qa, dx)));
                w = __fmul2_rn(__fmul2_rn(inv, inv), inv);
            } else {
                f = qa;
                w = inv;
            }
            if (NEAR) {
                w.x = r2.x >= d2 ? w.x : 0.f;
                w.y = r2.y >= d2 ? w.y : 0.f;
            }
            acc[m] = __ffma2_rn(f, w, acc[m]);
        }
    }
}

// Dipoles along axis K whose sources all lie in one plane normal to K (a flat face's
// leaf): the offset along K, dk = p_K - c, is the same for every source of the box, so
// the pairs only sum q_K / r^3 (r^2 = the in-plane offsets' squares + dk^2) and the
// caller multiplies the box's sum by dk once.  Two in-plane offsets instead of three.
template <bool NEAR, int NP, int K>
__device__ __forceinline__ void surf_pairs_plane(const float4* __restrict__ sp, const float4* __restrict__ sd,
                                                 int cnt, const float2* px, const float2* py, const float2* pz,
                                                 const float2* dk2, float2* acc) {
    const float d2 = (float)(kDelta * kDelta);
#pragma unroll 2
    for (int jj = 0; jj < cnt; ++jj) {
        const float4 y = sp[jj];
        const float4 dq = sd[jj];
        const float qk = K == 0 ? y.w : (K == 1 ? dq.x : dq.y);
        const float ya = K == 0 ? y.y : y.x, yb = K == 2 ? y.y : y.z;      // the in-plane coordinates
        const float2 na = make_float2(-ya, -ya), nb = make_float2(-yb, -yb), q2 = make_float2(qk, qk);
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const float2 da = __fadd2_rn(K == 0 ? py[m] : px[m], na);
            const float2 db = __fadd2_rn(K == 2 ? py[m] : pz[m], nb);
            const float2 r2 = __ffma2_rn(da, da, __ffma2_rn(db, db, dk2[m]));
            const float2 inv = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
            float2 w = __fmul2_rn(__fmul2_rn(inv, inv), inv);
            if (NEAR) {
                w.x = r2.x >= d2 ? w.x : 0.f;
                w.y = r2.y >= d2 ? w.y : 0.f;
            }
            acc[m] = __ffma2_rn(q2, w, acc[m]);
        }
    }
}

template <bool NEAR, int NP>
__device__ __forceinline__ void surf_pairs_plane_k(int k, const float4* __restrict__ sp,
                                                   const float4* __restrict__ sd, int cnt, const float2* px,
                                                   const float2* py, const float2* pz, const float2* dk2,
                                                   float2* acc) {
    if (k == 0) surf_pairs_plane<NEAR, NP, 0>(sp, sd, cnt, px, py, pz, dk2, acc);
    else if (k == 1) surf_pairs_plane<NEAR, NP, 1>(sp, sd, cnt, px, py, pz, dk2, acc);
    else surf_pairs_plane<NEAR, NP, 2>(sp, sd, cnt, px, py, pz, dk2, acc);
}

template <bool NEAR, bool DIPOLE, int NP, bool DIFF>
__device__ __forceinline__ void surf_pairs_ax(int ax, const float4* __restrict__ sp, const float4* __restrict__ sd,
                                              int cnt, const float2* px, const float2* py, const float2* pz,
                                              float2* acc, const float2* pp) {
    if (DIPOLE && ax == 0) surf_pairs<NEAR, DIPOLE, NP, DIFF, 0>(sp, sd, cnt, px, py, pz, acc, pp);
    else if (DIPOLE && ax == 1) surf_pairs<NEAR, DIPOLE, NP, DIFF, 1>(sp, sd, cnt, px, py, pz, acc, pp);
    else if (DIPOLE && ax == 2) surf_pairs<NEAR, DIPOLE, NP, DIFF, 2>(sp, sd, cnt, px, py, pz, acc, pp);
    else surf_pairs<NEAR, DIPOLE, NP, DIFF, 3>(sp, sd, cnt, px, py, pz, acc, pp);
}

//
// A block holds the whole check potential of its box, so it also writes the box's input
// for the tensor-core projection that follows: the potential scaled by the power of two
// that puts its largest entry into [2^14, 2^15) (exponent in bexp[b]) and split into
// FP16 hi and lo terms (Qp per box, zero past Q) -- the box split done in the producer.
// DIFF: the X list of a gradient kernel -- each check potential less the sources'
// potential at the box centre (see surf_pairs), so that FP32 and the split keep the
// variation across a box far smaller than its distance to the sources.
template <bool DIPOLE, int NP, int NT, bool DIFF = false>
__global__ void __launch_bounds__(NT)
k_surf_f(const int* __restrict__ boxes, const int* __restrict__ off, const int* __restrict__ idx, int down,
         const float4* __restrict__ bcf, const int64_t* __restrict__ rng, const float* __restrict__ sxf, int64_t ns,
         const float* __restrict__ qs, const float* __restrict__ surf, int Q, int Qp, __half* __restrict__ vin_h,
         __half* __restrict__ vin_l, int* __restrict__ bexp, const int* __restrict__ bax) {
    __shared__ float4 sp[NT];
    __shared__ float4 sd[(DIPOLE || DIFF) ? NT : 1];
    const int b = boxes[blockIdx.x];
    const float4 bh = bcf[3 * b], bl = bcf[3 * b + 1], br = bcf[3 * b + 2];
    const float rf = down ? br.y : br.x;
    float2 px[NP], py[NP], pz[NP], acc[NP], pp[DIFF ? NP : 1];
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        float c[2][3];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = threadIdx.x + (2 * m + h) * NT;
            const int kk = k < Q ? k : 0;
#pragma unroll
            for (int d = 0; d < 3; ++d) c[h][d] = rf * surf[3 * kk + d];
        }
        px[m] = make_float2(c[0][0], c[1][0]);
        py[m] = make_float2(c[0][1], c[1][1]);
        pz[m] = make_float2(c[0][2], c[1][2]);
        if (DIFF) pp[m] = __ffma2_rn(pz[m], pz[m], __ffma2_rn(py[m], py[m], __fmul2_rn(px[m], px[m])));
        acc[m] = make_float2(0.f, 0.f);
    }
    const float margin = (float)(2.0 * kDelta);
    for (int e = off[blockIdx.x]; e < off[blockIdx.x + 1]; ++e) {
        const int a = idx[e];
        const int64_t sb = rng[4 * a], se = rng[4 * a + 1];
        // max-norm separation between the source cube and the check surface
        const float4 ah = bcf[3 * a], al = bcf[3 * a + 1];
        const float dm = fmaxf(fabsf((ah.x - bh.x) + (al.x - bl.x)),
                               fmaxf(fabsf((ah.y - bh.y) + (al.y - bl.y)), fabsf((ah.z - bh.z) + (al.z - bl.z))));
        const bool near = fmaxf(dm - ah.w - rf, rf - dm - ah.w) <= margin;
        // the source box's dipole axis (0..2), 3, or 4 + the axis of a box in one plane
        // (the plane form only at 2 NP <= 4 points a thread: above, its extra registers spill)
        const int ax0 = (DIPOLE && bax && se > sb) ? bax[a] : 3;
        const bool plane = DIPOLE && NP <= 2 && ax0 >= 4;
        const int ax = ax0 >= 4 && !plane ? ax0 - 4 : ax0;
        float2 dk[NP], dk2[NP], accb[NP];
        if (plane) {
            // the plane's offset from the box centre, formed as the staged sources' are
            const int k = ax - 4;
            const float c = k == 0 ? (sxf[sb] - bh.x) + (sxf[3 * ns + sb] - bl.x)
                          : k == 1 ? (sxf[ns + sb] - bh.y) + (sxf[4 * ns + sb] - bl.y)
                                   : (sxf[2 * ns + sb] - bh.z) + (sxf[5 * ns + sb] - bl.z);
#pragma unroll
            for (int m = 0; m < NP; ++m) {
                dk[m] = __fadd2_rn(k == 0 ? px[m] : (k == 1 ? py[m] : pz[m]), make_float2(-c, -c));
                dk2[m] = __fmul2_rn(dk[m], dk[m]);
                accb[m] = make_float2(0.f, 0.f);
            }
        }
        for (int64_t j0 = sb; j0 < se; j0 += NT) {
            const int64_t j = j0 + threadIdx.x;
            if (j < se) {
                sp[threadIdx.x] = make_float4((sxf[j] - bh.x) + (sxf[3 * ns + j] - bl.x),
                                              (sxf[ns + j] - bh.y) + (sxf[4 * ns + j] - bl.y),
                                              (sxf[2 * ns + j] - bh.z) + (sxf[5 * ns + j] - bl.z), qs[j]);
                if (DIPOLE) sd[threadIdx.x] = make_float4(qs[ns + j], qs[2 * ns + j], 0.f, 0.f);
                if (DIFF) {
                    const float4 y = sp[threadIdx.x];
                    const float yy = fmaf(y.z, y.z, fmaf(y.y, y.y, y.x * y.x));
                    const float ry = sqrtf(yy);
                    sd[threadIdx.x] = make_float4(1.0f / ry, ry, 0.f, 0.f);
                }
            }
            __syncthreads();
            const int cnt = (int)((se - j0) < (int64_t)NT ? (se - j0) : (int64_t)NT);
            if (plane) {
                if (near) surf_pairs_plane_k<true, NP>(ax - 4, sp, sd, cnt, px, py, pz, dk2, accb);
                else surf_pairs_plane_k<false, NP>(ax - 4, sp, sd, cnt, px, py, pz, dk2, accb);
            } else if (near) {
                surf_pairs_ax<true, DIPOLE, NP, DIFF>(ax, sp, sd, cnt, px, py, pz, acc, pp);
            } else {
                surf_pairs_ax<false, DIPOLE, NP, DIFF>(ax, sp, sd, cnt, px, py, pz, acc, pp);
            }
            __syncthreads();
        }
        if (plane) {
#pragma unroll
            for (int m = 0; m < NP; ++m) acc[m] = __ffma2_rn(accb[m], dk[m], acc[m]);
        }
    }
    // the box's largest |potential| (points past Q hold partial sums of a repeated point)
    __shared__ float s_red[NT / 32];
    float mx = 0.f;
#pragma unroll
    for (int m = 0; m < NP; ++m) {
        const int k0 = threadIdx.x + 2 * m * NT, k1 = k0 + NT;
        if (k0 < Q) mx = fmaxf(mx, fabsf(acc[m].x));
        if (k1 < Q) mx = fmaxf(mx, fabsf(acc[m].y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = s_red[0];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) mx = fmaxf(mx, s_red[w]);
    int ex = mx > 0.f ? 14 - ilogbf(mx) : 0;
    ex = max(-100, min(100, ex));
    if (threadIdx.x == 0) bexp[b] = ex;
    const float sc = __int_as_float((127 + ex) << 23);
    __half* hb = vin_h + (size_t)b * Qp;
    __half* lb = vin_l + (size_t)b * Qp;
#pragma unroll
    for (int m = 0; m < NP; ++m) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = threadIdx.x + (2 * m + h) * NT;
            if (k < Qp) {
                const float x = k < Q ? (h ? acc[m].y : acc[m].x) * sc : 0.f;
                const __half hh = __float2half_rn(x);
                hb[k] = hh;
                lb[k] = __float2half_rn(x - __half2float(hh));
            }
        }
    }
    for (int k = threadIdx.x + 2 * NP * NT; k < Qp; k += NT) {
        hb[k] = __float2half_rn(0.f);
        lb[k] = __float2half_rn(0.f);
    }
}

// Point slots of the FP32 surface kernel's shapes (NT threads x 2 NP points): the
// smallest that holds n points.  The X list keeps the 128-thread shapes.
int surf_slots(int n) {
    for (int v : {256, 384, 512, 576, 768, 1024})
        if (n <= v) return v;
    return 0;
}
int surf_slots_full(int n) { return n <= 1024 ? (n + 255) / 256 * 256 : 0; }

// Per-box FP32 table of the surface kernel: {centre hi, half-width}, {centre lo, 0},
// {up-check radius, down-check radius, 0, 0}, each rounded once from FP64.
__global__ void k_box_f(const double* __restrict__ ctr, const int* __restrict__ lvl, double root_h, int nbox,
                        float4* __restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    const double h = ldexp(root_h, -lvl[b]);
    float hi[3], lo[3];
    for (int d = 0; d < 3; ++d) {
        const double c = ctr[3 * b + d];
        hi[d] = (float)c;
        lo[d] = (float)(c - (double)hi[d]);
    }
    out[3 * b] = make_float4(hi[0], hi[1], hi[2], (float)h);
    out[3 * b + 1] = make_float4(lo[0], lo[1], lo[2], 0.f);
    out[3 * b + 2] = make_float4((float)(kUpCheck * h), (float)(kDnCheck * h), 0.f, 0.f);
}

// Sources -> check surfaces of a CSR list of boxes (S2U: leaves and themselves; X list:
// boxes and their X sources).  FP32 through k_surf_f, which writes the split input of
// the projection that follows (out unused); FP64 through k_src2surf, adding into out.
template <typename Real>
int launch_surf(const Plan& P, const Tree& T, bool dl, int nbox, const int* boxes, const int* off, const int* idx,
                double radius, const Real* q, const Real* surf, Real* out, cudaStream_t s) {
    if (nbox <= 0) return KIFMM_OK;
    if constexpr (std::is_same<Real, float>::value) {
        (void)out;
        (void)surf;
        // S2U evaluates the skeleton of the up-check surface (ks points, rows of ks);
        // the X list the whole down-check surface (Q points, rows of Qp)
        const int down = radius == kDnCheck ? 1 : 0;
        const int npts = down ? P.Q : P.ops->ks, stride = down ? P.Qp : P.ops->ks;
        const float* sf = down ? P.surf_f.p : P.ops->surf_up.p;
        const int slots = down ? surf_slots_full(P.Q) : surf_slots(npts);
        const bool diff = down && !dl && gradient_kernel(P.kernel);
        switch (slots * 2 + (dl ? 1 : 0)) {
#define KF_SURF(NP, NT)                                                                                          \
    case 2 * (2 * NP * NT):                                                                                      \
        if (diff)                                                                                                \
            k_surf_f<false, NP, NT, true><<<nbox, NT, 0, s>>>(boxes, off, idx, down, P.bcf.p, T.rng.p, P.sxf.p,  \
                                                              T.ns, q, sf, npts, stride, P.sin_h.p, P.sin_l.p,   \
                                                              P.sexp.p, nullptr);                                \
        else                                                                                                     \
            k_surf_f<false, NP, NT><<<nbox, NT, 0, s>>>(boxes, off, idx, down, P.bcf.p, T.rng.p, P.sxf.p, T.ns, q,  \
                                                        sf, npts, stride, P.sin_h.p, P.sin_l.p, P.sexp.p, nullptr); \
        break;                                                                                                   \
    case 2 * (2 * NP * NT) + 1:                                                                                  \
        k_surf_f<true, NP, NT><<<nbox, NT, 0, s>>>(boxes, off, idx, down, P.bcf.p, T.rng.p, P.sxf.p, T.ns, q, sf,    \
                                                   npts, stride, P.sin_h.p, P.sin_l.p, P.sexp.p, P.bax.p);       \
        break;
            KF_SURF(1, 128) KF_SURF(2, 96) KF_SURF(2, 128) KF_SURF(3, 96) KF_SURF(3, 128) KF_SURF(4, 128)
#undef KF_SURF
            default:
                set_error("check surface of %d points exceeds the FP32 surface kernel", npts);
                return KIFMM_ERR_UNSUPPORTED;
        }
    } else {
        if (dl)
            k_src2surf<Real, true><<<nbox, kSurfThreads, 0, s>>>(boxes, off, idx, radius, T.lvl.p, T.ctr.p, T.root_h,
                                                                 T.rng.p, T.sxyz.p, T.ns, q, surf, P.Q, P.Qp, out);
        else
            k_src2surf<Real, false><<<nbox, kSurfThreads, 0, s>>>(boxes, off, idx, radius, T.lvl.p, T.ctr.p,
                                                                  T.root_h, T.rng.p, T.sxyz.p, T.ns, q, surf, P.Q,
                                                                  P.Qp, out);
    }
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

// ---------------------------------------------------------------- grouped pair GEMM (U2U, M2L, L2L)
// Every tile shares one operator: out[pout[j]] += Op . in[pin[j]] for its pairs.
// CUDA-core SGEMM/DGEMM blocking: 64 rows x 64 pairs per pass, 4x4 per thread.
template <typename Real>
__device__ __forceinline__ void pair_gemm_body(const Real* __restrict__ ops, int Q, int Qp,
                                               const int4* __restrict__ tiles, const int* __restrict__ pin,
                                               const int* __restrict__ pout, const Real* __restrict__ in,
                                               Real* __restrict__ out) {
    constexpr int BM = 64, BN = kPairTile, BK = 16;
    __shared__ Real As[BK][BM + 4];
    __shared__ Real Bs[BK][BN + 4];
    __shared__ int s_in[BN], s_out[BN];
    int4 t = tiles[blockIdx.x];
    const Real* Op = ops + (size_t)t.x * Qp * Qp;
    int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    for (int jb = 0; jb < t.z; jb += BN) {  // tiles may hold several blocks of BN pairs
    const int cnt = t.z - jb;
    __syncthreads();
    for (int j = threadIdx.x; j < BN; j += blockDim.x) {
        s_in[j] = j < cnt ? pin[t.y + jb + j] : -1;
        s_out[j] = j < cnt ? pout[t.y + jb + j] : -1;
    }
    __syncthreads();
    for (int row0 = 0; row0 < Q; row0 += BM) {
        Real acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0;
        for (int k0 = 0; k0 < Qp; k0 += BK) {
            for (int e = threadIdx.x; e < BM * BK; e += blockDim.x) {
                int r = e / BK, kk = e % BK;
                int row = row0 + r;
                As[kk][r] = row < Qp ? Op[(size_t)row * Qp + k0 + kk] : (Real)0;
            }
            for (int e = threadIdx.x; e < BN * BK; e += blockDim.x) {
                int j = e / BK, kk = e % BK;
                int bi = s_in[j];
                Bs[kk][j] = bi >= 0 ? in[(size_t)bi * Qp + k0 + kk] : (Real)0;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                Real a[4], bv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bv[j];
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int row = row0 + ty * 4 + i;
            if (row >= Q) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int ob = s_out[tx * 4 + j];
                if (ob >= 0) atomicAdd(&out[(size_t)ob * Qp + row], acc[i][j]);
            }
        }
    }
    }
}

// One kernel name per translation so profiles tell them apart.
#define KF_PAIR_KERNEL(NAME)                                                                              \
    template <typename Real>                                                                              \
    __global__ void __launch_bounds__(256)                                                               \
        NAME(const Real* __restrict__ ops, int Q, int Qp, const int4* __restrict__ tiles,                \
             const int* __restrict__ pin, const int* __restrict__ pout, const Real* __restrict__ in,     \
             Real* __restrict__ out) {                                                                    \
        pair_gemm_body<Real>(ops, Q, Qp, tiles, pin, pout, in, out);                                      \
    }
KF_PAIR_KERNEL(k_u2u_gemm)
KF_PAIR_KERNEL(k_m2l_gemm)
KF_PAIR_KERNEL(k_l2l_gemm)
#undef KF_PAIR_KERNEL

// ---------------------------------------------------------------- mean removal (ADL)
// The adjoint double layer needs only the gradient of the far field.  A constant
// potential has none, so each box's down-check potential is shifted to zero mean
// before it is passed on; otherwise the large constant carried down from coarse
// levels would be stored in FP32 and its rounding amplified by 2^level when the
// leaf rows differentiate it.
template <typename Real>
__global__ void __launch_bounds__(128) k_center(int box0, int Q, int Qp, Real* __restrict__ d) {
    __shared__ double red[128];
    Real* v = d + (size_t)(box0 + blockIdx.x) * Qp;
    double s = 0;
    for (int k = threadIdx.x; k < Q; k += blockDim.x) s += (double)v[k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    Real mean = (Real)(red[0] / Q);
    for (int k = threadIdx.x; k < Q; k += blockDim.x) v[k] -= mean;
}

// ---------------------------------------------------------------- D2T
// res[t] = T[t] . d[leaf(t)]: one block per target leaf, one warp per target row.
template <typename Real>
__global__ void __launch_bounds__(128)
k_d2t(const int* __restrict__ leaves, const int64_t* __restrict__ rng, const Real* __restrict__ T,
      const Real* __restrict__ d, int Qp, Real* __restrict__ res) {
    extern __shared__ unsigned char smem_raw[];
    Real* ds = reinterpret_cast<Real*>(smem_raw);
    int b = leaves[blockIdx.x];
    for (int k = threadIdx.x; k < Qp; k += blockDim.x) ds[k] = d[(size_t)b * Qp + k];
    __syncthreads();
    int64_t tb = rng[4 * b + 2], te = rng[4 * b + 3];
    int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if constexpr (std::is_same<Real, float>::value) {
        // FP32 rows (Qp a multiple of 16): 16-byte streaming loads, read once
        const float4* ds4 = reinterpret_cast<const float4*>(ds);
        for (int64_t t = tb + warp; t < te; t += blockDim.x / 32) {
            const float4* row = reinterpret_cast<const float4*>(T + (size_t)t * Qp);
            float s = 0.f;
#pragma unroll 2
            for (int k = lane; k < Qp / 4; k += 32) {
                const float4 a = __ldcs(row + k), c = ds4[k];
                s = fmaf(a.x, c.x, fmaf(a.y, c.y, fmaf(a.z, c.z, fmaf(a.w, c.w, s))));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) res[t] = s;
        }
    } else {
        for (int64_t t = tb + warp; t < te; t += blockDim.x / 32) {
            const Real* row = T + (size_t)t * Qp;
            Real s = 0;
            for (int k = lane; k < Qp; k += 32) s += row[k] * ds[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) res[t] = s;
        }
    }
}

// ---------------------------------------------------------------- P2P (U and W lists) + scatter
// One block per target leaf, one thread per target; source boxes staged in shared
// memory relative to the target leaf's centre.
// KIND 0: q/r   1: (q n_j).(x - y)/r^3   2: q n_i.(x - y)/r^3   3: q (x - y)/r^3 (three
// components, written to out[tperm[t] + c nt] with the far field res[t + c nt])
template <typename Real, int KIND>
__global__ void k_p2p(const int* __restrict__ leaves, const int* __restrict__ off, const int* __restrict__ idx,
                      const int64_t* __restrict__ rng, const double* __restrict__ ctr,
                      const double* __restrict__ sxyz, int64_t ns, const double* __restrict__ txyz,
                      int64_t nt, const Real* __restrict__ qs, const Real* __restrict__ tnrm,
                      const Real* __restrict__ res, const int64_t* __restrict__ tperm,
                      double* __restrict__ out) {
    extern __shared__ unsigned char smem_raw[];
    Real* sx = reinterpret_cast<Real*>(smem_raw);
    Real* sy = sx + blockDim.x;
    Real* sz = sy + blockDim.x;
    Real* s0 = sz + blockDim.x;
    Real* s1 = s0 + blockDim.x;
    Real* s2 = s1 + blockDim.x;
    int b = leaves[blockIdx.x];
    double cx = ctr[3 * b], cy = ctr[3 * b + 1], cz = ctr[3 * b + 2];
    int64_t tb = rng[4 * b + 2], te = rng[4 * b + 3];
    const Real d2 = (Real)(kDelta * kDelta);
    for (int64_t t0 = tb; t0 < te; t0 += blockDim.x) {
        int64_t t = t0 + threadIdx.x;
        bool valid = t < te;
        int64_t tt = valid ? t : tb;
        Real xt = (Real)(txyz[tt] - cx), yt = (Real)(txyz[nt + tt] - cy), zt = (Real)(txyz[2 * nt + tt] - cz);
        Real nx = 0, ny = 0, nz = 0;
        if (KIND == 2) {
            nx = tnrm[tt];
            ny = tnrm[nt + tt];
            nz = tnrm[2 * nt + tt];
        }
        Real acc = 0, acc2 = 0, acc3 = 0;
        for (int e = off[blockIdx.x]; e < off[blockIdx.x + 1]; ++e) {
            int a = idx[e];
            int64_t sb = rng[4 * a], se = rng[4 * a + 1];
            for (int64_t j0 = sb; j0 < se; j0 += blockDim.x) {
                int64_t j = j0 + threadIdx.x;
                if (j < se) {
                    sx[threadIdx.x] = (Real)(sxyz[j] - cx);
                    sy[threadIdx.x] = (Real)(sxyz[ns + j] - cy);
                    sz[threadIdx.x] = (Real)(sxyz[2 * ns + j] - cz);
                    s0[threadIdx.x] = qs[j];
                    if (KIND == 1) {
                        s1[threadIdx.x] = qs[ns + j];
                        s2[threadIdx.x] = qs[2 * ns + j];
                    }
                }
                __syncthreads();
                int cnt = (int)((se - j0) < (int64_t)blockDim.x ? (se - j0) : (int64_t)blockDim.x);
                for (int jj = 0; jj < cnt; ++jj) {
                    Real dx = xt - sx[jj], dy = yt - sy[jj], dz = zt - sz[jj];
                    Real r2 = dx * dx + dy * dy + dz * dz;
                    Real inv = RT<Real>::rsq(r2);
                    Real v;
                    if (KIND == 3) {
                        const Real w = (r2 >= d2) ? s0[jj] * (inv * inv * inv) : (Real)0;
                        acc += w * dx;
                        acc2 += w * dy;
                        acc3 += w * dz;
                        continue;
                    }
                    if (KIND == 0) v = s0[jj] * inv;
                    else if (KIND == 1) v = (s0[jj] * dx + s1[jj] * dy + s2[jj] * dz) * (inv * inv * inv);
                    else v = s0[jj] * (nx * dx + ny * dy + nz * dz) * (inv * inv * inv);
                    acc += (r2 >= d2) ? v : (Real)0;
                }
                __syncthreads();
            }
        }
        if (valid) {
            out[tperm[t]] = (double)(acc + res[t]);
            if (KIND == 3) {
                out[tperm[t] + nt] = (double)(acc2 + res[t + nt]);
                out[tperm[t] + 2 * nt] = (double)(acc3 + res[t + 2 * nt]);
            }
        }
    }
}

// FP32 near field (mixed form), one warp per work unit.  A unit is at most kP2PUnitSrc
// sources of one target leaf (pieces of its U-, W- and X-list source ranges); units run
// heaviest first, and a leaf spread over several units adds into its zeroed outputs
// with FP64 atomics (the first unit also adds the far field).  Lanes form 4 source
// groups of 8: lane (g, r) holds targets t0 + 8 i + r (i < T) of the current pass of
// at most 8 T targets, packed in pairs so that every step is one FP32x2 instruction for
// two pair evaluations, and takes sources g, g + 4, ... of each chunk of 32; the four
// partial sums of a target meet by shuffles at the end.
//
// Chunks are double-buffered: while one chunk is evaluated, cp.async copies the next
// chunk's raw source data (FP32 hi/lo coordinates and densities or dipoles) into shared
// memory; each lane then turns its source into the staged form the pair loop reads by
// shared-memory broadcast, every value already duplicated as a float2 pair.
//
// Accuracy (Sec. III.A.1 asks for the discrete sum; these are the steps that keep the
// FP32 evaluation at the single layer's accuracy for all three kernels):
//  - Offsets are taken from the leaf centre.  Each range has an exponent E with every
//    coordinate offset of the leaf's targets and the range's sources below 2^E (from
//    the boxes' extents).  For the double layers an offset is split as hi + lo, hi on the
//    grid g = 2^(E-10) (11 significant bits), lo the FP32 remainder; normals (ADL) and
//    dipoles q n_j (DL) likewise, on the grid 2^-10 or 2^(k-10) with 2^k above the
//    dipole's largest component.  Products of two hi parts have at most 22 significant
//    bits on a common grid, so the sums n_hi . t_hi - n_hi . s_hi (ADL) and
//    m_hi . t_hi - m_hi . s_hi (DL) are exact in FP32.  The rest, m_hi . (t_lo - s_lo) +
//    m_lo . (t - s) with the full FP32 offsets t and s in the second product (the lo
//    parts of close points are not small next to their separation), is 2^-10 smaller
//    and carries FP32 rounding only.  On a curved surface n . (x - y) between neighbours
//    is about |x - y|^2 / 2R, and this is what keeps it from cancellation.  A unit's
//    ranges are ordered by E and the targets split once per exponent.
//  - The tolerance radius (pair skipped when r^2 < 1e-10) is tested only on ranges
//    flagged kRangeExcl at set-up, which an FP64 scan found to hold a pair within 4
//    delta (the leaf's own range always does: each target is among its sources).
//  - r^2 from FP32 offsets is good to 2^-24 of the offsets, not of the separation.
//    Ranges flagged kRangeCorr (by the same scan: a pair closer than 2^(E-5) -- a target
//    close to a source relative to the boxes, such as a volume target near the surface
//    -- or between delta/2 and 4 delta) are skipped here and evaluated by a second launch
//    of this kernel, CORR, one range per unit, which adds to each difference of FP32
//    offsets the difference of their exact rounding errors (t - s = (tf - sf) + (te - se),
//    the first term exact for close points).  Coincident points (closer than delta/2: a
//    target among its own sources) are excluded in either launch.
constexpr int kP2PWarps = 8;
// range flags, in the start index's high bits: a pair may lie within 4 delta (test the
// tolerance radius); a pair is close (the corrected-distance launch); the range's offset
// exponent E + 128 (bits 48..55)
constexpr long long kRangeExcl = 1LL << 62;
constexpr long long kRangeCorr = 1LL << 61;
constexpr long long kRangeIdx = (1LL << 48) - 1;
// a range takes the corrected distance when a pair lies closer than 2^(Er - kCloseBits)
constexpr int kCloseBits = 5;
__host__ __device__ inline int range_exp(long long fl) { return (int)((fl >> 48) & 255) - 128; }
constexpr int kP2PUnitSrc = 2048;
// Larger target leaves of the single layer and the field go to the block kernel (a
// thread per target, sources staged once per leaf): at leaf 128 on the 64-sphere pack it
// takes 2.56 ms against 4.04 ms for two 64-target passes of the warp kernel.  The double
// layers always take the warp kernel, in passes, for its exact products.
constexpr int kP2PWarpMaxLeaf = 64;
// unit flags (int4 .w): bit 0 the leaf's first unit, bit 1 the leaf spans several units;
// bits 8..9 the dipoles' axis of a KIND 4 unit; bits 16..30 one plus the unit's one pass
// of 8 kMaxT targets, or 0 for all of the leaf's targets (the passes of a leaf share no
// targets, so they are dealt to separate warps: each pass walks all of its sources anyway)
constexpr int kUnitFirst = 1, kUnitSplit = 2, kUnitPassShift = 16;

// targets per lane per pass (plain and corrected-distance launches) and float4 entries
// staged per source, by kernel: as many targets as keep each kernel within 128
// registers, so two blocks share an SM
template <int KIND> struct NearShape;
template <> struct NearShape<0> { static constexpr int kMaxT = 8, kMaxTCorr = 6, kStage = 4, kRaw = 7; };
template <> struct NearShape<1> { static constexpr int kMaxT = 4, kMaxTCorr = 4, kStage = 7, kRaw = 12; };
template <> struct NearShape<2> { static constexpr int kMaxT = 4, kMaxTCorr = 2, kStage = 7, kRaw = 7; };
template <> struct NearShape<3> { static constexpr int kMaxT = 8, kMaxTCorr = 6, kStage = 4, kRaw = 7; };
// 4: the double layer on a unit whose dipoles all lie along one coordinate axis (flat
// faces normal to an axis): n . (x - y) has one term, no cancellation between terms
template <> struct NearShape<4> { static constexpr int kMaxT = 8, kMaxTCorr = 1, kStage = 2, kRaw = 9; };

__device__ __forceinline__ float2 lo2(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(float4 a) { return make_float2(a.z, a.w); }
// 2^k as a float (k in [-126, 127])
__device__ __forceinline__ float exp2i(int k) { return __int_as_float((k + 127) << 23); }
// x rounded to the grid of quantum g (|x| < 2^22 g), by adding and removing
// magic = 1.5 * 2^23 * g
__device__ __forceinline__ float grid_round(float x, float magic) { return __fsub_rn(__fadd_rn(x, magic), magic); }

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// A source's offset from the leaf centre, from FP32 hi/lo coordinates (ph, pl) and the
// centre's (ch, cl): a + rest with a = fl(ph - ch) and rest its error plus pl - cl.
__device__ __forceinline__ void src_offset(float ph, float pl, float ch, float cl, float& a, float& rest) {
    a = __fsub_rn(ph, ch);
    const float bb = __fsub_rn(a, ph);
    const float err = __fadd_rn(__fsub_rn(ph, __fsub_rn(a, bb)), __fsub_rn(-ch, bb));
    rest = __fadd_rn(__fsub_rn(pl, cl), err);
}

// One point's offset from the leaf centre in the forms the pair loop uses: full FP32
// offset f, its exact rounding error e (f + e = the offset to FP32^2 accuracy) and, for
// the double layers, the split hi (on the grid of magic) + lo with f = fl(hi + lo).
template <bool SPLIT>
__device__ __forceinline__ void offset_forms(float a, float rest, float magic, float& f, float& e, float& hi,
                                             float& lo) {
    if (SPLIT) {
        hi = grid_round(a, magic);
        lo = __fadd_rn(__fsub_rn(a, hi), rest);
        f = __fadd_rn(hi, lo);
        e = __fsub_rn(lo, __fsub_rn(f, hi));          // exact: |hi| >= |lo| or hi = 0
    } else {
        f = __fadd_rn(a, rest);                       // two-sum of a and rest
        const float bb = __fsub_rn(f, a);
        e = __fadd_rn(__fsub_rn(a, __fsub_rn(f, bb)), __fsub_rn(rest, bb));
        hi = f;
        lo = 0.f;
    }
}

template <int KIND, int T, bool CORR>
__device__ __forceinline__ void p2p_pass(int lane, int e0, int e1, const longlong2* __restrict__ ranges, int flags,
                                         float4 cb0, float4 cb1, const float* __restrict__ sxf, int64_t ns,
                                         const float* __restrict__ txf, int64_t nt, const float* __restrict__ qs,
                                         const float* __restrict__ tnrm_f, const float* __restrict__ res,
                                         const int64_t* __restrict__ tperm, double* __restrict__ out, int64_t t0,
                                         int64_t te, float4* __restrict__ st, float* __restrict__ raw) {
    using S = NearShape<KIND>;
    constexpr int TP = (T + 1) / 2;
    constexpr bool ACC = KIND == 1 || KIND == 2;     // double layers: exact hi products
    constexpr int NC = KIND == 3 ? 3 : 1;            // output components
    const int g = lane >> 3, r = lane & 7;
    const float chx = cb0.x, chy = cb0.y, chz = cb0.z, clx = cb1.x, cly = cb1.y, clz = cb1.z;
    const float d2 = (float)(kDelta * kDelta);
    const int axis = (flags >> 8) & 3;                   // KIND 4: the dipoles' axis, made the third
                                                         // coordinate of targets and sources

    // targets: offsets from the leaf centre, formed from FP32 hi/lo coordinates exactly as
    // the sources' below (a target and the same point as a source agree bit for bit), and
    // for the double layers split on the grid of the current range's exponent
    float2 tfx[TP], tfy[TP], tfz[TP], acc[TP], acc2[NC > 1 ? TP : 1], acc3[NC > 1 ? TP : 1];
    float2 thx[ACC ? TP : 1], thy[ACC ? TP : 1], thz[ACC ? TP : 1];   // DL: t hi;  ADL: n hi
    float2 tlx[ACC ? TP : 1], tly[ACC ? TP : 1], tlz[ACC ? TP : 1];   // DL: t lo;  ADL: -n lo
    float2 tca[KIND == 2 ? TP : 1], tcb[KIND == 2 ? TP : 1];          // ADL: -n_hi.t_hi, -(n_hi.t_lo + n_lo.t)
    float2 tex[CORR ? TP : 1], tey[CORR ? TP : 1], tez[CORR ? TP : 1]; // rounding errors of tf
    auto split_targets = [&](float magic) {
#pragma unroll
        for (int m = 0; m < TP; ++m) {
            float c[2][14];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int64_t t = t0 + 8 * (2 * m + h) + r;
                t = t < te ? t : t0;              // padding slots evaluate a real target, unused
                float a[3], rest[3], th[3], tl[3];
                src_offset(txf[t], txf[3 * nt + t], chx, clx, a[0], rest[0]);
                src_offset(txf[nt + t], txf[4 * nt + t], chy, cly, a[1], rest[1]);
                src_offset(txf[2 * nt + t], txf[5 * nt + t], chz, clz, a[2], rest[2]);
#pragma unroll
                for (int d = 0; d < 3; ++d) offset_forms<ACC>(a[d], rest[d], magic, c[h][d], c[h][11 + d], th[d], tl[d]);
                if (KIND == 4) {
                    const float ck = axis == 0 ? c[h][0] : (axis == 1 ? c[h][1] : c[h][2]);
                    if (axis == 0) c[h][0] = c[h][2];
                    else if (axis == 1) c[h][1] = c[h][2];
                    c[h][2] = ck;
                }
                if (KIND == 1) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        c[h][3 + d] = th[d];
                        c[h][6 + d] = tl[d];
                    }
                } else if (KIND == 2) {
                    // the normal on the grid 2^-10 (magic 1.5 * 2^13) and its remainder
                    float nh[3], nl[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        nh[d] = grid_round(tnrm_f[d * nt + t], 12288.0f);
                        nl[d] = __fadd_rn(__fsub_rn(tnrm_f[d * nt + t], nh[d]), tnrm_f[(3 + d) * nt + t]);
                        c[h][3 + d] = nh[d];
                        c[h][6 + d] = -nl[d];
                    }
                    // n_hi . t_hi exact (22-bit products on one grid); n_hi . t_lo + n_lo . t
                    c[h][9] = -__fmaf_rn(nh[2], th[2], __fmaf_rn(nh[1], th[1], __fmul_rn(nh[0], th[0])));
                    c[h][10] = -__fmaf_rn(nl[2], c[h][2], __fmaf_rn(nl[1], c[h][1], __fmaf_rn(nl[0], c[h][0],
                               __fmaf_rn(nh[2], tl[2], __fmaf_rn(nh[1], tl[1], __fmul_rn(nh[0], tl[0]))))));
                }
            }
            tfx[m] = make_float2(c[0][0], c[1][0]);
            tfy[m] = make_float2(c[0][1], c[1][1]);
            tfz[m] = make_float2(c[0][2], c[1][2]);
            if (ACC) {
                thx[m] = make_float2(c[0][3], c[1][3]);
                thy[m] = make_float2(c[0][4], c[1][4]);
                thz[m] = make_float2(c[0][5], c[1][5]);
                tlx[m] = make_float2(c[0][6], c[1][6]);
                tly[m] = make_float2(c[0][7], c[1][7]);
                tlz[m] = make_float2(c[0][8], c[1][8]);
            }
            if (KIND == 2) {
                tca[m] = make_float2(c[0][9], c[1][9]);
                tcb[m] = make_float2(c[0][10], c[1][10]);
            }
            if (CORR) {
                tex[m] = make_float2(c[0][11], c[1][11]);
                tey[m] = make_float2(c[0][12], c[1][12]);
                tez[m] = make_float2(c[0][13], c[1][13]);
            }
        }
    };
#pragma unroll
    for (int m = 0; m < TP; ++m) {
        acc[m] = make_float2(0.f, 0.f);
        if (NC > 1) acc2[m] = acc3[m] = make_float2(0.f, 0.f);
    }
    if (!ACC) split_targets(0.f);

    // raw rows per source: hi x|y|z, lo x|y|z, then q (SL, ADL, field) or q n_j hi x|y|z
    // and lo x|y|z (DL)
    auto issue = [&](int64_t j, int buf) {
        if (j >= 0) {
            float* rw = raw + buf * (S::kRaw * 32) + lane;
#pragma unroll
            for (int d = 0; d < 6; ++d) cp_async4(rw + 32 * d, sxf + d * ns + j);
#pragma unroll
            for (int d = 0; d < S::kRaw - 6; ++d) cp_async4(rw + 32 * (6 + d), qs + d * ns + j);
        }
        cp_async_commit();
    };

    // groups of ranges with one exponent (the unit's ranges are ordered by it); the double
    // layers split their targets for each group's grid
    for (int gb = e0; gb < e1;) {
        const int E = range_exp(ranges[gb].x);
        int ge = gb + 1;
        if (ACC)
            while (ge < e1 && range_exp(ranges[ge].x) == E) ++ge;
        else
            ge = e1;
        const float magic = 1.5f * exp2i(E + 13);        // rounds to the grid 2^(E-10)
        if (ACC) split_targets(magic);
        // Chunks of 32 sources run across the group's ranges (a leaf's neighbour boxes hold
        // a few dozen sources each), skipping the ranges of the other launch (the
        // corrected-distance ranges are the CORR instance's, and only its).  take() walks
        // the warp-uniform position (e, j0) past the next chunk; each lane gets its source
        // j (-1: none) and whether its range needs the tolerance-radius select.
        int e = gb;
        int64_t j0 = ranges[e].x & kRangeIdx, se = ranges[e].y;
        long long fl = ranges[e].x & ~kRangeIdx;
        auto take = [&](int64_t& j, bool& ex) -> int {
            j = -1;
            ex = false;
            int got = 0;
            while (e < ge && got < 32) {
                const bool mine = ((fl & kRangeCorr) != 0) == CORR;
                if (mine && j0 < se) {
                    const int n = (int)(se - j0 < 32 - got ? se - j0 : 32 - got);
                    if (lane >= got && lane < got + n) {
                        j = j0 + (lane - got);
                        ex = (fl & kRangeExcl) != 0;
                    }
                    got += n;
                    j0 += n;
                }
                if ((!mine || j0 >= se) && ++e < ge) {
                    j0 = ranges[e].x & kRangeIdx;
                    se = ranges[e].y;
                    fl = ranges[e].x & ~kRangeIdx;
                }
            }
            return got;
        };
        int64_t jn;
        bool exn;
        int cnt = take(jn, exn);
        bool excl = __any_sync(0xffffffffu, exn);
        if (cnt > 0) issue(jn, 0);
        int buf = 0;
        while (cnt > 0) {
            // the next chunk, whose copy overlaps this one's evaluation
            const int ncnt = take(jn, exn);
            const bool nexcl = __any_sync(0xffffffffu, exn);
            if (ncnt > 0) {
                issue(jn, buf ^ 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncwarp();
            // stage this lane's source of the chunk
            if (lane < cnt) {
                const float* rw = raw + buf * (S::kRaw * 32) + lane;
                float a[3], rest[3], sf[3], se_[3], sh[3], sl[3];
                src_offset(rw[0], rw[96], chx, clx, a[0], rest[0]);
                src_offset(rw[32], rw[128], chy, cly, a[1], rest[1]);
                src_offset(rw[64], rw[160], chz, clz, a[2], rest[2]);
    #pragma unroll
                for (int d = 0; d < 3; ++d) offset_forms<ACC>(a[d], rest[d], magic, sf[d], se_[d], sh[d], sl[d]);
                if (KIND == 4) {
                    const float sk = axis == 0 ? sf[0] : (axis == 1 ? sf[1] : sf[2]);
                    if (axis == 0) sf[0] = sf[2];
                    else if (axis == 1) sf[1] = sf[2];
                    sf[2] = sk;
                }
                st[lane] = make_float4(-sf[0], -sf[0], -sf[1], -sf[1]);
                if (KIND == 4) {
                    const float mk = axis == 0 ? rw[192] : (axis == 1 ? rw[224] : rw[256]);
                    st[32 + lane] = make_float4(-sf[2], -sf[2], mk, mk);
                } else if (KIND == 0 || KIND == 3) {
                    const float q = rw[192];
                    st[32 + lane] = make_float4(-sf[2], -sf[2], q, q);
                    if (CORR) {
                        st[64 + lane] = make_float4(-se_[0], -se_[0], -se_[1], -se_[1]);
                        st[96 + lane] = make_float4(-se_[2], -se_[2], 0.f, 0.f);
                    }
                } else if (KIND == 1) {
                    const float mf[3] = {rw[192], rw[224], rw[256]}, ml[3] = {rw[288], rw[320], rw[352]};
                    const float mmax = fmaxf(fabsf(mf[0]), fmaxf(fabsf(mf[1]), fabsf(mf[2])));
                    // 2^k > mmax; k clamped so that the magic number stays a normal float
                    int k = ((__float_as_int(mmax) >> 23) & 255) - 126;
                    k = max(-120, min(k, 110));
                    const float mmag = 1.5f * exp2i(k + 13);
                    float mh[3], mlo[3];
    #pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        mh[d] = grid_round(mf[d], mmag);
                        mlo[d] = __fadd_rn(__fsub_rn(mf[d], mh[d]), ml[d]);
                    }
                    // a_j = m_hi . s_hi (exact), b_j = m_hi . s_lo + m_lo . s
                    const float aj = __fmaf_rn(mh[2], sh[2], __fmaf_rn(mh[1], sh[1], __fmul_rn(mh[0], sh[0])));
                    const float bj = __fmaf_rn(mlo[2], sf[2], __fmaf_rn(mlo[1], sf[1], __fmaf_rn(mlo[0], sf[0],
                                     __fmaf_rn(mh[2], sl[2], __fmaf_rn(mh[1], sl[1], __fmul_rn(mh[0], sl[0]))))));
                    st[32 + lane] = make_float4(-sf[2], -sf[2], -aj, -aj);
                    st[64 + lane] = make_float4(mh[0], mh[0], mh[1], mh[1]);
                    st[96 + lane] = make_float4(mh[2], mh[2], -bj, -bj);
                    st[128 + lane] = make_float4(mlo[0], mlo[0], mlo[1], mlo[1]);
                    st[160 + lane] = make_float4(mlo[2], mlo[2], -se_[0], -se_[0]);
                    if (CORR) st[192 + lane] = make_float4(-se_[1], -se_[1], -se_[2], -se_[2]);
                } else {
                    const float q = rw[192];
                    st[32 + lane] = make_float4(-sf[2], -sf[2], q, q);
                    st[64 + lane] = make_float4(sh[0], sh[0], sh[1], sh[1]);
                    st[96 + lane] = make_float4(sh[2], sh[2], sl[0], sl[0]);
                    st[128 + lane] = make_float4(sl[1], sl[1], sl[2], sl[2]);
                    if (CORR) {
                        st[160 + lane] = make_float4(-se_[0], -se_[0], -se_[1], -se_[1]);
                        st[192 + lane] = make_float4(-se_[2], -se_[2], 0.f, 0.f);
                    }
                }
            }
            __syncwarp();
            constexpr int kJJ = (KIND == 1 && CORR) ? 1 : 2;   // two sources in flight; the DL corrected launch would spill
    #pragma unroll kJJ
            for (int jj = g; jj < cnt; jj += 4) {
                const float4 A = st[jj], B = st[32 + jj];
                float4 C, D, F, G, H;
                if (KIND == 1 || KIND == 2) {
                    C = st[64 + jj];
                    D = st[96 + jj];
                    F = st[128 + jj];
                }
                if (KIND == 1) G = st[160 + jj];
                // the sources' rounding errors -e (CORR): x in ex.x, y in ey.x, z in ez.x
                float2 ex, ey, ez;
                if (CORR) {
                    if (KIND == 0 || KIND == 3) {
                        C = st[64 + jj];
                        D = st[96 + jj];
                        ex = lo2(C), ey = hi2(C), ez = lo2(D);
                    } else if (KIND == 1) {
                        H = st[192 + jj];
                        ex = hi2(G), ey = lo2(H), ez = hi2(H);
                    } else {
                        G = st[160 + jj];
                        H = st[192 + jj];
                        ex = lo2(G), ey = hi2(G), ez = lo2(H);
                    }
                }
    #pragma unroll
                for (int m = 0; m < TP; ++m) {
                    float2 dx = __fadd2_rn(tfx[m], lo2(A)), dy = __fadd2_rn(tfy[m], hi2(A)),
                           dz = __fadd2_rn(tfz[m], lo2(B));
                    if (CORR) {
                        // t - s = (tf - sf) + (te - se): the first difference is exact for close
                        // points, the second carries what FP32 offsets dropped
                        dx = __fadd2_rn(dx, __fadd2_rn(tex[m], ex));
                        dy = __fadd2_rn(dy, __fadd2_rn(tey[m], ey));
                        dz = __fadd2_rn(dz, __fadd2_rn(tez[m], ez));
                    }
                    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                    float2 w = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
                    float2 num;
                    if (KIND == 3) {
                        // q (t - s) / r^3, three components
                        float2 w3 = __fmul2_rn(__fmul2_rn(w, w), __fmul2_rn(w, hi2(B)));
                        if (excl) {
                            w3.x = r2.x >= d2 ? w3.x : 0.f;
                            w3.y = r2.y >= d2 ? w3.y : 0.f;
                        }
                        acc[m] = __ffma2_rn(dx, w3, acc[m]);
                        acc2[m] = __ffma2_rn(dy, w3, acc2[m]);
                        acc3[m] = __ffma2_rn(dz, w3, acc3[m]);
                        continue;
                    }
                    if (KIND == 0) {
                        num = hi2(B);                                         // q
                    } else if (KIND == 4) {
                        w = __fmul2_rn(__fmul2_rn(w, w), w);                  // 1/r^3
                        num = __fmul2_rn(hi2(B), dz);                         // m_k (t - s)_k
                    } else if (KIND == 1) {
                        w = __fmul2_rn(__fmul2_rn(w, w), w);                  // 1/r^3
                        // m_hi . t_hi - a_j (exact) + m_hi . t_lo + m_lo . t - b_j
                        const float2 nh = __ffma2_rn(lo2(D), thz[m], __ffma2_rn(hi2(C), thy[m],
                                          __ffma2_rn(lo2(C), thx[m], hi2(B))));
                        const float2 cr = __ffma2_rn(lo2(G), tfz[m], __ffma2_rn(hi2(F), tfy[m], __ffma2_rn(lo2(F), tfx[m],
                                          __ffma2_rn(lo2(D), tlz[m], __ffma2_rn(hi2(C), tly[m],
                                          __ffma2_rn(lo2(C), tlx[m], hi2(D)))))));
                        num = __fadd2_rn(nh, cr);
                    } else {
                        w = __fmul2_rn(hi2(B), __fmul2_rn(__fmul2_rn(w, w), w));   // q/r^3
                        // n_hi . s_hi - n_hi . t_hi (exact) + n_hi . s_lo + n_lo . s - b_i = -n . d
                        // (the staged -s times the stored -n_lo)
                        const float2 nh = __ffma2_rn(lo2(D), thz[m], __ffma2_rn(hi2(C), thy[m],
                                          __ffma2_rn(lo2(C), thx[m], tca[m])));
                        const float2 cr = __ffma2_rn(lo2(B), tlz[m], __ffma2_rn(hi2(A), tly[m], __ffma2_rn(lo2(A), tlx[m],
                                          __ffma2_rn(hi2(F), thz[m], __ffma2_rn(lo2(F), thy[m],
                                          __ffma2_rn(hi2(D), thx[m], tcb[m]))))));
                        num = __fadd2_rn(nh, cr);
                    }
                    if (excl) {
                        w.x = r2.x >= d2 ? w.x : 0.f;
                        w.y = r2.y >= d2 ? w.y : 0.f;
                    }
                    acc[m] = __ffma2_rn(num, w, acc[m]);
                }
            }
            __syncwarp();
            buf ^= 1;
            cnt = ncnt;
            excl = nexcl;
        }
        gb = ge;
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
#pragma unroll
        for (int i = 0; i < T; ++i) {
            const float2 a = c == 0 ? acc[i >> 1] : (c == 1 ? acc2[i >> 1] : acc3[i >> 1]);
            float v = (i & 1) ? a.y : a.x;
            v += __shfl_xor_sync(0xffffffffu, v, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 16);
            if (KIND == 2) v = -v;
            const int64_t t = t0 + 8 * i + r;
            if (g == 0 && t < te) {
                // res (the far field) is added here, or later by the caller when null; the
                // corrected-range launch only adds its share
                const float far = (res && !CORR) ? res[t + c * nt] : 0.f;
                double* o = out + tperm[t] + c * nt;
                if (CORR) atomicAdd(o, (double)v);
                else if (!(flags & kUnitSplit)) *o = (double)(v + far);                   // the leaf's only unit
                else atomicAdd(o, (double)((flags & kUnitFirst) ? v + far : v));         // one of several
            }
        }
    }
}

template <int KIND, bool CORR>
__global__ void __launch_bounds__(32 * kP2PWarps, 2)
k_p2p_warp(const int* __restrict__ leaves, int nunits, const int4* __restrict__ units,
           const longlong2* __restrict__ ranges, const int64_t* __restrict__ rng, const float4* __restrict__ bcf,
           const float* __restrict__ sxf, int64_t ns, const float* __restrict__ txf, int64_t nt,
           const float* __restrict__ qs, const float* __restrict__ tnrm_f, const float* __restrict__ res,
           const int64_t* __restrict__ tperm, double* __restrict__ out) {
    using S = NearShape<KIND>;
    extern __shared__ float4 p2p_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ui = blockIdx.x * kP2PWarps + warp;
    if (ui >= nunits) return;                     // whole warp; no block-wide barrier below
    const int4 u = units[ui];                     // (leaf, first range, end range, flags)
    const int b = leaves[u.x];
    const float4 cb0 = bcf[3 * b], cb1 = bcf[3 * b + 1];   // leaf centre, FP32 hi and lo
    const int64_t tb = rng[4 * b + 2], te = rng[4 * b + 3];
    if (!CORR && u.y == u.z) {                    // no sources (all exact zeros): the far field alone
        constexpr int NC = KIND == 3 ? 3 : 1;     // the leaf's only unit, so a plain store
        for (int64_t t = tb + lane; t < te; t += 32)
            for (int c = 0; c < NC; ++c) out[tperm[t] + c * nt] = res ? (double)res[t + c * nt] : 0.0;
        return;
    }
    float4* st = p2p_smem + warp * (S::kStage * 32 + S::kRaw * 16);
    float* raw = reinterpret_cast<float*>(st + S::kStage * 32);
    constexpr int kMaxT = CORR ? S::kMaxTCorr : S::kMaxT;
    const int pass = u.w >> kUnitPassShift;
    const int64_t tf = pass ? tb + (int64_t)(pass - 1) * (8 * kMaxT) : tb;
    const int64_t tl = pass && tf + 8 * kMaxT < te ? tf + 8 * kMaxT : te;
    for (int64_t t0 = tf; t0 < tl; t0 += 8 * kMaxT) {
        const int n = (int)(tl - t0 < 8 * kMaxT ? tl - t0 : 8 * kMaxT);
        const int64_t tend = t0 + n;
        switch ((n + 7) >> 3) {
#define KF_PASS(TT)                                                                                              \
    case TT:                                                                                                     \
        if constexpr (TT <= kMaxT)                                                                               \
            p2p_pass<KIND, TT, CORR>(lane, u.y, u.z, ranges, u.w, cb0, cb1, sxf, ns, txf, nt, qs, tnrm_f, res,   \
                                     tperm, out, t0, tend, st, raw);                                             \
        break;
            KF_PASS(1) KF_PASS(2) KF_PASS(3) KF_PASS(4) KF_PASS(5) KF_PASS(6) KF_PASS(7) KF_PASS(8)
#undef KF_PASS
        }
    }
}

template <int KIND>
constexpr size_t p2p_warp_smem() {
    return (size_t)kP2PWarps * (NearShape<KIND>::kStage * 32 * sizeof(float4) + NearShape<KIND>::kRaw * 2 * 32 * sizeof(float));
}

// Dynamic shared memory of the near-field kernels (above the 48 KB default for some).
int set_p2p_smem(int kind) {
#define KF_SMEM(K)                                                                                              \
    KF_CHECK_CUDA(cudaFuncSetAttribute(k_p2p_warp<K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                       (int)p2p_warp_smem<K>()));                                              \
    KF_CHECK_CUDA(cudaFuncSetAttribute(k_p2p_warp<K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                       (int)p2p_warp_smem<K>()));
    switch (kind) {
    case 0: KF_SMEM(0) break;
    case 1: KF_SMEM(1) break;
    case 2: KF_SMEM(2) break;
    case 3: KF_SMEM(3) break;
    default: KF_SMEM(4) break;
    }
#undef KF_SMEM
    return KIFMM_OK;
}

// Mixed plans evaluate the near field with the warp kernel, except single-layer and
// field plans with a leaf above kP2PWarpMaxLeaf targets.
inline bool warp_near(const Plan& P) {
    const bool plain = P.kernel == KIFMM_KERNEL_SL || P.kernel == KIFMM_KERNEL_FIELD;
    return !P.fp64 && (!plain || P.max_trg_leaf <= kP2PWarpMaxLeaf);
}

// Set-up scan of the near-field ranges: for range i (sources [ranges[i].x, .y) of the
// target leaf leaves[rleaf[i]]), the smallest FP64 squared distance between one of the
// leaf's targets and one of the range's sources, over all pairs (minr2[2i]) and over the
// pairs at least delta/2 apart (minr2[2i + 1]; coincident points, a target among its own
// sources above all, are skipped whatever the precision).  One warp per range.
__global__ void k_range_min_r2(int nr, const longlong2* __restrict__ ranges, const int* __restrict__ rleaf,
                               const int* __restrict__ leaves, const int64_t* __restrict__ rng,
                               const double* __restrict__ sxyz, int64_t ns, const double* __restrict__ txyz,
                               int64_t nt, double* __restrict__ minr2) {
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= nr) return;
    const int64_t j0 = ranges[i].x & kRangeIdx, j1 = ranges[i].y;
    const int b = leaves[rleaf[i]];
    const int64_t tb = rng[4 * b + 2], te = rng[4 * b + 3];
    const double half2 = 0.25 * kDelta * kDelta;
    double best = 1e300, best_far = 1e300;
    for (int64_t j = j0 + lane; j < j1; j += 32) {
        const double sx = sxyz[j], sy = sxyz[ns + j], sz = sxyz[2 * ns + j];
        for (int64_t t = tb; t < te; ++t) {
            const double dx = txyz[t] - sx, dy = txyz[nt + t] - sy, dz = txyz[2 * nt + t] - sz;
            const double r2 = dx * dx + dy * dy + dz * dz;
            best = fmin(best, r2);
            if (r2 >= half2) best_far = fmin(best_far, r2);
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
        best_far = fmin(best_far, __shfl_xor_sync(0xffffffffu, best_far, o));
    }
    if (lane == 0) {
        minr2[2 * i] = best;
        minr2[2 * i + 1] = best_far;
    }
}

// out[tperm[t] + c nt] += res[t + c nt] for the nc output components: the far field,
// after a near field that ran beside it.
__global__ void k_add_far(const int64_t* __restrict__ tperm, const float* __restrict__ res, int64_t nt, int nc,
                          double* __restrict__ out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int64_t o = tperm[t];
    for (int c = 0; c < nc; ++c) out[o + c * nt] += (double)res[t + c * nt];
}

// f[i] = near[i] + res[itperm[i]] in input order (res null: f[i] = near[i]), written
// once and in order, so f may be a host buffer.
__global__ void k_add_far_io(const int64_t* __restrict__ itperm, const float* __restrict__ res,
                             const double* __restrict__ near, int64_t nt, int nc, double* __restrict__ f) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nt) return;
    const int64_t t = itperm[i];
    for (int c = 0; c < nc; ++c) f[i + c * nt] = res ? near[i + c * nt] + (double)res[t + c * nt] : near[i + c * nt];
}

// ---------------------------------------------------------------- set-up kernels
// x = hi + lo with hi = fl32(x), lo = fl32(x - hi): 6 x n SoA (hi x|y|z, lo x|y|z).
__global__ void k_split_xyz(const double* __restrict__ xyz, int64_t n, float* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int d = 0; d < 3; ++d) {
        const double v = xyz[d * n + i];
        const float h = (float)v;
        out[d * n + i] = h;
        out[(3 + d) * n + i] = (float)(v - (double)h);
    }
}

// Sorted normals: FP64 (outd) and FP32 (outf; with lo, also the FP32 remainders as rows
// 3..5, which the mixed near field's exact products read).
__global__ void k_gather_nrm(const double* __restrict__ nrm, const int64_t* __restrict__ perm, int64_t n,
                             double* __restrict__ outd, float* __restrict__ outf, bool lo) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    for (int d = 0; d < 3; ++d) {
        double v = nrm[d * n + j];
        if (outd) outd[d * n + i] = v;
        if (outf) {
            const float h = (float)v;
            outf[d * n + i] = h;
            if (lo) outf[(3 + d) * n + i] = (float)(v - (double)h);
        }
    }
}

// D2T row descriptors: target position in its leaf's unit frame, its normal, scale.
// grad: rows of the target-normal derivative, with the normal tnrm (ADL) or, tnrm
// null, the unit vector of coordinate axis (field component).
__global__ void k_d2t_rows(const int* __restrict__ tleaf_of, int64_t nt, const double* __restrict__ txyz,
                           const double* __restrict__ tnrm, int axis, const int* __restrict__ lvl,
                           const double* __restrict__ ctr, double root_h, bool adl, double* apts,
                           double* anrm, double* ascale, int64_t* orow) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int b = tleaf_of[t];
    double r = ldexp(root_h, -lvl[b]);
    for (int d = 0; d < 3; ++d) {
        apts[3 * t + d] = (txyz[d * nt + t] - ctr[3 * b + d]) / r;
        anrm[3 * t + d] = adl ? (tnrm ? tnrm[d * nt + t] : (d == axis ? 1.0 : 0.0)) : 0.0;
    }
    ascale[t] = adl ? 1.0 / r : 1.0;
    orow[t] = t;
}

int octant_of(const Tree& T, int b) {
    return ((T.h_coord[3 * b] & 1) << 2) | ((T.h_coord[3 * b + 1] & 1) << 1) | (T.h_coord[3 * b + 2] & 1);
}

bool has_src(const Tree& T, int b) { return T.h_rng[4 * b + 1] > T.h_rng[4 * b]; }
bool has_trg(const Tree& T, int b) { return T.h_rng[4 * b + 3] > T.h_rng[4 * b + 2]; }

// Group (op, in, out) triples by op into tiles of <= cap pairs.
struct Triple {
    int op, in, out;
};

// Stable order of tr by op: a counting sort (ops are small non-negative operator ids).
void sort_by_op(std::vector<Triple>& tr) {
    int nop = 0;
    for (const Triple& x : tr) nop = std::max(nop, x.op + 1);
    std::vector<size_t> at((size_t)nop + 1, 0);
    for (const Triple& x : tr) ++at[(size_t)x.op + 1];
    for (int o = 0; o < nop; ++o) at[(size_t)o + 1] += at[(size_t)o];
    std::vector<Triple> out(tr.size());
    for (const Triple& x : tr) out[at[(size_t)x.op]++] = x;
    tr.swap(out);
}

void make_tiles(std::vector<Triple>& tr, std::vector<int4>& tiles, std::vector<int>& pin,
                std::vector<int>& pout, int cap) {
    sort_by_op(tr);
    size_t base = pin.size();
    size_t i = 0;
    while (i < tr.size()) {
        size_t j = i;
        while (j < tr.size() && tr[j].op == tr[i].op && j - i < (size_t)cap) ++j;
        tiles.push_back(make_int4(tr[i].op, (int)(base + i), (int)(j - i), 0));
        i = j;
    }
    for (auto& t : tr) {
        pin.push_back(t.in);
        pout.push_back(t.out);
    }
}

// Work list of the persistent tensor-core M2L, whose CTA c of G takes tiles c, c + G,
// c + 2G, ...  Target boxes of one level whose V lists hold the same offsets are
// grouped.  Each run of cap of them, or a last run of at least 3/4 cap, forms a chain:
// one tile per offset, every tile with the same targets in the same columns.  One CTA
// takes a chain's tiles back to back (tile.w = 1 on all but the last), so it writes
// each target once per chain instead of once per offset.  The other pairs form tiles
// by offset as before.  Chains (longest first), then those tiles in offset order, go
// to the CTA with the fewest tiles.  (Counting a chained tile as half a plain one, for
// the scatter it skips, measured slower: 0.564 against 0.535 ms on the 1M cube.)  A
// chain longer than a CTA's share of all tiles is cut into near-equal pieces, each
// written once, so no CTA waits on one long chain.
// kcount receives each CTA's tile count, and the interleaved list is padded with empty
// tiles that no CTA reads.  With no chain the plain offset-sorted list is kept (kcount
// empty).
void m2l_schedule(std::vector<Triple>& tr, const std::vector<int>& level, int cap, int G,
                  std::vector<int4>& tiles, std::vector<int>& pin, std::vector<int>& pout,
                  std::vector<int>& kcount, int64_t* chain_pairs) {
    *chain_pairs = 0;
    kcount.clear();
    // order by (target, offset): the V lists arrive target by target, so only each
    // target's own list needs sorting
    auto by_out_op = [](const Triple& a, const Triple& b) { return a.out != b.out ? a.out < b.out : a.op < b.op; };
    bool grouped = true;
    for (size_t i = 1; i < tr.size() && grouped; ++i) grouped = tr[i - 1].out <= tr[i].out;
    if (grouped) {
        for (size_t i = 0; i < tr.size();) {
            size_t j = i;
            while (j < tr.size() && tr[j].out == tr[i].out) ++j;
            std::stable_sort(tr.begin() + i, tr.begin() + j, by_out_op);
            i = j;
        }
    } else {
        std::stable_sort(tr.begin(), tr.end(), by_out_op);
    }
    // targets by (level, offsets of the V list), members in box order; groups are
    // visited in the order of their (level, offsets) keys
    struct KeyHash {
        size_t operator()(const std::pair<int, std::vector<int>>& k) const {
            uint64_t h = 1469598103934665603ull ^ (uint64_t)(uint32_t)k.first;
            for (int x : k.second) h = (h ^ (uint64_t)(uint32_t)x) * 1099511628211ull;
            return (size_t)h;
        }
    };
    std::unordered_map<std::pair<int, std::vector<int>>, std::vector<std::pair<int, size_t>>, KeyHash> hgroups;
    for (size_t i = 0; i < tr.size();) {
        size_t j = i;
        std::vector<int> sig;
        while (j < tr.size() && tr[j].out == tr[i].out) sig.push_back(tr[j++].op);
        hgroups[{level[tr[i].out], std::move(sig)}].push_back({tr[i].out, i});
        i = j;
    }
    std::vector<const std::pair<const std::pair<int, std::vector<int>>, std::vector<std::pair<int, size_t>>>*> groups;
    groups.reserve(hgroups.size());
    for (const auto& kv : hgroups)
        if (kv.second.size() * 4 >= (size_t)cap * 3 && kv.first.second.size() >= 2) groups.push_back(&kv);
    std::sort(groups.begin(), groups.end(), [](const auto* a, const auto* b) { return a->first < b->first; });
    std::vector<std::vector<int4>> chains;
    std::vector<int> cpin, cpout;
    std::vector<char> chained(tr.size(), 0);
    for (const auto* kvp : groups) {
        const auto& kv = *kvp;
        const std::vector<int>& sig = kv.first.second;
        const auto& mem = kv.second;
        for (size_t c0 = 0; c0 < mem.size(); c0 += (size_t)cap) {
            const size_t n = std::min(mem.size() - c0, (size_t)cap);
            if (n * 4 < (size_t)cap * 3 || sig.size() < 2) break;
            std::vector<int4> ch;
            for (size_t o = 0; o < sig.size(); ++o) {
                ch.push_back(make_int4(sig[o], (int)cpin.size(), (int)n, o + 1 < sig.size() ? 1 : 0));
                for (size_t m = c0; m < c0 + n; ++m) {
                    const size_t t = mem[m].second + o;    // the member's pair of offset sig[o]
                    cpin.push_back(tr[t].in);
                    cpout.push_back(tr[t].out);
                    chained[t] = 1;
                }
            }
            *chain_pairs += (int64_t)(n * sig.size());
            chains.push_back(std::move(ch));
        }
    }
    std::vector<Triple> rest;
    for (size_t i = 0; i < tr.size(); ++i)
        if (!chained[i]) rest.push_back(tr[i]);
    if (chains.empty()) {
        make_tiles(rest, tiles, pin, pout, cap);
        return;
    }
    std::vector<int4> single;
    std::vector<int> spin, spout;
    make_tiles(rest, single, spin, spout, cap);
    size_t total = single.size();
    for (const auto& ch : chains) total += ch.size();
    const size_t share = std::max<size_t>(2, total / (size_t)G);
    std::vector<std::vector<int4>> pieces;
    for (auto& ch : chains) {
        const size_t np = (ch.size() + share - 1) / share;
        for (size_t q = 0; q < np; ++q) {
            const size_t a = ch.size() * q / np, b = ch.size() * (q + 1) / np;
            std::vector<int4> pc(ch.begin() + a, ch.begin() + b);
            pc.back().w = 0;                              // the piece's targets are written here
            pieces.push_back(std::move(pc));
        }
    }
    chains.swap(pieces);
    // pair lists: the chains' first, then the others'
    const int sbase = (int)cpin.size();
    pin = cpin;
    pout = cpout;
    pin.insert(pin.end(), spin.begin(), spin.end());
    pout.insert(pout.end(), spout.begin(), spout.end());
    std::vector<std::vector<int4>> list(G);
    using Load = std::pair<int, int>;   // (tiles so far, CTA)
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
    for (int c = 0; c < G; ++c) heap.push({0, c});
    std::stable_sort(chains.begin(), chains.end(),
                     [](const std::vector<int4>& a, const std::vector<int4>& b) { return a.size() > b.size(); });
    auto deal = [&](const int4* t, size_t n) {
        Load l = heap.top();
        heap.pop();
        list[l.second].insert(list[l.second].end(), t, t + n);
        heap.push({l.first + (int)n, l.second});
    };
    for (const auto& ch : chains) deal(ch.data(), ch.size());
    for (int4 t : single) {
        t.y += sbase;
        deal(&t, 1);
    }
    size_t kmax = 0;
    for (const auto& l : list) kmax = std::max(kmax, l.size());
    tiles.assign((size_t)G * kmax, make_int4(0, 0, 0, 0));   // padding: empty tiles
    kcount.resize(G);
    for (int c = 0; c < G; ++c) {
        kcount[c] = (int)list[c].size();
        for (size_t k = 0; k < list[c].size(); ++k) tiles[(size_t)c + k * G] = list[c][k];
    }
}

int upload_tiles(PairTiles& pt, const std::vector<int4>& tiles, const std::vector<int>& pin,
                 const std::vector<int>& pout, cudaStream_t s) {
    KF_TRY(pt.tiles.upload(tiles, s));
    KF_TRY(pt.pin.upload(pin, s));
    KF_TRY(pt.pout.upload(pout, s));
    pt.ntiles = (int)tiles.size();
    pt.npairs = (int64_t)pin.size();
    return KIFMM_OK;
}

// Remove the row mean of every column of every operator (FP64), then round.
// Used for the adjoint double layer, whose targets see only gradients: the
// constant part of a down-check potential is dropped before it is stored in the
// working precision, so its rounding is relative to the potential's variation.

// Operators of Mr rows (Q of them valid) by Kc columns, op-major.
template <typename Real>
__global__ void k_center_ops(const double* __restrict__ in, int Q, int Mr, int Kc, bool center,
                             Real* __restrict__ out) {
    int op = blockIdx.y;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Kc) return;
    const double* A = in + (size_t)op * Mr * Kc;
    Real* O = out + (size_t)op * Mr * Kc;
    double mean = 0;
    if (center) {
        for (int i = 0; i < Q; ++i) mean += A[(size_t)i * Kc + j];
        mean /= Q;
    }
    for (int i = 0; i < Mr; ++i) O[(size_t)i * Kc + j] = i < Q ? (Real)(A[(size_t)i * Kc + j] - mean) : (Real)0;
}

// Rows K_o P of one translation family (0 M2M', 1 M2L', 2 L2L') for every operator o,
// in FP64: P is Q x C (row-major), out is op-major with Qp rows (Q used) of Kc columns.
int translation_ops(const Plan& P, const HostPinv& h, int which, int C, int Kc, const double* dP, double* out,
                    cudaStream_t s) {
    std::vector<double> apts, ascale, bpts;
    std::vector<int> bset;
    std::vector<int64_t> orow;
    translation_rows(h, which, apts, bset, orow, ascale, bpts, P.Qp);
    DBuf<double> da, dsc, db;
    DBuf<int> dbs;
    DBuf<int64_t> dor;
    KF_TRY(da.upload(apts, s));
    KF_TRY(dsc.upload(ascale, s));
    KF_TRY(db.upload(bpts, s));
    KF_TRY(dbs.upload(bset, s));
    KF_TRY(dor.upload(orow, s));
    RowSpec rs;
    rs.nrows = (int)bset.size();
    rs.apts = da.p;
    rs.ascale = dsc.p;
    rs.bset = dbs.p;
    rs.orow = dor.p;
    rs.bpts = db.p;
    KF_TRY(build_rows<double>(rs, P.Q, C, Kc, dP, 0, out, s));
    KF_CHECK_CUDA(cudaStreamSynchronize(s));   // the row descriptors are freed on return
    return KIFMM_OK;
}

// The three translation families in FP64, each operator K_o P with P the up (M2M',
// M2L') or down (L2L') pseudo-inverse (Q x Q, stored Qp wide); op-major, Qp x Qp each.
int build_ops(Plan& P, const HostPinv& h, double* m2m, double* m2l, double* l2l, cudaStream_t s) {
    DBuf<double> dPu, dPd;
    KF_TRY(dPu.upload(h.Pu, s));
    KF_TRY(dPd.upload(h.Pd, s));
    double* outs[3] = {m2m, m2l, l2l};
    const int nops[3] = {8, kNumOffsets, 8};
    for (int which = 0; which < 3; ++which) {
        DBuf<double> tmp;
        KF_TRY(tmp.alloc((size_t)nops[which] * P.Qp * P.Qp));
        KF_CHECK_CUDA(cudaMemsetAsync(tmp.p, 0, tmp.bytes(), s));
        KF_TRY(translation_ops(P, h, which, P.Q, P.Qp, which == 2 ? dPd.p : dPu.p, tmp.p, s));
        bool center = gradient_kernel(P.kernel) && which != 0;
        dim3 grid(div_up(P.Qp, 128), nops[which]);
        k_center_ops<double><<<grid, 128, 0, s>>>(tmp.p, P.Q, P.Qp, P.Qp, center, outs[which]);
        KF_CHECK_LAUNCH();
        KF_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    return KIFMM_OK;
}

// The Chebyshev engine's tables (cheb_host_tables), centred like build_ops's for the
// gradient kernels: a constant shift of the node values moves the interpolant by that
// constant, so the rows' mean carries no gradient.
int build_cheb_ops(Plan& P, double* m2m, double* m2l, double* l2l, cudaStream_t s) {
    std::vector<double> hm2m, hm2l, hl2l;
    cheb_host_tables(P.p, P.Qp, hm2m, hm2l, hl2l);
    const std::vector<double>* src[3] = {&hm2m, &hm2l, &hl2l};
    double* outs[3] = {m2m, m2l, l2l};
    const int nops[3] = {8, kNumOffsets, 8};
    for (int which = 0; which < 3; ++which) {
        DBuf<double> tmp;
        KF_TRY(tmp.upload(*src[which], s));
        const bool center = gradient_kernel(P.kernel) && which != 0;
        dim3 grid(div_up(P.Qp, 128), nops[which]);
        k_center_ops<double><<<grid, 128, 0, s>>>(tmp.p, P.Q, P.Qp, P.Qp, center, outs[which]);
        KF_CHECK_LAUNCH();
        KF_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    return KIFMM_OK;
}

// out[op] (Kr x Kc) = L (Kr x Q, row-major) . A[op] (Q of Mr rows x Kc), set-up only:
// FP64 products, rounded once.  64 x 64 outputs per block, 4 x 4 per thread.
__global__ void k_left_mul(const double* __restrict__ L, const double* __restrict__ A, int Q, int Mr, int Kr,
                           int Kc, float* __restrict__ out) {
    __shared__ double Ls[16][65];
    __shared__ double As[16][65];
    const int op = blockIdx.z, r0 = blockIdx.y * 64, c0 = blockIdx.x * 64;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const double* Ao = A + (size_t)op * Mr * Kc;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < Q; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int r = e >> 4, k = e & 15;          // L: 16 neighbouring k of one row
            Ls[k][r] = (r0 + r < Kr && k0 + k < Q) ? L[(size_t)(r0 + r) * Q + k0 + k] : 0.0;
            const int kk = e >> 6, c = e & 63;          // A: 64 neighbouring columns of one row
            As[kk][c] = (k0 + kk < Q && c0 + c < Kc) ? Ao[(size_t)(k0 + kk) * Kc + c0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += Ls[k][ty * 4 + i] * As[k][tx * 4 + j];
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = r0 + ty * 4 + i, c = c0 + tx * 4 + j;
            if (r < Kr && c < Kc) out[((size_t)op * Kr + r) * Kc + c] = (float)acc[i][j];
        }
}

// Mixed-precision tables.  With P = W U^T (U: Q x r orthonormal, W = P U), every
// check-space operator K P that is followed by another pseudo-inverse only through
// its range can act between projections: a box's up-check potential enters as
// U_u^T u (ru values), its down-check potential is kept as U_d^T d (rd values), and
//   M2M'' = U_u^T (1/2 K_c W_u)    (Ku x Ku)
//   M2L'' = U_d^T C K_o W_u        (Kd x Ku)
//   L2L'' = U_d^T C K_c W_d        (Kd x Kd)
// with C the row-mean removal for ADL (identity otherwise), plus the projections
// U_u^T and U_d^T C of the leaves' and X-list boxes' full check potentials.  The
// products are exact: U^T U = I, so the chain reproduces K P ... K P.  Built in FP64,
// rounded once to FP32 (then split into two-term FP16 by the caller).
int build_projected(Plan& P, const HostPinv& h, OpTables* t, const std::vector<double>& Eup, DBuf<float>* f32,
                    cudaStream_t s) {
    const int Q = P.Q, Qp = P.Qp, Ku = t->Ku, Kd = t->Kd;
    const bool adl = gradient_kernel(P.kernel);
    std::vector<double> Lu((size_t)Ku * Q, 0.0), Ld((size_t)Kd * Q, 0.0);
    for (int j = 0; j < h.ru; ++j)
        for (int i = 0; i < Q; ++i) Lu[(size_t)j * Q + i] = h.Uu[(size_t)i * h.ru + j];
    for (int j = 0; j < h.rd; ++j)
        for (int i = 0; i < Q; ++i) Ld[(size_t)j * Q + i] = h.Ud[(size_t)i * h.rd + j];
    DBuf<double> dLu, dLd, dWu, dWd;
    KF_TRY(dLu.upload(Lu, s));
    KF_TRY(dLd.upload(Ld, s));
    KF_TRY(dWu.upload(h.Wu, s));
    KF_TRY(dWd.upload(h.Wd, s));
    const int nops[3] = {8, kNumOffsets, 8};
    for (int which = 0; which < 3; ++which) {
        const int C = which == 2 ? h.rd : h.ru, Kc = which == 2 ? Kd : Ku, Kr = which == 0 ? Ku : Kd;
        DBuf<double> tmp, cen;
        KF_TRY(tmp.alloc((size_t)nops[which] * Qp * Kc));
        KF_CHECK_CUDA(cudaMemsetAsync(tmp.p, 0, tmp.bytes(), s));
        KF_TRY(translation_ops(P, h, which, C, Kc, which == 2 ? dWd.p : dWu.p, tmp.p, s));
        const double* A = tmp.p;
        if (adl && which != 0) {
            KF_TRY(cen.alloc(tmp.n));
            dim3 grid(div_up(Kc, 128), nops[which]);
            k_center_ops<double><<<grid, 128, 0, s>>>(tmp.p, Q, Qp, Kc, true, cen.p);
            KF_CHECK_LAUNCH();
            A = cen.p;
        }
        dim3 grid(div_up(Kc, 64), div_up(Kr, 64), nops[which]);
        k_left_mul<<<grid, 256, 0, s>>>(which == 0 ? dLu.p : dLd.p, A, Q, Qp, Kr, Kc, f32[which].p);
        KF_CHECK_LAUNCH();
        KF_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    // projections U_u^T E (from the ks skeleton potentials; E interpolates the whole
    // up-check surface) and U_d^T C, zero padded to K x ks and K x Qp
    for (int f = 3; f < kFamilies; ++f) {
        const std::vector<double>& L = f == 3 ? Lu : Ld;
        const int K = f == 3 ? Ku : Kd, W = f == 3 ? t->ks : Qp;
        std::vector<float> ut((size_t)K * W, 0.f);
        for (int j = 0; j < K; ++j) {
            if (f == 3) {
                for (int m = 0; m < t->ks; ++m) {
                    double acc = 0.0;
                    for (int i = 0; i < Q; ++i) acc += L[(size_t)j * Q + i] * Eup[(size_t)i * t->ks + m];
                    ut[(size_t)j * W + m] = (float)acc;
                }
                continue;
            }
            double mean = 0.0;
            if (adl) {
                for (int i = 0; i < Q; ++i) mean += L[(size_t)j * Q + i];
                mean /= Q;
            }
            for (int i = 0; i < Q; ++i) ut[(size_t)j * W + i] = (float)(L[(size_t)j * Q + i] - mean);
        }
        KF_CHECK_CUDA(cudaMemcpyAsync(f32[f].p, ut.data(), ut.size() * sizeof(float), cudaMemcpyHostToDevice, s));
        KF_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    return KIFMM_OK;
}

// Per-target evaluation rows G(x_t, 2.95 s) P: P = Pd (Q wide, stored Qp) or, factored,
// Wd (rd wide, stored Kd).
template <typename Real>
int build_d2t(Plan& P, const HostPinv& h, bool factored, int Kd, const std::vector<int>& tleaf_of, int axis,
              Real* out, cudaStream_t s) {
    const Tree& T = P.tree->t;
    int64_t nt = T.nt;
    DBuf<int> dleaf;
    KF_TRY(dleaf.upload(tleaf_of, s));
    DBuf<double> apts, anrm, ascale, bpts, dPd;
    DBuf<int64_t> orow;
    KF_TRY(apts.alloc(3 * nt));
    KF_TRY(anrm.alloc(3 * nt));
    KF_TRY(ascale.alloc(nt));
    KF_TRY(orow.alloc(nt));
    std::vector<double> hb(3 * (size_t)h.Q);
    for (size_t i = 0; i < hb.size(); ++i) hb[i] = kDnEquiv * h.surf[i];
    KF_TRY(bpts.upload(hb, s));
    KF_TRY(dPd.upload(factored ? h.Wd : h.Pd, s));
    const int C = factored ? h.rd : P.Q, Kc = factored ? Kd : P.Qp;
    const double* txyz = T.same ? T.sxyz.p : T.txyz.p;
    const bool adl = gradient_kernel(P.kernel);
    const double* tn = P.kernel == KIFMM_KERNEL_ADL ? P.tnrm_d.p : nullptr;
    k_d2t_rows<<<div_up(nt, 256), 256, 0, s>>>(dleaf.p, nt, txyz, tn, axis, T.lvl.p, T.ctr.p, T.root_h, adl,
                                               apts.p, anrm.p, ascale.p, orow.p);
    KF_CHECK_LAUNCH();
    // build in chunks of rows to bound the launch size
    const int64_t chunk = 1 << 20;
    for (int64_t r0 = 0; r0 < nt; r0 += chunk) {
        RowSpec rs;
        rs.nrows = (int)std::min<int64_t>(chunk, nt - r0);
        rs.apts = apts.p + 3 * r0;
        rs.anrm = anrm.p + 3 * r0;
        rs.ascale = ascale.p + r0;
        rs.bset = nullptr;
        rs.orow = orow.p + r0;
        rs.bpts = bpts.p;
        KF_TRY(build_rows<Real>(rs, P.Q, C, Kc, dPd.p, adl ? 1 : 0, out, s));
    }
    KF_CHECK_CUDA(cudaStreamSynchronize(s));
    return KIFMM_OK;
}

// The translation tables for P's key from the process-wide cache, or built now.  Entries
// are weak: tables live as long as some plan holds them.
int get_tables(Plan& P, const HostPinv& h, cudaStream_t s) {
    static std::mutex mu;
    static std::vector<std::weak_ptr<OpTables>> cache;
    int dev = 0;
    KF_CHECK_CUDA(cudaGetDevice(&dev));
    const bool centered = gradient_kernel(P.kernel);
    std::lock_guard<std::mutex> lock(mu);
    for (auto it = cache.begin(); it != cache.end();) {
        std::shared_ptr<OpTables> t = it->lock();
        if (!t) {
            it = cache.erase(it);
            continue;
        }
        if (t->device == dev && t->p == P.p && t->cut_up == P.cut_up && t->cut_dn == P.cut_dn &&
            t->cap_up == P.cap_up && t->cap_dn == P.cap_dn && t->fp64 == P.fp64 &&
            t->cheb == P.cheb &&
            t->centered == centered) {
            P.ops = t;
            return KIFMM_OK;
        }
        ++it;
    }
    auto t = std::make_shared<OpTables>();
    t->device = dev;
    t->p = P.p;
    t->cut_up = P.cut_up;
    t->cut_dn = P.cut_dn;
    t->cap_up = P.cap_up;
    t->cap_dn = P.cap_dn;
    t->cheb = P.cheb;
    t->fp64 = P.fp64;
    t->centered = centered;
    const size_t QQ = (size_t)P.Qp * P.Qp;
    if (P.fp64) {
        KF_TRY(t->m2m_d.alloc(8 * QQ));
        KF_TRY(t->m2l_d.alloc(kNumOffsets * QQ));
        KF_TRY(t->l2l_d.alloc(8 * QQ));
        KF_CHECK_CUDA(cudaMemsetAsync(t->m2m_d.p, 0, t->m2m_d.bytes(), s));
        KF_CHECK_CUDA(cudaMemsetAsync(t->m2l_d.p, 0, t->m2l_d.bytes(), s));
        KF_CHECK_CUDA(cudaMemsetAsync(t->l2l_d.p, 0, t->l2l_d.bytes(), s));
        t->ru = P.cheb ? P.Q : h.ru;
        t->rd = P.cheb ? P.Q : h.rd;
        if (P.cheb)
            KF_TRY(build_cheb_ops(P, t->m2m_d.p, t->m2l_d.p, t->l2l_d.p, s));
        else
            KF_TRY(build_ops(P, h, t->m2m_d.p, t->m2l_d.p, t->l2l_d.p, s));
    } else {
        // translations between projections (see build_projected), two-term FP16
        t->ru = h.ru;
        t->rd = h.rd;
        t->Ku = (h.ru + 15) / 16 * 16;
        t->Kd = (h.rd + 15) / 16 * 16;
        // S2U on a skeleton of the up-check surface: the pivots above kSkelTol, rounded
        // up to the surface kernel's next shape (all Q points once that shape holds them)
        std::vector<int> sk;
        std::vector<double> Eup;
        {
            const UpPivots& f = host_up_pivots(P.p);
            const int kt = up_pivot_count(f, kSkelTol);
            const int slots = surf_slots(std::min(kt, h.Q));
            if (slots == 0 || slots >= h.Q) {
                t->ks = h.Q;
                sk.resize(h.Q);
                for (int i = 0; i < h.Q; ++i) sk[i] = i;
                Eup.assign((size_t)h.Q * h.Q, 0.0);
                for (int i = 0; i < h.Q; ++i) Eup[(size_t)i * h.Q + i] = 1.0;
            } else {
                t->ks = slots;
                up_skeleton(f, slots, sk, Eup);
            }
            std::vector<float> su(3 * (size_t)t->ks);
            for (int m = 0; m < t->ks; ++m)
                for (int d = 0; d < 3; ++d) su[3 * m + d] = (float)h.surf[3 * (size_t)sk[m] + d];
            KF_TRY(t->surf_up.upload(su, s));
        }
        DBuf<float> f32[kFamilies];
        const int nops[kFamilies] = {8, kNumOffsets, 8, 1, 1};
        const int rows[kFamilies] = {t->Ku, t->Kd, t->Kd, t->Ku, t->Kd};
        const int cols[kFamilies] = {t->Ku, t->Ku, t->Kd, t->ks, P.Qp};
        for (int f = 0; f < kFamilies; ++f) {
            KF_TRY(f32[f].alloc((size_t)nops[f] * rows[f] * cols[f]));
            KF_CHECK_CUDA(cudaMemsetAsync(f32[f].p, 0, f32[f].bytes(), s));
        }
        KF_TRY(build_projected(P, h, t.get(), Eup, f32, s));
        for (int f = 0; f < kFamilies; ++f) {
            KF_TRY(t->tab_h[f].alloc(f32[f].n));
            KF_TRY(t->tab_l[f].alloc(f32[f].n));
            KF_TRY(tc_split_table(f32[f].p, t->tab_h[f].p, t->tab_l[f].p, f32[f].n, &t->texp[f], s));
            KF_TRY(tc_make_map(&t->tmaps[f][0], t->tab_h[f].p, nops[f], rows[f], cols[f]));
            KF_TRY(tc_make_map(&t->tmaps[f][1], t->tab_l[f].p, nops[f], rows[f], cols[f]));
        }
    }
    KF_CHECK_CUDA(cudaStreamSynchronize(s));
    P.ops = t;
    cache.push_back(t);
    return KIFMM_OK;
}

int setup(Plan& P, const double* src_nrm, const double* trg_nrm, cudaStream_t s) {
    Tree& T = P.tree->t;
    // wall-clock time of each set-up phase, the device work of the phase included
    const auto t_start = std::chrono::steady_clock::now();
    auto t_last = t_start;
    auto stamp = [&](int k) -> int {
        KF_CHECK_CUDA(cudaStreamSynchronize(s));
        const auto now = std::chrono::steady_clock::now();
        P.setup_ms[k] = std::chrono::duration<double, std::milli>(now - t_last).count();
        t_last = now;
        return KIFMM_OK;
    };
    // mixed form: ranks capped at 256, the rows one tensor-core work item covers, so that
    // M2L'' and L2L'' (and for kernels other than DL M2M'') take one row group; the
    // double layer keeps its larger upward rank (dipole sources need it).  The
    // Chebyshev engine has no pseudo-inverses (its order only picks the surface
    // operators computed here, which it leaves unused).
    P.fp64 = P.prec == KIFMM_PREC_FP64;
    P.cap_dn = P.fp64 || P.cheb ? 0 : kMixedMaxRank;
    P.cap_up = P.fp64 || P.cheb || P.kernel == KIFMM_KERNEL_DL ? 0 : kMixedMaxRank;
    const HostPinv& h = host_pinv(P.cheb ? 2 : P.p, P.cut_up, P.cut_dn, P.cap_up, P.cap_dn);
    P.Q = P.cheb ? P.p * P.p * P.p : h.Q;
    P.Qp = (P.Q + 15) / 16 * 16;
    KF_TRY(P.err.alloc(1));
    KF_CHECK_CUDA(cudaMemsetAsync(P.err.p, 0, sizeof(int), s));

    // sorted normals
    if (P.kernel == KIFMM_KERNEL_DL) {
        KF_TRY(P.snrm.alloc(3 * T.ns));
        k_gather_nrm<<<div_up(T.ns, 256), 256, 0, s>>>(src_nrm, T.sperm.p, T.ns, P.snrm.p, nullptr, false);
        KF_CHECK_LAUNCH();
    }
    if (P.kernel == KIFMM_KERNEL_ADL) {
        const int64_t* tp = T.same ? T.sperm.p : T.tperm.p;
        KF_TRY(P.tnrm_d.alloc(3 * T.nt));
        if (!P.fp64) KF_TRY(P.tnrm_f.alloc(6 * T.nt));
        k_gather_nrm<<<div_up(T.nt, 256), 256, 0, s>>>(trg_nrm, tp, T.nt, P.tnrm_d.p,
                                                       P.fp64 ? nullptr : P.tnrm_f.p, true);
        KF_CHECK_LAUNCH();
    }

    // surfaces (the Chebyshev engine: its box nodes)
    {
        const std::vector<double> pts = P.cheb ? cheb_nodes(P.p) : h.surf;
        std::vector<float> sf(pts.begin(), pts.end());
        KF_TRY(P.surf_d.upload(pts, s));
        KF_TRY(P.surf_f.upload(sf, s));
    }

    // operators: shared tables of this key, built once
    KF_TRY(get_tables(P, h, s));
    KF_TRY(stamp(0));
    // mixed: tiles sized for the tensor-core GEMM of each family's row count; FP64:
    // CUDA-core blocks of kPairTile
    const int cap_up = P.fp64 ? kPairTile : tc_tile_pairs(P.ops->Ku);
    const int cap_dn = P.fp64 ? kPairTile : tc_tile_pairs(P.ops->Kd);
    if (!P.fp64) {
        const int kz = std::max(P.ops->Ku, P.ops->Kd);
        KF_TRY(P.bexp.alloc(T.nbox));
        KF_TRY(P.vin_h.alloc((size_t)T.nbox * kz));
        KF_TRY(P.vin_l.alloc((size_t)T.nbox * kz));
        KF_TRY(P.sexp.alloc(T.nbox));
        KF_TRY(P.sin_h.alloc((size_t)T.nbox * P.Qp));
        KF_TRY(P.sin_l.alloc((size_t)T.nbox * P.Qp));
        KF_TRY(P.sxf.alloc(6 * (size_t)T.ns));
        k_split_xyz<<<div_up(T.ns, 256), 256, 0, s>>>(T.sxyz.p, T.ns, P.sxf.p);
        KF_CHECK_LAUNCH();
        if (!T.same && T.nt > 0) {
            KF_TRY(P.txf.alloc(6 * (size_t)T.nt));
            k_split_xyz<<<div_up(T.nt, 256), 256, 0, s>>>(T.txyz.p, T.nt, P.txf.p);
            KF_CHECK_LAUNCH();
        }
        KF_TRY(P.bcf.alloc(3 * (size_t)T.nbox));
        k_box_f<<<div_up(T.nbox, 256), 256, 0, s>>>(T.ctr.p, T.lvl.p, T.root_h, T.nbox, P.bcf.p);
        KF_CHECK_LAUNCH();
    }

    // work lists (host bookkeeping over the tree's lists)
    std::vector<int> s2u_box, s2u_off{0}, s2u_idx, p2l_box, p2l_off{0}, p2l_idx, tleaf, p2p_off{0}, p2p_idx;
    std::vector<int> tleaf_of(T.nt, 0);
    // Double layer: a near-field source box whose dipoles all lie along one coordinate
    // axis and whose points share one coordinate c along it adds exactly zero to a
    // target leaf whose targets all have that coordinate c too (n.(x - y) = 0 for every
    // pair, in any precision; the interior of a flat face).  Such boxes are left out of
    // the near-field lists, detected by exact equality.
    P.near_zero_pairs = 0;
    P.near_pairs = 0;
    std::vector<double> hsx, hsn, htx;
    std::vector<signed char> plane_k;           // per box: the axis, -1 none, -2 not yet known
    std::vector<double> plane_c;
    if (P.kernel == KIFMM_KERNEL_DL && T.ns > 0) {
        KF_TRY(download(hsx, T.sxyz.p, 3 * (size_t)T.ns, s));
        KF_TRY(download(hsn, P.snrm.p, 3 * (size_t)T.ns, s));
        if (!T.same && T.nt > 0) KF_TRY(download(htx, T.txyz.p, 3 * (size_t)T.nt, s));
        plane_k.assign(T.nbox, -2);
        plane_c.assign(T.nbox, 0.0);
    }
    auto src_plane = [&](int a) -> int {        // the box's plane axis (its coordinate in plane_c)
        if (plane_k[a] != -2) return plane_k[a];
        int k = -1;
        const int64_t j0 = T.h_rng[4 * a], j1 = T.h_rng[4 * a + 1];
        if (j1 > j0) {
            for (int d = 0; d < 3; ++d)
                if (hsn[(size_t)d * T.ns + j0] != 0.0 && hsn[(size_t)((d + 1) % 3) * T.ns + j0] == 0.0 &&
                    hsn[(size_t)((d + 2) % 3) * T.ns + j0] == 0.0)
                    k = d;
            const double c = k >= 0 ? hsx[(size_t)k * T.ns + j0] : 0.0;
            for (int64_t j = j0; j < j1 && k >= 0; ++j)
                if (hsn[(size_t)((k + 1) % 3) * T.ns + j] != 0.0 || hsn[(size_t)((k + 2) % 3) * T.ns + j] != 0.0 ||
                    hsn[(size_t)k * T.ns + j] == 0.0 || hsx[(size_t)k * T.ns + j] != c)
                    k = -1;
            plane_c[a] = c;
        }
        plane_k[a] = (signed char)k;
        return k;
    };
    // DL: a source box's dipole axis (0..2; 3 mixed).  A leaf's near-field units hold boxes
    // of one axis each, so that as many as can take the one-term kernel do (a cube's
    // edges), and the surface kernel takes one term for such boxes too.
    std::vector<signed char> box_ax;
    if (!plane_k.empty()) box_ax.assign(T.nbox, -1);
    auto axis_class = [&](int a) -> int {
        if (box_ax.empty()) return 0;
        if (box_ax[a] >= 0) return box_ax[a];
        int k = 3;
        const int64_t j0 = T.h_rng[4 * a], j1 = T.h_rng[4 * a + 1];
        for (int d = 0; d < 3 && j1 > j0; ++d)
            if (hsn[(size_t)d * T.ns + j0] != 0.0) k = k == 3 ? d : 4;
        if (k == 4) k = 3;
        for (int64_t j = j0; j < j1 && k < 3; ++j)
            if (hsn[(size_t)k * T.ns + j] == 0.0 || hsn[(size_t)((k + 1) % 3) * T.ns + j] != 0.0 ||
                hsn[(size_t)((k + 2) % 3) * T.ns + j] != 0.0)
                k = 3;
        box_ax[a] = (signed char)k;
        return k;
    };
    auto zero_pair = [&](int b, int a) -> bool {  // source box a adds exactly zero to leaf b
        if (plane_k.empty()) return false;
        const int k = src_plane(a);
        if (k < 0) return false;
        const std::vector<double>& tx = T.same ? hsx : htx;
        const int64_t ntp = T.same ? T.ns : T.nt;
        const double c = plane_c[a];
        for (int64_t q = T.h_rng[4 * b + 2]; q < T.h_rng[4 * b + 3]; ++q)
            if (tx[(size_t)k * ntp + q] != c) return false;
        return true;
    };
    for (int b = 0; b < T.nbox; ++b) {
        int l = T.h_lvl[b];
        if (T.h_leaf[b] && has_src(T, b) && l >= 2) {
            s2u_box.push_back(b);
            s2u_idx.push_back(b);
            s2u_off.push_back((int)s2u_idx.size());
        }
        // X list: a leaf with fewer targets than check points takes its X sources
        // directly, with its U and W sources (|A| x n_t kernel evaluations, exact, instead
        // of |A| x Q onto its down-check surface); other boxes go through the surface
        const int64_t ntb = T.h_rng[4 * b + 3] - T.h_rng[4 * b + 2];
        const bool x_direct = T.h_leaf[b] && ntb < P.Q;
        if (has_trg(T, b) && T.h_x_off[b + 1] > T.h_x_off[b] && !x_direct) {
            p2l_box.push_back(b);
            for (int k = T.h_x_off[b]; k < T.h_x_off[b + 1]; ++k) {
                p2l_idx.push_back(T.h_x_idx[k]);
                P.n_xpairs += T.h_rng[4 * T.h_x_idx[k] + 1] - T.h_rng[4 * T.h_x_idx[k]];
            }
            p2l_off.push_back((int)p2l_idx.size());
        }
        if (T.h_leaf[b] && has_trg(T, b)) {
            tleaf.push_back(b);
            auto add = [&](int a) {
                const int64_t pairs = ntb * (T.h_rng[4 * a + 1] - T.h_rng[4 * a]);
                if (zero_pair(b, a)) {
                    P.near_zero_pairs += pairs;
                } else {
                    p2p_idx.push_back(a);
                    P.near_pairs += pairs;
                }
            };
            for (int k = T.h_u_off[b]; k < T.h_u_off[b + 1]; ++k) add(T.h_u_idx[k]);
            for (int k = T.h_w_off[b]; k < T.h_w_off[b + 1]; ++k) add(T.h_w_idx[k]);
            if (x_direct)
                for (int k = T.h_x_off[b]; k < T.h_x_off[b + 1]; ++k) add(T.h_x_idx[k]);
            p2p_off.push_back((int)p2p_idx.size());
            for (int64_t t = T.h_rng[4 * b + 2]; t < T.h_rng[4 * b + 3]; ++t) tleaf_of[t] = b;
            P.max_trg_leaf = std::max<int>(P.max_trg_leaf, (int)(T.h_rng[4 * b + 3] - T.h_rng[4 * b + 2]));
        }
    }
    P.n_s2u = (int)s2u_box.size();
    P.n_p2l = (int)p2l_box.size();
    P.n_tleaf = (int)tleaf.size();
    KF_TRY(P.s2u_box.upload(s2u_box, s));
    KF_TRY(P.s2u_off.upload(s2u_off, s));
    KF_TRY(P.s2u_idx.upload(s2u_idx, s));
    KF_TRY(P.p2l_box.upload(p2l_box, s));
    KF_TRY(P.p2l_off.upload(p2l_off, s));
    KF_TRY(P.p2l_idx.upload(p2l_idx, s));
    KF_TRY(P.tleaf.upload(tleaf, s));
    KF_TRY(P.p2p_off.upload(p2p_off, s));
    KF_TRY(P.p2p_idx.upload(p2p_idx, s));
    if (!P.fp64 && !box_ax.empty()) {
        std::vector<int> hbax(T.nbox, 3);
        // 4 + k: every source of the box in one plane normal to its dipoles' axis k
        auto code = [&](int a) { return src_plane(a) >= 0 ? 4 + src_plane(a) : axis_class(a); };
        for (int a : s2u_idx) hbax[a] = code(a);
        for (int a : p2l_idx) hbax[a] = code(a);
        KF_TRY(P.bax.upload(hbax, s));
    }
    // mixed: near-field work units of at most kP2PUnitSrc sources, heaviest first.  Each
    // range carries its offset exponent E (2^E above every coordinate offset of the leaf's
    // targets and the range's sources, from the boxes' extents) and the flags of an FP64
    // scan of its pairs; within a unit the ranges are ordered by E, so the targets are
    // split anew only when it changes.  Ranges with close pairs are also dealt, one per
    // unit, to the corrected-distance launch.
    if (!P.fp64) {
        struct Unit {
            int4 u;
            int64_t work;
        };
        std::vector<Unit> units;
        std::vector<longlong2> ranges;
        std::vector<int> rleaf;
        std::vector<double> rext;              // per range: largest coordinate offset of its pairs
        auto half = [&](int box) { return std::ldexp(T.root_h, -T.h_lvl[box]); };
        auto exp_of = [](double ext) { return std::max(-100, std::min(100, std::ilogb(ext * (1.0 + 1e-12)) + 1)); };
        std::vector<int> lb;
        for (size_t li = 0; li < tleaf.size(); ++li) {
            const int b = tleaf[li];
            const int64_t ntg = T.h_rng[4 * b + 3] - T.h_rng[4 * b + 2];
            const double hb = half(b);
            const size_t u0 = units.size();
            int r0 = (int)ranges.size();
            int64_t cnt = 0;
            auto close_unit = [&]() {
                // order the unit's ranges by exponent
                std::vector<int> ord(ranges.size() - r0);
                std::iota(ord.begin(), ord.end(), r0);
                std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
                    return range_exp(ranges[x].x) < range_exp(ranges[y].x);
                });
                std::vector<longlong2> rg;
                std::vector<double> re;
                for (int i : ord) {
                    rg.push_back(ranges[i]);
                    re.push_back(rext[i]);
                }
                std::copy(rg.begin(), rg.end(), ranges.begin() + r0);
                std::copy(re.begin(), re.end(), rext.begin() + r0);
                units.push_back({make_int4((int)li, r0, (int)ranges.size(), 0), ntg * cnt});
                r0 = (int)ranges.size();
                cnt = 0;
            };
            lb.assign(p2p_idx.begin() + p2p_off[li], p2p_idx.begin() + p2p_off[li + 1]);
            if (!box_ax.empty())
                std::stable_sort(lb.begin(), lb.end(), [&](int x, int y) { return axis_class(x) < axis_class(y); });
            int cls_cur = -1;
            for (const int a : lb) {
                const int cls = axis_class(a);
                if (cnt > 0 && cls != cls_cur) close_unit();
                cls_cur = cls;
                const double ha = half(a);
                double box_ext = hb;
                for (int d = 0; d < 3; ++d) {
                    const double ca = (2 * T.h_coord[3 * a + d] + 1) * ha, cb = (2 * T.h_coord[3 * b + d] + 1) * hb;
                    box_ext = std::max(box_ext, std::fabs(ca - cb) + ha);
                }
                const long long ebits = (long long)(exp_of(box_ext) + 128) << 48;
                int64_t j0 = T.h_rng[4 * a], j1 = T.h_rng[4 * a + 1];
                while (j0 < j1) {
                    const int64_t take = std::min<int64_t>(j1 - j0, kP2PUnitSrc - cnt);
                    ranges.push_back(make_longlong2(j0 | ebits, j0 + take));
                    rleaf.push_back((int)li);
                    rext.push_back(box_ext);
                    cnt += take;
                    j0 += take;
                    if (cnt == kP2PUnitSrc) close_unit();
                }
            }
            if (cnt > 0 || units.size() == u0) close_unit();
            const bool split = units.size() - u0 > 1;
            P.p2p_multi = P.p2p_multi || split;
            P.n_p2p_split += split ? 1 : 0;
            for (size_t i = u0; i < units.size(); ++i)
                units[i].u.w = (i == u0 ? kUnitFirst : 0) | (split ? kUnitSplit : 0);
        }
        // FP64 scan: the closest pair of each range
        const int nr = (int)ranges.size();
        std::vector<int4> hcu;
        std::vector<longlong2> hcr;
        if (nr > 0) {
            DBuf<longlong2> dr;
            DBuf<int> drl;
            DBuf<double> dmin;
            KF_TRY(dr.upload(ranges, s));
            KF_TRY(drl.upload(rleaf, s));
            KF_TRY(dmin.alloc(2 * (size_t)nr));
            const double* txyz = T.same ? T.sxyz.p : T.txyz.p;
            k_range_min_r2<<<div_up((int64_t)nr * 32, 256), 256, 0, s>>>(nr, dr.p, drl.p, P.tleaf.p, T.rng.p, T.sxyz.p,
                                                                       T.ns, txyz, T.nt, dmin.p);
            KF_CHECK_LAUNCH();
            std::vector<double> minr2;
            KF_TRY(download(minr2, dmin.p, 2 * (size_t)nr, s));
            const double excl2 = (4.0 * kDelta) * (4.0 * kDelta);
            for (int r = 0; r < nr; ++r) {
                // FP32 offsets of this range's pairs are good to 2^-24 of 2^Er: a pair much
                // closer than that takes the corrected distance, and so does a pair between
                // delta/2 and 4 delta, whose exclusion it then decides to FP32 accuracy
                const double close = std::ldexp(1.0, range_exp(ranges[r].x) - kCloseBits);
                if (minr2[2 * r] < excl2) ranges[r].x |= kRangeExcl;
                if (minr2[2 * r + 1] < std::max(close * close, excl2)) {
                    ranges[r].x |= kRangeCorr;
                    hcu.push_back(make_int4(rleaf[r], (int)hcr.size(), (int)hcr.size() + 1, kUnitSplit));
                    hcr.push_back(ranges[r]);
                }
            }
        }
        // double layer: units whose sources' dipoles all lie along one coordinate axis take
        // the one-term kernel (KIND 4), dealt after the others
        std::vector<char> is_axis(units.size(), 0);
        if (P.kernel == KIFMM_KERNEL_DL && T.ns > 0) {
            std::vector<double> hn;
            KF_TRY(download(hn, P.snrm.p, 3 * (size_t)T.ns, s));
            std::vector<signed char> ax(T.ns);
            for (int64_t j = 0; j < T.ns; ++j) {
                const double c[3] = {hn[j], hn[T.ns + j], hn[2 * T.ns + j]};
                ax[j] = -1;
                for (int k = 0; k < 3; ++k)
                    if (c[(k + 1) % 3] == 0.0 && c[(k + 2) % 3] == 0.0 && c[k] != 0.0) ax[j] = (signed char)k;
            }
            // run[j]: end of the run of equal axis codes from j
            std::vector<int64_t> run(T.ns);
            for (int64_t j = T.ns - 1; j >= 0; --j)
                run[j] = (j + 1 < T.ns && ax[j + 1] == ax[j]) ? run[j + 1] : j + 1;
            for (size_t i = 0; i < units.size(); ++i) {
                int k = -2;
                for (int r = units[i].u.y; r < units[i].u.z && k != -1; ++r) {
                    const int64_t j0 = ranges[r].x & kRangeIdx, j1 = ranges[r].y;
                    const int kr = (run[j0] >= j1) ? ax[j0] : -1;
                    k = (k == -2 || k == kr) ? kr : -1;
                }
                if (k >= 0) {
                    is_axis[i] = 1;
                    units[i].u.w |= k << 8;
                }
            }
        }
        // one unit per pass of the leaf's targets (empty units keep the whole leaf)
        {
            auto pass_targets = [&](bool axis) {
                const int k = axis ? 4 : P.kernel == KIFMM_KERNEL_SL ? 0 : P.kernel == KIFMM_KERNEL_DL ? 1
                                        : P.kernel == KIFMM_KERNEL_ADL ? 2 : 3;
                const int mt = k == 0 ? NearShape<0>::kMaxT : k == 1 ? NearShape<1>::kMaxT
                             : k == 2 ? NearShape<2>::kMaxT : k == 3 ? NearShape<3>::kMaxT : NearShape<4>::kMaxT;
                return (int64_t)8 * mt;
            };
            std::vector<Unit> pu;
            std::vector<char> pa;
            pu.reserve(units.size());
            for (size_t i = 0; i < units.size(); ++i) {
                const int b = tleaf[units[i].u.x];
                const int64_t ntg = T.h_rng[4 * b + 3] - T.h_rng[4 * b + 2];
                const int64_t pt = pass_targets(is_axis[i] != 0);
                const int64_t np = (ntg + pt - 1) / pt;
                if (units[i].u.y == units[i].u.z || np <= 1) {
                    pu.push_back(units[i]);
                    pa.push_back(is_axis[i]);
                    continue;
                }
                const int64_t per = units[i].work / ntg;      // sources of the unit
                for (int64_t k = 0; k < np; ++k) {
                    Unit v = units[i];
                    v.u.w |= (int)(k + 1) << kUnitPassShift;
                    v.work = std::min(pt, ntg - k * pt) * per;
                    pu.push_back(v);
                    pa.push_back(is_axis[i]);
                }
            }
            units.swap(pu);
            is_axis.swap(pa);
        }
        std::vector<size_t> ord(units.size());
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) {
            if (is_axis[x] != is_axis[y]) return is_axis[x] < is_axis[y];
            return units[x].work > units[y].work;
        });
        std::vector<int4> hu(units.size());
        P.n_p2p_axis = 0;
        P.near_axis_pairs = 0;
        for (size_t i = 0; i < units.size(); ++i) {
            hu[i] = units[ord[i]].u;
            P.n_p2p_axis += is_axis[ord[i]];
            if (is_axis[ord[i]]) P.near_axis_pairs += units[ord[i]].work;
        }
        KF_TRY(P.p2p_units.upload(hu, s));
        KF_TRY(P.p2p_ranges.upload(ranges, s));
        KF_TRY(P.p2p_cunits.upload(hcu, s));
        KF_TRY(P.p2p_cranges.upload(hcr, s));
        P.n_p2p_units = (int)hu.size();
        P.n_p2p_corr = (int)hcu.size();
        for (int k = 0; k < 5; ++k) KF_TRY(set_p2p_smem(k));
    }
    KF_TRY(stamp(1));

    // U2U: per parent level, (child -> parent) grouped by the child's octant
    {
        std::vector<int4> tiles;
        std::vector<int> pin, pout;
        P.u2u.level_tile.assign(T.nlev + 1, 0);
        for (int l = 0; l < T.nlev; ++l) {
            P.u2u.level_tile[l] = (int)tiles.size();
            if (l >= 2) {
                std::vector<Triple> tr;
                for (int b = T.level_off[l]; b < T.level_off[l + 1]; ++b) {
                    if (T.h_leaf[b] || !has_src(T, b)) continue;
                    for (int o = 0; o < 8; ++o) {
                        int c = T.h_child[8 * b + o];
                        if (c >= 0 && has_src(T, c)) tr.push_back({o, c, b});
                    }
                }
                make_tiles(tr, tiles, pin, pout, cap_up);
            }
        }
        P.u2u.level_tile[T.nlev] = (int)tiles.size();
        KF_TRY(upload_tiles(P.u2u, tiles, pin, pout, s));
    }
    // M2L: all V pairs grouped by offset
    {
        std::vector<int4> tiles;
        std::vector<int> pin, pout;
        std::vector<Triple> tr;
        tr.reserve(T.nv);
        for (int b = 0; b < T.nbox; ++b)
            for (int k = T.h_v_off[b]; k < T.h_v_off[b + 1]; ++k) {
                int a = T.h_v_idx[k];
                int ox = T.h_coord[3 * a] - T.h_coord[3 * b], oy = T.h_coord[3 * a + 1] - T.h_coord[3 * b + 1],
                    oz = T.h_coord[3 * a + 2] - T.h_coord[3 * b + 2];
                tr.push_back({(ox + 3) * 49 + (oy + 3) * 7 + (oz + 3), a, b});
            }
        // mixed: chains of targets that share their V list's offsets, when one work item
        // covers all of an operator's rows (Kd <= 256) and the kernel runs one CTA per SM
        P.m2l_chain_pairs = 0;
        if (!P.fp64 && P.ops->Kd <= 256) {
            int dev = 0, nsm = 0;
            KF_CHECK_CUDA(cudaGetDevice(&dev));
            KF_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
            std::vector<int> kcount;
            m2l_schedule(tr, T.h_lvl, cap_dn, nsm, tiles, pin, pout, kcount, &P.m2l_chain_pairs);
            if (!kcount.empty()) KF_TRY(P.m2l.kcount.upload(kcount, s));
        } else {
            make_tiles(tr, tiles, pin, pout, cap_dn);
        }
        KF_TRY(upload_tiles(P.m2l, tiles, pin, pout, s));
    }
    // L2L: per child level >= 3, (parent -> child) grouped by the child's octant
    {
        std::vector<int4> tiles;
        std::vector<int> pin, pout;
        P.l2l.level_tile.assign(T.nlev + 1, 0);
        for (int l = 0; l < T.nlev; ++l) {
            P.l2l.level_tile[l] = (int)tiles.size();
            if (l >= 3) {
                std::vector<Triple> tr;
                for (int b = T.level_off[l]; b < T.level_off[l + 1]; ++b)
                    if (has_trg(T, b)) tr.push_back({octant_of(T, b), T.h_parent[b], b});
                make_tiles(tr, tiles, pin, pout, cap_dn);
            }
        }
        P.l2l.level_tile[T.nlev] = (int)tiles.size();
        KF_TRY(upload_tiles(P.l2l, tiles, pin, pout, s));
    }
    // mixed: projections of the S2U leaves' up-check potentials and of the X-list
    // boxes' down-check potentials (one (box -> box) tile list each), and the
    // projected potentials of every box
    if (!P.fp64) {
        for (int up = 1; up >= 0; --up) {
            std::vector<int4> tiles;
            std::vector<int> pin, pout;
            std::vector<Triple> tr;
            for (int b : up ? s2u_box : p2l_box) tr.push_back({0, b, b});
            make_tiles(tr, tiles, pin, pout, up ? cap_up : cap_dn);
            KF_TRY(upload_tiles(up ? P.proj_up : P.proj_x, tiles, pin, pout, s));
        }
        KF_TRY(P.zu.alloc((size_t)T.nbox * P.ops->Ku));
        KF_TRY(P.zd.alloc((size_t)T.nbox * P.ops->Kd));
        int prio_lo = 0, prio_hi = 0;
        KF_CHECK_CUDA(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
        KF_CHECK_CUDA(cudaStreamCreateWithPriority(&P.near_stream, cudaStreamNonBlocking, prio_lo));
        KF_CHECK_CUDA(cudaStreamCreateWithPriority(&P.far_stream, cudaStreamNonBlocking, prio_hi));
        KF_CHECK_CUDA(cudaEventCreateWithFlags(&P.ev_fork, cudaEventDisableTiming));
        KF_CHECK_CUDA(cudaEventCreateWithFlags(&P.ev_join, cudaEventDisableTiming));
        KF_CHECK_CUDA(cudaEventCreateWithFlags(&P.ev_far, cudaEventDisableTiming));
        KF_CHECK_CUDA(cudaEventCreateWithFlags(&P.ev_zero, cudaEventDisableTiming));
    }

    KF_TRY(stamp(2));
    // per-target evaluation rows and buffers
    size_t nbq = (size_t)T.nbox * P.Qp;
    if (P.fp64) {
        KF_TRY(P.d2t_d.alloc((size_t)P.nc * T.nt * P.Qp));
        if (P.cheb) {
            DBuf<int> dleaf;
            KF_TRY(dleaf.upload(tleaf_of, s));
            for (int c = 0; c < P.nc; ++c)
                KF_TRY(cheb_rows(P, T, dleaf.p, P.kernel == KIFMM_KERNEL_ADL ? P.tnrm_d.p : nullptr, c,
                                 gradient_kernel(P.kernel), P.d2t_d.p + (size_t)c * T.nt * P.Qp, s));
            KF_CHECK_CUDA(cudaStreamSynchronize(s));
        } else {
            for (int c = 0; c < P.nc; ++c)
                KF_TRY(build_d2t<double>(P, h, false, 0, tleaf_of, c, P.d2t_d.p + (size_t)c * T.nt * P.Qp, s));
        }
        KF_TRY(P.u_d.alloc(nbq));
        KF_TRY(P.d_d.alloc(nbq));
        KF_TRY(P.res_d.alloc((size_t)P.nc * T.nt));
        KF_TRY(P.q_d.alloc(3 * T.ns));
    } else {
        // rows G W_d, reading the projected down-check potentials
        KF_TRY(P.d2t_f.alloc((size_t)P.nc * T.nt * P.ops->Kd));
        for (int c = 0; c < P.nc; ++c)
            KF_TRY(build_d2t<float>(P, h, true, P.ops->Kd, tleaf_of, c, P.d2t_f.p + (size_t)c * T.nt * P.ops->Kd, s));
        // (no FP32 check potentials: S2U and X write the projections' split inputs)
        KF_TRY(P.res_f.alloc((size_t)P.nc * T.nt));
        // DL: the dipoles q n_j as FP32 and their FP32 remainders (6 rows); else 3 rows
        KF_TRY(P.q_f.alloc((P.kernel == KIFMM_KERNEL_DL ? 6 : 3) * T.ns));
    }
    KF_TRY(stamp(3));
    P.setup_ms[4] = std::chrono::duration<double, std::milli>(t_last - t_start).count();

    P.device_bytes = 0;
    for (size_t b : {(size_t)P.ops->bytes(), P.d2t_d.bytes(), P.d2t_f.bytes(), P.u_d.bytes(), P.d_d.bytes(),
                     P.res_d.bytes(), P.q_d.bytes(), P.u_f.bytes(), P.d_f.bytes(), P.res_f.bytes(),
                     P.q_f.bytes(), P.snrm.bytes(), P.tnrm_d.bytes(), P.tnrm_f.bytes(),
                     P.bexp.bytes(), P.vin_h.bytes(), P.vin_l.bytes(), P.sexp.bytes(), P.sin_h.bytes(),
                     P.sin_l.bytes(), P.sxf.bytes(), P.txf.bytes(), P.bcf.bytes(), P.zu.bytes(),
                     P.zd.bytes()})
        P.device_bytes += (int64_t)b;
    return KIFMM_OK;
}

template <typename Real>
struct Bufs {
    const Real *m2m, *m2l, *l2l, *d2t, *surf, *tnrm;
    Real *u, *d, *res, *q;
};

enum { kU2U = 0, kM2L = 1, kL2L = 2 };

template <typename Real>
int run_pairs(const Plan& P, int which, const PairTiles& pt, int t0, int t1, const Real* ops, const Real* in,
              Real* out, int b0, int b1, cudaStream_t s, int& launches);

// Evaluated near-field pairs per target below which the near field starts after M2L
// (the 1M cube at 128 points per leaf: 52, once its exact zeros are left out; at 192:
// 298; curved surfaces: several hundred).
constexpr int64_t kLateNearPairs = 100;

// Mixed precision: two-term FP16 on the tensor cores (tcgen05), every translation
// between projected check potentials (see build_projected): U2U in the up basis (ru of
// Ku per box), M2L from the up to the down basis, L2L in the down basis (rd of Kd).
// The input vectors of a launch (boxes [b0, b1)) are scaled and split first.
template <>
int run_pairs<float>(const Plan& P, int which, const PairTiles& pt, int t0, int t1, const float* ops,
                     const float* z, float* out, int b0, int b1, cudaStream_t s, int& launches) {
    (void)ops;  // the tensor-core path reads the split tables through their TMA maps
    const OpTables& o = *P.ops;
    const bool in_up = which != kL2L, out_up = which == kU2U;
    const int K = in_up ? o.Ku : o.Kd, r = in_up ? o.ru : o.rd;
    const int Mr = out_up ? o.Ku : o.Kd, M = out_up ? o.ru : o.rd;
    // split even without tiles: M2L reads the splits the upward pass leaves behind
    if (b1 > b0) {
        KF_TRY(tc_box_split(z, r, K, b0, b1, P.vin_h.p, P.vin_l.p, P.bexp.p, s));
        ++launches;
    }
    if (t1 <= t0) return KIFMM_OK;
    const CUtensorMap* m = o.tmaps[which];
    // a chained M2L list (per-CTA counts) was dealt to one CTA per SM of this device
    const int* kc = (t0 == 0 && t1 == pt.ntiles) ? pt.kcount.p : nullptr;
    if (kc) {
        int dev = 0, nsm = 0;
        KF_CHECK_CUDA(cudaGetDevice(&dev));
        KF_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        if ((size_t)nsm != pt.kcount.n || (int64_t)pt.ntiles < nsm) {
            set_error("M2L work list was built for %zu SMs, the device has %d", pt.kcount.n, nsm);
            return KIFMM_ERR_CUDA;
        }
    }
    KF_TRY(launch_pair_tc(which, m[0], m[1], o.texp[which], M, Mr, K, Mr, pt.tiles.p + t0, t1 - t0, pt.pin.p,
                          pt.pout.p, P.bexp.p, P.vin_h.p, P.vin_l.p, out, P.err.p, s, kc));
    ++launches;
    return KIFMM_OK;
}

// Mixed: projection of the full check potentials of the boxes in pt's tiles onto the up
// (fam 3) or down (fam 4) basis, added into z.  Their split inputs (sin_h/sin_l, Qp per
// box, exponents in sexp) were written by the surface kernel that computed them.
int project(const Plan& P, int fam, const PairTiles& pt, float* z, cudaStream_t s, int& launches) {
    if (pt.ntiles == 0) return KIFMM_OK;
    const OpTables& o = *P.ops;
    const int Mr = fam == 3 ? o.Ku : o.Kd, M = fam == 3 ? o.ru : o.rd, Kp = fam == 3 ? o.ks : P.Qp;
    const CUtensorMap* m = o.tmaps[fam];
    KF_TRY(launch_pair_tc(3, m[0], m[1], o.texp[fam], M, Mr, Kp, Mr, pt.tiles.p, pt.ntiles, pt.pin.p,
                          pt.pout.p, P.sexp.p, P.sin_h.p, P.sin_l.p, z, P.err.p, s));
    launches += 2;
    return KIFMM_OK;
}

// FP64: CUDA-core blocked GEMM.
template <>
int run_pairs<double>(const Plan& P, int which, const PairTiles& pt, int t0, int t1, const double* ops,
                      const double* in, double* out, int b0, int b1, cudaStream_t s, int& launches) {
    (void)b0;
    (void)b1;
    using Real = double;
    if (t1 <= t0) return KIFMM_OK;
    auto kern = which == kU2U ? k_u2u_gemm<Real> : which == kM2L ? k_m2l_gemm<Real> : k_l2l_gemm<Real>;
    kern<<<t1 - t0, 256, 0, s>>>(ops, P.Q, P.Qp, pt.tiles.p + t0, pt.pin.p, pt.pout.p, in, out);
    KF_CHECK_LAUNCH();
    ++launches;
    return KIFMM_OK;
}

template <typename Real>
int matvec(Plan& P, const Bufs<Real>& B, const double* q, double* out, cudaStream_t s) {
    const Tree& T = P.tree->t;
    const size_t nbq = (size_t)T.nbox * P.Qp;
    int launches = 0;
    cudaEvent_t* slot = nullptr;
    if (P.profile) {
        if (P.slots_used == (int)P.ev_slots.size() && P.ev_slots.size() < 4096) {
            std::vector<cudaEvent_t> e(kPhaseEvents, nullptr);
            for (auto& x : e) KF_CHECK_CUDA(cudaEventCreate(&x));
            P.ev_slots.push_back(e);
        }
        if (P.slots_used < (int)P.ev_slots.size()) slot = P.ev_slots[P.slots_used++].data();
    }
    auto mark = [&](int i, cudaStream_t on = nullptr) -> int {
        if (slot) KF_CHECK_CUDA(cudaEventRecord(slot[i], on ? on : s));
        return KIFMM_OK;
    };
    // the near field on stream ns; res: the far field to add, or null (added later)
    auto near_field = [&](cudaStream_t ns, const Real* res) -> int {
        const double* txyz = T.same ? T.sxyz.p : T.txyz.p;
        const int64_t* tperm = T.same ? T.sperm.p : T.tperm.p;
        // FP32: the warp kernel over the near-field units (the single layer's leaves above
        // kP2PWarpMaxLeaf targets, and FP64: a block per leaf, whose staged sources serve
        // all of the leaf's targets at once)
        bool done = false;
        if constexpr (std::is_same<Real, float>::value) {
          if (warp_near(P)) {
            if (P.p2p_multi) {
                KF_CHECK_CUDA(cudaMemsetAsync(out, 0, (size_t)P.nc * T.nt * sizeof(double), ns));
                ++launches;
            }
#define KF_P2PW(KIND, CORR, NU, UNITS, RANGES)                                                                 \
    k_p2p_warp<KIND, CORR><<<(unsigned)div_up(NU, kP2PWarps), 32 * kP2PWarps, p2p_warp_smem<KIND>(), ns>>>(      \
        P.tleaf.p, NU, UNITS, RANGES, T.rng.p, P.bcf.p, P.sxf.p, T.ns, T.same ? P.sxf.p : P.txf.p, T.nt, B.q,     \
        P.tnrm_f.p, res, tperm, out)
#define KF_P2PK(CORR, NU, UNITS, RANGES)                                                                        \
    if (P.kernel == KIFMM_KERNEL_SL) KF_P2PW(0, CORR, NU, UNITS, RANGES);                                       \
    else if (P.kernel == KIFMM_KERNEL_DL) KF_P2PW(1, CORR, NU, UNITS, RANGES);                                  \
    else if (P.kernel == KIFMM_KERNEL_ADL) KF_P2PW(2, CORR, NU, UNITS, RANGES);                                 \
    else KF_P2PW(3, CORR, NU, UNITS, RANGES);
            {
                const int ngen = P.n_p2p_units - P.n_p2p_axis;
                if (ngen > 0 || P.n_p2p_axis == 0) KF_P2PK(false, ngen, P.p2p_units.p, P.p2p_ranges.p)
                if (P.n_p2p_axis) {
                    if (ngen > 0) {
                        KF_CHECK_LAUNCH();
                        ++launches;
                    }
                    KF_P2PW(4, false, P.n_p2p_axis, P.p2p_units.p + ngen, P.p2p_ranges.p);
                }
            }
            // the ranges with close pairs, added after the plain launch (same stream)
            if (P.n_p2p_corr) {
                KF_CHECK_LAUNCH();
                ++launches;
                KF_P2PK(true, P.n_p2p_corr, P.p2p_cunits.p, P.p2p_cranges.p)
            }
#undef KF_P2PK
#undef KF_P2PW
            done = true;
          }
        }
        if (!done) {
        int threads = std::min(256, std::max(32, (P.max_trg_leaf + 31) / 32 * 32));
        size_t smem = 6 * threads * sizeof(Real);
#define KF_P2P(KIND)                                                                                     \
    k_p2p<Real, KIND><<<P.n_tleaf, threads, smem, ns>>>(P.tleaf.p, P.p2p_off.p, P.p2p_idx.p, T.rng.p,     \
                                                        T.ctr.p, T.sxyz.p, T.ns, txyz, T.nt, B.q, B.tnrm, \
                                                        res, tperm, out)
        if (P.kernel == KIFMM_KERNEL_SL) KF_P2P(0);
        else if (P.kernel == KIFMM_KERNEL_DL) KF_P2P(1);
        else if (P.kernel == KIFMM_KERNEL_ADL) KF_P2P(2);
        else KF_P2P(3);
#undef KF_P2P
        }
        KF_CHECK_LAUNCH();
        ++launches;
        return KIFMM_OK;
    };
    // mixed, warp near field: it runs on its own stream beside the far field (forked
    // after the gather) and the far field is added once both are done
    const bool near_overlap = std::is_same<Real, float>::value && P.n_tleaf && P.near_stream && warp_near(P) &&
                              !P.serial;
    const bool dl = P.kernel == KIFMM_KERNEL_DL;
    // mixed DL: the FP32 remainders of the dipoles too (the near field's exact products)
    const bool dl_lo = dl && std::is_same<Real, float>::value;
    KF_TRY(mark(0));
    if (P.io_in)
        k_scatter_q<Real><<<div_up(T.ns, 256), 256, 0, s>>>(q, P.isperm.p, T.ns, dl ? P.snrm.p : nullptr, B.q,
                                                            dl_lo);
    else
        k_gather_q<Real><<<div_up(T.ns, 256), 256, 0, s>>>(q, T.sperm.p, T.ns, dl ? P.snrm.p : nullptr, B.q,
                                                           dl_lo);
    KF_CHECK_LAUNCH();
    ++launches;
    const cudaStream_t s_in = s;                  // the caller's stream
    // the near field on its stream, enqueued once the far field's first kernel is (so
    // that kernel's blocks, not the near field's, take the SMs first)
    auto fork_near = [&]() -> int {
        KF_CHECK_CUDA(cudaStreamWaitEvent(P.near_stream, P.ev_fork, 0));
        KF_TRY(mark(9, P.near_stream));
        KF_TRY(near_field(P.near_stream, nullptr));
        KF_TRY(mark(10, P.near_stream));
        KF_CHECK_CUDA(cudaEventRecord(P.ev_join, P.near_stream));
        return KIFMM_OK;
    };
    if (near_overlap) {
        KF_CHECK_CUDA(cudaEventRecord(P.ev_fork, s));
        KF_CHECK_CUDA(cudaStreamWaitEvent(P.far_stream, P.ev_fork, 0));
        s = P.far_stream;                         // the far-field phases below
    }
    constexpr bool mixed_form = std::is_same<Real, float>::value;
    if constexpr (!mixed_form) {
        KF_CHECK_CUDA(cudaMemsetAsync(B.u, 0, nbq * sizeof(Real), s));
        KF_CHECK_CUDA(cudaMemsetAsync(B.d, 0, nbq * sizeof(Real), s));
        launches += 2;
    }
    // the vectors the translations act on: check potentials (FP64) or, mixed, their
    // projections (zu, zd); mixed S2U and X write their full potentials as the split
    // input of a projection, which adds them into zu / zd
    constexpr bool mixed = std::is_same<Real, float>::value;
    Real* up = B.u;
    Real* dn = B.d;
    int dw = P.Qp;
    if constexpr (mixed) {
        up = P.zu.p;
        dn = P.zd.p;
        dw = P.ops->Kd;
        // zeroed on the near field's stream when there is one, beside S2U (which does not
        // touch them); the far field waits before its first accumulation into them
        const cudaStream_t zs = near_overlap ? P.near_stream : s;
        if (near_overlap) KF_CHECK_CUDA(cudaStreamWaitEvent(zs, P.ev_fork, 0));
        KF_CHECK_CUDA(cudaMemsetAsync(up, 0, P.zu.bytes(), zs));
        KF_CHECK_CUDA(cudaMemsetAsync(dn, 0, P.zd.bytes(), zs));
        if (near_overlap) KF_CHECK_CUDA(cudaEventRecord(P.ev_zero, zs));
        launches += 2;
    }
    KF_TRY(mark(1));
    // S2U
    if (P.n_s2u) {
        if constexpr (std::is_same<Real, double>::value) {
            if (P.cheb)
                KF_TRY(cheb_s2m(P, T, dl, P.n_s2u, P.s2u_box.p, P.s2u_off.p, P.s2u_idx.p, B.q, B.u, s));
            else
                KF_TRY(launch_surf<Real>(P, T, dl, P.n_s2u, P.s2u_box.p, P.s2u_off.p, P.s2u_idx.p, kUpCheck, B.q,
                                         B.surf, B.u, s));
        } else {
            KF_TRY(launch_surf<Real>(P, T, dl, P.n_s2u, P.s2u_box.p, P.s2u_off.p, P.s2u_idx.p, kUpCheck, B.q, B.surf,
                                     B.u, s));
        }
        ++launches;
    }
    // A near field much smaller than the far field (few evaluated pairs per target, as on
    // flat faces) starts after M2L, beside the coarse L2L levels and D2T, rather than
    // beside S2U and the upward pass, whose arithmetic it would slow.
    const bool late_near = near_overlap && P.near_pairs < kLateNearPairs * T.nt;
    if (near_overlap && !late_near) KF_TRY(fork_near());
    KF_TRY(mark(2));
    // mixed: the leaves' projections; U2U, deepest parents first
    if constexpr (mixed) {
        if (near_overlap) KF_CHECK_CUDA(cudaStreamWaitEvent(s, P.ev_zero, 0));
        KF_TRY(project(P, 3, P.proj_up, up, s, launches));
    }
    for (int l = T.nlev - 1; l >= 2; --l)
        KF_TRY(run_pairs<Real>(P, kU2U, P.u2u, P.u2u.level_tile[l], P.u2u.level_tile[l + 1], B.m2m, up, up,
                               T.level_off[std::min(l + 1, T.nlev)], T.level_off[std::min(l + 2, T.nlev)], s,
                               launches));
    KF_TRY(mark(3));
    // X list (mixed: then the X boxes' projections), then V list
    if (P.n_p2l) {
        // (the Chebyshev engine: X sources straight onto the box's nodes)
        KF_TRY(launch_surf<Real>(P, T, dl, P.n_p2l, P.p2l_box.p, P.p2l_off.p, P.p2l_idx.p, P.cheb ? 1.0 : kDnCheck,
                                 B.q, B.surf, B.d, s));
        ++launches;
        if constexpr (mixed) KF_TRY(project(P, 4, P.proj_x, dn, s, launches));
    }
    KF_TRY(mark(4));
    // the upward pass split levels 3 and deeper (mixed); level 2 is split here
    KF_TRY(run_pairs<Real>(P, kM2L, P.m2l, 0, P.m2l.ntiles, B.m2l, up, dn, T.level_off[std::min(2, T.nlev)],
                           T.level_off[std::min(3, T.nlev)], s, launches));
    if (late_near) {
        KF_CHECK_CUDA(cudaEventRecord(P.ev_fork, s));
        KF_TRY(fork_near());
    }
    KF_TRY(mark(5));
    // L2L, coarsest children first (ADL in FP64: each level's potentials shifted to zero
    // mean first; the mixed tables carry that centring)
    const bool center = !mixed && gradient_kernel(P.kernel);
    for (int l = 2; l < T.nlev; ++l) {
        if (l >= 3)
            KF_TRY(run_pairs<Real>(P, kL2L, P.l2l, P.l2l.level_tile[l], P.l2l.level_tile[l + 1], B.l2l, dn, dn,
                                   T.level_off[l - 1], T.level_off[l], s, launches));
        int nl = T.level_off[l + 1] - T.level_off[l];
        if (center && nl > 0) {
            k_center<Real><<<nl, 128, 0, s>>>(T.level_off[l], P.Q, P.Qp, B.d);
            KF_CHECK_LAUNCH();
            ++launches;
        }
    }
    KF_TRY(mark(6));
    if (P.n_tleaf) {
        for (int c = 0; c < P.nc; ++c) {
            k_d2t<Real><<<P.n_tleaf, 128, dw * sizeof(Real), s>>>(P.tleaf.p, T.rng.p, B.d2t + (size_t)c * T.nt * dw,
                                                                  dn, dw, B.res + (size_t)c * T.nt);
            KF_CHECK_LAUNCH();
            ++launches;
        }
    }
    KF_TRY(mark(7));
    if (!near_overlap) {
        KF_TRY(mark(9));
        if (P.n_tleaf) KF_TRY(near_field(s, B.res));
        KF_TRY(mark(10));
    }
    if (near_overlap) {
        // join both streams on the caller's, then add the far field into the near sums
        KF_CHECK_CUDA(cudaEventRecord(P.ev_far, s));
        s = s_in;
        KF_CHECK_CUDA(cudaStreamWaitEvent(s, P.ev_far, 0));
        KF_CHECK_CUDA(cudaStreamWaitEvent(s, P.ev_join, 0));
        if (P.io_out)
            k_add_far_io<<<(unsigned)div_up(T.nt, 256), 256, 0, s>>>(P.itperm.p, reinterpret_cast<const float*>(B.res),
                                                                     out, T.nt, P.nc, P.io_out);
        else
            k_add_far<<<(unsigned)div_up(T.nt, 256), 256, 0, s>>>(T.same ? T.sperm.p : T.tperm.p,
                                                                  reinterpret_cast<const float*>(B.res), T.nt, P.nc,
                                                                  out);
        KF_CHECK_LAUNCH();
        ++launches;
    } else if (P.io_out) {
        k_add_far_io<<<(unsigned)div_up(T.nt, 256), 256, 0, s>>>(P.itperm.p, nullptr, out, T.nt, P.nc, P.io_out);
        KF_CHECK_LAUNCH();
        ++launches;
    }
    KF_TRY(mark(8));
    P.launches = launches;
    return KIFMM_OK;
}

}  // namespace

int plan_matvec(Plan& P, const double* q, double* out, cudaStream_t s) {
    if (P.fp64) {
        Bufs<double> B{P.ops->m2m_d.p, P.ops->m2l_d.p, P.ops->l2l_d.p, P.d2t_d.p, P.surf_d.p, P.tnrm_d.p,
                       P.u_d.p,   P.d_d.p,   P.res_d.p, P.q_d.p};
        return matvec<double>(P, B, q, out, s);
    }
    Bufs<float> B{nullptr, nullptr, nullptr, P.d2t_f.p, P.surf_f.p, P.tnrm_f.p,
                  P.u_f.p,   P.d_f.p,   P.res_f.p, P.q_f.p};
    return matvec<float>(P, B, q, out, s);
}

}  // namespace kifmm

using namespace kifmm;

extern "C" int kifmm_fmm_setup(kifmm_tree tree, int kernel, int p, int precision, double pinv_cutoff,
                               const double* src_nrm, const double* trg_nrm, void* stream, kifmm_plan* out) {
    clear_error();
    KF_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    KF_ARG(tree != nullptr, "tree is NULL");
    KF_ARG(kernel >= KIFMM_KERNEL_SL && kernel <= KIFMM_KERNEL_FIELD, "unknown kernel");
    KF_ARG(p >= 2 && p <= 16, "p must be in [2, 16]");
    const bool cheb = (precision & KIFMM_ENGINE_CHEB) != 0;
    precision &= ~KIFMM_ENGINE_CHEB;
    KF_ARG(precision == KIFMM_PREC_FP64 || precision == KIFMM_PREC_MIXED, "unknown precision");
    KF_ARG(!cheb || precision == KIFMM_PREC_FP64, "the Chebyshev engine runs in FP64 only");
    KF_ARG(!cheb || (p >= 2 && p <= kChebMaxN), "Chebyshev order must be in [2, 8]");
    KF_ARG(pinv_cutoff == 0.0 || (pinv_cutoff > 0.0 && pinv_cutoff < 1.0), "pinv_cutoff must be 0 or in (0,1)");
    KF_ARG(kernel != KIFMM_KERNEL_DL || src_nrm != nullptr, "DL needs src_nrm");
    KF_ARG(kernel != KIFMM_KERNEL_ADL || trg_nrm != nullptr, "ADL needs trg_nrm");
    int dev = 0;
    KF_CHECK_CUDA(cudaGetDevice(&dev));
    KF_ARG(dev == tree->t.device, "tree was built on another device");
    kifmm_plan pl = new (std::nothrow) kifmm_plan_s;
    if (!pl) {
        set_error("host allocation failed");
        return KIFMM_ERR_OOM;
    }
    Plan& P = pl->P;
    P.tree = tree;
    P.kernel = kernel;
    P.cheb = cheb;
    P.nc = kernel == KIFMM_KERNEL_FIELD ? 3 : 1;
    P.p = p;
    P.prec = precision;
    // default truncations: FP64 1e-9; mixed 1e-8, except the double layer's Pu at 1e-9
    // (dipole sources need the smaller singular directions of the upward surface)
    if (pinv_cutoff > 0) {
        P.cut_up = P.cut_dn = pinv_cutoff;
    } else if (precision == KIFMM_PREC_FP64) {
        P.cut_up = P.cut_dn = 1e-9;
    } else {
        P.cut_dn = 1e-8;
        P.cut_up = kernel == KIFMM_KERNEL_DL ? 1e-9 : 1e-8;
    }
    int rc = setup(P, src_nrm, trg_nrm, (cudaStream_t)stream);
    if (rc != KIFMM_OK) {
        delete pl;
        return rc;
    }
    *out = pl;
    return KIFMM_OK;
}

extern "C" int kifmm_fmm_matvec(kifmm_plan plan, const double* q, double* out, void* stream) {
    clear_error();
    KF_ARG(plan && q && out, "NULL plan, q or out");
    return plan_matvec(plan->P, q, out, (cudaStream_t)stream);
}

namespace kifmm {
namespace {

// Capture the launches of one matvec (q, out as plan_matvec takes them; no profiling
// events inside the graph) and instantiate them into *exec (destroyed first if set).
int capture_matvec(Plan& P, const double* q, double* out, cudaGraphExec_t* exec) {
    if (*exec) {
        KF_CHECK_CUDA(cudaGraphExecDestroy(*exec));
        *exec = nullptr;
    }
    if (!P.cap_stream) KF_CHECK_CUDA(cudaStreamCreateWithFlags(&P.cap_stream, cudaStreamNonBlocking));
    const bool prof = P.profile;
    const int launches = P.launches;
    P.profile = false;
    KF_CHECK_CUDA(cudaStreamBeginCapture(P.cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = plan_matvec(P, q, out, P.cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(P.cap_stream, &g);
    P.profile = prof;
    P.launches = launches;
    if (rc != KIFMM_OK || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        if (rc == KIFMM_OK) {
            set_error("matvec capture failed: %s", cudaGetErrorString(ce));
            rc = KIFMM_ERR_CUDA;
        }
        cudaGetLastError();
        return rc;
    }
    // keep the stream priorities of the overlapped near and far fields
    cudaError_t ie = cudaGraphInstantiate(exec, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        *exec = nullptr;
        set_error("matvec graph instantiation failed: %s", cudaGetErrorString(ie));
        return KIFMM_ERR_CUDA;
    }
    return KIFMM_OK;
}

// Where a buffer of the host-buffer matvec lives: 0 pageable host memory, 1 page-locked
// host memory (*dev: the address kernels use for it), 2 device or managed memory.
int buffer_kind(const void* p, const void** dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeHost && a.devicePointer) {
        *dev = a.devicePointer;
        return 1;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
        *dev = p;
        return 2;
    }
    return 0;
}

// First use of the host-buffer matvec: inverse permutations and the staging of the
// near sums (q's staging is allocated when a pageable q first arrives).
int ensure_host_io(Plan& P, cudaStream_t s) {
    const Tree& T = P.tree->t;
    if (P.isperm.p || (T.ns == 0 && T.nt == 0)) return KIFMM_OK;
    KF_TRY(P.isperm.alloc(std::max<int64_t>(T.ns, 1)));
    KF_TRY(P.itperm.alloc(std::max<int64_t>(T.nt, 1)));
    KF_TRY(P.out_stage.alloc(std::max<int64_t>((int64_t)P.nc * T.nt, 1)));
    if (T.ns) k_invert_perm<<<(unsigned)div_up(T.ns, 256), 256, 0, s>>>(T.sperm.p, T.ns, P.isperm.p);
    if (T.nt)
        k_invert_perm<<<(unsigned)div_up(T.nt, 256), 256, 0, s>>>(T.same ? T.sperm.p : T.tperm.p, T.nt,
                                                                   P.itperm.p);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

}  // namespace
}  // namespace kifmm

namespace kifmm {
// The matvec as a replay of its captured launches (captured again when q or out change).
int plan_matvec_graph(Plan& P, const double* q, double* out, cudaStream_t s) {
    if (!P.gexec || P.g_q != q || P.g_out != out) {
        KF_TRY(capture_matvec(P, q, out, &P.gexec));
        P.g_q = q;
        P.g_out = out;
    }
    KF_CHECK_CUDA(cudaGraphLaunch(P.gexec, s));
    return KIFMM_OK;
}
}  // namespace kifmm

extern "C" int kifmm_fmm_matvec_graph(kifmm_plan plan, const double* q, double* out, void* stream) {
    clear_error();
    KF_ARG(plan && q && out, "NULL plan, q or out");
    return plan_matvec_graph(plan->P, q, out, (cudaStream_t)stream);
}

extern "C" int kifmm_fmm_matvec_host(kifmm_plan plan, const double* q, double* out, int graph, void* stream) {
    clear_error();
    KF_ARG(plan && q && out, "NULL plan, q or out");
    Plan& P = plan->P;
    const Tree& T = P.tree->t;
    cudaStream_t s = (cudaStream_t)stream;
    KF_TRY(ensure_host_io(P, s));
    const void* qd = nullptr;
    const void* od = nullptr;
    const int kq = buffer_kind(q, &qd), ko = buffer_kind(out, &od);
    // input: page-locked q is read in place (in input order) by the first kernel
    const double* q_use = q;
    bool in_host = false;
    if (kq == 1) {
        q_use = static_cast<const double*>(qd);
        in_host = true;
    } else if (kq == 0) {
        if (!P.q_stage.p) KF_TRY(P.q_stage.alloc(std::max<int64_t>(T.ns, 1)));
        if (T.ns)
            KF_CHECK_CUDA(cudaMemcpyAsync(P.q_stage.p, q, T.ns * sizeof(double), cudaMemcpyHostToDevice, s));
        q_use = P.q_stage.p;
    }
    // output: the near sums go to the staging buffer; the last kernel writes f into a
    // page-locked out directly, a pageable one is copied after the matvec
    double* out_use = out;
    double* io_out = nullptr;
    if (ko == 1) {
        out_use = P.out_stage.p;
        io_out = static_cast<double*>(const_cast<void*>(od));
    } else if (ko == 0) {
        out_use = P.out_stage.p;
    }
    P.io_in = in_host;
    P.io_out = io_out;
    int rc = KIFMM_OK;
    if (graph) {
        if (!P.hexec || P.h_q != q_use || P.h_out != out_use || P.h_io_out != io_out) {
            rc = capture_matvec(P, q_use, out_use, &P.hexec);
            if (rc == KIFMM_OK) {
                P.h_q = q_use;
                P.h_out = out_use;
                P.h_io_out = io_out;
            }
        }
        if (rc == KIFMM_OK) {
            cudaError_t e = cudaGraphLaunch(P.hexec, s);
            if (e != cudaSuccess) {
                set_error("%s", cudaGetErrorString(e));
                rc = KIFMM_ERR_CUDA;
            }
        }
    } else {
        rc = plan_matvec(P, q_use, out_use, s);
    }
    P.io_in = false;
    P.io_out = nullptr;
    if (rc != KIFMM_OK) return rc;
    if (ko == 0 && T.nt)
        KF_CHECK_CUDA(cudaMemcpyAsync(out, P.out_stage.p, (size_t)P.nc * T.nt * sizeof(double),
                                      cudaMemcpyDeviceToHost, s));
    return KIFMM_OK;
}

extern "C" int kifmm_plan_get_stats(kifmm_plan plan, kifmm_plan_stats* st) {
    clear_error();
    KF_ARG(plan && st, "NULL plan or stats");
    const Plan& P = plan->P;
    st->kernel = P.kernel;
    st->p = P.p;
    st->q_points = P.Q;
    st->precision = P.prec | (P.cheb ? KIFMM_ENGINE_CHEB : 0);
    st->pinv_cutoff = P.cut_dn;
    st->pinv_cutoff_up = P.cut_up;
    st->device_bytes = P.device_bytes;
    st->m2l_pairs = P.m2l.npairs;
    st->u2u_pairs = P.u2u.npairs;
    st->l2l_pairs = P.l2l.npairs;
    st->s2u_leaves = P.n_s2u;
    st->x_pairs = P.n_xpairs;
    st->launches_per_matvec = P.launches;
    st->rank_up = P.ops ? P.ops->ru : 0;
    st->rank_down = P.ops ? P.ops->rd : 0;
    st->m2l_width = P.fp64 ? P.Q : st->rank_up;
    st->m2l_rows = P.fp64 ? P.Q : st->rank_down;
    st->near_units = P.n_p2p_units;
    st->near_split_leaves = P.n_p2p_split;
    st->near_overlap = (!P.fp64 && P.near_stream && P.n_tleaf && warp_near(P)) ? 1 : 0;
    st->near_corr_ranges = P.n_p2p_corr;
    st->near_axis_units = P.n_p2p_axis;
    st->near_pairs = P.near_pairs;
    st->s2u_points = (P.fp64 || !P.ops) ? P.Q : P.ops->ks;
    st->m2l_chain_pairs = P.m2l_chain_pairs;
    for (int k = 0; k < 5; ++k) st->setup_ms[k] = P.setup_ms[k];
    st->near_axis_pairs = P.near_axis_pairs;
    st->near_zero_pairs = P.near_zero_pairs;
    return KIFMM_OK;
}

extern "C" int kifmm_up_skeleton(int p, int k, int32_t* idx, double* E, int32_t* k_tol) {
    clear_error();
    KF_ARG(p >= 2 && p <= 16, "p must be in [2, 16]");
    const int Q = 6 * (p - 1) * (p - 1) + 2;
    KF_ARG(k >= 1 && k <= Q, "k must be in [1, Q]");
    const UpPivots& f = host_up_pivots(p);
    if (k_tol) *k_tol = up_pivot_count(f, kSkelTol);
    if (idx || E) {
        std::vector<int> sk;
        std::vector<double> e;
        up_skeleton(f, k, sk, e);
        if (idx)
            for (int m = 0; m < k; ++m) idx[m] = sk[m];
        if (E) std::copy(e.begin(), e.end(), E);
    }
    return KIFMM_OK;
}

extern "C" int kifmm_plan_profile(kifmm_plan plan, int enable, double* phases) {
    clear_error();
    KF_ARG(plan, "NULL plan");
    Plan& P = plan->P;
    if (phases) {
        // mean over the matvecs recorded since the last read:
        // {gather, s2u, u2u, x, m2l, l2l, d2t, p2p, total}.  p2p is the near field's own
        // time (events 9, 10), which overlaps the far-field phases when it runs on its own
        // stream; then [7, 8) is the join and the far-field add
        constexpr int L = 8;
        for (int i = 0; i <= L; ++i) phases[i] = 0;
        for (int k = 0; k < P.slots_used; ++k) {
            const std::vector<cudaEvent_t>& e = P.ev_slots[k];
            KF_CHECK_CUDA(cudaEventSynchronize(e[L]));
            float ms;
            for (int i = 0; i < L - 1; ++i) {
                KF_CHECK_CUDA(cudaEventElapsedTime(&ms, e[i], e[i + 1]));
                phases[i] += ms;
            }
            KF_CHECK_CUDA(cudaEventElapsedTime(&ms, e[9], e[10]));
            phases[L - 1] += ms;
            KF_CHECK_CUDA(cudaEventElapsedTime(&ms, e[0], e[L]));
            phases[L] += ms;
        }
        if (P.slots_used)
            for (int i = 0; i <= L; ++i) phases[i] /= P.slots_used;
        P.slots_used = 0;
    }
    P.profile = enable != 0;
    P.serial = enable == 2;
    return KIFMM_OK;
}

extern "C" int kifmm_plan_check(kifmm_plan plan) {
    clear_error();
    KF_ARG(plan, "NULL plan");
    int h = 0;
    KF_CHECK_CUDA(cudaMemcpy(&h, plan->P.err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        set_error("a tensor-core translation GEMM gave up waiting on its pipeline (code %d)", h);
        return KIFMM_ERR_TIMEOUT;
    }
    return KIFMM_OK;
}

extern "C" int kifmm_plan_destroy(kifmm_plan plan) {
    clear_error();
    delete plan;
    return KIFMM_OK;
}
