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
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <queue>
#include <type_traits>

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

template <typename Real> struct RT;
template <> struct RT<float> {
    static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
};
template <> struct RT<double> {
    static __device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
};

// ---------------------------------------------------------------- gather
// lo: also write the rounding remainders of the dipoles (3 more rows, compensated
// near field)
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
template <bool NEAR, bool DIPOLE, int NP>
__device__ __forceinline__ void surf_pairs(const float4* __restrict__ sp, const float4* __restrict__ sd, int cnt,
                                           const float2* px, const float2* py, const float2* pz, float2* acc) {
    const float d2 = (float)(kDelta * kDelta);
#pragma unroll 2
    for (int jj = 0; jj < cnt; ++jj) {
        const float4 y = sp[jj];
        const float2 nx = make_float2(-y.x, -y.x), ny = make_float2(-y.y, -y.y), nz = make_float2(-y.z, -y.z);
        float2 qa = make_float2(y.w, y.w), qb, qc;
        if (DIPOLE) {
            const float4 dq = sd[jj];
            qb = make_float2(dq.x, dq.x);
            qc = make_float2(dq.y, dq.y);
        }
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const float2 dx = __fadd2_rn(px[m], nx), dy = __fadd2_rn(py[m], ny), dz = __fadd2_rn(pz[m], nz);
            const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
            const float2 inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
            float2 v;
            if (DIPOLE) {
                const float2 num = __ffma2_rn(qc, dz, __ffma2_rn(qb, dy, __fmul2_rn(qa, dx)));
                v = __fmul2_rn(num, __fmul2_rn(__fmul2_rn(inv, inv), inv));
            } else {
                v = __fmul2_rn(qa, inv);
            }
            if (NEAR) {
                v.x = r2.x >= d2 ? v.x : 0.f;
                v.y = r2.y >= d2 ? v.y : 0.f;
            }
            acc[m] = __fadd2_rn(acc[m], v);
        }
    }
}

//
// A block holds the whole check potential of its box, so it also writes the box's input
// for the tensor-core projection that follows: the potential scaled by the power of two
// that puts its largest entry into [2^14, 2^15) (exponent in bexp[b]) and split into
// FP16 hi and lo terms (Qp per box, zero past Q) -- the box split done in the producer.
template <bool DIPOLE, int NP, int NT>
__global__ void __launch_bounds__(NT)
k_surf_f(const int* __restrict__ boxes, const int* __restrict__ off, const int* __restrict__ idx, int down,
         const float4* __restrict__ bcf, const int64_t* __restrict__ rng, const float* __restrict__ sxf, int64_t ns,
         const float* __restrict__ qs, const float* __restrict__ surf, int Q, int Qp, __half* __restrict__ vin_h,
         __half* __restrict__ vin_l, int* __restrict__ bexp) {
    __shared__ float4 sp[NT];
    __shared__ float4 sd[DIPOLE ? NT : 1];
    const int b = boxes[blockIdx.x];
    const float4 bh = bcf[3 * b], bl = bcf[3 * b + 1], br = bcf[3 * b + 2];
    const float rf = down ? br.y : br.x;
    float2 px[NP], py[NP], pz[NP], acc[NP];
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
        for (int64_t j0 = sb; j0 < se; j0 += NT) {
            const int64_t j = j0 + threadIdx.x;
            if (j < se) {
                sp[threadIdx.x] = make_float4((sxf[j] - bh.x) + (sxf[3 * ns + j] - bl.x),
                                              (sxf[ns + j] - bh.y) + (sxf[4 * ns + j] - bl.y),
                                              (sxf[2 * ns + j] - bh.z) + (sxf[5 * ns + j] - bl.z), qs[j]);
                if (DIPOLE) sd[threadIdx.x] = make_float4(qs[ns + j], qs[2 * ns + j], 0.f, 0.f);
            }
            __syncthreads();
            const int cnt = (int)((se - j0) < (int64_t)NT ? (se - j0) : (int64_t)NT);
            if (near)
                surf_pairs<true, DIPOLE, NP>(sp, sd, cnt, px, py, pz, acc);
            else
                surf_pairs<false, DIPOLE, NP>(sp, sd, cnt, px, py, pz, acc);
            __syncthreads();
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
        switch (slots * 2 + (dl ? 1 : 0)) {
#define KF_SURF(NP, NT)                                                                                          \
    case 2 * (2 * NP * NT):                                                                                      \
        k_surf_f<false, NP, NT><<<nbox, NT, 0, s>>>(boxes, off, idx, down, P.bcf.p, T.rng.p, P.sxf.p, T.ns, q, sf,   \
                                                    npts, stride, P.sin_h.p, P.sin_l.p, P.sexp.p);               \
        break;                                                                                                   \
    case 2 * (2 * NP * NT) + 1:                                                                                  \
        k_surf_f<true, NP, NT><<<nbox, NT, 0, s>>>(boxes, off, idx, down, P.bcf.p, T.rng.p, P.sxf.p, T.ns, q, sf,    \
                                                   npts, stride, P.sin_h.p, P.sin_l.p, P.sexp.p);                \
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
// KIND 0: q/r   1: (q n_j).(x - y)/r^3   2: q n_i.(x - y)/r^3
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
        Real acc = 0;
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
                    if (KIND == 0) v = s0[jj] * inv;
                    else if (KIND == 1) v = (s0[jj] * dx + s1[jj] * dy + s2[jj] * dz) * (inv * inv * inv);
                    else v = s0[jj] * (nx * dx + ny * dy + nz * dz) * (inv * inv * inv);
                    acc += (r2 >= d2) ? v : (Real)0;
                }
                __syncthreads();
            }
        }
        if (valid) out[tperm[t]] = (double)(acc + res[t]);
    }
}

// FP32 near field, one warp per target leaf.  Lanes form 4 source groups of 8: lane
// (g, r) holds targets t0 + 8 i + r (i < T) of the current pass of at most 64 targets and
// takes sources j = g, g + 4, ... of every 32 staged by the warp; the four partial sums
// of a target meet by shuffles at the end.  Staged sources are float4 (position relative
// to the leaf centre and q -- or q n_j for the double layer, spread over two float4), so
// one shared-memory broadcast load feeds T pair evaluations.  Source positions come as
// FP32 hi/lo pairs (split once per plan) and the offset from the leaf centre is formed
// from them in FP32, to within 2 ulp of that offset, with no FP64 arithmetic per pair or
// per staged source.  A lane's targets are packed in pairs (the last pair of an odd
// count repeats a target and drops it), so each step is one FP32x2 instruction for two
// pair evaluations, with the scalar form's round-to-nearest operations.
// Work is split into units of at most kP2PUnitSrc sources of one leaf (its U- and
// W-list source ranges, cut where needed) and the units run heaviest first: on
// adaptive geometries a few leaves next to dense regions carry W lists of tens of
// thousands of sources, and one warp per leaf left them running alone at the end.  A
// leaf with several units adds into its outputs with FP64 atomics (the output is
// zeroed first); the first unit also adds the far field.
constexpr int kP2PWarps = 8;
constexpr long long kFarRange = 1LL << 62;   // range flag: W/X sources, not adjacent to the leaf
constexpr int kP2PUnitSrc = 2048;
// Larger target leaves go to the block kernel (a thread per target, sources staged once
// per leaf): at leaf 128 on the 64-sphere pack it takes 2.56 ms against 4.04 ms for two
// 64-target passes of this kernel, and 3.70 ms for a packed variant with two targets
// per thread and half the threads.
constexpr int kP2PWarpMaxLeaf = 64;

template <int KIND, int T>
__device__ __forceinline__ void p2p_pass(int lane, int e0, int e1, const longlong2* __restrict__ ranges,
                                         int flags, double cx, double cy, double cz,
                                         const float* __restrict__ sxf, int64_t ns,
                                         const double* __restrict__ txyz, int64_t nt,
                                         const float* __restrict__ qs, const float* __restrict__ tnrm,
                                         const float* __restrict__ res, const int64_t* __restrict__ tperm,
                                         double* __restrict__ out, int64_t t0, int64_t te, float4* st) {
    const int g = lane >> 3, r = lane & 7;
    constexpr int TP = (T + 1) / 2;
    float2 tx[TP], ty[TP], tz[TP], acc[TP], nx[TP], ny[TP], nz[TP];
#pragma unroll
    for (int m = 0; m < TP; ++m) {
        float c[2][6];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int64_t t = t0 + 8 * (2 * m + h) + r;
            t = t < te ? t : t0;                  // padding slots evaluate a real target, unused
            c[h][0] = (float)(txyz[t] - cx);
            c[h][1] = (float)(txyz[nt + t] - cy);
            c[h][2] = (float)(txyz[2 * nt + t] - cz);
            if (KIND == 2) {
                c[h][3] = tnrm[t];
                c[h][4] = tnrm[nt + t];
                c[h][5] = tnrm[2 * nt + t];
            }
        }
        tx[m] = make_float2(c[0][0], c[1][0]);
        ty[m] = make_float2(c[0][1], c[1][1]);
        tz[m] = make_float2(c[0][2], c[1][2]);
        if (KIND == 2) {
            nx[m] = make_float2(c[0][3], c[1][3]);
            ny[m] = make_float2(c[0][4], c[1][4]);
            nz[m] = make_float2(c[0][5], c[1][5]);
        }
        acc[m] = make_float2(0.f, 0.f);
    }
    // the leaf centre as FP32 hi + lo; a source's offset from it is (yh - ch) + (yl - cl)
    const float chx = (float)cx, chy = (float)cy, chz = (float)cz;
    const float clx = (float)(cx - (double)chx), cly = (float)(cy - (double)chy), clz = (float)(cz - (double)chz);
    const float d2 = (float)(kDelta * kDelta);
    // chunks of 32 sources over the leaf's source boxes, the next one prefetched into
    // registers while the current one is evaluated
    int e = e0;
    int64_t j0 = 0, se = 0;
    if (e < e1) {
        j0 = ranges[e].x & ~kFarRange;
        se = ranges[e].y;
    }
    float ph[3], pl[3], pq[3];
    auto fetch = [&](int64_t jb, int64_t je) {
        const int64_t j = jb + lane;
        if (j < je) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                ph[d] = sxf[d * ns + j];
                pl[d] = sxf[(3 + d) * ns + j];
            }
            pq[0] = qs[j];
            if (KIND == 1) {
                pq[1] = qs[ns + j];
                pq[2] = qs[2 * ns + j];
            }
        }
    };
    while (e < e1) {
        fetch(j0, se);
        const int64_t j = j0 + lane;
        if (j < se) {
            st[lane] = make_float4((ph[0] - chx) + (pl[0] - clx), (ph[1] - chy) + (pl[1] - cly),
                                   (ph[2] - chz) + (pl[2] - clz), pq[0]);
            if (KIND == 1) st[32 + lane] = make_float4(pq[1], pq[2], 0.f, 0.f);
        }
        const int cnt = (int)(se - j0 < 32 ? se - j0 : 32);
        // advance to the next chunk and prefetch it
        j0 += 32;
        while (j0 >= se && ++e < e1) {
            j0 = ranges[e].x & ~kFarRange;
            se = ranges[e].y;
        }
        __syncwarp();
#pragma unroll 1
        for (int jj = g; jj < cnt; jj += 4) {
            const float4 sp = st[jj];
            float4 sd = make_float4(0.f, 0.f, 0.f, 0.f);
            if (KIND == 1) sd = st[32 + jj];
            const float2 mx = make_float2(-sp.x, -sp.x), my = make_float2(-sp.y, -sp.y),
                         mz = make_float2(-sp.z, -sp.z), qa = make_float2(sp.w, sp.w);
#pragma unroll
            for (int m = 0; m < TP; ++m) {
                const float2 dx = __fadd2_rn(tx[m], mx), dy = __fadd2_rn(ty[m], my), dz = __fadd2_rn(tz[m], mz);
                const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                const float2 inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                float2 v;
                if (KIND == 0) {
                    v = __fmul2_rn(qa, inv);
                } else {
                    const float2 i3 = __fmul2_rn(__fmul2_rn(inv, inv), inv);
                    float2 num;
                    if (KIND == 1)
                        num = __ffma2_rn(make_float2(sd.y, sd.y), dz,
                                         __ffma2_rn(make_float2(sd.x, sd.x), dy, __fmul2_rn(qa, dx)));
                    else
                        num = __fmul2_rn(qa, __ffma2_rn(nz[m], dz, __ffma2_rn(ny[m], dy, __fmul2_rn(nx[m], dx))));
                    v = __fmul2_rn(num, i3);
                }
                v.x = r2.x >= d2 ? v.x : 0.f;
                v.y = r2.y >= d2 ? v.y : 0.f;
                acc[m] = __fadd2_rn(acc[m], v);
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int i = 0; i < T; ++i) {
        float v = (i & 1) ? acc[i >> 1].y : acc[i >> 1].x;
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        const int64_t t = t0 + 8 * i + r;
        if (g == 0 && t < te) {
            // res (the far field) is added here, or later by the caller when null
            const float far = res ? res[t] : 0.f;
            if (!(flags & 2)) out[tperm[t]] = (double)(v + far);                          // the leaf's only unit
            else atomicAdd(out + tperm[t], (double)((flags & 1) ? v + far : v));         // one of several
        }
    }
}

// ---- compensated near field (KIFMM_PREC_MIXED_CN), double and adjoint double layer.
// On a curved surface n.(x - y) between close neighbours is about |x - y|^2 / (2 R),
// far below |x - y|: plain FP32 loses the digits to cancellation (positions rounded to
// 2^-24 of the leaf size, normals or dipoles to 2^-24).  Here every offset from the
// leaf centre is a pair hi + lo with hi on a grid of 2^(e-19) (e: the leaf half-width's
// binade), so the difference of two hi parts is exact in FP32; normals and dipoles are
// hi + lo pairs too; the dot product of the hi parts is formed with error-free
// transformations (FMA two-products, two-sums) and the cross terms are added in FP32.
// W- and X-list sources (ranges flagged kFarRange) are not adjacent to the leaf, so
// there the plain FP32 evaluation (of the same hi + lo offsets) is accurate enough.
__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2b(float a) { return make_float2(a, a); }

// a . b (3-vectors, packed pairs) as hi + lo
__device__ __forceinline__ void dot3_ef(float2 ax, float2 ay, float2 az, float2 bx, float2 by, float2 bz,
                                        float2& hi, float2& lo) {
    const float2 p1 = __fmul2_rn(ax, bx), p2 = __fmul2_rn(ay, by), p3 = __fmul2_rn(az, bz);
    const float2 e1 = __ffma2_rn(ax, bx, f2neg(p1)), e2 = __ffma2_rn(ay, by, f2neg(p2)),
                 e3 = __ffma2_rn(az, bz, f2neg(p3));
    const float2 s = __fadd2_rn(p1, p2), z = __fadd2_rn(s, f2neg(p1));
    const float2 t1 = __fadd2_rn(__fadd2_rn(p1, f2neg(__fadd2_rn(s, f2neg(z)))), __fadd2_rn(p2, f2neg(z)));
    const float2 u = __fadd2_rn(s, p3), z2 = __fadd2_rn(u, f2neg(s));
    const float2 t2 = __fadd2_rn(__fadd2_rn(s, f2neg(__fadd2_rn(u, f2neg(z2)))), __fadd2_rn(p3, f2neg(z2)));
    hi = u;
    lo = __fadd2_rn(__fadd2_rn(__fadd2_rn(e1, e2), __fadd2_rn(e3, t1)), t2);
}

// x rounded to the grid of quantum g (|x| < 2^22 g), by the magic-number sum
__device__ __forceinline__ float grid_round(float x, float magic) { return __fsub_rn(__fadd_rn(x, magic), magic); }

// A source's offset from the leaf centre as hi (on the grid) + lo, from its FP32
// hi/lo coordinates and the centre's.
__device__ __forceinline__ void src_offset_ef(float ph, float pl, float ch, float cl, float magic, float& oh,
                                              float& ol) {
    const float a = __fsub_rn(ph, ch);                         // two-sum of ph and -ch
    const float bb = __fsub_rn(a, ph);
    const float err = __fadd_rn(__fsub_rn(ph, __fsub_rn(a, bb)), __fsub_rn(-ch, bb));
    const float rest = __fadd_rn(__fsub_rn(pl, cl), err);
    oh = grid_round(a, magic);
    ol = __fadd_rn(__fsub_rn(a, oh), rest);
}

template <int KIND, int T>
__device__ __forceinline__ void p2p_pass_cn(int lane, int e0, int e1, const longlong2* __restrict__ ranges,
                                            int flags, double cx, double cy, double cz, float hbox,
                                            const float* __restrict__ sxf, int64_t ns,
                                            const double* __restrict__ txyz, int64_t nt,
                                            const float* __restrict__ qs, const double* __restrict__ tnrm_d,
                                            const float* __restrict__ res, const int64_t* __restrict__ tperm,
                                            double* __restrict__ out, int64_t t0, int64_t te, float4* st) {
    static_assert(KIND == 1 || KIND == 2, "compensated form for the double layers");
    const int g = lane >> 3, r = lane & 7;
    constexpr int TP = (T + 1) / 2;
    const double quantum = ldexp(1.0, ilogbf(hbox) - 19);
    const float magic = (float)(1.5 * 8388608.0 * quantum);    // 1.5 * 2^23 * quantum
    float2 thx[TP], thy[TP], thz[TP], tlx[TP], tly[TP], tlz[TP], acc[TP];
    float2 nhx[TP], nhy[TP], nhz[TP], nlx[TP], nly[TP], nlz[TP];
#pragma unroll
    for (int m = 0; m < TP; ++m) {
        float c[2][12];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int64_t t = t0 + 8 * (2 * m + h) + r;
            t = t < te ? t : t0;                  // padding slots evaluate a real target, unused
            const double o[3] = {txyz[t] - cx, txyz[nt + t] - cy, txyz[2 * nt + t] - cz};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double oh = rint(o[d] / quantum) * quantum;
                c[h][d] = (float)oh;
                c[h][3 + d] = (float)(o[d] - oh);
                if (KIND == 2) {
                    const double nd = tnrm_d[d * nt + t];
                    c[h][6 + d] = (float)nd;
                    c[h][9 + d] = (float)(nd - (double)(float)nd);
                }
            }
        }
        thx[m] = make_float2(c[0][0], c[1][0]);
        thy[m] = make_float2(c[0][1], c[1][1]);
        thz[m] = make_float2(c[0][2], c[1][2]);
        tlx[m] = make_float2(c[0][3], c[1][3]);
        tly[m] = make_float2(c[0][4], c[1][4]);
        tlz[m] = make_float2(c[0][5], c[1][5]);
        if (KIND == 2) {
            nhx[m] = make_float2(c[0][6], c[1][6]);
            nhy[m] = make_float2(c[0][7], c[1][7]);
            nhz[m] = make_float2(c[0][8], c[1][8]);
            nlx[m] = make_float2(c[0][9], c[1][9]);
            nly[m] = make_float2(c[0][10], c[1][10]);
            nlz[m] = make_float2(c[0][11], c[1][11]);
        }
        acc[m] = make_float2(0.f, 0.f);
    }
    const float chx = (float)cx, chy = (float)cy, chz = (float)cz;
    const float clx = (float)(cx - (double)chx), cly = (float)(cy - (double)chy), clz = (float)(cz - (double)chz);
    const float d2 = (float)(kDelta * kDelta);
    int e = e0;
    int64_t j0 = 0, se = 0;
    bool far = false;
    if (e < e1) {
        j0 = ranges[e].x & ~kFarRange;
        far = (ranges[e].x & kFarRange) != 0;
        se = ranges[e].y;
    }
    while (e < e1) {
        const int64_t j = j0 + lane;
        if (j < se) {
            float oh[3], ol[3];
            src_offset_ef(sxf[j], sxf[3 * ns + j], chx, clx, magic, oh[0], ol[0]);
            src_offset_ef(sxf[ns + j], sxf[4 * ns + j], chy, cly, magic, oh[1], ol[1]);
            src_offset_ef(sxf[2 * ns + j], sxf[5 * ns + j], chz, clz, magic, oh[2], ol[2]);
            // A: (offset hi, q or dipole hi x), B: (offset lo, dipole hi y), C: (dipole hi z, dipole lo)
            st[lane] = make_float4(oh[0], oh[1], oh[2], qs[j]);
            if (KIND == 1) {
                st[32 + lane] = make_float4(ol[0], ol[1], ol[2], qs[ns + j]);
                st[64 + lane] = make_float4(qs[2 * ns + j], qs[3 * ns + j], qs[4 * ns + j], qs[5 * ns + j]);
            } else {
                st[32 + lane] = make_float4(ol[0], ol[1], ol[2], 0.f);
            }
        }
        const int cnt = (int)(se - j0 < 32 ? se - j0 : 32);
        const bool chunk_far = far;               // a chunk lies within one range
        j0 += 32;
        while (j0 >= se && ++e < e1) {
            j0 = ranges[e].x & ~kFarRange;
            far = (ranges[e].x & kFarRange) != 0;
            se = ranges[e].y;
        }
        __syncwarp();
#pragma unroll 1
        for (int jj = g; jj < cnt; jj += 4) {
            const float4 sa = st[jj], sb = st[32 + jj];
            float4 sc = make_float4(0.f, 0.f, 0.f, 0.f);
            if (KIND == 1) sc = st[64 + jj];
#pragma unroll
            for (int m = 0; m < TP; ++m) {
                // d = t - s as hi (exact: both on the grid) + lo
                const float2 dhx = __fadd2_rn(thx[m], f2b(-sa.x)), dhy = __fadd2_rn(thy[m], f2b(-sa.y)),
                             dhz = __fadd2_rn(thz[m], f2b(-sa.z));
                const float2 dlx = __fadd2_rn(tlx[m], f2b(-sb.x)), dly = __fadd2_rn(tly[m], f2b(-sb.y)),
                             dlz = __fadd2_rn(tlz[m], f2b(-sb.z));
                const float2 dx = __fadd2_rn(dhx, dlx), dy = __fadd2_rn(dhy, dly), dz = __fadd2_rn(dhz, dlz);
                const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
                const float2 inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                const float2 i3 = __fmul2_rn(__fmul2_rn(inv, inv), inv);
                if (chunk_far) {                  // W/X sources: no cancellation worth the cost
                    const float2 num = KIND == 1
                        ? __ffma2_rn(f2b(sc.x), dz, __ffma2_rn(f2b(sb.w), dy, __fmul2_rn(f2b(sa.w), dx)))
                        : __fmul2_rn(f2b(sa.w), __ffma2_rn(nhz[m], dz, __ffma2_rn(nhy[m], dy, __fmul2_rn(nhx[m], dx))));
                    float2 v = __fmul2_rn(num, i3);
                    v.x = r2.x >= d2 ? v.x : 0.f;
                    v.y = r2.y >= d2 ? v.y : 0.f;
                    acc[m] = __fadd2_rn(acc[m], v);
                    continue;
                }
                float2 hi, lo, corr;
                if (KIND == 1) {                  // (q n_j) . d, dipole hi (sa.w, sb.w, sc.x), lo (sc.y..w)
                    dot3_ef(f2b(sa.w), f2b(sb.w), f2b(sc.x), dhx, dhy, dhz, hi, lo);
                    corr = __ffma2_rn(f2b(sa.w), dlx, __ffma2_rn(f2b(sb.w), dly, __fmul2_rn(f2b(sc.x), dlz)));
                    corr = __ffma2_rn(f2b(sc.y), dhx, __ffma2_rn(f2b(sc.z), dhy, __ffma2_rn(f2b(sc.w), dhz, corr)));
                } else {                          // n_i . d, normal hi / lo per target
                    dot3_ef(nhx[m], nhy[m], nhz[m], dhx, dhy, dhz, hi, lo);
                    corr = __ffma2_rn(nhx[m], dlx, __ffma2_rn(nhy[m], dly, __fmul2_rn(nhz[m], dlz)));
                    corr = __ffma2_rn(nlx[m], dhx, __ffma2_rn(nly[m], dhy, __ffma2_rn(nlz[m], dhz, corr)));
                }
                float2 v = __fadd2_rn(hi, __fadd2_rn(lo, corr));
                v = KIND == 1 ? __fmul2_rn(v, i3) : __fmul2_rn(__fmul2_rn(f2b(sa.w), v), i3);
                v.x = r2.x >= d2 ? v.x : 0.f;
                v.y = r2.y >= d2 ? v.y : 0.f;
                acc[m] = __fadd2_rn(acc[m], v);
            }
        }
        __syncwarp();
    }
#pragma unroll
    for (int i = 0; i < T; ++i) {
        float v = (i & 1) ? acc[i >> 1].y : acc[i >> 1].x;
        v += __shfl_xor_sync(0xffffffffu, v, 8);
        v += __shfl_xor_sync(0xffffffffu, v, 16);
        const int64_t t = t0 + 8 * i + r;
        if (g == 0 && t < te) {
            const float far = res ? res[t] : 0.f;
            if (!(flags & 2)) out[tperm[t]] = (double)(v + far);
            else atomicAdd(out + tperm[t], (double)((flags & 1) ? v + far : v));
        }
    }
}

template <int KIND, bool CN>
__global__ void __launch_bounds__(32 * kP2PWarps)
k_p2p_warp(const int* __restrict__ leaves, int nunits, const int4* __restrict__ units,
           const longlong2* __restrict__ ranges, const int64_t* __restrict__ rng, const double* __restrict__ ctr,
           const float* __restrict__ sxf,
           int64_t ns, const double* __restrict__ txyz, int64_t nt, const float* __restrict__ qs,
           const float* __restrict__ tnrm, const double* __restrict__ tnrm_d, const float4* __restrict__ bcf,
           const float* __restrict__ res, const int64_t* __restrict__ tperm, double* __restrict__ out) {
    __shared__ float4 stage[kP2PWarps][CN ? (KIND == 1 ? 96 : 64) : (KIND == 1 ? 64 : 32)];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ui = blockIdx.x * kP2PWarps + warp;
    if (ui >= nunits) return;                     // whole warp; no block-wide barrier below
    const int4 u = units[ui];                     // (leaf, first range, end range, flags)
    const int b = leaves[u.x];
    const double cx = ctr[3 * b], cy = ctr[3 * b + 1], cz = ctr[3 * b + 2];
    const int64_t tb = rng[4 * b + 2], te = rng[4 * b + 3];
    const int e0 = u.y, e1 = u.z;
    float4* st = stage[warp];
    // passes of up to 8 kMaxT targets (the compensated form keeps four per lane)
    constexpr int kMaxT = CN ? 4 : 8;
    for (int64_t t0 = tb; t0 < te; t0 += 8 * kMaxT) {
        const int n = (int)(te - t0 < 8 * kMaxT ? te - t0 : 8 * kMaxT);
        const int64_t tend = t0 + n;
        switch ((n + 7) >> 3) {
#define KF_PASS(TT)                                                                                        \
    case TT:                                                                                               \
        if constexpr (TT <= kMaxT) {                                                                       \
            if constexpr (CN)                                                                              \
                p2p_pass_cn<KIND == 0 ? 1 : KIND, TT>(lane, e0, e1, ranges, u.w, cx, cy, cz, bcf[3 * b].w, sxf, \
                                                      ns, txyz, nt, qs, tnrm_d, res, tperm, out, t0, tend, st); \
            else                                                                                           \
                p2p_pass<KIND, TT>(lane, e0, e1, ranges, u.w, cx, cy, cz, sxf, ns, txyz, nt, qs, tnrm, res,  \
                                   tperm, out, t0, tend, st);                                              \
        }                                                                                                  \
        break;
            KF_PASS(1) KF_PASS(2) KF_PASS(3) KF_PASS(4) KF_PASS(5) KF_PASS(6) KF_PASS(7) KF_PASS(8)
#undef KF_PASS
        }
    }
}

// out[tperm[t]] += res[t]: the far field, after a near field that ran beside it.
__global__ void k_add_far(const int64_t* __restrict__ tperm, const float* __restrict__ res, int64_t nt,
                          double* __restrict__ out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < nt) out[tperm[t]] += (double)res[t];
}

// f[i] = near[i] + res[itperm[i]] in input order (res null: f[i] = near[i]), written
// once and in order, so f may be a host buffer.
__global__ void k_add_far_io(const int64_t* __restrict__ itperm, const float* __restrict__ res,
                             const double* __restrict__ near, int64_t nt, double* __restrict__ f) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nt) return;
    f[i] = res ? near[i] + (double)res[itperm[i]] : near[i];
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

__global__ void k_gather_nrm(const double* __restrict__ nrm, const int64_t* __restrict__ perm, int64_t n,
                             double* __restrict__ outd, float* __restrict__ outf) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    for (int d = 0; d < 3; ++d) {
        double v = nrm[d * n + j];
        if (outd) outd[d * n + i] = v;
        if (outf) outf[d * n + i] = (float)v;
    }
}

// D2T row descriptors: target position in its leaf's unit frame, its normal, scale.
__global__ void k_d2t_rows(const int* __restrict__ tleaf_of, int64_t nt, const double* __restrict__ txyz,
                           const double* __restrict__ tnrm, const int* __restrict__ lvl,
                           const double* __restrict__ ctr, double root_h, bool adl, double* apts,
                           double* anrm, double* ascale, int64_t* orow) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int b = tleaf_of[t];
    double r = ldexp(root_h, -lvl[b]);
    for (int d = 0; d < 3; ++d) {
        apts[3 * t + d] = (txyz[d * nt + t] - ctr[3 * b + d]) / r;
        anrm[3 * t + d] = adl ? tnrm[d * nt + t] : 0.0;
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

void make_tiles(std::vector<Triple>& tr, std::vector<int4>& tiles, std::vector<int>& pin,
                std::vector<int>& pout, int cap) {
    std::stable_sort(tr.begin(), tr.end(), [](const Triple& a, const Triple& b) { return a.op < b.op; });
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
    std::stable_sort(tr.begin(), tr.end(),
                     [](const Triple& a, const Triple& b) { return a.out != b.out ? a.out < b.out : a.op < b.op; });
    // targets by (level, offsets of the V list), members in box order
    std::map<std::pair<int, std::vector<int>>, std::vector<std::pair<int, size_t>>> groups;
    for (size_t i = 0; i < tr.size();) {
        size_t j = i;
        std::vector<int> sig;
        while (j < tr.size() && tr[j].out == tr[i].out) sig.push_back(tr[j++].op);
        groups[{level[tr[i].out], sig}].push_back({tr[i].out, i});
        i = j;
    }
    std::vector<std::vector<int4>> chains;
    std::vector<int> cpin, cpout;
    std::vector<char> chained(tr.size(), 0);
    for (auto& kv : groups) {
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
        bool center = P.kernel == KIFMM_KERNEL_ADL && which != 0;
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
    const bool adl = P.kernel == KIFMM_KERNEL_ADL;
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
int build_d2t(Plan& P, const HostPinv& h, bool factored, int Kd, const std::vector<int>& tleaf_of, Real* out,
              cudaStream_t s) {
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
    bool adl = P.kernel == KIFMM_KERNEL_ADL;
    k_d2t_rows<<<div_up(nt, 256), 256, 0, s>>>(dleaf.p, nt, txyz, adl ? P.tnrm_d.p : nullptr, T.lvl.p,
                                               T.ctr.p, T.root_h, adl, apts.p, anrm.p, ascale.p, orow.p);
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
    const bool centered = P.kernel == KIFMM_KERNEL_ADL;
    std::lock_guard<std::mutex> lock(mu);
    for (auto it = cache.begin(); it != cache.end();) {
        std::shared_ptr<OpTables> t = it->lock();
        if (!t) {
            it = cache.erase(it);
            continue;
        }
        if (t->device == dev && t->p == P.p && t->cutoff == P.cutoff && t->fp64 == P.fp64 &&
            t->centered == centered) {
            P.ops = t;
            return KIFMM_OK;
        }
        ++it;
    }
    auto t = std::make_shared<OpTables>();
    t->device = dev;
    t->p = P.p;
    t->cutoff = P.cutoff;
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
        t->ru = h.ru;
        t->rd = h.rd;
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
    const HostPinv& h = host_pinv(P.p, P.cutoff);
    P.Q = h.Q;
    P.Qp = (h.Q + 15) / 16 * 16;
    P.fp64 = P.prec == KIFMM_PREC_FP64;
    P.cnear = P.prec == KIFMM_PREC_MIXED_CN && P.kernel != KIFMM_KERNEL_SL;
    KF_TRY(P.err.alloc(1));
    KF_CHECK_CUDA(cudaMemsetAsync(P.err.p, 0, sizeof(int), s));

    // sorted normals
    if (P.kernel == KIFMM_KERNEL_DL) {
        KF_TRY(P.snrm.alloc(3 * T.ns));
        k_gather_nrm<<<div_up(T.ns, 256), 256, 0, s>>>(src_nrm, T.sperm.p, T.ns, P.snrm.p, nullptr);
        KF_CHECK_LAUNCH();
    }
    if (P.kernel == KIFMM_KERNEL_ADL) {
        const int64_t* tp = T.same ? T.sperm.p : T.tperm.p;
        KF_TRY(P.tnrm_d.alloc(3 * T.nt));
        if (!P.fp64) KF_TRY(P.tnrm_f.alloc(3 * T.nt));
        k_gather_nrm<<<div_up(T.nt, 256), 256, 0, s>>>(trg_nrm, tp, T.nt, P.tnrm_d.p,
                                                       P.fp64 ? nullptr : P.tnrm_f.p);
        KF_CHECK_LAUNCH();
    }

    // surfaces
    {
        std::vector<float> sf(h.surf.begin(), h.surf.end());
        KF_TRY(P.surf_d.upload(h.surf, s));
        KF_TRY(P.surf_f.upload(sf, s));
    }

    // operators: shared tables of this key, built once
    KF_TRY(get_tables(P, h, s));
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
        KF_TRY(P.bcf.alloc(3 * (size_t)T.nbox));
        k_box_f<<<div_up(T.nbox, 256), 256, 0, s>>>(T.ctr.p, T.lvl.p, T.root_h, T.nbox, P.bcf.p);
        KF_CHECK_LAUNCH();
    }

    // work lists (host bookkeeping over the tree's lists)
    std::vector<int> s2u_box, s2u_off{0}, s2u_idx, p2l_box, p2l_off{0}, p2l_idx, tleaf, p2p_off{0}, p2p_idx;
    std::vector<int> tleaf_of(T.nt, 0);
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
            for (int k = T.h_u_off[b]; k < T.h_u_off[b + 1]; ++k) p2p_idx.push_back(T.h_u_idx[k]);
            for (int k = T.h_w_off[b]; k < T.h_w_off[b + 1]; ++k) p2p_idx.push_back(T.h_w_idx[k]);
            if (x_direct)
                for (int k = T.h_x_off[b]; k < T.h_x_off[b + 1]; ++k) p2p_idx.push_back(T.h_x_idx[k]);
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
    // mixed: near-field work units of at most kP2PUnitSrc sources, heaviest first
    if (!P.fp64) {
        struct Unit {
            int4 u;
            int64_t work;
        };
        std::vector<Unit> units;
        std::vector<longlong2> ranges;
        for (size_t li = 0; li < tleaf.size(); ++li) {
            const int b = tleaf[li];
            const int64_t ntg = T.h_rng[4 * b + 3] - T.h_rng[4 * b + 2];
            const size_t u0 = units.size();
            int r0 = (int)ranges.size();
            int64_t cnt = 0;
            const int n_u = T.h_u_off[b + 1] - T.h_u_off[b];   // the U list comes first
            for (int k = p2p_off[li]; k < p2p_off[li + 1]; ++k) {
                const int a = p2p_idx[k];
                // W- and X-list boxes are not adjacent to the leaf; flagged when their
                // max-norm gap also exceeds twice the tolerance radius
                long long far = 0;
                if (k - p2p_off[li] >= n_u) {
                    const double ha = std::ldexp(T.root_h, -T.h_lvl[a]), hb = std::ldexp(T.root_h, -T.h_lvl[b]);
                    double dc = 0.0;
                    for (int d = 0; d < 3; ++d) {
                        const double ca = (2 * T.h_coord[3 * a + d] + 1) * ha, cb = (2 * T.h_coord[3 * b + d] + 1) * hb;
                        dc = std::max(dc, std::fabs(ca - cb));
                    }
                    if (dc - ha - hb > 2.0 * kDelta) far = kFarRange;
                }
                int64_t j0 = T.h_rng[4 * a], j1 = T.h_rng[4 * a + 1];
                while (j0 < j1) {
                    const int64_t take = std::min<int64_t>(j1 - j0, kP2PUnitSrc - cnt);
                    ranges.push_back(make_longlong2(j0 | far, j0 + take));
                    cnt += take;
                    j0 += take;
                    if (cnt == kP2PUnitSrc) {
                        units.push_back({make_int4((int)li, r0, (int)ranges.size(), 0), ntg * cnt});
                        r0 = (int)ranges.size();
                        cnt = 0;
                    }
                }
            }
            if (cnt > 0 || units.size() == u0)
                units.push_back({make_int4((int)li, r0, (int)ranges.size(), 0), ntg * cnt});
            const bool split = units.size() - u0 > 1;
            P.p2p_multi = P.p2p_multi || split;
            P.n_p2p_split += split ? 1 : 0;
            for (size_t i = u0; i < units.size(); ++i) units[i].u.w = (i == u0 ? 1 : 0) | (split ? 2 : 0);
        }
        std::stable_sort(units.begin(), units.end(), [](const Unit& x, const Unit& y) { return x.work > y.work; });
        std::vector<int4> hu(units.size());
        for (size_t i = 0; i < units.size(); ++i) hu[i] = units[i].u;
        KF_TRY(P.p2p_units.upload(hu, s));
        KF_TRY(P.p2p_ranges.upload(ranges, s));
        P.n_p2p_units = (int)hu.size();
    }

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
    }

    // per-target evaluation rows and buffers
    size_t nbq = (size_t)T.nbox * P.Qp;
    if (P.fp64) {
        KF_TRY(P.d2t_d.alloc((size_t)T.nt * P.Qp));
        KF_TRY(build_d2t<double>(P, h, false, 0, tleaf_of, P.d2t_d.p, s));
        KF_TRY(P.u_d.alloc(nbq));
        KF_TRY(P.d_d.alloc(nbq));
        KF_TRY(P.res_d.alloc(T.nt));
        KF_TRY(P.q_d.alloc(3 * T.ns));
    } else {
        // rows G W_d, reading the projected down-check potentials
        KF_TRY(P.d2t_f.alloc((size_t)T.nt * P.ops->Kd));
        KF_TRY(build_d2t<float>(P, h, true, P.ops->Kd, tleaf_of, P.d2t_f.p, s));
        // (no FP32 check potentials: S2U and X write the projections' split inputs)
        KF_TRY(P.res_f.alloc(T.nt));
        KF_TRY(P.q_f.alloc((P.cnear ? 6 : 3) * T.ns));
    }
    KF_CHECK_CUDA(cudaStreamSynchronize(s));

    P.device_bytes = 0;
    for (size_t b : {(size_t)P.ops->bytes(), P.d2t_d.bytes(), P.d2t_f.bytes(), P.u_d.bytes(), P.d_d.bytes(),
                     P.res_d.bytes(), P.q_d.bytes(), P.u_f.bytes(), P.d_f.bytes(), P.res_f.bytes(),
                     P.q_f.bytes(), P.snrm.bytes(), P.tnrm_d.bytes(), P.tnrm_f.bytes(),
                     P.bexp.bytes(), P.vin_h.bytes(), P.vin_l.bytes(), P.sexp.bytes(), P.sin_h.bytes(),
                     P.sin_l.bytes(), P.sxf.bytes(), P.bcf.bytes(), P.zu.bytes(),
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
        // FP32 with leaves of up to 64 targets: a warp per leaf; larger leaves (and FP64):
        // a block per leaf, whose staged sources serve all of the leaf's targets at once
        bool done = false;
        if constexpr (std::is_same<Real, float>::value) {
          if (P.max_trg_leaf <= kP2PWarpMaxLeaf) {
            const unsigned grid = (unsigned)((P.n_p2p_units + kP2PWarps - 1) / kP2PWarps);
            if (P.p2p_multi) {
                KF_CHECK_CUDA(cudaMemsetAsync(out, 0, (size_t)T.nt * sizeof(double), ns));
                ++launches;
            }
#define KF_P2PW(KIND, CN)                                                                                    \
    k_p2p_warp<KIND, CN><<<grid, 32 * kP2PWarps, 0, ns>>>(P.tleaf.p, P.n_p2p_units, P.p2p_units.p,           \
                                                          P.p2p_ranges.p, T.rng.p, T.ctr.p, P.sxf.p, T.ns, txyz, \
                                                          T.nt, B.q, B.tnrm, P.tnrm_d.p, P.bcf.p, res, tperm, out)
            if (P.kernel == KIFMM_KERNEL_SL) KF_P2PW(0, false);
            else if (P.kernel == KIFMM_KERNEL_DL) {
                if (P.cnear) KF_P2PW(1, true);
                else KF_P2PW(1, false);
            } else {
                if (P.cnear) KF_P2PW(2, true);
                else KF_P2PW(2, false);
            }
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
        else KF_P2P(2);
#undef KF_P2P
        }
        KF_CHECK_LAUNCH();
        ++launches;
        return KIFMM_OK;
    };
    // mixed, warp near field: it runs on its own stream beside the far field (forked
    // after the gather) and the far field is added once both are done
    const bool near_overlap = std::is_same<Real, float>::value && P.n_tleaf && P.near_stream &&
                              P.max_trg_leaf <= kP2PWarpMaxLeaf;
    const bool dl = P.kernel == KIFMM_KERNEL_DL;
    KF_TRY(mark(0));
    if (P.io_in)
        k_scatter_q<Real><<<div_up(T.ns, 256), 256, 0, s>>>(q, P.isperm.p, T.ns, dl ? P.snrm.p : nullptr, B.q,
                                                            P.cnear && dl);
    else
        k_gather_q<Real><<<div_up(T.ns, 256), 256, 0, s>>>(q, T.sperm.p, T.ns, dl ? P.snrm.p : nullptr, B.q,
                                                           P.cnear && dl);
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
        KF_CHECK_CUDA(cudaMemsetAsync(up, 0, P.zu.bytes(), s));
        KF_CHECK_CUDA(cudaMemsetAsync(dn, 0, P.zd.bytes(), s));
        launches += 2;
    }
    KF_TRY(mark(1));
    // S2U
    if (P.n_s2u) {
        KF_TRY(launch_surf<Real>(P, T, dl, P.n_s2u, P.s2u_box.p, P.s2u_off.p, P.s2u_idx.p, kUpCheck, B.q, B.surf,
                                 B.u, s));
        ++launches;
    }
    if (near_overlap) KF_TRY(fork_near());
    KF_TRY(mark(2));
    // mixed: the leaves' projections; U2U, deepest parents first
    if constexpr (mixed) KF_TRY(project(P, 3, P.proj_up, up, s, launches));
    for (int l = T.nlev - 1; l >= 2; --l)
        KF_TRY(run_pairs<Real>(P, kU2U, P.u2u, P.u2u.level_tile[l], P.u2u.level_tile[l + 1], B.m2m, up, up,
                               T.level_off[std::min(l + 1, T.nlev)], T.level_off[std::min(l + 2, T.nlev)], s,
                               launches));
    KF_TRY(mark(3));
    // X list (mixed: then the X boxes' projections), then V list
    if (P.n_p2l) {
        KF_TRY(launch_surf<Real>(P, T, dl, P.n_p2l, P.p2l_box.p, P.p2l_off.p, P.p2l_idx.p, kDnCheck, B.q, B.surf,
                                 B.d, s));
        ++launches;
        if constexpr (mixed) KF_TRY(project(P, 4, P.proj_x, dn, s, launches));
    }
    KF_TRY(mark(4));
    // the upward pass split levels 3 and deeper (mixed); level 2 is split here
    KF_TRY(run_pairs<Real>(P, kM2L, P.m2l, 0, P.m2l.ntiles, B.m2l, up, dn, T.level_off[std::min(2, T.nlev)],
                           T.level_off[std::min(3, T.nlev)], s, launches));
    KF_TRY(mark(5));
    // L2L, coarsest children first (ADL in FP64: each level's potentials shifted to zero
    // mean first; the mixed tables carry that centring)
    const bool center = !mixed && P.kernel == KIFMM_KERNEL_ADL;
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
        k_d2t<Real><<<P.n_tleaf, 128, dw * sizeof(Real), s>>>(P.tleaf.p, T.rng.p, B.d2t, dn, dw, B.res);
        KF_CHECK_LAUNCH();
        ++launches;
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
                                                                     out, T.nt, P.io_out);
        else
            k_add_far<<<(unsigned)div_up(T.nt, 256), 256, 0, s>>>(T.same ? T.sperm.p : T.tperm.p,
                                                                  reinterpret_cast<const float*>(B.res), T.nt, out);
        KF_CHECK_LAUNCH();
        ++launches;
    } else if (P.io_out) {
        k_add_far_io<<<(unsigned)div_up(T.nt, 256), 256, 0, s>>>(P.itperm.p, nullptr, out, T.nt, P.io_out);
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
    KF_ARG(kernel >= KIFMM_KERNEL_SL && kernel <= KIFMM_KERNEL_ADL, "unknown kernel");
    KF_ARG(p >= 2 && p <= 16, "p must be in [2, 16]");
    KF_ARG(precision == KIFMM_PREC_FP64 || precision == KIFMM_PREC_MIXED || precision == KIFMM_PREC_MIXED_CN,
           "unknown precision");
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
    P.p = p;
    P.prec = precision;
    P.cutoff = pinv_cutoff > 0 ? pinv_cutoff : (precision == KIFMM_PREC_FP64 ? 1e-9 : 1e-8);
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
    KF_TRY(P.out_stage.alloc(std::max<int64_t>(T.nt, 1)));
    if (T.ns) k_invert_perm<<<(unsigned)div_up(T.ns, 256), 256, 0, s>>>(T.sperm.p, T.ns, P.isperm.p);
    if (T.nt)
        k_invert_perm<<<(unsigned)div_up(T.nt, 256), 256, 0, s>>>(T.same ? T.sperm.p : T.tperm.p, T.nt,
                                                                   P.itperm.p);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

}  // namespace
}  // namespace kifmm

extern "C" int kifmm_fmm_matvec_graph(kifmm_plan plan, const double* q, double* out, void* stream) {
    clear_error();
    KF_ARG(plan && q && out, "NULL plan, q or out");
    Plan& P = plan->P;
    if (!P.gexec || P.g_q != q || P.g_out != out) {
        KF_TRY(capture_matvec(P, q, out, &P.gexec));
        P.g_q = q;
        P.g_out = out;
    }
    KF_CHECK_CUDA(cudaGraphLaunch(P.gexec, (cudaStream_t)stream));
    return KIFMM_OK;
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
        KF_CHECK_CUDA(cudaMemcpyAsync(out, P.out_stage.p, T.nt * sizeof(double), cudaMemcpyDeviceToHost, s));
    return KIFMM_OK;
}

extern "C" int kifmm_plan_get_stats(kifmm_plan plan, kifmm_plan_stats* st) {
    clear_error();
    KF_ARG(plan && st, "NULL plan or stats");
    const Plan& P = plan->P;
    st->kernel = P.kernel;
    st->p = P.p;
    st->q_points = P.Q;
    st->precision = P.prec;
    st->pinv_cutoff = P.cutoff;
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
    st->near_overlap = (!P.fp64 && P.near_stream && P.n_tleaf && P.max_trg_leaf <= kP2PWarpMaxLeaf) ? 1 : 0;
    st->s2u_points = (P.fp64 || !P.ops) ? P.Q : P.ops->ks;
    st->m2l_chain_pairs = P.m2l_chain_pairs;
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
