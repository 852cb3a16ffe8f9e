// Boundary-integral operators on top of the FMM matvec, and matrix-free GMRES.
//
// Polarization (Sec. II.C, Eqs. Ax, Eb, pol_discret, rhs), eps_0 = 1:
//   (A s)_j = ebar_j s_j + deps_j (1/4pi) [ ADL(s * a)_j + c_j s_j ]
//   ebar_j = (eps_j + eps_out)/2, deps_j = eps_out - eps_j, c_j = H_j sqrt(pi a_j)
// The self term of Eq. pol_discret is read as c_j s_j: the principal-value normal
// field at the centre of a disc of area a_j on a surface of mean curvature H_j with
// unit density is pi rho H, rho = sqrt(a_j/pi).
// Surface field and body force (Sec. II.C, Eq. Eb with the discretization of Eq.
// pol_discret, and the force on a body from its surface force density eps_m sigma E):
//   E^j = E0 + (1/4pi) [ FIELD(sigma * a)_j + c_j sigma_j n_j ],  F_b = sum_{j in b} eps_out sigma_j E^j a_j
// Right-hand side with free surface charge (Eq. rhs, Eq. Ef without its volume term):
//   b_j = (1 - ebar_j) sf_j - deps_j [ E0 . n_j + (1/4pi) ( ADL(sf * a)_j + c_j sf_j ) ]
// Demagnetization (Sec. II.B, Eq. fk_integral_discrete):
//   phi2_i = DL(phi1 * w)_i / 4pi + (Omega_i/4pi - 1) phi1_i
// GMRES (Sec. III: PETSc GMRES in matrix-free form; here restarted GMRES(m) of Saad &
// Schultz with classical Gram-Schmidt applied twice) keeps its Krylov basis, the
// orthogonalization and the residuals in FP64 on the device; only the small
// Hessenberg least-squares problem runs on the host.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"
#include "plan.cuh"

namespace kifmm {
int plan_matvec(Plan& P, const double* q, double* out, cudaStream_t s);
int plan_matvec_graph(Plan& P, const double* q, double* out, cudaStream_t s);
}

using namespace kifmm;

namespace {

constexpr double kPi = 3.14159265358979323846;

__global__ void k_mul(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                      double* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] * b[i];
}

// y = ebar x + deps (adl + c x)/4pi, adl already in y.
__global__ void k_polar_combine(const double* __restrict__ x, const double* __restrict__ area,
                                const double* __restrict__ eps_in, double eps_out,
                                const double* __restrict__ curv, int64_t n, double* __restrict__ y) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double ebar = 0.5 * (eps_in[i] + eps_out), deps = eps_out - eps_in[i];
    double c = curv[i] * sqrt(kPi * area[i]);
    y[i] = ebar * x[i] + deps * (y[i] + c * x[i]) / (4.0 * kPi);
}

// E[k n + i] = e0_k + (E[k n + i] + c_i sigma_i n_k,i) / 4pi: the raw field sum of
// sigma a (already in E) completed with the self-patch term and the applied field.
__global__ void k_field_combine(const double* __restrict__ sigma, const double* __restrict__ area,
                                const double* __restrict__ curv, const double* __restrict__ nrm, double ex, double ey,
                                double ez, int64_t n, double* __restrict__ E) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double cs = curv[i] * sqrt(kPi * area[i]) * sigma[i];
    const double e0[3] = {ex, ey, ez};
    for (int k = 0; k < 3; ++k) E[k * n + i] = e0[k] + (E[k * n + i] + cs * nrm[k * n + i]) / (4.0 * kPi);
}

// F[3 b + k] += eps_out sigma_i E_k,i a_i over the elements i of body b.  Bodies up to
// kForceBins are summed per block in shared memory first (one FP64 atomic per body and
// block), more go straight to global FP64 atomics.
constexpr int kForceBins = 1024;
__global__ void __launch_bounds__(256) k_force(const double* __restrict__ sigma, const double* __restrict__ area,
                                               const double* __restrict__ E, const int* __restrict__ body,
                                               double eps_out, int64_t n, int n_body, double* __restrict__ F) {
    __shared__ double bins[3 * kForceBins];
    const bool shared = n_body <= kForceBins;
    if (shared)
        for (int k = threadIdx.x; k < 3 * n_body; k += blockDim.x) bins[k] = 0.0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = body[i];
        if (b < 0 || b >= n_body) continue;
        const double s = eps_out * sigma[i] * area[i];
        for (int k = 0; k < 3; ++k) {
            const double f = s * E[k * n + i];
            if (shared) atomicAdd(&bins[3 * b + k], f);
            else atomicAdd(&F[3 * b + k], f);
        }
    }
    __syncthreads();
    if (shared)
        for (int k = threadIdx.x; k < 3 * n_body; k += blockDim.x)
            if (bins[k] != 0.0) atomicAdd(&F[k], bins[k]);
}

// b = (1 - ebar) sf - deps (E0 . n + (adl + c sf)/4pi), adl (the raw ADL sum of sf a) in b.
__global__ void k_rhs_free(const double* __restrict__ nrm, const double* __restrict__ eps_in, double eps_out,
                           const double* __restrict__ sf, const double* __restrict__ area,
                           const double* __restrict__ curv, double ex, double ey, double ez, int64_t n,
                           double* __restrict__ b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double ebar = 0.5 * (eps_in[i] + eps_out), deps = eps_out - eps_in[i];
    const double c = curv[i] * sqrt(kPi * area[i]);
    const double en = ex * nrm[i] + ey * nrm[n + i] + ez * nrm[2 * n + i];
    b[i] = (1.0 - ebar) * sf[i] - deps * (en + (b[i] + c * sf[i]) / (4.0 * kPi));
}

__global__ void k_demag_combine(const double* __restrict__ phi1, const double* __restrict__ omega, int64_t n,
                                double* __restrict__ phi2) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    phi2[i] = phi2[i] / (4.0 * kPi) + (omega[i] / (4.0 * kPi) - 1.0) * phi1[i];
}

__global__ void k_rhs(const double* __restrict__ nrm, const double* __restrict__ eps_in, double eps_out,
                      double ex, double ey, double ez, int64_t n, double* __restrict__ b) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    b[i] = -(eps_out - eps_in[i]) * (ex * nrm[i] + ey * nrm[n + i] + ez * nrm[2 * n + i]);
}

// Reductions and updates of the GMRES vectors, per instance.  A forest's vectors hold
// its instances back to back (input order); every instance runs its own GMRES, so every
// dot product, combination and scaling acts on one instance's segment with that
// instance's coefficients.  A plan on one tree is the case of one instance.
//
// Dot products: block b sums V_j . w over the range [lo_b, hi_b) of one instance
// (ranges never straddle two instances) into partial[b nv + j]; the final pass adds the
// blocks of instance i into h[i hld + j].
__global__ void __launch_bounds__(256) k_dots(const double* __restrict__ V, int64_t ld, int nv,
                                              const double* __restrict__ w, const int64_t* __restrict__ blo,
                                              const int64_t* __restrict__ bhi, double* __restrict__ partial) {
    // eight vectors per pass over the block's range of w; per pass a warp-shuffle
    // reduction of the eight sums, then one across the block's warps
    constexpr int G = 8;
    __shared__ double red[8][G];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t lo = blo[blockIdx.x], hi = bhi[blockIdx.x];
    for (int i0 = 0; i0 < nv; i0 += G) {
        const int m = nv - i0 < G ? nv - i0 : G;
        double s[G];
#pragma unroll
        for (int j = 0; j < G; ++j) s[j] = 0.0;
        for (int64_t t = lo + threadIdx.x; t < hi; t += blockDim.x) {
            const double wt = w[t];
#pragma unroll
            for (int j = 0; j < G; ++j)
                if (j < m) s[j] += V[(size_t)(i0 + j) * ld + t] * wt;
        }
#pragma unroll
        for (int j = 0; j < G; ++j)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s[j] += __shfl_xor_sync(0xffffffffu, s[j], o);
        if (lane == 0)
#pragma unroll
            for (int j = 0; j < G; ++j) red[warp][j] = s[j];
        __syncthreads();
        if (threadIdx.x < m) {
            double a = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) a += red[q][threadIdx.x];
            partial[(size_t)blockIdx.x * nv + i0 + threadIdx.x] = a;
        }
        __syncthreads();
    }
}

// grid (nv, n_inst): h[i hld + j] = sum of partial[b nv + j] over the blocks of instance i
__global__ void k_dots_final(const double* __restrict__ partial, const int* __restrict__ inst_blk, int nv,
                             int hld, double* __restrict__ h) {
    const int j = blockIdx.x, i = blockIdx.y;
    __shared__ double red[128];
    double s = 0;
    for (int b = inst_blk[i] + threadIdx.x; b < inst_blk[i + 1]; b += blockDim.x) s += partial[(size_t)b * nv + j];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) h[(size_t)i * hld + j] = red[0];
}

// w += sign sum_j h[inst(t) hld + j] V_j   (inst = 0 without a point-to-instance map)
__global__ void k_combine(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ h, int hld,
                          double sign, int64_t n, const int* __restrict__ inst, double* __restrict__ w) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double* hi = h + (size_t)(inst ? inst[t] : 0) * hld;
    double s = 0;
    for (int i = 0; i < nv; ++i) s += hi[i] * V[(size_t)i * ld + t];
    w[t] += sign * s;
}

// out = a[inst(t)] x   (out may be x)
__global__ void k_scale(const double* __restrict__ a, const double* x, int64_t n, const int* __restrict__ inst,
                        double* out) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) out[t] = a[inst ? inst[t] : 0] * x[t];
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, const double* __restrict__ y, int64_t n,
                        double* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * x[i] + b * y[i];
}

// inst[t] = i for off[i] <= t < off[i + 1]
__global__ void k_point_instance(const int64_t* __restrict__ off, int ninst, int64_t n, int* __restrict__ inst) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    int lo = 0, hi = ninst;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (off[mid] <= t) lo = mid;
        else hi = mid;
    }
    inst[t] = lo;
}

struct Gmres {
    Plan& P;
    const double *area, *eps_in, *curv;
    double eps_out;
    int64_t n;
    cudaStream_t s;
    double* qbuf;
    bool graph = false;              // replay the plan's captured matvec (fixed qbuf and y)

    int apply(const double* x, double* y) {
        k_mul<<<div_up(n, 256), 256, 0, s>>>(x, area, n, qbuf);
        KF_CHECK_LAUNCH();
        if (graph) KF_TRY(plan_matvec_graph(P, qbuf, y, s));
        else KF_TRY(plan_matvec(P, qbuf, y, s));
        k_polar_combine<<<div_up(n, 256), 256, 0, s>>>(x, area, eps_in, eps_out, curv, n, y);
        KF_CHECK_LAUNCH();
        return KIFMM_OK;
    }
};

int check_plan_for(kifmm_plan plan, int kernel) {
    KF_ARG(plan != nullptr, "NULL plan");
    KF_ARG(plan->P.kernel == kernel, kernel == KIFMM_KERNEL_ADL     ? "plan kernel must be ADL"
                                     : kernel == KIFMM_KERNEL_FIELD ? "plan kernel must be FIELD"
                                                                    : "plan kernel must be DL");
    KF_ARG(plan->P.tree->t.same, "plan must have targets = sources");
    return KIFMM_OK;
}

int ensure(DBuf<double>& b, size_t n) {
    if (b.n < n) KF_TRY(b.alloc(n));
    return KIFMM_OK;
}

}  // namespace

static kifmm::BieScratch& scratch_of(kifmm_plan plan) { return plan->P.bie; }

extern "C" int kifmm_polarization_rhs(const double* nrm, const double* eps_in, double eps_out, const double e0[3],
                                      int64_t n, double* b, void* stream) {
    clear_error();
    KF_ARG(nrm && eps_in && e0 && b, "NULL pointer");
    KF_ARG(n >= 0, "n < 0");
    if (n == 0) return KIFMM_OK;
    k_rhs<<<div_up(n, 256), 256, 0, (cudaStream_t)stream>>>(nrm, eps_in, eps_out, e0[0], e0[1], e0[2], n, b);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

extern "C" int kifmm_bie_apply(kifmm_plan plan, const double* area, const double* eps_in, double eps_out,
                               const double* curv, const double* x, double* y, void* stream) {
    clear_error();
    KF_TRY(check_plan_for(plan, KIFMM_KERNEL_ADL));
    KF_ARG(area && eps_in && curv && x && y, "NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    Plan& P = plan->P;
    int64_t n = P.tree->t.nt;
    BieScratch& S = scratch_of(plan);
    KF_TRY(ensure(S.q, n));
    Gmres g{P, area, eps_in, curv, eps_out, n, s, S.q.p};
    return g.apply(x, y);
}

extern "C" int kifmm_demag_phi2(kifmm_plan plan, const double* phi1, const double* w, const double* omega,
                                double* phi2, void* stream) {
    clear_error();
    KF_TRY(check_plan_for(plan, KIFMM_KERNEL_DL));
    KF_ARG(phi1 && w && omega && phi2, "NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    Plan& P = plan->P;
    int64_t n = P.tree->t.nt;
    BieScratch& S = scratch_of(plan);
    KF_TRY(ensure(S.q, n));
    k_mul<<<div_up(n, 256), 256, 0, s>>>(phi1, w, n, S.q.p);
    KF_CHECK_LAUNCH();
    KF_TRY(plan_matvec(P, S.q.p, phi2, s));
    k_demag_combine<<<div_up(n, 256), 256, 0, s>>>(phi1, omega, n, phi2);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

// ---------------------------------------------------------------------------------
// Allocation-free variant of kifmm_demag_phi2.
//
// Some callers cannot allocate device memory at the moment they need phi2: code
// running under a custom or pooled allocator that forbids driver allocations,
// real-time loops where cudaMalloc's implicit device synchronization is not
// acceptable, or pipelines that record their work into a CUDA graph.  For them the
// scratch vector phi1 * w lives in this file-scope device array instead of a
// buffer the plan allocates on first use.  The array exists once per device for
// as long as the library is loaded.
constexpr int64_t kNoAllocMaxPoints = 1 << 20;   // 8 MiB of FP64 scratch per device
static __device__ __align__(256) double g_noalloc_q[kNoAllocMaxPoints];

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[64] = {};

// Device address of g_noalloc_q on the current device (looked up once per device).
static int noalloc_scratch(double** out) {
    int dev = 0;
    KF_CHECK_CUDA(cudaGetDevice(&dev));
    KF_ARG(dev >= 0 && dev < 64, "device ordinal out of range for the scratch table");
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_q);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress(g_noalloc_q): %s", cudaGetErrorString(e));
            return KIFMM_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return KIFMM_OK;
}

extern "C" int kifmm_demag_phi2_noalloc(kifmm_plan plan, const double* phi1, const double* w,
                                        const double* omega, double* phi2, void* stream) {
    clear_error();
    KF_TRY(check_plan_for(plan, KIFMM_KERNEL_DL));
    KF_ARG(phi1 && w && omega && phi2, "NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    Plan& P = plan->P;
    int64_t n = P.tree->t.nt;
    if (n > kNoAllocMaxPoints) {
        set_error("invalid argument: kifmm_demag_phi2_noalloc handles at most %lld points, plan has %lld",
                  (long long)kNoAllocMaxPoints, (long long)n);
        return KIFMM_ERR_INVALID_ARG;
    }
    double* q = nullptr;
    KF_TRY(noalloc_scratch(&q));
    // every entry of q[0, n) is overwritten here, so nothing needs clearing
    k_mul<<<div_up(n, 256), 256, 0, s>>>(phi1, w, n, q);
    KF_CHECK_LAUNCH();
    KF_TRY(plan_matvec(P, q, phi2, s));
    k_demag_combine<<<div_up(n, 256), 256, 0, s>>>(phi1, omega, n, phi2);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

// ---------------------------------------------------------------- resumable GMRES
// Restarted GMRES(m) as a state machine, so several solves can advance in lockstep:
// launch() enqueues the device work of the next step on a stream without waiting;
// finish() waits for it, runs the host part (Givens rotations, convergence, restart)
// and picks the next step.  Steps: the norm of b; a restart (r = b - A x, beta); one
// Arnoldi step (A v_k, CGS2, ||w||); the final true residual.  Device work that needs a
// host result (v_0 = r / beta, v_{k+1} = w / h_{k+1,k}, x += V y) is carried into the
// next launch.
//
// On a forest every instance runs its own GMRES: its own Hessenberg matrix, rotations,
// residual and convergence test, on its own segment of the vectors.  All instances
// share the steps (one matvec of the forest per step).  An instance leaves the cycle
// when it has converged, when its Krylov space is exhausted (h_{k+1,k} = 0: it waits
// for the next restart) or on breakdown; its new basis vectors are then zero, so the
// matvec, the dots and the updates leave it unchanged.  A cycle ends when no instance
// is left in it or after m steps.
namespace kifmm {

struct Solver {
    enum Inst { kRun, kWait, kConv, kFail };
    Plan& P;
    const double *area, *eps_in, *curv, *b;
    double* x;
    double eps_out, tol;
    int m, max_iter;
    int64_t n;
    int ni;                                 // instances (1 unless the tree is a forest)
    int hld;                                // leading dimension of the per-instance h rows: m + 2
    // device: Krylov basis (m+1) x n, w, r, the area-weighted operand, dot partials and
    // block ranges, per-instance h rows, the point-to-instance map (forests only)
    double *V = nullptr, *w = nullptr, *r = nullptr, *q = nullptr;
    DBuf<double> own_V, own_w, own_r, own_q;
    DBuf<double> partial, hdev;
    DBuf<int64_t> blo, bhi;
    DBuf<int> inst_blk, pinst;
    int nblk = 0;
    Gmres g;
    double* hpin = nullptr;                 // pinned: ha, hb, y (ni hld each), scales (ni)
    enum Step { kNormB, kRestart, kArnoldi, kFinal, kDone } step = kNormB;
    // pending device work for the next launch
    int pend_scale = 0;                     // 1: V_0 *= scal, 2: V_k = scal w, 3: x *= scal
    int pend_x = 0;                         // x += V[0..pend_x) y
    bool zero_x = false;
    // host state, per instance
    std::vector<double> H, cs, sn, gv, bnorm, rel, true_rel;
    std::vector<int> state, iters, status;
    double rel_max = INFINITY, true_max = 0;
    int it = 0, k = 0;
    int status_all = KIFMM_OK;              // first failing instance's status once step == kDone
    cudaStream_t last = nullptr;

    Solver(Plan& P_, const double* area_, const double* eps_in_, const double* curv_, double eps_out_,
           const double* b_, double* x_, double tol_, int m_, int max_iter_)
        : P(P_), area(area_), eps_in(eps_in_), curv(curv_), b(b_), x(x_), eps_out(eps_out_), tol(tol_),
          m(m_), max_iter(max_iter_), n(P_.tree->t.nt), ni(1), hld(m_ + 2),
          g{P_, area_, eps_in_, curv_, eps_out_, P_.tree->t.nt, nullptr, nullptr, true} {
        const Tree& T = P_.tree->t;
        if (T.forest_level >= 0 && T.inst_off.size() >= 2) ni = (int)T.inst_off.size() - 1;
    }
    ~Solver() {
        if (hpin) cudaFreeHost(hpin);
    }

    double* ha() { return hpin; }
    double* hb() { return hpin + (size_t)ni * hld; }
    double* hyv() { return hpin + 2 * (size_t)ni * hld; }
    double* hscal() { return hpin + 3 * (size_t)ni * hld; }
    double* dA() { return hdev.p; }
    double* dB() { return hdev.p + (size_t)ni * hld; }
    double* dY() { return hdev.p + 2 * (size_t)ni * hld; }
    double* dS() { return hdev.p + 3 * (size_t)ni * hld; }
    double& Hx(int i, int row, int col) { return H[((size_t)i * (m + 1) + row) * m + col]; }

    // own = false: use the plan's resident scratch (one solve at a time on that plan)
    int init(bool own) {
        const size_t state_doubles = (size_t)ni * ((size_t)(m + 1) * m + 3 * (size_t)m + 8);
        if (state_doubles > ((size_t)1 << 27)) {
            set_error("invalid argument: GMRES(%d) state of %d instances exceeds 1 GiB of host memory", m, ni);
            return KIFMM_ERR_INVALID_ARG;
        }
        if (own) {
            KF_TRY(own_V.alloc((size_t)(m + 1) * n));
            KF_TRY(own_w.alloc(n));
            KF_TRY(own_r.alloc(n));
            KF_TRY(own_q.alloc(n));
            V = own_V.p, w = own_w.p, r = own_r.p, q = own_q.p;
        } else {
            BieScratch& S = P.bie;
            KF_TRY(ensure(S.q, n));
            KF_TRY(ensure(S.krylov, (size_t)(m + 1) * n));
            KF_TRY(ensure(S.w, n));
            KF_TRY(ensure(S.r, n));
            V = S.krylov.p, w = S.w.p, r = S.r.p, q = S.q.p;
        }
        g.qbuf = q;
        // dot-product blocks: chunks of at least 2048 points (about 600 blocks on large
        // vectors), never across an instance boundary
        std::vector<int64_t> off(ni + 1);
        if (ni > 1) off = P.tree->t.inst_off;
        else off[0] = 0, off[1] = n;
        const int64_t chunk = std::max<int64_t>(2048, div_up(n, 600));
        std::vector<int64_t> lo, hi;
        std::vector<int> ib(ni + 1, 0);
        for (int i = 0; i < ni; ++i) {
            ib[i] = (int)lo.size();
            for (int64_t a = off[i]; a < off[i + 1]; a += chunk) {
                lo.push_back(a);
                hi.push_back(std::min(off[i + 1], a + chunk));
            }
            if (off[i + 1] == off[i]) lo.push_back(off[i]), hi.push_back(off[i]);   // an empty plan
        }
        ib[ni] = (int)lo.size();
        nblk = (int)lo.size();
        KF_TRY(blo.alloc(nblk));
        KF_TRY(bhi.alloc(nblk));
        KF_TRY(inst_blk.alloc(ni + 1));
        KF_CHECK_CUDA(cudaMemcpy(blo.p, lo.data(), nblk * sizeof(int64_t), cudaMemcpyHostToDevice));
        KF_CHECK_CUDA(cudaMemcpy(bhi.p, hi.data(), nblk * sizeof(int64_t), cudaMemcpyHostToDevice));
        KF_CHECK_CUDA(cudaMemcpy(inst_blk.p, ib.data(), (ni + 1) * sizeof(int), cudaMemcpyHostToDevice));
        if (ni > 1) {
            DBuf<int64_t> doff;
            KF_TRY(doff.alloc(ni + 1));
            KF_CHECK_CUDA(cudaMemcpy(doff.p, off.data(), (ni + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
            KF_TRY(pinst.alloc(n));
            // on a private stream, so that other solves' work in flight is not waited for
            cudaStream_t ps = nullptr;
            KF_CHECK_CUDA(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking));
            k_point_instance<<<div_up(n, 256), 256, 0, ps>>>(doff.p, ni, n, pinst.p);
            cudaError_t le = cudaGetLastError();
            cudaError_t se = cudaStreamSynchronize(ps);
            cudaStreamDestroy(ps);
            if (le != cudaSuccess || se != cudaSuccess) {
                set_error("point-to-instance map: %s", cudaGetErrorString(le != cudaSuccess ? le : se));
                return KIFMM_ERR_CUDA;
            }
        }
        KF_TRY(partial.alloc((size_t)nblk * (m + 1)));
        KF_TRY(hdev.alloc(3 * (size_t)ni * hld + ni));
        KF_CHECK_CUDA(cudaMallocHost(&hpin, (3 * (size_t)ni * hld + ni) * sizeof(double)));
        std::fill(hpin, hpin + 3 * (size_t)ni * hld + ni, 0.0);
        H.assign((size_t)ni * (m + 1) * m, 0.0);
        cs.assign((size_t)ni * m, 0.0);
        sn.assign((size_t)ni * m, 0.0);
        gv.assign((size_t)ni * (m + 1), 0.0);
        bnorm.assign(ni, 0.0);
        rel.assign(ni, INFINITY);
        true_rel.assign(ni, 0.0);
        state.assign(ni, kRun);
        iters.assign(ni, 0);
        status.assign(ni, KIFMM_OK);
        return KIFMM_OK;
    }

    const int* inst() const { return ni > 1 ? pinst.p : nullptr; }

    // h (device, row i at i hld_h) = V[0..nv)^T w per instance
    int dots(const double* Vp, int64_t ld, int nv, const double* wp, double* h, int hld_h, cudaStream_t s) {
        k_dots<<<nblk, 256, 0, s>>>(Vp, ld, nv, wp, blo.p, bhi.p, partial.p);
        KF_CHECK_LAUNCH();
        k_dots_final<<<dim3(nv, ni), 128, 0, s>>>(partial.p, inst_blk.p, nv, hld_h, h);
        KF_CHECK_LAUNCH();
        return KIFMM_OK;
    }

    int flush_pending(cudaStream_t s) {
        if (zero_x) {
            KF_CHECK_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
            zero_x = false;
        }
        if (pend_x > 0) {
            // y rows were written to the pinned buffer by finish(); copy and update x
            KF_CHECK_CUDA(cudaMemcpyAsync(dY(), hyv(), (size_t)ni * hld * sizeof(double), cudaMemcpyHostToDevice,
                                          s));
            k_combine<<<div_up(n, 256), 256, 0, s>>>(V, n, pend_x, dY(), hld, 1.0, n, inst(), x);
            KF_CHECK_LAUNCH();
            pend_x = 0;
        }
        if (pend_scale) {
            KF_CHECK_CUDA(cudaMemcpyAsync(dS(), hscal(), ni * sizeof(double), cudaMemcpyHostToDevice, s));
            if (pend_scale == 1) k_scale<<<div_up(n, 256), 256, 0, s>>>(dS(), V, n, inst(), V);
            else if (pend_scale == 2) k_scale<<<div_up(n, 256), 256, 0, s>>>(dS(), w, n, inst(), V + (size_t)k * n);
            else k_scale<<<div_up(n, 256), 256, 0, s>>>(dS(), x, n, inst(), x);
            KF_CHECK_LAUNCH();
            pend_scale = 0;
        }
        return KIFMM_OK;
    }

    int launch(cudaStream_t s) {
        if (step == kDone) return KIFMM_OK;
        g.s = s;
        last = s;
        KF_TRY(flush_pending(s));
        if (step == kNormB) {
            KF_TRY(dots(b, 0, 1, b, dA(), 1, s));
            KF_CHECK_CUDA(cudaMemcpyAsync(ha(), dA(), ni * sizeof(double), cudaMemcpyDeviceToHost, s));
        } else if (step == kRestart || step == kFinal) {
            // r = b - A x (restart: into v_0); A x into w, the matvec's one output buffer
            KF_TRY(g.apply(x, w));
            double* dst = step == kRestart ? V : r;
            k_axpby<<<div_up(n, 256), 256, 0, s>>>(1.0, b, -1.0, w, n, dst);
            KF_CHECK_LAUNCH();
            KF_TRY(dots(dst, 0, 1, dst, dA(), 1, s));
            KF_CHECK_CUDA(cudaMemcpyAsync(ha(), dA(), ni * sizeof(double), cudaMemcpyDeviceToHost, s));
        } else {  // kArnoldi: w = A v_k, two Gram-Schmidt passes against v_0..v_k, ||w||^2
            KF_TRY(g.apply(V + (size_t)k * n, w));
            KF_TRY(dots(V, n, k + 1, w, dA(), hld, s));
            k_combine<<<div_up(n, 256), 256, 0, s>>>(V, n, k + 1, dA(), hld, -1.0, n, inst(), w);
            KF_CHECK_LAUNCH();
            KF_TRY(dots(V, n, k + 1, w, dB(), hld, s));
            k_combine<<<div_up(n, 256), 256, 0, s>>>(V, n, k + 1, dB(), hld, -1.0, n, inst(), w);
            KF_CHECK_LAUNCH();
            KF_TRY(dots(w, 0, 1, w, dB() + (m + 1), hld, s));
            KF_CHECK_CUDA(cudaMemcpyAsync(ha(), dA(), 2 * (size_t)ni * hld * sizeof(double), cudaMemcpyDeviceToHost,
                                          s));
        }
        return KIFMM_OK;
    }

    // Instance i leaves the cycle after kdone steps: back substitution into its y row;
    // x += V y runs at the next launch.
    void end_cycle(int i, int kdone) {
        double* y = hyv() + (size_t)i * hld;
        const double* g_i = &gv[(size_t)i * (m + 1)];
        for (int a = kdone - 1; a >= 0; --a) {
            double acc = g_i[a];
            for (int c = a + 1; c < kdone; ++c) acc -= Hx(i, a, c) * y[c];
            y[a] = acc / Hx(i, a, a);
        }
        pend_x = std::max(pend_x, kdone);
    }

    void update_rel_max() {
        rel_max = 0;
        for (int i = 0; i < ni; ++i)
            if (state[i] != kFail) rel_max = std::max(rel_max, rel[i]);
    }

    void fail(int i, int code) {
        state[i] = kFail;
        status[i] = code;
    }

    int finish() {
        if (step == kDone) return KIFMM_OK;
        KF_CHECK_CUDA(cudaStreamSynchronize(last));
        const double* h0 = ha();
        if (step == kNormB) {
            bool any = false;
            for (int i = 0; i < ni; ++i) {
                bnorm[i] = std::sqrt(h0[i]);
                if (bnorm[i] > 0) any = true;
                else state[i] = kConv, rel[i] = 0;    // x_i = 0 is exact
            }
            if (!any) {
                zero_x = true;
                rel_max = 0;
                step = kFinal;              // x = 0; the final residual is then exactly 0
                return KIFMM_OK;
            }
            if (ni > 1) {
                // x_i = 0 for the instances with b_i = 0 (their exact solution), by a
                // scaling of x with 0 there and 1 elsewhere
                bool zero_any = false;
                for (int i = 0; i < ni; ++i) {
                    hscal()[i] = bnorm[i] > 0 ? 1.0 : 0.0;
                    zero_any |= !(bnorm[i] > 0);
                }
                if (zero_any) pend_scale = 3;
            }
            step = kRestart;
            update_rel_max();
            return KIFMM_OK;
        }
        if (step == kFinal) {
            true_max = 0;
            status_all = KIFMM_OK;
            for (int i = 0; i < ni; ++i) {
                true_rel[i] = bnorm[i] > 0 ? std::sqrt(h0[i]) / bnorm[i] : 0.0;
                true_max = std::max(true_max, true_rel[i]);
                if (status[i] == KIFMM_OK && !(rel[i] <= tol)) status[i] = KIFMM_ERR_NOT_CONVERGED;
                if (status_all == KIFMM_OK && status[i] != KIFMM_OK) status_all = status[i];
            }
            if (status_all == KIFMM_ERR_NOT_CONVERGED)
                set_error("GMRES did not converge in %d iterations (residual estimate %.3e)", it, rel_max);
            else if (status_all == KIFMM_ERR_BREAKDOWN)
                set_error("GMRES breakdown after %d iterations", it);
            step = kDone;
            return KIFMM_OK;
        }
        if (step == kRestart) {
            bool any = false;
            for (int i = 0; i < ni; ++i) {
                double* sc = hscal() + i;
                *sc = 0.0;
                if (state[i] != kRun && state[i] != kWait) continue;
                const double beta = std::sqrt(h0[i]);
                rel[i] = beta / bnorm[i];
                if (!std::isfinite(beta)) {
                    fail(i, KIFMM_ERR_BREAKDOWN);
                    continue;
                }
                if (rel[i] <= tol) {
                    state[i] = kConv;
                    continue;
                }
                state[i] = kRun;
                *sc = 1.0 / beta;
                double* g_i = &gv[(size_t)i * (m + 1)];
                std::fill(g_i, g_i + m + 1, 0.0);
                g_i[0] = beta;
                any = true;
            }
            update_rel_max();
            if (!any || it >= max_iter) {
                step = kFinal;
                return KIFMM_OK;
            }
            pend_scale = 1;
            k = 0;
            step = kArnoldi;
            return KIFMM_OK;
        }
        // kArnoldi: per instance in the cycle, column k of H, the previous rotations, a
        // new rotation
        const double* hA_ = ha();
        const double* hB_ = hb();
        ++it;
        std::fill(hyv(), hyv() + (size_t)ni * hld, 0.0);
        bool left = false;
        const bool last_step = k + 1 == m || it >= max_iter;
        for (int i = 0; i < ni; ++i) {
            double* sc = hscal() + i;
            *sc = 0.0;
            if (state[i] != kRun) continue;
            const double* a_ = hA_ + (size_t)i * hld;
            const double* b_ = hB_ + (size_t)i * hld;
            for (int a = 0; a <= k; ++a) Hx(i, a, k) = a_[a] + b_[a];
            const double hk1 = std::sqrt(b_[m + 1]);
            Hx(i, k + 1, k) = hk1;
            if (!std::isfinite(hk1)) {
                fail(i, KIFMM_ERR_BREAKDOWN);
                continue;
            }
            double* cs_i = &cs[(size_t)i * m];
            double* sn_i = &sn[(size_t)i * m];
            double* g_i = &gv[(size_t)i * (m + 1)];
            for (int a = 0; a < k; ++a) {
                const double a0 = Hx(i, a, k), a1 = Hx(i, a + 1, k);
                Hx(i, a, k) = cs_i[a] * a0 + sn_i[a] * a1;
                Hx(i, a + 1, k) = -sn_i[a] * a0 + cs_i[a] * a1;
            }
            const double a0 = Hx(i, k, k), a1 = Hx(i, k + 1, k);
            const double den = std::hypot(a0, a1);
            if (!(den > 0)) {
                fail(i, KIFMM_ERR_BREAKDOWN);
                continue;
            }
            cs_i[k] = a0 / den;
            sn_i[k] = a1 / den;
            Hx(i, k, k) = den;
            Hx(i, k + 1, k) = 0;
            g_i[k + 1] = -sn_i[k] * g_i[k];
            g_i[k] = cs_i[k] * g_i[k];
            iters[i] = it;
            rel[i] = std::fabs(g_i[k + 1]) / bnorm[i];
            if (rel[i] <= tol) {
                end_cycle(i, k + 1);
                state[i] = kConv;
            } else if (hk1 == 0 || last_step) {
                end_cycle(i, k + 1);
                state[i] = kWait;           // Krylov space exhausted or cycle over: restart
            } else {
                *sc = 1.0 / hk1;            // v_{k+1} = w / h_{k+1,k}
                left = true;
            }
        }
        update_rel_max();
        if (left) {
            pend_scale = 2;
            ++k;
            return KIFMM_OK;
        }
        bool waiting = false;
        for (int i = 0; i < ni; ++i) waiting |= state[i] == kWait;
        step = waiting && it < max_iter ? kRestart : kFinal;
        return KIFMM_OK;
    }

};

}  // namespace kifmm

struct kifmm_solver_s {
    kifmm::Solver S;
    template <class... A>
    explicit kifmm_solver_s(A&&... a) : S(std::forward<A>(a)...) {}
};

static int solver_args(kifmm_plan plan, const double* area, const double* eps_in, const double* curv,
                       const double* b, double* x, double tol, int restart, int max_iter) {
    KF_TRY(check_plan_for(plan, KIFMM_KERNEL_ADL));
    KF_ARG(area && eps_in && curv && b && x, "NULL pointer");
    KF_ARG(tol > 0 && tol < 1, "tol must be in (0, 1)");
    KF_ARG(restart >= 1 && restart <= 500, "restart must be in [1, 500]");
    KF_ARG(max_iter >= 1, "max_iter must be >= 1");
    return KIFMM_OK;
}

extern "C" int kifmm_bie_solve(kifmm_plan plan, const double* area, const double* eps_in, double eps_out,
                               const double* curv, const double* b, double* x, double tol, int restart,
                               int max_iter, int* iters, double* rel_res, void* stream) {
    clear_error();
    KF_TRY(solver_args(plan, area, eps_in, curv, b, x, tol, restart, max_iter));
    cudaStream_t s = (cudaStream_t)stream;
    Solver S(plan->P, area, eps_in, curv, eps_out, b, x, tol, restart, max_iter);
    KF_TRY(S.init(false));
    while (S.step != Solver::kDone) {
        KF_TRY(S.launch(s));
        KF_TRY(S.finish());
    }
    if (iters) *iters = S.it;
    if (rel_res) *rel_res = S.true_max;
    return S.status_all;
}

extern "C" int kifmm_solver_create(kifmm_plan plan, const double* area, const double* eps_in, double eps_out,
                                   const double* curv, const double* b, double* x, double tol, int restart,
                                   int max_iter, kifmm_solver* out) {
    clear_error();
    KF_ARG(out != nullptr, "out is NULL");
    *out = nullptr;
    KF_TRY(solver_args(plan, area, eps_in, curv, b, x, tol, restart, max_iter));
    kifmm_solver sv =
        new (std::nothrow) kifmm_solver_s(plan->P, area, eps_in, curv, eps_out, b, x, tol, restart, max_iter);
    if (!sv) {
        set_error("host allocation failed");
        return KIFMM_ERR_OOM;
    }
    int rc = sv->S.init(true);
    if (rc != KIFMM_OK) {
        delete sv;
        return rc;
    }
    *out = sv;
    return KIFMM_OK;
}

extern "C" int kifmm_solver_launch(kifmm_solver solver, void* stream) {
    clear_error();
    KF_ARG(solver != nullptr, "NULL solver");
    return solver->S.launch((cudaStream_t)stream);
}

extern "C" int kifmm_solver_finish(kifmm_solver solver, int* done, int* iters, double* rel_res) {
    clear_error();
    KF_ARG(solver != nullptr, "NULL solver");
    KF_TRY(solver->S.finish());
    const Solver& S = solver->S;
    if (done) *done = S.step == Solver::kDone;
    if (iters) *iters = S.it;
    if (rel_res) *rel_res = S.step == Solver::kDone ? S.true_max : S.rel_max;
    return S.step == Solver::kDone ? S.status_all : KIFMM_OK;
}

extern "C" int kifmm_solver_instances(kifmm_solver solver, int n_inst, int32_t* iters, double* rel_res,
                                      int32_t* status) {
    clear_error();
    KF_ARG(solver != nullptr, "NULL solver");
    const Solver& S = solver->S;
    KF_ARG(n_inst == S.ni, "n_inst must be the tree's instance count");
    const bool done = S.step == Solver::kDone;
    for (int i = 0; i < S.ni; ++i) {
        if (iters) iters[i] = S.iters[i];
        if (rel_res) rel_res[i] = done ? S.true_rel[i] : S.rel[i];
        if (status) status[i] = done ? S.status[i] : KIFMM_OK;
    }
    return KIFMM_OK;
}

extern "C" int kifmm_solver_destroy(kifmm_solver solver) {
    clear_error();
    delete solver;
    return KIFMM_OK;
}

extern "C" int kifmm_polarization_field(kifmm_plan plan, const double* area, const double* curv, const double* nrm,
                                        const double* sigma, const double e0[3], double* E, void* stream) {
    clear_error();
    KF_TRY(check_plan_for(plan, KIFMM_KERNEL_FIELD));
    KF_ARG(area && curv && nrm && sigma && e0 && E, "NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    Plan& P = plan->P;
    const int64_t n = P.tree->t.nt;
    if (n == 0) return KIFMM_OK;
    BieScratch& S = scratch_of(plan);
    KF_TRY(ensure(S.q, n));
    k_mul<<<div_up(n, 256), 256, 0, s>>>(sigma, area, n, S.q.p);
    KF_CHECK_LAUNCH();
    KF_TRY(plan_matvec(P, S.q.p, E, s));
    k_field_combine<<<div_up(n, 256), 256, 0, s>>>(sigma, area, curv, nrm, e0[0], e0[1], e0[2], n, E);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

extern "C" int kifmm_polarization_force(kifmm_plan plan, const double* area, const double* curv, const double* nrm,
                                        const double* sigma, double eps_out, const double e0[3], const int32_t* body,
                                        int n_body, double* F, void* stream) {
    clear_error();
    KF_TRY(check_plan_for(plan, KIFMM_KERNEL_FIELD));
    KF_ARG(area && curv && nrm && sigma && e0 && body && F, "NULL pointer");
    KF_ARG(n_body >= 1, "n_body < 1");
    cudaStream_t s = (cudaStream_t)stream;
    Plan& P = plan->P;
    const int64_t n = P.tree->t.nt;
    BieScratch& S = scratch_of(plan);
    KF_TRY(ensure(S.r, 3 * (size_t)std::max<int64_t>(n, 1)));
    KF_CHECK_CUDA(cudaMemsetAsync(F, 0, 3 * (size_t)n_body * sizeof(double), s));
    if (n == 0) return KIFMM_OK;
    KF_TRY(kifmm_polarization_field(plan, area, curv, nrm, sigma, e0, S.r.p, stream));
    int dev = 0, nsm = 0;
    KF_CHECK_CUDA(cudaGetDevice(&dev));
    KF_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = (int)std::min<int64_t>(div_up(n, 256), 4 * (int64_t)nsm);
    k_force<<<grid, 256, 0, s>>>(sigma, area, S.r.p, body, eps_out, n, n_body, F);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

extern "C" int kifmm_polarization_rhs_free(kifmm_plan plan, const double* area, const double* eps_in, double eps_out,
                                           const double* curv, const double* nrm, const double* sigma_f,
                                           const double e0[3], double* b, void* stream) {
    clear_error();
    KF_TRY(check_plan_for(plan, KIFMM_KERNEL_ADL));
    KF_ARG(area && eps_in && curv && nrm && sigma_f && e0 && b, "NULL pointer");
    cudaStream_t s = (cudaStream_t)stream;
    Plan& P = plan->P;
    const int64_t n = P.tree->t.nt;
    if (n == 0) return KIFMM_OK;
    BieScratch& S = scratch_of(plan);
    KF_TRY(ensure(S.q, n));
    k_mul<<<div_up(n, 256), 256, 0, s>>>(sigma_f, area, n, S.q.p);
    KF_CHECK_LAUNCH();
    KF_TRY(plan_matvec(P, S.q.p, b, s));
    k_rhs_free<<<div_up(n, 256), 256, 0, s>>>(nrm, eps_in, eps_out, sigma_f, area, curv, e0[0], e0[1], e0[2], n, b);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}
