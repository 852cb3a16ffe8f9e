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

// partial[blk * nv + i] = sum over this block's stride of V[i] . w  (i < nv)
constexpr int kDotBlocks = 304;
__global__ void k_dots(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ w,
                       int64_t n, double* __restrict__ partial) {
    __shared__ double red[256];
    for (int i = 0; i < nv; ++i) {
        const double* v = V + (size_t)i * ld;
        double s = 0;
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
            s += v[t] * w[t];
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(size_t)blockIdx.x * nv + i] = red[0];
        __syncthreads();
    }
}

__global__ void k_dots_final(const double* __restrict__ partial, int nblk, int nv, double* __restrict__ h) {
    int i = blockIdx.x;
    __shared__ double red[256];
    double s = 0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(size_t)b * nv + i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) h[i] = red[0];
}

// w -= sum_i h[i] V[i]   (sign = -1)   or   x += sum_i h[i] V[i]   (sign = +1)
__global__ void k_combine(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ h,
                          double sign, int64_t n, double* __restrict__ w) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    double s = 0;
    for (int i = 0; i < nv; ++i) s += h[i] * V[(size_t)i * ld + t];
    w[t] += sign * s;
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, const double* __restrict__ y, int64_t n,
                        double* __restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * x[i] + b * y[i];
}

struct Gmres {
    Plan& P;
    const double *area, *eps_in, *curv;
    double eps_out;
    int64_t n;
    cudaStream_t s;
    double* qbuf;
    DBuf<double> partial, hdev;

    int apply(const double* x, double* y) {
        k_mul<<<div_up(n, 256), 256, 0, s>>>(x, area, n, qbuf);
        KF_CHECK_LAUNCH();
        KF_TRY(plan_matvec(P, qbuf, y, s));
        k_polar_combine<<<div_up(n, 256), 256, 0, s>>>(x, area, eps_in, eps_out, curv, n, y);
        KF_CHECK_LAUNCH();
        return KIFMM_OK;
    }
    // h (device, nv) = V[0..nv)^T w
    int dots(const double* V, int64_t ld, int nv, const double* w, double* h) {
        k_dots<<<kDotBlocks, 256, 0, s>>>(V, ld, nv, w, n, partial.p);
        KF_CHECK_LAUNCH();
        k_dots_final<<<nv, 256, 0, s>>>(partial.p, kDotBlocks, nv, h);
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
namespace kifmm {

struct Solver {
    Plan& P;
    const double *area, *eps_in, *curv, *b;
    double* x;
    double eps_out, tol;
    int m, max_iter;
    int64_t n;
    // device: Krylov basis (m+1) x n, w, r, the area-weighted operand, dot partials, h
    double *V = nullptr, *w = nullptr, *r = nullptr, *q = nullptr;
    DBuf<double> own_V, own_w, own_r, own_q;
    Gmres g;
    double* hpin = nullptr;                 // pinned host copies: ha (m+2), hb (m+2), scalar
    enum Step { kNormB, kRestart, kArnoldi, kFinal, kDone } step = kNormB;
    // pending device work for the next launch
    double scale_v0 = 0, scale_next = 0;
    int pend_x = 0;                         // x += V[0..pend_x) y
    bool zero_x = false;
    // host state
    std::vector<double> H, cs, sn, gv, y;
    double bnorm = 0, rel = INFINITY, true_rel = 0;
    int it = 0, k = 0;
    int status = KIFMM_OK;                  // final status once step == kDone
    cudaStream_t last = nullptr;

    Solver(Plan& P_, const double* area_, const double* eps_in_, const double* curv_, double eps_out_,
           const double* b_, double* x_, double tol_, int m_, int max_iter_)
        : P(P_), area(area_), eps_in(eps_in_), curv(curv_), b(b_), x(x_), eps_out(eps_out_), tol(tol_),
          m(m_), max_iter(max_iter_), n(P_.tree->t.nt), g{P_, area_, eps_in_, curv_, eps_out_, P_.tree->t.nt,
                                                            nullptr, nullptr, {}, {}} {}
    ~Solver() {
        if (hpin) cudaFreeHost(hpin);
    }

    // own = false: use the plan's resident scratch (one solve at a time on that plan)
    int init(bool own) {
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
        KF_TRY(g.partial.alloc((size_t)kDotBlocks * (m + 1)));
        KF_TRY(g.hdev.alloc(3 * (size_t)(m + 2)));
        KF_CHECK_CUDA(cudaMallocHost(&hpin, (2 * (size_t)(m + 2) + 1) * sizeof(double)));
        H.assign((size_t)(m + 1) * m, 0.0);
        cs.assign(m, 0.0);
        sn.assign(m, 0.0);
        gv.assign(m + 1, 0.0);
        y.assign(m, 0.0);
        return KIFMM_OK;
    }

    double* hA() { return g.hdev.p; }
    double* hB() { return g.hdev.p + (m + 2); }
    double* hy() { return g.hdev.p + 2 * (m + 2); }

    int flush_pending(cudaStream_t s) {
        if (zero_x) {
            KF_CHECK_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
            zero_x = false;
        }
        if (pend_x > 0) {
            // y was written to the pinned buffer by finish(); copy and update x
            KF_CHECK_CUDA(cudaMemcpyAsync(hy(), hpin, pend_x * sizeof(double), cudaMemcpyHostToDevice, s));
            k_combine<<<div_up(n, 256), 256, 0, s>>>(V, n, pend_x, hy(), 1.0, n, x);
            KF_CHECK_LAUNCH();
            pend_x = 0;
        }
        if (scale_v0 != 0) {
            k_axpby<<<div_up(n, 256), 256, 0, s>>>(scale_v0, V, 0.0, V, n, V);
            KF_CHECK_LAUNCH();
            scale_v0 = 0;
        }
        if (scale_next != 0) {
            k_axpby<<<div_up(n, 256), 256, 0, s>>>(scale_next, w, 0.0, w, n, V + (size_t)k * n);
            KF_CHECK_LAUNCH();
            scale_next = 0;
        }
        return KIFMM_OK;
    }

    int launch(cudaStream_t s) {
        if (step == kDone) return KIFMM_OK;
        g.s = s;
        last = s;
        KF_TRY(flush_pending(s));
        if (step == kNormB) {
            KF_TRY(g.dots(b, 0, 1, b, hA()));
            KF_CHECK_CUDA(cudaMemcpyAsync(hpin, hA(), sizeof(double), cudaMemcpyDeviceToHost, s));
        } else if (step == kRestart || step == kFinal) {
            // r = b - A x (restart: into v_0)
            KF_TRY(g.apply(x, r));
            double* dst = step == kRestart ? V : r;
            k_axpby<<<div_up(n, 256), 256, 0, s>>>(1.0, b, -1.0, r, n, dst);
            KF_CHECK_LAUNCH();
            KF_TRY(g.dots(dst, 0, 1, dst, hA()));
            KF_CHECK_CUDA(cudaMemcpyAsync(hpin, hA(), sizeof(double), cudaMemcpyDeviceToHost, s));
        } else {  // kArnoldi: w = A v_k, two Gram-Schmidt passes against v_0..v_k, ||w||^2
            KF_TRY(g.apply(V + (size_t)k * n, w));
            KF_TRY(g.dots(V, n, k + 1, w, hA()));
            k_combine<<<div_up(n, 256), 256, 0, s>>>(V, n, k + 1, hA(), -1.0, n, w);
            KF_CHECK_LAUNCH();
            KF_TRY(g.dots(V, n, k + 1, w, hB()));
            k_combine<<<div_up(n, 256), 256, 0, s>>>(V, n, k + 1, hB(), -1.0, n, w);
            KF_CHECK_LAUNCH();
            KF_TRY(g.dots(w, 0, 1, w, hB() + (m + 1)));
            KF_CHECK_CUDA(cudaMemcpyAsync(hpin, hA(), (k + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
            KF_CHECK_CUDA(cudaMemcpyAsync(hpin + (m + 2), hB(), (m + 2) * sizeof(double),
                                          cudaMemcpyDeviceToHost, s));
        }
        return KIFMM_OK;
    }

    // End of a cycle: back substitution, then x += V y at the next launch.
    void end_cycle(int kdone) {
        for (int i = kdone - 1; i >= 0; --i) {
            double acc = gv[i];
            for (int j = i + 1; j < kdone; ++j) acc -= H[(size_t)i * m + j] * y[j];
            y[i] = acc / H[(size_t)i * m + i];
        }
        for (int i = 0; i < kdone; ++i) hpin[i] = y[i];   // read by the next launch's copy
        pend_x = kdone;
    }

    int finish() {
        if (step == kDone) return KIFMM_OK;
        KF_CHECK_CUDA(cudaStreamSynchronize(last));
        if (step == kNormB) {
            bnorm = std::sqrt(hpin[0]);
            if (!(bnorm > 0)) {
                zero_x = true;
                rel = true_rel = 0;
                step = kFinal;              // x = 0; the final residual is then exactly 0
                return KIFMM_OK;
            }
            step = kRestart;
            return KIFMM_OK;
        }
        if (step == kFinal) {
            true_rel = bnorm > 0 ? std::sqrt(hpin[0]) / bnorm : 0.0;
            if (status == KIFMM_OK && !(rel <= tol)) {
                set_error("GMRES did not converge in %d iterations (residual estimate %.3e)", it, rel);
                status = KIFMM_ERR_NOT_CONVERGED;
            }
            step = kDone;
            return KIFMM_OK;
        }
        if (step == kRestart) {
            const double beta = std::sqrt(hpin[0]);
            rel = beta / bnorm;
            if (!std::isfinite(beta)) return breakdown();
            if (rel <= tol || it >= max_iter) {
                step = kFinal;
                return KIFMM_OK;
            }
            scale_v0 = 1.0 / beta;
            std::fill(gv.begin(), gv.end(), 0.0);
            gv[0] = beta;
            k = 0;
            step = kArnoldi;
            return KIFMM_OK;
        }
        // kArnoldi: column k of H, the previous rotations, a new rotation
        const double* ha = hpin;
        const double* hb = hpin + (m + 2);
        for (int i = 0; i <= k; ++i) H[(size_t)i * m + k] = ha[i] + hb[i];
        const double hk1 = std::sqrt(hb[m + 1]);
        H[(size_t)(k + 1) * m + k] = hk1;
        if (!std::isfinite(hk1)) return breakdown();
        for (int i = 0; i < k; ++i) {
            const double a0 = H[(size_t)i * m + k], a1 = H[(size_t)(i + 1) * m + k];
            H[(size_t)i * m + k] = cs[i] * a0 + sn[i] * a1;
            H[(size_t)(i + 1) * m + k] = -sn[i] * a0 + cs[i] * a1;
        }
        const double a0 = H[(size_t)k * m + k], a1 = H[(size_t)(k + 1) * m + k];
        const double den = std::hypot(a0, a1);
        if (!(den > 0)) return breakdown();
        cs[k] = a0 / den;
        sn[k] = a1 / den;
        H[(size_t)k * m + k] = den;
        H[(size_t)(k + 1) * m + k] = 0;
        gv[k + 1] = -sn[k] * gv[k];
        gv[k] = cs[k] * gv[k];
        ++it;
        rel = std::fabs(gv[k + 1]) / bnorm;
        if (rel <= tol || hk1 == 0 || k + 1 == m || it >= max_iter) {
            end_cycle(k + 1);
            step = (rel <= tol || it >= max_iter) ? kFinal : kRestart;
            return KIFMM_OK;
        }
        if (hk1 > 0) scale_next = 1.0 / hk1;   // v_{k+1} = w / h_{k+1,k}
        ++k;
        return KIFMM_OK;
    }

    int breakdown() {
        set_error("GMRES breakdown after %d iterations", it);
        status = KIFMM_ERR_BREAKDOWN;
        step = kFinal;
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
    if (rel_res) *rel_res = S.true_rel;
    return S.status;
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
    if (rel_res) *rel_res = S.step == Solver::kDone ? S.true_rel : S.rel;
    return S.step == Solver::kDone ? S.status : KIFMM_OK;
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
