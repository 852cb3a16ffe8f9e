// Boundary-integral operators on top of the FMM matvec, and matrix-free GMRES.
//
// Polarization (Sec. II.C, Eqs. Ax, Eb, pol_discret, rhs), eps_0 = 1:
//   (A s)_j = ebar_j s_j + deps_j (1/4pi) [ ADL(s * a)_j + c_j s_j ]
//   ebar_j = (eps_j + eps_out)/2, deps_j = eps_out - eps_j, c_j = H_j sqrt(pi a_j)
// The self term of Eq. pol_discret is read as c_j s_j: the principal-value normal
// field at the centre of a disc of area a_j on a surface of mean curvature H_j with
// unit density is pi rho H, rho = sqrt(a_j/pi).
// Demagnetization (Sec. II.B, Eq. fk_integral_discrete):
//   phi2_i = DL(phi1 * w)_i / 4pi + (Omega_i/4pi - 1) phi1_i
// GMRES (Sec. III: PETSc GMRES in matrix-free form; here restarted GMRES(m) of Saad &
// Schultz with classical Gram-Schmidt applied twice) keeps its Krylov basis, the
// orthogonalization and the residuals in FP64 on the device; only the small
// Hessenberg least-squares problem runs on the host.
#include <cmath>
#include <mutex>
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
    KF_ARG(plan->P.kernel == kernel, kernel == KIFMM_KERNEL_ADL ? "plan kernel must be ADL" : "plan kernel must be DL");
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

extern "C" int kifmm_bie_solve(kifmm_plan plan, const double* area, const double* eps_in, double eps_out,
                               const double* curv, const double* b, double* x, double tol, int restart,
                               int max_iter, int* iters, double* rel_res, void* stream) {
    clear_error();
    KF_TRY(check_plan_for(plan, KIFMM_KERNEL_ADL));
    KF_ARG(area && eps_in && curv && b && x, "NULL pointer");
    KF_ARG(tol > 0 && tol < 1, "tol must be in (0, 1)");
    KF_ARG(restart >= 1 && restart <= 500, "restart must be in [1, 500]");
    KF_ARG(max_iter >= 1, "max_iter must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    Plan& P = plan->P;
    const int64_t n = P.tree->t.nt;
    const int m = restart;
    BieScratch& S = scratch_of(plan);
    KF_TRY(ensure(S.q, n));
    KF_TRY(ensure(S.krylov, (size_t)(m + 1) * n));
    KF_TRY(ensure(S.w, n));
    KF_TRY(ensure(S.r, n));
    Gmres g{P, area, eps_in, curv, eps_out, n, s, S.q.p};
    KF_TRY(g.partial.alloc((size_t)kDotBlocks * (m + 1)));
    KF_TRY(g.hdev.alloc(3 * (size_t)(m + 2)));
    double* V = S.krylov.p;
    double* w = S.w.p;
    double* hA = g.hdev.p;
    double* hB = g.hdev.p + (m + 2);
    double* hy = g.hdev.p + 2 * (m + 2);

    double bn2 = 0;
    KF_TRY(g.dots(b, 0, 1, b, hA));
    KF_CHECK_CUDA(cudaMemcpyAsync(&bn2, hA, sizeof(double), cudaMemcpyDeviceToHost, s));
    KF_CHECK_CUDA(cudaStreamSynchronize(s));
    double bnorm = std::sqrt(bn2);
    if (iters) *iters = 0;
    if (rel_res) *rel_res = 0;
    if (!(bnorm > 0)) {
        KF_CHECK_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
        KF_CHECK_CUDA(cudaStreamSynchronize(s));
        return KIFMM_OK;
    }
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m), ha(m + 2), hb(m + 2);
    int it = 0;
    double rel = INFINITY;
    bool converged = false, breakdown = false;
    while (it < max_iter && !converged) {
        // r = b - A x
        KF_TRY(g.apply(x, S.r.p));
        k_axpby<<<div_up(n, 256), 256, 0, s>>>(1.0, b, -1.0, S.r.p, n, V);
        KF_CHECK_LAUNCH();
        KF_TRY(g.dots(V, 0, 1, V, hA));
        double beta2;
        KF_CHECK_CUDA(cudaMemcpyAsync(&beta2, hA, sizeof(double), cudaMemcpyDeviceToHost, s));
        KF_CHECK_CUDA(cudaStreamSynchronize(s));
        double beta = std::sqrt(beta2);
        rel = beta / bnorm;
        if (!std::isfinite(beta)) {
            breakdown = true;
            break;
        }
        if (rel <= tol) {
            converged = true;
            break;
        }
        k_axpby<<<div_up(n, 256), 256, 0, s>>>(1.0 / beta, V, 0.0, V, n, V);
        KF_CHECK_LAUNCH();
        std::fill(gv.begin(), gv.end(), 0.0);
        gv[0] = beta;
        int kdone = 0;
        for (int k = 0; k < m && it < max_iter; ++k) {
            KF_TRY(g.apply(V + (size_t)k * n, w));
            KF_TRY(g.dots(V, n, k + 1, w, hA));
            k_combine<<<div_up(n, 256), 256, 0, s>>>(V, n, k + 1, hA, -1.0, n, w);
            KF_CHECK_LAUNCH();
            KF_TRY(g.dots(V, n, k + 1, w, hB));
            k_combine<<<div_up(n, 256), 256, 0, s>>>(V, n, k + 1, hB, -1.0, n, w);
            KF_CHECK_LAUNCH();
            KF_TRY(g.dots(w, 0, 1, w, hB + (m + 1)));
            KF_CHECK_CUDA(cudaMemcpyAsync(ha.data(), hA, (k + 1) * sizeof(double), cudaMemcpyDeviceToHost, s));
            KF_CHECK_CUDA(cudaMemcpyAsync(hb.data(), hB, (m + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
            KF_CHECK_CUDA(cudaStreamSynchronize(s));
            for (int i = 0; i <= k; ++i) H[(size_t)i * m + k] = ha[i] + hb[i];
            double hk1 = std::sqrt(hb[m + 1]);
            H[(size_t)(k + 1) * m + k] = hk1;
            if (!std::isfinite(hk1)) {
                breakdown = true;
                break;
            }
            if (hk1 > 0) {
                k_axpby<<<div_up(n, 256), 256, 0, s>>>(1.0 / hk1, w, 0.0, w, n, V + (size_t)(k + 1) * n);
                KF_CHECK_LAUNCH();
            }
            for (int i = 0; i < k; ++i) {
                double a0 = H[(size_t)i * m + k], a1 = H[(size_t)(i + 1) * m + k];
                H[(size_t)i * m + k] = cs[i] * a0 + sn[i] * a1;
                H[(size_t)(i + 1) * m + k] = -sn[i] * a0 + cs[i] * a1;
            }
            double a0 = H[(size_t)k * m + k], a1 = H[(size_t)(k + 1) * m + k];
            double den = std::hypot(a0, a1);
            if (!(den > 0)) {
                breakdown = true;
                break;
            }
            cs[k] = a0 / den;
            sn[k] = a1 / den;
            H[(size_t)k * m + k] = den;
            H[(size_t)(k + 1) * m + k] = 0;
            gv[k + 1] = -sn[k] * gv[k];
            gv[k] = cs[k] * gv[k];
            ++it;
            kdone = k + 1;
            rel = std::fabs(gv[k + 1]) / bnorm;
            if (rel <= tol || hk1 == 0) break;
        }
        if (kdone > 0) {
            for (int i = kdone - 1; i >= 0; --i) {
                double acc = gv[i];
                for (int j = i + 1; j < kdone; ++j) acc -= H[(size_t)i * m + j] * y[j];
                y[i] = acc / H[(size_t)i * m + i];
            }
            KF_CHECK_CUDA(cudaMemcpyAsync(hy, y.data(), kdone * sizeof(double), cudaMemcpyHostToDevice, s));
            k_combine<<<div_up(n, 256), 256, 0, s>>>(V, n, kdone, hy, 1.0, n, x);
            KF_CHECK_LAUNCH();
            KF_CHECK_CUDA(cudaStreamSynchronize(s));
        }
        if (breakdown) break;
        if (rel <= tol) converged = true;
    }
    // true residual
    KF_TRY(g.apply(x, S.r.p));
    k_axpby<<<div_up(n, 256), 256, 0, s>>>(1.0, b, -1.0, S.r.p, n, S.r.p);
    KF_CHECK_LAUNCH();
    KF_TRY(g.dots(S.r.p, 0, 1, S.r.p, hA));
    double rr;
    KF_CHECK_CUDA(cudaMemcpyAsync(&rr, hA, sizeof(double), cudaMemcpyDeviceToHost, s));
    KF_CHECK_CUDA(cudaStreamSynchronize(s));
    if (iters) *iters = it;
    if (rel_res) *rel_res = std::sqrt(rr) / bnorm;
    if (breakdown) {
        set_error("GMRES breakdown after %d iterations", it);
        return KIFMM_ERR_BREAKDOWN;
    }
    if (!converged) {
        set_error("GMRES did not converge in %d iterations (residual estimate %.3e)", it, rel);
        return KIFMM_ERR_NOT_CONVERGED;
    }
    return KIFMM_OK;
}
