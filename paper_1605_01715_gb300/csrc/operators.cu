// KIFMM translation operators (Ying, Biros & Zorin 2004), built in FP64.
//
// Surfaces: the p x p x p grid points on the boundary of the cube [-1,1]^3,
// Q = 6(p-1)^2 + 2 of them, scaled by 1.05 (equivalent surface of the upward pass,
// check surface of the downward pass) or 2.95 (the other two) box half-widths.
// Check-to-equivalent maps are pseudo-inverses of the 1/r kernel matrices, from a
// one-sided Jacobi SVD truncated at cutoff * sigma_max.
//
// The matvec keeps only check potentials.  Each pseudo-inverse is folded into the
// operator that follows it, so no ill-conditioned equivalent density is ever
// rounded to the working precision:
//   M2M'_o = 1/2 K(2.95 s, c_o + 0.525 s) Pu      child up-check  -> parent up-check
//   M2L'_t = K(1.05 s, 2t + 1.05 s) Pu              source up-check -> target down-check
//   L2L'_o = K(c_o + 0.525 s, 2.95 s) Pd           parent down-check -> child down-check
//   D2T_i  = G(x_i, 2.95 s) Pd                     leaf down-check  -> target value
// (unit frames: the larger box has half-width 1; the scale factors of the 1/r kernel
// cancel against those of the pseudo-inverses).  The 1/r kernel is the paper's K_r,
// the kernel its far field is built on (Sec. III.A.1, Eq. p2m; Sec. III.A.2).
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "operators.cuh"

namespace kifmm {

std::vector<double> surface_points(int p) {
    std::vector<double> s;
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j)
            for (int k = 0; k < p; ++k) {
                if (i != 0 && i != p - 1 && j != 0 && j != p - 1 && k != 0 && k != p - 1) continue;
                s.push_back(-1.0 + 2.0 * i / (p - 1));
                s.push_back(-1.0 + 2.0 * j / (p - 1));
                s.push_back(-1.0 + 2.0 * k / (p - 1));
            }
    return s;
}

// Pseudo-inverse of the n x n matrix A (row-major) by one-sided Jacobi SVD
// (Hestenes): rotate column pairs of A until mutually orthogonal, A V = U S.
// Pairs are visited in round-robin order so each round's rotations are disjoint.
std::vector<double> pinv_jacobi(const std::vector<double>& A_rm, int n, double cutoff, std::vector<double>* U,
                                std::vector<double>* W, int* rank, int max_rank) {
    std::vector<double> a((size_t)n * n), v((size_t)n * n, 0.0);  // column-major
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) a[(size_t)j * n + i] = A_rm[(size_t)i * n + j];
    for (int j = 0; j < n; ++j) v[(size_t)j * n + j] = 1.0;
    int m = n + (n & 1);               // players in the round-robin schedule
    std::vector<int> ring(m);
    for (int i = 0; i < m; ++i) ring[i] = i;
    const double eps = 1e-15;
    for (int sweep = 0; sweep < 60; ++sweep) {
        int rotated = 0;
        for (int round = 0; round < m - 1; ++round) {
#pragma omp parallel for reduction(+ : rotated) schedule(static)
            for (int k = 0; k < m / 2; ++k) {
                int p = ring[k], q = ring[m - 1 - k];
                if (p >= n || q >= n) continue;
                if (p > q) std::swap(p, q);
                double* ap = &a[(size_t)p * n];
                double* aq = &a[(size_t)q * n];
                double alpha = 0, beta = 0, gamma = 0;
                for (int i = 0; i < n; ++i) {
                    alpha += ap[i] * ap[i];
                    beta += aq[i] * aq[i];
                    gamma += ap[i] * aq[i];
                }
                if (std::fabs(gamma) <= eps * std::sqrt(alpha * beta) || gamma == 0.0) continue;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < n; ++i) {
                    double x = ap[i], y = aq[i];
                    ap[i] = c * x - s * y;
                    aq[i] = s * x + c * y;
                }
                double* vp = &v[(size_t)p * n];
                double* vq = &v[(size_t)q * n];
                for (int i = 0; i < n; ++i) {
                    double x = vp[i], y = vq[i];
                    vp[i] = c * x - s * y;
                    vq[i] = s * x + c * y;
                }
                ++rotated;
            }
            // rotate the ring, keeping ring[0] fixed
            int last = ring[m - 1];
            for (int i = m - 1; i > 1; --i) ring[i] = ring[i - 1];
            ring[1] = last;
        }
        if (rotated == 0) break;
    }
    std::vector<double> sig(n);
    double smax = 0;
    for (int j = 0; j < n; ++j) {
        double s2 = 0;
        for (int i = 0; i < n; ++i) s2 += a[(size_t)j * n + i] * a[(size_t)j * n + i];
        sig[j] = std::sqrt(s2);
        smax = std::max(smax, sig[j]);
    }
    // pinv = V diag(1/s) U^T with u_j = a_j / s_j  =>  pinv[r][c] = sum_j v[r][j] a[c][j] / s_j^2
    // kept: s_j > cutoff s_max, and at most max_rank of them (the largest) when max_rank > 0
    double thresh = cutoff * smax;
    if (max_rank > 0) {
        std::vector<double> s(sig);
        std::sort(s.begin(), s.end(), std::greater<double>());
        if ((int)s.size() > max_rank && s[max_rank] > thresh) thresh = s[max_rank];
    }
    std::vector<double> w(n);
    for (int j = 0; j < n; ++j) w[j] = (sig[j] > thresh) ? 1.0 / (sig[j] * sig[j]) : 0.0;
    std::vector<double> P((size_t)n * n);
#pragma omp parallel for schedule(static)
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            double acc = 0;
            for (int j = 0; j < n; ++j) acc += v[(size_t)j * n + r] * a[(size_t)j * n + c] * w[j];
            P[(size_t)r * n + c] = acc;
        }
    if (U && W && rank) {
        // kept triplets in index order: u_j = a_j / s_j, w_j = v_j / s_j
        std::vector<int> kept;
        for (int j = 0; j < n; ++j)
            if (w[j] > 0) kept.push_back(j);
        const int r = (int)kept.size();
        U->assign((size_t)n * r, 0.0);
        W->assign((size_t)n * r, 0.0);
        for (int k = 0; k < r; ++k) {
            const int j = kept[k];
            for (int i = 0; i < n; ++i) {
                (*U)[(size_t)i * r + k] = a[(size_t)j * n + i] / sig[j];
                (*W)[(size_t)i * r + k] = v[(size_t)j * n + i] / sig[j];
            }
        }
        *rank = r;
    }
    return P;
}

static std::vector<double> kernel_matrix(const std::vector<double>& x, double sx,
                                         const std::vector<double>& y, double sy) {
    int n = (int)x.size() / 3, m = (int)y.size() / 3;
    std::vector<double> K((size_t)n * m);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double dx = sx * x[3 * i] - sy * y[3 * j], dy = sx * x[3 * i + 1] - sy * y[3 * j + 1],
                   dz = sx * x[3 * i + 2] - sy * y[3 * j + 2];
            K[(size_t)i * m + j] = 1.0 / std::sqrt(dx * dx + dy * dy + dz * dz);
        }
    return K;
}

const HostPinv& host_pinv(int p, double cut_up, double cut_dn, int max_up, int max_dn) {
    static std::mutex mu;
    static std::map<std::tuple<int, double, double, int, int>, HostPinv> cache;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_tuple(p, cut_up, cut_dn, max_up, max_dn);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    HostPinv h;
    h.p = p;
    h.surf = surface_points(p);
    h.Q = (int)h.surf.size() / 3;
    h.Pu = pinv_jacobi(kernel_matrix(h.surf, kUpCheck, h.surf, kUpEquiv), h.Q, cut_up, &h.Uu, &h.Wu, &h.ru, max_up);
    h.Pd = pinv_jacobi(kernel_matrix(h.surf, kDnCheck, h.surf, kDnEquiv), h.Q, cut_dn, &h.Ud, &h.Wd, &h.rd, max_dn);
    return cache.emplace(key, std::move(h)).first->second;
}

const UpPivots& host_up_pivots(int p) {
    static std::mutex mu;
    static std::map<int, UpPivots> cache;
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(p);
    if (it != cache.end()) return it->second;
    const std::vector<double> s = surface_points(p);
    const int n = (int)s.size() / 3;
    // a: column j = row j of K(check, equivalent), i.e. column j of A (column-major)
    std::vector<double> a = kernel_matrix(s, kUpCheck, s, kUpEquiv);
    UpPivots f;
    f.n = n;
    f.perm.resize(n);
    for (int j = 0; j < n; ++j) f.perm[j] = j;
    std::vector<double> v(n);
    for (int i = 0; i < n; ++i) {
        // the trailing column of largest norm (norms recomputed, not downdated)
        int best = i;
        double bn = -1.0;
        for (int j = i; j < n; ++j) {
            const double* c = &a[(size_t)j * n];
            double t = 0.0;
            for (int r = i; r < n; ++r) t += c[r] * c[r];
            if (t > bn) {
                bn = t;
                best = j;
            }
        }
        if (best != i) {
            std::swap_ranges(a.begin() + (size_t)i * n, a.begin() + (size_t)(i + 1) * n, a.begin() + (size_t)best * n);
            std::swap(f.perm[i], f.perm[best]);
        }
        // Householder reflection taking column i's trailing part to alpha e_i
        double* c = &a[(size_t)i * n];
        const double nx = std::sqrt(bn > 0 ? bn : 0.0);
        if (nx == 0.0) continue;
        const double alpha = c[i] > 0 ? -nx : nx;
        double vn = 0.0;
        for (int r = i; r < n; ++r) {
            v[r] = c[r] - (r == i ? alpha : 0.0);
            vn += v[r] * v[r];
        }
        c[i] = alpha;
        for (int r = i + 1; r < n; ++r) c[r] = 0.0;
        if (vn == 0.0) continue;
#pragma omp parallel for schedule(static)
        for (int j = i + 1; j < n; ++j) {
            double* cj = &a[(size_t)j * n];
            double t = 0.0;
            for (int r = i; r < n; ++r) t += v[r] * cj[r];
            t = 2.0 * t / vn;
            for (int r = i; r < n; ++r) cj[r] -= t * v[r];
        }
    }
    f.R.assign((size_t)n * n, 0.0);
    for (int c = 0; c < n; ++c)
        for (int r = 0; r <= c; ++r) f.R[(size_t)r * n + c] = a[(size_t)c * n + r];
    return cache.emplace(p, std::move(f)).first->second;
}

int up_pivot_count(const UpPivots& f, double tol) {
    if (f.n == 0) return 0;
    const double r0 = std::fabs(f.R[0]);
    int k = 0;
    for (int i = 0; i < f.n; ++i)
        if (std::fabs(f.R[(size_t)i * f.n + i]) > tol * r0) ++k;
    return k;
}

void up_skeleton(const UpPivots& f, int k, std::vector<int>& idx, std::vector<double>& E) {
    const int n = f.n;
    k = std::max(0, std::min(k, n));
    idx.assign(f.perm.begin(), f.perm.begin() + k);
    E.assign((size_t)n * k, 0.0);
    for (int m = 0; m < k; ++m) E[(size_t)f.perm[m] * k + m] = 1.0;
    // column j of T = R11^-1 R12 by back substitution, one per non-skeleton point
#pragma omp parallel for schedule(static)
    for (int j = k; j < n; ++j) {
        std::vector<double> t(k);
        for (int m = k - 1; m >= 0; --m) {
            double acc = f.R[(size_t)m * n + j];
            for (int l = m + 1; l < k; ++l) acc -= f.R[(size_t)m * n + l] * t[l];
            t[m] = acc / f.R[(size_t)m * n + m];
        }
        for (int m = 0; m < k; ++m) E[(size_t)f.perm[j] * k + m] = t[m];
    }
}

// out[orow[r]*Cp + j] = ascale[r] * sum_m G(a_r, b_{bset[r], m}) P[m][j],  j < C; 0 for C <= j < Cp
// (P is Q x C: the Q points of a b set by C columns)
// G = 1/|a-b| (kfun 0) or n_r.(a-b)/|a-b|^3 (kfun 1).  8 rows per block.
template <typename Real>
__global__ void k_build_rows(int nrows, const double* __restrict__ apts, const double* __restrict__ anrm,
                             const double* __restrict__ ascale, const int* __restrict__ bset,
                             const int64_t* __restrict__ orow, const double* __restrict__ bpts, int Q,
                             int C, int Cp, const double* __restrict__ P, int kfun, Real* __restrict__ out) {
    extern __shared__ double Ks[];  // [8][Q]
    const int R = 8;
    int r0 = blockIdx.x * R;
    for (int e = threadIdx.x; e < R * Q; e += blockDim.x) {
        int r = e / Q, m = e % Q;
        int row = r0 + r;
        double val = 0.0;
        if (row < nrows) {
            const double* b = bpts + ((size_t)(bset ? bset[row] : 0) * Q + m) * 3;
            double dx = apts[3 * row] - b[0], dy = apts[3 * row + 1] - b[1], dz = apts[3 * row + 2] - b[2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double inv = 1.0 / sqrt(r2);
            if (kfun == 0) {
                val = inv;
            } else {
                double nd = anrm[3 * row] * dx + anrm[3 * row + 1] * dy + anrm[3 * row + 2] * dz;
                val = nd * inv * inv * inv;
            }
        }
        Ks[r * Q + m] = val;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < Cp; j += blockDim.x) {
        double acc[8];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = 0.0;
        if (j < C) {
            for (int m = 0; m < Q; ++m) {
                double pm = P[(size_t)m * C + j];
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] += Ks[r * Q + m] * pm;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            int row = r0 + r;
            if (row < nrows) out[(size_t)orow[row] * Cp + j] = (Real)(ascale[row] * acc[r]);
        }
    }
}

template <typename Real>
int build_rows(const RowSpec& rs, int Q, int C, int Cp, const double* dP, int kfun, Real* out,
               cudaStream_t s) {
    if (rs.nrows == 0) return KIFMM_OK;
    size_t smem = 8 * (size_t)Q * sizeof(double);
    if (smem > 48 * 1024)
        KF_CHECK_CUDA(cudaFuncSetAttribute(k_build_rows<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
    k_build_rows<Real><<<div_up(rs.nrows, 8), 256, smem, s>>>(rs.nrows, rs.apts, rs.anrm, rs.ascale,
                                                              rs.bset, rs.orow, rs.bpts, Q, C, Cp, dP, kfun,
                                                              out);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

template int build_rows<float>(const RowSpec&, int, int, int, const double*, int, float*, cudaStream_t);
template int build_rows<double>(const RowSpec&, int, int, int, const double*, int, double*, cudaStream_t);

// Host-side row descriptors of the three translation-operator tables.
void translation_rows(const HostPinv& h, int which, std::vector<double>& apts, std::vector<int>& bset,
                      std::vector<int64_t>& orow, std::vector<double>& ascale,
                      std::vector<double>& bpts, int Qp) {
    const int Q = h.Q;
    const std::vector<double>& s = h.surf;
    apts.clear();
    bset.clear();
    orow.clear();
    ascale.clear();
    bpts.clear();
    auto oct_center = [](int o, double c[3]) {
        c[0] = ((o >> 2) & 1) ? 0.5 : -0.5;
        c[1] = ((o >> 1) & 1) ? 0.5 : -0.5;
        c[2] = (o & 1) ? 0.5 : -0.5;
    };
    if (which == 0) {  // M2M'
        for (int o = 0; o < 8; ++o) {
            double c[3];
            oct_center(o, c);
            for (int m = 0; m < Q; ++m)
                for (int d = 0; d < 3; ++d) bpts.push_back(c[d] + 0.5 * kUpEquiv * s[3 * m + d]);
            for (int i = 0; i < Q; ++i) {
                for (int d = 0; d < 3; ++d) apts.push_back(kUpCheck * s[3 * i + d]);
                bset.push_back(o);
                orow.push_back((int64_t)o * Qp + i);
                ascale.push_back(0.5);
            }
        }
    } else if (which == 1) {  // M2L'
        for (int g = 0; g < kNumOffsets; ++g) {
            int ox = g / 49 - 3, oy = (g / 7) % 7 - 3, oz = g % 7 - 3;
            for (int m = 0; m < Q; ++m) {
                bpts.push_back(2.0 * ox + kUpEquiv * s[3 * m]);
                bpts.push_back(2.0 * oy + kUpEquiv * s[3 * m + 1]);
                bpts.push_back(2.0 * oz + kUpEquiv * s[3 * m + 2]);
            }
            if (std::max(std::abs(ox), std::max(std::abs(oy), std::abs(oz))) <= 1) continue;
            for (int i = 0; i < Q; ++i) {
                for (int d = 0; d < 3; ++d) apts.push_back(kDnCheck * s[3 * i + d]);
                bset.push_back(g);
                orow.push_back((int64_t)g * Qp + i);
                ascale.push_back(1.0);
            }
        }
    } else {  // L2L'
        for (int m = 0; m < Q; ++m)
            for (int d = 0; d < 3; ++d) bpts.push_back(kDnEquiv * s[3 * m + d]);
        for (int o = 0; o < 8; ++o) {
            double c[3];
            oct_center(o, c);
            for (int i = 0; i < Q; ++i) {
                for (int d = 0; d < 3; ++d) apts.push_back(c[d] + 0.5 * kDnCheck * s[3 * i + d]);
                bset.push_back(0);
                orow.push_back((int64_t)o * Qp + i);
                ascale.push_back(1.0);
            }
        }
    }
}

}  // namespace kifmm
