// The Chebyshev-interpolation far field (the black-box FMM the paper's ScalFMM runs:
// Sec. I and Sec. III.A.1, Eq. p2m) as a second engine behind the same plan: n
// Chebyshev nodes per dimension in every box, Q = n^3.
//
// With S_n(x, y) = prod_d S(x_d, y_d), S(x, u) = 1/n + (2/n) sum_{k=1}^{n-1} T_k(x) T_k(u)
// on [-1, 1] (box coordinates: u = (y - c)/h, h the half-width):
//   S2M  W_m = sum_j S_n(xbar_m, u_j) q_j          (double layer: the source-side
//        derivative, W_m = (1/h) sum_j q_j n_j . grad_u S_n(xbar_m, u_j) -- Eq. p2m)
//   M2M  W_parent = sum over children of S_n(xbar_m, c_o + xbar_m' / 2) W_child
//   M2L  L_m = sum_m' K(xbar_m, 2t + xbar_m') W_m' / h   (t: the source box's offset)
//   L2L  L_child,m = sum_m' S_n(xbar_m', c_o + xbar_m / 2) L_parent,m'
//   L2P  f(x) = sum_m S_n(xbar_m, u) L_m           (gradient kernels: minus its gradient / h)
// The plan's FP64 form carries these in its check-potential slots: the upward vector is
// W / h (so M2L is one table per offset at every level and M2M takes a factor 1/2), the
// downward one L; X-list sources are evaluated at the nodes directly, W-list sources in
// the near field, as in the other engine.
#include <cmath>
#include <vector>

#include "cheb.cuh"

namespace kifmm {

namespace {

constexpr double kPi = 3.14159265358979323846;

// T_k(u), k < n
inline void cheb_t(int n, double u, double* t) {
    t[0] = 1.0;
    if (n > 1) t[1] = u;
    for (int k = 2; k < n; ++k) t[k] = 2.0 * u * t[k - 1] - t[k - 2];
}

// S(xbar_i, u) for the n nodes of one dimension
inline void cheb_s(int n, const double* xb, double u, double* s) {
    double tu[kChebMaxN];
    cheb_t(n, u, tu);
    for (int i = 0; i < n; ++i) {
        double tx[kChebMaxN];
        cheb_t(n, xb[i], tx);
        double v = 1.0 / n;
        for (int k = 1; k < n; ++k) v += 2.0 / n * tx[k] * tu[k];
        s[i] = v;
    }
}

}  // namespace

std::vector<double> cheb_nodes_1d(int n) {
    std::vector<double> x(n);
    for (int i = 0; i < n; ++i) x[i] = std::cos((2.0 * i + 1.0) * kPi / (2.0 * n));
    return x;
}

std::vector<double> cheb_nodes(int n) {
    const std::vector<double> x = cheb_nodes_1d(n);
    std::vector<double> p;
    p.reserve(3 * (size_t)n * n * n);
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n; ++b)
            for (int c = 0; c < n; ++c) {
                p.push_back(x[a]);
                p.push_back(x[b]);
                p.push_back(x[c]);
            }
    return p;
}

void cheb_host_tables(int n, int Qp, std::vector<double>& m2m, std::vector<double>& m2l, std::vector<double>& l2l) {
    const int Q = n * n * n;
    const std::vector<double> xb = cheb_nodes_1d(n), nodes = cheb_nodes(n);
    m2m.assign(8 * (size_t)Qp * Qp, 0.0);
    l2l.assign(8 * (size_t)Qp * Qp, 0.0);
    m2l.assign((size_t)kNumOffsets * Qp * Qp, 0.0);
    for (int o = 0; o < 8; ++o) {
        const double co[3] = {((o >> 2) & 1) ? 0.5 : -0.5, ((o >> 1) & 1) ? 0.5 : -0.5, (o & 1) ? 0.5 : -0.5};
        // S(xbar_i, c_o + xbar_k / 2) per dimension: sc[d][k][i]
        std::vector<double> sc(3 * (size_t)n * n);
        for (int d = 0; d < 3; ++d)
            for (int k = 0; k < n; ++k) cheb_s(n, xb.data(), co[d] + 0.5 * xb[k], &sc[((size_t)d * n + k) * n]);
        for (int m = 0; m < Q; ++m) {
            const int i0 = m / (n * n), i1 = (m / n) % n, i2 = m % n;          // parent node
            for (int mc = 0; mc < Q; ++mc) {
                const int k0 = mc / (n * n), k1 = (mc / n) % n, k2 = mc % n;   // child node
                const double v = sc[((size_t)0 * n + k0) * n + i0] * sc[((size_t)1 * n + k1) * n + i1] *
                                 sc[((size_t)2 * n + k2) * n + i2];
                m2m[(size_t)o * Qp * Qp + (size_t)m * Qp + mc] = 0.5 * v;      // W/h: child h = parent h / 2
                l2l[(size_t)o * Qp * Qp + (size_t)mc * Qp + m] = v;            // child node mc <- parent node m
            }
        }
    }
    for (int g = 0; g < kNumOffsets; ++g) {
        const int ox = g / 49 - 3, oy = (g / 7) % 7 - 3, oz = g % 7 - 3;
        if (std::max(std::abs(ox), std::max(std::abs(oy), std::abs(oz))) <= 1) continue;
        double* T = &m2l[(size_t)g * Qp * Qp];
        for (int m = 0; m < Q; ++m)
            for (int mp = 0; mp < Q; ++mp) {
                const double dx = nodes[3 * m] - (2.0 * ox + nodes[3 * mp]);
                const double dy = nodes[3 * m + 1] - (2.0 * oy + nodes[3 * mp + 1]);
                const double dz = nodes[3 * m + 2] - (2.0 * oz + nodes[3 * mp + 2]);
                T[(size_t)m * Qp + mp] = 1.0 / std::sqrt(dx * dx + dy * dy + dz * dz);
            }
    }
}

namespace {

// The node table of one dimension, passed by value: t[i][k] = T_k(xbar_i).
struct ChebTx {
    double t[kChebMaxN * kChebMaxN];
};

// S(xbar_i, u) and dS/du for the n nodes of one dimension, from T_k(u) and
// T'_k(u) = k U_{k-1}(u) (U_0 = 1, U_1 = 2u, U_j = 2u U_{j-1} - U_{j-2}).
template <bool DERIV>
__device__ __forceinline__ void dev_cheb_s(int n, const ChebTx& tx, double u, double* s, double* ds) {
    double t[kChebMaxN], dt[kChebMaxN], uu[kChebMaxN];
    t[0] = 1.0;
    uu[0] = 1.0;
    if (n > 1) {
        t[1] = u;
        uu[1] = 2.0 * u;
    }
    for (int k = 2; k < n; ++k) {
        t[k] = 2.0 * u * t[k - 1] - t[k - 2];
        uu[k] = 2.0 * u * uu[k - 1] - uu[k - 2];
    }
    dt[0] = 0.0;
    for (int k = 1; k < n; ++k) dt[k] = k * uu[k - 1];
    for (int i = 0; i < n; ++i) {
        double v = 1.0 / n, dv = 0.0;
        for (int k = 1; k < n; ++k) {
            v += 2.0 / n * tx.t[i * kChebMaxN + k] * t[k];
            if (DERIV) dv += 2.0 / n * tx.t[i * kChebMaxN + k] * dt[k];
        }
        s[i] = v;
        if (DERIV) ds[i] = dv;
    }
}

ChebTx make_tx(int n) {
    ChebTx tx{};
    const std::vector<double> xb = cheb_nodes_1d(n);
    for (int i = 0; i < n; ++i) cheb_t(n, xb[i], &tx.t[(size_t)i * kChebMaxN]);
    return tx;
}

// S2M for the leaves of a CSR list (each leaf and itself): one block per box, threads
// over the Q nodes; each staged source carries its 3n interpolation weights (and, for
// dipoles, 3n derivatives).  out[b Qp + m] = W_m / h (monopoles) or the double layer's
// (1/h^2) sum_j q_j n_j . grad_u S_n.
template <bool DL>
__global__ void __launch_bounds__(128)
k_cheb_s2m(const int* __restrict__ boxes, const int* __restrict__ off, const int* __restrict__ idx, int n,
           const ChebTx tx, int Q, int Qp, const int* __restrict__ lvl, const double* __restrict__ ctr, double root_h,
           const int64_t* __restrict__ rng, const double* __restrict__ sxyz, int64_t ns, const double* __restrict__ qs,
           double* __restrict__ out) {
    constexpr int kStage = 32;
    constexpr int W = DL ? 6 : 3;          // weight rows per dimension set: S (and S')
    __shared__ double sw[kStage][W * kChebMaxN];
    __shared__ double sq[kStage][3];
    const int b = boxes[blockIdx.x];
    const double h = ldexp(root_h, -lvl[b]), ih = 1.0 / h;
    const double c[3] = {ctr[3 * b], ctr[3 * b + 1], ctr[3 * b + 2]};
    constexpr int kPer = (kChebMaxN * kChebMaxN * kChebMaxN + 127) / 128;
    double acc[kPer];
#pragma unroll
    for (int i = 0; i < kPer; ++i) acc[i] = 0.0;
    for (int e = off[blockIdx.x]; e < off[blockIdx.x + 1]; ++e) {
        const int a = idx[e];
        const int64_t sb = rng[4 * a], se = rng[4 * a + 1];
        for (int64_t j0 = sb; j0 < se; j0 += kStage) {
            const int cnt = (int)((se - j0) < kStage ? (se - j0) : kStage);
            if (threadIdx.x < cnt) {
                const int64_t j = j0 + threadIdx.x;
                for (int d = 0; d < 3; ++d) {
                    const double u = (sxyz[d * ns + j] - c[d]) * ih;
                    dev_cheb_s<DL>(n, tx, u, &sw[threadIdx.x][d * kChebMaxN], DL ? &sw[threadIdx.x][(3 + d) * kChebMaxN] : nullptr);
                    sq[threadIdx.x][d] = DL ? qs[d * ns + j] : (d == 0 ? qs[j] : 0.0);
                }
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kPer; ++i) {
                const int m = threadIdx.x + 128 * i;
                if (m < Q) {
                    const int i0 = m / (n * n), i1 = (m / n) % n, i2 = m % n;
                    double v = acc[i];
                    for (int jj = 0; jj < cnt; ++jj) {
                        const double* wv = sw[jj];
                        if (DL) {
                            const double sx = wv[i0], sy = wv[kChebMaxN + i1], sz = wv[2 * kChebMaxN + i2];
                            const double gx = wv[3 * kChebMaxN + i0], gy = wv[4 * kChebMaxN + i1],
                                         gz = wv[5 * kChebMaxN + i2];
                            v += sq[jj][0] * gx * sy * sz + sq[jj][1] * sx * gy * sz + sq[jj][2] * sx * sy * gz;
                        } else {
                            v += sq[jj][0] * wv[i0] * wv[kChebMaxN + i1] * wv[2 * kChebMaxN + i2];
                        }
                    }
                    acc[i] = v;
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        const int m = threadIdx.x + 128 * i;
        if (m < Qp) out[(size_t)b * Qp + m] = m < Q ? acc[i] * (DL ? ih * ih : ih) : 0.0;
    }
}

// L2P rows: row t of Qp = the interpolation weights S_n(xbar_m, u_t) of its leaf's nodes,
// or (gradient kernels) -(1/h) nvec . grad_u S_n with nvec the target normal (tnrm) or
// the unit vector of coordinate axis: the kernels n_i . (r_i - r_j)/|r_i - r_j|^3 and
// (r_i - r_j)/|r_i - r_j|^3 are minus the gradient of 1/|r_i - r_j| at the target.
template <bool GRAD>
__global__ void k_cheb_rows(const int* __restrict__ tleaf_of, int64_t nt, const double* __restrict__ txyz,
                            const double* __restrict__ tnrm, int axis, const int* __restrict__ lvl,
                            const double* __restrict__ ctr, double root_h, int n, const ChebTx tx, int Q, int Qp,
                            double* __restrict__ out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int b = tleaf_of[t];
    const double h = ldexp(root_h, -lvl[b]), ih = 1.0 / h;
    double s[3][kChebMaxN], ds[3][kChebMaxN];
    for (int d = 0; d < 3; ++d) dev_cheb_s<GRAD>(n, tx, (txyz[d * nt + t] - ctr[3 * b + d]) * ih, s[d], ds[d]);
    double nv[3] = {0.0, 0.0, 0.0};
    if (GRAD)
        for (int d = 0; d < 3; ++d) nv[d] = tnrm ? tnrm[d * nt + t] : (d == axis ? 1.0 : 0.0);
    double* row = out + (size_t)t * Qp;
    for (int m = 0; m < Qp; ++m) {
        double v = 0.0;
        if (m < Q) {
            const int i0 = m / (n * n), i1 = (m / n) % n, i2 = m % n;
            if (GRAD)
                v = -ih * (nv[0] * ds[0][i0] * s[1][i1] * s[2][i2] + nv[1] * s[0][i0] * ds[1][i1] * s[2][i2] +
                           nv[2] * s[0][i0] * s[1][i1] * ds[2][i2]);
            else
                v = s[0][i0] * s[1][i1] * s[2][i2];
        }
        row[m] = v;
    }
}

}  // namespace

int cheb_s2m(const Plan& P, const Tree& T, bool dl, int nbox, const int* boxes, const int* off, const int* idx,
             const double* q, double* out, cudaStream_t s) {
    if (nbox <= 0) return KIFMM_OK;
    const ChebTx tx = make_tx(P.p);
    if (dl)
        k_cheb_s2m<true><<<nbox, 128, 0, s>>>(boxes, off, idx, P.p, tx, P.Q, P.Qp, T.lvl.p, T.ctr.p, T.root_h,
                                              T.rng.p, T.sxyz.p, T.ns, q, out);
    else
        k_cheb_s2m<false><<<nbox, 128, 0, s>>>(boxes, off, idx, P.p, tx, P.Q, P.Qp, T.lvl.p, T.ctr.p, T.root_h,
                                               T.rng.p, T.sxyz.p, T.ns, q, out);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

int cheb_rows(const Plan& P, const Tree& T, const int* tleaf_of, const double* tnrm, int axis, bool grad, double* out,
              cudaStream_t s) {
    if (T.nt == 0) return KIFMM_OK;
    const ChebTx tx = make_tx(P.p);
    const double* txyz = T.same ? T.sxyz.p : T.txyz.p;
    if (grad)
        k_cheb_rows<true><<<div_up(T.nt, 128), 128, 0, s>>>(tleaf_of, T.nt, txyz, tnrm, axis, T.lvl.p, T.ctr.p,
                                                            T.root_h, P.p, tx, P.Q, P.Qp, out);
    else
        k_cheb_rows<false><<<div_up(T.nt, 128), 128, 0, s>>>(tleaf_of, T.nt, txyz, tnrm, axis, T.lvl.p, T.ctr.p,
                                                             T.root_h, P.p, tx, P.Q, P.Qp, out);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}

}  // namespace kifmm
