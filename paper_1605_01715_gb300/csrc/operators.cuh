// KIFMM operator construction (FP64 host SVD + FP64 device builder).
#pragma once

#include <vector>

#include "common.cuh"

namespace kifmm {

constexpr double kUpEquiv = 1.05;   // upward equivalent surface / half-width
constexpr double kUpCheck = 2.95;   // upward check surface
constexpr double kDnCheck = 1.05;   // downward check surface
constexpr double kDnEquiv = 2.95;   // downward equivalent surface

struct HostPinv {
    int p = 0, Q = 0;
    std::vector<double> surf;       // Q x 3 unit-cube surface points
    std::vector<double> Pu, Pd;     // Q x Q row-major pseudo-inverses (unit box)
    // Factored form of the same pseudo-inverses, P = W U^T over the r kept singular
    // triplets (A V = U S, kept: s_j > cutoff s_max): U (Q x r, orthonormal columns, a
    // basis of the check space P acts on) and W = V S^-1 = P U (Q x r), row-major.
    int ru = 0, rd = 0;
    std::vector<double> Uu, Wu, Ud, Wd;
};

std::vector<double> surface_points(int p);
// Pseudo-inverse (n x n, row-major) by one-sided Jacobi SVD; U and W (n x rank,
// row-major) of its factored form when requested.
// Singular values above cutoff * sigma_max are kept, and at most max_rank of them (the
// largest) when max_rank > 0.
std::vector<double> pinv_jacobi(const std::vector<double>& A_rm, int n, double cutoff,
                                std::vector<double>* U = nullptr, std::vector<double>* W = nullptr,
                                int* rank = nullptr, int max_rank = 0);
// Pu truncated at cut_up * sigma_max and to at most max_up singular triplets, Pd at
// cut_dn * sigma_max and max_dn (0: no cap); cached per (p, cuts, caps).
const HostPinv& host_pinv(int p, double cut_up, double cut_dn, int max_up = 0, int max_dn = 0);

// Column-pivoted Householder QR of A = K(2.95 s_i, 1.05 s_j)^T, the transposed map from
// the upward equivalent surface to the upward check surface (both Q points of the unit
// box), in FP64: A[:, perm] = Q R.  Its pivots order the check points so that the first
// k of them interpolate the rest (up_skeleton).  Cached per order.
struct UpPivots {
    int n = 0;
    std::vector<int> perm;          // check point of each pivot position
    std::vector<double> R;          // n x n upper triangle, row-major
};
const UpPivots& host_up_pivots(int p);
// Pivots with |R_ii| > tol |R_00|.
int up_pivot_count(const UpPivots& f, double tol);
// Skeleton of the upward check surface (an interpolative decomposition; the method
// itself evaluates all Q points): idx = the first k pivots and E (Q x k, row-major)
// with E[idx[m]][m] = 1 and, for every other point, the row T = R11^-1 R12 gives.  The
// potential u of any upward equivalent density, and so of any source inside the box,
// then satisfies u(c_i) = sum_m E[i][m] u(c_idx[m]) up to the QR's truncation after k
// pivots.  k = n gives the identity.
void up_skeleton(const UpPivots& f, int k, std::vector<int>& idx, std::vector<double>& E);

// Device row descriptors for build_rows (all device pointers); a table row is
// ascale * G(a, B) P with P an (Q x C) matrix, stored C of Cp wide (zero padding).
struct RowSpec {
    int nrows = 0;
    const double* apts = nullptr;    // 3 per row
    const double* anrm = nullptr;    // 3 per row (kfun 1)
    const double* ascale = nullptr;  // 1 per row
    const int* bset = nullptr;       // 1 per row (NULL: set 0)
    const int64_t* orow = nullptr;   // output row index per row
    const double* bpts = nullptr;    // sets of Q points, 3 doubles each
};

template <typename Real>
int build_rows(const RowSpec& rs, int Q, int C, int Cp, const double* dP, int kfun, Real* out, cudaStream_t s);

// which: 0 = M2M', 1 = M2L', 2 = L2L'
void translation_rows(const HostPinv& h, int which, std::vector<double>& apts, std::vector<int>& bset,
                      std::vector<int64_t>& orow, std::vector<double>& ascale, std::vector<double>& bpts,
                      int Qp);

}  // namespace kifmm
