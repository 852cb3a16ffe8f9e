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
std::vector<double> pinv_jacobi(const std::vector<double>& A_rm, int n, double cutoff,
                                std::vector<double>* U = nullptr, std::vector<double>* W = nullptr,
                                int* rank = nullptr);
const HostPinv& host_pinv(int p, double cutoff);

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
