// The Chebyshev-interpolation far field (see cheb.cu): node sets, translation tables and
// the two kernels that differ from the equivalent-density engine's.
#pragma once

#include <vector>

#include "common.cuh"
#include "plan.cuh"

namespace kifmm {

constexpr int kChebMaxN = 8;          // nodes per dimension (Q = n^3 <= 512)

// the n nodes cos((2i + 1) pi / 2n) of [-1, 1]; the n^3 box nodes, x outermost (Q x 3)
std::vector<double> cheb_nodes_1d(int n);
std::vector<double> cheb_nodes(int n);
// Unit-box tables (FP64, Qp x Qp each, row = output node): M2M (8, with the factor 1/2
// of the upward vector W / h), M2L (343 offsets; near ones zero), L2L (8).
void cheb_host_tables(int n, int Qp, std::vector<double>& m2m, std::vector<double>& m2l, std::vector<double>& l2l);
// S2M of the boxes of a CSR list into out (nbox x Qp, the upward vector W / h).
int cheb_s2m(const Plan& P, const Tree& T, bool dl, int nbox, const int* boxes, const int* off, const int* idx,
             const double* q, double* out, cudaStream_t s);
// L2P rows (T.nt x Qp): interpolation weights, or for grad the gradient along tnrm
// (per target) or, tnrm null, along coordinate axis.
int cheb_rows(const Plan& P, const Tree& T, const int* tleaf_of, const double* tnrm, int axis, bool grad, double* out,
              cudaStream_t s);

}  // namespace kifmm
