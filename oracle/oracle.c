/*
 * Oracle for the Laplace boundary sums -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg load this
 * library.  It shares no code with the CUDA path.  Everything here is the plain
 * O(N^2) definition in FP64, one target at a time, sources summed in index
 * order:
 *
 *   the discrete kernel sum f(r_i) = sum_j K(r_i, r_j) q_j   (Sec. II.A, Eq. sum_fmm)
 *
 * with q_j = sigma_j * w_j (density times quadrature weight, Sec. III.A.1) and
 *
 *   SL : K = 1 / |r_i - r_j|                                  (the 1/r kernel K_r of Sec. III.A.1)
 *   DL : K = n_j . (r_i - r_j) / |r_i - r_j|^3               (Eq. kernel, source normal)
 *   ADL: K = n_i . (r_i - r_j) / |r_i - r_j|^3               (Eq. kernel_pol dotted with the
 *                                                             target normal as in Eq. Ax)
 *
 * A pair closer than the tolerance radius delta contributes nothing (Sec. III.A.1,
 * the 1e-5 tolerance radius around each target); the test is |r_i - r_j|^2 < delta^2.
 * The sums are raw: the 1/(4 pi) prefactors of Eqs. fk_integral and Eb are
 * applied by the boundary-integral operators above this layer.
 *
 * Layouts: coordinates and normals are structure-of-arrays, x[0..n) then y then z.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORACLE_SL = 0, ORACLE_DL = 1, ORACLE_ADL = 2 };

static double pair_value(int kernel, double dx, double dy, double dz, double r2,
                         const double* src_nrm, int64_t ns, int64_t j,
                         const double* trg_nrm, int64_t nt, int64_t i)
{
    double r = sqrt(r2);
    if (kernel == ORACLE_SL)
        return 1.0 / r;
    if (kernel == ORACLE_DL) {
        double nd = src_nrm[j] * dx + src_nrm[ns + j] * dy + src_nrm[2 * ns + j] * dz;
        return nd / (r2 * r);
    }
    double nd = trg_nrm[i] * dx + trg_nrm[nt + i] * dy + trg_nrm[2 * nt + i] * dz;
    return nd / (r2 * r);
}

/* out[k] = sum_j K(trg[t], src[j]) q[j] for t = idx[k] (idx == NULL: t = k, nidx = nt).
 * Returns 0, or -1 on a bad argument. */
int oracle_direct(int kernel,
                  const double* trg, const double* trg_nrm, int64_t nt,
                  const int64_t* idx, int64_t nidx,
                  const double* src, const double* src_nrm, const double* q, int64_t ns,
                  double delta, double* out, int nthreads)
{
    if (kernel < ORACLE_SL || kernel > ORACLE_ADL) return -1;
    if (kernel == ORACLE_DL && !src_nrm) return -1;
    if (kernel == ORACLE_ADL && !trg_nrm) return -1;
    if (!idx) nidx = nt;
    const double d2 = delta * delta;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t k = 0; k < nidx; ++k) {
        int64_t i = idx ? idx[k] : k;
        double xi = trg[i], yi = trg[nt + i], zi = trg[2 * nt + i];
        double acc = 0.0;
        for (int64_t j = 0; j < ns; ++j) {
            double dx = xi - src[j], dy = yi - src[ns + j], dz = zi - src[2 * ns + j];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < d2) continue;
            acc += q[j] * pair_value(kernel, dx, dy, dz, r2, src_nrm, ns, j, trg_nrm, nt, i);
        }
        out[k] = acc;
    }
    return 0;
}

/* Number of OpenMP threads a parallel region uses (for reporting). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
