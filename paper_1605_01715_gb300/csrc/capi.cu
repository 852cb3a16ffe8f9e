// Error reporting, version, and the one-point quadrature rule of Sec. III.
#include <stdarg.h>

#include <cmath>

#include "common.cuh"

namespace kifmm {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = 0; }

namespace {

// Per triangle: centroid; on a sphere the spherical-triangle area R^2 E with the
// excess from tan(E/2) = |a.(b x c)| / (1 + a.b + b.c + c.a) (Van Oosterom &
// Strackee 1983) and the radial normal at the centroid; otherwise the flat area and
// the unit facet normal of the vertex winding (Sec. III, electrostatic implementation).
__global__ void k_quadrature(const double* __restrict__ tri, const double* __restrict__ sph, int64_t n,
                             double* __restrict__ xyz, double* __restrict__ w, double* __restrict__ nrm) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    double A[3], B[3], C[3], c[3];
    for (int d = 0; d < 3; ++d) {
        A[d] = tri[9 * t + d];
        B[d] = tri[9 * t + 3 + d];
        C[d] = tri[9 * t + 6 + d];
        c[d] = (A[d] + B[d] + C[d]) / 3.0;
        xyz[d * n + t] = c[d];
    }
    double R = sph[4 * t + 3];
    if (R > 0) {
        double o[3] = {sph[4 * t], sph[4 * t + 1], sph[4 * t + 2]};
        double a[3], b[3], e[3];
        double la = 0, lb = 0, le = 0;
        for (int d = 0; d < 3; ++d) {
            a[d] = A[d] - o[d];
            b[d] = B[d] - o[d];
            e[d] = C[d] - o[d];
            la += a[d] * a[d];
            lb += b[d] * b[d];
            le += e[d] * e[d];
        }
        la = sqrt(la);
        lb = sqrt(lb);
        le = sqrt(le);
        for (int d = 0; d < 3; ++d) {
            a[d] /= la;
            b[d] /= lb;
            e[d] /= le;
        }
        double bx = b[1] * e[2] - b[2] * e[1], by = b[2] * e[0] - b[0] * e[2], bz = b[0] * e[1] - b[1] * e[0];
        double trip = fabs(a[0] * bx + a[1] * by + a[2] * bz);
        double den = 1.0 + (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) + (b[0] * e[0] + b[1] * e[1] + b[2] * e[2]) +
                     (e[0] * a[0] + e[1] * a[1] + e[2] * a[2]);
        w[t] = R * R * 2.0 * atan2(trip, den);
        double r[3], lr = 0;
        for (int d = 0; d < 3; ++d) {
            r[d] = c[d] - o[d];
            lr += r[d] * r[d];
        }
        lr = sqrt(lr);
        for (int d = 0; d < 3; ++d) nrm[d * n + t] = r[d] / lr;
    } else {
        double u[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        double v[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
        double x[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
        double l = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        w[t] = 0.5 * l;
        for (int d = 0; d < 3; ++d) nrm[d * n + t] = x[d] / l;
    }
}

}  // namespace
}  // namespace kifmm

using namespace kifmm;

extern "C" const char* kifmm_last_error(void) { return g_err; }

extern "C" const char* kifmm_version(void) { return "kifmm 0.1 sm_103a"; }

extern "C" int kifmm_quadrature_points(const double* tri, const double* sph, int64_t n_tri, double* xyz, double* w,
                                       double* nrm, void* stream) {
    clear_error();
    KF_ARG(n_tri >= 0, "n_tri < 0");
    if (n_tri == 0) return KIFMM_OK;
    KF_ARG(tri && sph && xyz && w && nrm, "NULL pointer");
    k_quadrature<<<div_up(n_tri, 256), 256, 0, (cudaStream_t)stream>>>(tri, sph, n_tri, xyz, w, nrm);
    KF_CHECK_LAUNCH();
    return KIFMM_OK;
}
