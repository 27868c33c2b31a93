// geometry.cuh -- device helpers for the geometry of the map x = xi + grad phi
// (Sec. II): the symmetric triad e = I + Hess phi, its determinant sqrt g and
// smallest eigenvalue lambda0, the compression limiter C(lambda0) of App. A,
// and the CIC weights of a tracer.  Shared by the step kernels and the
// adjoint kernels.
#pragma once

#include "recon_internal.cuh"

namespace recon {

struct Sym3 {
    double xx, yy, zz, xy, xz, yz;
};

// Hessian of f at node (i,j,k): 3-point second differences on the diagonal,
// 4-point centred cross differences off it.
__device__ inline Sym3 hessian(const Dims& d, const double* __restrict__ f, int i, int j, int k) {
    const double c = f[cell_index(d, i, j, k)];
    Sym3 H;
    H.xx = f[cell_index(d, i + 1, j, k)] - 2.0 * c + f[cell_index(d, i - 1, j, k)];
    H.yy = f[cell_index(d, i, j + 1, k)] - 2.0 * c + f[cell_index(d, i, j - 1, k)];
    H.zz = f[cell_index(d, i, j, k + 1)] - 2.0 * c + f[cell_index(d, i, j, k - 1)];
    H.xy = 0.25 * (f[cell_index(d, i + 1, j + 1, k)] - f[cell_index(d, i + 1, j - 1, k)] -
                   f[cell_index(d, i - 1, j + 1, k)] + f[cell_index(d, i - 1, j - 1, k)]);
    H.xz = 0.25 * (f[cell_index(d, i + 1, j, k + 1)] - f[cell_index(d, i + 1, j, k - 1)] -
                   f[cell_index(d, i - 1, j, k + 1)] + f[cell_index(d, i - 1, j, k - 1)]);
    H.yz = 0.25 * (f[cell_index(d, i, j + 1, k + 1)] - f[cell_index(d, i, j + 1, k - 1)] -
                   f[cell_index(d, i, j - 1, k + 1)] + f[cell_index(d, i, j - 1, k - 1)]);
    return H;
}

__device__ inline double det3(const Sym3& e) {
    return e.xx * (e.yy * e.zz - e.yz * e.yz) - e.xy * (e.xy * e.zz - e.yz * e.xz) +
           e.xz * (e.xy * e.yz - e.yy * e.xz);
}

// det(e - lam I) and its derivative in lam.
__device__ inline void charpoly(const Sym3& e, double lam, double& p, double& dp) {
    const double a = e.xx - lam, b = e.yy - lam, c = e.zz - lam;
    p = a * (b * c - e.yz * e.yz) - e.xy * (e.xy * c - e.yz * e.xz) + e.xz * (e.xy * e.yz - b * e.xz);
    dp = -((b * c - e.yz * e.yz) + (a * c - e.xz * e.xz) + (a * b - e.xy * e.xy));
}

// Smallest eigenvalue of a symmetric 3x3 matrix: the trigonometric closed form
// of the characteristic cubic (O. K. Smith, CACM 4, 168, 1961), then Newton
// steps on det(e - lam I) while they reduce |det|.
__device__ inline double min_eig_sym3(const Sym3& e) {
    const double p1 = e.xy * e.xy + e.xz * e.xz + e.yz * e.yz;
    const double q = (e.xx + e.yy + e.zz) * (1.0 / 3.0);
    const double b11 = e.xx - q, b22 = e.yy - q, b33 = e.zz - q;
    const double p2 = b11 * b11 + b22 * b22 + b33 * b33 + 2.0 * p1;
    if (!(p2 > 0.0)) return q;
    const double pp = sqrt(p2 * (1.0 / 6.0));
    const double ip = 1.0 / pp;
    Sym3 B;
    B.xx = b11 * ip, B.yy = b22 * ip, B.zz = b33 * ip;
    B.xy = e.xy * ip, B.xz = e.xz * ip, B.yz = e.yz * ip;
    double r = 0.5 * det3(B);
    r = fmin(1.0, fmax(-1.0, r));
    const double ang = acos(r) * (1.0 / 3.0);
    double lam = q + 2.0 * pp * cos(ang + 2.0943951023931957);  // + 2 pi / 3
    double p, dp;
    charpoly(e, lam, p, dp);
    for (int it = 0; it < 3; ++it) {
        if (p == 0.0 || dp == 0.0) break;
        const double cand = lam - p / dp;
        double pc, dpc;
        charpoly(e, cand, pc, dpc);
        if (!(fabs(pc) < fabs(p))) break;
        lam = cand, p = pc, dp = dpc;
    }
    return lam;
}

__device__ inline double climit(int reading, double xi_m, double lambda0) {
    const double lam = lambda0 > 1e-12 ? lambda0 : 1e-12;
    const double q = xi_m / lam;
    double v;
    if (reading == 1) v = q - (q - 1.0 > 0.0 ? 1.0 : 0.0);       // literal
    else if (reading == 2) v = q * (q - 1.0 > 0.0 ? 1.0 : 0.0);  // step
    else v = q - 1.0 > 0.0 ? q - 1.0 : 0.0;                      // soft
    return 4.0 * v * v;
}

// CIC weights along one axis for grid coordinate home + off: lower node and
// fraction toward the upper one.
__device__ inline void cic_offset(int home, double off, int& i0, double& f) {
    const double fl = floor(off);
    f = off - fl;
    i0 = home + (int)fl;
}

}  // namespace recon
