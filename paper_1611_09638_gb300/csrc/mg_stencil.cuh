// mg_stencil.cuh -- the per-node arithmetic of the multigrid levels that are
// not streamed (App. A's 7-point operator with face coefficients
// (a + a_nbr)/2 and spacing factors h_a^-2), shared by the one-kernel-per-
// phase path, the single-block coarse V-cycle and the cluster coarse V-cycle
// so that all three compute every node identically; and the layout of the
// coarsest level's inverse.
#pragma once

#include "recon_internal.cuh"

namespace recon {

// Seven-point operator pieces at a node: diagonal D and off-diagonal sum O,
// so that (L u)_c = O - D u_c.
template <typename T>
struct Stencil7 {
    T diag, off;
};

// From the node's coefficient ac and its neighbours' coefficients a* and
// values u* (x: i, y: j, z: k; p: +1, m: -1).
template <typename T>
__device__ inline Stencil7<T> stencil7v(T hx, T hy, T hz, T ac, T axp, T axm, T ayp, T aym, T azp,
                                        T azm, T uxp, T uxm, T uyp, T uym, T uzp, T uzm) {
    const T h = T(0.5);
    T apx = h * (ac + axp) * hx, amx = h * (ac + axm) * hx;
    T apy = h * (ac + ayp) * hy, amy = h * (ac + aym) * hy;
    T apz = h * (ac + azp) * hz, amz = h * (ac + azm) * hz;
    Stencil7<T> s;
    s.diag = (apx + amx) + (apy + amy) + (apz + amz);
    s.off = (apx * uxp + amx * uxm) + (apy * uyp + amy * uym) + (apz * uzp + amz * uzm);
    return s;
}

// At node c = (i, j, k) of a periodic level stored as one array.
template <typename T>
__device__ inline Stencil7<T> stencil7(const Dims& d, T hx, T hy, T hz, int i, int j, int k, int c,
                                       const T* __restrict__ u, const T* __restrict__ a) {
    const int xp = cell_index(d, i + 1, j, k), xm = cell_index(d, i - 1, j, k);
    const int yp = cell_index(d, i, j + 1, k), ym = cell_index(d, i, j - 1, k);
    const int zp = cell_index(d, i, j, k + 1), zm = cell_index(d, i, j, k - 1);
    return stencil7v<T>(hx, hy, hz, a[c], a[xp], a[xm], a[yp], a[ym], a[zp], a[zm], u[xp], u[xm], u[yp],
                        u[ym], u[zp], u[zm]);
}

// The same pieces from face sums G (face coefficient x 2) of the six faces.
template <typename T>
__device__ inline Stencil7<T> stencil7g(T hx, T hy, T hz, T gpx, T gmx, T gpy, T gmy, T gpz, T gmz,
                                        T uxp, T uxm, T uyp, T uym, T uzp, T uzm) {
    const T h = T(0.5);
    T apx = h * gpx * hx, amx = h * gmx * hx;
    T apy = h * gpy * hy, amy = h * gmy * hy;
    T apz = h * gpz * hz, amz = h * gmz * hz;
    Stencil7<T> s;
    s.diag = (apx + amx) + (apy + amy) + (apz + amz);
    s.off = (apx * uxp + amx * uxm) + (apy * uyp + amy * uym) + (apz * uzp + amz * uzm);
    return s;
}

// At node c = (i, j, k) of a level: from its nodal coefficient a, or (face)
// from its face sums g (x faces, then y, then z, each d.cells long).
template <typename T>
__device__ inline Stencil7<T> stencil7_any(const Dims& d, T hx, T hy, T hz, int i, int j, int k, int c,
                                           const T* __restrict__ u, const T* __restrict__ a, int face) {
    if (!face) return stencil7<T>(d, hx, hy, hz, i, j, k, c, u, a);
    const int xp = cell_index(d, i + 1, j, k), xm = cell_index(d, i - 1, j, k);
    const int yp = cell_index(d, i, j + 1, k), ym = cell_index(d, i, j - 1, k);
    const int zp = cell_index(d, i, j, k + 1), zm = cell_index(d, i, j, k - 1);
    const T* gx = a;
    const T* gy = a + d.cells;
    const T* gz = a + 2 * (size_t)d.cells;
    return stencil7g<T>(hx, hy, hz, gx[c], gx[xm], gy[c], gy[ym], gz[c], gz[zm], u[xp], u[xm], u[yp], u[ym],
                        u[zp], u[zm]);
}

// The coarsest (4^3) level is solved with the inverse of the bordered system
// [L 1; 1^T 0] (kNb x kNb), stored as the augmented matrix [I | M^-1]
// (kNb rows of kW doubles) that the Gauss-Jordan kernel leaves behind.
constexpr int kNc = 64, kNb = 65, kW = 130;

}  // namespace recon
