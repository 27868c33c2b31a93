// mg_kernels.cu -- variable-coefficient multigrid kernels for the linearised
// elliptic equation of App. A (Eq. elliptic with x ~ xi):
//     L u = sum_a h_a^-2 [A+ (u+ - u) - A- (u - u-)],  A+- = (a + a+-) / 2,
// red-black Gauss-Seidel smoothing (red = (i+j+k) even first), residual,
// full-weighting restriction, trilinear prolongation, and a dense solve of the
// 4^3 coarsest level with the mean constraint.  Templated on float (mixed mode)
// and double.
#include "mg_stencil.cuh"
#include "recon_internal.cuh"
#include "reduce.cuh"

namespace recon {

namespace {

constexpr int kThreads = 256;

inline int nblocks(long long work) { return (int)((work + kThreads - 1) / kThreads); }

// One colour of a red-black Gauss-Seidel sweep; thread t owns the t-th node
// of that colour (nodes of a colour alternate along the fastest axis).
template <typename T>
__global__ void k_rbgs_colour(Dims d, T hx, T hy, T hz, int colour, T* __restrict__ u,
                              const T* __restrict__ f, const T* __restrict__ a, int face) {
    const int half = d.cells >> 1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= half) return;
    const int hs2 = d.s2 - 1;
    const int kk = t & ((1 << hs2) - 1);
    const int j = (t >> hs2) & (d.n1 - 1);
    const int i = t >> (d.s1 + hs2);
    const int k = 2 * kk + ((i + j + colour) & 1);
    const int c = cell_index(d, i, j, k);
    Stencil7<T> s = stencil7_any<T>(d, hx, hy, hz, i, j, k, c, u, a, face);
    u[c] = (s.off - f[c]) / s.diag;
}

// One colour of a red-black sweep of the finest FP64 level (unit spacing)
// from the stored face coefficients A = (a_c + a_n) / 2 (F: +x, +y, +z face
// of each node) and the inverse of the node's diagonal D = sum of its six A:
// u_c = (sum_n A_n u_n - f_c) / D_c in 8 FP64 instructions per node, since
// FP64 issue, not memory, bounds this sweep on GB300.
__global__ void k_rbgs_colour64_unit(Dims d, int colour, double* __restrict__ u,
                                     const double* __restrict__ f, const double* __restrict__ F,
                                     const double* __restrict__ inv_d) {
    const int half = d.cells >> 1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= half) return;
    const int hs2 = d.s2 - 1;
    const int kk = t & ((1 << hs2) - 1);
    const int j = (t >> hs2) & (d.n1 - 1);
    const int i = t >> (d.s1 + hs2);
    const int k = 2 * kk + ((i + j + colour) & 1);
    const int c = cell_index(d, i, j, k);
    const int n0 = cell_index(d, i + 1, j, k), n1 = cell_index(d, i - 1, j, k);
    const int n2 = cell_index(d, i, j + 1, k), n3 = cell_index(d, i, j - 1, k);
    const int n4 = cell_index(d, i, j, k + 1), n5 = cell_index(d, i, j, k - 1);
    const size_t n = (size_t)d.cells;
    double o = F[c] * u[n0];
    o = fma(F[n1], u[n1], o);
    o = fma(F[n + c], u[n2], o);
    o = fma(F[n + n3], u[n3], o);
    o = fma(F[2 * n + c], u[n4], o);
    o = fma(F[2 * n + n5], u[n5], o);
    u[c] = (o - f[c]) * inv_d[c];
}

// FP64 residual r = f - L u of the finest level (unit spacing) from the
// stored face coefficients A (F) and node diagonals D: since
// L u = sum_n A_n u_n - D u_c, r = f + D u_c - sum_n A_n u_n is a chain of
// seven FMAs.  The FP64 issue rate, not memory, bounds this kernel on GB300,
// so coefficients are read rather than recomputed.  The rounding error of the
// undifferenced form is ~8 eps D |u|, i.e. ~1e-12 relative to |f| even for
// the smoothest mode of a 512^3 grid, far below the stopping tolerance.
// Optionally also writes r in FP32 (the next V-cycle's right-hand side);
// always the per-block partial sums of r^2.  With the FP32 copy (mixed mode)
// r^2 is summed from it on the FP32 pipe, one FP64 instruction fewer per
// node.  The norm only decides the multigrid stopping test: each thread's
// FP32 sum covers cells / (kRedBlocks * kRedThreads) nodes (54 at 256^3, 431
// at 512^3), so its relative error stays below ~3e-5, and the block sums
// are FP64.
__global__ void k_residual64_to32(Dims d, const double* __restrict__ u,
                                  const double* __restrict__ f, const double* __restrict__ F,
                                  const double* __restrict__ D, float* __restrict__ r32,
                                  double* __restrict__ partials) {
    double acc = 0.0;
    float acc32 = 0.f;
    const size_t n = (size_t)d.cells;
    const double* __restrict__ Fx = F;
    const double* __restrict__ Fy = F + n;
    const double* __restrict__ Fz = F + 2 * n;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.cells; c += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_coords(d, c, i, j, k);
        const int n0 = cell_index(d, i + 1, j, k), n1 = cell_index(d, i - 1, j, k);
        const int n2 = cell_index(d, i, j + 1, k), n3 = cell_index(d, i, j - 1, k);
        const int n4 = cell_index(d, i, j, k + 1), n5 = cell_index(d, i, j, k - 1);
        double r = fma(D[c], u[c], f[c]);
        r = fma(-Fx[c], u[n0], r);
        r = fma(-Fx[n1], u[n1], r);
        r = fma(-Fy[c], u[n2], r);
        r = fma(-Fy[n3], u[n3], r);
        r = fma(-Fz[c], u[n4], r);
        r = fma(-Fz[n5], u[n5], r);
        if (r32) {
            const float rf = (float)r;
            r32[c] = rf;
            acc32 = fmaf(rf, rf, acc32);
        } else {
            acc = fma(r, r, acc);
        }
    }
    acc += (double)acc32;
    acc = block_reduce<OpSum>(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// Face coefficients A = (a_c + a_{c + e_a}) / 2 of a unit-spacing level, one
// array per axis, the node diagonal D = sum of the node's six A, and
// optionally 1 / D.
__global__ void k_faces64(Dims d, const double* __restrict__ a, double* __restrict__ F,
                          double* __restrict__ D, double* __restrict__ inv_d) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.cells) return;
    int i, j, k;
    cell_coords(d, c, i, j, k);
    const size_t n = (size_t)d.cells;
    const double ac = a[c];
    const double xp = 0.5 * (ac + a[cell_index(d, i + 1, j, k)]);
    const double xm = 0.5 * (ac + a[cell_index(d, i - 1, j, k)]);
    const double yp = 0.5 * (ac + a[cell_index(d, i, j + 1, k)]);
    const double ym = 0.5 * (ac + a[cell_index(d, i, j - 1, k)]);
    const double zp = 0.5 * (ac + a[cell_index(d, i, j, k + 1)]);
    const double zm = 0.5 * (ac + a[cell_index(d, i, j, k - 1)]);
    F[c] = xp, F[n + c] = yp, F[2 * n + c] = zp;
    const double dg = ((xp + xm) + (yp + ym)) + (zp + zm);
    D[c] = dg;
    if (inv_d) inv_d[c] = 1.0 / dg;
}

// Full weighting: weights (1/4, 1/2, 1/4) along every coarsened axis.
template <typename T>
__global__ void k_restrict(Dims df, Dims dc, int cx, int cy, int cz, const T* __restrict__ in,
                           T* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= dc.cells) return;
    int I, J, K;
    cell_coords(dc, c, I, J, K);
    const int fi = cx ? 2 * I : I, fj = cy ? 2 * J : J, fk = cz ? 2 * K : K;
    T acc = T(0);
    for (int oi = -cx; oi <= cx; ++oi) {
        const T wi = cx ? (oi == 0 ? T(0.5) : T(0.25)) : T(1);
        for (int oj = -cy; oj <= cy; ++oj) {
            const T wj = cy ? (oj == 0 ? T(0.5) : T(0.25)) : T(1);
            for (int ok = -cz; ok <= cz; ++ok) {
                const T wk = cz ? (ok == 0 ? T(0.5) : T(0.25)) : T(1);
                acc += wi * wj * wk * in[cell_index(df, fi + oi, fj + oj, fk + ok)];
            }
        }
    }
    out[c] = acc;
}

// Residual r = f - L u evaluated at the fine nodes of each coarse node's
// full-weighting stencil and restricted at once (the fine residual is never
// stored): per node the 7-point residual f - L u followed by the full weighting.
template <typename T>
__global__ void k_resid_restrict(Dims df, Dims dc, int cx, int cy, int cz, T hx, T hy, T hz,
                                 const T* __restrict__ u, const T* __restrict__ f,
                                 const T* __restrict__ a, int face, T* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= dc.cells) return;
    int I, J, K;
    cell_coords(dc, c, I, J, K);
    const int fi = cx ? 2 * I : I, fj = cy ? 2 * J : J, fk = cz ? 2 * K : K;
    T acc = T(0);
    for (int oi = -cx; oi <= cx; ++oi) {
        const T wi = cx ? (oi == 0 ? T(0.5) : T(0.25)) : T(1);
        for (int oj = -cy; oj <= cy; ++oj) {
            const T wj = cy ? (oj == 0 ? T(0.5) : T(0.25)) : T(1);
            for (int ok = -cz; ok <= cz; ++ok) {
                const T wk = cz ? (ok == 0 ? T(0.5) : T(0.25)) : T(1);
                const int i = (fi + oi) & (df.n0 - 1), j = (fj + oj) & (df.n1 - 1),
                          k = (fk + ok) & (df.n2 - 1);
                const int n = cell_index(df, i, j, k);
                Stencil7<T> s = stencil7_any<T>(df, hx, hy, hz, i, j, k, n, u, a, face);
                const T r = f[n] - (s.off - s.diag * u[n]);
                acc += wi * wj * wk * r;
            }
        }
    }
    out[c] = acc;
}

// Face sums of the coarse level (every axis halved) from the fine level's
// nodal coefficient a (face sum a_c + a_n) or its face sums (fine_face).  A
// coarse face between coarse nodes I and I + 1 along an axis spans the two
// fine faces 2I|2I+1 and 2I+1|2I+2 of each fine line along that axis: in
// series they conduct as the harmonic mean of the two, and the 3 x 3 lines
// around the coarse line are weighted (1/4, 1/2, 1/4) in both transverse
// axes.  For a constant coefficient this is the re-discretised face; where
// the coefficient jumps it keeps the flux a fine-grid path can carry, which
// full weighting of a nodal coefficient does not.
__global__ void k_faces_line(Dims df, Dims dc, const float* __restrict__ in, int fine_face,
                             float* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= dc.cells) return;
    int I, J, K;
    cell_coords(dc, c, I, J, K);
    const int f0[3] = {2 * I, 2 * J, 2 * K};
    const float w[3] = {0.25f, 0.5f, 0.25f};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;  // transverse axes
        float acc = 0.f;
        for (int o1 = -1; o1 <= 1; ++o1)
            for (int o2 = -1; o2 <= 1; ++o2) {
                int p[3];
                p[ax] = f0[ax];
                p[t1] = f0[t1] + o1;
                p[t2] = f0[t2] + o2;
                const int e0 = cell_index(df, p[0], p[1], p[2]);
                p[ax] += 1;
                const int e1 = cell_index(df, p[0], p[1], p[2]);
                p[ax] += 1;
                const int e2 = cell_index(df, p[0], p[1], p[2]);
                float g1, g2;
                if (fine_face) {
                    const float* g = in + (size_t)ax * df.cells;
                    g1 = g[e0], g2 = g[e1];
                } else {
                    g1 = in[e0] + in[e1], g2 = in[e1] + in[e2];
                }
                acc += w[o1 + 1] * w[o2 + 1] * __fdividef(2.f * g1 * g2, g1 + g2);
            }
        out[(size_t)ax * dc.cells + c] = acc;
    }
}

// Trilinear prolongation of the coarse correction, added to the fine field.
template <typename T>
__global__ void k_prolong_add(Dims df, Dims dc, int cx, int cy, int cz, const T* __restrict__ uc,
                              T* __restrict__ u) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= df.cells) return;
    int i, j, k;
    cell_coords(df, c, i, j, k);
    int ii[2], jj[2], kk[2];
    T wi[2], wj[2], wk[2];
    int ni, nj, nk;
    if (!cx) { ii[0] = i; wi[0] = T(1); ni = 1; }
    else if (!(i & 1)) { ii[0] = i >> 1; wi[0] = T(1); ni = 1; }
    else { ii[0] = i >> 1; ii[1] = (i >> 1) + 1; wi[0] = wi[1] = T(0.5); ni = 2; }
    if (!cy) { jj[0] = j; wj[0] = T(1); nj = 1; }
    else if (!(j & 1)) { jj[0] = j >> 1; wj[0] = T(1); nj = 1; }
    else { jj[0] = j >> 1; jj[1] = (j >> 1) + 1; wj[0] = wj[1] = T(0.5); nj = 2; }
    if (!cz) { kk[0] = k; wk[0] = T(1); nk = 1; }
    else if (!(k & 1)) { kk[0] = k >> 1; wk[0] = T(1); nk = 1; }
    else { kk[0] = k >> 1; kk[1] = (k >> 1) + 1; wk[0] = wk[1] = T(0.5); nk = 2; }
    T acc = T(0);
    for (int p = 0; p < ni; ++p)
        for (int q = 0; q < nj; ++q)
            for (int r = 0; r < nk; ++r)
                acc += wi[p] * wj[q] * wk[r] * uc[cell_index(dc, ii[p], jj[q], kk[r])];
    u[c] += acc;
}

// Coarsest level (64 nodes): Gauss-Jordan inversion with partial pivoting of
// the bordered system [L 1; 1^T 0] (65 x 65), in FP64, by one block working
// on the augmented matrix [M | I] (65 x 130) in shared memory; the result is
// written to global memory in the same layout.
constexpr int kInvThreads = 1024;
constexpr size_t kInvSmem = sizeof(double) * kNb * kW;

template <typename T>
__global__ void __launch_bounds__(kInvThreads) k_coarse_invert(Dims d, double hx, double hy,
                                                              double hz, const T* __restrict__ a,
                                                              int face, double* __restrict__ out) {
    extern __shared__ double aug[];
    __shared__ double fac[kNb];
    __shared__ int piv_row;
    const int t = threadIdx.x;
    for (int e = t; e < kNb * kW; e += blockDim.x) aug[e] = 0.0;
    __syncthreads();
    if (t < kNc) {
        const int c = t;
        int i, j, k;
        cell_coords(d, c, i, j, k);
        const int nb[6] = {cell_index(d, i + 1, j, k), cell_index(d, i - 1, j, k),
                           cell_index(d, i, j + 1, k), cell_index(d, i, j - 1, k),
                           cell_index(d, i, j, k + 1), cell_index(d, i, j, k - 1)};
        const double hh[3] = {hx, hy, hz};
        double diag = 0.0;
        for (int q = 0; q < 6; ++q) {
            // face sum of face q: the +1 face of node c, or the +1 face of
            // its -1 neighbour
            const double g = face ? (double)a[(size_t)(q >> 1) * d.cells + ((q & 1) ? nb[q] : c)]
                                  : (double)a[c] + (double)a[nb[q]];
            double w = 0.5 * g * hh[q >> 1];
            diag += w;
            aug[c * kW + nb[q]] += w;  // row c of L; distinct neighbours on 4^3
        }
        aug[c * kW + c] -= diag;
        aug[c * kW + kNc] = 1.0;
        aug[kNc * kW + c] = 1.0;
    }
    __syncthreads();
    for (int r = t; r < kNb; r += blockDim.x) aug[r * kW + kNb + r] = 1.0;
    __syncthreads();
    for (int p = 0; p < kNb; ++p) {
        if (t < 32) {
            // largest |entry| of column p at or below row p; the first such
            // row on ties (as a serial scan with a strict comparison)
            int best = -1;
            double bv = -1.0;
            for (int r = p + t; r < kNb; r += 32) {
                const double v = fabs(aug[r * kW + p]);
                if (v > bv) bv = v, best = r;
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_down_sync(0xffffffffu, bv, o);
                const int ob = __shfl_down_sync(0xffffffffu, best, o);
                if (ob >= 0 && (ov > bv || (ov == bv && (best < 0 || ob < best)))) bv = ov, best = ob;
            }
            if (t == 0) piv_row = best;
        }
        __syncthreads();
        const int pr = piv_row;
        if (pr != p)
            for (int cc = t; cc < kW; cc += blockDim.x) {
                const double x = aug[p * kW + cc];
                aug[p * kW + cc] = aug[pr * kW + cc];
                aug[pr * kW + cc] = x;
            }
        __syncthreads();
        const double pv = aug[p * kW + p];
        __syncthreads();
        for (int cc = t; cc < kW; cc += blockDim.x) aug[p * kW + cc] /= pv;
        __syncthreads();
        for (int r = t; r < kNb; r += blockDim.x) fac[r] = aug[r * kW + p];
        __syncthreads();
        for (int e = t; e < kNb * kW; e += blockDim.x) {
            const int r = e / kW, cc = e - r * kW;
            if (r != p) aug[e] -= fac[r] * aug[p * kW + cc];
        }
        __syncthreads();
    }
    for (int e = t; e < kNb * kW; e += blockDim.x) out[e] = aug[e];
}

template <typename T>
__global__ void k_coarse_solve(const double* __restrict__ aug, const T* __restrict__ f,
                               T* __restrict__ u) {
    const int r = threadIdx.x;
    if (r >= kNc) return;
    double acc = 0.0;
    for (int c = 0; c < kNc; ++c) acc += aug[r * kW + kNb + c] * (double)f[c];
    u[r] = (T)acc;
}

__global__ void k_to_f32(int cells, const double* __restrict__ x, float* __restrict__ y) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < cells) y[c] = (float)x[c];
}

__global__ void k_correct(int cells, double* __restrict__ u, const float* __restrict__ e) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < cells) u[c] += (double)e[c];
}

}  // namespace

template <typename T>
void launch_rbgs_sweep(const Level& L, T* u, const T* f, const T* a, cudaStream_t st) {
    const int half = L.d.cells >> 1;
    launch_counter() += 2;
    for (int colour = 0; colour < 2; ++colour)
        k_rbgs_colour<T><<<nblocks(half), kThreads, 0, st>>>(L.d, (T)L.h2i[0], (T)L.h2i[1],
                                                             (T)L.h2i[2], colour, u, f, a, L.face);
}

template <typename T>
void launch_restrict(const Level& fine, const Level& coarse, const T* in, T* out, cudaStream_t st) {
    launch_counter()++;
    k_restrict<T><<<nblocks(coarse.d.cells), kThreads, 0, st>>>(
        fine.d, coarse.d, fine.coarsen[0], fine.coarsen[1], fine.coarsen[2], in, out);
}

template <typename T>
void launch_resid_restrict(const Level& fine, const Level& coarse, const T* u, const T* f,
                           const T* a, T* out, cudaStream_t st) {
    launch_counter()++;
    k_resid_restrict<T><<<nblocks(coarse.d.cells), kThreads, 0, st>>>(
        fine.d, coarse.d, fine.coarsen[0], fine.coarsen[1], fine.coarsen[2], (T)fine.h2i[0],
        (T)fine.h2i[1], (T)fine.h2i[2], u, f, a, fine.face, out);
}

void launch_faces_line(const Level& fine, const Level& coarse, const float* in, float* out,
                       cudaStream_t st) {
    launch_counter()++;
    k_faces_line<<<nblocks(coarse.d.cells), kThreads, 0, st>>>(fine.d, coarse.d, in, fine.face, out);
}

template <typename T>
void launch_prolong_add(const Level& fine, const Level& coarse, const T* uc, T* u, cudaStream_t st) {
    launch_counter()++;
    k_prolong_add<T><<<nblocks(fine.d.cells), kThreads, 0, st>>>(
        fine.d, coarse.d, fine.coarsen[0], fine.coarsen[1], fine.coarsen[2], uc, u);
}

template <typename T>
void launch_coarse_invert(const Level& L, const T* a, double* minv, cudaStream_t st) {
    allow_smem((const void*)k_coarse_invert<T>, (int)kInvSmem);
    launch_counter()++;
    k_coarse_invert<T><<<1, kInvThreads, kInvSmem, st>>>(L.d, L.h2i[0], L.h2i[1], L.h2i[2], a,
                                                         L.face, minv);
}

template <typename T>
void launch_coarse_solve(const double* minv, const T* f, T* u, cudaStream_t st) {
    launch_counter()++;
    k_coarse_solve<T><<<1, kNc, 0, st>>>(minv, f, u);
}

void launch_to_f32(int cells, const double* x, float* y, cudaStream_t st) {
    launch_counter()++;
    k_to_f32<<<nblocks(cells), kThreads, 0, st>>>(cells, x, y);
}

void launch_residual64_to32(const Level& L, const double* u, const double* f, const double* F,
                            const double* D, float* r32, double* partials, cudaStream_t st) {
    launch_counter()++;
    k_residual64_to32<<<kRedBlocks, kRedThreads, 0, st>>>(L.d, u, f, F, D, r32, partials);
}

void launch_residual_norm64(const Level& L, const double* u, const double* f, const double* F,
                            const double* D, double* partials, cudaStream_t st) {
    launch_counter()++;
    k_residual64_to32<<<kRedBlocks, kRedThreads, 0, st>>>(L.d, u, f, F, D, nullptr, partials);
}

void launch_rbgs_sweep64_unit(const Level& L, double* u, const double* f, const double* F,
                              const double* inv_d, cudaStream_t st) {
    const int half = L.d.cells >> 1;
    launch_counter() += 2;
    for (int colour = 0; colour < 2; ++colour)
        k_rbgs_colour64_unit<<<nblocks(half), kThreads, 0, st>>>(L.d, colour, u, f, F, inv_d);
}

void launch_faces64(const Level& L, const double* a, double* F, double* D, double* inv_d,
                    cudaStream_t st) {
    launch_counter()++;
    k_faces64<<<nblocks(L.d.cells), kThreads, 0, st>>>(L.d, a, F, D, inv_d);
}

void launch_correct(int cells, double* u, const float* e, cudaStream_t st) {
    launch_counter()++;
    k_correct<<<nblocks(cells), kThreads, 0, st>>>(cells, u, e);
}

#define RECON_INSTANTIATE(T)                                                                    \
    template void launch_rbgs_sweep<T>(const Level&, T*, const T*, const T*, cudaStream_t);   \
    template void launch_restrict<T>(const Level&, const Level&, const T*, T*, cudaStream_t);  \
    template void launch_resid_restrict<T>(const Level&, const Level&, const T*, const T*,     \
                                           const T*, T*, cudaStream_t);                       \
    template void launch_prolong_add<T>(const Level&, const Level&, const T*, T*,              \
                                        cudaStream_t);                                        \
    template void launch_coarse_invert<T>(const Level&, const T*, double*, cudaStream_t);      \
    template void launch_coarse_solve<T>(const double*, const T*, T*, cudaStream_t);
RECON_INSTANTIATE(float)
RECON_INSTANTIATE(double)
#undef RECON_INSTANTIATE

}  // namespace recon

// ---------------------------------------------------------------------------
// The coarse end of the V-cycle in one block: every level from l0 (at most
// kCoarseMaxCells nodes) down to the 4^3 level is smoothed, restricted, solved
// and prolonged in shared memory, with the same per-node arithmetic as the
// kernels above, so a V-cycle launches one kernel for all of these levels.

namespace recon {

namespace {

template <typename T>
__device__ inline void sm_sweep_colour(const Dims& d, T hx, T hy, T hz, int colour, T* u,
                                       const T* f, const T* a) {
    const int half = d.cells >> 1, hs2 = d.s2 - 1;
    for (int t = threadIdx.x; t < half; t += blockDim.x) {
        const int kk = t & ((1 << hs2) - 1);
        const int j = (t >> hs2) & (d.n1 - 1);
        const int i = t >> (d.s1 + hs2);
        const int k = 2 * kk + ((i + j + colour) & 1);
        const int c = cell_index(d, i, j, k);
        Stencil7<T> s = stencil7<T>(d, hx, hy, hz, i, j, k, c, u, a);
        u[c] = (s.off - f[c]) / s.diag;
    }
}

template <typename T>
__device__ inline void sm_sweeps(const Dims& d, T hx, T hy, T hz, int nu, T* u, const T* f,
                                 const T* a) {
    for (int s = 0; s < nu; ++s)
        for (int colour = 0; colour < 2; ++colour) {
            sm_sweep_colour<T>(d, hx, hy, hz, colour, u, f, a);
            __syncthreads();
        }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_vcycle(CoarseSet cs, const T* __restrict__ f_top,
                                                        T* __restrict__ u_top,
                                                        const double* __restrict__ aug,
                                                        int zero_u) {
    extern __shared__ unsigned char smem_raw[];
    T* base = reinterpret_cast<T*>(smem_raw);
    T *u[kCoarseMaxLevels], *f[kCoarseMaxLevels], *a[kCoarseMaxLevels], *r[kCoarseMaxLevels];
    {
        T* q = base;
        for (int l = 0; l < cs.nlev; ++l) {
            const int n = cs.lv[l].d.cells;
            u[l] = q, f[l] = q + n, a[l] = q + 2 * n, r[l] = q + 3 * n;
            q += 4 * n;
        }
    }
    for (int l = 0; l < cs.nlev; ++l) {
        const T* ag = reinterpret_cast<const T*>(cs.a[l]);
        for (int c = threadIdx.x; c < cs.lv[l].d.cells; c += blockDim.x) a[l][c] = ag[c];
    }
    for (int c = threadIdx.x; c < cs.lv[0].d.cells; c += blockDim.x) {
        f[0][c] = f_top[c];
        u[0][c] = zero_u ? T(0) : u_top[c];
    }
    // the 4^3 inverse (its kNc x kNc block of the augmented matrix) in shared
    // memory, after the levels (8-byte aligned: 4 arrays of whole levels)
    double* minv = reinterpret_cast<double*>(u[cs.nlev - 1] + 4 * cs.lv[cs.nlev - 1].d.cells);
    for (int e = threadIdx.x; e < kNc * kNc; e += blockDim.x) minv[e] = aug[(e / kNc) * kW + kNb + (e % kNc)];
    __syncthreads();
    const int last = cs.nlev - 1;
    // down
    for (int l = 0; l < last; ++l) {
        const Level& L = cs.lv[l];
        const T hx = (T)L.h2i[0], hy = (T)L.h2i[1], hz = (T)L.h2i[2];
        sm_sweeps<T>(L.d, hx, hy, hz, cs.nu1, u[l], f[l], a[l]);
        for (int c = threadIdx.x; c < L.d.cells; c += blockDim.x) {
            int i, j, k;
            cell_coords(L.d, c, i, j, k);
            Stencil7<T> s = stencil7<T>(L.d, hx, hy, hz, i, j, k, c, u[l], a[l]);
            r[l][c] = f[l][c] - (s.off - s.diag * u[l][c]);
        }
        __syncthreads();
        const Dims& dc = cs.lv[l + 1].d;
        const int cx = L.coarsen[0], cy = L.coarsen[1], cz = L.coarsen[2];
        for (int c = threadIdx.x; c < dc.cells; c += blockDim.x) {
            int I, J, K;
            cell_coords(dc, c, I, J, K);
            const int fi = cx ? 2 * I : I, fj = cy ? 2 * J : J, fk = cz ? 2 * K : K;
            T acc = T(0);
            for (int oi = -cx; oi <= cx; ++oi) {
                const T wi = cx ? (oi == 0 ? T(0.5) : T(0.25)) : T(1);
                for (int oj = -cy; oj <= cy; ++oj) {
                    const T wj = cy ? (oj == 0 ? T(0.5) : T(0.25)) : T(1);
                    for (int ok = -cz; ok <= cz; ++ok) {
                        const T wk = cz ? (ok == 0 ? T(0.5) : T(0.25)) : T(1);
                        acc += wi * wj * wk * r[l][cell_index(L.d, fi + oi, fj + oj, fk + ok)];
                    }
                }
            }
            f[l + 1][c] = acc;
            u[l + 1][c] = T(0);
        }
        __syncthreads();
    }
    // coarsest: u = M^-1 [f; 0]
    if (threadIdx.x < kNc) {
        double acc = 0.0;
        for (int c = 0; c < kNc; ++c) acc += minv[threadIdx.x * kNc + c] * (double)f[last][c];
        u[last][threadIdx.x] = (T)acc;
    }
    __syncthreads();
    // up
    for (int l = last - 1; l >= 0; --l) {
        const Level& L = cs.lv[l];
        const Dims& dc = cs.lv[l + 1].d;
        const int cx = L.coarsen[0], cy = L.coarsen[1], cz = L.coarsen[2];
        for (int c = threadIdx.x; c < L.d.cells; c += blockDim.x) {
            int i, j, k;
            cell_coords(L.d, c, i, j, k);
            int ii[2], jj[2], kk[2];
            T wi[2], wj[2], wk[2];
            int ni, nj, nk;
            if (!cx) { ii[0] = i; wi[0] = T(1); ni = 1; }
            else if (!(i & 1)) { ii[0] = i >> 1; wi[0] = T(1); ni = 1; }
            else { ii[0] = i >> 1; ii[1] = (i >> 1) + 1; wi[0] = wi[1] = T(0.5); ni = 2; }
            if (!cy) { jj[0] = j; wj[0] = T(1); nj = 1; }
            else if (!(j & 1)) { jj[0] = j >> 1; wj[0] = T(1); nj = 1; }
            else { jj[0] = j >> 1; jj[1] = (j >> 1) + 1; wj[0] = wj[1] = T(0.5); nj = 2; }
            if (!cz) { kk[0] = k; wk[0] = T(1); nk = 1; }
            else if (!(k & 1)) { kk[0] = k >> 1; wk[0] = T(1); nk = 1; }
            else { kk[0] = k >> 1; kk[1] = (k >> 1) + 1; wk[0] = wk[1] = T(0.5); nk = 2; }
            T acc = T(0);
            for (int p = 0; p < ni; ++p)
                for (int q = 0; q < nj; ++q)
                    for (int rr = 0; rr < nk; ++rr)
                        acc += wi[p] * wj[q] * wk[rr] * u[l + 1][cell_index(dc, ii[p], jj[q], kk[rr])];
            u[l][c] += acc;
        }
        __syncthreads();
        sm_sweeps<T>(L.d, (T)L.h2i[0], (T)L.h2i[1], (T)L.h2i[2], cs.nu2, u[l], f[l], a[l]);
    }
    for (int c = threadIdx.x; c < cs.lv[0].d.cells; c += blockDim.x) u_top[c] = u[0][c];
}

}  // namespace

template <typename T>
bool launch_coarse_vcycle(const CoarseSet& cs, const T* f_top, T* u_top, const double* minv,
                          bool zero_u, cudaStream_t st) {
    size_t cells = 0;
    for (int l = 0; l < cs.nlev; ++l) cells += cs.lv[l].d.cells;
    const size_t sm = 4 * cells * sizeof(T) + kNc * kNc * sizeof(double);
    if (cs.nlev < 1 || cs.nlev > kCoarseMaxLevels || sm > kCoarseMaxSmem) return false;
    allow_smem((const void*)k_coarse_vcycle<T>, (int)kCoarseMaxSmem);
    launch_counter()++;
    k_coarse_vcycle<T><<<1, 1024, sm, st>>>(cs, f_top, u_top, minv, zero_u ? 1 : 0);
    return true;
}

template bool launch_coarse_vcycle<float>(const CoarseSet&, const float*, float*, const double*,
                                          bool, cudaStream_t);
template bool launch_coarse_vcycle<double>(const CoarseSet&, const double*, double*,
                                           const double*, bool, cudaStream_t);

}  // namespace recon
