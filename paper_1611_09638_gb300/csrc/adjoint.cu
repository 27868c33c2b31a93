// adjoint.cu -- the vector-Jacobian product of the map rho -> delta_r of a
// solve (Sec. II, App. A, tracer re-deposit form) with the step lengths held
// at the values the forward solve chose, and the per-step checkpoints the
// forward solve keeps for it.
//
// The reverse sweep visits the steps k = K-1 .. 0 and, with the step's state
// (phi_k, the tracer offsets and phidot_k, kept by the forward solve),
// recomputes m_k, the triad e_k and the node velocities V_k = e_k^-1 grad
// dphi_k, then pulls the adjoints back through: the phi update, the tracer
// advance xi -= alpha V(xi) (the transpose of the CIC interpolation is a CIC
// scatter, done with FP64 atomics), V = e^-1 G, dphi = S phidot - mean, the
// linear solve (an adjoint solve with the same symmetric operator, run by the
// host with the multigrid of the forward solve), the coefficient
// a = max(m, a_min), s = S t - mean, the source t = Sigma + C(lambda0) + E
// (d lambda0 = v^T de v, v the eigenvector of lambda0), the Hessian e = I +
// Hess phi, and the CIC deposit of the tracers' masses.  Every other step is
// a gather, so only the scatter's summation order varies between runs.
#include "geometry.cuh"
#include "recon_internal.cuh"
#include "reduce.cuh"

namespace recon {

namespace {

constexpr int kThreads = 256;
inline int nblocks(long long work) { return (int)((work + kThreads - 1) / kThreads); }

// Unit eigenvector of a symmetric e for its (simple) eigenvalue lam: the
// largest cross product of two rows of e - lam I.
__device__ inline void eigvec_sym3(const Sym3& e, double lam, double v[3]) {
    const double r0[3] = {e.xx - lam, e.xy, e.xz};
    const double r1[3] = {e.xy, e.yy - lam, e.yz};
    const double r2[3] = {e.xz, e.yz, e.zz - lam};
    double c[3][3];
    const double* A[3] = {r0, r0, r1};
    const double* B[3] = {r1, r2, r2};
    int best = 0;
    double bn = -1.0;
    for (int q = 0; q < 3; ++q) {
        c[q][0] = A[q][1] * B[q][2] - A[q][2] * B[q][1];
        c[q][1] = A[q][2] * B[q][0] - A[q][0] * B[q][2];
        c[q][2] = A[q][0] * B[q][1] - A[q][1] * B[q][0];
        const double nn = c[q][0] * c[q][0] + c[q][1] * c[q][1] + c[q][2] * c[q][2];
        if (nn > bn) bn = nn, best = q;
    }
    const double inv = bn > 0.0 ? 1.0 / sqrt(bn) : 0.0;
    v[0] = c[best][0] * inv, v[1] = c[best][1] * inv, v[2] = c[best][2] * inv;
}

// dC / d lambda0 of the compression limiter (zero where lambda0 is clamped).
__device__ inline double climit_deriv(int reading, double xi_m, double lambda0) {
    if (!(lambda0 > 1e-12)) return 0.0;
    const double q = xi_m / lambda0, dq = -xi_m / (lambda0 * lambda0);
    const double h = q - 1.0 > 0.0 ? 1.0 : 0.0;
    double v, dv;
    if (reading == 1) v = q - h, dv = dq;              // literal
    else if (reading == 2) v = q * h, dv = h * dq;     // step
    else v = q - 1.0 > 0.0 ? q - 1.0 : 0.0, dv = h * dq;  // soft
    return 8.0 * v * dv;
}

__device__ inline Sym3 load_e6(const double* e6, size_t n, int c) {
    Sym3 e;
    e.xx = e6[c], e.yy = e6[n + c], e.zz = e6[2 * n + c];
    e.xy = e6[3 * n + c], e.xz = e6[4 * n + c], e.yz = e6[5 * n + c];
    return e;
}

// ---- checkpoints of the forward solve (slot ctl->k)

__global__ void k_ckpt_state(const Ctl* __restrict__ ctl, int cells, const double* __restrict__ phi,
                             const double* __restrict__ ox, const double* __restrict__ oy,
                             const double* __restrict__ oz, double* __restrict__ base) {
    double* dst = base + (size_t)ctl->k * 5 * (size_t)cells;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += gridDim.x * blockDim.x) {
        dst[c] = phi[c];
        dst[(size_t)cells + c] = ox[c];
        dst[2 * (size_t)cells + c] = oy[c];
        dst[3 * (size_t)cells + c] = oz[c];
    }
}

__global__ void k_ckpt_phidot(const Ctl* __restrict__ ctl, int cells,
                              const double* __restrict__ phidot, double* __restrict__ base) {
    double* dst = base + (size_t)ctl->k * 5 * (size_t)cells + 4 * (size_t)cells;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += gridDim.x * blockDim.x)
        dst[c] = phidot[c];
}

// ---- reverse sweep

// delta_r = -lap_7 phi: phibar = -lap_7 gbar (the stencil is symmetric).
__global__ void k_adj_lap(Dims d, const double* __restrict__ gbar, double* __restrict__ phibar) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.cells) return;
    int i, j, k;
    cell_coords(d, c, i, j, k);
    const double g = gbar[c];
    const double acc = (gbar[cell_index(d, i + 1, j, k)] + gbar[cell_index(d, i - 1, j, k)] - 2.0 * g) +
                       (gbar[cell_index(d, i, j + 1, k)] + gbar[cell_index(d, i, j - 1, k)] - 2.0 * g) +
                       (gbar[cell_index(d, i, j, k + 1)] + gbar[cell_index(d, i, j, k - 1)] - 2.0 * g);
    phibar[c] = -acc;
}

// Tracer advance xi_{k+1} = xi_k - alpha sum_corners W(xi_k) V(corner):
// Vbar(corner) -= alpha W xibar (scatter), xibar -= alpha sum dW (V . xibar).
__global__ void k_adj_tracers(Dims d, const double* __restrict__ ox, const double* __restrict__ oy,
                              const double* __restrict__ oz, const double* __restrict__ vx,
                              const double* __restrict__ vy, const double* __restrict__ vz,
                              const double* __restrict__ alpha_p, double* __restrict__ xbx,
                              double* __restrict__ xby, double* __restrict__ xbz,
                              double* __restrict__ vbx, double* __restrict__ vby,
                              double* __restrict__ vbz) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.cells) return;
    const double al = *alpha_p;
    int i, j, k;
    cell_coords(d, c, i, j, k);
    int i0, j0, k0;
    double fx, fy, fz;
    cic_offset(i, ox[c], i0, fx);
    cic_offset(j, oy[c], j0, fy);
    cic_offset(k, oz[c], k0, fz);
    const double bx = xbx[c], by = xby[c], bz = xbz[c];
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (int di = 0; di < 2; ++di) {
        const double wx = di ? fx : 1.0 - fx, sx = di ? 1.0 : -1.0;
        for (int dj = 0; dj < 2; ++dj) {
            const double wy = dj ? fy : 1.0 - fy, sy = dj ? 1.0 : -1.0;
            for (int dk = 0; dk < 2; ++dk) {
                const double wz = dk ? fz : 1.0 - fz, sz = dk ? 1.0 : -1.0;
                const int q = cell_index(d, i0 + di, j0 + dj, k0 + dk);
                const double w = wx * wy * wz;
                const double vd = vx[q] * bx + vy[q] * by + vz[q] * bz;
                ax += sx * wy * wz * vd, ay += wx * sy * wz * vd, az += wx * wy * sz * vd;
                atomicAdd(vbx + q, -al * w * bx);
                atomicAdd(vby + q, -al * w * by);
                atomicAdd(vbz + q, -al * w * bz);
            }
        }
    }
    xbx[c] = bx - al * ax, xby[c] = by - al * ay, xbz[c] = bz - al * az;
}

// V = e^-1 G: Gbar = e^-1 Vbar, ebar = -Gbar V^T, kept as the diagonal
// entries and the symmetrised quarter (ebar_ab + ebar_ba) / 4 of the others
// (the weight the cross stencil of Hess phi gives them).
__global__ void k_adj_velocity(Dims d, const double* __restrict__ e6, const double* __restrict__ v3,
                               const double* __restrict__ vb3, double* __restrict__ gb3,
                               double* __restrict__ eb6) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.cells) return;
    const size_t n = (size_t)d.cells;
    const Sym3 e = load_e6(e6, n, c);
    const double Axx = e.yy * e.zz - e.yz * e.yz, Ayy = e.xx * e.zz - e.xz * e.xz;
    const double Azz = e.xx * e.yy - e.xy * e.xy, Axy = e.xz * e.yz - e.xy * e.zz;
    const double Axz = e.xy * e.yz - e.yy * e.xz, Ayz = e.xy * e.xz - e.xx * e.yz;
    const double inv = 1.0 / det3(e);
    const double bx = vb3[c], by = vb3[n + c], bz = vb3[2 * n + c];
    const double gx = (Axx * bx + Axy * by + Axz * bz) * inv;
    const double gy = (Axy * bx + Ayy * by + Ayz * bz) * inv;
    const double gz = (Axz * bx + Ayz * by + Azz * bz) * inv;
    gb3[c] = gx, gb3[n + c] = gy, gb3[2 * n + c] = gz;
    const double Vx = v3[c], Vy = v3[n + c], Vz = v3[2 * n + c];
    eb6[c] = -gx * Vx, eb6[n + c] = -gy * Vy, eb6[2 * n + c] = -gz * Vz;
    eb6[3 * n + c] = -0.25 * (gx * Vy + gy * Vx);
    eb6[4 * n + c] = -0.25 * (gx * Vz + gz * Vx);
    eb6[5 * n + c] = -0.25 * (gy * Vz + gz * Vy);
}

// dbar = alpha phibar + G^T Gbar (G: central differences), with block sums.
__global__ void k_adj_dbar(Dims d, const double* __restrict__ alpha_p,
                           const double* __restrict__ phibar, const double* __restrict__ gb3,
                           double* __restrict__ dbar, double* __restrict__ psum) {
    const size_t n = (size_t)d.cells;
    const double al = *alpha_p;
    double s = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.cells; c += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_coords(d, c, i, j, k);
        const double g = 0.5 * ((gb3[cell_index(d, i - 1, j, k)] - gb3[cell_index(d, i + 1, j, k)]) +
                                (gb3[n + cell_index(d, i, j - 1, k)] - gb3[n + cell_index(d, i, j + 1, k)]) +
                                (gb3[2 * n + cell_index(d, i, j, k - 1)] -
                                 gb3[2 * n + cell_index(d, i, j, k + 1)]));
        const double v = fma(al, phibar[c], g);
        dbar[c] = v;
        s += v;
    }
    s = block_reduce<OpSum>(s);
    if (threadIdx.x == 0) psum[blockIdx.x] = s;
}

// Coefficient: abar_j = (1/2) sum over the six faces of node j of
// (lam_n - lam_j)(pd_n - pd_j); mbar = abar where m > a_min (a = max(m,
// a_min)), else 0.  Also the block sums of lam.
__global__ void k_adj_coef(Dims d, const double* __restrict__ lam, const double* __restrict__ pd,
                           const double* __restrict__ m, double a_min, double* __restrict__ mbar,
                           double* __restrict__ psum) {
    double s = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.cells; c += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_coords(d, c, i, j, k);
        const double lc = lam[c], pc = pd[c];
        const int nb[6] = {cell_index(d, i + 1, j, k), cell_index(d, i - 1, j, k),
                           cell_index(d, i, j + 1, k), cell_index(d, i, j - 1, k),
                           cell_index(d, i, j, k + 1), cell_index(d, i, j, k - 1)};
        double acc = 0.0;
        for (int q = 0; q < 6; ++q) acc = fma(lam[nb[q]] - lc, pd[nb[q]] - pc, acc);
        mbar[c] = m[c] > a_min ? 0.5 * acc : 0.0;
        s += lc;
    }
    s = block_reduce<OpSum>(s);
    if (threadIdx.x == 0) psum[blockIdx.x] = s;
}

// Source t = (1 - m) + C(lambda0) + E(sqrt g, 1 - m): mbar += tbar dt/dm,
// ebar += tbar C'(lambda0) v v^T (same storage as k_adj_velocity).
__global__ void k_adj_source(Dims d, SourceParams sp, const double* __restrict__ e6,
                             const double* __restrict__ m, const double* __restrict__ tbar,
                             double* __restrict__ mbar, double* __restrict__ eb6) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.cells) return;
    const size_t n = (size_t)d.cells;
    const Sym3 e = load_e6(e6, n, c);
    const double tb = tbar[c];
    const double Sig = 1.0 - m[c];
    const double sg = Sig > 0.0 ? 1.0 : (Sig < 0.0 ? -1.0 : 0.0);
    const double hE = det3(e) - sp.v_m > 0.0 ? 1.0 : 0.0;
    mbar[c] += tb * (-1.0 + 2.0 * hE * sg);
    const double gersh = fmin(fmin(e.xx - fabs(e.xy) - fabs(e.xz), e.yy - fabs(e.xy) - fabs(e.yz)),
                              e.zz - fabs(e.xz) - fabs(e.yz));
    if (sp.climiter == 1 || gersh < sp.xi_m) {
        const double lam = min_eig_sym3(e);
        const double lb = tb * climit_deriv(sp.climiter, sp.xi_m, lam);
        if (lb != 0.0) {
            double v[3];
            eigvec_sym3(e, lam, v);
            eb6[c] += lb * v[0] * v[0];
            eb6[n + c] += lb * v[1] * v[1];
            eb6[2 * n + c] += lb * v[2] * v[2];
            eb6[3 * n + c] += 0.5 * lb * v[0] * v[1];
            eb6[4 * n + c] += 0.5 * lb * v[0] * v[2];
            eb6[5 * n + c] += 0.5 * lb * v[1] * v[2];
        }
    }
}

// phibar += Hess^T ebar: the second differences and the cross stencils are
// symmetric, so the transpose gathers with the same stencils.
__global__ void k_adj_hess(Dims d, const double* __restrict__ eb6, double* __restrict__ phibar) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.cells) return;
    const size_t n = (size_t)d.cells;
    int i, j, k;
    cell_coords(d, c, i, j, k);
    const double* Ex = eb6;
    const double* Ey = eb6 + n;
    const double* Ez = eb6 + 2 * n;
    const double* Xxy = eb6 + 3 * n;
    const double* Xxz = eb6 + 4 * n;
    const double* Xyz = eb6 + 5 * n;
    double acc = (Ex[cell_index(d, i + 1, j, k)] + Ex[cell_index(d, i - 1, j, k)] - 2.0 * Ex[c]) +
                 (Ey[cell_index(d, i, j + 1, k)] + Ey[cell_index(d, i, j - 1, k)] - 2.0 * Ey[c]) +
                 (Ez[cell_index(d, i, j, k + 1)] + Ez[cell_index(d, i, j, k - 1)] - 2.0 * Ez[c]);
    acc += Xxy[cell_index(d, i + 1, j + 1, k)] - Xxy[cell_index(d, i + 1, j - 1, k)] -
           Xxy[cell_index(d, i - 1, j + 1, k)] + Xxy[cell_index(d, i - 1, j - 1, k)];
    acc += Xxz[cell_index(d, i + 1, j, k + 1)] - Xxz[cell_index(d, i + 1, j, k - 1)] -
           Xxz[cell_index(d, i - 1, j, k + 1)] + Xxz[cell_index(d, i - 1, j, k - 1)];
    acc += Xyz[cell_index(d, i, j + 1, k + 1)] - Xyz[cell_index(d, i, j + 1, k - 1)] -
           Xyz[cell_index(d, i, j - 1, k + 1)] + Xyz[cell_index(d, i, j - 1, k - 1)];
    phibar[c] += acc;
}

// m = CIC deposit of the masses w at the tracers: wbar += W . mbar,
// xibar += w dW . mbar (a gather per tracer).
__global__ void k_adj_deposit(Dims d, const double* __restrict__ ox, const double* __restrict__ oy,
                              const double* __restrict__ oz, const double* __restrict__ w,
                              const double* __restrict__ mbar, double* __restrict__ wbar,
                              double* __restrict__ xbx, double* __restrict__ xby,
                              double* __restrict__ xbz) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.cells) return;
    int i, j, k;
    cell_coords(d, c, i, j, k);
    int i0, j0, k0;
    double fx, fy, fz;
    cic_offset(i, ox[c], i0, fx);
    cic_offset(j, oy[c], j0, fy);
    cic_offset(k, oz[c], k0, fz);
    double sw = 0.0, ax = 0.0, ay = 0.0, az = 0.0;
    for (int di = 0; di < 2; ++di) {
        const double wx = di ? fx : 1.0 - fx, sx = di ? 1.0 : -1.0;
        for (int dj = 0; dj < 2; ++dj) {
            const double wy = dj ? fy : 1.0 - fy, sy = dj ? 1.0 : -1.0;
            for (int dk = 0; dk < 2; ++dk) {
                const double wz = dk ? fz : 1.0 - fz, sz = dk ? 1.0 : -1.0;
                const double mb = mbar[cell_index(d, i0 + di, j0 + dj, k0 + dk)];
                sw = fma(wx * wy * wz, mb, sw);
                ax = fma(sx * wy * wz, mb, ax), ay = fma(wx * sy * wz, mb, ay), az = fma(wx * wy * sz, mb, az);
            }
        }
    }
    const double wc = w[c];
    wbar[c] += sw;
    xbx[c] += wc * ax, xby[c] += wc * ay, xbz[c] += wc * az;
}

__global__ void k_adj_dot(int cells, const double* __restrict__ a, const double* __restrict__ b,
                          double* __restrict__ psum) {
    double s = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += gridDim.x * blockDim.x)
        s = fma(a[c], b[c], s);
    s = block_reduce<OpSum>(s);
    if (threadIdx.x == 0) psum[blockIdx.x] = s;
}

// w = rho / rho_bar, rho_bar = sum(rho) / n:
// grad_j = (wbar_j - sum_c wbar_c w_c / n) / rho_bar.
__global__ void k_adj_final(int cells, const double* __restrict__ wbar,
                            const double* __restrict__ sum_wbw, const double* __restrict__ sum_rho,
                            double* __restrict__ grad) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cells) return;
    const double nn = (double)cells;
    const double rho_bar = *sum_rho / nn;
    grad[c] = (wbar[c] - *sum_wbw / nn) / rho_bar;
}

}  // namespace

void launch_ckpt_state(const Ctl* ctl, int cells, const double* phi, const double* ox,
                       const double* oy, const double* oz, double* base, cudaStream_t st) {
    launch_counter()++;
    k_ckpt_state<<<kRedBlocks, kRedThreads, 0, st>>>(ctl, cells, phi, ox, oy, oz, base);
}
void launch_ckpt_phidot(const Ctl* ctl, int cells, const double* phidot, double* base,
                        cudaStream_t st) {
    launch_counter()++;
    k_ckpt_phidot<<<kRedBlocks, kRedThreads, 0, st>>>(ctl, cells, phidot, base);
}
void launch_adj_lap(const Dims& d, const double* gbar, double* phibar, cudaStream_t st) {
    launch_counter()++;
    k_adj_lap<<<nblocks(d.cells), kThreads, 0, st>>>(d, gbar, phibar);
}
void launch_adj_tracers(const Dims& d, const double* ox, const double* oy, const double* oz,
                        const double* v3, const double* alpha, double* xb3, double* vb3,
                        cudaStream_t st) {
    const size_t n = (size_t)d.cells;
    launch_counter()++;
    k_adj_tracers<<<nblocks(d.cells), kThreads, 0, st>>>(d, ox, oy, oz, v3, v3 + n, v3 + 2 * n, alpha,
                                                         xb3, xb3 + n, xb3 + 2 * n, vb3, vb3 + n,
                                                         vb3 + 2 * n);
}
void launch_adj_velocity(const Dims& d, const double* e6, const double* v3, const double* vb3,
                         double* gb3, double* eb6, cudaStream_t st) {
    launch_counter()++;
    k_adj_velocity<<<nblocks(d.cells), kThreads, 0, st>>>(d, e6, v3, vb3, gb3, eb6);
}
void launch_adj_dbar(const Dims& d, const double* alpha, const double* phibar, const double* gb3,
                     double* dbar, double* psum, cudaStream_t st) {
    launch_counter()++;
    k_adj_dbar<<<kRedBlocks, kRedThreads, 0, st>>>(d, alpha, phibar, gb3, dbar, psum);
}
void launch_adj_coef(const Dims& d, const double* lam, const double* pd, const double* m,
                     double a_min, double* mbar, double* psum, cudaStream_t st) {
    launch_counter()++;
    k_adj_coef<<<kRedBlocks, kRedThreads, 0, st>>>(d, lam, pd, m, a_min, mbar, psum);
}
void launch_adj_source(const Dims& d, const SourceParams& sp, const double* e6, const double* m,
                       const double* tbar, double* mbar, double* eb6, cudaStream_t st) {
    launch_counter()++;
    k_adj_source<<<nblocks(d.cells), kThreads, 0, st>>>(d, sp, e6, m, tbar, mbar, eb6);
}
void launch_adj_hess(const Dims& d, const double* eb6, double* phibar, cudaStream_t st) {
    launch_counter()++;
    k_adj_hess<<<nblocks(d.cells), kThreads, 0, st>>>(d, eb6, phibar);
}
void launch_adj_deposit(const Dims& d, const double* ox, const double* oy, const double* oz,
                        const double* w, const double* mbar, double* wbar, double* xb3,
                        cudaStream_t st) {
    const size_t n = (size_t)d.cells;
    launch_counter()++;
    k_adj_deposit<<<nblocks(d.cells), kThreads, 0, st>>>(d, ox, oy, oz, w, mbar, wbar, xb3, xb3 + n,
                                                         xb3 + 2 * n);
}
void launch_adj_dot(int cells, const double* a, const double* b, double* psum, cudaStream_t st) {
    launch_counter()++;
    k_adj_dot<<<kRedBlocks, kRedThreads, 0, st>>>(cells, a, b, psum);
}
void launch_adj_final(int cells, const double* wbar, const double* sum_wbw, const double* sum_rho,
                      double* grad, cudaStream_t st) {
    launch_counter()++;
    k_adj_final<<<nblocks(cells), kThreads, 0, st>>>(cells, wbar, sum_wbw, sum_rho, grad);
}

}  // namespace recon
