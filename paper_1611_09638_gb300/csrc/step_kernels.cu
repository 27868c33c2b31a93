// step_kernels.cu -- kernels of one moving-mesh step (Sec. II, App. A) other
// than the multigrid solve: CIC deposits in 64-bit fixed point, geometry of
// the map x = xi + grad phi, the limited source of Eq. (elliptic), the
// smoothing operator S, the step limiter, the mesh advance and the outputs.
#include "checked.cuh"
#include "geometry.cuh"
#include "recon_internal.cuh"
#include "reduce.cuh"

namespace recon {

namespace {

constexpr int kThreads = 256;
inline int nblocks(long long work) { return (int)((work + kThreads - 1) / kThreads); }

// ---------------------------------------------------------------- helpers

// lambda_min(M) > floor by Sylvester's criterion on M - floor I.
__device__ inline bool pd_above(Sym3 M, double floor) {
    M.xx -= floor, M.yy -= floor, M.zz -= floor;
    return M.xx > 0.0 && (M.xx * M.yy - M.xy * M.xy) > 0.0 && det3(M) > 0.0;
}

// 1 / n for a power of two n (< 2^1023), exactly, from the exponent bits
// (integer work only; x * inv_pow2(n) equals x / n bit for bit).
__device__ inline double inv_pow2(int n) {
    return __longlong_as_double((long long)(1023 - (__ffs(n) - 1)) << 52);
}

// The eight CIC corner charges of one tracer in fixed point.  The offset of
// the tracer from its home node is rounded on each axis to 2^-52 of a cell
// (fixed_axis): the lower node is home + floor and f the fraction in units of
// 2^-52.  The mass M = llrint(w scale) is split exactly,
// first along x into M1 = M f_x / 2^52 rounded to nearest and M0 = M - M1, then each part
// along y, then along z, so the charges are non-negative integers that sum to
// M exactly (mass conservation per tracer).  The splits are 64 x 64-bit
// integer multiplies (upper halves): the FP64 work per tracer is four
// scalings and four conversions, against some 35 FP64 instructions for FP64
// corner weights.  The rounding of a charge is below one unit (1 / scale) of
// the fixed point, like llrint of an FP64 product, and the position's below
// 2^-53 cells, the rounding of an FP64 offset between 1/2 and 1 cell.
struct CicCharges {
    int i0, j0, k0;               // lower corner
    unsigned long long c[2][2][2];  // charges at (i0 + di, j0 + dj, k0 + dk)
};

constexpr int kFracBits = 52;

// The fixed-point position of a tracer along one axis: the offset from its
// home node rounded to 2^-kFracBits of a cell (|off| < 2^11), as the lower
// node and the fraction f in [0, 2^kFracBits).
__device__ inline void fixed_axis(int home, double off, int& i0, unsigned long long& f) {
    const long long q = __double2ll_rn(off * 4503599627370496.0);  // off 2^52
    i0 = home + (int)(q >> kFracBits);                              // floor
    f = (unsigned long long)q & ((1ull << kFracBits) - 1);
}

// m f / 2^52 rounded to nearest (the upper half of m (f 2^12), plus one where
// the lower half is at least 2^63) and the rest m - that: an exact split
// without a bias toward either side.
__device__ inline void split_fixed(unsigned long long m, unsigned long long f, unsigned long long& lo,
                                   unsigned long long& hi) {
    const unsigned long long y = f << (64 - kFracBits);
    hi = __umul64hi(m, y) + ((m * y) >> 63);
    lo = m - hi;
}

// The split of M over the corners for the fractions fx, fy, fz.
__device__ inline void split_charges(unsigned long long M, unsigned long long fx, unsigned long long fy,
                                     unsigned long long fz, CicCharges& r) {
    unsigned long long mx[2], mxy[2][2];
    split_fixed(M, fx, mx[0], mx[1]);
#pragma unroll
    for (int di = 0; di < 2; ++di) {
        split_fixed(mx[di], fy, mxy[di][0], mxy[di][1]);
#pragma unroll
        for (int dj = 0; dj < 2; ++dj) split_fixed(mxy[di][dj], fz, r.c[di][dj][0], r.c[di][dj][1]);
    }
}

__device__ inline CicCharges cic_charges(int i, int j, int k, double ox, double oy, double oz, double w,
                                         double scale) {
    CicCharges r;
    unsigned long long fx, fy, fz;
    fixed_axis(i, ox, r.i0, fx);
    fixed_axis(j, oy, r.j0, fy);
    fixed_axis(k, oz, r.k0, fz);
    split_charges((unsigned long long)__double2ll_rn(w * scale), fx, fy, fz, r);
    return r;
}


// ---------------------------------------------------------------- kernels

__global__ void k_validate_grid(int cells, const double* __restrict__ rho, double* ps, double* pb) {
    double s = 0.0, bad = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += gridDim.x * blockDim.x) {
        const double v = rho[c];
        if (!(v >= 0.0) || !isfinite(v)) bad = 1.0;
        else s += v;
    }
    s = block_reduce<OpSum>(s);
    if (threadIdx.x == 0) ps[blockIdx.x] = s;
    bad = block_reduce<OpMax>(bad);
    if (threadIdx.x == 0) pb[blockIdx.x] = bad;
}

__global__ void k_validate_particles(int64_t np, const double* __restrict__ pos,
                                     const double* __restrict__ mass, double* ps, double* pb) {
    double s = 0.0, bad = 0.0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < np;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double x = pos[3 * p], y = pos[3 * p + 1], z = pos[3 * p + 2];
        if (!isfinite(x) || !isfinite(y) || !isfinite(z)) bad = 1.0;
        const double m = mass ? mass[p] : 1.0;
        if (!(m >= 0.0) || !isfinite(m)) bad = 1.0;
        else s += m;
    }
    s = block_reduce<OpSum>(s);
    if (threadIdx.x == 0) ps[blockIdx.x] = s;
    bad = block_reduce<OpMax>(bad);
    if (threadIdx.x == 0) pb[blockIdx.x] = bad;
}

__global__ void k_deposit_particles(Dims d, int64_t np, const double* __restrict__ pos,
                                    const double* __restrict__ mass, double inv_h, double scale,
                                    unsigned long long* __restrict__ mfix) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    // the position wrapped into [0, n) grid units, then as fixed_axis does
    // for an offset from node 0 (the same integer charges as the tracers')
    // (x * inv_pow2(n) is x / n exactly: n is a power of two)
    auto wrap = [](double x, int n) { return x - (double)n * floor(x * inv_pow2(n)); };
    CicCharges q;
    unsigned long long fx, fy, fz;
    fixed_axis(0, wrap(pos[3 * p] * inv_h, d.n0), q.i0, fx);
    fixed_axis(0, wrap(pos[3 * p + 1] * inv_h, d.n1), q.j0, fy);
    fixed_axis(0, wrap(pos[3 * p + 2] * inv_h, d.n2), q.k0, fz);
    const double m = mass ? mass[p] : 1.0;
    split_charges((unsigned long long)__double2ll_rn(m * scale), fx, fy, fz, q);
    for (int di = 0; di < 2; ++di)
        for (int dj = 0; dj < 2; ++dj)
            for (int dk = 0; dk < 2; ++dk)
                atomicAdd(&mfix[cell_index(d, q.i0 + di, q.j0 + dj, q.k0 + dk)], q.c[di][dj][dk]);
}

__global__ void k_fix_to_double(int cells, unsigned long long* __restrict__ mfix, double inv_scale,
                                double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cells) return;
    out[c] = (double)(long long)mfix[c] * inv_scale;
    mfix[c] = 0ull;
}

__global__ void k_init_tracers(int cells, const double* __restrict__ rho,
                               const double* __restrict__ sum_rho,
                               double* __restrict__ w, double* __restrict__ ox,
                               double* __restrict__ oy, double* __restrict__ oz,
                               double* __restrict__ phi, float* __restrict__ phi32) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cells) return;
    const double inv_rho_bar = 1.0 / (*sum_rho / (double)cells);
    w[c] = rho[c] * inv_rho_bar;
    ox[c] = 0.0, oy[c] = 0.0, oz[c] = 0.0;
    phi[c] = 0.0;
    phi32[c] = 0.0f;
}

// Deposit of the tracers on the deformed mesh: tracer c (home node c, mass
// w_c) sits at curvilinear coordinate c + offset.
__global__ void k_deposit_tracers(Dims d, const double* __restrict__ ox,
                                  const double* __restrict__ oy, const double* __restrict__ oz,
                                  const double* __restrict__ w, double scale,
                                  unsigned long long* __restrict__ mfix) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.cells) return;
    int i, j, k;
    cell_coords(d, c, i, j, k);
    const CicCharges q = cic_charges(i, j, k, ox[c], oy[c], oz[c], w[c], scale);
    for (int di = 0; di < 2; ++di)
        for (int dj = 0; dj < 2; ++dj)
            for (int dk = 0; dk < 2; ++dk)
                atomicAdd(&mfix[cell_index(d, q.i0 + di, q.j0 + dj, q.k0 + dk)], q.c[di][dj][dk]);
}

// The same deposit (same fixed-point values) with shared-memory accumulation:
// a block takes the tracers whose home nodes form a DTI x DTJ x DTK tile and
// adds each corner weight into a copy of the tile plus DH nodes on every side
// held in shared memory, then adds the non-zero cells of that copy to the
// grid.  A tracer whose stencil leaves the copy adds to the grid directly.
// The fixed-point sums are integers, so the result is bit-identical to
// k_deposit_tracers while the grid sees ~4x fewer atomics.  The corner
// charges are cic_charges' exact integer split of the tracer's mass.
constexpr int DTI = 8, DTJ = 16, DTK = 32, DH = 2;
constexpr int DRI = DTI + 2 * DH, DRJ = DTJ + 2 * DH, DRK = DTK + 2 * DH;
constexpr int DCELLS = DRI * DRJ * DRK;
constexpr size_t kDepSmem = sizeof(unsigned long long) * DCELLS;

__global__ void __launch_bounds__(256) k_deposit_tracers_tiled(Dims d, const double* __restrict__ ox,
                                                               const double* __restrict__ oy,
                                                               const double* __restrict__ oz,
                                                               const double* __restrict__ w,
                                                               double scale,
                                                               unsigned long long* __restrict__ mfix) {
    extern __shared__ unsigned long long acc[];
    const int t = threadIdx.x;
    for (int e = t; e < DCELLS; e += blockDim.x) acc[e] = 0ull;
    __syncthreads();
    const int ti = blockIdx.z * DTI, tj = blockIdx.y * DTJ, tk = blockIdx.x * DTK;
    for (int q = t; q < DTI * DTJ * DTK; q += blockDim.x) {
        const int li = q / (DTJ * DTK), lj = (q / DTK) % DTJ, lk = q % DTK;
        const int i = ti + li, j = tj + lj, k = tk + lk;
        const int c = cell_index(d, i, j, k);
        const CicCharges ch = cic_charges(i, j, k, ox[c], oy[c], oz[c], w[c], scale);
        const int i0 = ch.i0, j0 = ch.j0, k0 = ch.k0;
        const int bi = i0 - ti + DH, bj = j0 - tj + DH, bk = k0 - tk + DH;
        const bool local = bi >= 0 && bi + 1 < DRI && bj >= 0 && bj + 1 < DRJ && bk >= 0 && bk + 1 < DRK;
        for (int di = 0; di < 2; ++di) {
            for (int dj = 0; dj < 2; ++dj) {
                for (int dk = 0; dk < 2; ++dk) {
                    const unsigned long long qv = ch.c[di][dj][dk];
                    if (local)
                        atomicAdd(&acc[RC_OFF(((bi + di) * DRJ + (bj + dj)) * DRK + (bk + dk), DCELLS, 401)], qv);
                    else
                        atomicAdd(&mfix[cell_index(d, i0 + di, j0 + dj, k0 + dk)], qv);
                }
            }
        }
    }
    __syncthreads();
    for (int e = t; e < DCELLS; e += blockDim.x) {
        const unsigned long long v = acc[e];
        if (!v) continue;  // every contribution is >= 0, so 0 means none
        const int ri = e / (DRJ * DRK), rj = (e / DRK) % DRJ, rk = e % DRK;
        atomicAdd(&mfix[cell_index(d, ti - DH + ri, tj - DH + rj, tk - DH + rk)], v);
    }
}

// m from the fixed-point accumulator (which is cleared for the next deposit),
// coefficient a = max(m, a_min) in FP64 and FP32, and partial sums of m.
__global__ void k_mass_coef(int cells, unsigned long long* __restrict__ mfix, double inv_scale,
                            double a_min, double* __restrict__ m, double* __restrict__ a64,
                            float* __restrict__ a32, double* __restrict__ part) {
    double s = 0.0;
    const int stride = gridDim.x * blockDim.x;
    auto one = [&](int c, long long q) {
        const double v = (double)q * inv_scale;
        mfix[c] = 0ull;
        m[c] = v;
        const double a = v > a_min ? v : a_min;
        a64[c] = a;
        if (a32) a32[c] = (float)a;
        s += v;
    };
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    // four loads in flight per thread; the nodes are summed in the same order
    for (; c + 3 * stride < cells; c += 4 * stride) {
        long long q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = (long long)mfix[c + u * stride];
#pragma unroll
        for (int u = 0; u < 4; ++u) one(c + u * stride, q[u]);
    }
    for (; c < cells; c += stride) one(c, (long long)mfix[c]);
    s = block_reduce<OpSum>(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// Source of App. A Eq. (elliptic) before smoothing: t = Sigma + C + E with
// Sigma = 1 - m, C(lambda0) the compression limiter of the triad
// e = I + Hess phi and E = -2 H(sqrt_g - v_m) |Sigma| the expansion limiter.
// lambda0 only matters where it is below xi_m (for the soft and step readings
// C vanishes above it); the Gershgorin bound skips the eigenvalue elsewhere.
__global__ void k_geometry_source(Dims d, SourceParams sp, const double* __restrict__ phi,
                                  const double* __restrict__ m, double* __restrict__ t,
                                  double* __restrict__ e6, double* __restrict__ psum,
                                  double* __restrict__ pmin) {
    double s = 0.0, mdet = INFINITY;
    const size_t n = (size_t)d.cells;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.cells; c += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_coords(d, c, i, j, k);
        Sym3 e = hessian(d, phi, i, j, k);
        e.xx += 1.0, e.yy += 1.0, e.zz += 1.0;
        // the triad is kept for the limiter and the advance of this step
        e6[c] = e.xx, e6[n + c] = e.yy, e6[2 * n + c] = e.zz;
        e6[3 * n + c] = e.xy, e6[4 * n + c] = e.xz, e6[5 * n + c] = e.yz;
        const double g = det3(e);
        double C = 0.0;
        const double gersh =
            fmin(fmin(e.xx - fabs(e.xy) - fabs(e.xz), e.yy - fabs(e.xy) - fabs(e.yz)),
                 e.zz - fabs(e.xz) - fabs(e.yz));
        if (sp.climiter == 1 || gersh < sp.xi_m) C = climit(sp.climiter, sp.xi_m, min_eig_sym3(e));
        const double Sigma = 1.0 - m[c];
        const double E = g - sp.v_m > 0.0 ? -2.0 * fabs(Sigma) : 0.0;
        const double v = Sigma + C + E;
        t[c] = v;
        s += v;
        mdet = fmin(mdet, g);
    }
    s = block_reduce<OpSum>(s);
    if (threadIdx.x == 0) psum[blockIdx.x] = s;
    mdet = block_reduce<OpMin>(mdet);
    if (threadIdx.x == 0) pmin[blockIdx.x] = mdet;
}

// One axis of the smoothing operator S (a weighted mean over the 3x3x3
// neighbourhood, separable into (w, 1-2w, w) along each axis): out =
// w in[-1] + (1-2w) in[0] + w in[+1] along `axis`, minus (*shift_sum / cells)
// when shift_sum is given; optional per-block sums of out and out^2.  Three
// passes (k, j, i) cost 9 FP64 instructions per node against 27 for the
// direct 27-point sum.
__global__ void k_smooth_axis(Dims d, int axis, double ws, const double* __restrict__ in,
                              const double* __restrict__ shift_sum, double* __restrict__ out,
                              float* __restrict__ out32, double* __restrict__ psum,
                              double* __restrict__ psq) {
    const double w1 = 1.0 - 2.0 * ws;
    const double shift = shift_sum ? *shift_sum / (double)d.cells : 0.0;
    const int di = axis == 0, dj = axis == 1, dk = axis == 2;
    double s = 0.0, q = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.cells; c += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_coords(d, c, i, j, k);
        const double v = fma(ws, in[cell_index(d, i - di, j - dj, k - dk)] +
                                     in[cell_index(d, i + di, j + dj, k + dk)],
                             w1 * in[c]) - shift;
        out[c] = v;
        if (out32) out32[c] = (float)v;
        s += v;
        q = fma(v, v, q);
    }
    if (psum) {
        s = block_reduce<OpSum>(s);
        if (threadIdx.x == 0) psum[blockIdx.x] = s;
    }
    if (psq) {
        q = block_reduce<OpSum>(q);
        if (threadIdx.x == 0) psq[blockIdx.x] = q;
    }
}

// S in one pass: a block takes SJ x SK tiles of the (j, k) plane and streams
// SCI planes along i; each plane (with a one-node ring) is staged in shared
// memory and smoothed along k, then along j, and each thread keeps the last
// two (j, k)-smoothed values of its column in registers for the pass along
// i.  The three passes use the expressions of k_smooth_axis in the same order
// (k, j, i), so the output equals the three-kernel form bit for bit; only the
// order of the partial sums differs.  The grid is kRedBlocks blocks looping
// over the tiles, so the partial sums are those of fixed blocks.
constexpr int SJ = 8, SK = 32, SCI = 16;

__global__ void __launch_bounds__(256) k_smooth_S_stream(Dims d, double ws,
                                                         const double* __restrict__ in,
                                                         const double* __restrict__ shift_sum,
                                                         double* __restrict__ out,
                                                         float* __restrict__ out32,
                                                         double* __restrict__ psum,
                                                         double* __restrict__ psq) {
    __shared__ double pl[SJ + 2][SK + 2];  // plane with a one-node ring
    __shared__ double sk[SJ + 2][SK];      // smoothed along k
    const double w1 = 1.0 - 2.0 * ws;
    const double shift = shift_sum ? *shift_sum / (double)d.cells : 0.0;
    const int t = threadIdx.x, lj = t / SK, lk = t % SK;
    const int tiles_k = d.n2 / SK, tiles_j = d.n1 / SJ;
    const int ntiles = tiles_k * tiles_j * (d.n0 / SCI);
    double s = 0.0, q = 0.0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tk = tile % tiles_k, tj = (tile / tiles_k) % tiles_j, ti = tile / (tiles_k * tiles_j);
        const int k0 = tk * SK, j0 = tj * SJ, i0 = ti * SCI;
        double a2 = 0.0, a1 = 0.0;  // (j, k)-smoothed values of planes p - 2, p - 1
        for (int p = i0 - 1; p <= i0 + SCI; ++p) {
            for (int e = t; e < (SJ + 2) * (SK + 2); e += blockDim.x) {
                const int r = e / (SK + 2), c = e - r * (SK + 2);
                pl[r][c] = in[cell_index(d, p, j0 - 1 + r, k0 - 1 + c)];
            }
            __syncthreads();
            for (int e = t; e < (SJ + 2) * SK; e += blockDim.x) {
                const int r = e / SK, c = e - r * SK;
                sk[r][c] = fma(ws, pl[r][c] + pl[r][c + 2], w1 * pl[r][c + 1]);
            }
            __syncthreads();
            const double v = fma(ws, sk[lj][lk] + sk[lj + 2][lk], w1 * sk[lj + 1][lk]);
            if (p > i0) {  // plane p - 1 is complete
                const double o = fma(ws, a2 + v, w1 * a1) - shift;
                const int c = cell_index(d, p - 1, j0 + lj, k0 + lk);
                out[c] = o;
                if (out32) out32[c] = (float)o;
                s += o;
                q = fma(o, o, q);
            }
            a2 = a1, a1 = v;
            __syncthreads();  // pl and sk are refilled for the next plane
        }
    }
    if (psum) {
        s = block_reduce<OpSum>(s);
        if (threadIdx.x == 0) psum[blockIdx.x] = s;
    }
    if (psq) {
        q = block_reduce<OpSum>(q);
        if (threadIdx.x == 0) psq[blockIdx.x] = q;
    }
}

template <typename T>
struct Hess3 {
    T xx, yy, zz, xy, xz, yz;
};

// Hessian in FP32 of an FP32 copy, and the largest |value| it read.
__device__ inline Hess3<float> hessian32(const Dims& d, const float* __restrict__ f, int i, int j,
                                         int k, float& vmax) {
    float v[19];
    v[0] = f[cell_index(d, i, j, k)];
    v[1] = f[cell_index(d, i + 1, j, k)], v[2] = f[cell_index(d, i - 1, j, k)];
    v[3] = f[cell_index(d, i, j + 1, k)], v[4] = f[cell_index(d, i, j - 1, k)];
    v[5] = f[cell_index(d, i, j, k + 1)], v[6] = f[cell_index(d, i, j, k - 1)];
    v[7] = f[cell_index(d, i + 1, j + 1, k)], v[8] = f[cell_index(d, i + 1, j - 1, k)];
    v[9] = f[cell_index(d, i - 1, j + 1, k)], v[10] = f[cell_index(d, i - 1, j - 1, k)];
    v[11] = f[cell_index(d, i + 1, j, k + 1)], v[12] = f[cell_index(d, i + 1, j, k - 1)];
    v[13] = f[cell_index(d, i - 1, j, k + 1)], v[14] = f[cell_index(d, i - 1, j, k - 1)];
    v[15] = f[cell_index(d, i, j + 1, k + 1)], v[16] = f[cell_index(d, i, j + 1, k - 1)];
    v[17] = f[cell_index(d, i, j - 1, k + 1)], v[18] = f[cell_index(d, i, j - 1, k - 1)];
    vmax = 0.0f;
#pragma unroll
    for (int q = 0; q < 19; ++q) vmax = fmaxf(vmax, fabsf(v[q]));
    Hess3<float> H;
    H.xx = v[1] - 2.0f * v[0] + v[2];
    H.yy = v[3] - 2.0f * v[0] + v[4];
    H.zz = v[5] - 2.0f * v[0] + v[6];
    H.xy = 0.25f * (v[7] - v[8] - v[9] + v[10]);
    H.xz = 0.25f * (v[11] - v[12] - v[13] + v[14]);
    H.yz = 0.25f * (v[15] - v[16] - v[17] + v[18]);
    return H;
}

// Sylvester's test of N = M - floor I in FP32 with a bound on its error:
// returns +1 when N is certainly positive definite, -1 when it certainly is
// not, 0 when FP32 cannot tell.  eps bounds the error of every entry of M;
// the minors' bounds add the propagated entry errors and the FP32 roundings
// of their own evaluation (u = 2^-24).
__device__ inline int sylvester32(float xx, float yy, float zz, float xy, float xz, float yz,
                                  float floor, float eps) {
    constexpr float u = 5.96046448e-8f;
    xx -= floor, yy -= floor, zz -= floor;
    const float big = fmaxf(fmaxf(fabsf(xx), fabsf(yy)), fmaxf(fabsf(zz),
                            fmaxf(fabsf(xy), fmaxf(fabsf(xz), fabsf(yz)))));
    const float en = eps + 2.0f * u * (big + floor);  // entries of N
    const float m1 = xx;
    const float m2 = xx * yy - xy * xy;
    const float m3 = xx * (yy * zz - yz * yz) - xy * (xy * zz - yz * xz) + xz * (xy * yz - yy * xz);
    const float e1 = en;
    const float e2 = 4.0f * en * big + en * en + 8.0f * u * big * big;
    const float e3 = 9.0f * en * big * big + 3.0f * en * en * big + en * en * en + 72.0f * u * big * big * big;
    if (m1 < -e1 || m2 < -e2 || m3 < -e3) return -1;
    if (m1 > e1 && m2 > e2 && m3 > e3) return 1;
    return 0;
}

// Step limiter, per node: the smallest k in [0, kmax] with
// lambda_min(e + 2^-k Hess dphi) > floor (kmax + 1 if none), e = I + Hess phi
// the FP64 triad stored by k_geometry_source, and max_a |central grad_a
// dphi|.  Both are max-reduced over the grid.
// Each alpha is first tested in FP32 on Hessians of FP32 copies of phi and
// dphi, with a bound on every rounding involved (an entry of a Hessian
// combines at most four stencil values of magnitude <= vmax; the FP32 copies
// and at most four operations each round by 2^-24 relative, so 32 u vmax
// bounds its error with room to spare).  Only when FP32 cannot certify the answer does the node
// take the FP64 test (Sylvester's criterion on the FP64 triad); where FP32
// certifies it, the FP64 test gives the same answer, so every decision is the
// FP64 one while most nodes issue no FP64 arithmetic beyond the move limit.
__global__ void k_limiter(Dims d, LimiterParams lp, const double* __restrict__ e6,
                          const double* __restrict__ dphi, const float* __restrict__ phi32,
                          const float* __restrict__ dphi32, double* __restrict__ pk,
                          double* __restrict__ pg) {
    constexpr float u = 5.96046448e-8f;
    double kk = 0.0;
    unsigned long long gbits = 0ull;  // max |G| as the bits of a non-negative double
    const size_t n = (size_t)d.cells;
    const float floor32 = (float)lp.lambda_floor;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.cells; c += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_coords(d, c, i, j, k);
        // move limit: central differences of dphi in FP64 (the max is taken on
        // the bit patterns, 0.5 is applied once per block)
        const double gx = dphi[cell_index(d, i + 1, j, k)] - dphi[cell_index(d, i - 1, j, k)];
        const double gy = dphi[cell_index(d, i, j + 1, k)] - dphi[cell_index(d, i, j - 1, k)];
        const double gz = dphi[cell_index(d, i, j, k + 1)] - dphi[cell_index(d, i, j, k - 1)];
        const unsigned long long mask = 0x7fffffffffffffffull;
        gbits = max(gbits, (unsigned long long)__double_as_longlong(gx) & mask);
        gbits = max(gbits, (unsigned long long)__double_as_longlong(gy) & mask);
        gbits = max(gbits, (unsigned long long)__double_as_longlong(gz) & mask);
        float vm0, vm1;
        const Hess3<float> A = hessian32(d, phi32, i, j, k, vm0);
        const Hess3<float> B = hessian32(d, dphi32, i, j, k, vm1);
        bool have64 = false;
        Sym3 e, H1;
        int kn = lp.kmax + 1;
        float al = 1.0f;
        for (int q = 0; q <= lp.kmax; ++q, al *= 0.5f) {
            const float mxx = 1.0f + A.xx + al * B.xx, myy = 1.0f + A.yy + al * B.yy;
            const float mzz = 1.0f + A.zz + al * B.zz, mxy = A.xy + al * B.xy;
            const float mxz = A.xz + al * B.xz, myz = A.yz + al * B.yz;
            const float big = fmaxf(fmaxf(fabsf(mxx), fabsf(myy)),
                                    fmaxf(fabsf(mzz), fmaxf(fabsf(mxy), fmaxf(fabsf(mxz), fabsf(myz)))));
            // inputs and Hessian arithmetic (|entry| <= 4 vmax), then the two
            // additions forming M
            const float eps = 32.0f * u * (vm0 + al * vm1) + 4.0f * u * (big + 1.0f);
            const int v = sylvester32(mxx, myy, mzz, mxy, mxz, myz, floor32, eps);
            bool pass;
            if (v != 0) {
                pass = v > 0;
            } else {
                if (!have64) {
                    e.xx = e6[c], e.yy = e6[n + c], e.zz = e6[2 * n + c];
                    e.xy = e6[3 * n + c], e.xz = e6[4 * n + c], e.yz = e6[5 * n + c];
                    H1 = hessian(d, dphi, i, j, k);
                    have64 = true;
                }
                const double al64 = ldexp(1.0, -q);
                Sym3 M;
                M.xx = e.xx + al64 * H1.xx, M.yy = e.yy + al64 * H1.yy, M.zz = e.zz + al64 * H1.zz;
                M.xy = e.xy + al64 * H1.xy, M.xz = e.xz + al64 * H1.xz, M.yz = e.yz + al64 * H1.yz;
                pass = pd_above(M, lp.lambda_floor);
            }
            if (pass) {
                kn = q;
                break;
            }
        }
        kk = fmax(kk, (double)kn);
    }
    kk = block_reduce<OpMax>(kk);
    if (threadIdx.x == 0) pk[blockIdx.x] = kk;
    double gm = 0.5 * __longlong_as_double((long long)gbits);
    gm = block_reduce<OpMax>(gm);
    if (threadIdx.x == 0) pg[blockIdx.x] = gm;
}

// V = e^-1 G at every node: e = I + Hess phi (before the step; stored by
// k_geometry_source), G the central-difference gradient of dphi; e^-1 from
// the adjugate of the symmetric e.
__global__ void k_node_velocity(Dims d, const double* __restrict__ e6,
                                const double* __restrict__ dphi, double* __restrict__ vx,
                                double* __restrict__ vy, double* __restrict__ vz) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.cells) return;
    int i, j, k;
    cell_coords(d, c, i, j, k);
    const size_t n = (size_t)d.cells;
    Sym3 e;
    e.xx = e6[c], e.yy = e6[n + c], e.zz = e6[2 * n + c];
    e.xy = e6[3 * n + c], e.xz = e6[4 * n + c], e.yz = e6[5 * n + c];
    // twice the central-difference gradient of dphi (the 1/2 goes with 1/det)
    const double gx = dphi[cell_index(d, i + 1, j, k)] - dphi[cell_index(d, i - 1, j, k)];
    const double gy = dphi[cell_index(d, i, j + 1, k)] - dphi[cell_index(d, i, j - 1, k)];
    const double gz = dphi[cell_index(d, i, j, k + 1)] - dphi[cell_index(d, i, j, k - 1)];
    // e^-1 = adj(e) / det e with the six cofactors of the symmetric e
    const double Axx = e.yy * e.zz - e.yz * e.yz, Ayy = e.xx * e.zz - e.xz * e.xz;
    const double Azz = e.xx * e.yy - e.xy * e.xy, Axy = e.xz * e.yz - e.xy * e.zz;
    const double Axz = e.xy * e.yz - e.yy * e.xz, Ayz = e.xy * e.xz - e.xx * e.yz;
    const double hinv = 0.5 / (e.xx * Axx + e.xy * Axy + e.xz * Axz);
    vx[c] = (Axx * gx + Axy * gy + Axz * gz) * hinv;
    vy[c] = (Axy * gx + Ayy * gy + Ayz * gz) * hinv;
    vz[c] = (Axz * gx + Ayz * gy + Azz * gz) * hinv;
}

// The step's node displacement alpha V = alpha e^-1 G (V as in
// k_node_velocity) in fixed point with kDispBits fractional bits, for the
// tracer advance's integer interpolation.  The step limiter bounds it by
// d_max / lambda_floor (50 cells at the defaults); values beyond kDispMax
// cells, which no valid step produces, are held at that bound.
constexpr int kDispBits = 53;
constexpr long long kDispMax = 1ll << (kDispBits + 7);  // 128 cells
__global__ void k_node_displacement(Dims d, const double* __restrict__ e6,
                                    const double* __restrict__ dphi, const double* __restrict__ alpha_p,
                                    long long* __restrict__ dx, long long* __restrict__ dy,
                                    long long* __restrict__ dz) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.cells) return;
    int i, j, k;
    cell_coords(d, c, i, j, k);
    const size_t n = (size_t)d.cells;
    Sym3 e;
    e.xx = e6[c], e.yy = e6[n + c], e.zz = e6[2 * n + c];
    e.xy = e6[3 * n + c], e.xz = e6[4 * n + c], e.yz = e6[5 * n + c];
    const double gx = dphi[cell_index(d, i + 1, j, k)] - dphi[cell_index(d, i - 1, j, k)];
    const double gy = dphi[cell_index(d, i, j + 1, k)] - dphi[cell_index(d, i, j - 1, k)];
    const double gz = dphi[cell_index(d, i, j, k + 1)] - dphi[cell_index(d, i, j, k - 1)];
    const double Axx = e.yy * e.zz - e.yz * e.yz, Ayy = e.xx * e.zz - e.xz * e.xz;
    const double Azz = e.xx * e.yy - e.xy * e.xy, Axy = e.xz * e.yz - e.xy * e.zz;
    const double Axz = e.xy * e.yz - e.yy * e.xz, Ayz = e.xy * e.xz - e.xx * e.yz;
    // 1/2 of the central differences, alpha and 2^kDispBits in one factor
    const double hinv = (0.5 * 9007199254740992.0) * *alpha_p / (e.xx * Axx + e.xy * Axy + e.xz * Axz);
    auto fix = [](double v) {
        const long long q = __double2ll_rn(v);  // saturates beyond the int64 range
        return q > kDispMax ? kDispMax : (q < -kDispMax ? -kDispMax : q);
    };
    dx[c] = fix((Axx * gx + Axy * gy + Axz * gz) * hinv);
    dy[c] = fix((Axy * gx + Ayy * gy + Ayz * gz) * hinv);
    dz[c] = fix((Axz * gx + Ayz * gy + Azz * gz) * hinv);
}

// App. A's linear density update (the variant that carries m instead of
// re-depositing tracers): K = m e^-1 at every node, e = I + Hess phi the
// stored triad (symmetric, so K is too: xx, yy, zz, xy, xz, yz).
__global__ void k_mass_tensor(Dims d, const double* __restrict__ e6, const double* __restrict__ m,
                              double* __restrict__ K6) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.cells) return;
    const size_t n = (size_t)d.cells;
    Sym3 e;
    e.xx = e6[c], e.yy = e6[n + c], e.zz = e6[2 * n + c];
    e.xy = e6[3 * n + c], e.xz = e6[4 * n + c], e.yz = e6[5 * n + c];
    const double cxx = e.yy * e.zz - e.yz * e.yz, cyy = e.xx * e.zz - e.xz * e.xz;
    const double czz = e.xx * e.yy - e.xy * e.xy, cxy = e.xz * e.yz - e.xy * e.zz;
    const double cxz = e.xy * e.yz - e.xz * e.yy, cyz = e.xy * e.xz - e.xx * e.yz;
    const double s = m[c] / det3(e);
    K6[c] = cxx * s, K6[n + c] = cyy * s, K6[2 * n + c] = czz * s;
    K6[3 * n + c] = cxy * s, K6[4 * n + c] = cxz * s, K6[5 * n + c] = cyz * s;
}

// m += alpha d_mu(K^{mu nu} d_nu v) in flux form: per axis the second
// difference with face coefficients (K_c + K_n)/2, per axis pair the
// difference of centred differences taken at the two neighbours.
__global__ void k_mass_update(Dims d, const double* __restrict__ K6, const double* __restrict__ v,
                              const double* __restrict__ alpha_p, double* __restrict__ m) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.cells) return;
    const double alpha = *alpha_p;
    int i, j, k;
    cell_coords(d, c, i, j, k);
    const size_t n = (size_t)d.cells;
    const int o[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    const int off[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};  // K6 slot of (a, b)
    const double vc = v[c];
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int pl = cell_index(d, i + o[a][0], j + o[a][1], k + o[a][2]);
        const int mi = cell_index(d, i - o[a][0], j - o[a][1], k - o[a][2]);
        const double* Ka = K6 + off[a][a] * n;
        acc += 0.5 * (Ka[c] + Ka[pl]) * (v[pl] - vc) - 0.5 * (Ka[c] + Ka[mi]) * (vc - v[mi]);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (b == a) continue;
            const double* Kab = K6 + off[a][b] * n;
            const int pi = i + o[a][0], pj = j + o[a][1], pk = k + o[a][2];
            const int qi = i - o[a][0], qj = j - o[a][1], qk = k - o[a][2];
            const double dp = v[cell_index(d, pi + o[b][0], pj + o[b][1], pk + o[b][2])] -
                              v[cell_index(d, pi - o[b][0], pj - o[b][1], pk - o[b][2])];
            const double dm = v[cell_index(d, qi + o[b][0], qj + o[b][1], qk + o[b][2])] -
                              v[cell_index(d, qi - o[b][0], qj - o[b][1], qk - o[b][2])];
            acc += 0.25 * (Kab[pl] * dp - Kab[mi] * dm);
        }
    }
    m[c] += alpha * acc;
}

// a = max(m, a_min) in FP64 (and FP32) with partial sums of m, for the
// variant whose m is carried rather than deposited.
__global__ void k_coef_from_m(int cells, const double* __restrict__ m, double a_min,
                              double* __restrict__ a64, float* __restrict__ a32,
                              double* __restrict__ part) {
    double s = 0.0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += gridDim.x * blockDim.x) {
        const double v = m[c];
        const double a = v > a_min ? v : a_min;
        a64[c] = a;
        if (a32) a32[c] = (float)a;
        s += v;
    }
    s = block_reduce<OpSum>(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// phi += alpha (dphi - mean) without moving tracers.
__global__ void k_phi_advance(int cells, const double* __restrict__ alpha_p,
                              const double* __restrict__ dphi, const double* __restrict__ sum_dphi,
                              double* __restrict__ phi, float* __restrict__ phi32) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cells) return;
    const double alpha = *alpha_p;
    const double mean = *sum_dphi * inv_pow2(cells);
    const double pn = phi[c] + alpha * (dphi[c] - mean);
    phi[c] = pn;
    phi32[c] = (float)pn;
}

// (b - a) f / 2^52 rounded to nearest, added to a: one step of linear
// interpolation of fixed-point values with a fraction f of fixed_axis
// (|b - a| <= 2^61; the 128-bit product's upper half is the floor, its lower
// half's top bit the rounding).
__device__ inline long long lerp_fixed(long long a, long long b, unsigned long long f) {
    const long long x = (b - a) * 2, y = (long long)(f << (63 - kFracBits));
    const unsigned long long low = (unsigned long long)x * (unsigned long long)y;
    return a + __mul64hi(x, y) + (long long)(low >> 63);
}

// Tracers move by -alpha V(xi), V CIC-interpolated from the nodes, in fixed
// point: the offsets are rounded to 2^-52 cell as in cic_charges, and the
// node displacements alpha V (k_node_displacement, 2^-kDispBits cells) are
// interpolated by integer linear interpolation along k, then j, then i, each
// step rounded to nearest (rounding down instead biases every move by about a
// unit the same way, which the 40-step 32^3 trajectory amplified to 3e-6 in
// R_k); the result leaves as one FP64 subtraction per axis.
// phi += alpha (dphi - mean), mean = *sum_dphi / cells.
__global__ void k_advance(Dims d, const long long* __restrict__ dx, const long long* __restrict__ dy,
                          const long long* __restrict__ dz, const double* __restrict__ alpha_p,
                          const double* __restrict__ dphi, const double* __restrict__ sum_dphi,
                          double* __restrict__ ox, double* __restrict__ oy,
                          double* __restrict__ oz, double* __restrict__ phi,
                          float* __restrict__ phi32) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.cells) return;
    const double alpha = *alpha_p;
    int i, j, k;
    cell_coords(d, c, i, j, k);
    const double px = ox[c], py = oy[c], pz = oz[c];
    int i0, j0, k0;
    unsigned long long fx, fy, fz;
    fixed_axis(i, px, i0, fx);
    fixed_axis(j, py, j0, fy);
    fixed_axis(k, pz, k0, fz);
    int nb[2][2][2];
#pragma unroll
    for (int di = 0; di < 2; ++di)
#pragma unroll
        for (int dj = 0; dj < 2; ++dj)
#pragma unroll
            for (int dk = 0; dk < 2; ++dk) nb[di][dj][dk] = cell_index(d, i0 + di, j0 + dj, k0 + dk);
    auto interp = [&](const long long* __restrict__ D) {
        long long cx[2];
#pragma unroll
        for (int di = 0; di < 2; ++di) {
            const long long c0 = lerp_fixed(D[nb[di][0][0]], D[nb[di][0][1]], fz);
            const long long c1 = lerp_fixed(D[nb[di][1][0]], D[nb[di][1][1]], fz);
            cx[di] = lerp_fixed(c0, c1, fy);
        }
        return lerp_fixed(cx[0], cx[1], fx);
    };
    constexpr double unit = 1.0 / 9007199254740992.0;  // 2^-kDispBits
    ox[c] = fma(-(double)interp(dx), unit, px);
    oy[c] = fma(-(double)interp(dy), unit, py);
    oz[c] = fma(-(double)interp(dz), unit, pz);
    const double mean = *sum_dphi * inv_pow2(d.cells);
    const double pn = phi[c] + alpha * (dphi[c] - mean);
    phi[c] = pn;
    phi32[c] = (float)pn;
}

__global__ void k_delta_r(Dims d, const double* __restrict__ phi, double* __restrict__ out,
                          double* __restrict__ pmax) {
    double mx = -INFINITY;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.cells; c += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_coords(d, c, i, j, k);
        const double p = phi[c];
        const double lap = (phi[cell_index(d, i + 1, j, k)] - 2.0 * p + phi[cell_index(d, i - 1, j, k)]) +
                           (phi[cell_index(d, i, j + 1, k)] - 2.0 * p + phi[cell_index(d, i, j - 1, k)]) +
                           (phi[cell_index(d, i, j, k + 1)] - 2.0 * p + phi[cell_index(d, i, j, k - 1)]);
        out[c] = -lap;
        mx = fmax(mx, -lap);
    }
    mx = block_reduce<OpMax>(mx);
    if (threadIdx.x == 0) pmax[blockIdx.x] = mx;
}

__global__ void k_mesh_x(Dims d, const double* __restrict__ phi, double h, double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= d.cells) return;
    int i, j, k;
    cell_coords(d, c, i, j, k);
    out[3 * c + 0] = ((double)i + 0.5 * (phi[cell_index(d, i + 1, j, k)] - phi[cell_index(d, i - 1, j, k)])) * h;
    out[3 * c + 1] = ((double)j + 0.5 * (phi[cell_index(d, i, j + 1, k)] - phi[cell_index(d, i, j - 1, k)])) * h;
    out[3 * c + 2] = ((double)k + 0.5 * (phi[cell_index(d, i, j, k + 1)] - phi[cell_index(d, i, j, k - 1)])) * h;
}

__global__ void k_geometry_out(Dims d, const double* __restrict__ phi, double* __restrict__ det,
                               double* __restrict__ lam, double* __restrict__ pdet,
                               double* __restrict__ plam) {
    double md = INFINITY, ml = INFINITY;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d.cells; c += gridDim.x * blockDim.x) {
        int i, j, k;
        cell_coords(d, c, i, j, k);
        Sym3 e = hessian(d, phi, i, j, k);
        e.xx += 1.0, e.yy += 1.0, e.zz += 1.0;
        const double g = det3(e);
        if (det) det[c] = g;
        md = fmin(md, g);
        // lambda0 >= the Gershgorin bound, so without a per-node output the
        // eigenvalue is needed only where that bound is below the running min
        const double gersh =
            fmin(fmin(e.xx - fabs(e.xy) - fabs(e.xz), e.yy - fabs(e.xy) - fabs(e.yz)),
                 e.zz - fabs(e.xz) - fabs(e.yz));
        if (lam || gersh < ml) {
            const double l = min_eig_sym3(e);
            if (lam) lam[c] = l;
            ml = fmin(ml, l);
        }
    }
    md = block_reduce<OpMin>(md);
    if (threadIdx.x == 0) pdet[blockIdx.x] = md;
    ml = block_reduce<OpMin>(ml);
    if (threadIdx.x == 0) plam[blockIdx.x] = ml;
}

__global__ void k_scale(int cells, const double* __restrict__ in, double s, double* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < cells) out[c] = in[c] * s;
}

template <class Op>
__global__ void k_finish(const double* __restrict__ partials, double* __restrict__ scalars, int slot) {
    double v = Op::id();
    for (int b = threadIdx.x; b < kRedBlocks; b += blockDim.x) v = Op::op(v, partials[b]);
    v = block_reduce<Op>(v);
    if (threadIdx.x == 0) scalars[slot] = v;
}

}  // namespace

void finish_reduce(const double* partials, int op, double* scalars, int slot, cudaStream_t st) {
    if (op == 0) { launch_counter()++; k_finish<OpSum><<<1, 1024, 0, st>>>(partials, scalars, slot); }
    else if (op == 1) { launch_counter()++; k_finish<OpMin><<<1, 1024, 0, st>>>(partials, scalars, slot); }
    else { launch_counter()++; k_finish<OpMax><<<1, 1024, 0, st>>>(partials, scalars, slot); }
}

void launch_validate_grid(int cells, const double* rho, double* ps, double* pb, cudaStream_t st) {
    launch_counter()++;
    k_validate_grid<<<kRedBlocks, kRedThreads, 0, st>>>(cells, rho, ps, pb);
}

void launch_validate_particles(int64_t np, const double* pos, const double* mass, double* ps,
                               double* pb, cudaStream_t st) {
    launch_counter()++;
    k_validate_particles<<<kRedBlocks, kRedThreads, 0, st>>>(np, pos, mass, ps, pb);
}

void launch_deposit_particles(const Dims& d, int64_t np, const double* pos, const double* mass,
                              double inv_h, double scale, unsigned long long* mfix, cudaStream_t st) {
    if (np <= 0) return;
    launch_counter()++;
    k_deposit_particles<<<(unsigned)((np + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        d, np, pos, mass, inv_h, scale, mfix);
}

void launch_fix_to_double(int cells, unsigned long long* mfix, double inv_scale, double* out,
                          cudaStream_t st) {
    launch_counter()++;
    k_fix_to_double<<<nblocks(cells), kThreads, 0, st>>>(cells, mfix, inv_scale, out);
}

void launch_init_tracers(int cells, const double* rho, const double* sum_rho, double* w,
                         double* ox, double* oy, double* oz, double* phi, float* phi32,
                         cudaStream_t st) {
    launch_counter()++;
    k_init_tracers<<<nblocks(cells), kThreads, 0, st>>>(cells, rho, sum_rho, w, ox, oy, oz, phi,
                                                        phi32);
}

void launch_deposit_tracers(const Dims& d, const double* ox, const double* oy, const double* oz,
                            const double* w, double scale, unsigned long long* mfix,
                            cudaStream_t st) {
    launch_counter()++;
    if (d.n0 % DTI == 0 && d.n1 % DTJ == 0 && d.n2 % DTK == 0) {
        allow_smem((const void*)k_deposit_tracers_tiled, (int)kDepSmem);
        dim3 grid(d.n2 / DTK, d.n1 / DTJ, d.n0 / DTI);
        k_deposit_tracers_tiled<<<grid, 256, kDepSmem, st>>>(d, ox, oy, oz, w, scale, mfix);
        return;
    }
    k_deposit_tracers<<<nblocks(d.cells), kThreads, 0, st>>>(d, ox, oy, oz, w, scale, mfix);
}

void launch_mass_coef(int cells, unsigned long long* mfix, double inv_scale, double a_min,
                      double* m, double* a64, float* a32, double* partials, cudaStream_t st) {
    launch_counter()++;
    k_mass_coef<<<kRedBlocks, kRedThreads, 0, st>>>(cells, mfix, inv_scale, a_min, m, a64, a32,
                                                    partials);
}

void launch_geometry_source(const Dims& d, const SourceParams& sp, const double* phi,
                            const double* m, double* t, double* e6, double* part_sum,
                            double* part_min, cudaStream_t st) {
    launch_counter()++;
    k_geometry_source<<<kRedBlocks, kRedThreads, 0, st>>>(d, sp, phi, m, t, e6, part_sum, part_min);
}

void launch_smooth_S(const Dims& d, double s_side, const double* in, const double* shift_sum,
                     double* out, float* out32, double* tmp2, double* part_sum, double* part_sq,
                     cudaStream_t st) {
    if (d.n2 % SK == 0 && d.n1 % SJ == 0 && d.n0 % SCI == 0) {
        launch_counter()++;
        k_smooth_S_stream<<<kRedBlocks, 256, 0, st>>>(d, s_side, in, shift_sum, out, out32, part_sum,
                                                      part_sq);
        return;
    }
    launch_counter() += 3;
    k_smooth_axis<<<kRedBlocks, kRedThreads, 0, st>>>(d, 2, s_side, in, nullptr, tmp2, nullptr,
                                                      nullptr, nullptr);
    k_smooth_axis<<<kRedBlocks, kRedThreads, 0, st>>>(d, 1, s_side, tmp2, nullptr,
                                                      tmp2 + d.cells, nullptr, nullptr, nullptr);
    k_smooth_axis<<<kRedBlocks, kRedThreads, 0, st>>>(d, 0, s_side, tmp2 + d.cells, shift_sum,
                                                      out, out32, part_sum, part_sq);
}

void launch_limiter(const Dims& d, const LimiterParams& lp, const double* e6, const double* dphi,
                    const float* phi32, const float* dphi32, double* part_k, double* part_g,
                    cudaStream_t st) {
    launch_counter()++;
    k_limiter<<<kRedBlocks, kRedThreads, 0, st>>>(d, lp, e6, dphi, phi32, dphi32, part_k, part_g);
}

void launch_node_velocity(const Dims& d, const double* e6, const double* dphi, double* vx,
                          double* vy, double* vz, cudaStream_t st) {
    launch_counter()++;
    k_node_velocity<<<nblocks(d.cells), kThreads, 0, st>>>(d, e6, dphi, vx, vy, vz);
}

void launch_node_displacement(const Dims& d, const double* e6, const double* dphi, const double* alpha,
                              long long* dx, long long* dy, long long* dz, cudaStream_t st) {
    launch_counter()++;
    k_node_displacement<<<nblocks(d.cells), kThreads, 0, st>>>(d, e6, dphi, alpha, dx, dy, dz);
}

void launch_advance(const Dims& d, const long long* dx, const long long* dy, const long long* dz,
                    const double* alpha, const double* dphi, const double* sum_dphi, double* ox,
                    double* oy, double* oz, double* phi, float* phi32, cudaStream_t st) {
    launch_counter()++;
    k_advance<<<nblocks(d.cells), kThreads, 0, st>>>(d, dx, dy, dz, alpha, dphi, sum_dphi, ox, oy,
                                                     oz, phi, phi32);
}

void launch_mass_literal(const Dims& d, const double* e6, const double* dphi,
                         const double* alpha, double* m, double* K6, cudaStream_t st) {
    launch_counter() += 2;
    k_mass_tensor<<<nblocks(d.cells), kThreads, 0, st>>>(d, e6, m, K6);
    k_mass_update<<<nblocks(d.cells), kThreads, 0, st>>>(d, K6, dphi, alpha, m);
}

void launch_coef_from_m(int cells, const double* m, double a_min, double* a64, float* a32,
                        double* partials, cudaStream_t st) {
    launch_counter()++;
    k_coef_from_m<<<kRedBlocks, kRedThreads, 0, st>>>(cells, m, a_min, a64, a32, partials);
}

void launch_phi_advance(int cells, const double* alpha, const double* dphi,
                        const double* sum_dphi, double* phi, float* phi32, cudaStream_t st) {
    launch_counter()++;
    k_phi_advance<<<nblocks(cells), kThreads, 0, st>>>(cells, alpha, dphi, sum_dphi, phi, phi32);
}

void launch_delta_r(const Dims& d, const double* phi, double* out, double* part_max,
                    cudaStream_t st) {
    launch_counter()++;
    k_delta_r<<<kRedBlocks, kRedThreads, 0, st>>>(d, phi, out, part_max);
}

void launch_mesh_x(const Dims& d, const double* phi, double h, double* out, cudaStream_t st) {
    launch_counter()++;
    k_mesh_x<<<nblocks(d.cells), kThreads, 0, st>>>(d, phi, h, out);
}

void launch_geometry_out(const Dims& d, const double* phi, double* det, double* lam,
                         double* part_min_det, double* part_min_lam, cudaStream_t st) {
    launch_counter()++;
    k_geometry_out<<<kRedBlocks, kRedThreads, 0, st>>>(d, phi, det, lam, part_min_det, part_min_lam);
}

void launch_scale(int cells, const double* in, double s, double* out, cudaStream_t st) {
    launch_counter()++;
    k_scale<<<nblocks(cells), kThreads, 0, st>>>(cells, in, s, out);
}

int bounds_fail_steps() { return bounds_fail_take(); }

}  // namespace recon
