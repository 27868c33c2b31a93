// coarse_cluster.cu -- the coarse end of the V-cycle (App. A's multigrid)
// from a 32^3 level down, in one launch of one thread-block cluster.
//
// A level of 32^3 nodes is too large for one block's shared memory and too
// small to fill the GPU, so launching one kernel per phase (two colours per
// sweep, residual and restriction, prolongation) leaves it bound by launch
// gaps.  Here a cluster of kCR blocks holds the 32^3 and 16^3 levels in
// distributed shared memory, four (two) consecutive i-planes per block, and
// every phase ends with the cluster's hardware barrier.  A node whose
// i-neighbour lives in another block reads it from that block's shared memory
// (cluster.map_shared_rank).  Block 0 then gathers the 16^3 residual,
// runs the 8^3 and 4^3 levels alone (block barriers), and solves the 4^3
// level exactly with the stored inverse of the bordered system; the other
// blocks read the 8^3 correction back from it.  The per-node arithmetic is
// that of mg_stencil.cuh and the loop orders are those of the per-phase
// kernels (k_rbgs_colour, k_resid_restrict, k_prolong_add) and of the
// single-block coarse V-cycle, so the result is the same bit for bit.  With
// coarse levels given by face sums (Level::face) the same phases read the
// x face sums where they read a, and the y and z sums of their own planes.
#include <cooperative_groups.h>

#include "checked.cuh"
#include "mg_stencil.cuh"
#include "recon_internal.cuh"

namespace cg = cooperative_groups;

namespace recon {

namespace {

constexpr int kCR = 8;      // blocks of the cluster (portable cluster size)
constexpr int kCT = 1024;   // threads per block
constexpr int kCN = 32;     // edge of the top level

// One level's four arrays (u, f, a, r) in a block's shared memory.  The
// level functions take its edge N and planes per block P as template
// arguments: the block holds global planes [rank P, rank P + P) of the N^3
// level, and plane gi is owned by block gi / P.
template <typename T>
struct CLev {
    T *u, *f, *a, *r;
    T *gy, *gz;  // face-sum levels: a holds the x face sums, these the y and z ones
    T hx, hy, hz;
};

// Plane gi (periodic) of array X of an N^3 level: this block's own shared
// memory, or the owner's through the cluster's distributed shared memory.
template <typename T, int N, int P>
__device__ inline T* plane_of(T* X, int gi, int self) {
    gi &= N - 1;
    const int owner = RC_OFF(gi / P, kCR, 301);  // a block of the cluster
    T* base = owner == self ? X : cg::this_cluster().map_shared_rank(X, owner);
    return base + (gi - owner * P) * (N * N);
}

// One colour of a red-black sweep on the block's planes (colour: (i + j + k)
// parity; in-plane neighbours wrap periodically).
template <typename T, int N, int P, bool FACE>
__device__ void cl_sweep(const CLev<T>& L, int colour, int self) {
    constexpr int n = N, nn = n * n, hn = n >> 1, m = n - 1;
    constexpr int half = P * nn / 2;
    for (int t = threadIdx.x; t < half; t += blockDim.x) {
        const int lp = t / (nn / 2), rem = t - lp * (nn / 2);
        const int j = rem / hn, kk = rem - j * hn;
        const int gi = self * P + lp;
        const int k = 2 * kk + ((gi + j + colour) & 1);
        const int o = j * n + k, c = lp * nn + o;
        const T* up = plane_of<T, N, P>(L.u, gi + 1, self);
        const T* um = plane_of<T, N, P>(L.u, gi - 1, self);
        const T* ap = plane_of<T, N, P>(L.a, gi + 1, self);
        const T* am = plane_of<T, N, P>(L.a, gi - 1, self);
        const T* uc = L.u + lp * nn;
        const T* ac = L.a + lp * nn;
        const int yp = ((j + 1) & m) * n + k, ym = ((j - 1) & m) * n + k;
        const int zp = j * n + ((k + 1) & m), zm = j * n + ((k - 1) & m);
        Stencil7<T> s;
        if constexpr (FACE) {
            const T* gy = L.gy + lp * nn;
            const T* gz = L.gz + lp * nn;
            s = stencil7g<T>(L.hx, L.hy, L.hz, ac[o], am[o], gy[o], gy[ym], gz[o], gz[zm], up[o], um[o],
                             uc[yp], uc[ym], uc[zp], uc[zm]);
        } else {
            s = stencil7v<T>(L.hx, L.hy, L.hz, ac[o], ap[o], am[o], ac[yp], ac[ym], ac[zp], ac[zm], up[o], um[o],
                             uc[yp], uc[ym], uc[zp], uc[zm]);
        }
        L.u[c] = (s.off - L.f[c]) / s.diag;
    }
}

// r = f - L u on the block's planes.
template <typename T, int N, int P, bool FACE>
__device__ void cl_resid(const CLev<T>& L, int self) {
    constexpr int n = N, nn = n * n, m = n - 1;
    for (int c = threadIdx.x; c < P * nn; c += blockDim.x) {
        const int lp = c / nn, o = c - lp * nn;
        const int j = o / n, k = o & m;
        const int gi = self * P + lp;
        const T* up = plane_of<T, N, P>(L.u, gi + 1, self);
        const T* um = plane_of<T, N, P>(L.u, gi - 1, self);
        const T* ap = plane_of<T, N, P>(L.a, gi + 1, self);
        const T* am = plane_of<T, N, P>(L.a, gi - 1, self);
        const T* uc = L.u + lp * nn;
        const T* ac = L.a + lp * nn;
        const int yp = ((j + 1) & m) * n + k, ym = ((j - 1) & m) * n + k;
        const int zp = j * n + ((k + 1) & m), zm = j * n + ((k - 1) & m);
        Stencil7<T> s;
        if constexpr (FACE) {
            const T* gy = L.gy + lp * nn;
            const T* gz = L.gz + lp * nn;
            s = stencil7g<T>(L.hx, L.hy, L.hz, ac[o], am[o], gy[o], gy[ym], gz[o], gz[zm], up[o], um[o],
                             uc[yp], uc[ym], uc[zp], uc[zm]);
        } else {
            s = stencil7v<T>(L.hx, L.hy, L.hz, ac[o], ap[o], am[o], ac[yp], ac[ym], ac[zp], ac[zm], up[o], um[o],
                             uc[yp], uc[ym], uc[zp], uc[zm]);
        }
        L.r[c] = L.f[c] - (s.off - s.diag * uc[o]);
    }
}

// Full weighting of the fine residual into the coarse right-hand side on the
// coarse planes the block holds (all of them when PC == NC); u = 0 there.
// self: the calling block (fine planes are read from whichever block holds
// them); the coarse planes start at plane cself * PC.
template <typename T, int NF, int PF, int NC, int PC>
__device__ void cl_restrict(const CLev<T>& F, const CLev<T>& C, int self, int cself) {
    constexpr int n = NC, nn = n * n, m = n - 1, fn = NF, fm = fn - 1;
    for (int c = threadIdx.x; c < PC * nn; c += blockDim.x) {
        const int lp = c / nn, o = c - lp * nn;
        const int J = o / n, K = o & m;
        const int I = cself * PC + lp;
        T acc = T(0);
        for (int oi = -1; oi <= 1; ++oi) {
            const T wi = oi == 0 ? T(0.5) : T(0.25);
            const T* rp = plane_of<T, NF, PF>(F.r, 2 * I + oi, self);
            for (int oj = -1; oj <= 1; ++oj) {
                const T wj = oj == 0 ? T(0.5) : T(0.25);
                const int row = ((2 * J + oj) & fm) * fn;
                for (int ok = -1; ok <= 1; ++ok) {
                    const T wk = ok == 0 ? T(0.5) : T(0.25);
                    acc += wi * wj * wk * rp[row + ((2 * K + ok) & fm)];
                }
            }
        }
        C.f[c] = acc;
        C.u[c] = T(0);
    }
}

// Trilinear prolongation of the coarse field, added on the fine planes the
// block holds (coarse planes are read from whichever block holds them).
template <typename T, int NC, int PC, int NF, int PF>
__device__ void cl_prolong(const CLev<T>& C, const CLev<T>& F, int self) {
    constexpr int n = NF, nn = n * n, m = n - 1, cn = NC, cm = cn - 1;
    for (int c = threadIdx.x; c < PF * nn; c += blockDim.x) {
        const int lp = c / nn, o = c - lp * nn;
        const int j = o / n, k = o & m;
        const int i = self * PF + lp;
        int ii[2], jj[2], kk[2];
        T wi[2], wj[2], wk[2];
        int ni, nj, nk;
        if (!(i & 1)) { ii[0] = i >> 1; wi[0] = T(1); ni = 1; }
        else { ii[0] = i >> 1; ii[1] = (i >> 1) + 1; wi[0] = wi[1] = T(0.5); ni = 2; }
        if (!(j & 1)) { jj[0] = j >> 1; wj[0] = T(1); nj = 1; }
        else { jj[0] = j >> 1; jj[1] = (j >> 1) + 1; wj[0] = wj[1] = T(0.5); nj = 2; }
        if (!(k & 1)) { kk[0] = k >> 1; wk[0] = T(1); nk = 1; }
        else { kk[0] = k >> 1; kk[1] = (k >> 1) + 1; wk[0] = wk[1] = T(0.5); nk = 2; }
        T acc = T(0);
        for (int p = 0; p < ni; ++p) {
            const T* cp = plane_of<T, NC, PC>(C.u, ii[p], self);
            for (int q = 0; q < nj; ++q)
                for (int r = 0; r < nk; ++r)
                    acc += wi[p] * wj[q] * wk[r] * cp[(jj[q] & cm) * cn + (kk[r] & cm)];
        }
        F.u[c] += acc;
    }
}

// Levels: 0 = 32^3 and 1 = 16^3 spread over the cluster; 2 = 8^3 and
// 3 = 4^3 held by block 0 alone.
constexpr int N0 = kCN, P0 = N0 / kCR, N1 = kCN / 2, P1 = N1 / kCR, N2 = kCN / 4, P2 = N2,
              N3 = kCN / 8, P3 = N3;
static_assert(P0 >= 1 && P1 >= 1 && N3 * N3 * N3 == kNc, "level split");

template <typename T, bool FACE>
__global__ void __cluster_dims__(kCR, 1, 1) __launch_bounds__(kCT)
    k_coarse_cluster(CoarseSet cs, const T* __restrict__ f_top, T* __restrict__ u_top,
                     const double* __restrict__ aug, int zero_u) {
    cg::cluster_group cluster = cg::this_cluster();
    const int self = (int)cluster.block_rank();
    extern __shared__ unsigned char smem_raw[];
    T* q = reinterpret_cast<T*>(smem_raw);
    CLev<T> L[4];
    const int sz[4] = {P0 * N0 * N0, P1 * N1 * N1, P2 * N2 * N2, P3 * N3 * N3};
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        L[l].u = q, L[l].f = q + sz[l], L[l].a = q + 2 * sz[l], L[l].r = q + 3 * sz[l];
        q += 4 * sz[l];
        if (FACE) {
            L[l].gy = q, L[l].gz = q + sz[l];
            q += 2 * sz[l];
        }
        L[l].hx = (T)cs.lv[l].h2i[0], L[l].hy = (T)cs.lv[l].h2i[1], L[l].hz = (T)cs.lv[l].h2i[2];
    }
    // the block's planes of a (or of the three face sums), f and u; block 0
    // also the whole 8^3 and 4^3 coefficients
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if (l >= 2 && self != 0) continue;
        const T* ag = reinterpret_cast<const T*>(cs.a[l]);
        const int base = l >= 2 ? 0 : self * sz[l];
        for (int c = threadIdx.x; c < sz[l]; c += blockDim.x) L[l].a[c] = ag[base + c];
        if (FACE) {
            const int cells = cs.lv[l].d.cells;
            for (int c = threadIdx.x; c < sz[l]; c += blockDim.x) {
                L[l].gy[c] = ag[cells + base + c];
                L[l].gz[c] = ag[2 * cells + base + c];
            }
        }
    }
    for (int c = threadIdx.x; c < sz[0]; c += blockDim.x) {
        L[0].f[c] = f_top[self * sz[0] + c];
        L[0].u[c] = zero_u ? T(0) : u_top[self * sz[0] + c];
    }
    // block 0: the 4^3 inverse (its kNc x kNc block of the augmented matrix),
    // read once here so that the exact solve later runs from shared memory
    double* minv = reinterpret_cast<double*>(q);
    if (self == 0)
        for (int e = threadIdx.x; e < kNc * kNc; e += blockDim.x)
            minv[e] = aug[(e / kNc) * kW + kNb + (e % kNc)];
    cluster.sync();
    // down: the two distributed levels
    for (int s = 0; s < cs.nu1; ++s)
        for (int colour = 0; colour < 2; ++colour) {
            cl_sweep<T, N0, P0, FACE>(L[0], colour, self);
            cluster.sync();
        }
    cl_resid<T, N0, P0, FACE>(L[0], self);
    cluster.sync();
    cl_restrict<T, N0, P0, N1, P1>(L[0], L[1], self, self);
    cluster.sync();
    for (int s = 0; s < cs.nu1; ++s)
        for (int colour = 0; colour < 2; ++colour) {
            cl_sweep<T, N1, P1, FACE>(L[1], colour, self);
            cluster.sync();
        }
    cl_resid<T, N1, P1, FACE>(L[1], self);
    cluster.sync();
    // block 0: the 8^3 and 4^3 levels and the exact 4^3 solve
    if (self == 0) {
        cl_restrict<T, N1, P1, N2, P2>(L[1], L[2], 0, 0);
        __syncthreads();
        for (int s = 0; s < cs.nu1; ++s)
            for (int colour = 0; colour < 2; ++colour) {
                cl_sweep<T, N2, P2, FACE>(L[2], colour, 0);
                __syncthreads();
            }
        cl_resid<T, N2, P2, FACE>(L[2], 0);
        __syncthreads();
        cl_restrict<T, N2, P2, N3, P3>(L[2], L[3], 0, 0);
        __syncthreads();
        if (threadIdx.x < kNc) {
            double acc = 0.0;
            for (int c = 0; c < kNc; ++c) acc += minv[threadIdx.x * kNc + c] * (double)L[3].f[c];
            L[3].u[threadIdx.x] = (T)acc;
        }
        __syncthreads();
        cl_prolong<T, N3, P3, N2, P2>(L[3], L[2], 0);
        __syncthreads();
        for (int s = 0; s < cs.nu2; ++s)
            for (int colour = 0; colour < 2; ++colour) {
                cl_sweep<T, N2, P2, FACE>(L[2], colour, 0);
                __syncthreads();
            }
    }
    cluster.sync();
    // up: the two distributed levels (the 8^3 field is read from block 0)
    cl_prolong<T, N2, P2, N1, P1>(L[2], L[1], self);
    cluster.sync();
    for (int s = 0; s < cs.nu2; ++s)
        for (int colour = 0; colour < 2; ++colour) {
            cl_sweep<T, N1, P1, FACE>(L[1], colour, self);
            cluster.sync();
        }
    cl_prolong<T, N1, P1, N0, P0>(L[1], L[0], self);
    cluster.sync();
    for (int s = 0; s < cs.nu2; ++s)
        for (int colour = 0; colour < 2; ++colour) {
            cl_sweep<T, N0, P0, FACE>(L[0], colour, self);
            cluster.sync();
        }
    for (int c = threadIdx.x; c < sz[0]; c += blockDim.x) u_top[self * sz[0] + c] = L[0].u[c];
}

template <typename T, bool FACE>
constexpr int cluster_smem() {
    // the four levels' arrays (u, f, r and a or the three face sums), then the
    // 4^3 inverse (8-byte aligned: every level's arrays are a multiple of 8
    // bytes long)
    return (FACE ? 6 : 4) * (P0 * N0 * N0 + P1 * N1 * N1 + P2 * N2 * N2 + P3 * N3 * N3) * (int)sizeof(T) +
           kNc * kNc * (int)sizeof(double);
}

}  // namespace

bool coarse_cluster_fits(const CoarseSet& cs) {
    if (cs.nlev != 4) return false;
    for (int l = 0; l < 4; ++l) {
        const Dims& d = cs.lv[l].d;
        if (cs.lv[l].face != cs.lv[0].face) return false;  // one form for the whole set
        const int n = kCN >> l;
        if (d.n0 != n || d.n1 != n || d.n2 != n) return false;
        if (l < 3 && !(cs.lv[l].coarsen[0] && cs.lv[l].coarsen[1] && cs.lv[l].coarsen[2])) return false;
    }
    return true;
}

template <typename T>
bool launch_coarse_cluster(const CoarseSet& cs, const T* f, T* u, const double* minv, bool zero_u,
                           cudaStream_t st) {
    if (!coarse_cluster_fits(cs)) return false;
    launch_counter()++;
    if constexpr (sizeof(T) == sizeof(float)) {
        if (cs.lv[0].face) {
            constexpr int smem = cluster_smem<T, true>();
            allow_smem((const void*)k_coarse_cluster<T, true>, smem);
            k_coarse_cluster<T, true><<<kCR, kCT, smem, st>>>(cs, f, u, minv, zero_u ? 1 : 0);
            return true;
        }
    }
    constexpr int smem = cluster_smem<T, false>();
    allow_smem((const void*)k_coarse_cluster<T, false>, smem);
    k_coarse_cluster<T, false><<<kCR, kCT, smem, st>>>(cs, f, u, minv, zero_u ? 1 : 0);
    return true;
}

template bool launch_coarse_cluster<float>(const CoarseSet&, const float*, float*, const double*, bool,
                                           cudaStream_t);
template bool launch_coarse_cluster<double>(const CoarseSet&, const double*, double*, const double*, bool,
                                            cudaStream_t);

int bounds_fail_cluster() { return bounds_fail_take(); }

}  // namespace recon
