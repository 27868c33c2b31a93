// coarse_cluster.cu -- the coarse end of the V-cycle (App. A's multigrid)
// from a 32^3 level down, in one launch of one thread-block cluster.
//
// A level of 32^3 nodes is too large for one block's shared memory and too
// small to fill the GPU, so launching one kernel per phase (two colours per
// sweep, residual and restriction, prolongation) leaves it bound by launch
// gaps.  Here a cluster of kCR blocks holds the 32^3 and 16^3 levels in
// distributed shared memory, four (two) consecutive i-planes per block, and
// every phase ends with the cluster's hardware barrier.  A node
// whose i-neighbour lives in another block reads it from that block's shared
// memory (cluster.map_shared_rank).  Block 0 then gathers the 16^3 residual,
// runs the 8^3 and 4^3 levels alone (block barriers), and solves the 4^3
// level exactly with the stored inverse of the bordered system; the other
// blocks read the 8^3 correction back from it.  The per-node arithmetic is
// that of mg_stencil.cuh and the loop orders are those of the per-phase
// kernels (k_rbgs_colour, k_resid_restrict, k_prolong_add) and of the
// single-block coarse V-cycle, so the result is the same bit for bit.
#include <cooperative_groups.h>

#include "mg_stencil.cuh"
#include "recon_internal.cuh"

namespace cg = cooperative_groups;

namespace recon {

namespace {

constexpr int kCR = 8;      // blocks of the cluster (portable cluster size)
constexpr int kCT = 1024;   // threads per block
constexpr int kCN = 32;     // edge of the top level

// One level's four arrays (u, f, a, r) in a block's shared memory: the block
// holds global planes [rank P, rank P + P) of an n^3 level; planes are owned
// by block gi / P.
template <typename T>
struct CLev {
    T *u, *f, *a, *r;
    int n, lg, P;     // edge, log2 edge, planes per block
    T hx, hy, hz;
};

template <typename T>
__device__ inline T* plane_of(const CLev<T>& L, T* X, int gi, int self) {
    gi &= L.n - 1;
    const int owner = gi / L.P;
    T* base = owner == self ? X : cg::this_cluster().map_shared_rank(X, owner);
    return base + (gi - owner * L.P) * (L.n * L.n);
}

// One colour of a red-black sweep on the block's planes (colour: (i + j + k)
// parity; in-plane neighbours wrap periodically).
template <typename T>
__device__ void cl_sweep(const CLev<T>& L, int colour, int self) {
    const int n = L.n, nn = n * n, hn = n >> 1, m = n - 1;
    const int half = L.P * nn / 2;
    for (int t = threadIdx.x; t < half; t += blockDim.x) {
        const int lp = t / (nn / 2), rem = t - lp * (nn / 2);
        const int j = rem / hn, kk = rem - j * hn;
        const int gi = self * L.P + lp;
        const int k = 2 * kk + ((gi + j + colour) & 1);
        const int o = j * n + k, c = lp * nn + o;
        const T* up = plane_of(L, L.u, gi + 1, self);
        const T* um = plane_of(L, L.u, gi - 1, self);
        const T* ap = plane_of(L, L.a, gi + 1, self);
        const T* am = plane_of(L, L.a, gi - 1, self);
        const T* uc = L.u + lp * nn;
        const T* ac = L.a + lp * nn;
        const int yp = ((j + 1) & m) * n + k, ym = ((j - 1) & m) * n + k;
        const int zp = j * n + ((k + 1) & m), zm = j * n + ((k - 1) & m);
        const Stencil7<T> s = stencil7v<T>(L.hx, L.hy, L.hz, ac[o], ap[o], am[o], ac[yp], ac[ym], ac[zp], ac[zm],
                                           up[o], um[o], uc[yp], uc[ym], uc[zp], uc[zm]);
        L.u[c] = (s.off - L.f[c]) / s.diag;
    }
}

// r = f - L u on the block's planes.
template <typename T>
__device__ void cl_resid(const CLev<T>& L, int self) {
    const int n = L.n, nn = n * n, m = n - 1;
    for (int c = threadIdx.x; c < L.P * nn; c += blockDim.x) {
        const int lp = c / nn, o = c - lp * nn;
        const int j = o >> L.lg, k = o & m;
        const int gi = self * L.P + lp;
        const T* up = plane_of(L, L.u, gi + 1, self);
        const T* um = plane_of(L, L.u, gi - 1, self);
        const T* ap = plane_of(L, L.a, gi + 1, self);
        const T* am = plane_of(L, L.a, gi - 1, self);
        const T* uc = L.u + lp * nn;
        const T* ac = L.a + lp * nn;
        const int yp = ((j + 1) & m) * n + k, ym = ((j - 1) & m) * n + k;
        const int zp = j * n + ((k + 1) & m), zm = j * n + ((k - 1) & m);
        const Stencil7<T> s = stencil7v<T>(L.hx, L.hy, L.hz, ac[o], ap[o], am[o], ac[yp], ac[ym], ac[zp], ac[zm],
                                           up[o], um[o], uc[yp], uc[ym], uc[zp], uc[zm]);
        L.r[c] = L.f[c] - (s.off - s.diag * uc[o]);
    }
}

// Full weighting of the fine residual into the coarse right-hand side on the
// coarse planes the block holds (all of them when C.P == C.n); u = 0 there.
// self: the calling block (fine planes are read from whichever block holds
// them); C's planes start at plane cself * C.P.
template <typename T>
__device__ void cl_restrict(const CLev<T>& F, const CLev<T>& C, int self, int cself) {
    const int n = C.n, nn = n * n, m = n - 1, fn = F.n, fm = fn - 1;
    for (int c = threadIdx.x; c < C.P * nn; c += blockDim.x) {
        const int lp = c / nn, o = c - lp * nn;
        const int J = o >> C.lg, K = o & m;
        const int I = cself * C.P + lp;
        T acc = T(0);
        for (int oi = -1; oi <= 1; ++oi) {
            const T wi = oi == 0 ? T(0.5) : T(0.25);
            const T* rp = plane_of(F, F.r, 2 * I + oi, self);
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
template <typename T>
__device__ void cl_prolong(const CLev<T>& C, const CLev<T>& F, int self) {
    const int n = F.n, nn = n * n, m = n - 1, cn = C.n, cm = cn - 1;
    for (int c = threadIdx.x; c < F.P * nn; c += blockDim.x) {
        const int lp = c / nn, o = c - lp * nn;
        const int j = o >> F.lg, k = o & m;
        const int i = self * F.P + lp;
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
            const T* cp = plane_of(C, C.u, ii[p], self);
            for (int q = 0; q < nj; ++q)
                for (int r = 0; r < nk; ++r)
                    acc += wi[p] * wj[q] * wk[r] * cp[((jj[q] & cm) << C.lg) + (kk[r] & cm)];
        }
        F.u[c] += acc;
    }
}

// Levels: 0 = 32^3 and 1 = 16^3 spread over the cluster; 2 = 8^3 and
// 3 = 4^3 held by block 0 alone.
template <typename T>
__global__ void __cluster_dims__(kCR, 1, 1) __launch_bounds__(kCT)
    k_coarse_cluster(CoarseSet cs, const T* __restrict__ f_top, T* __restrict__ u_top,
                     const double* __restrict__ aug, int zero_u) {
    cg::cluster_group cluster = cg::this_cluster();
    const int self = (int)cluster.block_rank();
    extern __shared__ unsigned char smem_raw[];
    T* q = reinterpret_cast<T*>(smem_raw);
    CLev<T> L[4];
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const int n = kCN >> l;
        const int P = l == 0 ? n / kCR : (l == 1 ? n / kCR : n);
        const int sz = P * n * n;
        L[l].u = q, L[l].f = q + sz, L[l].a = q + 2 * sz, L[l].r = q + 3 * sz;
        q += 4 * sz;
        L[l].n = n, L[l].lg = 5 - l, L[l].P = P;
        L[l].hx = (T)cs.lv[l].h2i[0], L[l].hy = (T)cs.lv[l].h2i[1], L[l].hz = (T)cs.lv[l].h2i[2];
    }
    // the block's planes of a, f and u; block 0 also the whole 8^3 and 4^3 a
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        if (l >= 2 && self != 0) continue;
        const T* ag = reinterpret_cast<const T*>(cs.a[l]);
        const int base = (l >= 2 ? 0 : self * L[l].P) * L[l].n * L[l].n;
        for (int c = threadIdx.x; c < L[l].P * L[l].n * L[l].n; c += blockDim.x) L[l].a[c] = ag[base + c];
    }
    {
        const int base = self * L[0].P * kCN * kCN;
        for (int c = threadIdx.x; c < L[0].P * kCN * kCN; c += blockDim.x) {
            L[0].f[c] = f_top[base + c];
            L[0].u[c] = zero_u ? T(0) : u_top[base + c];
        }
    }
    cluster.sync();
    // down: the two distributed levels
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        for (int s = 0; s < cs.nu1; ++s)
            for (int colour = 0; colour < 2; ++colour) {
                cl_sweep<T>(L[l], colour, self);
                cluster.sync();
            }
        cl_resid<T>(L[l], self);
        cluster.sync();
        if (l == 0) {
            cl_restrict<T>(L[0], L[1], self, self);
            cluster.sync();
        }
    }
    // block 0: the 8^3 and 4^3 levels and the exact 4^3 solve
    if (self == 0) {
        cl_restrict<T>(L[1], L[2], 0, 0);
        __syncthreads();
        for (int s = 0; s < cs.nu1; ++s)
            for (int colour = 0; colour < 2; ++colour) {
                cl_sweep<T>(L[2], colour, 0);
                __syncthreads();
            }
        cl_resid<T>(L[2], 0);
        __syncthreads();
        cl_restrict<T>(L[2], L[3], 0, 0);
        __syncthreads();
        if (threadIdx.x < kNc) {
            double acc = 0.0;
            for (int c = 0; c < kNc; ++c) acc += aug[threadIdx.x * kW + kNb + c] * (double)L[3].f[c];
            L[3].u[threadIdx.x] = (T)acc;
        }
        __syncthreads();
        cl_prolong<T>(L[3], L[2], 0);
        __syncthreads();
        for (int s = 0; s < cs.nu2; ++s)
            for (int colour = 0; colour < 2; ++colour) {
                cl_sweep<T>(L[2], colour, 0);
                __syncthreads();
            }
    }
    cluster.sync();
    // up: the two distributed levels (the 8^3 field is read from block 0)
#pragma unroll
    for (int l = 1; l >= 0; --l) {
        cl_prolong<T>(L[l + 1], L[l], self);
        cluster.sync();
        for (int s = 0; s < cs.nu2; ++s)
            for (int colour = 0; colour < 2; ++colour) {
                cl_sweep<T>(L[l], colour, self);
                cluster.sync();
            }
    }
    {
        const int base = self * L[0].P * kCN * kCN;
        for (int c = threadIdx.x; c < L[0].P * kCN * kCN; c += blockDim.x) u_top[base + c] = L[0].u[c];
    }
}

template <typename T>
constexpr int cluster_smem() {
    int floats = 0;
    for (int l = 0; l < 4; ++l) {
        const int n = kCN >> l;
        const int P = l <= 1 ? n / kCR : n;
        floats += 4 * P * n * n;
    }
    return floats * (int)sizeof(T);
}

}  // namespace

bool coarse_cluster_fits(const CoarseSet& cs) {
    if (cs.nlev != 4) return false;
    for (int l = 0; l < 4; ++l) {
        const Dims& d = cs.lv[l].d;
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
    constexpr int smem = cluster_smem<T>();
    allow_smem((const void*)k_coarse_cluster<T>, smem);
    launch_counter()++;
    k_coarse_cluster<T><<<kCR, kCT, smem, st>>>(cs, f, u, minv, zero_u ? 1 : 0);
    return true;
}

template bool launch_coarse_cluster<float>(const CoarseSet&, const float*, float*, const double*, bool,
                                           cudaStream_t);
template bool launch_coarse_cluster<double>(const CoarseSet&, const double*, double*, const double*, bool,
                                            cudaStream_t);

}  // namespace recon
