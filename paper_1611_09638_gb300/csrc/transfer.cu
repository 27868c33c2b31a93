// transfer.cu -- residual and full-weighting restriction of an FP32 level in
// one streaming pass (App. A's multigrid: the coarse right-hand side of a
// V-cycle is R (f - L u), with L the 7-point variable-coefficient operator
// with face coefficients (a + a_nbr)/2 and R the tensor (1/4, 1/2, 1/4)
// weighting on the fine nodes 2I-1, 2I, 2I+1 of each axis).
//
// The per-coarse-node kernel in mg_kernels.cu evaluates the 27 fine residuals
// of each coarse node's stencil, so every fine residual is computed 27/8
// times.  Here a block owns a 8 x 32 tile of the coarse (J, K) plane, i.e. a
// 16 x 64 tile of the fine plane, and streams fine planes along i.  Each
// thread owns one coarse node and the 2 x 2 fine columns (2J, 2J+1) x (2K,
// 2K+1) under it for the whole stream: u and a of its columns for planes
// p - 1 .. p + 1 and f of plane p are carried in registers (one 8-byte shared
// load per row and plane), so the residual of its four nodes reads from
// shared memory only the rows above and below (8-byte loads) and takes the
// columns left and right from the neighbouring lanes by warp shuffles.  The
// block's low-side ring of residuals (row -1 and column -1, 81 nodes) is
// computed from shared memory by three warps.  Every thread stores the
// residuals of its lower fine row; after the plane's barrier the next
// iteration weights plane p in j and k (the row above from shared memory,
// the column to the left by shuffles) and applies the i weights in registers
// (an odd plane 2I+1 closes coarse plane I and opens I+1).  The residuals
// alternate between two buffers, so one block-wide barrier per plane
// suffices.  u and a are held for four planes (p-1 .. p+1 and the one being
// fetched), f for two; each plane is fetched with 16-byte cp.async copies.
// DRAM traffic is one read of u, a, f and one write of the coarse plane.
#include "async_copy.cuh"
#include "checked.cuh"
#include "recon_internal.cuh"

namespace recon {

namespace {

constexpr int RT = 256;                 // threads: one per coarse node of the tile
constexpr int FJ = 16, FK = 64;         // fine tile rows (j) and columns (k)
constexpr int RH = 2, RKO = 4;          // halo rows / columns held
constexpr int RRJ = FJ + 2 * RH;        // 20 rows per plane
constexpr int RRK = FK + 2 * RKO;       // 72 columns per plane
constexpr int RPL = RRJ * RRK;          // floats per plane
constexpr int RCH = RRK / 4;            // 16-byte chunks per row
constexpr int NUA = RRJ * RCH;          // chunks of a u (or a) plane: 360
constexpr int NFC = (FJ + 1) * RCH;     // chunks of an f plane (rows -1 .. FJ-1): 306
constexpr int NRING = (FK + 1) + FJ;    // low-side ring residuals: row -1 and column -1: 81
constexpr int SUA = 4, SFF = 2;         // ring slots of u / a and of f
constexpr int RSMEM = (int)sizeof(float) * RPL * (2 * SUA + SFF + 2);
// FACE: also the y and z face sums of a plane, two slots each (read for the
// residual plane only)
constexpr int RSMEM_FACE = RSMEM + (int)sizeof(float) * RPL * 2 * SFF;
static_assert(NUA <= 2 * RT && NFC <= 2 * RT && NRING <= RT, "fetch rounds");
static_assert((FJ / 2) * (FK / 2) == RT && FK / 2 == 32, "one coarse node per thread, a coarse row per warp");

// The residual f - L u at a node from its coefficient c, the neighbours'
// coefficients and values (x: i, y: j, z: k; p: +1, m: -1), u at the node
// and f.  ISO: one spacing on every axis; hx then holds hh = h^-2 / 2,
// applied once to the sums of the face sums c + a_n (see k_rbgs_stream).
template <bool ISO>
__device__ __forceinline__ float resid_node(float c, float apx, float amx, float apy, float amy, float apz,
                                            float amz, float upx, float umx, float upy, float umy,
                                            float upz, float umz, float uc, float f, float hx, float hy,
                                            float hz) {
    if (ISO) {
        const float px = c + apx, mx = c + amx, py = c + apy, my = c + amy, pz = c + apz, mz = c + amz;
        const float diag = (px + mx) + (py + my) + (pz + mz);
        const float off = (px * upx + mx * umx) + (py * upy + my * umy) + (pz * upz + mz * umz);
        return fmaf(-hx, fmaf(-diag, uc, off), f);
    }
    const float px = 0.5f * (c + apx) * hx, mx = 0.5f * (c + amx) * hx;
    const float py = 0.5f * (c + apy) * hy, my = 0.5f * (c + amy) * hy;
    const float pz = 0.5f * (c + apz) * hz, mz = 0.5f * (c + amz) * hz;
    const float diag = (px + mx) + (py + my) + (pz + mz);
    const float off = (px * upx + mx * umx) + (py * upy + my * umy) + (pz * upz + mz * umz);
    return f - (off - diag * uc);
}

// The residual of an isotropic level given by face sums G of the node's six
// faces (hx holds hh, as in resid_node).
__device__ __forceinline__ float resid_face(float gpx, float gmx, float gpy, float gmy, float gpz, float gmz,
                                            float upx, float umx, float upy, float umy, float upz,
                                            float umz, float uc, float f, float hx) {
    const float diag = (gpx + gmx) + (gpy + gmy) + (gpz + gmz);
    const float off = (gpx * upx + gmx * umx) + (gpy * upy + gmy * umy) + (gpz * upz + gmz * umz);
    return fmaf(-hx, fmaf(-diag, uc, off), f);
}

// FACE: the fine level is given by face sums (a points at its x, y and z
// face-sum arrays): the x sums ride in the registers that hold a, the y and z
// sums of the residual plane come from shared memory.
template <bool ISO, int CIc, bool FACE>
__global__ void __launch_bounds__(RT) k_resid_restrict_stream(Dims df, Dims dc, float hx, float hy,
                                                              float hz,
                                                              const float* __restrict__ u,
                                                              const float* __restrict__ f,
                                                              const float* __restrict__ a,
                                                              float* __restrict__ out) {
    extern __shared__ float4 smem_f4[];
    float* su = reinterpret_cast<float*>(smem_f4);
    float* sa = su + SUA * RPL;
    float* sf = sa + SUA * RPL;
    float* sr = sf + SFF * RPL;  // two residual planes
    float* sy = sr + 2 * RPL;    // FACE: y and z face sums
    float* sz = sy + SFF * RPL;
    static_assert(!FACE || ISO, "face sums: isotropic levels");
    const float* gyg = FACE ? a + df.cells : nullptr;
    const float* gzg = FACE ? a + 2 * (size_t)df.cells : nullptr;
    const int t = threadIdx.x;
    const int K0c = blockIdx.x * (FK / 2), J0c = blockIdx.y * (FJ / 2), I0c = blockIdx.z * CIc;
    const int k0 = 2 * K0c, j0 = 2 * J0c;
    const int pS = 2 * I0c - 1;  // first residual plane of the block (odd)
    const int plane = df.n1 * df.n2;

    // ---- offsets fixed for the whole block -------------------------------
    // smem offset of fine (row jj, column kk) relative to the tile origin is
    // (jj + RH) * RRK + kk + RKO, the same in every plane buffer.
    int ua_s[2], ua_g[2], f_s[2], f_g[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int e = t + m * RT;
        const int r = e / RCH, ch = e - r * RCH;
        const int gk = (k0 - RKO + ch * 4) & (df.n2 - 1);
        // (RC_OFF: checked against the extent in the RECON_CHECKED build)
        ua_s[m] = e < NUA ? RC_OFF(r * RRK + ch * 4, RPL - 3, 201) : -1;
        ua_g[m] = RC_OFF((((j0 + r - RH) & (df.n1 - 1)) << df.s2) + gk, plane - 3, 202);
        f_s[m] = e < NFC ? RC_OFF((r + 1) * RRK + ch * 4, RPL - 3, 203) : -1;  // fine row r - 1
        f_g[m] = RC_OFF((((j0 + r - 1) & (df.n1 - 1)) << df.s2) + gk, plane - 3, 204);
    }
    // warp jc = coarse row, lane kc = coarse column: fine rows 2 jc, 2 jc + 1
    // (offsets e0, e1 of the column pair 2 kc, 2 kc + 1)
    const int jc = t >> 5, kc = t & 31;
    // every read around the quad lies in [e0 - RRK - 1, e1 + RRK + 2)
    const int e0 = RRK + 1 + RC_OFF((2 * jc + RH) * RRK + 2 * kc + RKO - RRK - 1, RPL - 3 * RRK - 2, 205);
    const int e1 = e0 + RRK;
    const int out_o = RC_OFF(((J0c + jc) << dc.s2) + K0c + kc, dc.n1 * dc.n2, 206);
    // ring residual of thread t < NRING: row -1 (columns -1 .. FK-1) or
    // column -1 (rows 0 .. FJ-1)
    int ring_e = t < FK + 1 ? (RH - 1) * RRK + RKO + t - 1
                            : (t < NRING ? (t - (FK + 1) + RH) * RRK + RKO - 1 : -1);
    if (ring_e >= 0) ring_e = RRK + RC_OFF(ring_e - RRK, RPL - 2 * RRK, 207);  // with rows +- 1

    // Plane p is held in u / a slot (p - pS + 1) mod SUA and f slot
    // (p - pS) mod SFF; the plane loop is unrolled (p = pS + it), so every
    // slot offset and register index is a compile-time constant.
    auto gplane = [&](int p) { return (p & (df.n0 - 1)) * plane; };
    auto fetch_ua = [&](int p, int so) {
        const int g = gplane(p);
#pragma unroll
        for (int m = 0; m < 2; ++m)
            if (ua_s[m] >= 0) {
                cp_async16(su + so + ua_s[m], u + g + ua_g[m]);
                cp_async16(sa + so + ua_s[m], a + g + ua_g[m]);
            }
    };
    auto fetch_f = [&](int p, int so) {
        const int g = gplane(p);
#pragma unroll
        for (int m = 0; m < 2; ++m)
            if (f_s[m] >= 0) cp_async16(sf + so + f_s[m], f + g + f_g[m]);
        if (FACE) {
#pragma unroll
            for (int m = 0; m < 2; ++m)
                if (ua_s[m] >= 0) {
                    cp_async16(sy + so + ua_s[m], gyg + g + ua_g[m]);
                    cp_async16(sz + so + ua_s[m], gzg + g + ua_g[m]);
                }
        }
    };
    auto ld2 = [](const float* p) { return *reinterpret_cast<const float2*>(p); };
    const unsigned full = 0xffffffffu;

    // U, A: the thread's u and a (rows 0 and 1 of its quad) for plane x at
    // index (x - pS + 1) & 3; Rp: its residuals of the previous plane.
    float2 U[4][2], A[4][2];
    float Rp[4] = {0.f, 0.f, 0.f, 0.f};

    fetch_ua(pS - 1, 0 * RPL);
    fetch_ua(pS, 1 * RPL);
    fetch_ua(pS + 1, 2 * RPL);
    fetch_f(pS, 0 * RPL);
    cp_commit();
    cp_wait_all();
    __syncthreads();
#pragma unroll
    for (int x = 0; x < 2; ++x) {
        U[x][0] = ld2(su + x * RPL + e0), U[x][1] = ld2(su + x * RPL + e1);
        A[x][0] = ld2(sa + x * RPL + e0), A[x][1] = ld2(sa + x * RPL + e1);
    }

    float acc = 0.f;
#pragma unroll
    for (int it = 0; it <= 2 * CIc + 1; ++it) {
        const int p = pS + it;
        if (it < 2 * CIc) {
            fetch_ua(p + 2, ((it + 3) % SUA) * RPL);
            fetch_f(p + 1, ((it + 1) % SFF) * RPL);
        }
        cp_commit();
        // (1/4, 1/2, 1/4) weights in j and k around fine node (2 jc, 2 kc) of
        // plane p - 1, whose residuals were stored before the last barrier
        if (it >= 1) {
            const float* rb = sr + ((it - 1) & 1) * RPL;
            const float2 up = ld2(rb + e0 - RRK);  // row 2 jc - 1
            float la = __shfl_up_sync(full, up.y, 1);
            float l0 = __shfl_up_sync(full, Rp[1], 1), l1 = __shfl_up_sync(full, Rp[3], 1);
            if (kc == 0) la = rb[e0 - RRK - 1], l0 = rb[e0 - 1], l1 = rb[e1 - 1];
            const float s = 0.25f * (0.25f * la + 0.5f * up.x + 0.25f * up.y) +
                            0.5f * (0.25f * l0 + 0.5f * Rp[0] + 0.25f * Rp[1]) +
                            0.25f * (0.25f * l1 + 0.5f * Rp[2] + 0.25f * Rp[3]);
            if ((it - 1) & 1) {
                acc += 0.5f * s;
            } else {  // p - 1 = 2I + 1 (odd) closes coarse plane I and opens I + 1
                if (it > 1)
                    out[RC_OFF(((I0c - 1 + ((it - 1) >> 1)) << (dc.s1 + dc.s2)) + out_o, dc.cells, 208)] =
                        acc + 0.25f * s;
                acc = 0.25f * s;
            }
        }
        if (it == 2 * CIc + 1) break;
        // residual r = f - L u of plane p at the thread's four nodes
        const int iq = (it + 1) & 3, im1 = it & 3, ip1 = (it + 2) & 3;
        const int cu = ((it + 1) % SUA) * RPL, mu = (it % SUA) * RPL;
        const int pu = ((it + 2) % SUA) * RPL, cf = (it % SFF) * RPL;
        U[ip1][0] = ld2(su + pu + e0), U[ip1][1] = ld2(su + pu + e1);
        A[ip1][0] = ld2(sa + pu + e0), A[ip1][1] = ld2(sa + pu + e1);
        const float2 f0 = ld2(sf + cf + e0), f1 = ld2(sf + cf + e1);
        const float2 ua = ld2(su + cu + e0 - RRK), ub = ld2(su + cu + e1 + RRK);  // rows 2jc-1, 2jc+2
        const float2 aa = ld2(sa + cu + e0 - RRK), ab = ld2(sa + cu + e1 + RRK);
        const float2 u0 = U[iq][0], u1 = U[iq][1], a0 = A[iq][0], a1 = A[iq][1];
        // columns 2 kc - 1 and 2 kc + 2 from the neighbouring lanes (the tile's
        // edge columns from shared memory)
        float ul0 = __shfl_up_sync(full, u0.y, 1), ul1 = __shfl_up_sync(full, u1.y, 1);
        float al0 = __shfl_up_sync(full, a0.y, 1), al1 = __shfl_up_sync(full, a1.y, 1);
        float ur0 = __shfl_down_sync(full, u0.x, 1), ur1 = __shfl_down_sync(full, u1.x, 1);
        float ar0 = __shfl_down_sync(full, a0.x, 1), ar1 = __shfl_down_sync(full, a1.x, 1);
        if (kc == 0) {
            ul0 = su[cu + e0 - 1], ul1 = su[cu + e1 - 1];
            al0 = sa[cu + e0 - 1], al1 = sa[cu + e1 - 1];
        }
        if (kc == 31) {
            ur0 = su[cu + e0 + 2], ur1 = su[cu + e1 + 2];
            ar0 = sa[cu + e0 + 2], ar1 = sa[cu + e1 + 2];
        }
        const float2 up0 = U[ip1][0], up1 = U[ip1][1], um0 = U[im1][0], um1 = U[im1][1];
        const float2 ap0 = A[ip1][0], ap1 = A[ip1][1], am0 = A[im1][0], am1 = A[im1][1];
        float r00, r01, r10, r11;
        if constexpr (FACE) {
            // x sums: a0/a1 (plane p), am0/am1 (plane p - 1); y sums of rows
            // 2jc - 1 .. 2jc + 1 and z sums of columns 2kc - 1 .. 2kc + 1
            const float2 gym = ld2(sy + cf + e0 - RRK), gy0 = ld2(sy + cf + e0), gy1 = ld2(sy + cf + e1);
            const float2 gz0 = ld2(sz + cf + e0), gz1 = ld2(sz + cf + e1);
            const float gzl0 = sz[cf + e0 - 1], gzl1 = sz[cf + e1 - 1];
            r00 = resid_face(a0.x, am0.x, gy0.x, gym.x, gz0.x, gzl0, up0.x, um0.x, u1.x, ua.x, u0.y, ul0, u0.x,
                             f0.x, hx);
            r01 = resid_face(a0.y, am0.y, gy0.y, gym.y, gz0.y, gz0.x, up0.y, um0.y, u1.y, ua.y, ur0, u0.x, u0.y,
                             f0.y, hx);
            r10 = resid_face(a1.x, am1.x, gy1.x, gy0.x, gz1.x, gzl1, up1.x, um1.x, ub.x, u0.x, u1.y, ul1, u1.x,
                             f1.x, hx);
            r11 = resid_face(a1.y, am1.y, gy1.y, gy0.y, gz1.y, gz1.x, up1.y, um1.y, ub.y, u0.y, ur1, u1.x, u1.y,
                             f1.y, hx);
        } else {
            r00 = resid_node<ISO>(a0.x, ap0.x, am0.x, a1.x, aa.x, a0.y, al0, up0.x, um0.x, u1.x, ua.x,
                                  u0.y, ul0, u0.x, f0.x, hx, hy, hz);
            r01 = resid_node<ISO>(a0.y, ap0.y, am0.y, a1.y, aa.y, ar0, a0.x, up0.y, um0.y, u1.y, ua.y,
                                  ur0, u0.x, u0.y, f0.y, hx, hy, hz);
            r10 = resid_node<ISO>(a1.x, ap1.x, am1.x, ab.x, a0.x, a1.y, al1, up1.x, um1.x, ub.x, u0.x,
                                  u1.y, ul1, u1.x, f1.x, hx, hy, hz);
            r11 = resid_node<ISO>(a1.y, ap1.y, am1.y, ab.y, a0.y, ar1, a1.x, up1.y, um1.y, ub.y, u0.y,
                                  ur1, u1.x, u1.y, f1.y, hx, hy, hz);
        }
        float* rw = sr + (it & 1) * RPL;
        *reinterpret_cast<float2*>(rw + e1) = make_float2(r10, r11);  // read by the coarse row below
        Rp[0] = r00, Rp[1] = r01, Rp[2] = r10, Rp[3] = r11;
        // the low-side ring from shared memory
        if (ring_e >= 0) {
            const int e = ring_e;
            const float* ac = sa + cu;
            const float* uq = su + cu;
            if constexpr (FACE)
                rw[e] = resid_face(ac[e], sa[mu + e], sy[cf + e], sy[cf + e - RRK], sz[cf + e], sz[cf + e - 1],
                                   su[pu + e], su[mu + e], uq[e + RRK], uq[e - RRK], uq[e + 1], uq[e - 1], uq[e],
                                   sf[cf + e], hx);
            else
                rw[e] = resid_node<ISO>(ac[e], sa[pu + e], sa[mu + e], ac[e + RRK], ac[e - RRK], ac[e + 1],
                                        ac[e - 1], su[pu + e], su[mu + e], uq[e + RRK], uq[e - RRK], uq[e + 1],
                                        uq[e - 1], uq[e], sf[cf + e], hx, hy, hz);
        }
        cp_wait_all();
        __syncthreads();
    }
}

// Blocks of the kernel resident at once on each device (0: not yet asked).
constexpr int kMaxDevices = 64;
int g_resident[kMaxDevices] = {};
std::mutex g_resident_mu;

template <bool ISO, int CIc, bool FACE>
void launch_rr(dim3 grid, const Dims& df, const Dims& dc, float hx, float hy, float hz,
               const float* u, const float* f, const float* a, float* out, cudaStream_t st) {
    constexpr int smem = FACE ? RSMEM_FACE : RSMEM;
    allow_smem((const void*)k_resid_restrict_stream<ISO, CIc, FACE>, smem);
    k_resid_restrict_stream<ISO, CIc, FACE><<<grid, RT, smem, st>>>(df, dc, hx, hy, hz, u, f, a, out);
}

template <bool ISO, bool FACE = false>
void launch_rr_ci(int ci, dim3 grid, const Dims& df, const Dims& dc, float hx, float hy, float hz,
                  const float* u, const float* f, const float* a, float* out, cudaStream_t st) {
    switch (ci) {
        case 1: launch_rr<ISO, 1, FACE>(grid, df, dc, hx, hy, hz, u, f, a, out, st); break;
        case 2: launch_rr<ISO, 2, FACE>(grid, df, dc, hx, hy, hz, u, f, a, out, st); break;
        case 4: launch_rr<ISO, 4, FACE>(grid, df, dc, hx, hy, hz, u, f, a, out, st); break;
        case 8: launch_rr<ISO, 8, FACE>(grid, df, dc, hx, hy, hz, u, f, a, out, st); break;
        default: launch_rr<ISO, 16, FACE>(grid, df, dc, hx, hy, hz, u, f, a, out, st); break;
    }
}

}  // namespace

namespace {

// Coarse planes per block from the cost model: fewest rounds of resident
// blocks times the planes each block streams (2 CIc + 1 residual planes and a
// start-up).
int model_rr_ci(const Level& fine, const Level& coarse) {
    const Dims& df = fine.d;
    int dev = 0;
    cudaGetDevice(&dev);
    int resident = 0;
    {
        std::lock_guard<std::mutex> lock(g_resident_mu);
        int& r = g_resident[(dev >= 0 && dev < kMaxDevices) ? dev : 0];
        if (!r) {
            allow_smem((const void*)k_resid_restrict_stream<true, 8, false>, RSMEM);
            int sms = 0, per_sm = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_resid_restrict_stream<true, 8, false>,
                                                          RT, RSMEM);
            r = sms * per_sm > 0 ? sms * per_sm : 1;
        }
        resident = r;
    }
    const long long tiles = (long long)(df.n2 / FK) * (df.n1 / FJ);
    const int n0c = coarse.d.n0;
    int best = 0;
    long long best_cost = 0;
    for (int ci = 1; ci <= 16 && ci <= n0c; ci *= 2) {
        if (n0c % ci) continue;
        const long long blocks = tiles * (n0c / ci);
        const long long cost = ((blocks + resident - 1) / resident) * (2 * ci + 2);
        if (!best || cost < best_cost) best = ci, best_cost = cost;
    }
    return best;
}

bool iso(const Level& L) { return L.h2i[0] == L.h2i[1] && L.h2i[1] == L.h2i[2]; }

bool rr_fits(const Level& fine) {
    const Dims& df = fine.d;
    return fine.coarsen[0] && fine.coarsen[1] && fine.coarsen[2] && df.n2 % FK == 0 && df.n1 % FJ == 0 &&
           df.n0 >= 4;
}

void launch_rr_level(const Level& fine, const Level& coarse, int ci, const float* u, const float* f,
                     const float* a, float* out, cudaStream_t st) {
    const Dims& df = fine.d;
    dim3 grid(df.n2 / FK, df.n1 / FJ, coarse.d.n0 / ci);
    launch_counter()++;
    if (fine.h2i[0] == fine.h2i[1] && fine.h2i[1] == fine.h2i[2]) {
        const float hh = (float)(0.5 * fine.h2i[0]);  // 2^-(2l+1): exact
        if (fine.face)
            launch_rr_ci<true, true>(ci, grid, df, coarse.d, hh, hh, hh, u, f, a, out, st);
        else
            launch_rr_ci<true>(ci, grid, df, coarse.d, hh, hh, hh, u, f, a, out, st);
    } else {
        launch_rr_ci<false>(ci, grid, df, coarse.d, (float)fine.h2i[0], (float)fine.h2i[1],
                            (float)fine.h2i[2], u, f, a, out, st);
    }
}

}  // namespace

// Coarse planes per block: the level's tuned value, else the cost model's.
int launch_resid_restrict_stream(const Level& fine, const Level& coarse, const float* u,
                                 const float* f, const float* a, float* out, cudaStream_t st) {
    if (!rr_fits(fine) || (fine.face && !iso(fine))) return 0;
    int ci = fine.tune[2];
    if (!ci || coarse.d.n0 % ci) ci = model_rr_ci(fine, coarse);
    launch_rr_level(fine, coarse, ci, u, f, a, out, st);
    return 1;
}

void tune_resid_restrict_level(Level& fine, const Level& coarse, const float* u, const float* f,
                               const float* a, float* out, cudaStream_t st) {
    if (!rr_fits(fine) || (fine.face && !iso(fine))) return;
    float best_ms = 0.f;
    int best = 0;
    // two rounds, the first only bringing the clocks up
    for (int round = 0; round < 2; ++round)
        for (int ci = 1; ci <= 16 && ci <= coarse.d.n0; ci *= 2) {
            if (coarse.d.n0 % ci) continue;
            const float ms = time_launches(st, 5, [&] { launch_rr_level(fine, coarse, ci, u, f, a, out, st); });
            if (round == 1 && (!best || ms < best_ms)) best = ci, best_ms = ms;
        }
    fine.tune[2] = best;
}

int bounds_fail_transfer() { return bounds_fail_take(); }

}  // namespace recon
