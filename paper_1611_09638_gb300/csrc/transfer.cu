// transfer.cu -- residual and full-weighting restriction of an FP32 level in
// one streaming pass (App. A's multigrid: the coarse right-hand side of a
// V-cycle is R (f - L u), with L the 7-point variable-coefficient operator
// with face coefficients (a + a_nbr)/2 and R the tensor (1/4, 1/2, 1/4)
// weighting on the fine nodes 2I-1, 2I, 2I+1 of each axis).
//
// The per-coarse-node kernel in mg_kernels.cu evaluates the 27 fine residuals
// of each coarse node's stencil, so every fine residual is computed 27/8
// times.  Here a block owns a 8 x 32 tile of the coarse (J, K) plane, i.e. a
// 16 x 64 tile of the fine plane, and streams fine planes along i: the
// residual of fine plane p is computed once per node on the tile plus its
// low-side ring (17 x 65 nodes) into shared memory, weighted in j and k there,
// and the i weights are applied in registers (an odd plane 2I+1 closes coarse
// plane I and opens I+1).  u and a are held for four planes (p-1 .. p+1 and
// the one being fetched), f for two; each plane is fetched with 16-byte
// cp.async copies.  DRAM traffic is one read of u, a, f and one write of the
// coarse plane.
#include "async_copy.cuh"
#include "recon_internal.cuh"

namespace recon {

namespace {

constexpr int RT = 256;                 // threads
constexpr int FJ = 16, FK = 64;         // fine tile rows (j) and columns (k)
constexpr int RH = 2, RKO = 4;          // halo rows / columns held
constexpr int RRJ = FJ + 2 * RH;        // 20 rows per plane
constexpr int RRK = FK + 2 * RKO;       // 72 columns per plane
constexpr int RPL = RRJ * RRK;          // floats per plane
constexpr int RCH = RRK / 4;            // 16-byte chunks per row
constexpr int NUA = RRJ * RCH;          // chunks of a u (or a) plane: 360
constexpr int NFC = (FJ + 1) * RCH;     // chunks of an f plane (rows -1 .. FJ-1): 306
constexpr int NRES = (FJ + 1) * (FK + 1);  // residual nodes (rows and columns -1 .. F-1): 1105
constexpr int RES_T = (NRES + RT - 1) / RT;  // residual nodes per thread: 5
constexpr int SUA = 4, SFF = 2;         // ring slots of u / a and of f
constexpr int RSMEM = (int)sizeof(float) * RPL * (2 * SUA + SFF + 1);
static_assert(NUA <= 2 * RT && NFC <= 2 * RT, "fetch rounds");
static_assert((FJ / 2) * (FK / 2) == RT, "one coarse node per thread");

// ISO: one spacing on every axis; hx then holds hh = h^-2 / 2, applied once
// to the sums of the face sums c + a_n (see k_rbgs_stream).
template <bool ISO, int CIc>
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
    float* sr = sf + SFF * RPL;
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
        ua_s[m] = e < NUA ? r * RRK + ch * 4 : -1;
        ua_g[m] = (((j0 + r - RH) & (df.n1 - 1)) << df.s2) + gk;
        f_s[m] = e < NFC ? (r + 1) * RRK + ch * 4 : -1;  // fine row r - 1
        f_g[m] = (((j0 + r - 1) & (df.n1 - 1)) << df.s2) + gk;
    }
    int res_e[RES_T];
#pragma unroll
    for (int m = 0; m < RES_T; ++m) {
        const int e = t + m * RT;
        const int r = e / (FK + 1), c = e - r * (FK + 1);  // fine row r - 1, column c - 1
        res_e[m] = e < NRES ? (r + 1) * RRK + c + RKO - 1 : -1;
    }
    const int jc = t >> 5, kc = t & 31;
    const int rc_e = (2 * jc + RH) * RRK + 2 * kc + RKO;
    const int out_o = ((J0c + jc) << dc.s2) + K0c + kc;

    // Plane p is held in u / a slot (p - pS + 1) mod SUA and f slot
    // (p - pS) mod SFF; the plane loop is unrolled (p = pS + it), so every
    // slot offset is a compile-time constant.
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
    };

    fetch_ua(pS - 1, 0 * RPL);
    fetch_ua(pS, 1 * RPL);
    fetch_ua(pS + 1, 2 * RPL);
    fetch_f(pS, 0 * RPL);
    cp_commit();
    cp_wait_all();
    __syncthreads();

    float acc = 0.f;
#pragma unroll
    for (int it = 0; it <= 2 * CIc; ++it) {
        const int p = pS + it;
        if (it < 2 * CIc) {
            fetch_ua(p + 2, ((it + 3) % SUA) * RPL);
            fetch_f(p + 1, ((it + 1) % SFF) * RPL);
        }
        cp_commit();
        // residual r = f - L u of plane p on the tile and its low-side ring
        {
            const int cu = ((it + 1) % SUA) * RPL, mu = (it % SUA) * RPL;
            const int pu = ((it + 2) % SUA) * RPL, cf = (it % SFF) * RPL;
            const float* ac = sa + cu;
            const float* uc = su + cu;
#pragma unroll
            for (int m = 0; m < RES_T; ++m) {
                const int e = res_e[m];
                if (e < 0) continue;
                const float c = ac[e];
                if (ISO) {
                    const float px = c + sa[pu + e], mx = c + sa[mu + e];
                    const float py = c + ac[e + RRK], my = c + ac[e - RRK];
                    const float pz = c + ac[e + 1], mz = c + ac[e - 1];
                    const float diag = (px + mx) + (py + my) + (pz + mz);
                    const float off = (px * su[pu + e] + mx * su[mu + e]) +
                                      (py * uc[e + RRK] + my * uc[e - RRK]) +
                                      (pz * uc[e + 1] + mz * uc[e - 1]);
                    sr[e] = fmaf(-hx, fmaf(-diag, uc[e], off), sf[cf + e]);
                } else {
                    const float apx = 0.5f * (c + sa[pu + e]) * hx, amx = 0.5f * (c + sa[mu + e]) * hx;
                    const float apy = 0.5f * (c + ac[e + RRK]) * hy, amy = 0.5f * (c + ac[e - RRK]) * hy;
                    const float apz = 0.5f * (c + ac[e + 1]) * hz, amz = 0.5f * (c + ac[e - 1]) * hz;
                    const float diag = (apx + amx) + (apy + amy) + (apz + amz);
                    const float off = (apx * su[pu + e] + amx * su[mu + e]) +
                                      (apy * uc[e + RRK] + amy * uc[e - RRK]) +
                                      (apz * uc[e + 1] + amz * uc[e - 1]);
                    sr[e] = sf[cf + e] - (off - diag * uc[e]);
                }
            }
        }
        __syncthreads();
        // (1/4, 1/2, 1/4) weights in j and k around fine node (2 jc, 2 kc)
        const float* R = sr + rc_e;
        const float s = 0.25f * (0.25f * R[-RRK - 1] + 0.5f * R[-RRK] + 0.25f * R[-RRK + 1]) +
                        0.5f * (0.25f * R[-1] + 0.5f * R[0] + 0.25f * R[1]) +
                        0.25f * (0.25f * R[RRK - 1] + 0.5f * R[RRK] + 0.25f * R[RRK + 1]);
        if (!(it & 1)) {  // p = 2I + 1 (odd) closes coarse plane I and opens I + 1
            if (it > 0) out[((I0c - 1 + (it >> 1)) << (dc.s1 + dc.s2)) + out_o] = acc + 0.25f * s;
            acc = 0.25f * s;
        } else {
            acc += 0.5f * s;
        }
        cp_wait_all();
        __syncthreads();
    }
}

// Blocks of the kernel resident at once on each device (0: not yet asked).
constexpr int kMaxDevices = 64;
int g_resident[kMaxDevices] = {};
std::mutex g_resident_mu;

template <bool ISO, int CIc>
void launch_rr(dim3 grid, const Dims& df, const Dims& dc, float hx, float hy, float hz,
               const float* u, const float* f, const float* a, float* out, cudaStream_t st) {
    allow_smem((const void*)k_resid_restrict_stream<ISO, CIc>, RSMEM);
    k_resid_restrict_stream<ISO, CIc><<<grid, RT, RSMEM, st>>>(df, dc, hx, hy, hz, u, f, a, out);
}

template <bool ISO>
void launch_rr_ci(int ci, dim3 grid, const Dims& df, const Dims& dc, float hx, float hy, float hz,
                  const float* u, const float* f, const float* a, float* out, cudaStream_t st) {
    switch (ci) {
        case 1: launch_rr<ISO, 1>(grid, df, dc, hx, hy, hz, u, f, a, out, st); break;
        case 2: launch_rr<ISO, 2>(grid, df, dc, hx, hy, hz, u, f, a, out, st); break;
        case 4: launch_rr<ISO, 4>(grid, df, dc, hx, hy, hz, u, f, a, out, st); break;
        case 8: launch_rr<ISO, 8>(grid, df, dc, hx, hy, hz, u, f, a, out, st); break;
        default: launch_rr<ISO, 16>(grid, df, dc, hx, hy, hz, u, f, a, out, st); break;
    }
}

}  // namespace

int launch_resid_restrict_stream(const Level& fine, const Level& coarse, const float* u,
                                 const float* f, const float* a, float* out, cudaStream_t st) {
    const Dims& df = fine.d;
    if (!fine.coarsen[0] || !fine.coarsen[1] || !fine.coarsen[2]) return 0;
    if (df.n2 % FK || df.n1 % FJ || df.n0 < 4) return 0;
    int dev = 0;
    cudaGetDevice(&dev);
    int resident = 0;
    {
        std::lock_guard<std::mutex> lock(g_resident_mu);
        int& r = g_resident[(dev >= 0 && dev < kMaxDevices) ? dev : 0];
        if (!r) {
            allow_smem((const void*)k_resid_restrict_stream<true, 8>, RSMEM);
            int sms = 0, per_sm = 0;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_resid_restrict_stream<true, 8>, RT,
                                                          RSMEM);
            r = sms * per_sm > 0 ? sms * per_sm : 1;
        }
        resident = r;
    }
    // coarse planes per block: fewest rounds of resident blocks times the
    // planes each block streams (2 CIc + 1 residual planes and a start-up)
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
    dim3 grid(df.n2 / FK, df.n1 / FJ, n0c / best);
    launch_counter()++;
    if (fine.h2i[0] == fine.h2i[1] && fine.h2i[1] == fine.h2i[2]) {
        const float hh = (float)(0.5 * fine.h2i[0]);  // 2^-(2l+1): exact
        launch_rr_ci<true>(best, grid, df, coarse.d, hh, hh, hh, u, f, a, out, st);
    } else {
        launch_rr_ci<false>(best, grid, df, coarse.d, (float)fine.h2i[0], (float)fine.h2i[1],
                            (float)fine.h2i[2], u, f, a, out, st);
    }
    return 1;
}

}  // namespace recon
