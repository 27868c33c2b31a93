// smoother.cu -- one full red-black Gauss-Seidel sweep (red, then black) of
// L u = f in FP32 (App. A, Eq. elliptic with x ~ xi; the 7-point
// variable-coefficient operator with face coefficients (a + a_nbr)/2) in a
// single pass over memory.
//
// Each block owns a TJ x TK tile of the (j, k) plane and streams CI planes
// along i.  At iteration q the red update of plane q runs on the tile plus a
// one-node ring (it reads old black values on a two-node ring), then the black
// update of plane q - 1 runs on the tile from those red values, and plane q - 1
// of the tile is written out.  u is read from u_old and written to u_new
// (another buffer), so halos read by a block are never values another block
// has already updated: the result equals the in-place sweep node for node.
// Shared memory holds rings of six u and a planes (tile + two-node ring in j,
// four-node in k so that every row is whole 16-byte chunks) and four f
// planes; while planes q and q - 1 are updated, the 16-byte cp.async copies
// of plane q + 3 (u, a) and q + 2 (f) are issued and those of the plane
// before them complete.  DRAM traffic is one read of u, a, f and one write
// of u.  With u_old == nullptr the sweep starts from u = 0 and u is not read.
//
// Every shared-memory and global offset a thread uses is computed once per
// block, and the plane loop is unrolled so that the ring slots are
// compile-time constants: the per-plane work is the cp.async issue, the
// stencil arithmetic and the stores.
#include "async_copy.cuh"
#include "recon_internal.cuh"

namespace recon {

namespace {

constexpr int TJ = 8, TK = 64, NT = 256;
constexpr int H = 2;                   // rows of halo (stencil ring of the red stage + 1)
constexpr int KO = 4;                  // columns of halo: one 16-byte chunk
constexpr int RJ = TJ + 2 * H;         // 12 rows held per plane
constexpr int RK = TK + 2 * KO;        // 72 columns held per plane
constexpr int PL = RJ * RK;            // floats per plane
constexpr int CH = RK / 4;             // 16-byte chunks per row
constexpr int SU = 6, SF = 4;          // ring slots of u / a and of f (two planes ahead)
constexpr int SMEM = (int)sizeof(float) * PL * (2 * SU + SF);
constexpr int NUA = RJ * CH;           // chunks of one u (or a) plane: 216
constexpr int NF = (TJ + 2) * CH;      // chunks of one f plane (rows of the red ring): 180
constexpr int NR = (TJ + 2) * ((TK + 2) / 2);  // red nodes on tile + ring: 330
constexpr int NB = TJ * (TK / 2);      // black nodes on the tile: 256
constexpr int NO = TJ * TK;            // outputs per plane: 512
static_assert(NUA <= NT && NF <= NT && NB == NT && NO == 2 * NT && NR <= 2 * NT, "tile");
static_assert(TJ % 2 == 0 && RK % 2 == 0 && TK == 64, "row-pair colour mapping");
static_assert(NR == 330 && (TJ + 2) * 32 == 320, "red task split");

// ISO: the level has one spacing on every axis, so every face coefficient
// carries the same factor hh = h^-2 / 2: the update sums the face sums
// c + a_n and applies hh once, u = (sum (c + a_n) u_n - f / hh) / sum (c + a_n)
// (1 / hh is a power of two); otherwise each face is scaled by its axis.
// PRO: the sweep also applies the coarse-grid correction of the V-cycle
// first: u_old + P(uc) is swept, P the trilinear prolongation from the
// coarse level dc (every axis halved).  Each thread issues the loads of its
// 4-node chunk of u and of the 6 or 12 coarse values the chunk's
// interpolation needs at the start of an iteration and combines and stores
// them to shared memory at its end, so the loads overlap the iteration's
// updates.
// COR: the swept values are also added to the FP64 field u64 (the defect
// correction phidot += e of the mixed-precision solve) as they are written;
// the u64 values are loaded at the start of the iteration that writes them.
template <bool ISO, int CI, bool PRO, bool COR>
__global__ void __launch_bounds__(NT) k_rbgs_stream(Dims d, float hx, float hy, float hz,
                                                    const float* __restrict__ u_old,
                                                    float* __restrict__ u_new,
                                                    const float* __restrict__ f,
                                                    const float* __restrict__ a,
                                                    const float* __restrict__ uc, Dims dc,
                                                    double* __restrict__ u64) {
    extern __shared__ float4 smem_f4[];
    float* su = reinterpret_cast<float*>(smem_f4);
    float* sa = su + SU * PL;
    float* sf = sa + SU * PL;
    const int t = threadIdx.x;
    const int k0 = blockIdx.x * TK, j0 = blockIdx.y * TJ, i0 = blockIdx.z * CI;
    static_assert(CI % 2 == 0, "the plane parity of iteration it is (it + 1) & 1");
    const int plane = d.n1 * d.n2;

    // ---- offsets fixed for the whole block -------------------------------
    // fetch: this thread's chunk of a u/a plane and of an f plane
    int ua_s = -1, ua_g = 0, f_s = -1, f_g = 0;
    if (t < NUA) {
        const int r = t / CH, ch = t - r * CH;
        ua_s = r * RK + ch * 4;
        ua_g = (((j0 + r - H) & (d.n1 - 1)) << d.s2) + ((k0 - KO + ch * 4) & (d.n2 - 1));
    }
    if (t < NF) {
        const int r = t / CH, ch = t - r * CH;
        f_s = (r + 1) * RK + ch * 4;
        f_g = (((j0 + r - 1) & (d.n1 - 1)) << d.s2) + ((k0 - KO + ch * 4) & (d.n2 - 1));
    }
    // Colour nodes are assigned so that each warp takes 16 nodes of a row and
    // the 16 nodes below them in the next row: the colours alternate from row
    // to row and RK is even, so the two half-warps read opposite bank parities
    // and the stride-2 access is free of bank conflicts.
    // Red tasks r = t and t + NT cover the 33 red nodes c = 0 .. 32 of each of
    // the ring rows jj = -1 .. TJ: r < 320 takes c = 1 .. 32 by row pairs, and
    // r = 320 .. 329 takes c = 0 of the ten rows.  Stored: smem offset of the
    // node with zero parity shift and the row's parity (the shift is
    // (q + j0 + jj + k0 - 1) & 1, i.e. the plane parity xor the row's).
    int red_e[2], red_p[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int r = t + m * NT;
        int jj = 0, c = -1;
        if (r < 320) {
            const int wt = r >> 5, lane = r & 31;
            jj = 2 * (wt >> 1) + (lane >> 4) - 1;
            c = 1 + 16 * (wt & 1) + (lane & 15);
        } else if (r < NR) {
            jj = r - 320 - 1;
            c = 0;
        }
        if (c >= 0) {
            red_e[m] = (jj + H) * RK + (2 * c - 1 + KO);
            red_p[m] = (j0 + jj + k0 - 1) & 1;
        } else {
            red_e[m] = -1, red_p[m] = 0;
        }
    }
    // black node t on the tile: 4 row pairs x 2 chunks of 16 of the 32 black
    // nodes per row; shift (p + j0 + jj + k0 + 1) & 1
    const int bw = t >> 5, blane = t & 31;
    const int blk_row = 2 * (bw >> 1) + (blane >> 4), blk_c = 16 * (bw & 1) + (blane & 15);
    const int blk_e = (blk_row + H) * RK + (2 * blk_c + KO);
    const int blk_p = (j0 + blk_row + k0 + 1) & 1;
    // the node offsets for an even and an odd plane
    int red0[2], red1[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) red0[m] = red_e[m] + red_p[m], red1[m] = red_e[m] + (1 ^ red_p[m]);
    const int blk0 = blk_e + blk_p, blk1 = blk_e + (1 ^ blk_p);
    // outputs t and t + NT
    int out_s[2], out_g[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int e = t + m * NT;
        const int jj = e / TK, kk = e - jj * TK;
        out_s[m] = (jj + H) * RK + (kk + KO);
        out_g[m] = ((j0 + jj) << d.s2) + k0 + kk;
    }

    // Plane x is held in ring slot (x - (i0 - 2)) mod SU of u and a and
    // (x - (i0 - 2)) mod SF of f.  The plane loop is unrolled, so with
    // q = i0 - 1 + it every slot offset below is a compile-time constant.
    // Copies run two planes ahead: iteration it issues u, a of plane q + 3
    // and f of plane q + 2 and then waits only for the previous iteration's
    // copies, so one group is always in flight while a plane is updated.
    auto pbase = [&](int q) { return (q & (d.n0 - 1)) * plane; };
    auto fetch_ua = [&](int q, int slot) {
        if (ua_s >= 0) {
            const int so = slot + ua_s, g = pbase(q) + ua_g;
            if (!PRO) {
                if (u_old) cp_async16(su + so, u_old + g);
                else *reinterpret_cast<float4*>(su + so) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            cp_async16(sa + so, a + g);
        }
    };
    // PRO: coarse offsets of this thread's chunk (fine row gj, fine columns
    // gk .. gk + 3 with gk a multiple of 4): rows J0, J1 (weights wj0, wj1)
    // and columns K0, K0 + 1 (an aligned pair: K0 is even) and K0 + 2.
    int o0 = 0, o1 = 0, o02 = 0, o12 = 0;
    float wj0 = 1.f, wj1 = 0.f;
    if (PRO && ua_s >= 0) {
        const int gj = (ua_g >> d.s2) & (d.n1 - 1), gk = ua_g & (d.n2 - 1);
        const int J0 = gj >> 1, oj = gj & 1;
        const int r0 = J0 << dc.s2, r1 = ((J0 + oj) & (dc.n1 - 1)) << dc.s2;
        wj0 = oj ? 0.5f : 1.f, wj1 = oj ? 0.5f : 0.f;
        const int K0 = gk >> 1, K2 = (K0 + 2) & (dc.n2 - 1);
        o0 = r0 + K0, o1 = r1 + K0, o02 = r0 + K2, o12 = r1 + K2;
    }
    const int cplane = dc.n1 * dc.n2;
    // The raw values one chunk's u + P(uc) needs: u itself and, per coarse
    // plane (one for an even fine plane, two for an odd one), the pairs at
    // (J0 | J1, K0..K0+1) and the values at K0 + 2.  pro_load issues the loads;
    // pro_value combines them later, so the loads stay in flight meanwhile.
    struct ProRaw {
        float4 u;
        float2 a, b, c, e;
        float a2, b2, c2, e2;
        bool odd;
    };
    auto pro_load = [&](int q) -> ProRaw {
        ProRaw r{};
        if (!PRO || ua_s < 0) return r;
        const int gi = q & (d.n0 - 1);
        const int I0 = gi >> 1;
        const float* p0 = uc + I0 * cplane;
        r.a = __ldg(reinterpret_cast<const float2*>(p0 + o0));
        r.b = __ldg(reinterpret_cast<const float2*>(p0 + o1));
        r.a2 = __ldg(p0 + o02), r.b2 = __ldg(p0 + o12);
        r.odd = gi & 1;
        if (r.odd) {  // odd fine plane: coarse planes I0 and I0 + 1
            const float* p1 = uc + ((I0 + 1) & (dc.n0 - 1)) * cplane;
            r.c = __ldg(reinterpret_cast<const float2*>(p1 + o0));
            r.e = __ldg(reinterpret_cast<const float2*>(p1 + o1));
            r.c2 = __ldg(p1 + o02), r.e2 = __ldg(p1 + o12);
        }
        r.u = __ldg(reinterpret_cast<const float4*>(u_old + pbase(q) + ua_g));
        return r;
    };
    auto pro_value = [&](const ProRaw& r) -> float4 {
        float k0v = fmaf(wj1, r.b.x, wj0 * r.a.x), k1v = fmaf(wj1, r.b.y, wj0 * r.a.y);
        float k2v = fmaf(wj1, r.b2, wj0 * r.a2);
        if (r.odd) {
            k0v = 0.5f * (k0v + fmaf(wj1, r.e.x, wj0 * r.c.x));
            k1v = 0.5f * (k1v + fmaf(wj1, r.e.y, wj0 * r.c.y));
            k2v = 0.5f * (k2v + fmaf(wj1, r.e2, wj0 * r.c2));
        }
        return make_float4(r.u.x + k0v, r.u.y + 0.5f * (k0v + k1v), r.u.z + k1v,
                           r.u.w + 0.5f * (k1v + k2v));
    };
    auto pro_store = [&](int slot, const float4& v) {
        if (PRO && ua_s >= 0) *reinterpret_cast<float4*>(su + slot + ua_s) = v;
    };
    auto fetch_f = [&](int q, int slot) {
        if (f_s >= 0) cp_async16(sf + slot + f_s, f + pbase(q) + f_g);
    };
    // Gauss-Seidel value at smem offset e of the plane in slots (cu, mu, pu)
    // of u and a (current, previous, next plane) and cf of f.
    const float ihh = 1.0f / hx;  // ISO: hx holds hh, a power of two
    auto gs = [&](int cu, int mu, int pu, int cf, int e) -> float {
        const float* ac = sa + cu;
        const float* uc = su + cu;
        const float c = ac[e];
        if (ISO) {
            const float px = c + sa[pu + e], mx = c + sa[mu + e];
            const float py = c + ac[e + RK], my = c + ac[e - RK];
            const float pz = c + ac[e + 1], mz = c + ac[e - 1];
            const float diag = (px + mx) + (py + my) + (pz + mz);
            const float off = (px * su[pu + e] + mx * su[mu + e]) + (py * uc[e + RK] + my * uc[e - RK]) +
                              (pz * uc[e + 1] + mz * uc[e - 1]);
            return __fdividef(fmaf(-ihh, sf[cf + e], off), diag);
        }
        const float apx = 0.5f * (c + sa[pu + e]) * hx, amx = 0.5f * (c + sa[mu + e]) * hx;
        const float apy = 0.5f * (c + ac[e + RK]) * hy, amy = 0.5f * (c + ac[e - RK]) * hy;
        const float apz = 0.5f * (c + ac[e + 1]) * hz, amz = 0.5f * (c + ac[e - 1]) * hz;
        const float diag = (apx + amx) + (apy + amy) + (apz + amz);
        const float off = (apx * su[pu + e] + amx * su[mu + e]) + (apy * uc[e + RK] + amy * uc[e - RK]) +
                          (apz * uc[e + 1] + amz * uc[e - 1]);
        return __fdividef(off - sf[cf + e], diag);
    };

    // prologue: u, a of planes i0-2 .. i0 and f of plane i0-1 (waited for);
    // u, a of plane i0+1 and f of plane i0 (left in flight)
    fetch_ua(i0 - 2, 0 * PL);
    fetch_ua(i0 - 1, 1 * PL);
    fetch_ua(i0, 2 * PL);
    fetch_f(i0 - 1, 1 * PL);
    cp_commit();
    if (PRO) {
        pro_store(0 * PL, pro_value(pro_load(i0 - 2)));
        pro_store(1 * PL, pro_value(pro_load(i0 - 1)));
        pro_store(2 * PL, pro_value(pro_load(i0)));
        pro_store(3 * PL, pro_value(pro_load(i0 + 1)));
    }
    cp_wait_all();
    __syncthreads();
    fetch_ua(i0 + 1, 3 * PL);
    fetch_f(i0, 2 * PL);
    cp_commit();

#pragma unroll
    for (int it = 0; it < CI + 2; ++it) {
        const int q = i0 - 1 + it;  // plane of the red update
        ProRaw pend;                // PRO: raw values of plane q + 3, stored below
        double cor[2] = {0.0, 0.0}; // COR: u64 at this thread's outputs of plane q - 1
        if (COR && it >= 2) {
            const int gb = pbase(q - 1);
#pragma unroll
            for (int m = 0; m < 2; ++m) cor[m] = u64[gb + out_g[m]];
        }
        if (it < CI) {
            if (PRO) pend = pro_load(q + 3);
            fetch_ua(q + 3, ((it + 4) % SU) * PL);
            fetch_f(q + 2, ((it + 3) % SF) * PL);
        }
        cp_commit();
        // red update of plane q on the tile + 1-node ring (reads old black)
        {
            const int cu = ((it + 1) % SU) * PL, mu = (it % SU) * PL, pu = ((it + 2) % SU) * PL;
            const int cf = ((it + 1) % SF) * PL;
#pragma unroll
            for (int m = 0; m < 2; ++m)
                if (red_e[m] >= 0) {
                    const int e = ((it + 1) & 1) ? red1[m] : red0[m];
                    su[cu + e] = gs(cu, mu, pu, cf, e);
                }
        }
        __syncthreads();
        // black update of plane p = q - 1 on the tile, then write the tile
        if (it >= 2) {
            const int cu = (it % SU) * PL, mu = ((it - 1) % SU) * PL, pu = ((it + 1) % SU) * PL;
            const int cf = (it % SF) * PL;
            const int e = (it & 1) ? blk1 : blk0;
            su[cu + e] = gs(cu, mu, pu, cf, e);
            __syncthreads();
            const int gb = pbase(q - 1);
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const float v = su[cu + out_s[m]];
                u_new[gb + out_g[m]] = v;
                if (COR) u64[gb + out_g[m]] = cor[m] + (double)v;
            }
        }
        // the slot of plane q + 3 was last read in the previous iteration
        if (PRO && it < CI) pro_store(((it + 4) % SU) * PL, pro_value(pend));
        cp_wait_prior();
        __syncthreads();
    }
}

constexpr int CIS = 16;  // planes streamed per block

template <bool PRO, bool COR>
void launch_sweep(const Level& L, const float* u_old, float* u_new, const float* f, const float* a,
                  const float* uc, const Dims& dc, double* u64, cudaStream_t st) {
    allow_smem((const void*)k_rbgs_stream<true, CIS, PRO, COR>, SMEM);
    allow_smem((const void*)k_rbgs_stream<false, CIS, PRO, COR>, SMEM);
    const Dims& d = L.d;
    dim3 grid(d.n2 / TK, d.n1 / TJ, d.n0 / CIS);
    launch_counter()++;
    if (L.h2i[0] == L.h2i[1] && L.h2i[1] == L.h2i[2]) {
        const float hh = (float)(0.5 * L.h2i[0]);  // 2^-(2l+1): exact
        k_rbgs_stream<true, CIS, PRO, COR><<<grid, NT, SMEM, st>>>(d, hh, hh, hh, u_old, u_new, f, a, uc,
                                                                   dc, u64);
    } else {
        k_rbgs_stream<false, CIS, PRO, COR><<<grid, NT, SMEM, st>>>(
            d, (float)L.h2i[0], (float)L.h2i[1], (float)L.h2i[2], u_old, u_new, f, a, uc, dc, u64);
    }
}

bool stream_fits(const Dims& d) { return d.n2 % TK == 0 && d.n1 % TJ == 0 && d.n0 % CIS == 0; }

}  // namespace

// One sweep u_new <- RBGS(u_old) in one pass when the level is a multiple of
// the tile; returns the number of sweeps done (1), or 0 with nothing launched.
template <>
int launch_rbgs_fused<float>(const Level& L, const float* u_old, float* u_new, const float* f,
                             const float* a, int nsweeps, cudaStream_t st) {
    if (nsweeps < 1 || !stream_fits(L.d)) return 0;
    launch_sweep<false, false>(L, u_old, u_new, f, a, nullptr, L.d, nullptr, st);
    return 1;
}

bool rbgs_prolong_fits(const Level& fine) {
    return fine.coarsen[0] && fine.coarsen[1] && fine.coarsen[2] && stream_fits(fine.d);
}

// The first post-smoothing sweep with the coarse correction folded in:
// u_new <- RBGS(u_old + P(uc)); returns 1, or 0 with nothing launched.
int launch_rbgs_prolong(const Level& fine, const Level& coarse, const float* uc, const float* u_old,
                        float* u_new, const float* f, const float* a, cudaStream_t st) {
    if (!rbgs_prolong_fits(fine) || !u_old) return 0;
    launch_sweep<true, false>(fine, u_old, u_new, f, a, uc, coarse.d, nullptr, st);
    return 1;
}

// A sweep that also adds its result to the FP64 field u64:
// u_new <- RBGS(u_old), u64 += u_new; returns 1, or 0 with nothing launched.
int launch_rbgs_correct(const Level& L, const float* u_old, float* u_new, const float* f,
                        const float* a, double* u64, cudaStream_t st) {
    if (!stream_fits(L.d) || !u_old) return 0;
    launch_sweep<false, true>(L, u_old, u_new, f, a, nullptr, L.d, u64, st);
    return 1;
}

// FP64 levels are bound by the FP64 issue rate, not by memory: the ring nodes
// the streaming kernel recomputes would cost more than the traffic they save,
// so FP64 sweeps use the in-place two-colour kernels.
template <>
int launch_rbgs_fused<double>(const Level&, const double*, double*, const double*,
                              const double*, int, cudaStream_t) {
    return 0;
}

}  // namespace recon
