// smoother.cu -- one full red-black Gauss-Seidel sweep (red, then black) of
// L u = f in FP32 (App. A, Eq. elliptic with x ~ xi; the 7-point
// variable-coefficient operator with face coefficients (a + a_nbr)/2) in a
// single pass over memory.
//
// Each block owns a TJ x TK tile of the (j, k) plane and streams CI planes
// along i.  Every thread owns two adjacent columns (k, k + 1) of one row of
// the tile for the whole stream.  In a plane exactly one of the two is red,
// and the red column of plane q is the black column of plane q - 1, so at
// iteration q a thread updates the red node of plane q and then the black
// node of plane q - 1 in the same column.  Along i every value a thread needs
// is its own: u, a and f of its two columns are read once per plane as one
// 8-byte shared load each and carried in registers, the red value of plane q
// is the black update's i + 1 neighbour and the red value of plane q - 2 its
// i - 1 neighbour.  Only the in-plane neighbours (rows j +- 1 and the column
// across the pair boundary) come from shared memory: 6 shared loads per
// update instead of 14.  Black values never go to shared memory: a plane's
// two outputs leave the thread as one 8-byte store.
//
// The red update also runs on a one-node ring around the tile (rows -1 and
// TJ, columns -1 and TK), from old black values on a two-node ring; the
// black update of the tile's edge nodes reads those ring values.  u is read
// from u_old and written to u_new (another buffer), so halos read by a block
// are never values another block has already updated: the result equals the
// in-place sweep node for node.  Shared memory holds rings of SU planes of u,
// a and f (u and a: tile + two-node ring in j, four-node in k so that every
// row is whole 16-byte chunks; f: tile + one-node ring), all fetched with
// 16-byte cp.async copies PD planes ahead of the one waited for (loading f
// straight into registers instead left the warps waiting on those loads).
// The stages of an iteration touch disjoint data (red writes red nodes of
// plane q and reads black ones, black reads red nodes of plane q - 1), so one
// block-wide barrier per plane suffices.  DRAM traffic is one read of u, a, f
// and one write of u.  With u_old == nullptr the sweep starts from u = 0 and
// u is not read.
//
// Tiles clear of the periodic seams (the 12 x 72 window of a plane lies
// inside the grid) stage their planes with the Tensor Memory Accelerator
// instead: one thread copies each field's whole window of a plane (a 72 x 12
// box of a rank-3 tensor map, which lands in exactly the ring slot's layout)
// and the block waits on that slot's mbarrier; tiles on a seam keep the
// per-thread 16-byte copies.  Both fill the slots with the same values.
//
// Every shared-memory and global offset a thread uses is computed once per
// block, and the plane loop is unrolled so that ring slots and register
// indices are compile-time constants.
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "async_copy.cuh"
#include "checked.cuh"
#include "recon_internal.cuh"
#include "tma.cuh"

namespace recon {

// Set by a sweep whose wait for a bulk copy gave up (read and cleared by
// sweep_wait_failed after a solve).
__device__ int g_sweep_wait_fail;

namespace {

constexpr int TJ = 8, TK = 64, NT = 256;
constexpr int H = 2;                   // rows of halo (stencil ring of the red stage + 1)
constexpr int KO = 4;                  // columns of halo: one 16-byte chunk
constexpr int RJ = TJ + 2 * H;         // 12 rows held per plane
constexpr int RK = TK + 2 * KO;        // 72 columns held per plane
constexpr int PL = RJ * RK;            // floats per plane
constexpr int CH = RK / 4;             // 16-byte chunks per row
constexpr int PD = 2;                  // planes of copies in flight ahead of the one waited for
static_assert(PD >= 2, "the prolongation is applied one iteration before a plane is read");
constexpr int SU = 3 + PD;             // ring slots of u, a and f
constexpr int MBAR = 8 * SU;           // one mbarrier per ring slot (bulk copies)
constexpr int SMEM = (int)sizeof(float) * PL * 3 * SU + MBAR;
// FACE: u, the three face-sum planes and f
constexpr int SMEM_FACE = (int)sizeof(float) * PL * 5 * SU + MBAR;
static_assert((sizeof(float) * PL) % 128 == 0, "every ring slot starts on a 128-byte boundary");

// Tensor maps of one sweep's inputs: u_old, a (or the x face sums), f, and
// the y and z face sums of a FACE level; on = 0 where none apply.
struct SweepMaps {
    CUtensorMap m[5];
    int on;
};
constexpr int NUA = RJ * CH;           // chunks of one u (or a) plane: 216
constexpr int NF = (TJ + 2) * CH;      // chunks of one f plane (rows of the red ring): 180
constexpr int NRING = 2 * (TK / 2 + 1) + TJ;  // red ring nodes per plane: 74
static_assert(NUA <= NT && NRING <= NT, "tile");
static_assert(TJ * TK == 2 * NT && TK == 64 && TJ % 2 == 0, "two columns per thread, row pairs per warp");
static_assert(RK % 32 == 8 && ((TJ + 1) * RK) % 32 == 8, "bank parity of the row pairs");

// The Gauss-Seidel value of a node from its coefficient c, the neighbours'
// coefficients and values (x: i, y: j, z: k; p: +1, m: -1) and f.
// ISO: the level has one spacing on every axis, so every face coefficient
// carries the same factor hh = h^-2 / 2: the update sums the face sums
// c + a_n and applies hh once, u = (sum (c + a_n) u_n - f / hh) / sum (c + a_n)
// (1 / hh is a power of two, passed as s0); otherwise each face is scaled by
// its axis (s0, s1, s2 = h_i^-2, h_j^-2, h_k^-2).
template <bool ISO>
__device__ __forceinline__ float gs_node(float c, float apx, float amx, float apy, float amy, float apz,
                                         float amz, float upx, float umx, float upy, float umy,
                                         float upz, float umz, float f, float s0, float s1, float s2) {
    if (ISO) {
        const float px = c + apx, mx = c + amx, py = c + apy, my = c + amy, pz = c + apz, mz = c + amz;
        const float diag = (px + mx) + (py + my) + (pz + mz);
        const float off = (px * upx + mx * umx) + (py * upy + my * umy) + (pz * upz + mz * umz);
        return __fdividef(fmaf(-s0, f, off), diag);
    }
    const float px = 0.5f * (c + apx) * s0, mx = 0.5f * (c + amx) * s0;
    const float py = 0.5f * (c + apy) * s1, my = 0.5f * (c + amy) * s1;
    const float pz = 0.5f * (c + apz) * s2, mz = 0.5f * (c + amz) * s2;
    const float diag = (px + mx) + (py + my) + (pz + mz);
    const float off = (px * upx + mx * umx) + (py * upy + my * umy) + (pz * upz + mz * umz);
    return __fdividef(off - f, diag);
}

// The same update on an isotropic level whose operator is given by its face
// sums G (2 x the face coefficient) of the six faces of the node.
__device__ __forceinline__ float gs_face(float gpx, float gmx, float gpy, float gmy, float gpz, float gmz,
                                         float upx, float umx, float upy, float umy, float upz,
                                         float umz, float f, float s0) {
    const float diag = (gpx + gmx) + (gpy + gmy) + (gpz + gmz);
    const float off = (gpx * upx + gmx * umx) + (gpy * upy + gmy * umy) + (gpz * upz + gmz * umz);
    return __fdividef(fmaf(-s0, f, off), diag);
}

// the value of column z (0: k, 1: k + 1) of a pair, and of the other column
__device__ __forceinline__ float pick(float2 v, int z) { return z ? v.y : v.x; }
__device__ __forceinline__ float other(float2 v, int z) { return z ? v.x : v.y; }

// PRO: the sweep also applies the coarse-grid correction of the V-cycle
// first: u_old + P(uc) is swept, P the trilinear prolongation from the
// coarse level dc (every axis halved).  u_old arrives by the same cp.async
// copies as in the plain sweep; a plane's copies are waited for at the end of
// the iteration before the one that first reads it, and there each thread
// adds P(uc) to its own 4-node chunk in shared memory, from the 6 or 12
// coarse values (an L2-resident level) it loaded at the start of that
// iteration.
// COR: the swept values are also added to the FP64 field u64 (the defect
// correction phidot += e of the mixed-precision solve) as they are written;
// the u64 values are loaded one iteration before the one that writes them.
// FACE: the level's operator is given by face sums (a points at the x, y and
// z face-sum arrays, one after another): the x sums of the thread's columns
// are carried in registers like a, the y and z sums of the plane come from
// shared memory (isotropic levels only; two blocks per SM).
// tm: tensor maps of u_old, a (or the x face sums), f and the y and z face
// sums, each with a 72 x 12 x 1 box; tm.on = 0: every tile uses cp.async.
// Registers are capped so that 4 blocks (3 with PRO) stay resident per SM.
template <bool ISO, int CI, bool PRO, bool COR, bool FACE>
__global__ void __launch_bounds__(NT, FACE ? 2 : (PRO ? 3 : 4)) k_rbgs_stream(Dims d, float hx, float hy, float hz,
                                                    const float* __restrict__ u_old,
                                                    float* __restrict__ u_new,
                                                    const float* __restrict__ f,
                                                    const float* __restrict__ a,
                                                    const float* __restrict__ uc, Dims dc,
                                                    double* __restrict__ u64,
                                                    const __grid_constant__ SweepMaps tm) {
    extern __shared__ __align__(128) float4 smem_f4[];
    float* su = reinterpret_cast<float*>(smem_f4);
    float* sa = su + SU * PL;  // a, or (FACE) the x face sums
    float* sy = sa + SU * PL;  // FACE: y and z face sums
    float* sz = sy + SU * PL;
    float* sf = FACE ? sz + SU * PL : sy;
    const int t = threadIdx.x;
    const int k0 = blockIdx.x * TK, j0 = blockIdx.y * TJ, i0 = blockIdx.z * CI;
    static_assert(CI % 2 == 0, "the parity of plane i0 - 1 + it is (it + 1) & 1");
    static_assert(!FACE || (ISO && !COR), "face sums: isotropic coarse levels");
    const float* gy = FACE ? a + d.cells : nullptr;
    const float* gz = FACE ? a + 2 * (size_t)d.cells : nullptr;
    const int plane = d.n1 * d.n2;
    const float s0 = ISO ? 1.0f / hx : hx;  // ISO: hx holds hh, a power of two

    // ---- offsets fixed for the whole block -------------------------------
    // fetch: this thread's 16-byte chunk of a u/a plane and of an f plane
    // (RC_OFF: the RECON_CHECKED build checks each offset against the extent
    // it addresses; otherwise it is the offset itself)
    int ua_s = -1, ua_g = 0;
    if (t < NUA) {
        const int r = t / CH, ch = t - r * CH;
        ua_s = RC_OFF(r * RK + ch * 4, PL - 3, 101);
        ua_g = RC_OFF((((j0 + r - H) & (d.n1 - 1)) << d.s2) + ((k0 - KO + ch * 4) & (d.n2 - 1)), plane - 3, 102);
    }
    int f_s = -1, f_g = 0;
    if (t < NF) {
        const int r = t / CH, ch = t - r * CH;
        f_s = RC_OFF((r + 1) * RK + ch * 4, PL - 3, 103);
        f_g = RC_OFF((((j0 + r - 1) & (d.n1 - 1)) << d.s2) + ((k0 - KO + ch * 4) & (d.n2 - 1)), plane - 3, 104);
    }
    // Columns: warp w takes rows 2 (w / 2) and 2 (w / 2) + 1 (one per half
    // warp) and column pairs 16 (w & 1) .. + 15.  The red column of a pair in
    // plane q is k = q + j (mod 2) (red: i + j + k even), so the two half
    // warps use opposite bank parities (RK = 8 mod 32) and the stride-2
    // accesses are free of bank conflicts.  z[m]: the offset (0 or 1) in the
    // pair of the column updated at iterations of parity m (plane
    // q = i0 - 1 + it has the parity of it + 1).
    const int w = t >> 5, lane = t & 31;
    const int jj = 2 * (w >> 1) + (lane >> 4), pr = 16 * (w & 1) + (lane & 15);
    const int jg = j0 + jj;
    int z[2], ez[2], en[2];
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        z[m] = (m + 1 + jg) & 1;
        // the node and its rows j +- 1 lie in the plane buffer
        ez[m] = RK + RC_OFF((jj + H) * RK + KO + 2 * pr + z[m] - RK, PL - 2 * RK, 105);
        en[m] = RC_OFF(ez[m] + (z[m] ? 1 : -1), PL, 106);  // the k neighbour in the adjacent pair
    }
    const int ep = RC_OFF((jj + H) * RK + KO + 2 * pr, PL - 1, 107);  // the pair in a plane buffer (8-byte aligned)
    const int gp = RC_OFF((jg << d.s2) + k0 + 2 * pr, plane - 1, 108);   // the pair in a global plane
    // Ring tasks (threads t < NRING): the red node of row -1 or TJ (t < 66:
    // the 33 red nodes of each row) or of column -1 or TK of tile row t - 66.
    // ring_e: smem offset of the node in a plane of even and of odd q - i0.
    int ring_e[2] = {-1, -1};
    if (t < NRING) {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            int rj, kc;
            if (t < 64) {  // half warps: rows -1 and TJ (opposite bank parities), nodes 0 .. 31
                rj = (t & 16) ? TJ : -1;
                const int c = 16 * (t >> 5) + (t & 15);
                kc = 2 * c - 1 + ((m + j0 + rj + k0 - 1) & 1);
            } else if (t < 66) {  // node 32 of rows -1 and TJ
                rj = t == 64 ? -1 : TJ;
                kc = 2 * 32 - 1 + ((m + j0 + rj + k0 - 1) & 1);
            } else {              // the red one of columns -1 and TK
                rj = t - 66;
                kc = ((m + j0 + rj + k0 - 1) & 1) ? TK : -1;
            }
            ring_e[m] = RK + RC_OFF((rj + H) * RK + KO + kc - RK, PL - 2 * RK, 109);  // with rows +- 1
        }
    }

    // Plane x is held in ring slot (x - (i0 - 2)) mod SU of u, a and f.  The
    // plane loop is unrolled, so with q = i0 - 1 + it every slot offset below
    // is a compile-time constant.  Iteration it issues the copies of plane
    // q + 1 + PD and, before its barrier, waits for those the next iteration
    // reads.
    auto pbase = [&](int q) { return (q & (d.n0 - 1)) * plane; };
    // Bulk copies: plane x sits in ring slot r % SU, r = x - (i0 - 2), and is
    // that slot's (r / SU)-th fill, so it completes the phase of parity
    // (r / SU) & 1 of the slot's mbarrier.  f is read on rows 1 .. TJ only;
    // its box brings the same 12 rows as u's.
    unsigned long long* mbar = reinterpret_cast<unsigned long long*>(sf + SU * PL);
    const bool tma = tm.on && j0 >= H && j0 + TJ + H <= d.n1 && k0 >= KO && k0 + TK + KO <= d.n2;
    auto tma_issue = [&](int x, bool with_f) {
        const int r = x - (i0 - 2), slot = (r % SU) * PL;
        unsigned long long* bar = mbar + r % SU;
        const int kx = k0 - KO, jy = j0 - H, iz = x & (d.n0 - 1);
        const unsigned nfield = (u_old ? 1u : 0u) + (FACE ? 3u : 1u) + (with_f ? 1u : 0u);
        mbar_arrive_expect(bar, nfield * (unsigned)(sizeof(float) * PL));
        if (u_old) tma_load_3d(su + slot, &tm.m[0], kx, jy, iz, bar);
        tma_load_3d(sa + slot, &tm.m[1], kx, jy, iz, bar);
        if (FACE) {
            tma_load_3d(sy + slot, &tm.m[3], kx, jy, iz, bar);
            tma_load_3d(sz + slot, &tm.m[4], kx, jy, iz, bar);
        }
        if (with_f) tma_load_3d(sf + slot, &tm.m[2], kx, jy, iz, bar);
    };
    auto tma_wait = [&](int x) {
        const int r = x - (i0 - 2);
        mbar_wait(mbar + r % SU, (unsigned)((r / SU) & 1), &g_sweep_wait_fail);
    };
    // the sweep from u = 0: this thread's chunk of a u slot (both paths)
    auto zero_u = [&](int slot) {
        if (ua_s >= 0) *reinterpret_cast<float4*>(su + slot + ua_s) = make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto fetch_ua = [&](int q, int slot) {
        if (ua_s >= 0) {
            const int so = slot + ua_s, g = pbase(q) + ua_g;
            if (u_old) cp_async16(su + so, u_old + g);
            else *reinterpret_cast<float4*>(su + so) = make_float4(0.f, 0.f, 0.f, 0.f);
            cp_async16(sa + so, a + g);
            if (FACE) {
                cp_async16(sy + so, gy + g);
                cp_async16(sz + so, gz + g);
            }
        }
    };
    // f is read for the planes of the red updates, i0 - 1 .. i0 + CI
    auto fetch_f = [&](int q, int slot) {
        if (f_s >= 0) cp_async16(sf + slot + f_s, f + pbase(q) + f_g);
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
    if (PRO && ua_s >= 0) {  // pairs at o0, o1; single values at o02, o12
        o0 = RC_OFF(o0, cplane - 1, 110), o1 = RC_OFF(o1, cplane - 1, 111);
        o02 = RC_OFF(o02, cplane, 112), o12 = RC_OFF(o12, cplane, 113);
    }
    // The coarse values one chunk's P(uc) needs: per coarse plane (one for an
    // even fine plane, two for an odd one), the pairs at (J0 | J1, K0..K0+1)
    // and the values at K0 + 2.  pro_load issues the loads; pro_value combines
    // them with the chunk of u later, so the loads stay in flight meanwhile.
    struct ProRaw {
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
        return r;
    };
    auto pro_value = [&](const ProRaw& r, const float4& u) -> float4 {
        float k0v = fmaf(wj1, r.b.x, wj0 * r.a.x), k1v = fmaf(wj1, r.b.y, wj0 * r.a.y);
        float k2v = fmaf(wj1, r.b2, wj0 * r.a2);
        if (r.odd) {
            k0v = 0.5f * (k0v + fmaf(wj1, r.e.x, wj0 * r.c.x));
            k1v = 0.5f * (k1v + fmaf(wj1, r.e.y, wj0 * r.c.y));
            k2v = 0.5f * (k2v + fmaf(wj1, r.e2, wj0 * r.c2));
        }
        return make_float4(u.x + k0v, u.y + 0.5f * (k0v + k1v), u.z + k1v, u.w + 0.5f * (k1v + k2v));
    };
    // u + P(uc) in place on this thread's chunk of the plane in ring slot
    // `slot` (its own copies of that plane have completed)
    auto pro_apply = [&](int slot, const ProRaw& r) {
        if (PRO && ua_s >= 0) {
            float4* p = reinterpret_cast<float4*>(su + slot + ua_s);
            *p = pro_value(r, *p);
        }
    };
    auto own = [&](const float* buf, int slot) { return *reinterpret_cast<const float2*>(buf + slot + ep); };

    // Registers, indexed by plane x as (x - (i0 - 2)) & 3 (plane q: (it + 1) & 3):
    // U, A: old u and a of the pair (planes q - 1 .. q + 1 and q - 2 .. q + 1);
    // F: f of the pair (q - 1 .. q); R: the red value of the column updated
    // for that plane (q - 2 .. q).
    float2 U[4], A[4], F[4];
    float R[4];
    double2 cor = make_double2(0.0, 0.0);  // COR: u64 at the pair of the plane written next

    // prologue: u, a of planes i0-2 .. i0 (waited for); with PD = 2 also
    // plane i0+1 (left in flight)
    if (tma) {
        if (t == 0) {
            for (int r = 0; r < SU; ++r) mbar_init(mbar + r, 1);
            mbar_init_fence();
        }
        __syncthreads();
        if (t == 0) {
            tma_issue(i0 - 2, false);
            tma_issue(i0 - 1, true);
            tma_issue(i0, true);
        }
        if (!u_old) zero_u(0 * PL), zero_u(1 * PL), zero_u(2 * PL);
    } else {
        fetch_ua(i0 - 2, 0 * PL);
        fetch_ua(i0 - 1, 1 * PL);
        fetch_ua(i0, 2 * PL);
        fetch_f(i0 - 1, 1 * PL);
        fetch_f(i0, 2 * PL);
        cp_commit();
    }
    auto wait_prologue = [&] {
        if (tma) tma_wait(i0 - 2), tma_wait(i0 - 1), tma_wait(i0);
        else cp_wait_all();
    };
    if (PRO) {  // the three planes read first: their coarse values, then u + P(uc)
        const ProRaw r0 = pro_load(i0 - 2), r1 = pro_load(i0 - 1), r2 = pro_load(i0);
        wait_prologue();
        pro_apply(0 * PL, r0);
        pro_apply(1 * PL, r1);
        pro_apply(2 * PL, r2);
    } else {
        wait_prologue();
    }
    __syncthreads();
    if (PD == 2) {
        if (tma) {
            if (t == 0) tma_issue(i0 + 1, true);
            if (!u_old) zero_u(3 * PL);
        } else {
            fetch_ua(i0 + 1, 3 * PL);
            fetch_f(i0 + 1, 3 * PL);
            cp_commit();
        }
    }
    U[0] = own(su, 0 * PL), U[1] = own(su, 1 * PL);
    A[0] = own(sa, 0 * PL), A[1] = own(sa, 1 * PL);

#pragma unroll
    for (int it = 0; it < CI + 2; ++it) {
        const int q = i0 - 1 + it;                 // plane of the red update
        const int iq = (it + 1) & 3;               // register index of plane q
        const int im1 = it & 3, ip1 = (it + 2) & 3, im2 = (it + 3) & 3;  // q - 1, q + 1, q - 2
        const int cu = ((it + 1) % SU) * PL, mu = (it % SU) * PL, pu = ((it + 2) % SU) * PL;
        const int zz = z[it & 1], e = ez[it & 1], en_ = en[it & 1];
        const bool fetch = it <= CI + 1 - PD;
        // PRO: plane q + PD (copied in the previous iteration, first read in
        // the next one) gets u + P(uc) at the end of this iteration
        const bool prolong = PRO && it <= CI + 2 - PD;
        ProRaw pend;
        if (prolong) pend = pro_load(q + PD);
        if (fetch) {
            if (tma) {
                // the slot last held plane q - 4, read for the last time
                // before the previous iteration's barrier
                if (t == 0) {
                    fence_async_smem();
                    tma_issue(q + 1 + PD, it + PD <= CI);
                }
                if (!u_old) zero_u(((it + 2 + PD) % SU) * PL);
            } else {
                fetch_ua(q + 1 + PD, ((it + 2 + PD) % SU) * PL);
                if (it + PD <= CI) fetch_f(q + 1 + PD, ((it + 2 + PD) % SU) * PL);
            }
        }
        cp_commit();
        const double2 cor_now = cor;
        if (COR && it >= 1 && it <= CI) cor = *reinterpret_cast<const double2*>(u64 + pbase(q) + gp);
        U[ip1] = own(su, pu);
        A[ip1] = own(sa, pu);
        F[iq] = own(sf, cu);

        // red update of plane q at this thread's column
        {
            const float* ap = sa + cu;
            const float* up = su + cu;
            const float uN = up[en_];
            const float uW = other(U[iq], zz);
            float r;
            if constexpr (FACE) {
                r = gs_face(pick(A[iq], zz), pick(A[im1], zz), sy[cu + e], sy[cu + e - RK], sz[cu + e],
                            sz[cu + e - 1], pick(U[ip1], zz), pick(U[im1], zz), up[e + RK], up[e - RK],
                            zz ? uN : uW, zz ? uW : uN, pick(F[iq], zz), s0);
            } else {
                const float aN = ap[en_];
                const float aW = other(A[iq], zz);
                r = gs_node<ISO>(pick(A[iq], zz), pick(A[ip1], zz), pick(A[im1], zz), ap[e + RK],
                                 ap[e - RK], zz ? aN : aW, zz ? aW : aN, pick(U[ip1], zz),
                                 pick(U[im1], zz), up[e + RK], up[e - RK], zz ? uN : uW,
                                 zz ? uW : uN, pick(F[iq], zz), s0, hy, hz);
            }
            R[iq] = r;
            if (it >= 1 && it <= CI) su[cu + e] = r;  // the black update of plane q reads it
        }
        // red update of plane q at the ring node (the black updates read
        // planes i0 .. i0 + CI - 1 only)
        if (it >= 1 && it <= CI && t < NRING) {
            const int r = ring_e[(it + 1) & 1];
            const float* ac = sa + cu;
            const float* uq = su + cu;
            if constexpr (FACE)
                su[cu + r] = gs_face(ac[r], sa[mu + r], sy[cu + r], sy[cu + r - RK], sz[cu + r],
                                     sz[cu + r - 1], su[pu + r], su[mu + r], uq[r + RK], uq[r - RK],
                                     uq[r + 1], uq[r - 1], sf[cu + r], s0);
            else
                su[cu + r] = gs_node<ISO>(ac[r], sa[pu + r], sa[mu + r], ac[r + RK], ac[r - RK], ac[r + 1],
                                          ac[r - 1], su[pu + r], su[mu + r], uq[r + RK], uq[r - RK],
                                          uq[r + 1], uq[r - 1], sf[cu + r], s0, hy, hz);
        }
        // black update of plane q - 1 at the same column; write plane q - 1
        if (it >= 2) {
            const float* ap = sa + mu;
            const float* up = su + mu;
            const float uN = up[en_];
            const float uW = R[im1];
            float b;
            if constexpr (FACE) {
                b = gs_face(pick(A[im1], zz), pick(A[im2], zz), sy[mu + e], sy[mu + e - RK], sz[mu + e],
                            sz[mu + e - 1], R[iq], R[im2], up[e + RK], up[e - RK], zz ? uN : uW,
                            zz ? uW : uN, pick(F[im1], zz), s0);
            } else {
                const float aN = ap[en_];
                const float aW = other(A[im1], zz);
                b = gs_node<ISO>(pick(A[im1], zz), pick(A[iq], zz), pick(A[im2], zz), ap[e + RK],
                                 ap[e - RK], zz ? aN : aW, zz ? aW : aN, R[iq], R[im2],
                                 up[e + RK], up[e - RK], zz ? uN : uW, zz ? uW : uN,
                                 pick(F[im1], zz), s0, hy, hz);
            }
            const float2 v = zz ? make_float2(R[im1], b) : make_float2(b, R[im1]);
            const int g = pbase(q - 1) + gp;
            *reinterpret_cast<float2*>(u_new + g) = v;
            if (COR)
                *reinterpret_cast<double2*>(u64 + g) =
                    make_double2(cor_now.x + (double)v.x, cor_now.y + (double)v.y);
        }
        if (tma) {
            if (it <= CI + 2 - PD) tma_wait(q + PD);  // planes up to i0 + CI + 1 were fetched
        } else if (PD == 1) {
            cp_wait_all();
        } else {
            cp_wait_prior();
        }
        // this thread's copies of plane q + PD are complete (bulk copies: the
        // whole plane); no one reads that slot before the barrier
        if (prolong) pro_apply(((it + 1 + PD) % SU) * PL, pend);
        __syncthreads();
    }
}

// Planes streamed per block: 16 where the level gives enough blocks (a
// round of resident blocks per SM streams fewer halo planes), 8 or 4 on
// small levels, where fewer planes per block put more blocks to work.  The
// choice minimises rounds of resident blocks times (planes + prologue).
constexpr int kCIs[3] = {4, 8, 16};
constexpr int kMaxDevices = 64;

// The map of one grid array with the sweep's 72 x 12 x 1 box, from a cache
// keyed by device, address and shape (the solver's buffers live as long as
// their handle; a map only records an address and a shape).
bool plane_map(CUtensorMap* out, const float* base, const Dims& d) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, int, int, int>, CUtensorMap> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, (const void*)base, d.n0, d.n1, d.n2);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it == cache.end()) {
        CUtensorMap m;
        if (!encode_grid_map(&m, base, d.n0, d.n1, d.n2, RK, RJ)) return false;
        it = cache.emplace(key, m).first;
    }
    *out = it->second;
    return true;
}

// Maps for a sweep of level L where some tile is clear of the seams
// (n2 >= 4 TK, n1 >= 4 TJ) and the level allows bulk copies.
template <bool FACE>
void sweep_maps(SweepMaps& m, const Level& L, const float* u_old, const float* f, const float* a) {
    std::memset(&m, 0, sizeof(m));
    const Dims& d = L.d;
    if (!L.tma || d.n2 < 4 * TK || d.n1 < 4 * TJ) return;
    bool ok = (!u_old || plane_map(&m.m[0], u_old, d)) && plane_map(&m.m[1], a, d) && plane_map(&m.m[2], f, d);
    if (FACE) ok = ok && plane_map(&m.m[3], a + d.cells, d) && plane_map(&m.m[4], a + 2 * (size_t)d.cells, d);
    m.on = ok ? 1 : 0;
}

template <bool ISO, int CI, bool PRO, bool COR, bool FACE = false>
void launch_ci(dim3 grid, const Level& L, float hx, float hy, float hz, const float* u_old, float* u_new,
               const float* f, const float* a, const float* uc, const Dims& dc, double* u64, cudaStream_t st) {
    constexpr int smem = FACE ? SMEM_FACE : SMEM;
    SweepMaps maps;
    sweep_maps<FACE>(maps, L, u_old, f, a);
    allow_smem((const void*)k_rbgs_stream<ISO, CI, PRO, COR, FACE>, smem);
    k_rbgs_stream<ISO, CI, PRO, COR, FACE><<<grid, NT, smem, st>>>(L.d, hx, hy, hz, u_old, u_new, f, a, uc,
                                                                   dc, u64, maps);
}

// Blocks of the PRO (or plain; FACE or nodal) variant resident at once on the
// current device.
template <bool PRO, bool FACE>
int resident_blocks() {
    static int cache[kMaxDevices] = {};
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    int& r = cache[(dev >= 0 && dev < kMaxDevices) ? dev : 0];
    if (!r) {
        constexpr int smem = FACE ? SMEM_FACE : SMEM;
        allow_smem((const void*)k_rbgs_stream<true, 16, PRO, false, FACE>, smem);
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rbgs_stream<true, 16, PRO, false, FACE>, NT,
                                                      smem);
        r = sms * per_sm > 0 ? sms * per_sm : 1;
    }
    return r;
}

// The cost model's choice of planes per block.
template <bool PRO>
int model_ci(const Dims& d, bool face) {
    const long long tiles = (long long)(d.n2 / TK) * (d.n1 / TJ);
    const int resident = face ? resident_blocks<PRO, true>() : resident_blocks<PRO, false>();
    int ci = 0;
    long long best = 0;
    for (int ci_try : kCIs) {
        if (d.n0 % ci_try) continue;
        const long long blocks = tiles * (d.n0 / ci_try);
        const long long cost = ((blocks + resident - 1) / resident) * (ci_try + 4);
        if (!ci || cost < best) ci = ci_try, best = cost;
    }
    return ci;
}

// ci: planes per block (0: the level's tuned value, else the cost model's).
// A level given by face sums (L.face) runs the FACE variant (isotropic levels).
template <bool PRO, bool COR>
void launch_sweep(const Level& L, const float* u_old, float* u_new, const float* f, const float* a,
                  const float* uc, const Dims& dc, double* u64, cudaStream_t st, int ci = 0) {
    const Dims& d = L.d;
    if (!ci) ci = L.tune[PRO ? 1 : 0];
    if (!ci || d.n0 % ci) ci = model_ci<PRO>(d, L.face != 0);
    dim3 grid(d.n2 / TK, d.n1 / TJ, d.n0 / ci);
    launch_counter()++;
    const bool iso = L.h2i[0] == L.h2i[1] && L.h2i[1] == L.h2i[2];
    // ISO: hh = 2^-(2l+1), exact in FP32
    const float hx = iso ? (float)(0.5 * L.h2i[0]) : (float)L.h2i[0];
    const float hy = iso ? hx : (float)L.h2i[1], hz = iso ? hx : (float)L.h2i[2];
    if constexpr (!COR) {
        if (L.face) {
            if (ci == 4) launch_ci<true, 4, PRO, false, true>(grid, L, hx, hy, hz, u_old, u_new, f, a, uc, dc, u64, st);
            else if (ci == 8) launch_ci<true, 8, PRO, false, true>(grid, L, hx, hy, hz, u_old, u_new, f, a, uc, dc, u64, st);
            else launch_ci<true, 16, PRO, false, true>(grid, L, hx, hy, hz, u_old, u_new, f, a, uc, dc, u64, st);
            return;
        }
    }
#define RECON_SWEEP_CI(CI)                                                                          \
    (iso ? launch_ci<true, CI, PRO, COR>(grid, L, hx, hy, hz, u_old, u_new, f, a, uc, dc, u64, st)   \
         : launch_ci<false, CI, PRO, COR>(grid, L, hx, hy, hz, u_old, u_new, f, a, uc, dc, u64, st))
    if (ci == 4) RECON_SWEEP_CI(4);
    else if (ci == 8) RECON_SWEEP_CI(8);
    else RECON_SWEEP_CI(16);
#undef RECON_SWEEP_CI
}

bool stream_fits(const Dims& d) { return d.n2 % TK == 0 && d.n1 % TJ == 0 && d.n0 % kCIs[0] == 0; }

bool iso_level(const Level& L) { return L.h2i[0] == L.h2i[1] && L.h2i[1] == L.h2i[2]; }

}  // namespace

// One sweep u_new <- RBGS(u_old) in one pass when the level is a multiple of
// the tile; returns the number of sweeps done (1), or 0 with nothing launched.
template <>
int launch_rbgs_fused<float>(const Level& L, const float* u_old, float* u_new, const float* f,
                             const float* a, int nsweeps, cudaStream_t st) {
    if (nsweeps < 1 || !stream_fits(L.d) || (L.face && !iso_level(L))) return 0;
    launch_sweep<false, false>(L, u_old, u_new, f, a, nullptr, L.d, nullptr, st);
    return 1;
}

bool rbgs_prolong_fits(const Level& fine) {
    return fine.coarsen[0] && fine.coarsen[1] && fine.coarsen[2] && stream_fits(fine.d);
}

// The first post-smoothing sweep with the coarse correction folded in:
// u_new <- RBGS(u_old + P(uc)), and with u64 also u64 += u_new; returns 1,
// or 0 with nothing launched.
int launch_rbgs_prolong(const Level& fine, const Level& coarse, const float* uc, const float* u_old,
                        float* u_new, const float* f, const float* a, cudaStream_t st, double* u64) {
    if (!rbgs_prolong_fits(fine) || !u_old || (fine.face && !iso_level(fine))) return 0;
    if (u64)
        launch_sweep<true, true>(fine, u_old, u_new, f, a, uc, coarse.d, u64, st);
    else
        launch_sweep<true, false>(fine, u_old, u_new, f, a, uc, coarse.d, nullptr, st);
    return 1;
}

// A sweep that also adds its result to the FP64 field u64:
// u_new <- RBGS(u_old), u64 += u_new; returns 1, or 0 with nothing launched.
int launch_rbgs_correct(const Level& L, const float* u_old, float* u_new, const float* f,
                        const float* a, double* u64, cudaStream_t st) {
    if (!stream_fits(L.d) || !u_old || L.face) return 0;
    launch_sweep<false, true>(L, u_old, u_new, f, a, nullptr, L.d, u64, st);
    return 1;
}

void tune_sweep_level(Level& L, const Level* coarse, const float* uc, float* u, float* w,
                      const float* f, const float* a, cudaStream_t st) {
    if (!stream_fits(L.d) || (L.face && !iso_level(L))) return;
    for (int pro = 0; pro < 2; ++pro) {
        if (pro && !(coarse && uc && rbgs_prolong_fits(L))) continue;
        float best_ms = 0.f;
        int best = 0;
        // two rounds over the candidates, the first only bringing the clocks
        // up, so that the kept timings compare like with like
        for (int round = 0; round < 2; ++round)
            for (int ci : kCIs) {
                if (L.d.n0 % ci) continue;
                const float ms = time_launches(st, 5, [&] {
                    if (pro)
                        launch_sweep<true, false>(L, u, w, f, a, uc, coarse->d, nullptr, st, ci);
                    else
                        launch_sweep<false, false>(L, u, w, f, a, nullptr, L.d, nullptr, st, ci);
                });
                if (round == 1 && (!best || ms < best_ms)) best = ci, best_ms = ms;
            }
        L.tune[pro] = best;
    }
}

bool encode_grid_map(CUtensorMap* map, const float* base, int n0, int n1, int n2, int box_k, int box_j) {
    using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Encode fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (Encode)p;
        cudaGetLastError();
    });
    if (!fn || ((uintptr_t)base & 15)) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)n2, (cuuint64_t)n1, (cuuint64_t)n0};
    const cuuint64_t strides[2] = {(cuuint64_t)n2 * sizeof(float), (cuuint64_t)n2 * n1 * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)box_k, (cuuint32_t)box_j, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int bounds_fail_smoother() { return bounds_fail_take(); }

bool sweep_wait_failed() {
    int v = 0;
    const int zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_sweep_wait_fail, sizeof(int)) != cudaSuccess) return false;
    if (v) cudaMemcpyToSymbol(g_sweep_wait_fail, &zero, sizeof(int));
    return v != 0;
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
