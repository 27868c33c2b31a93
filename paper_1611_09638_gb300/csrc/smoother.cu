// smoother.cu -- NS full red-black Gauss-Seidel sweeps (red, then black,
// NS times) of L u = f (App. A, Eq. elliptic with x ~ xi; the 7-point
// variable-coefficient operator with face coefficients (a + a_nbr)/2) in a
// single pass over memory.
//
// Each block owns a TJ x TK tile of the (j, k) plane and streams planes along
// i.  The 2 NS colour updates form a pipeline of stages: at iteration q, stage
// s (colour s % 2, 0 = red) updates plane q - s on the tile grown by a ring of
// 2 NS - 1 - s nodes in j and k.  Every stage reads only values that earlier
// stages (or the initial load, for stage 0) have brought to the state the
// sweep order prescribes, so the result equals NS in-place sweeps node for
// node; the last stage's plane is written out.  u is read from u_old and
// written to u_new (another buffer), so halos read by a block are never values
// another block has already updated.  Shared memory holds rings of u and a
// planes (tile + 2 NS-node ring; rows padded to 16-byte chunks) and of f
// planes; plane q + 2 is fetched with 16-byte cp.async copies while plane q is
// processed.  DRAM traffic for NS sweeps is one read
// of u, a, f and one write of u.  With u_old == nullptr the sweeps start from
// u = 0 and u is not read.
#include "recon_internal.cuh"

namespace recon {

namespace {

__device__ inline void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ inline void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Division of the smoother update: the fast approximate reciprocal in FP32
// (a smoother needs no correctly rounded quotient), IEEE in FP64.
__device__ inline float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ inline double fast_div(double a, double b) { return a / b; }

template <typename T, int NS, int TJ, int TK>
struct SweepShape {
    static constexpr int H = 2 * NS;  // halo of the loaded planes (rows)
    static constexpr int V = 16 / (int)sizeof(T);  // elements per 16-byte copy
    static constexpr int KO = V;      // column halo, rounded up to one 16-byte chunk
    static_assert(H <= KO, "column halo must cover the stencil halo");
    static constexpr int RJ = TJ + 2 * H, RK = TK + 2 * KO, PL = RJ * RK;
    static constexpr int CH = RK / V;  // 16-byte chunks per row
    static constexpr int SU = 2 * NS + 3;  // u / a ring slots
    static constexpr int SF = 2 * NS + 1;  // f ring slots
    static constexpr int smem = (int)sizeof(T) * PL * (2 * SU + SF);
};

__device__ inline void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}

template <typename T, int NS, int TJ, int TK, int NT>
__global__ void __launch_bounds__(NT) k_rbgs_stream(Dims d, T hx, T hy, T hz, int CI,
                                                    const T* __restrict__ u_old,
                                                    T* __restrict__ u_new,
                                                    const T* __restrict__ f,
                                                    const T* __restrict__ a) {
    using S = SweepShape<T, NS, TJ, TK>;
    constexpr int H = S::H, KO = S::KO, V = S::V, CH = S::CH, RK = S::RK, PL = S::PL;
    constexpr int SU = S::SU, SF = S::SF;
    constexpr int NST = 2 * NS;  // stages
    extern __shared__ unsigned char smem_raw[];
    T* su = reinterpret_cast<T*>(smem_raw);
    T* sa = su + SU * PL;
    T* sf = sa + SU * PL;
    const int k0 = blockIdx.x * TK, j0 = blockIdx.y * TJ, i0 = blockIdx.z * CI;
    const int iend = i0 + CI;
    const int q0 = i0 - (NST - 1), q1 = iend - 1 + (NST - 1);
    const int base = q0 - 1;  // first plane held

    auto su_of = [&](int q) { return su + ((q - base) % SU) * PL; };
    auto sa_of = [&](int q) { return sa + ((q - base) % SU) * PL; };
    auto sf_of = [&](int q) { return sf + ((q - base) % SF) * PL; };
    // old u and a of plane q: rows j0-H .. j0+TJ+H-1, columns k0-KO ..
    // k0+TK+KO-1, in 16-byte chunks (n2 is a multiple of the chunk, so a chunk
    // never straddles the periodic seam)
    auto fetch_ua = [&](int q) {
        T* du = su_of(q);
        T* da = sa_of(q);
        for (int e = threadIdx.x; e < S::RJ * CH; e += NT) {
            const int r = e / CH, ch = e - r * CH;
            const int g = cell_index(d, q, j0 + r - H, k0 - KO + ch * V);
            const int o = r * RK + ch * V;
            if (u_old) cp_async16(du + o, u_old + g);
            else *reinterpret_cast<float4*>(du + o) = make_float4(0.f, 0.f, 0.f, 0.f);
            cp_async16(da + o, a + g);
        }
    };
    // f of plane q on the rows of the widest stage region (tile + H - 1)
    auto fetch_f = [&](int q) {
        constexpr int FJ = TJ + 2 * (H - 1);
        T* df = sf_of(q);
        for (int e = threadIdx.x; e < FJ * CH; e += NT) {
            const int r = e / CH, ch = e - r * CH;
            const int g = cell_index(d, q, j0 + r - (H - 1), k0 - KO + ch * V);
            cp_async16(df + (r + 1) * RK + ch * V, f + g);
        }
    };

    const T half = T(0.5);
    // Gauss-Seidel value at smem offset e of plane q from its six neighbours.
    auto gs = [&](int q, int e) -> T {
        const T* uc = su_of(q);
        const T* um = su_of(q - 1);
        const T* up = su_of(q + 1);
        const T* ac = sa_of(q);
        const T* am = sa_of(q - 1);
        const T* ap = sa_of(q + 1);
        const T c = ac[e];
        const T apx = half * (c + ap[e]) * hx, amx = half * (c + am[e]) * hx;
        const T apy = half * (c + ac[e + RK]) * hy, amy = half * (c + ac[e - RK]) * hy;
        const T apz = half * (c + ac[e + 1]) * hz, amz = half * (c + ac[e - 1]) * hz;
        const T diag = (apx + amx) + (apy + amy) + (apz + amz);
        const T off = (apx * up[e] + amx * um[e]) + (apy * uc[e + RK] + amy * uc[e - RK]) +
                      (apz * uc[e + 1] + amz * uc[e - 1]);
        return fast_div(off - sf_of(q)[e], diag);
    };

    // prologue: u, a of planes q0-1 .. q0+1; f of plane q0
    fetch_ua(q0 - 1);
    fetch_ua(q0);
    fetch_ua(q0 + 1);
    fetch_f(q0);
    cp_commit();
    cp_wait_all();
    __syncthreads();

    for (int q = q0; q <= q1; ++q) {
        if (q + 2 <= q1 + 1) fetch_ua(q + 2);
        if (q + 1 <= q1) fetch_f(q + 1);
        cp_commit();
#pragma unroll
        for (int s = 0; s < NST; ++s) {
            const int p = q - s;
            const int ring = NST - 1 - s;  // region: tile + ring
            if (p >= i0 - ring && p <= iend - 1 + ring) {
                const int colour = s & 1;
                const int RJs = TJ + 2 * ring, RKs = TK + 2 * ring;
                const int NC = RKs / 2;  // nodes of one colour per row
                T* upl = su_of(p);
                for (int r = threadIdx.x; r < RJs * NC; r += NT) {
                    const int row = r / NC, c = r - row * NC;
                    const int jj = row - ring;
                    // first kk >= -ring with (p + j + k) of the stage's parity
                    const int sh = (p + j0 + jj + k0 - ring + colour) & 1;
                    const int kk = -ring + 2 * c + sh;
                    const int e = (jj + H) * RK + (kk + KO);
                    upl[e] = gs(p, e);
                }
            }
            __syncthreads();
        }
        const int pout = q - (NST - 1);
        if (pout >= i0 && pout < iend) {
            const T* upl = su_of(pout);
            for (int e = threadIdx.x; e < TJ * TK; e += NT) {
                const int jj = e / TK, kk = e - jj * TK;
                u_new[cell_index(d, pout, j0 + jj, k0 + kk)] = upl[(jj + H) * RK + (kk + KO)];
            }
        }
        cp_wait_all();
        __syncthreads();
    }
}

template <typename T, int NS, int TJ, int TK, int NT>
int launch_stream(const Level& L, const T* u_old, T* u_new, const T* f, const T* a, int CI,
                  cudaStream_t st) {
    const Dims& d = L.d;
    if (d.n2 % TK || d.n1 % TJ || d.n0 % CI) return 0;
    using S = SweepShape<T, NS, TJ, TK>;
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_rbgs_stream<T, NS, TJ, TK, NT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, S::smem);
        configured = true;
    }
    dim3 grid(d.n2 / TK, d.n1 / TJ, d.n0 / CI);
    launch_counter()++;
    k_rbgs_stream<T, NS, TJ, TK, NT><<<grid, NT, S::smem, st>>>(
        d, (T)L.h2i[0], (T)L.h2i[1], (T)L.h2i[2], CI, u_old, u_new, f, a);
    return NS;
}

}  // namespace

// Up to nsweeps sweeps u_new <- RBGS^k(u_old) in one pass when the level is a
// multiple of the tile; returns k, the number of sweeps done (0: nothing
// launched).  The single-sweep kernel is used: fusing two sweeps halves the
// DRAM traffic, but its wider rings and fewer resident blocks made it slower
// per sweep (1.38 vs 1.74 TB/s of algorithmic traffic on the 256^3 level).
template <>
int launch_rbgs_fused<float>(const Level& L, const float* u_old, float* u_new, const float* f,
                             const float* a, int nsweeps, cudaStream_t st) {
    if (nsweeps < 1) return 0;
    return launch_stream<float, 1, 8, 64, 256>(L, u_old, u_new, f, a, 16, st);
}
// FP64 levels are bound by the FP64 issue rate, not by memory: the ring nodes
// the streaming kernel recomputes would cost more than the traffic they save,
// so FP64 sweeps use the in-place two-colour kernel.
template <>
int launch_rbgs_fused<double>(const Level&, const double*, double*, const double*,
                              const double*, int, cudaStream_t) {
    return 0;
}

}  // namespace recon
