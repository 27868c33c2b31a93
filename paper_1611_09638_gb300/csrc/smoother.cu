// smoother.cu -- one full red-black Gauss-Seidel sweep (red, then black) of
// L u = f (App. A, Eq. elliptic with x ~ xi; the 7-point variable-coefficient
// operator with face coefficients (a + a_nbr)/2) in a single pass over memory.
//
// Each block owns a TJ x TK tile of the (j, k) plane and streams CI planes
// along i.  The red update of plane q is computed on the tile plus a one-node
// ring (it needs old values on a two-node ring), the black update of plane
// q - 1 then reads those red values from shared memory, and plane q - 1 of the
// tile is written out.  u is read from u_old and written to u_new (a second
// buffer), so halos read by a block are never values another block has
// already updated: the result equals the in-place sweep node for node.
// Shared memory holds rings of five u and a planes (tile + two-node ring)
// and three f planes; plane q+2 is fetched with cp.async while planes q and
// q-1 are updated.  DRAM traffic is one read of u, a, f and one write of u.
#include "recon_internal.cuh"

namespace recon {

namespace {

__device__ inline void cp_async4(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ inline void cp_async8(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ inline void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ inline void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

template <typename T>
__device__ inline void cp_async_elem(T* smem, const T* gmem) {
    if constexpr (sizeof(T) == 4) cp_async4(smem, gmem);
    else cp_async8(smem, gmem);
}

template <typename T, int TJ, int TK, int NT>
__global__ void __launch_bounds__(NT) k_rbgs_fused(Dims d, T hx, T hy, T hz, int CI,
                                                   const T* __restrict__ u_old,
                                                   T* __restrict__ u_new,
                                                   const T* __restrict__ f,
                                                   const T* __restrict__ a) {
    constexpr int RJ = TJ + 4, RK = TK + 4, PL = RJ * RK;  // tile + 2-node ring
    constexpr int R1J = TJ + 2, R1K = TK + 2;              // tile + 1-node ring
    extern __shared__ unsigned char smem_raw[];
    T* su = reinterpret_cast<T*>(smem_raw);  // u planes, ring of 5
    T* sa = su + 5 * PL;                      // a planes, ring of 5
    T* sf = sa + 5 * PL;                      // f planes, ring of 3
    const int k0 = blockIdx.x * TK, j0 = blockIdx.y * TJ, i0 = blockIdx.z * CI;
    const int iend = i0 + CI;
    const int base = i0 - 2;  // first plane held

    // While plane q is being updated, planes q-2 .. q+1 of u and a and planes
    // q-1, q of f are live; plane q+2 and f of q+1 are fetched meanwhile.
    auto su_of = [&](int q) { return su + ((q - base) % 5) * PL; };
    auto sa_of = [&](int q) { return sa + ((q - base) % 5) * PL; };
    auto sf_of = [&](int q) { return sf + ((q - base) % 3) * PL; };
    auto fetch_ua = [&](int q) {
        T* du = su_of(q);
        T* da = sa_of(q);
        for (int e = threadIdx.x; e < PL; e += NT) {
            const int r = e / RK;
            const int g = cell_index(d, q, j0 + r - 2, k0 + (e - r * RK) - 2);
            cp_async_elem(du + e, u_old + g);
            cp_async_elem(da + e, a + g);
        }
    };
    auto fetch_f = [&](int q) {
        T* df = sf_of(q);
        for (int e = threadIdx.x; e < R1J * R1K; e += NT) {
            const int r = e / R1K, c = e - r * R1K;
            const int g = cell_index(d, q, j0 + r - 1, k0 + c - 1);
            cp_async_elem(df + (r + 1) * RK + (c + 1), f + g);
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
        return (off - sf_of(q)[e]) / diag;
    };

    // prologue: u, a of planes i0-2 .. i0; f of plane i0-1
    fetch_ua(i0 - 2);
    fetch_ua(i0 - 1);
    fetch_ua(i0);
    fetch_f(i0 - 1);
    cp_commit();
    cp_wait_all();
    __syncthreads();

    for (int q = i0 - 1; q <= iend; ++q) {
        if (q + 2 <= iend + 1) fetch_ua(q + 2);
        if (q + 1 <= iend) fetch_f(q + 1);
        cp_commit();
        // red update of plane q on the tile + 1-node ring (reads old black)
        {
            constexpr int NR = R1K / 2;  // red nodes per ring row
            T* uq = su_of(q);
            for (int r = threadIdx.x; r < R1J * NR; r += NT) {
                const int row = r / NR, c = r - row * NR;
                const int jj = row - 1;
                const int s = (q + j0 + jj + k0 - 1) & 1;
                const int kk = -1 + 2 * c + s;
                const int e = (jj + 2) * RK + (kk + 2);
                uq[e] = gs(q, e);
            }
        }
        __syncthreads();
        // black update of plane p = q-1 on the tile, then write the tile
        const int p = q - 1;
        if (p >= i0) {
            constexpr int NB = TK / 2;
            T* upl = su_of(p);
            for (int b = threadIdx.x; b < TJ * NB; b += NT) {
                const int jj = b / NB, c = b - jj * NB;
                const int s = (p + j0 + jj + k0 + 1) & 1;
                const int kk = 2 * c + s;
                const int e = (jj + 2) * RK + (kk + 2);
                upl[e] = gs(p, e);
            }
            __syncthreads();
            for (int e = threadIdx.x; e < TJ * TK; e += NT) {
                const int jj = e / TK, kk = e - jj * TK;
                u_new[cell_index(d, p, j0 + jj, k0 + kk)] = upl[(jj + 2) * RK + (kk + 2)];
            }
        }
        cp_wait_all();
        __syncthreads();
    }
}

template <typename T, int TJ, int TK, int NT>
int smem_bytes() {
    return (int)sizeof(T) * 13 * (TJ + 4) * (TK + 4);
}

template <typename T, int TJ, int TK, int NT>
bool launch_fused(const Level& L, const T* u_old, T* u_new, const T* f, const T* a, int CI,
                  cudaStream_t st) {
    const Dims& d = L.d;
    if (d.n2 % TK || d.n1 % TJ || d.n0 % CI) return false;
    const int sm = smem_bytes<T, TJ, TK, NT>();
    static bool configured = false;
    if (!configured) {
        cudaFuncSetAttribute(k_rbgs_fused<T, TJ, TK, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        configured = true;
    }
    dim3 grid(d.n2 / TK, d.n1 / TJ, d.n0 / CI);
    launch_counter()++;
    k_rbgs_fused<T, TJ, TK, NT><<<grid, NT, sm, st>>>(d, (T)L.h2i[0], (T)L.h2i[1], (T)L.h2i[2], CI,
                                                       u_old, u_new, f, a);
    return true;
}

}  // namespace

// One full sweep u_new <- RBGS(u_old) when the level is a multiple of the
// tile; returns false (nothing launched) otherwise.
template <>
bool launch_rbgs_fused<float>(const Level& L, const float* u_old, float* u_new, const float* f,
                              const float* a, cudaStream_t st) {
    return launch_fused<float, 8, 64, 256>(L, u_old, u_new, f, a, 16, st);
}
template <>
bool launch_rbgs_fused<double>(const Level& L, const double* u_old, double* u_new, const double* f,
                               const double* a, cudaStream_t st) {
    return launch_fused<double, 8, 32, 128>(L, u_old, u_new, f, a, 16, st);
}

}  // namespace recon
