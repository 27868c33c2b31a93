// tma.cuh -- tiled bulk tensor copies (the Tensor Memory Accelerator) from
// global into shared memory, completed on a shared-memory mbarrier, and the
// host-side construction of their tensor maps.  Every wait is bounded: after
// about a second it gives up, records the failure in a device word that the
// host reads after the solve (RECON_E_TIMEOUT) and returns.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace recon {

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// makes the initialised barriers visible to the async proxy (the copies)
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// one arrival that also announces `bytes` of copies completing on this phase
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(unsigned long long* bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Waits for the phase of `bar` with the given parity to complete; false
// (and *fail set) if it has not after ~1 s.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* fail) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try(bar, parity))
        if (global_ns() - t0 > 1000000000ull) {
            atomicExch(fail, 1);
            return false;
        }
    return true;
}

// orders this thread's earlier generic-proxy accesses of shared memory
// (after a barrier: the whole block's) before later bulk copies into it
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// box of a rank-3 map at element coordinates (x, y, z), x innermost
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// A rank-3 FP32 map of an n0 x n1 x n2 grid (n2 fastest) whose box is
// box_k x box_j x 1 elements.  False where the driver offers no encoder or
// refuses the map (the caller then stages by per-thread copies).
bool encode_grid_map(CUtensorMap* map, const float* base, int n0, int n1, int n2, int box_k, int box_j);

}  // namespace recon
