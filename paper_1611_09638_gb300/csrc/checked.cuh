// checked.cuh -- index bounds checks of the RECON_CHECKED build.
//
// Built with -DRECON_CHECKED (librecon_checked.so), every shared-memory and
// global offset the streaming and tiled kernels compute is checked against
// the extent of the array it addresses before use.  A failed check never
// traps: it records the check's id in a device word of its translation unit
// (the first failure wins) and replaces the offset by 0, so the access stays
// inside the array and the kernel runs to its end.  recon_solve then returns
// RECON_E_CUDA naming the id.  Without RECON_CHECKED the checks compile to
// nothing and the offsets are used as computed.
#pragma once

#include <cuda_runtime.h>

namespace recon {

#ifdef RECON_CHECKED
// the first failed check of this translation unit (0: none)
static __device__ int g_bounds_fail;

__device__ __forceinline__ int checked_offset(long long idx, long long limit, int id) {
    if (idx < 0 || idx >= limit) {
        atomicCAS(&g_bounds_fail, 0, id);
        return 0;
    }
    return (int)idx;
}

// Reads and clears this translation unit's record (the current device).
static inline int bounds_fail_take() {
    int v = 0;
    const int zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_bounds_fail, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (v) cudaMemcpyToSymbol(g_bounds_fail, &zero, sizeof(int));
    return v;
}
// idx checked to lie in [0, limit): the offset, or 0 with the failure recorded
#define RC_OFF(idx, limit, id) ::recon::checked_offset((long long)(idx), (long long)(limit), (id))
#else
static inline int bounds_fail_take() { return 0; }
#define RC_OFF(idx, limit, id) (idx)
#endif

}  // namespace recon
