// reduce.cuh -- deterministic block reductions (fixed shuffle tree, fixed
// warp order), used by every kernel that emits per-block partials.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace recon {

struct OpSum {
    __device__ static double id() { return 0.0; }
    __device__ static double op(double a, double b) { return a + b; }
};
struct OpMin {
    __device__ static double id() { return INFINITY; }
    __device__ static double op(double a, double b) { return fmin(a, b); }
};
struct OpMax {
    __device__ static double id() { return -INFINITY; }
    __device__ static double op(double a, double b) { return fmax(a, b); }
};

// Reduce v over the block; the result is valid in thread 0.  blockDim.x must
// be a multiple of 32 and at most 1024.
template <class Op>
__device__ inline double block_reduce(double v) {
    __shared__ double warp_part[32];
    for (int o = 16; o > 0; o >>= 1) v = Op::op(v, __shfl_down_sync(0xffffffffu, v, o));
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();  // warp_part may still be read by a previous call
    if (lane == 0) warp_part[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    if (w == 0) {
        v = lane < nw ? warp_part[lane] : Op::id();
        for (int o = 16; o > 0; o >>= 1) v = Op::op(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    return v;
}

}  // namespace recon
