// async_copy.cuh -- 16-byte global-to-shared copies that bypass L1
// (cp.async.cg), used by the streaming stencil kernels to fetch the next plane
// while the current one is computed.
#pragma once

namespace recon {

__device__ inline void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ inline void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ inline void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }
// all but the most recently committed group complete
__device__ inline void cp_wait_prior() { asm volatile("cp.async.wait_group 1;\n" ::); }

}  // namespace recon
