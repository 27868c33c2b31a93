// noalloc.cu -- recon_deposit_cic_noalloc: the CIC particle deposit for
// callers that must not allocate device memory.
//
// recon_deposit accumulates particle masses in a 64-bit fixed-point grid and
// reduces partial sums in buffers that the handle allocates.  Some callers
// cannot allocate at the point where they need a deposit: code whose device
// memory is owned by another allocator that must account for every byte (a
// framework's caching allocator, a fixed memory pool), or loops where a
// cudaMalloc / cudaFree would synchronise the device.  For them this file
// keeps the scratch in a file-scope device array of fixed size, resident on
// every GPU that loads the library until the process exits.  The caller still
// passes the inputs and the output.  The call checks its inputs on the host
// after one synchronisation of its stream, so it cannot run inside a stream
// capture.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/recon.h"
#include "recon_internal.cuh"

namespace recon {
int set_last_error(int code, const char* msg);
}

namespace {

using recon::kRedBlocks;

// Largest grid the fixed scratch holds: 128^3 cells (16 MiB of accumulators).
constexpr long long kNoallocMaxCells = 1ll << 21;

struct NoallocScratch {
    unsigned long long acc[kNoallocMaxCells];  // fixed-point mass per cell
    double partials[2][kRedBlocks];            // per-block sums / flags
    double scalars[recon::SC_COUNT];           // finished reductions
};

// The scratch itself.  In host code this name is only a stand-in for the
// device symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

constexpr int kMaxDevices = 256;
std::mutex g_setup_mutex;
NoallocScratch* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does this set-up).  A cudaDeviceReset of
// that device ends the context the address belongs to; the entry point must
// not be used on that device afterwards in the same process.
int scratch_on_current_device(NoallocScratch** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return recon::set_last_error(RECON_E_CUDA, "cudaGetDevice failed");
    }
    if (dev < 0 || dev >= kMaxDevices) return recon::set_last_error(RECON_E_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            char msg[160];
            snprintf(msg, sizeof(msg), "cudaGetSymbolAddress of the deposit scratch failed: %s",
                     cudaGetErrorString(e));
            return recon::set_last_error(RECON_E_CUDA, msg);
        }
        g_scratch_addr[dev] = (NoallocScratch*)p;
    }
    *out = g_scratch_addr[dev];
    return RECON_OK;
}

// Device memory of the current device, or managed memory.
bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

}  // namespace

extern "C" int recon_deposit_cic_noalloc(int n0, int n1, int n2, double cell, const double* pos,
                                         const double* mass, int64_t np, double* rho,
                                         void* cuda_stream) {
    recon::set_last_error(RECON_OK, "");
    if (!pow2_in(n0, 2, 4096) || !pow2_in(n1, 2, 4096) || !pow2_in(n2, 2, 4096))
        return recon::set_last_error(RECON_E_INVALID, "grid dims must be powers of two in [2, 4096]");
    const long long cells = (long long)n0 * n1 * n2;
    if (cells > kNoallocMaxCells) {
        char msg[160];
        snprintf(msg, sizeof(msg),
                 "grid of %lld cells exceeds the %lld-cell (128^3) limit of the allocation-free deposit",
                 cells, kNoallocMaxCells);
        return recon::set_last_error(RECON_E_INVALID, msg);
    }
    if (!(cell > 0.0) || !std::isfinite(cell)) return recon::set_last_error(RECON_E_INVALID, "cell size must be positive");
    if (np <= 0 || !pos || !rho) return recon::set_last_error(RECON_E_INVALID, "need particles, positions and an output");
    if (!on_device(pos) || !on_device(rho) || (mass && !on_device(mass)))
        return recon::set_last_error(RECON_E_INVALID, "pos, mass and rho must be device memory of the current device");
    NoallocScratch* S = nullptr;
    int rc = scratch_on_current_device(&S);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const recon::Dims d = recon::make_dims(n0, n1, n2);

    // total mass and the finite / non-negative check (the scratch keeps the
    // previous call's values, so everything read here is written first)
    recon::launch_validate_particles(np, pos, mass, S->partials[0], S->partials[1], st);
    recon::finish_reduce(S->partials[0], 0, S->scalars, recon::SC_SUM_RHO, st);
    recon::finish_reduce(S->partials[1], 2, S->scalars, recon::SC_BAD, st);
    double host[2] = {0.0, 0.0};
    cudaError_t e = cudaMemcpyAsync(host, S->scalars + recon::SC_SUM_RHO, 2 * sizeof(double),
                                    cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return recon::set_last_error(RECON_E_CUDA, cudaGetErrorString(e));
    }
    if (host[1] != 0.0) return recon::set_last_error(RECON_E_NONFINITE, "particle positions or masses are not finite / negative");
    if (!(host[0] > 0.0)) return recon::set_last_error(RECON_E_INVALID, "total particle mass is zero");
    int ex = 0;
    std::frexp(host[0] > 1.0 ? host[0] : 1.0, &ex);
    const double scale = std::ldexp(1.0, 61 - ex);

    // the accumulators must start at zero; the conversion clears them again
    e = cudaMemsetAsync(S->acc, 0, sizeof(unsigned long long) * cells, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return recon::set_last_error(RECON_E_CUDA, cudaGetErrorString(e));
    }
    recon::launch_deposit_particles(d, np, pos, mass, 1.0 / cell, scale, S->acc, st);
    recon::launch_fix_to_double((int)cells, S->acc, 1.0 / scale, rho, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return recon::set_last_error(RECON_E_CUDA, cudaGetErrorString(e));
    return RECON_OK;
}
