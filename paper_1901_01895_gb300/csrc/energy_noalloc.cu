// mmf_energy_noalloc: the per-field energy reduction of mmf_energy for callers that
// cannot allocate device memory.
//
// Who cannot allocate: a process whose device memory is already claimed by another
// framework's caching allocator (a raw cudaMalloc can then fail although the pool
// has room), and latency-critical loops where cudaMalloc/cudaFree are not allowed
// because they synchronise the whole device and stall work on other streams.  Such
// callers pass only their input fields and a device output array; the reduction's
// partial sums go to a fixed buffer compiled into this library instead of memory
// obtained at run time.
//
// The buffer is a file-scope __device__ array of MMF_NOALLOC_ENERGY_MAX doubles
// (128 KiB); every GPU that loads this library holds it until the process exits.
// Host code cannot use the array's name as a device address, so the first call on
// each device looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it together with the device's current context; a call that finds
// another context current (the device was reset, or its primary context torn down and
// created again) looks the address up again instead of using a stale one.  The first
// call on a device, and the first after such a re-creation, should therefore come before
// any stream capture.  All calls share the one
// buffer: calls whose kernels overlap on the GPU (different streams, no ordering between
// them) race on it and must be serialised by the caller.  Each call overwrites every
// partial sum it later reads, so nothing has to be cleared between calls.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/mmf.h"
#include "kernels.h"

namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_energy_partials[MMF_NOALLOC_ENERGY_MAX];

std::mutex g_mu;
struct Slot {
    CUcontext ctx;      // context current when the address was looked up
    double* ptr;        // device address of g_energy_partials in that context
};
Slot g_slot[kMaxDevices] = {};
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn g_ctx_get_current = nullptr;   // cuCtxGetCurrent, through the runtime

// The calling thread's current context (NULL when none is current yet).
CUcontext current_context() {
    if (!g_ctx_get_current) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        g_ctx_get_current = (CtxGetCurrentFn)fn;
    }
    CUcontext c = nullptr;
    if (g_ctx_get_current(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

int noalloc_fail(int code, const std::string& msg) {
    mmf::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" int mmf_energy_noalloc(const void* fields, int P, int64_t N_t, double dt, double* out_dev, void* stream) {
    mmf::set_last_error("");
    if (!fields || !out_dev) return noalloc_fail(MMF_EINVAL, "fields and out_dev must be device pointers");
    if (P < 1) return noalloc_fail(MMF_EINVAL, "P must be >= 1");
    if (N_t < 16 || N_t > (1 << 17) || (N_t & (N_t - 1))) return noalloc_fail(MMF_EINVAL, "N_t must be a power of two in [16, 131072]");
    if (!(dt > 0) || !std::isfinite(dt)) return noalloc_fail(MMF_EINVAL, "dt must be positive");
    const int nblk = mmf::energy_blocks((int)N_t);
    if ((int64_t)P * nblk > MMF_NOALLOC_ENERGY_MAX)
        return noalloc_fail(MMF_EINVAL, "P * blocks(N_t) = " + std::to_string((int64_t)P * nblk) +
                                            " partial sums exceed the built-in buffer of " +
                                            std::to_string(MMF_NOALLOC_ENERGY_MAX));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(MMF_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(MMF_EINVAL, "device index out of range");
    double* partials = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        Slot& sl = g_slot[dev];
        const CUcontext ctx = current_context();
        if (!sl.ptr || !ctx || ctx != sl.ctx) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_energy_partials);
            if (e != cudaSuccess)
                return noalloc_fail(MMF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            sl.ptr = (double*)p;
            sl.ctx = current_context();   // the lookup makes the device's context current
        }
        partials = sl.ptr;
    }
    e = mmf::energy_launch((const float2*)fields, P, (int)N_t, dt, partials, nblk, out_dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return noalloc_fail(MMF_ECUDA, std::string("energy kernels: ") + cudaGetErrorString(e));
    return MMF_OK;
}
