// hobo_energy_fp64_noalloc: the float64 re-score without any allocation.
//
// Some callers cannot let a library allocate device memory: applications
// whose device memory is entirely reserved up front by their own pool (a
// framework's caching allocator, a fixed arena on a shared GPU), where any
// further allocation fails or fragments the pool, and latency-critical
// loops that must not risk the implicit synchronisation or the pool growth
// an allocation can bring.  For them this entry point keeps its scratch, the
// 64-bit integer accumulators of the re-score, in a fixed array in device
// memory declared at file scope, which the CUDA driver sets aside once for every
// GPU that loads the library and keeps until the process exits.
//
// Every call shares that one array per device, and the array keeps whatever
// the last call left in it: each call clears the words it uses before its
// kernels run.  Two calls whose work overlaps on the GPU (on different
// streams, without ordering between them) race on the array and give wrong
// results; callers must order them, for example by issuing them on one
// stream.
#include <string>
#include "hobo_internal.h"

namespace hobo {

// Largest batch one call accepts: 65,536 states x 8 bytes = 512 KiB per GPU.
constexpr int kNoAllocMaxStates = HOBO_NOALLOC_MAX_B;

static __device__ __align__(256) unsigned long long g_fix_scratch[kNoAllocMaxStates];

// Device address of g_fix_scratch on the current device.  In host code the
// symbol is only a stand-in and must never be passed to a kernel.  The
// address is looked up on every call, with the call's device current: after
// the first lookup on a device (which may load the library's device code
// there, so make that first call before any stream capture) it is a cheap
// host-side query, and no address is kept that a device reset could leave
// stale.
static cudaError_t scratch_for_current_device(void** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_fix_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

}  // namespace hobo

using namespace hobo;

static int hobo_energy_fp64_noalloc_impl(hobo_h h, const uint32_t* X, int B, double* E, void* stream)
{
    if (!h) { set_error("NULL instance"); return HOBO_ERR_ARG; }
    if (B < 0 || (B > 0 && (!X || !E))) { set_error("bad X/E/B"); return HOBO_ERR_ARG; }
    if (B > kNoAllocMaxStates) {
        set_error("hobo_energy_fp64_noalloc: B = " + std::to_string(B) + " exceeds the fixed scratch of " +
                  std::to_string(kNoAllocMaxStates) + " states");
        return HOBO_ERR_ARG;
    }
    if (B == 0) return HOBO_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess && dev != h->device) {
        set_error("hobo_energy_fp64_noalloc: the instance lives on another device than the current one");
        return HOBO_ERR_ARG;
    }
    void* scratch = nullptr;
    if (e == cudaSuccess) e = scratch_for_current_device(&scratch);
    cudaStream_t st = (cudaStream_t)stream;
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * (size_t)B, st);
    if (e == cudaSuccess)
        e = launch_energy_fp64_into(h, X, B, E, static_cast<unsigned long long*>(scratch), st);
    if (e != cudaSuccess) {
        set_error(std::string("hobo_energy_fp64_noalloc: ") + cudaGetErrorString(e));
        return HOBO_ERR_CUDA;
    }
    set_error("");
    return HOBO_OK;
}

// Under the same guard as the other entry points: the error messages build
// host strings, and the exact re-score's launcher a small host vector, so a
// failed host allocation becomes HOBO_ERR_OOM instead of an exception
// crossing the C ABI.
extern "C" int hobo_energy_fp64_noalloc(hobo_h h, const uint32_t* X, int B, double* E, void* stream)
{
    return hobo::guarded("hobo_energy_fp64_noalloc",
                         [&] { return hobo_energy_fp64_noalloc_impl(h, X, B, E, stream); });
}
