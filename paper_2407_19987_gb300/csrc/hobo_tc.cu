// tcgen05 tensor-core contraction of dense order-3 instances (placeholder:
// reports "not supported" until the kernel is in place).
#include "hobo_internal.h"

namespace hobo {

cudaError_t launch_energy_tc(const hobo_instance* h, const uint32_t* X, int B, float* E,
                             float* g_or_dE, bool flip_out, cudaStream_t st)
{
    (void)h; (void)X; (void)B; (void)E; (void)g_or_dE; (void)flip_out; (void)st;
    return cudaErrorNotSupported;
}

}  // namespace hobo
