// Instantiations of the tuned sweep kernel: dense order-3 slabs.
#include "sweep_impl.cuh"

namespace hobo {

template <>
cudaError_t dispatch_tuned<true, 1>(const SweepDev& p, cudaStream_t st)
{
    if (p.W <= 1) return run_tuned<1, true, 1>(p, st);
    if (p.W <= 2) return run_tuned<2, true, 1>(p, st);
    if (p.W <= 4) return run_tuned<4, true, 1>(p, st);
    if (p.W <= 8) return run_tuned<8, true, 1>(p, st);
    return run_tuned<16, true, 1>(p, st);
}

}  // namespace hobo
