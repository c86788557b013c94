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

cudaError_t dispatch_tuned_dense_reuse(const SweepDev& p, cudaStream_t st)
{
    if (p.W <= 1) return run_tuned<1, true, 1, true>(p, st);
    if (p.W <= 2) return run_tuned<2, true, 1, true>(p, st);
    if (p.W <= 4) return run_tuned<4, true, 1, true>(p, st);
    if (p.W <= 8) return run_tuned<8, true, 1, true>(p, st);
    return run_tuned<16, true, 1, true>(p, st);
}

template <>
cudaError_t dispatch_batch<true, 1>(const SweepDev* descs, const int2* items, int nitems, int* counter, int Nmax,
                                  int Wmax, int warps, int ctas, cudaStream_t st)
{
    if (Wmax <= 1) return run_batch<1, true, 1>(descs, items, nitems, counter, Nmax, warps, ctas, st);
    if (Wmax <= 2) return run_batch<2, true, 1>(descs, items, nitems, counter, Nmax, warps, ctas, st);
    if (Wmax <= 4) return run_batch<4, true, 1>(descs, items, nitems, counter, Nmax, warps, ctas, st);
    if (Wmax <= 8) return run_batch<8, true, 1>(descs, items, nitems, counter, Nmax, warps, ctas, st);
    return run_batch<16, true, 1>(descs, items, nitems, counter, Nmax, warps, ctas, st);
}

}  // namespace hobo
