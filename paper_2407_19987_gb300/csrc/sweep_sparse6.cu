// Instantiations of the tuned sweep kernel: term lists, up to six conditions per entry (order 5..8).
#include "sweep_impl.cuh"

namespace hobo {

template <>
cudaError_t dispatch_tuned<false, 6>(const SweepDev& p, cudaStream_t st)
{
    if (p.W <= 1) return run_tuned<1, false, 6>(p, st);
    if (p.W <= 2) return run_tuned<2, false, 6>(p, st);
    if (p.W <= 4) return run_tuned<4, false, 6>(p, st);
    if (p.W <= 8) return run_tuned<8, false, 6>(p, st);
    if (p.W <= 16) return run_tuned<16, false, 6>(p, st);
    return run_tuned<32, false, 6>(p, st);
}

template <>
cudaError_t dispatch_batch<false, 6>(const SweepDev* descs, const int2* items, int nitems, int* counter, int Nmax,
                                  int Wmax, int warps, int ctas, cudaStream_t st)
{
    if (Wmax <= 1) return run_batch<1, false, 6>(descs, items, nitems, counter, Nmax, warps, ctas, st);
    if (Wmax <= 2) return run_batch<2, false, 6>(descs, items, nitems, counter, Nmax, warps, ctas, st);
    if (Wmax <= 4) return run_batch<4, false, 6>(descs, items, nitems, counter, Nmax, warps, ctas, st);
    if (Wmax <= 8) return run_batch<8, false, 6>(descs, items, nitems, counter, Nmax, warps, ctas, st);
    if (Wmax <= 16) return run_batch<16, false, 6>(descs, items, nitems, counter, Nmax, warps, ctas, st);
    return run_batch<32, false, 6>(descs, items, nitems, counter, Nmax, warps, ctas, st);
}

}  // namespace hobo
