// Instantiations of the learned-proposal sweep kernel (N <= 256).
#include "sweep_impl.cuh"

namespace hobo {

#define HOBO_LEARNED_DISPATCH(DENSE, KU)                                                          \
    template <>                                                                                 \
    cudaError_t dispatch_learned<DENSE, KU>(const SweepDev& p, const LearnedDev& L, cudaStream_t st) \
    {                                                                                           \
        if (p.W <= 1) return run_learned<1, DENSE, KU>(p, L, st);                               \
        if (p.W <= 2) return run_learned<2, DENSE, KU>(p, L, st);                               \
        if (p.W <= 4) return run_learned<4, DENSE, KU>(p, L, st);                               \
        return run_learned<8, DENSE, KU>(p, L, st);                                             \
    }

HOBO_LEARNED_DISPATCH(true, 1)
HOBO_LEARNED_DISPATCH(false, 1)
HOBO_LEARNED_DISPATCH(false, 2)
HOBO_LEARNED_DISPATCH(false, 6)

}  // namespace hobo
