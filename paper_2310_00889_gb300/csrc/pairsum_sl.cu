// Pair-sum kernel instantiations for the single-layer (paper Eq. stokes-sl) kind.
#include "pairsum_kernels.cuh"

namespace sbq {

cudaError_t launch_pairsum_sl(int prec, int R, int W, int grid, const PairsumParams &p,
                              cudaStream_t s)
{
    return KindLauncher<KIND_SL>::launch(prec, R, W, grid, p, s);
}

int occupancy_pairsum_sl(int prec, int R, int W)
{
    return KindLauncher<KIND_SL>::occupancy(prec, R, W);
}

}  // namespace sbq
