// Pair-sum kernel instantiations for the double-layer (paper Eq. stokes-dl) kind.
#include "pairsum_kernels.cuh"

namespace sbq {

cudaError_t launch_pairsum_dl(int prec, int R, int W, int grid, const PairsumParams &p,
                              cudaStream_t s)
{
    return KindLauncher<KIND_DL>::launch(prec, R, W, grid, p, s);
}

int occupancy_pairsum_dl(int prec, int R, int W)
{
    return KindLauncher<KIND_DL>::occupancy(prec, R, W);
}

}  // namespace sbq
