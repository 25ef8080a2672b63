// Pair-sum kernel instantiations for the combined-field eta S + D (paper Eq. stokes-bie-new) kind.
#include "pairsum_kernels.cuh"

namespace sbq {

cudaError_t launch_pairsum_cf(int prec, int R, int W, int grid, const PairsumParams &p,
                              cudaStream_t s)
{
    return KindLauncher<KIND_CF>::launch(prec, R, W, grid, p, s);
}

int occupancy_pairsum_cf(int prec, int R, int W)
{
    return KindLauncher<KIND_CF>::occupancy(prec, R, W);
}

}  // namespace sbq
