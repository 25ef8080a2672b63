// Pair-sum kernel instantiations for the Laplace kinds (paper Sec. 4.1: single layer
// G = 1/(4 pi |r|), double layer dG/dn_y, combined field of Eq. laplace-bie-rep-new).
#include "pairsum_kernels.cuh"

namespace sbq {

cudaError_t launch_pairsum_laplace(int kind, int prec, int R, int W, int grid,
                                   const PairsumParams &p, cudaStream_t s)
{
    switch (kind) {
    case KIND_LSL: return KindLauncher<KIND_LSL>::launch(prec, R, W, grid, p, s);
    case KIND_LDL: return KindLauncher<KIND_LDL>::launch(prec, R, W, grid, p, s);
    case KIND_LCF: return KindLauncher<KIND_LCF>::launch(prec, R, W, grid, p, s);
    default: return cudaErrorInvalidValue;
    }
}

int occupancy_pairsum_laplace(int kind, int prec, int R, int W)
{
    switch (kind) {
    case KIND_LSL: return KindLauncher<KIND_LSL>::occupancy(prec, R, W);
    case KIND_LDL: return KindLauncher<KIND_LDL>::occupancy(prec, R, W);
    case KIND_LCF: return KindLauncher<KIND_LCF>::occupancy(prec, R, W);
    default: return 0;
    }
}

}  // namespace sbq
