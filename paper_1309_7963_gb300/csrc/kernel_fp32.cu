// FP32 bulk mode (compiled with --use_fast_math, which affects single precision only):
// transport, free paths and cross sections in float; collision boosts, event bookkeeping
// and evaporation widths stay in double.
#include "pnuc_kernels.cuh"

namespace pnuc {

cudaError_t launch_plain_fp32(const SimParams &p, int block, bool count, cudaStream_t s)
{
    return count ? dev::launch_plain<float, true>(p, block, s) : dev::launch_plain<float, false>(p, block, s);
}
cudaError_t launch_persistent_fp32(const SimParams &p, int grid, int block, bool count, cudaStream_t s)
{
    return count ? dev::launch_persistent<float, true>(p, grid, block, s)
                 : dev::launch_persistent<float, false>(p, grid, block, s);
}
cudaError_t launch_evap_fp32(const SimParams &p, int grid, int block, bool count, cudaStream_t s)
{
    return count ? dev::launch_evap<float, true>(p, grid, block, s) : dev::launch_evap<float, false>(p, grid, block, s);
}
int occupancy_persistent_fp32(int block, bool count)
{
    return count ? dev::occupancy_persistent<float, true>(block) : dev::occupancy_persistent<float, false>(block);
}

}  // namespace pnuc
