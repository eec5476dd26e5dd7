// FP32 persistent kernel with per-thread register caps of 80 and 64 (6 and 8 resident
// 128-thread blocks per SM), compiled with --use_fast_math like kernel_fp32.cu.
#include "pnuc_kernels.cuh"

namespace pnuc {

cudaError_t launch_persistent_fp32_capped(const SimParams &p, int grid, int block, int max_registers, cudaStream_t s)
{
    if (max_registers == 80) return dev::launch_persistent_capped<float, false, 6>(p, grid, block, s);
    return dev::launch_persistent_capped<float, false, 8>(p, grid, block, s);
}
int occupancy_persistent_fp32_capped(int block, int max_registers)
{
    if (max_registers == 80) return dev::occupancy_persistent_capped<float, false, 6>(block);
    return dev::occupancy_persistent_capped<float, false, 8>(block);
}

}  // namespace pnuc
