// FP64 deterministic mode: every step in double precision, compiled with --fmad=false so
// that the arithmetic is the plain IEEE sequence of the CPU oracle (results differ only
// where CUDA's and the host's libm round transcendental functions differently).
#include "pnuc_kernels.cuh"

namespace pnuc {

// one variant per level density (SimParams.level_density), as in kernel_fp32.cu
cudaError_t launch_plain_fp64(const SimParams &p, int block, cudaStream_t s)
{
    if (p.level_density == 1) return dev::launch_plain<double, true, false, true>(p, block, s);
    return dev::launch_plain<double, true>(p, block, s);
}
cudaError_t launch_persistent_fp64(const SimParams &p, int grid, int block, cudaStream_t s)
{
    return dev::launch_persistent<double, true>(p, grid, block, s);
}
cudaError_t launch_evap_fp64(const SimParams &p, int grid, int block, cudaStream_t s)
{
    if (p.level_density == 1) return dev::launch_evap<double, true, false, true>(p, grid, block, s);
    return dev::launch_evap<double, true>(p, grid, block, s);
}
int occupancy_persistent_fp64(int block) { return dev::occupancy_persistent<double, true>(block); }
int occupancy_evap_fp64(int block, bool ct)
{
    return ct ? dev::occupancy_evap<double, true, false, true>(block) : dev::occupancy_evap<double, true>(block);
}
cudaError_t launch_sorted_fp64(const SimParams &p, void *stacks, int grid, int block, cudaStream_t s)
{
    return dev::launch_sorted<double, true>(p, stacks, grid, block, s);
}
int occupancy_sorted_fp64(int block) { return dev::occupancy_sorted<double, true>(block); }
size_t sorted_stack_bytes_fp64() { return sizeof(dev::Particle<double>) * kStackCap; }

}  // namespace pnuc
