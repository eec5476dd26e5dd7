// FP32 bulk modes (compiled with --use_fast_math, which affects single precision only):
// transport, free paths, cross sections, channel parameters, the emission sampler and the
// evaporation decay in float; the NN collision boosts and the event's energy/momentum
// bookkeeping in double. PNUC_FP32 keeps the evaporation widths (their exponentials, the
// channel draw) in double; PNUC_FP32_SCALED evaluates them in float, scaled by the largest
// channel's exponential (the "scaled" evaporation kernels below).
#include "pnuc_kernels.cuh"

namespace pnuc {
namespace dev {
namespace {
// The FP32 cascade kernel capped at 96 registers: five resident 128-thread blocks per SM
// instead of four (3.5% faster on GB300 than the 105 registers it uses unbounded; caps of 80
// and 72 with six and seven blocks measured the same and 4% slower). The evaporation kernel
// fits 96 without spilling (five blocks per SM instead of four; the same time).
__global__ void __maxnreg__(96) persistent_kernel_f32(const SimParams P) { persistent_body<float, false>(P); }
__global__ void __maxnreg__(96) evap_kernel_f32(const SimParams P) { evap_body<float, false, false>(P); }
__global__ void __maxnreg__(96) evap_kernel_f32s(const SimParams P) { evap_body<float, false, true>(P); }
__global__ void __maxnreg__(96) evap_kernel_f32c(const SimParams P) { evap_body<float, false, false, true>(P); }

// The FP32 mode's width exponential on n arguments (pnuc_width_exp): e^x for x in [1, 256),
// -1 for other arguments.
__global__ void width_exp_kernel(const float *x, double *out, uint64_t n)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float v = x[i];
        out[i] = v >= 1.f && v < 256.f ? exp_fixed(v) : -1.0;
    }
}
}  // namespace
}  // namespace dev

cudaError_t launch_width_exp(const float *x, double *out, uint64_t n, int sm_count, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = (n + 255) / 256, cap = (uint64_t)sm_count * 8;
    dev::width_exp_kernel<<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, s>>>(x, out, n);
    return cudaGetLastError();
}

// The kernels that evaporate come in one variant per level density (SimParams.level_density:
// the Fermi gas, or the constant-temperature composite), so that the option's code is not in
// the default kernels.
cudaError_t launch_plain_fp32(const SimParams &p, int block, bool count, bool scaled, cudaStream_t s)
{
    if (p.level_density == 1)
        return count ? dev::launch_plain<float, true, false, true>(p, block, s)
                     : dev::launch_plain<float, false, false, true>(p, block, s);
    if (scaled)
        return count ? dev::launch_plain<float, true, true>(p, block, s) : dev::launch_plain<float, false, true>(p, block, s);
    return count ? dev::launch_plain<float, true>(p, block, s) : dev::launch_plain<float, false>(p, block, s);
}
cudaError_t launch_persistent_fp32(const SimParams &p, int grid, int block, bool count, cudaStream_t s)
{
    if (count) return dev::launch_persistent<float, true>(p, grid, block, s);
    return dev::launch_kernel(dev::persistent_kernel_f32, dev::persistent_smem_bytes<float>(p.n_targets, block), p, grid,
                              block, s);
}
cudaError_t launch_evap_fp32(const SimParams &p, int grid, int block, bool count, bool scaled, cudaStream_t s)
{
    if (p.level_density == 1) {
        if (count) return dev::launch_evap<float, true, false, true>(p, grid, block, s);
        return dev::launch_kernel(dev::evap_kernel_f32c, dev::evap_smem_bytes<float>(p.n_targets, block), p, grid,
                                  block, s);
    }
    if (scaled) {
        if (count) return dev::launch_evap<float, true, true>(p, grid, block, s);
        return dev::launch_kernel(dev::evap_kernel_f32s, dev::evap_smem_bytes<float, true>(p.n_targets, block), p,
                                  grid, block, s);
    }
    if (count) return dev::launch_evap<float, true>(p, grid, block, s);
    return dev::launch_kernel(dev::evap_kernel_f32, dev::evap_smem_bytes<float>(p.n_targets, block), p, grid, block, s);
}
cudaError_t launch_sorted_fp32(const SimParams &p, void *stacks, int grid, int block, bool count, cudaStream_t s)
{
    return count ? dev::launch_sorted<float, true>(p, stacks, grid, block, s)
                 : dev::launch_sorted<float, false>(p, stacks, grid, block, s);
}
int occupancy_sorted_fp32(int block, bool count)
{
    return count ? dev::occupancy_sorted<float, true>(block) : dev::occupancy_sorted<float, false>(block);
}
size_t sorted_stack_bytes_fp32() { return sizeof(dev::Particle<float>) * kStackCap; }
int occupancy_evap_fp32(int block, bool count, bool scaled, bool ct)
{
    if (ct) {
        if (count) return dev::occupancy_evap<float, true, false, true>(block);
        return dev::occupancy_of(dev::evap_kernel_f32c, dev::evap_smem_bytes<float>(kMaxTargets, block), block);
    }
    if (scaled) {
        if (count) return dev::occupancy_evap<float, true, true>(block);
        return dev::occupancy_of(dev::evap_kernel_f32s, dev::evap_smem_bytes<float, true>(kMaxTargets, block), block);
    }
    if (count) return dev::occupancy_evap<float, true>(block);
    return dev::occupancy_of(dev::evap_kernel_f32, dev::evap_smem_bytes<float>(kMaxTargets, block), block);
}
int occupancy_persistent_fp32(int block, bool count)
{
    if (count) return dev::occupancy_persistent<float, true>(block);
    return dev::occupancy_of(dev::persistent_kernel_f32, dev::persistent_smem_bytes<float>(kMaxTargets, block), block);
}

}  // namespace pnuc
