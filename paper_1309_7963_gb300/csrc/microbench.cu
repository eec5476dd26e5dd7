// Pipe-throughput microbenchmarks for the ALU roofline of the event kernels: FP32 FMA,
// FP64 FMA, special-function (reciprocal square root) and 32-bit integer multiply-add
// lane operations per second, each from eight independent dependency chains per thread
// on a grid of 8 x 256-thread blocks per SM.
#include "pnuc_internal.h"

namespace pnuc {
namespace {

constexpr int kChains = 8;

__global__ void peak_ffma(float *out, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3f + c;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5f) out[0] = s;
}

__global__ void peak_dfma(double *out, int iters, double a, double b)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-3 + c;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5) out[0] = s;
}

__global__ void peak_mufu(float *out, int iters)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = 1.f + threadIdx.x * 1e-4f + c;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __frsqrt_rn(x[c]) + 0.75f;
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5f) out[0] = s;
}

__global__ void peak_imad(unsigned *out, int iters, unsigned a, unsigned b)
{
    unsigned x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x + c;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= x[c];
    if (s == 12345u) out[0] = s;
}

template <typename F>
double time_kernel(F launch, int reps)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    launch();  // warm-up
    cudaEventRecord(a);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms * 1e-3 / reps;
}

}  // namespace

cudaError_t measure_peaks(int sm_count, double out[4])
{
    void *buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, 64);
    if (e != cudaSuccess) return e;
    const int blocks = 8 * sm_count, threads = 256;
    const double lanes = (double)blocks * threads * kChains;
    int it_f = 2048, it_d = 256, it_m = 1024, it_i = 2048;
    double t;
    t = time_kernel([&] { peak_ffma<<<blocks, threads>>>((float *)buf, it_f, 0.999f, 0.001f); }, 5);
    out[0] = lanes * it_f / t;
    t = time_kernel([&] { peak_dfma<<<blocks, threads>>>((double *)buf, it_d, 0.999, 0.001); }, 5);
    out[1] = lanes * it_d / t;
    t = time_kernel([&] { peak_mufu<<<blocks, threads>>>((float *)buf, it_m); }, 5);
    out[2] = lanes * it_m / t;
    t = time_kernel([&] { peak_imad<<<blocks, threads>>>((unsigned *)buf, it_i, 1664525u, 1013904223u); }, 5);
    out[3] = lanes * it_i / t;
    e = cudaGetLastError();
    cudaFree(buf);
    return e;
}

}  // namespace pnuc
