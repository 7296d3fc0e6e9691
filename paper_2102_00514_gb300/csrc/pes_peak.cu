// FMA throughput probe used as the ALU roofline denominator.
//
// Every thread runs 8 independent FMA chains (enough to cover the FMA
// latency) for a fixed number of rounds; the result is stored so the work is
// not eliminated. Grid: 8 blocks of 256 threads per SM.
#include <cuda_runtime.h>

#include "pes.h"

namespace {

constexpr int kChains = 8;
constexpr int kRounds = 4096;

template <typename T>
__global__ void fma_probe_kernel(T* out, T a, T b)
{
    T acc[kChains];
#pragma unroll
    for (int i = 0; i < kChains; ++i) acc[i] = T(threadIdx.x + i);
#pragma unroll 4
    for (int r = 0; r < kRounds; ++r)
#pragma unroll
        for (int i = 0; i < kChains; ++i) acc[i] = fma(acc[i], a, b);
    T s = T(0);
#pragma unroll
    for (int i = 0; i < kChains; ++i) s += acc[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
double probe(int sms)
{
    const int threads = 256, blocks = sms * 8;
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * threads * blocks) != cudaSuccess) return 0.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // the multiplier keeps values bounded: a = 1 - 2^-20, b = 2^-10
    const T a = T(1) - T(1.0 / 1048576.0), b = T(1.0 / 1024.0);
    fma_probe_kernel<T><<<blocks, threads>>>(out, a, b);   // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(e0);
        fma_probe_kernel<T><<<blocks, threads>>>(out, a, b);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    const double flops = 2.0 * kChains * (double)kRounds * threads * blocks;
    return flops / (best * 1e-3) / 1e9;
}

}  // namespace

extern "C" pes_status pes_measure_fma_peak(double* fp32_gflops, double* fp64_gflops)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PES_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PES_ERR_CUDA;
    if (fp32_gflops) *fp32_gflops = probe<float>(sms);
    if (fp64_gflops) *fp64_gflops = probe<double>(sms);
    return cudaGetLastError() == cudaSuccess ? PES_OK : PES_ERR_CUDA;
}
