// Launch helpers for one configuration of the persistent kernel; included by
// the per-configuration translation units (pes_k_*.cu), which instantiate them
// explicitly so that the configurations compile in parallel.
#pragma once

#include "pes_internal.h"

namespace pes {

template <typename T, int LIN, int NT>
cudaError_t launch_cfg(const KParams<T>& p, int nb, cudaStream_t st)
{
    auto kern = pes_persistent_kernel<T, LIN, NT>;
    const size_t smem = smem_bytes_for<NT>(sizeof(T));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    KParams<T> pc = p;
    void* args[] = {&pc};
    return cudaLaunchCooperativeKernel((const void*)kern, dim3(nb), dim3(NT), args, smem, st);
}

template <typename T, int LIN, int NT>
int capacity_cfg(int device)
{
    // a failing call returns its negated error code (the caller reports it)
    auto kern = pes_persistent_kernel<T, LIN, NT>;
    const size_t smem = smem_bytes_for<NT>(sizeof(T));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -(int)e;
    int per_sm = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem)) != cudaSuccess) return -(int)e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return -(int)e;
    return per_sm * sms;
}

}  // namespace pes

#define PES_INSTANTIATE(T, LIN, NT)                                                              \
    namespace pes {                                                                              \
    template cudaError_t launch_cfg<T, LIN, NT>(const KParams<T>&, int, cudaStream_t);           \
    template int capacity_cfg<T, LIN, NT>(int);                                                  \
    }
