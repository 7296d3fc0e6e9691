// Host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "pes_kernel.cuh"

namespace pes {

// One configuration of the persistent kernel (defined in pes_launch_impl.cuh,
// instantiated by the pes_k_*.cu translation units).
template <typename T, int LIN, int NT>
cudaError_t launch_cfg(const KParams<T>& p, int nb, cudaStream_t st);
template <typename T, int LIN, int NT>
int capacity_cfg(int device);

// Dispatch over the compiled configurations (pes_dispatch.cu). `lin` is one of
// LIN_ARRAYS / LIN_IEKS / LIN_CUBATURE; `nt` a compiled block size.
cudaError_t launch_persistent(const KParams<float>& p, int lin, int nt, int nb, cudaStream_t st);
cudaError_t launch_persistent(const KParams<double>& p, int lin, int nt, int nb, cudaStream_t st);
// Largest cooperative grid (co-resident blocks on the whole device), 0 if unsupported.
int coop_capacity(float, int lin, int nt, int device);
int coop_capacity(double, int lin, int nt, int device);
// Block sizes compiled per precision.
bool nt_supported(float, int nt);
bool nt_supported(double, int nt);

// Element-wise helpers (pes_aux.cu).
template <typename T>
cudaError_t launch_linearize(const KParams<T>& p, int lin, T* F, T* c, T* Qp, T* H, T* d, T* Rp, T* y_used,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_init_nominal(const int64_t* offsets, int B, int64_t N, const T* m0, const T* P0, T* x, T* P,
                                cudaStream_t st);
// Element-wise precision conversion.
template <typename Ti, typename To>
cudaError_t launch_convert_ff(const Ti* in, To* out, int64_t n, cudaStream_t st);
// Element-wise double -> T copy (model sensors into the kernel precision).
template <typename T>
cudaError_t launch_convert(const double* in, T* out, int n, cudaStream_t st);
// Caller layout [nc][N] <-> lane-major [nc][L][NL] (state k = lane * L + s).
template <typename T>
cudaError_t launch_lanes_transpose(const T* src, T* dst, int nc, int64_t N, int L, int NL, bool to_lanes,
                                   cudaStream_t st);
template <typename T>
cudaError_t launch_init_nominal_lanes(const int64_t* offsets, int B, int64_t N, int L, int NL, const T* m0,
                                      const T* P0, T* x, T* P, cudaStream_t st);
template <typename T, int LIN>
cudaError_t launch_sequential(const KParams<T>& p, cudaStream_t st);

cudaError_t launch_validate_offsets(const int64_t* offsets, int B, int64_t N, int* status, cudaStream_t st);

// Refinement of the final iteration (pes_refine.cu): the forward residual
// elements (`lin` LIN_IEKS or LIN_CUBATURE), the RTS residual elements, and
// the correction scan (cooperative: nb blocks of nt threads, nt 128 or 256).
struct RefineParams;
cudaError_t launch_refine_fwd(const RefineParams& p, int lin, cudaStream_t st);
cudaError_t launch_refine_bwd(const RefineParams& p, cudaStream_t st);
cudaError_t launch_refine_scan(const RefineParams& p, bool fwd, int nt, int nb, cudaStream_t st);
// Largest cooperative grid of the correction scan at nt threads (negated CUDA
// error code on failure).
int refine_scan_capacity(int nt, int device);

}  // namespace pes
