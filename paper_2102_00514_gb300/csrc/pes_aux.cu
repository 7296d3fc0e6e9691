// Element-wise kernels around the persistent smoother: offsets validation,
// nominal initialisation and the stand-alone linearisation (Eqs. 7-10).
#include <algorithm>

#include "pes_internal.h"

namespace pes {

// Grid-stride over the B gaps; any malformed entry raises ST_BADARG.
__global__ void validate_offsets_kernel(const int64_t* offsets, int B, int64_t N, int* status)
{
    const int stride = gridDim.x * blockDim.x;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += stride) {
        const int64_t lo = offsets[b], hi = offsets[b + 1];
        bool bad = !(hi > lo);
        if (b == 0 && lo != 0) bad = true;
        if (b == B - 1 && hi != N) bad = true;
        if (bad) atomicOr(status, ST_BADARG);
    }
}

cudaError_t launch_validate_offsets(const int64_t* offsets, int B, int64_t N, int* status, cudaStream_t st)
{
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((B + threads - 1) / threads, 4096);
    validate_offsets_kernel<<<blocks, threads, 0, st>>>(offsets, B, N, status);
    return cudaGetLastError();
}

// One thread per state: locate its trajectory by binary search.
PES_DEV int traj_of(const int64_t* offsets, int B, int64_t k)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(offsets + mid) <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__global__ void convert_kernel(const double* in, T* out, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = T(in[i]);
}

template <typename T>
cudaError_t launch_convert(const double* in, T* out, int n, cudaStream_t st)
{
    const int threads = 256;
    const int blocks = std::max(1, std::min((n + threads - 1) / threads, 1024));
    convert_kernel<T><<<blocks, threads, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

template <typename Ti, typename To>
__global__ void convert_ff_kernel(const Ti* in, To* out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = To(in[i]);
}

template <typename Ti, typename To>
cudaError_t launch_convert_ff(const Ti* in, To* out, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, 152 * 16));
    convert_ff_kernel<Ti, To><<<blocks, threads, 0, st>>>(in, out, n);
    return cudaGetLastError();
}

template cudaError_t launch_convert_ff<float, double>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_convert_ff<double, float>(const double*, float*, int64_t, cudaStream_t);

template cudaError_t launch_convert<float>(const double*, float*, int, cudaStream_t);
template cudaError_t launch_convert<double>(const double*, double*, int, cudaStream_t);

// Caller layout [nc][N] <-> the kernel's lane-major layout [nc][L][NL], where
// state k = lane * L + s sits at s * NL + lane. 32 x 32 tiles through shared
// memory keep both sides coalesced.
template <typename T, bool TO_LANES>
__global__ void lanes_transpose_kernel(const T* src, T* dst, int64_t N, int L, int NL, int64_t cs)
{
    __shared__ T tile[32][33];
    const int c = blockIdx.z;
    const int l0 = blockIdx.x * 32, s0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        if (TO_LANES) {
            // read: for lane l0 + r, steps s0 + tx (contiguous in the caller layout)
            const int l = l0 + r, s = s0 + tx;
            const int64_t k = (int64_t)l * L + s;
            if (l < NL && s < L && k < N) tile[r][tx] = src[(int64_t)c * N + k];
        } else {
            // read: for step s0 + r, lanes l0 + tx (contiguous in the lane layout)
            const int l = l0 + tx, s = s0 + r;
            const int64_t k = (int64_t)l * L + s;
            if (l < NL && s < L && k < N) tile[tx][r] = src[(int64_t)c * cs + (int64_t)s * NL + l];
        }
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        if (TO_LANES) {
            const int l = l0 + tx, s = s0 + r;
            const int64_t k = (int64_t)l * L + s;
            if (l < NL && s < L && k < N) dst[(int64_t)c * cs + (int64_t)s * NL + l] = tile[tx][r];
        } else {
            const int l = l0 + r, s = s0 + tx;
            const int64_t k = (int64_t)l * L + s;
            if (l < NL && s < L && k < N) dst[(int64_t)c * N + k] = tile[r][tx];
        }
    }
}

template <typename T>
cudaError_t launch_lanes_transpose(const T* src, T* dst, int nc, int64_t N, int L, int NL, bool to_lanes,
                                   cudaStream_t st)
{
    const dim3 grid((NL + 31) / 32, (L + 31) / 32, nc), block(32, 8);
    if (to_lanes) lanes_transpose_kernel<T, true><<<grid, block, 0, st>>>(src, dst, N, L, NL, (int64_t)L * NL);
    else lanes_transpose_kernel<T, false><<<grid, block, 0, st>>>(src, dst, N, L, NL, (int64_t)L * NL);
    return cudaGetLastError();
}

template cudaError_t launch_lanes_transpose<float>(const float*, float*, int, int64_t, int, int, bool, cudaStream_t);
template cudaError_t launch_lanes_transpose<double>(const double*, double*, int, int64_t, int, int, bool, cudaStream_t);

// Prior nominal in the lane-major layout: state k of trajectory b gets (m0_b, P0_b).
template <typename T>
__global__ void init_nominal_lanes_kernel(const int64_t* offsets, int B, int64_t N, int L, int NL, const T* m0,
                                          const T* P0, T* x, T* P)
{
    const int64_t cs = (int64_t)L * NL;
    const int64_t total = cs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(i / NL), l = (int)(i - (int64_t)s * NL);
        const int64_t k = (int64_t)l * L + s;
        if (k >= N) continue;
        const int b = traj_of(offsets, B, k);
        if (x)
#pragma unroll
            for (int c = 0; c < 5; ++c) x[c * cs + i] = m0[5 * b + c];
        if (P)
#pragma unroll
            for (int c = 0; c < 15; ++c) P[c * cs + i] = P0[15 * b + c];
    }
}

template <typename T>
cudaError_t launch_init_nominal_lanes(const int64_t* offsets, int B, int64_t N, int L, int NL, const T* m0,
                                      const T* P0, T* x, T* P, cudaStream_t st)
{
    const int threads = 256;
    const int64_t total = (int64_t)L * NL;
    const int blocks = (int)std::min<int64_t>((total + threads - 1) / threads, 152 * 32);
    init_nominal_lanes_kernel<T><<<blocks, threads, 0, st>>>(offsets, B, N, L, NL, m0, P0, x, P);
    return cudaGetLastError();
}

template cudaError_t launch_init_nominal_lanes<float>(const int64_t*, int, int64_t, int, int, const float*,
                                                      const float*, float*, float*, cudaStream_t);
template cudaError_t launch_init_nominal_lanes<double>(const int64_t*, int, int64_t, int, int, const double*,
                                                       const double*, double*, double*, cudaStream_t);

template <typename T>
__global__ void init_nominal_kernel(const int64_t* offsets, int B, int64_t N, const T* m0, const T* P0, T* x, T* P)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += stride) {
        const int b = traj_of(offsets, B, k);
        if (x)
#pragma unroll
            for (int i = 0; i < 5; ++i) x[i * N + k] = m0[5 * b + i];
        if (P)
#pragma unroll
            for (int i = 0; i < 15; ++i) P[i * N + k] = P0[15 * b + i];
    }
}

template <typename T>
cudaError_t launch_init_nominal(const int64_t* offsets, int B, int64_t N, const T* m0, const T* P0, T* x, T* P,
                                cudaStream_t st)
{
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((N + threads - 1) / threads, 152 * 32);
    init_nominal_kernel<T><<<blocks, threads, 0, st>>>(offsets, B, N, m0, P0, x, P);
    return cudaGetLastError();
}

// Linearisation in the paper's parametrisation (F, c, Q', H, d, R') of Eq. 11.
template <typename T, int LIN>
__global__ void linearize_kernel(const KParams<T> p, T* F, T* c, T* Qp, T* H, T* d, T* Rp, T* y_used)
{
    if (*(volatile int*)p.status & ST_BADARG) return;
    const int64_t N = p.N;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    bool ok = true;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += stride) {
        const int b = traj_of(p.offsets, p.B, k);
        const bool has_next = k + 1 < __ldg(p.offsets + b + 1);
        const bool has_obs = k > __ldg(p.offsets + b);
        if (has_next) {
            Trans<T> tr;
            ok &= get_trans<T, LIN>(p, k, k, tr);
            T Fx[5];
            mv(tr.F, tr.xn, Fx);
#pragma unroll
            for (int i = 0; i < 25; ++i) F[i * N + k] = tr.F[i];
#pragma unroll
            for (int i = 0; i < 5; ++i) c[i * N + k] = tr.fx[i] - Fx[i];
#pragma unroll
            for (int i = 0; i < 15; ++i) Qp[i * N + k] = tr.Q[i];
        } else {
#pragma unroll
            for (int i = 0; i < 25; ++i) F[i * N + k] = T(0);
#pragma unroll
            for (int i = 0; i < 5; ++i) c[i * N + k] = T(0);
#pragma unroll
            for (int i = 0; i < 15; ++i) Qp[i * N + k] = T(0);
        }
        if (has_obs) {
            Obs<T> ob;
            ok &= get_obs<T, LIN>(p, k, k, b, ob);
            T y[2];
            load_y(p, k, y);
            // h(xn), the measurement y_used and d = zbar - H xn with zbar = y_used - r_offset
            T hx[2];
            if (p.model.kind == MODEL_LINEAR) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    T v = p.model.d[r];
#pragma unroll
                    for (int l = 0; l < 5; ++l) v = fma(p.model.H[r * 5 + l], ob.xn[l], v);
                    hx[r] = v;
                }
            } else {
                T s[4];
                load_sensors(p.model, b, s);
                bearings(ob.xn, s, hx);
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const T yu = (p.model.kind == MODEL_LINEAR) ? y[r] : hx[r] + wrap_angle(y[r] - hx[r]);
                // innovation of x is r - H (x - xn) = yu - (zbar + H (x - xn)), so zbar = yu - r
                T Hx = T(0);
#pragma unroll
                for (int l = 0; l < 5; ++l) Hx = fma(ob.H[r * 5 + l], ob.xn[l], Hx);
                d[r * N + k] = (yu - ob.r[r]) - Hx;
                if (y_used) y_used[r * N + k] = yu;
            }
#pragma unroll
            for (int i = 0; i < 10; ++i) H[i * N + k] = ob.H[i];
#pragma unroll
            for (int i = 0; i < 3; ++i) Rp[i * N + k] = ob.R[i];
        } else {
#pragma unroll
            for (int i = 0; i < 10; ++i) H[i * N + k] = T(0);
#pragma unroll
            for (int i = 0; i < 2; ++i) d[i * N + k] = T(0);
#pragma unroll
            for (int i = 0; i < 3; ++i) Rp[i * N + k] = T(0);
            if (y_used) {
                y_used[k] = T(0);
                y_used[N + k] = T(0);
            }
        }
    }
    if (!ok) atomicOr(p.status, ST_NOT_PD);
}

template <typename T>
cudaError_t launch_linearize(const KParams<T>& p, int lin, T* F, T* c, T* Qp, T* H, T* d, T* Rp, T* y_used,
                             cudaStream_t st)
{
    const int threads = 128;
    const int blocks = (int)std::min<int64_t>((p.N + threads - 1) / threads, 152 * 16);
    if (lin == LIN_IEKS)
        linearize_kernel<T, LIN_IEKS><<<blocks, threads, 0, st>>>(p, F, c, Qp, H, d, Rp, y_used);
    else if (lin == LIN_GH)
        linearize_kernel<T, LIN_GH><<<blocks, threads, 0, st>>>(p, F, c, Qp, H, d, Rp, y_used);
    else
        linearize_kernel<T, LIN_CUBATURE><<<blocks, threads, 0, st>>>(p, F, c, Qp, H, d, Rp, y_used);
    return cudaGetLastError();
}

template cudaError_t launch_init_nominal<float>(const int64_t*, int, int64_t, const float*, const float*, float*,
                                                float*, cudaStream_t);
template cudaError_t launch_init_nominal<double>(const int64_t*, int, int64_t, const double*, const double*,
                                                 double*, double*, cudaStream_t);
template cudaError_t launch_linearize<float>(const KParams<float>&, int, float*, float*, float*, float*, float*,
                                             float*, float*, cudaStream_t);
template cudaError_t launch_linearize<double>(const KParams<double>&, int, double*, double*, double*, double*,
                                              double*, double*, double*, cudaStream_t);

}  // namespace pes
