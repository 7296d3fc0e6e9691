// The sequential counterpart of the iterated smoother on the GPU: one thread
// per trajectory runs the textbook extended (or cubature) Kalman filter and
// RTS smoother of Sec. 3's iteration over its whole trajectory, iterating
// until its own relative update meets the tolerance. It is the method the
// paper compares its parallel form against, moved onto the GPU, so that the
// two can be compared on the same device: it has no tree levels and no
// grid-wide barriers, but only B threads of parallelism.
//
// Per step it uses the same device operations as the parallel path: the
// linearisation (Eq. 10 or Eqs. 7-9), the prediction and update, and the
// smoothing element of Eq. 17 built from the filter's own prediction, which
// the backward pass applies to the next smoothed Gaussian (the RTS step).
#include "pes_internal.h"
#include "pes_kernel.cuh"

namespace pes {

namespace {

// Smoothing element of state k in the per-state scratch, component-major.
template <typename T>
PES_DEV void seq_store_el(const KParams<T>& p, int64_t k, const SElem<T>& el)
{
    const T* src = reinterpret_cast<const T*>(&el);
#pragma unroll
    for (int i = 0; i < HAND; ++i) p.hand[(size_t)i * p.N + k] = src[i];
}

template <typename T>
PES_DEV void seq_load_el(const KParams<T>& p, int64_t k, SElem<T>& el)
{
    T* dst = reinterpret_cast<T*>(&el);
#pragma unroll
    for (int i = 0; i < HAND; ++i) dst[i] = p.hand[(size_t)i * p.N + k];
}

// Write the smoothed moments of state k as the next nominal, accumulating the
// relative-update norm against the nominal they replace.
template <typename T>
PES_DEV void seq_write(const KParams<T>& p, int64_t k, const Gauss<T>& g, double& num, double& den)
{
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const double old = (double)p.x[(size_t)i * p.N + k], nw = (double)g.m[i];
        num += (nw - old) * (nw - old);
        den += nw * nw;
        p.x[(size_t)i * p.N + k] = g.m[i];
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) p.P[(size_t)i * p.N + k] = g.P[i];
}

// The Levenberg-Marquardt pseudo-measurement of state k's nominal (if any).
template <typename T>
PES_DEV void seq_damp(const KParams<T>& p, int64_t k, T* m, T* P)
{
    if (!(p.model.lm > T(0))) return;
    T xb[5];
    load_nominal(p, k, xb);
    FElem<T> dmp;
    felem_damping(dmp, xb, p.model.lm);
    Gauss<T> g, gd;
#pragma unroll
    for (int i = 0; i < 5; ++i) g.m[i] = m[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) g.P[i] = P[i];
    apply_filter(g, dmp, gd);
#pragma unroll
    for (int i = 0; i < 5; ++i) m[i] = gd.m[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) P[i] = gd.P[i];
}

template <typename T, int LIN>
__global__ void __launch_bounds__(64) sequential_smoother_kernel(const KParams<T> p)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= p.B) return;
    const int64_t a = p.offsets[b], e = p.offsets[b + 1];
    if (!(a >= 0 && e > a && e <= p.N)) {
        atomicOr(p.status, ST_BADARG);
        return;
    }
    const bool track = p.tol > 0.0;
    bool ok = true, converged = false;
    int it = 0;
    for (it = 0; it < p.iters; ++it) {
        // forward: filter, and the smoothing element of every state but the last
        T m[5], P[15];
        load_prior(p, b, m, P);
        seq_damp(p, a, m, P);
        for (int64_t k = a + 1; k < e; ++k) {
            Trans<T> tr;
            ok &= get_trans<T, LIN>(p, k - 1, k - 1, tr);
            T mp[5], FP[25], Pp[15];
            predict(tr, m, P, mp, FP, Pp);
            SElem<T> el;
            ok &= selem_from_prediction(m, P, FP, Pp, mp, el);
            seq_store_el(p, k - 1, el);
            Obs<T> ob;
            ok &= get_obs<T, LIN>(p, k, k, b, ob);
            ok &= kf_update(ob, mp, Pp, m, P);
            seq_damp(p, k, m, P);
        }
        // backward: the last state's smoothed moments are its filtered ones
        Gauss<T> g;
#pragma unroll
        for (int i = 0; i < 5; ++i) g.m[i] = m[i];
#pragma unroll
        for (int i = 0; i < 15; ++i) g.P[i] = P[i];
        double num = 0.0, den = 0.0;
        seq_write(p, e - 1, g, num, den);
        for (int64_t k = e - 2; k >= a; --k) {
            SElem<T> el;
            seq_load_el(p, k, el);
            Gauss<T> s;
            apply_smoother(el, g, s);
            g = s;
            seq_write(p, k, g, num, den);
        }
#pragma unroll
        for (int i = 0; i < 5; ++i)
            if (!isfinite((double)g.m[i])) ok = false;
        if (track) {
            const double r = den > 0.0 ? sqrt(num / den) : sqrt(num);
            if (r <= p.tol) {
                converged = true;
                ++it;
                break;
            }
        }
    }
    if (!ok) atomicOr(p.status, ST_NOT_PD);
    if (track) {
        if (p.traj_iters) p.traj_iters[b] = converged ? it : 0;
        if (!converged) atomicOr(p.status, ST_NOT_CONVERGED);
    }
    if (p.iters_done) atomicMax(p.iters_done, it);
}

}  // namespace

template <typename T, int LIN>
cudaError_t launch_sequential(const KParams<T>& p, cudaStream_t st)
{
    constexpr int threads = 64;
    const int blocks = (p.B + threads - 1) / threads;
    sequential_smoother_kernel<T, LIN><<<blocks, threads, 0, st>>>(p);
    return cudaGetLastError();
}

template cudaError_t launch_sequential<float, LIN_IEKS>(const KParams<float>&, cudaStream_t);
template cudaError_t launch_sequential<float, LIN_CUBATURE>(const KParams<float>&, cudaStream_t);
template cudaError_t launch_sequential<double, LIN_IEKS>(const KParams<double>&, cudaStream_t);
template cudaError_t launch_sequential<double, LIN_CUBATURE>(const KParams<double>&, cudaStream_t);
template cudaError_t launch_sequential<float, LIN_GH>(const KParams<float>&, cudaStream_t);
template cudaError_t launch_sequential<double, LIN_GH>(const KParams<double>&, cudaStream_t);

}  // namespace pes
