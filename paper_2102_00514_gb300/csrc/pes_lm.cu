// Device side of the Levenberg-Marquardt iteration with adaptive damping
// (Sec. 3 names the LM variant of the IEKS; the host loop is
// pes_ieks_run_lm in pes_api.cu): the MAP objective of every trajectory, the
// per-trajectory accept/reject decision and damping update, and the restore
// of a rejected trajectory's nominal. Objective arithmetic is in FP64 for
// either precision, so that the decisions do not turn on rounding.
#include "pes_internal.h"
#include "pes_lm.cuh"

namespace pes {

namespace {

PES_DEV int traj_of_k(const int64_t* off, int B, int64_t k)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// f(x) of the model in FP64
PES_DEV void f_model(const LMParams& p, const double* x, double* out)
{
    if (p.kind == MODEL_LINEAR) {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            double s = p.c[i];
#pragma unroll
            for (int l = 0; l < 5; ++l) s = fma(p.F[i * 5 + l], x[l], s);
            out[i] = s;
        }
        return;
    }
    const CTCoef<double> k = ct_coef(x[4], p.dt);
    double inc[5];
    ct_increment(x, k, inc);
    out[0] = x[0] + inc[0];
    out[1] = x[1] + inc[1];
    out[2] = inc[2];
    out[3] = inc[3];
    out[4] = inc[4];
}

// the measurement residual y - h(x), bearings on the branch nearest zero
PES_DEV void resid_model(const LMParams& p, int b, const double* x, const double* y, double* r)
{
    if (p.kind == MODEL_LINEAR) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            double s = p.d[i];
#pragma unroll
            for (int l = 0; l < 5; ++l) s = fma(p.H[i * 5 + l], x[l], s);
            r[i] = y[i] - s;
        }
        return;
    }
    const double* s = p.sensors + (p.sensors_per_traj ? 4 * b : 0);
#pragma unroll
    for (int i = 0; i < 2; ++i) r[i] = wrap_angle(y[i] - atan2(x[1] - s[2 * i + 1], x[0] - s[2 * i]));
}

PES_DEV double quad_sym(const double* S, const double* e, int n)
{
    double q = 0.0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const int a = i < j ? i : j, c = i < j ? j : i;
            const int ix = n == 5 ? si(a, c) : si2(a, c);
            q = fma(e[i] * S[ix], e[j], q);
        }
    return q;
}

// Contiguous runs of lanes that hold the same trajectory add their values
// into the run's first lane, which adds them to the trajectory's accumulator.
// Every lane of the warp calls (b < 0: a lane without a state, nothing added).
PES_DEV void warp_segment_add(double v, int b, double* acc)
{
    const unsigned grp = __match_any_sync(0xffffffffu, b);
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double o = __shfl_down_sync(0xffffffffu, v, off);
        const int src = lane + off;
        if (src < 32 && ((grp >> src) & 1u)) v += o;
    }
    if (b >= 0 && lane == __ffs(grp) - 1) atomicAdd(acc + b, v);
}

}  // namespace

// The MAP objective of every trajectory at the nominal x (PES_* layout of the
// smoother kernel: lane-major slots), added into p.cost; with p.xold, also the
// squared step ||x - xold||^2 into p.num and ||x||^2 into p.den.
template <typename T>
__global__ void lm_cost_kernel(const LMParams p, double* cost_out, const T* x, const T* xold, const T* y,
                               const T* m0, const T* P0)
{
    const int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = ix < p.cs;
    int64_t k = 0;
    int s = 0, lane = 0;
    if (valid) {
        s = (int)(ix / p.NL);
        lane = (int)(ix - (int64_t)s * p.NL);
        k = (int64_t)lane * p.L + s;
        valid = k < p.N;
    }
    // every lane stays to the warp's reductions; one without a state adds nothing
    const int b = valid ? traj_of_k(p.offsets, p.B, k) : -1;
    double xk[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    double J = 0.0;
    if (valid) {
#pragma unroll
    for (int c = 0; c < 5; ++c) xk[c] = (double)x[c * p.cs + ix];
    if (k == __ldg(p.offsets + b)) {
        // prior: 1/2 (x_0 - m0)^T P0^{-1} (x_0 - m0), by a Cholesky solve
        double P[15], e[5], Lc[25], rd[5];
#pragma unroll
        for (int c = 0; c < 15; ++c) P[c] = (double)P0[15 * b + c];
#pragma unroll
        for (int c = 0; c < 5; ++c) e[c] = xk[c] - (double)m0[5 * b + c];
        chol_pd(P, Lc, rd);
        double z[5];   // L z = e
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            double t = e[i];
#pragma unroll
            for (int l = 0; l < i; ++l) t = fma(-Lc[i * 5 + l], z[l], t);
            z[i] = t * rd[i];
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) J = fma(0.5 * z[i], z[i], J);
    } else {
        const int64_t ixp = s > 0 ? ix - p.NL : (int64_t)(p.L - 1) * p.NL + (lane - 1);
        double xp[5], fx[5], e[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) xp[c] = (double)x[c * p.cs + ixp];
        f_model(p, xp, fx);
#pragma unroll
        for (int c = 0; c < 5; ++c) e[c] = xk[c] - fx[c];
        J = 0.5 * quad_sym(p.Qi, e, 5);
        double yk[2] = {(double)y[ix], (double)y[p.cs + ix]}, r[2];
        resid_model(p, b, xk, yk, r);
        J = fma(0.5, quad_sym(p.Ri, r, 2), J);
    }
    }
    warp_segment_add(J, b, cost_out);
    if (xold) {
        double num = 0.0, den = 0.0;
        if (valid) {
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                const double dv = xk[c] - (double)xold[c * p.cs + ix];
                num = fma(dv, dv, num);
                den = fma(xk[c], xk[c], den);
            }
        }
        warp_segment_add(num, b, p.num);
        warp_segment_add(den, b, p.den);
    }
}

// Per trajectory: keep the step if it lowered the objective (damping / nu),
// else keep the nominal (damping * nu); record convergence (the step's
// relative size <= tol) and count the trajectories still unconverged.
template <typename T>
__global__ void lm_decide_kernel(const LMParams p, T* lam, int it, double tol, double nu)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= p.B) return;
    const bool acc = p.cost_new[b] < p.cost[b];
    const double num = p.num[b], den = p.den[b];
    const double rel = den > 0.0 ? sqrt(num / den) : sqrt(num);
    if (acc) {
        p.cost[b] = p.cost_new[b];
        lam[b] = (T)((double)lam[b] / nu);
        p.accepted[b] += 1;
        p.reject[b] = 0;
    } else {
        lam[b] = (T)((double)lam[b] * nu);
        p.reject[b] = 1;
    }
    if (tol > 0.0 && p.conv_iter[b] == 0 && rel <= tol) p.conv_iter[b] = it;
    if (p.conv_iter[b] == 0) atomicAdd(p.unconv, 1);
}

// A rejected trajectory's nominal and covariances go back to their values
// before the step.
template <typename T>
__global__ void lm_restore_kernel(const LMParams p, T* x, T* P, const T* xold, const T* Pold)
{
    const int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ix >= p.cs) return;
    const int s = (int)(ix / p.NL);
    const int lane = (int)(ix - (int64_t)s * p.NL);
    const int64_t k = (int64_t)lane * p.L + s;
    if (k >= p.N) return;
    const int b = traj_of_k(p.offsets, p.B, k);
    if (!p.reject[b]) return;
#pragma unroll
    for (int c = 0; c < 5; ++c) x[c * p.cs + ix] = xold[c * p.cs + ix];
#pragma unroll
    for (int c = 0; c < 15; ++c) P[c * p.cs + ix] = Pold[c * p.cs + ix];
}

template <typename T>
__global__ void lm_fill_kernel(T* lam, int B, double v)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) lam[b] = (T)v;
}

template <typename T>
cudaError_t launch_lm_cost(const LMParams& p, double* cost_out, const T* x, const T* xold, const T* y, const T* m0,
                           const T* P0, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((p.cs + 255) / 256);
    lm_cost_kernel<T><<<blocks, 256, 0, st>>>(p, cost_out, x, xold, y, m0, P0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lm_decide(const LMParams& p, T* lam, int it, double tol, double nu, cudaStream_t st)
{
    lm_decide_kernel<T><<<(p.B + 127) / 128, 128, 0, st>>>(p, lam, it, tol, nu);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lm_restore(const LMParams& p, T* x, T* P, const T* xold, const T* Pold, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((p.cs + 255) / 256);
    lm_restore_kernel<T><<<blocks, 256, 0, st>>>(p, x, P, xold, Pold);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lm_fill(T* lam, int B, double v, cudaStream_t st)
{
    lm_fill_kernel<T><<<(B + 127) / 128, 128, 0, st>>>(lam, B, v);
    return cudaGetLastError();
}

#define PES_LM_INSTANTIATE(T)                                                                                     \
    template cudaError_t launch_lm_cost<T>(const LMParams&, double*, const T*, const T*, const T*, const T*,      \
                                           const T*, cudaStream_t);                                               \
    template cudaError_t launch_lm_decide<T>(const LMParams&, T*, int, double, double, cudaStream_t);           \
    template cudaError_t launch_lm_restore<T>(const LMParams&, T*, T*, const T*, const T*, cudaStream_t);       \
    template cudaError_t launch_lm_fill<T>(T*, int, double, cudaStream_t);
PES_LM_INSTANTIATE(float)
PES_LM_INSTANTIATE(double)

}  // namespace pes
