// Kernels of the final iteration's refinement (pes_refine.cuh): the
// float-float residual elements of the filter and RTS recursions, one thread
// per state, and the FP32 scan that turns them into corrections.
#include "pes_internal.h"
#include "pes_refine.cuh"

namespace pes {

namespace {

PES_DEV void load20(const float* base, int64_t cs, int64_t ix, float* m, float* P)
{
#pragma unroll
    for (int c = 0; c < 5; ++c) m[c] = base[c * cs + ix];
#pragma unroll
    for (int c = 0; c < 15; ++c) P[c] = base[(5 + c) * cs + ix];
}

PES_DEV void store_elem(const RefineParams& p, int64_t ix, const float* A, const float* w, const float* s,
                        const float* r)
{
    float* e = p.elem + ix;
#pragma unroll
    for (int c = 0; c < 25; ++c) e[c * p.cs] = A[c];
#pragma unroll
    for (int c = 0; c < 5; ++c) e[(25 + c) * p.cs] = w[c];
#pragma unroll
    for (int c = 0; c < 5; ++c) e[(30 + c) * p.cs] = s[c];
#pragma unroll
    for (int c = 0; c < 15; ++c) e[(35 + c) * p.cs] = r[c];
}

// The elements are read-only while the correction scan runs: loads through
// the non-coherent path, which the compiler may move ahead of the scan's
// stores.
PES_DEV void load_elem(const RefineParams& p, int64_t ix, RElem& el)
{
    const float* e = p.elem + ix;
    float* d = reinterpret_cast<float*>(&el);
#pragma unroll
    for (int c = 0; c < RE; ++c) d[c] = __ldg(e + c * p.cs);
}

// (state, lane) of the thread's slot in the lane-major arrays; false past N.
PES_DEV bool slot_state(const RefineParams& p, int64_t ix, int& s, int& lane, int64_t& k)
{
    if (ix >= p.cs) return false;
    s = (int)(ix / p.NL);
    lane = (int)(ix - (int64_t)s * p.NL);
    k = (int64_t)lane * p.L + s;
    return k < p.N;
}

PES_DEV int64_t next_slot(const RefineParams& p, int64_t ix, int s, int lane)
{
    return (s + 1 < p.L) ? ix + p.NL : (int64_t)(lane + 1);
}

}  // namespace

constexpr int RT_THREADS = 128;   // threads per block of the residual kernels
constexpr size_t RT_SMEM = sizeof(float) * SCR_N * RT_THREADS;

// Forward residual elements. The thread of state k writes the element of
// state k + 1 (the Kalman step k -> k+1 from the FP32 filtered moments of k)
// and, for a trajectory's first state, its own (the prior: A = 0); it also
// stores the transition out of k for the RTS residuals.
template <int LIN>
__global__ void __launch_bounds__(RT_THREADS) refine_fwd_kernel(const RefineParams p)
{
    extern __shared__ float scr_raw[];
    const Scratch<RT_THREADS> sc{scr_raw + threadIdx.x};
    const int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int s, lane;
    int64_t k;
    if (!slot_state(p, ix, s, lane, k)) return;
    const int b = traj_of(p.offsets, p.B, k);
    const int64_t head = __ldg(p.offsets + b), next = __ldg(p.offsets + b + 1);
    float xf[5], Pf[15];
    load20(p.filt, p.cs, ix, xf, Pf);
    if (k == head) {
        float A[25], w[5], sres[5], r[15];
#pragma unroll
        for (int c = 0; c < 25; ++c) A[c] = 0.0f;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            w[c] = 0.0f;
            sres[c] = __fsub_rn(__ldg(p.m0 + 5 * b + c), xf[c]);
        }
#pragma unroll
        for (int c = 0; c < 15; ++c) r[c] = __fsub_rn(__ldg(p.P0 + 15 * b + c), Pf[c]);
        store_elem(p, ix, A, w, sres, r);
    }
    if (k + 1 >= next) return;
    const DevModel<float>& m = p.model;
    // transition k -> k+1 about the nominal of k; its slope goes to the scratch
    Trans<float> tr;
    bool ok = true;
    {
        float xn[5], Pn[15];
        load20(p.nom, p.cs, ix, xn, Pn);
        if (LIN == LIN_IEKS) {
            lin_trans_taylor(m, xn, tr);
#pragma unroll
            for (int c = 0; c < 25; ++c) sc[SCR_F + c] = tr.F[c];
        } else {
            float Lc[25], rdc[5];
            ok &= cub_factor(Pn, Lc, rdc);
            lin_trans_cubature(m, xn, Lc, rdc, tr);
            cub_trans_slope_ff(m, xn, Lc, sc);
        }
    }
    {
        float* t = p.trans + ix;
#pragma unroll 5
        for (int c = 0; c < 25; ++c) t[c * p.cs] = sc[SCR_F + c];
#pragma unroll
        for (int c = 0; c < 5; ++c) t[(25 + c) * p.cs] = tr.fx[c];
#pragma unroll
        for (int c = 0; c < 15; ++c) t[(30 + c) * p.cs] = tr.Q[c];
    }
    // observation of k + 1 about its nominal
    const int64_t ix1 = next_slot(p, ix, s, lane);
    Obs<float> ob;
    {
        float xn[5], Pn[15], y[2];
        load20(p.nom, p.cs, ix1, xn, Pn);
        y[0] = __ldg(p.y + ix1);
        y[1] = __ldg(p.y + p.cs + ix1);
        if (LIN == LIN_IEKS) {
            lin_obs_taylor(m, b, xn, y, ob);
        } else {
            float Lc[25], rdc[5];
            ok &= cub_factor(Pn, Lc, rdc);
            lin_obs_cubature(m, b, xn, Lc, rdc, y, ob);
        }
    }
    ff mf[5], Pff[15];
    float A[25], w[5];
    ok &= ff_kalman_step(tr, ob, xf, Pf, mf, Pff, A, w, sc);
    float x1[5], P1[15], sres[5], r[15];
    load20(p.filt, p.cs, ix1, x1, P1);
#pragma unroll
    for (int c = 0; c < 5; ++c) sres[c] = ff_to_f(ff_add_f(mf[c], -x1[c]));
#pragma unroll
    for (int c = 0; c < 15; ++c) r[c] = ff_to_f(ff_add_f(Pff[c], -P1[c]));
    store_elem(p, ix1, A, w, sres, r);
    if (!ok) atomicOr(p.status, ST_NOT_PD);
}

// RTS residual elements, one per state, from the refined filtered moments
// (FP32 value + the filter's correction) and the FP32 smoothed moments.
__global__ void __launch_bounds__(RT_THREADS) refine_bwd_kernel(const RefineParams p)
{
    extern __shared__ float scr_raw[];
    const Scratch<RT_THREADS> sc{scr_raw + threadIdx.x};
    const int64_t ix = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int s, lane;
    int64_t k;
    if (!slot_state(p, ix, s, lane, k)) return;
    const int b = traj_of(p.offsets, p.B, k);
    const int64_t next = __ldg(p.offsets + b + 1);
    // the refined filtered moments as float-float pairs
    auto filt_ff = [&](int c) { return two_sum(p.filt[c * p.cs + ix], p.dlt[c * p.cs + ix]); };
    float* el = p.elem + ix;
#pragma unroll
    for (int c = 0; c < 5; ++c) el[(25 + c) * p.cs] = 0.0f;
    if (k + 1 >= next) {
        // last state: smoothed = filtered
#pragma unroll 5
        for (int c = 0; c < 25; ++c) el[c * p.cs] = 0.0f;
#pragma unroll
        for (int c = 0; c < 20; ++c) el[(30 + c) * p.cs] = ff_to_f(ff_add_f(filt_ff(c), -p.xs[c * p.cs + ix]));
        return;
    }
    Trans<float> tr;
    {
        const float* t = p.trans + ix;
#pragma unroll 5
        for (int c = 0; c < 25; ++c) sc[SCR_F + c] = t[c * p.cs];
#pragma unroll
        for (int c = 0; c < 5; ++c) tr.fx[c] = t[(25 + c) * p.cs];
#pragma unroll
        for (int c = 0; c < 15; ++c) tr.Q[c] = t[(30 + c) * p.cs];
#pragma unroll
        for (int c = 0; c < 5; ++c) tr.xn[c] = p.nom[c * p.cs + ix];
    }
    const int64_t ix1 = next_slot(p, ix, s, lane);
    ff ms[5], dP[15];
    bool ok;
    {
        ff mf[5], Pf[15];
#pragma unroll
        for (int c = 0; c < 5; ++c) mf[c] = filt_ff(c);
#pragma unroll
        for (int c = 0; c < 15; ++c) Pf[c] = filt_ff(5 + c);
        float xs1[5], Ps1[15];
        load20(p.xs, p.cs, ix1, xs1, Ps1);
        ok = ff_rts_gain(tr, mf, Pf, xs1, Ps1, ms, dP, sc);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) el[(30 + c) * p.cs] = ff_to_f(ff_add_f(ms[c], -p.xs[c * p.cs + ix]));
    // covariance residuals, row by row: Pf + G dP G^T - Ps
#pragma unroll 1
    for (int i = 0; i < 5; ++i) {
        rts_cov_row(i, dP, sc, [&](int j, ff v) {
            const int e = si_rt(i, j);
            const ff Ps = ff_add(filt_ff(5 + e), v);
            el[(35 + e) * p.cs] = ff_to_f(ff_add_f(Ps, -p.xs[(5 + e) * p.cs + ix]));
        });
    }
    // G_ij = (G^T)_ji
#pragma unroll 1
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) el[(i * 5 + j) * p.cs] = sc[SCR_M + 2 * (j * 5 + i)];
    if (!ok) atomicOr(p.status, ST_NOT_PD);
}

// ---- the correction scan ---------------------------------------------------------

namespace {

PES_DEV void refine_barrier(const RefineParams& p)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(p.bar, 1u);
        const long long t0 = globaltimer_ns();
        unsigned polls = 0;
        while (ld_acquire(p.bar) < gridDim.x) {
            if (*(volatile int*)p.status & ST_TIMEOUT) break;
            if (++polls > (1u << 26) || globaltimer_ns() - t0 > p.timeout_ns) {
                atomicOr(p.status, ST_TIMEOUT);
                break;
            }
            __nanosleep(128);
        }
        __threadfence();
    }
    __syncthreads();
}

template <bool W>
__device__ __noinline__ void tree_compose(const RElem& b, const RElem& a, RElem& c)
{
    relem_compose<W>(b, a, c);
}

PES_DEV void rstate_zero(RState& d)
{
#pragma unroll
    for (int i = 0; i < 5; ++i) d.m[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < 15; ++i) d.P[i] = 0.0f;
}

}  // namespace

template <int NT>
constexpr size_t refine_smem_bytes()
{
    return sizeof(RElem) * 2 * NT + sizeof(RState) * (NT + 1);
}

// The correction recursion over every state: forward (FWD, the filter's, from
// a trajectory's first state; writes the corrections to p.dlt) or backward
// (the RTS smoother's, from a trajectory's last state; adds the corrections
// to p.xs). Lanes own the same chunks as the smoother kernel's (L steps of
// lane-major slot s * NL + lane). Three levels as in the smoother kernel: each
// lane composes its chunk's elements, a block tree and a grid-wide level give
// every lane the correction of the state before (after) its chunk, and each
// lane re-runs its chunk.
template <bool FWD, int NT>
__global__ void __launch_bounds__(NT, 1) refine_scan_kernel(const RefineParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RElem* el = reinterpret_cast<RElem*>(smem_raw);
    RElem* top = el + NT;
    RState* gs = reinterpret_cast<RState*>(top + NT);
    RState* gblock = gs + NT;
    constexpr bool W = FWD;
    const int t = threadIdx.x;
    const int lane = blockIdx.x * NT + t;
    const int64_t a = min((int64_t)lane * p.L, p.N);
    const int64_t e = min(a + (int64_t)p.L, p.N);
    // level 1: the chunk's composition (each new element applies after the
    // ones already composed: forward from the chunk's first state, backward
    // from its last)
    {
        RElem acc, ek, en;
        relem_identity(acc);
        const int n = (int)(e - a);
        if (n > 0) load_elem(p, (FWD ? 0 : n - 1) * (int64_t)p.NL + lane, en);
#pragma unroll 1
        for (int q = 0; q < n; ++q) {
            ek = en;
            const int sn = FWD ? q + 1 : n - 2 - q;   // the next state's step within the chunk
            if (q + 1 < n) load_elem(p, sn * (int64_t)p.NL + lane, en);
            relem_compose<W>(ek, acc, acc);
        }
        el[t] = acc;
    }
    __syncthreads();
    const bool half = t < NT / 2;
    const int to = 2 * t + 1, te = 2 * t;
    // level 2: up-sweep (forward: later after earlier; backward: earlier after later)
#pragma unroll 1
    for (int s = 1; s < NT; s <<= 1) {
        if (FWD) {
            if (half && ((to + 1) & (2 * s - 1)) == 0) tree_compose<W>(el[to], el[to - s], el[to]);
        } else {
            if (half && (te & (2 * s - 1)) == 0) tree_compose<W>(el[te], el[te + s], el[te]);
        }
        __syncthreads();
    }
    {
        const float* src = reinterpret_cast<const float*>(FWD ? &el[NT - 1] : &el[0]);
        for (int i = t; i < RE; i += NT) p.agg[(size_t)blockIdx.x * RE + i] = src[i];
    }
    refine_barrier(p);
    // level 3: the correction entering this block from the blocks before (after) it
    if (t == 0) rstate_zero(*gblock);
    const int j = blockIdx.x, nb = gridDim.x;
    if (FWD) {
#pragma unroll 1
        for (int c0 = 0; c0 < j; c0 += NT) {
            const int n = min(NT, j - c0);
            __syncthreads();
            for (int i = t; i < n * RE; i += NT) reinterpret_cast<float*>(top)[i] = __ldcg(p.agg + (size_t)c0 * RE + i);
            __syncthreads();
#pragma unroll 1
            for (int s = 1; s < n; s <<= 1) {
                if (half && (te & (2 * s - 1)) == 0 && te + s < n) tree_compose<W>(top[te + s], top[te], top[te]);
                __syncthreads();
            }
            if (t == 0) relem_apply<W>(top[0], *gblock, *gblock);
        }
    } else {
#pragma unroll 1
        for (int c1 = nb; c1 > j + 1;) {
            const int n = min(NT, c1 - (j + 1));
            const int c0 = c1 - n;
            __syncthreads();
            for (int i = t; i < n * RE; i += NT) reinterpret_cast<float*>(top)[i] = __ldcg(p.agg + (size_t)c0 * RE + i);
            __syncthreads();
#pragma unroll 1
            for (int s = 1; s < n; s <<= 1) {
                if (half && (te & (2 * s - 1)) == 0 && te + s < n) tree_compose<W>(top[te], top[te + s], top[te]);
                __syncthreads();
            }
            if (t == 0) relem_apply<W>(top[0], *gblock, *gblock);
            c1 = c0;
        }
    }
    __syncthreads();
    // level 4: down-sweep
    if (FWD) {
        if (t == NT - 1) gs[NT - 1] = *gblock;
        __syncthreads();
#pragma unroll 1
        for (int s = NT / 2; s >= 1; s >>= 1) {
            if (half && ((to + 1) & (2 * s - 1)) == 0) {
                const RState gin = gs[to];
                RState gr;
                relem_apply<W>(el[to - s], gin, gr);
                gs[to - s] = gin;
                gs[to] = gr;
            }
            __syncthreads();
        }
    } else {
        if (t == 0) gs[0] = *gblock;
        __syncthreads();
#pragma unroll 1
        for (int s = NT / 2; s >= 1; s >>= 1) {
            if (half && (te & (2 * s - 1)) == 0) {
                const RState gin = gs[te];
                RState gl;
                relem_apply<W>(el[te + s], gin, gl);
                gs[te + s] = gin;
                gs[te] = gl;
            }
            __syncthreads();
        }
    }
    RState d = gs[t];
    // level 5: re-run, the next state's element (and, backward, its FP32
    // smoothed moments) loaded one step ahead
    {
        const int n = (int)(e - a);
        RElem ek, en;
        float xn[20], xc[20];
        auto slot = [&](int q) { return (int64_t)(FWD ? q : n - 1 - q) * p.NL + lane; };
        if (n > 0) {
            load_elem(p, slot(0), en);
            if (!FWD)
#pragma unroll
                for (int c = 0; c < 20; ++c) xn[c] = p.xs[c * p.cs + slot(0)];
        }
        bool finite = true;
#pragma unroll 1
        for (int q = 0; q < n; ++q) {
            const int64_t ix = slot(q);
            ek = en;
            if (!FWD)
#pragma unroll
                for (int c = 0; c < 20; ++c) xc[c] = xn[c];
            if (q + 1 < n) {
                load_elem(p, slot(q + 1), en);
                if (!FWD)
#pragma unroll
                    for (int c = 0; c < 20; ++c) xn[c] = p.xs[c * p.cs + slot(q + 1)];
            }
            relem_apply<W>(ek, d, d);
            if (FWD) {
#pragma unroll
                for (int c = 0; c < 5; ++c) p.dlt[c * p.cs + ix] = d.m[c];
#pragma unroll
                for (int c = 0; c < 15; ++c) p.dlt[(5 + c) * p.cs + ix] = d.P[c];
            } else {
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    const float v = xc[c] + d.m[c];
                    finite = finite && isfinite(v);
                    p.xs[c * p.cs + ix] = v;
                }
#pragma unroll
                for (int c = 0; c < 15; ++c) p.xs[(5 + c) * p.cs + ix] = xc[5 + c] + d.P[c];
            }
        }
        if (!finite) atomicOr(p.status, ST_NONFINITE);
    }
}

// ---- launchers -----------------------------------------------------------------

cudaError_t launch_refine_fwd(const RefineParams& p, int lin, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((p.cs + RT_THREADS - 1) / RT_THREADS);
    auto kern = lin == LIN_IEKS ? refine_fwd_kernel<LIN_IEKS> : refine_fwd_kernel<LIN_CUBATURE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RT_SMEM);
    if (e != cudaSuccess) return e;
    kern<<<blocks, RT_THREADS, RT_SMEM, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_refine_bwd(const RefineParams& p, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((p.cs + RT_THREADS - 1) / RT_THREADS);
    cudaError_t e = cudaFuncSetAttribute(refine_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RT_SMEM);
    if (e != cudaSuccess) return e;
    refine_bwd_kernel<<<blocks, RT_THREADS, RT_SMEM, st>>>(p);
    return cudaGetLastError();
}

namespace {
template <bool FWD, int NT>
cudaError_t launch_scan_cfg(const RefineParams& p, int nb, cudaStream_t st)
{
    auto kern = refine_scan_kernel<FWD, NT>;
    const size_t smem = refine_smem_bytes<NT>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    RefineParams pc = p;
    void* args[] = {&pc};
    return cudaLaunchCooperativeKernel((const void*)kern, dim3(nb), dim3(NT), args, smem, st);
}

template <bool FWD, int NT>
int scan_capacity_cfg(int device)
{
    auto kern = refine_scan_kernel<FWD, NT>;
    const size_t smem = refine_smem_bytes<NT>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return -(int)e;
    int per_sm = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem)) != cudaSuccess) return -(int)e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess) return -(int)e;
    return per_sm * sms;
}
}  // namespace

cudaError_t launch_refine_scan(const RefineParams& p, bool fwd, int nt, int nb, cudaStream_t st)
{
    if (nt == 256) return fwd ? launch_scan_cfg<true, 256>(p, nb, st) : launch_scan_cfg<false, 256>(p, nb, st);
    if (nt == 128) return fwd ? launch_scan_cfg<true, 128>(p, nb, st) : launch_scan_cfg<false, 128>(p, nb, st);
    return cudaErrorInvalidValue;
}

int refine_scan_capacity(int nt, int device)
{
    int a, b;
    if (nt == 256) {
        a = scan_capacity_cfg<true, 256>(device);
        b = scan_capacity_cfg<false, 256>(device);
    } else if (nt == 128) {
        a = scan_capacity_cfg<true, 128>(device);
        b = scan_capacity_cfg<false, 128>(device);
    } else {
        return 0;
    }
    if (a < 0) return a;
    if (b < 0) return b;
    return a < b ? a : b;
}

}  // namespace pes
