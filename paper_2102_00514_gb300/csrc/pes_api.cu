// Host side of the C ABI declared in include/pes.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>

#include "pes.h"
#include "pes_handle.h"
#include "pes_trace.h"
#include "pes_internal.h"
#include "pes_lm.cuh"
#include "pes_refine.cuh"

using namespace pes;

namespace {

constexpr int kMaxBlocksPerSM = 2;   // largest occupancy of any compiled configuration
constexpr int kMaxThreads = 256;
constexpr int kMinStepsPerThread = 8;

pes_status fail(pes_handle* h, pes_status st, const char* fmt, ...)
{
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof(h->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

pes_status cuda_fail(pes_handle* h, cudaError_t e, const char* what)
{
    return fail(h, PES_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define PES_CUDA(h, call)                                 \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

size_t scalar_size(pes_precision p) { return p == PES_FP64 ? sizeof(double) : sizeof(float); }

pes_status check_common(pes_handle* h, pes_precision prec, const int64_t* offsets, int32_t B, int64_t N,
                        bool allow_mixed = false)
{
    if (!h) return PES_ERR_INVALID_ARG;
    const bool two_stage = (prec == PES_MIXED || prec == PES_REFINED);
    if (two_stage && !allow_mixed)
        return fail(h, PES_ERR_UNSUPPORTED, "PES_MIXED and PES_REFINED are only supported by pes_ieks_run");
    if (two_stage) return check_common(h, PES_FP32, offsets, B, N);
    if (prec != PES_FP32 && prec != PES_FP64) return fail(h, PES_ERR_INVALID_ARG, "unknown precision %d", (int)prec);
    if (!offsets) return fail(h, PES_ERR_INVALID_ARG, "offsets is NULL");
    if (B < 1) return fail(h, PES_ERR_INVALID_ARG, "B must be >= 1 (got %d)", (int)B);
    if (N < B) return fail(h, PES_ERR_INVALID_ARG, "N (%lld) must be >= B (%d)", (long long)N, (int)B);
    if (N > h->max_states) return fail(h, PES_ERR_INVALID_ARG, "N (%lld) exceeds max_states (%lld)", (long long)N, (long long)h->max_states);
    if (B > h->max_batch) return fail(h, PES_ERR_INVALID_ARG, "B (%d) exceeds max_batch (%d)", (int)B, (int)h->max_batch);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device)
        return fail(h, PES_ERR_INVALID_ARG, "the current device (%d) is not the handle's device (%d)", dev, h->device);
    return PES_OK;
}

// Kernel linearisation of a method: Taylor, the symmetric sigma-point rules
// (cubature, unscented: one kernel, parameterised), Gauss-Hermite.
int lin_of(pes_method method)
{
    return method == PES_IEKS ? LIN_IEKS : (method == PES_GAUSS_HERMITE ? LIN_GH : LIN_CUBATURE);
}

// Sigma-point rule of a method: the spread of the side points, twice a side
// point's weight, and the centre's covariance weight (pes.h, pes_method).
void sigma_rule(const pes_model& m, pes_method method, double& scale, double& w, double& w0c)
{
    const double n = 5.0;
    if (method == PES_UNSCENTED) {
        const double a = m.ut_alpha;
        const double lam = a * a * (n + m.ut_kappa) - n;
        scale = sqrt(n + lam);
        w = 1.0 / (n + lam);
        w0c = lam / (n + lam) + 1.0 - a * a + m.ut_beta;
    } else {
        scale = sqrt(n);
        w = 1.0 / n;
        w0c = 0.0;
    }
}

template <typename T>
DevModel<T> to_dev_model(const pes_model& m, const T* sensors_T, pes_method method)
{
    DevModel<T> d;
    memset(&d, 0, sizeof(d));
    double sc, w, w0c;
    sigma_rule(m, method, sc, w, w0c);
    d.sp_scale = T(sc);
    d.sp_w = T(w);
    d.sp_w0c = T(w0c);
    d.lm = T(m.lm_lambda);
    d.kind = m.kind;
    d.sensors_per_traj = m.sensors_per_traj;
    d.dt = T(m.dt);
    d.sensors = sensors_T;
    double Q[15] = {0}, R[3] = {0};
    if (m.kind == PES_MODEL_LINEAR) {
        memcpy(Q, m.Q, sizeof(Q));
        memcpy(R, m.R, sizeof(R));
        for (int i = 0; i < 25; ++i) d.F[i] = T(m.F[i]);
        for (int i = 0; i < 5; ++i) d.c[i] = T(m.c[i]);
        for (int i = 0; i < 10; ++i) d.H[i] = T(m.H[i]);
        for (int i = 0; i < 2; ++i) d.d[i] = T(m.d[i]);
    } else {
        const double dt = m.dt;
        if (m.q_form == 1) {
            for (int ax = 0; ax < 2; ++ax) {
                const int pp = ax, v = ax + 2;
                Q[si(pp, pp)] = m.q_c * dt * dt * dt / 3.0;
                Q[si(pp, v)] = m.q_c * dt * dt / 2.0;
                Q[si(v, v)] = m.q_c * dt;
            }
        } else {
            Q[si(2, 2)] = m.q_c * dt;
            Q[si(3, 3)] = m.q_c * dt;
        }
        Q[si(4, 4)] = m.q_w * dt;
        R[0] = m.r_std * m.r_std;
        R[2] = m.r_std * m.r_std;
    }
    for (int i = 0; i < 15; ++i) d.Q[i] = T(Q[i]);
    for (int i = 0; i < 3; ++i) d.R[i] = T(R[i]);
    return d;
}

// The model's sensors in the kernel precision, in the handle's workspace.
template <typename T>
pes_status device_model(pes_handle* h, const pes_model& m, int32_t B, cudaStream_t st, DevModel<T>& out);

pes_status check_method(pes_handle* h, pes_method method, const pes_model* m)
{
    if (method != PES_IEKS && method != PES_CUBATURE && method != PES_UNSCENTED && method != PES_GAUSS_HERMITE)
        return fail(h, PES_ERR_INVALID_ARG, "unknown method");
    if (method == PES_UNSCENTED) {
        if (!std::isfinite(m->ut_alpha) || m->ut_alpha == 0.0 || !std::isfinite(m->ut_beta) ||
            !std::isfinite(m->ut_kappa))
            return fail(h, PES_ERR_INVALID_ARG, "unscented parameters must be finite, alpha non-zero");
        const double lam = m->ut_alpha * m->ut_alpha * (5.0 + m->ut_kappa) - 5.0;
        if (!(5.0 + lam > 0.0)) return fail(h, PES_ERR_INVALID_ARG, "unscented rule needs n + lambda > 0");
    }
    return PES_OK;
}

pes_status check_model(pes_handle* h, const pes_model* m)
{
    if (m && !(m->lm_lambda >= 0.0 && std::isfinite(m->lm_lambda)))
        return fail(h, PES_ERR_INVALID_ARG, "lm_lambda must be finite and >= 0");
    if (!m) return fail(h, PES_ERR_INVALID_ARG, "model is NULL");
    if (m->kind == PES_MODEL_CT_BEARINGS) {
        if (!m->sensors) return fail(h, PES_ERR_INVALID_ARG, "model.sensors is NULL");
        if (!(m->dt > 0.0) || !(m->r_std > 0.0) || m->q_c < 0.0 || m->q_w < 0.0)
            return fail(h, PES_ERR_INVALID_ARG, "model needs dt > 0, r_std > 0, q_c >= 0, q_w >= 0");
        if (m->q_form != 0 && m->q_form != 1) return fail(h, PES_ERR_INVALID_ARG, "model.q_form must be 0 or 1");
        return PES_OK;
    }
    if (m->kind == PES_MODEL_LINEAR) return PES_OK;
    return fail(h, PES_ERR_INVALID_ARG, "unknown model kind %d", (int)m->kind);
}

// Block size per precision. PES_FP32_THREADS (128 or 256) overrides the FP32
// choice, for tuning.
// Threads per block and minimum steps per lane: the autotuned values of the
// handle if pes_autotune set them, else the defaults (256 threads for FP32,
// the 128 that the FP64 kernel is compiled for).
static_assert(std::extent<decltype(pes_handle::tune)>::value > LIN_GH, "one tuning slot per linearisation");

int choose_nt(const pes_handle* h, int lin, pes_precision prec)
{
    const pes_tune& t = h->tune[lin][prec == PES_FP64 ? 1 : 0];
    if (t.nt) return t.nt;
    return prec == PES_FP64 ? 128 : 256;
}

int choose_min_steps(const pes_handle* h, int lin, pes_precision prec)
{
    const pes_tune& t = h->tune[lin][prec == PES_FP64 ? 1 : 0];
    return t.min_steps ? t.min_steps : kMinStepsPerThread;
}

struct Shape {
    int nb, nt, L;
};

template <typename T>
pes_status make_shape(pes_handle* h, int lin, pes_precision prec, int64_t N, Shape& s)
{
    s.nt = choose_nt(h, lin, prec);
    const int min_steps = choose_min_steps(h, lin, prec);
    const int cap = coop_capacity(T(0), lin, s.nt, h->device);
    if (cap < 0) {
        cudaGetLastError();   // clear a sticky launch-configuration error
        return fail(h, PES_ERR_CUDA, "the smoother kernel's occupancy query failed: %s",
                    cudaGetErrorString((cudaError_t)(-cap)));
    }
    if (cap == 0) return fail(h, PES_ERR_CUDA, "the smoother kernel cannot be made co-resident on this device");
    const int64_t want = (N + (int64_t)s.nt * min_steps - 1) / ((int64_t)s.nt * min_steps);
    s.nb = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)cap, want, (int64_t)h->nb_max}));
    const int64_t lanes = (int64_t)s.nb * s.nt;
    s.L = (int)((N + lanes - 1) / lanes);
    return PES_OK;
}

template <typename T>
void fill_workspace(pes_handle* h, KParams<T>& p, const Shape& s)
{
    p.hand = static_cast<T*>(h->hand);
    p.lin = static_cast<T*>(h->lin);
    p.aggF = static_cast<T*>(h->aggF);
    p.aggS = static_cast<T*>(h->aggS);
    p.bar = h->bar;
    p.status = h->status;
    p.conv = h->conv;
    p.iters_done = h->iters_done;
    p.traj_iters = nullptr;
    p.L = s.L;
    p.NL = s.nb * s.nt;
    p.cs = p.lanes_layout ? (int64_t)s.L * p.NL : p.N;
    p.timeout_ns = h->timeout_ns;
    p.ptime = h->ptime;
    h->ptime_blocks = s.nb;
}

pes_status read_status(pes_handle* h, cudaStream_t st, int* iters = nullptr)
{
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
    int status = 0;
    PES_CUDA(h, cudaMemcpy(&status, h->status, sizeof(int), cudaMemcpyDeviceToHost));
    PES_CUDA(h, cudaMemset(h->status, 0, sizeof(int)));
    if (iters) PES_CUDA(h, cudaMemcpy(iters, h->iters_done, sizeof(int), cudaMemcpyDeviceToHost));
    if (status & ST_BADARG) return fail(h, PES_ERR_INVALID_ARG, "offsets are malformed (need 0 = o[0] < o[1] < ... < o[B] = N)");
    if (status & ST_TIMEOUT) return fail(h, PES_ERR_TIMEOUT, "a grid-wide wait exceeded its time limit");
    if (status & ST_NOT_PD) return fail(h, PES_ERR_NOT_PD, "a covariance or innovation matrix was not positive definite");
    if (status & ST_NONFINITE) return fail(h, PES_ERR_NONFINITE, "a non-finite smoothed mean was produced");
    if (status & ST_NOT_CONVERGED) return fail(h, PES_ERR_NOT_CONVERGED, "the tolerance was not reached within max_iters");
    return PES_OK;
}

template <typename T>
pes_status device_model(pes_handle* h, const pes_model& m, int32_t B, cudaStream_t st, DevModel<T>& out,
                        pes_method method)
{
    T* sensT = static_cast<T*>(h->sensT);
    out = to_dev_model<T>(m, sensT, method);
    if (m.kind == PES_MODEL_CT_BEARINGS) {
        const int n = 4 * (m.sensors_per_traj ? (int)B : 1);
        PES_CUDA(h, launch_convert<T>(m.sensors, sensT, n, st));
    }
    return PES_OK;
}

template <typename T>
pes_status run_persistent_shaped(pes_handle* h, KParams<T>& p, int lin, const Shape& s, cudaStream_t st)
{
    fill_workspace(h, p, s);
    // the grid barriers count arrivals up from 0; the timeout test starts the
    // count one short (all ones: -1), so that no barrier completes
    PES_CUDA(h, cudaMemsetAsync(h->bar, h->bar_short ? 0xFF : 0, sizeof(unsigned), st));
    if (p.mode == MODE_RUN && p.tol > 0.0) {
        PES_CUDA(h, cudaMemsetAsync(h->conv, 0, sizeof(double) * 4 * p.B, st));
        if (h->traj_iters) {
            PES_CUDA(h, cudaMemsetAsync(h->traj_iters, 0, sizeof(int) * p.B, st));
            p.traj_iters = h->traj_iters;
            h->traj_iters_B = p.B;
        }
    }
    cudaError_t e = launch_persistent(p, lin, s.nt, s.nb, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "cooperative launch of the smoother kernel");
    return PES_OK;
}

template <typename T>
pes_status run_persistent(pes_handle* h, KParams<T>& p, int lin, pes_precision prec, cudaStream_t st)
{
    Shape s;
    pes_status r = make_shape<T>(h, lin, prec, p.N, s);
    if (r != PES_OK) return r;
    return run_persistent_shaped(h, p, lin, s, st);
}

}  // namespace

template <typename T>
static pes_status filter_scan_t(pes_handle* h, const void* F, const void* c, const void* Qp, const void* H,
                                const void* d, const void* Rp, const void* y, const void* m0, const void* P0,
                                const int64_t* offsets, int32_t B, int64_t N, void* xf, void* Pf, pes_precision prec,
                                cudaStream_t st, double* loglik = nullptr)
{
    KParams<T> p{};
    p.N = N; p.offsets = offsets; p.B = B; p.mode = MODE_FILTER; p.iters = 1;
    if (loglik) PES_CUDA(h, cudaMemsetAsync(loglik, 0, sizeof(double) * B, st));
    p.loglik = loglik;
    p.F = (const T*)F; p.c = (const T*)c; p.Qp = (const T*)Qp; p.H = (const T*)H; p.d = (const T*)d;
    p.Rp = (const T*)Rp; p.y = (const T*)y; p.m0 = (const T*)m0; p.P0 = (const T*)P0;
    p.xf = (T*)xf; p.Pf = (T*)Pf;
    return run_persistent<T>(h, p, LIN_ARRAYS, prec, st);
}

template <typename T>
static pes_status smooth_scan_t(pes_handle* h, const void* F, const void* c, const void* Qp, const void* xf,
                                const void* Pf, const int64_t* offsets, int32_t B, int64_t N, void* xs, void* Ps,
                                pes_precision prec, cudaStream_t st)
{
    KParams<T> p{};
    p.N = N; p.offsets = offsets; p.B = B; p.mode = MODE_SMOOTH; p.iters = 1;
    p.F = (const T*)F; p.c = (const T*)c; p.Qp = (const T*)Qp;
    p.xf = (T*)xf; p.Pf = (T*)Pf; p.x = (T*)xs; p.P = (T*)Ps;
    return run_persistent<T>(h, p, LIN_ARRAYS, prec, st);
}

template <typename T>
static pes_status ieks_run_t(pes_handle* h, const pes_model* model, pes_method method, pes_precision prec,
                             const void* y, const int64_t* offsets, int32_t B, int64_t N, const void* m0,
                             const void* P0, const void* x_init, const void* P_init, int32_t max_iters, double tol,
                             void* x_out, void* P_out, int32_t* iters_used, cudaStream_t st)
{
    const int lin = lin_of(method);
    Shape s;
    pes_status r = make_shape<T>(h, lin, prec, N, s);
    if (r != PES_OK) return r;
    // the kernel's lane-major copies of x, P and y (state k = lane * L + s)
    const int NL = s.nb * s.nt;
    const int64_t cs = (int64_t)s.L * NL;
    T* lx = static_cast<T*>(h->lanes);
    T* lP = lx + 5 * cs;
    T* ly = lP + 15 * cs;
    PES_CUDA(h, launch_lanes_transpose<T>((const T*)y, ly, 2, N, s.L, NL, true, st));
    const bool cub = (method != PES_IEKS);
    if (x_init) PES_CUDA(h, launch_lanes_transpose<T>((const T*)x_init, lx, 5, N, s.L, NL, true, st));
    if (cub && P_init) PES_CUDA(h, launch_lanes_transpose<T>((const T*)P_init, lP, 15, N, s.L, NL, true, st));
    if (!x_init || (cub && !P_init))
        PES_CUDA(h, launch_init_nominal_lanes<T>(offsets, B, N, s.L, NL, (const T*)m0, (const T*)P0,
                                                 x_init ? nullptr : lx, (cub && !P_init) ? lP : nullptr, st));
    KParams<T> p{};
    p.N = N; p.offsets = offsets; p.B = B; p.mode = MODE_RUN; p.iters = max_iters; p.tol = tol;
    p.write_P_every_iter = tol > 0.0 ? 1 : 0;
    pes_status rm = device_model<T>(h, *model, B, st, p.model, method);
    if (rm != PES_OK) return rm;
    p.y = ly; p.m0 = (const T*)m0; p.P0 = (const T*)P0;
    p.x = lx; p.P = lP;
    p.lanes_layout = 1;
    r = run_persistent_shaped<T>(h, p, lin, s, st);
    if (r != PES_OK) return r;
    PES_CUDA(h, launch_lanes_transpose<T>(lx, (T*)x_out, 5, N, s.L, NL, false, st));
    PES_CUDA(h, launch_lanes_transpose<T>(lP, (T*)P_out, 15, N, s.L, NL, false, st));
    if (tol > 0.0 || iters_used) {
        int it = 0;
        r = read_status(h, st, &it);
        if (iters_used) *iters_used = it;
        return r;
    }
    return PES_OK;
}

// The sequential counterpart: one thread per trajectory over the caller's
// layout, the nominal held in x_out / P_out, smoothing elements in h->hand.
template <typename T>
static pes_status ieks_run_sequential_t(pes_handle* h, const pes_model* model, pes_method method, const void* y,
                                        const int64_t* offsets, int32_t B, int64_t N, const void* m0, const void* P0,
                                        const void* x_init, const void* P_init, int32_t max_iters, double tol,
                                        void* x_out, void* P_out, int32_t* iters_used, cudaStream_t st)
{
    const bool cub = (method != PES_IEKS);
    if (x_init && x_init != x_out) PES_CUDA(h, cudaMemcpyAsync(x_out, x_init, sizeof(T) * 5 * N, cudaMemcpyDeviceToDevice, st));
    if (cub && P_init && P_init != P_out)
        PES_CUDA(h, cudaMemcpyAsync(P_out, P_init, sizeof(T) * 15 * N, cudaMemcpyDeviceToDevice, st));
    if (!x_init || (cub && !P_init))
        PES_CUDA(h, launch_init_nominal<T>(offsets, B, N, (const T*)m0, (const T*)P0, x_init ? nullptr : (T*)x_out,
                                           (cub && !P_init) ? (T*)P_out : nullptr, st));
    KParams<T> p{};
    p.N = N; p.offsets = offsets; p.B = B; p.mode = MODE_RUN; p.iters = max_iters; p.tol = tol;
    pes_status rm = device_model<T>(h, *model, B, st, p.model, method);
    if (rm != PES_OK) return rm;
    p.y = (const T*)y; p.m0 = (const T*)m0; p.P0 = (const T*)P0;
    p.x = (T*)x_out; p.P = (T*)P_out;
    p.lanes_layout = 0;
    p.cs = N;
    p.hand = static_cast<T*>(h->hand);
    p.status = h->status;
    p.iters_done = h->iters_done;
    p.traj_iters = nullptr;
    PES_CUDA(h, cudaMemsetAsync(h->iters_done, 0, sizeof(int), st));
    if (tol > 0.0 && h->traj_iters) {
        PES_CUDA(h, cudaMemsetAsync(h->traj_iters, 0, sizeof(int) * B, st));
        p.traj_iters = h->traj_iters;
        h->traj_iters_B = B;
    }
    const cudaError_t e = !cub                           ? launch_sequential<T, LIN_IEKS>(p, st)
                          : method == PES_GAUSS_HERMITE ? launch_sequential<T, LIN_GH>(p, st)
                                                        : launch_sequential<T, LIN_CUBATURE>(p, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "launch of the sequential smoother");
    if (tol > 0.0 || iters_used) {
        int it = 0;
        pes_status r = read_status(h, st, &it);
        if (iters_used) *iters_used = it;
        return r;
    }
    return PES_OK;
}

// PES_MIXED: the first max_iters - 1 iterations in FP32, the last one (and so
// the returned means and smoother covariances) in FP64 from the FP32 nominal.
// Inputs and outputs are FP32 arrays; the FP64 copies live in h->mix.
static pes_status ieks_run_mixed(pes_handle* h, const pes_model* model, pes_method method, const void* y,
                                 const int64_t* offsets, int32_t B, int64_t N, const void* m0, const void* P0,
                                 const void* x_init, const void* P_init, int32_t max_iters, double tol, void* x_out,
                                 void* P_out, int32_t* iters_used, cudaStream_t st)
{
    if (!h->mix) {
        const size_t need = sizeof(double) * (22 * (size_t)h->max_states + 20 * (size_t)h->max_batch);
        PES_CUDA(h, cudaMalloc(&h->mix, need));
    }
    double* y64 = static_cast<double*>(h->mix);
    double* x64 = y64 + 2 * N;
    double* P64 = x64 + 5 * N;
    double* m064 = P64 + 15 * N;
    double* P064 = m064 + 5 * (size_t)B;
    int32_t it32 = 0;
    const bool cub = (method != PES_IEKS);
    const void* xi32 = x_init;
    const void* Pi32 = P_init;
    if (max_iters > 1) {
        pes::TraceRange trace_("FP32 iterations");
        pes_status r = ieks_run_t<float>(h, model, method, PES_FP32, y, offsets, B, N, m0, P0, x_init, P_init,
                                         max_iters - 1, tol, x_out, P_out, &it32, st);
        if (r != PES_OK && r != PES_ERR_NOT_CONVERGED) return r;
        xi32 = x_out;
        Pi32 = P_out;
    }
    pes::TraceRange trace_("final FP64 iteration");
    PES_CUDA(h, (launch_convert_ff<float, double>((const float*)y, y64, 2 * N, st)));
    PES_CUDA(h, (launch_convert_ff<float, double>((const float*)m0, m064, 5 * (int64_t)B, st)));
    PES_CUDA(h, (launch_convert_ff<float, double>((const float*)P0, P064, 15 * (int64_t)B, st)));
    if (xi32) PES_CUDA(h, (launch_convert_ff<float, double>((const float*)xi32, x64, 5 * N, st)));
    if (cub && Pi32) PES_CUDA(h, (launch_convert_ff<float, double>((const float*)Pi32, P64, 15 * N, st)));
    int32_t it64 = 0;
    const pes_status r = ieks_run_t<double>(h, model, method, PES_FP64, y64, offsets, B, N, m064, P064,
                                            xi32 ? x64 : nullptr, (cub && Pi32) ? P64 : nullptr, 1, tol, x64, P64,
                                            &it64, st);
    if (r != PES_OK && r != PES_ERR_NOT_CONVERGED) return r;
    PES_CUDA(h, (launch_convert_ff<double, float>(x64, (float*)x_out, 5 * N, st)));
    PES_CUDA(h, (launch_convert_ff<double, float>(P64, (float*)P_out, 15 * N, st)));
    if (iters_used) *iters_used = it32 + it64;
    PES_CUDA(h, cudaStreamSynchronize(st));
    return r;
}

// The refinement workspace: nominal and filtered moments (20 + 20 floats per
// slot), residual elements (RE), stored transitions (RT), the filter's
// correction (RD), for every lane-major slot the handle can hold.
static pes_status ensure_refine_workspace(pes_handle* h)
{
    if (h->refw) return PES_OK;
    const size_t slots = (size_t)h->max_states + (size_t)h->nl_max;
    PES_CUDA(h, cudaMalloc(&h->refw, sizeof(float) * (20 + 20 + RE + RT + RD) * slots));
    return PES_OK;
}

// PES_REFINED: the first max_iters - 1 iterations in FP32, then the final
// iteration in FP32 and its Newton refinement (pes_refine.cuh): float-float
// residuals of the filter and RTS recursions about the FP32 solution, and the
// corrections from two FP32 scans. Everything stays in the lane-major layout
// of the smoother kernel; the refinement workspace (155 floats per slot) is
// allocated by the first call on the handle.
static pes_status ieks_run_refined(pes_handle* h, const pes_model* model, pes_method method, const void* y,
                                   const int64_t* offsets, int32_t B, int64_t N, const void* m0, const void* P0,
                                   const void* x_init, const void* P_init, int32_t max_iters, double tol, void* x_out,
                                   void* P_out, int32_t* iters_used, cudaStream_t st)
{
    if (method == PES_GAUSS_HERMITE)
        return fail(h, PES_ERR_UNSUPPORTED, "PES_REFINED supports PES_IEKS, PES_CUBATURE and PES_UNSCENTED");
    if (model->lm_lambda > 0.0)
        return fail(h, PES_ERR_UNSUPPORTED, "PES_REFINED does not support Levenberg-Marquardt damping");
    const int lin = lin_of(method);
    Shape s;
    pes_status r = make_shape<float>(h, lin, PES_FP32, N, s);
    if (r != PES_OK) return r;
    const int cap = refine_scan_capacity(s.nt, h->device);
    if (cap < 0) {
        cudaGetLastError();
        return fail(h, PES_ERR_CUDA, "the refinement scan's occupancy query failed: %s",
                    cudaGetErrorString((cudaError_t)(-cap)));
    }
    if (cap < s.nb)
        return fail(h, PES_ERR_CUDA, "the refinement scan cannot be made co-resident (%d of %d blocks)", cap, s.nb);
    if ((r = ensure_refine_workspace(h)) != PES_OK) return r;
    const int NL = s.nb * s.nt;
    const int64_t cs = (int64_t)s.L * NL;
    float* lx = static_cast<float*>(h->lanes);
    float* lP = lx + 5 * cs;
    float* ly = lP + 15 * cs;
    float* nom = static_cast<float*>(h->refw);
    float* filt = nom + 20 * cs;
    float* elem = filt + 20 * cs;
    float* trans = elem + RE * cs;
    float* dlt = trans + RT * cs;
    PES_CUDA(h, launch_lanes_transpose<float>((const float*)y, ly, 2, N, s.L, NL, true, st));
    const bool cub = (method != PES_IEKS);
    if (x_init) PES_CUDA(h, launch_lanes_transpose<float>((const float*)x_init, lx, 5, N, s.L, NL, true, st));
    if (cub && P_init) PES_CUDA(h, launch_lanes_transpose<float>((const float*)P_init, lP, 15, N, s.L, NL, true, st));
    if (!x_init || (cub && !P_init))
        PES_CUDA(h, launch_init_nominal_lanes<float>(offsets, B, N, s.L, NL, (const float*)m0, (const float*)P0,
                                                     x_init ? nullptr : lx, (cub && !P_init) ? lP : nullptr, st));
    KParams<float> p{};
    p.N = N; p.offsets = offsets; p.B = B; p.mode = MODE_RUN;
    if ((r = device_model<float>(h, *model, B, st, p.model, method)) != PES_OK) return r;
    p.y = ly; p.m0 = (const float*)m0; p.P0 = (const float*)P0;
    p.x = lx; p.P = lP;
    p.lanes_layout = 1;
    int32_t it32 = 0;
    pes_status r32 = PES_OK;
    if (max_iters > 1) {
        pes::TraceRange trace_("FP32 iterations");
        p.iters = max_iters - 1;
        p.tol = tol;
        p.write_P_every_iter = tol > 0.0 ? 1 : 0;
        if ((r = run_persistent_shaped<float>(h, p, lin, s, st)) != PES_OK) return r;
        if (tol > 0.0) {
            r32 = read_status(h, st, &it32);
            if (r32 != PES_OK && r32 != PES_ERR_NOT_CONVERGED) return r32;
        } else {
            it32 = max_iters - 1;
        }
    }
    // the final iteration's nominal, then the iteration itself with its filtered moments kept
    PES_CUDA(h, cudaMemcpyAsync(nom, lx, sizeof(float) * 20 * cs, cudaMemcpyDeviceToDevice, st));
    p.iters = 1;
    p.tol = 0.0;
    p.write_P_every_iter = 1;
    p.fstore = filt;
    {
        pes::TraceRange trace_("final FP32 iteration");
        if ((r = run_persistent_shaped<float>(h, p, lin, s, st)) != PES_OK) return r;
    }
    {
        pes::TraceRange trace_refine_("refinement");
        RefineParams rp{};
        rp.N = N; rp.offsets = offsets; rp.B = B; rp.L = s.L; rp.NL = NL; rp.cs = cs;
        rp.model = p.model;
        rp.y = ly; rp.m0 = (const float*)m0; rp.P0 = (const float*)P0;
        rp.nom = nom; rp.filt = filt; rp.xs = lx;
        rp.elem = elem; rp.trans = trans; rp.dlt = dlt;
        rp.agg = static_cast<float*>(h->aggF);
        rp.bar = h->bar;
        rp.status = h->status;
        rp.timeout_ns = h->timeout_ns;
        PES_CUDA(h, launch_refine_fwd(rp, lin, st));
        PES_CUDA(h, cudaMemsetAsync(h->bar, 0, sizeof(unsigned), st));
        cudaError_t e = launch_refine_scan(rp, true, s.nt, s.nb, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "cooperative launch of the refinement scan");
        PES_CUDA(h, launch_refine_bwd(rp, st));
        PES_CUDA(h, cudaMemsetAsync(h->bar, 0, sizeof(unsigned), st));
        e = launch_refine_scan(rp, false, s.nt, s.nb, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "cooperative launch of the refinement scan");
    }
    PES_CUDA(h, launch_lanes_transpose<float>(lx, (float*)x_out, 5, N, s.L, NL, false, st));
    PES_CUDA(h, launch_lanes_transpose<float>(lP, (float*)P_out, 15, N, s.L, NL, false, st));
    if (tol > 0.0 || iters_used) {
        r = read_status(h, st);
        if (iters_used) *iters_used = it32 + 1;
        return r != PES_OK ? r : r32;
    }
    return PES_OK;
}

// Process and measurement noise of the model in FP64 (packed), as the
// kernels receive them.
static void model_noise(const pes_model& m, double Q[15], double R[3])
{
    for (int i = 0; i < 15; ++i) Q[i] = 0.0;
    for (int i = 0; i < 3; ++i) R[i] = 0.0;
    if (m.kind == PES_MODEL_LINEAR) {
        for (int i = 0; i < 15; ++i) Q[i] = m.Q[i];
        for (int i = 0; i < 3; ++i) R[i] = m.R[i];
        return;
    }
    const double dt = m.dt;
    if (m.q_form == 1) {
        for (int ax = 0; ax < 2; ++ax) {
            Q[si(ax, ax)] = m.q_c * dt * dt * dt / 3.0;
            Q[si(ax, ax + 2)] = m.q_c * dt * dt / 2.0;
            Q[si(ax + 2, ax + 2)] = m.q_c * dt;
        }
    } else {
        Q[si(2, 2)] = m.q_c * dt;
        Q[si(3, 3)] = m.q_c * dt;
    }
    Q[si(4, 4)] = m.q_w * dt;
    R[0] = R[2] = m.r_std * m.r_std;
}

// Inverse of a packed symmetric n x n (n <= 5) matrix by its Cholesky factor;
// false if it is not positive definite.
static bool inv_spd_packed(const double* S, int n, double* Si)
{
    auto at = [&](int i, int j) { return n == 5 ? S[si(std::min(i, j), std::max(i, j))] : S[std::min(i, j) + std::max(i, j)]; };
    double L[25] = {0}, X[25] = {0};
    for (int j = 0; j < n; ++j) {
        double d = at(j, j);
        for (int l = 0; l < j; ++l) d -= L[j * 5 + l] * L[j * 5 + l];
        if (!(d > 0.0)) return false;
        L[j * 5 + j] = std::sqrt(d);
        for (int i = j + 1; i < n; ++i) {
            double t = at(i, j);
            for (int l = 0; l < j; ++l) t -= L[i * 5 + l] * L[j * 5 + l];
            L[i * 5 + j] = t / L[j * 5 + j];
        }
    }
    for (int c = 0; c < n; ++c) {   // columns of S^{-1}: L L^T x = e_c
        double z[5];
        for (int i = 0; i < n; ++i) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int l = 0; l < i; ++l) t -= L[i * 5 + l] * z[l];
            z[i] = t / L[i * 5 + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double t = z[i];
            for (int l = i + 1; l < n; ++l) t -= L[l * 5 + i] * X[l * 5 + c];
            X[i * 5 + c] = t / L[i * 5 + i];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) Si[n == 5 ? si(i, j) : i + j] = 0.5 * (X[i * 5 + j] + X[j * 5 + i]);
    return true;
}

// The IEKS with Levenberg-Marquardt steps and adaptive per-trajectory damping
// (host loop; kernels in pes_lm.cu). Every iteration: keep the nominal, run
// one damped iteration of the smoother kernel with each trajectory's damping,
// evaluate the MAP objective, keep or undo each trajectory's step.
template <typename T>
static pes_status ieks_run_lm_t(pes_handle* h, const pes_model* model, pes_precision prec, const void* y,
                                const int64_t* offsets, int32_t B, int64_t N, const void* m0, const void* P0,
                                const void* x_init, int32_t max_iters, double tol, double lambda0, double nu,
                                void* x_out, void* P_out, int32_t* iters_used, double* lambda_out,
                                int32_t* accepted_out, int32_t* conv_out, cudaStream_t st)
{
    LMParams lp{};
    double Q[15], R[3];
    model_noise(*model, Q, R);
    if (!inv_spd_packed(Q, 5, lp.Qi) || !inv_spd_packed(R, 2, lp.Ri))
        return fail(h, PES_ERR_UNSUPPORTED,
                    "the MAP objective needs positive definite Q and R (q_form 1, or a linear model with them)");
    Shape s;
    pes_status r = make_shape<T>(h, LIN_IEKS, prec, N, s);
    if (r != PES_OK) return r;
    if ((r = ensure_refine_workspace(h)) != PES_OK) return r;
    if (!h->lmw) {
        const size_t per = 5 * sizeof(double) + 3 * sizeof(int);
        PES_CUDA(h, cudaMalloc(&h->lmw, per * (size_t)h->max_batch + 16));
    }
    const int NL = s.nb * s.nt;
    const int64_t cs = (int64_t)s.L * NL;
    T* lx = static_cast<T*>(h->lanes);
    T* lP = lx + 5 * cs;
    T* ly = lP + 15 * cs;
    T* xold = static_cast<T*>(h->refw);
    T* Pold = xold + 5 * cs;
    const size_t Bm = (size_t)h->max_batch;
    double* dw = static_cast<double*>(h->lmw);
    lp.cost = dw;
    lp.cost_new = dw + Bm;
    lp.num = dw + 2 * Bm;
    lp.den = dw + 3 * Bm;
    T* lam = reinterpret_cast<T*>(dw + 4 * Bm);
    int* iw = reinterpret_cast<int*>(dw + 5 * Bm);
    lp.reject = iw;
    lp.accepted = iw + Bm;
    lp.conv_iter = iw + 2 * Bm;
    lp.unconv = iw + 3 * Bm;
    lp.N = N; lp.offsets = offsets; lp.B = B; lp.L = s.L; lp.NL = NL; lp.cs = cs;
    lp.kind = model->kind;
    lp.dt = model->dt;
    lp.sensors = model->sensors;
    lp.sensors_per_traj = model->sensors_per_traj;
    for (int i = 0; i < 25; ++i) lp.F[i] = model->F[i];
    for (int i = 0; i < 5; ++i) lp.c[i] = model->c[i];
    for (int i = 0; i < 10; ++i) lp.H[i] = model->H[i];
    for (int i = 0; i < 2; ++i) lp.d[i] = model->d[i];
    PES_CUDA(h, launch_lanes_transpose<T>((const T*)y, ly, 2, N, s.L, NL, true, st));
    if (x_init) PES_CUDA(h, launch_lanes_transpose<T>((const T*)x_init, lx, 5, N, s.L, NL, true, st));
    // covariances start at the prior's: a trajectory whose every step is
    // rejected returns them
    PES_CUDA(h, launch_init_nominal_lanes<T>(offsets, B, N, s.L, NL, (const T*)m0, (const T*)P0,
                                             x_init ? nullptr : lx, lP, st));
    PES_CUDA(h, cudaMemsetAsync(lp.accepted, 0, 2 * Bm * sizeof(int), st));
    PES_CUDA(h, launch_lm_fill<T>(lam, B, lambda0, st));
    PES_CUDA(h, cudaMemsetAsync(lp.cost, 0, B * sizeof(double), st));
    PES_CUDA(h, launch_lm_cost<T>(lp, lp.cost, lx, nullptr, ly, (const T*)m0, (const T*)P0, st));
    KParams<T> p{};
    p.N = N; p.offsets = offsets; p.B = B; p.mode = MODE_RUN; p.iters = 1; p.tol = 0.0;
    if ((r = device_model<T>(h, *model, B, st, p.model, PES_IEKS)) != PES_OK) return r;
    p.model.lm = T(0);
    p.model.lm_traj = lam;
    p.y = ly; p.m0 = (const T*)m0; p.P0 = (const T*)P0;
    p.x = lx; p.P = lP;
    p.lanes_layout = 1;
    int it = 0;
    bool all = false;
    for (it = 1; it <= max_iters; ++it) {
        PES_CUDA(h, cudaMemcpyAsync(xold, lx, sizeof(T) * 20 * cs, cudaMemcpyDeviceToDevice, st));
        if ((r = run_persistent_shaped<T>(h, p, LIN_IEKS, s, st)) != PES_OK) return r;
        PES_CUDA(h, cudaMemsetAsync(lp.cost_new, 0, 3 * Bm * sizeof(double), st));
        PES_CUDA(h, cudaMemsetAsync(lp.unconv, 0, sizeof(int), st));
        PES_CUDA(h, launch_lm_cost<T>(lp, lp.cost_new, lx, xold, ly, (const T*)m0, (const T*)P0, st));
        PES_CUDA(h, launch_lm_decide<T>(lp, lam, it, tol, nu, st));
        PES_CUDA(h, launch_lm_restore<T>(lp, lx, lP, xold, Pold, st));
        if (tol > 0.0) {
            int un = 0;
            PES_CUDA(h, cudaMemcpyAsync(&un, lp.unconv, sizeof(int), cudaMemcpyDeviceToHost, st));
            PES_CUDA(h, cudaStreamSynchronize(st));
            if (un == 0) {
                all = true;
                break;
            }
        }
    }
    if (it > max_iters) it = max_iters;
    PES_CUDA(h, launch_lanes_transpose<T>(lx, (T*)x_out, 5, N, s.L, NL, false, st));
    PES_CUDA(h, launch_lanes_transpose<T>(lP, (T*)P_out, 15, N, s.L, NL, false, st));
    if (lambda_out) {
        T* tmp = new (std::nothrow) T[B];
        if (!tmp) return fail(h, PES_ERR_CUDA, "out of host memory");
        cudaError_t e = cudaMemcpyAsync(tmp, lam, sizeof(T) * B, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        for (int b = 0; b < B && e == cudaSuccess; ++b) lambda_out[b] = (double)tmp[b];
        delete[] tmp;
        if (e != cudaSuccess) return cuda_fail(h, e, "reading the dampings");
    }
    if (accepted_out)
        PES_CUDA(h, cudaMemcpyAsync(accepted_out, lp.accepted, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
    if (conv_out) PES_CUDA(h, cudaMemcpyAsync(conv_out, lp.conv_iter, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
    r = read_status(h, st);
    if (iters_used) *iters_used = it;
    if (r == PES_OK && tol > 0.0 && !all) r = fail(h, PES_ERR_NOT_CONVERGED, "the tolerance was not reached within max_iters");
    return r;
}

struct pes_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

pes_status pes_create(pes_handle** out, int64_t max_states, int32_t max_batch)
{
    if (!out || max_states < 1 || max_batch < 1) return PES_ERR_INVALID_ARG;
    *out = nullptr;
    pes_handle* h = new (std::nothrow) pes_handle();
    if (!h) return PES_ERR_CUDA;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        delete h;
        return PES_ERR_CUDA;
    }
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device);
    if (!coop) {
        delete h;
        return PES_ERR_UNSUPPORTED;
    }
    if (const char* env = getenv("PES_BARRIER_TIMEOUT_MS")) {
        const long long ms = atoll(env);
        if (ms > 0) h->timeout_ns = ms * 1000000LL;
    }
    if (const char* env = getenv("PES_TEST_BARRIER_SHORT")) h->bar_short = atoi(env) != 0;
    h->max_states = max_states;
    h->max_batch = max_batch;
    h->nb_max = h->num_sms * kMaxBlocksPerSM;
    h->nl_max = h->nb_max * kMaxThreads;
    const size_t hand_elems = (size_t)HAND * ((size_t)max_states + (size_t)h->nl_max);
    e = cudaMalloc(&h->hand, hand_elems * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->lanes, (size_t)22 * ((size_t)max_states + (size_t)h->nl_max) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->lin, (size_t)LINS * ((size_t)max_states + (size_t)h->nl_max) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->aggF, (size_t)h->nb_max * FE * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->aggS, (size_t)h->nb_max * SE * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->bar, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->conv, sizeof(double) * 4 * (size_t)max_batch);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->iters_done, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->traj_iters, sizeof(int) * (size_t)max_batch);
    if (e == cudaSuccess) e = cudaMalloc(&h->sensT, sizeof(double) * 4 * (size_t)max_batch);
    if (e == cudaSuccess && getenv("PES_PHASE_TIMES") && atoi(getenv("PES_PHASE_TIMES")) > 0) {
        e = cudaMalloc((void**)&h->ptime, sizeof(long long) * NPHASE * (size_t)h->nb_max);
        if (e == cudaSuccess) e = cudaMemset(h->ptime, 0, sizeof(long long) * NPHASE * (size_t)h->nb_max);
    }
    if (e == cudaSuccess) e = cudaMemset(h->status, 0, sizeof(int));
    if (e != cudaSuccess) {
        pes_destroy(h);
        return PES_ERR_CUDA;
    }
    *out = h;
    return PES_OK;
}

pes_status pes_destroy(pes_handle* h)
{
    if (!h) return PES_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    void* ptrs[] = {h->hand, h->lanes, h->lin, h->mix, h->refw, h->lmw, h->aggF, h->aggS, h->bar, h->status, h->conv, h->iters_done, h->traj_iters, h->sensT, h->ptime,
                    h->hy, h->hoff, h->hm0, h->hP0, h->hx, h->hP, h->hsens};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete h;
    return PES_OK;
}

const char* pes_last_error(const pes_handle* h) { return h ? h->err : "null handle"; }

pes_status pes_sync(pes_handle* h, void* stream)
{
    if (!h) return PES_ERR_INVALID_ARG;
    return read_status(h, (cudaStream_t)stream);
}

pes_status pes_debug_phase_times(pes_handle* h, double* mean_ns, double* max_ns, int32_t n)
{
    if (!h || !mean_ns || n < 1) return PES_ERR_INVALID_ARG;
    if (!h->ptime || h->ptime_blocks < 1) return fail(h, PES_ERR_UNSUPPORTED, "phase timing is off (set PES_PHASE_TIMES=1 before pes_create)");
    const int nb = h->ptime_blocks;
    long long* buf = (long long*)malloc(sizeof(long long) * NPHASE * nb);
    if (!buf) return PES_ERR_CUDA;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(buf, h->ptime, sizeof(long long) * NPHASE * nb, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        free(buf);
        return cuda_fail(h, e, "reading phase timestamps");
    }
    for (int i = 0; i < n && i < NPHASE - 1; ++i) {
        double sum = 0.0, mx = 0.0;
        int cnt = 0;
        for (int b = 0; b < nb; ++b) {
            const long long t0 = buf[b * NPHASE + i], t1 = buf[b * NPHASE + i + 1];
            if (t0 > 0 && t1 >= t0) {
                sum += double(t1 - t0);
                mx = std::max(mx, double(t1 - t0));
                ++cnt;
            }
        }
        mean_ns[i] = cnt ? sum / cnt : -1.0;
        if (max_ns) max_ns[i] = cnt ? mx : -1.0;
    }
    free(buf);
    return PES_OK;
}

pes_status pes_set_launch_shape(pes_handle* h, pes_method method, pes_precision prec, int32_t threads,
                                int32_t min_steps)
{
    if (!h) return PES_ERR_INVALID_ARG;
    if (prec != PES_FP32 && prec != PES_FP64) return fail(h, PES_ERR_INVALID_ARG, "launch shapes are per FP32 or FP64");
    if (method < PES_IEKS || method > PES_GAUSS_HERMITE) return fail(h, PES_ERR_INVALID_ARG, "unknown method");
    const bool defaults = (threads == 0 && min_steps == 0);
    const bool compiled = prec == PES_FP64 ? nt_supported(0.0, threads) : nt_supported(0.0f, threads);
    if (!defaults && (!compiled || min_steps < 1 || min_steps > (1 << 20)))
        return fail(h, PES_ERR_INVALID_ARG, "no compiled launch of %d threads with at least %d steps per lane",
                    (int)threads, (int)min_steps);
    pes_tune& slot = h->tune[lin_of(method)][prec == PES_FP64 ? 1 : 0];
    slot.nt = threads;
    slot.min_steps = min_steps;
    return PES_OK;
}

pes_status pes_launch_shape(pes_handle* h, pes_method method, pes_precision prec, int64_t N, int32_t* blocks,
                            int32_t* threads, int32_t* steps_per_thread)
{
    if (!h || N < 1) return PES_ERR_INVALID_ARG;
    if (prec == PES_MIXED) return PES_ERR_UNSUPPORTED;
    if (prec == PES_REFINED) prec = PES_FP32;   // its iterations run the FP32 kernel
    const int lin = lin_of(method);
    Shape s;
    pes_status r = (prec == PES_FP64) ? make_shape<double>(h, lin, prec, N, s) : make_shape<float>(h, lin, prec, N, s);
    if (r != PES_OK) return r;
    if (blocks) *blocks = s.nb;
    if (threads) *threads = s.nt;
    if (steps_per_thread) *steps_per_thread = s.L;
    return PES_OK;
}

pes_status pes_ieks_graph_create(pes_handle* h, const pes_model* model, pes_method method, pes_precision prec,
                                 const void* y, const int64_t* offsets, int32_t B, int64_t N, const void* m0,
                                 const void* P0, const void* x_init, const void* P_init, int32_t iters, void* x_out,
                                 void* P_out, pes_graph** out)
{
    pes::TraceRange trace_("pes_ieks_graph_create");
    if (!h || !out) return PES_ERR_INVALID_ARG;
    *out = nullptr;
    if (prec == PES_MIXED) return fail(h, PES_ERR_UNSUPPORTED, "PES_MIXED synchronises and cannot be captured");
    if (prec == PES_REFINED) {
        // allocate outside the capture
        const pes_status ra = ensure_refine_workspace(h);
        if (ra != PES_OK) return ra;
    }
    cudaStream_t cs = nullptr;
    PES_CUDA(h, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    pes_status r = PES_OK;
    if (e == cudaSuccess) {
        r = pes_ieks_run(h, model, method, prec, y, offsets, B, N, m0, P0, x_init, P_init, iters, 0.0, x_out, P_out,
                         nullptr, cs);
        const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);   // ends the capture whatever happened
        if (r == PES_OK && e2 != cudaSuccess) r = cuda_fail(h, e2, "stream capture of the smoother");
    } else {
        r = cuda_fail(h, e, "cudaStreamBeginCapture");
    }
    cudaStreamDestroy(cs);
    cudaGraphExec_t exec = nullptr;
    if (r == PES_OK) {
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) r = cuda_fail(h, e, "cudaGraphInstantiate");
    }
    if (r != PES_OK) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return r;
    }
    pes_graph* g = new (std::nothrow) pes_graph();
    if (!g) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return fail(h, PES_ERR_CUDA, "out of host memory");
    }
    g->graph = graph;
    g->exec = exec;
    *out = g;
    return PES_OK;
}

pes_status pes_graph_launch(pes_graph* g, void* stream)
{
    if (!g) return PES_ERR_INVALID_ARG;
    return cudaGraphLaunch(g->exec, (cudaStream_t)stream) == cudaSuccess ? PES_OK : PES_ERR_CUDA;
}

pes_status pes_graph_destroy(pes_graph* g)
{
    if (!g) return PES_ERR_INVALID_ARG;
    cudaGraphExecDestroy(g->exec);
    cudaGraphDestroy(g->graph);
    delete g;
    return PES_OK;
}

pes_status pes_autotune(pes_handle* h, const pes_model* model, pes_method method, pes_precision prec, const void* y,
                        const int64_t* offsets, int32_t B, int64_t N, const void* m0, const void* P0,
                        int32_t iters, void* x_scratch, void* P_scratch, int32_t* threads, int32_t* min_steps,
                        float* ms_per_run, void* stream)
{
    pes::TraceRange trace_("pes_autotune");
    if (!h) return PES_ERR_INVALID_ARG;
    if (prec != PES_FP32 && prec != PES_FP64) return fail(h, PES_ERR_INVALID_ARG, "autotune FP32 or FP64");
    if (iters < 1 || !x_scratch || !P_scratch) return fail(h, PES_ERR_INVALID_ARG, "iters >= 1 and scratch needed");
    cudaStream_t st = (cudaStream_t)stream;
    const int lin = lin_of(method);
    pes_tune& slot = h->tune[lin][prec == PES_FP64 ? 1 : 0];
    const pes_tune saved = slot;
    const int nts32[] = {128, 256}, nts64[] = {128};
    const int* nts = prec == PES_FP64 ? nts64 : nts32;
    const int n_nt = prec == PES_FP64 ? 1 : 2;
    const int steps[] = {4, 8, 16, 32, 64, 128};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PES_CUDA(h, cudaEventCreate(&e0));
    PES_CUDA(h, cudaEventCreate(&e1));
    float best = 1e30f;
    pes_tune best_t;
    int seen_nb[16], seen_nt[16], n_seen = 0;
    pes_status r = PES_OK;
    for (int a = 0; a < n_nt && r == PES_OK; ++a) {
        for (int b = 0; b < 6 && r == PES_OK; ++b) {
            slot.nt = nts[a];
            slot.min_steps = steps[b];
            Shape s;
            r = (prec == PES_FP64) ? make_shape<double>(h, lin, prec, N, s) : make_shape<float>(h, lin, prec, N, s);
            if (r != PES_OK) break;
            bool dup = false;   // candidates that give the same launch are timed once
            for (int q = 0; q < n_seen; ++q) dup |= (seen_nb[q] == s.nb && seen_nt[q] == s.nt);
            if (dup) continue;
            seen_nb[n_seen] = s.nb;
            seen_nt[n_seen++] = s.nt;
            float ms = 1e30f;
            for (int rep = 0; rep < 2 && r == PES_OK; ++rep) {   // the first run warms up
                cudaEventRecord(e0, st);
                r = pes_ieks_run(h, model, method, prec, y, offsets, B, N, m0, P0, nullptr, nullptr, iters, 0.0,
                                 x_scratch, P_scratch, nullptr, stream);
                cudaEventRecord(e1, st);
                if (r == PES_OK) r = pes_sync(h, stream);
                float t = 0.f;
                if (r == PES_OK && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && rep == 1) ms = t;
            }
            if (r == PES_OK && ms < best) {
                best = ms;
                best_t = slot;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != PES_OK) {
        slot = saved;
        return r;
    }
    slot = best_t;
    if (threads) *threads = best_t.nt;
    if (min_steps) *min_steps = best_t.min_steps;
    if (ms_per_run) *ms_per_run = best;
    return PES_OK;
}

pes_status pes_linearize(pes_handle* h, const pes_model* model, pes_method method, pes_precision prec,
                         const void* x_nom, const void* P_nom, const void* y, const int64_t* offsets, int32_t B,
                         int64_t N, void* F, void* c, void* Qp, void* H, void* d, void* Rp, void* y_used,
                         void* stream)
{
    pes::TraceRange trace_("pes_linearize");
    pes_status r = check_common(h, prec, offsets, B, N);
    if (r != PES_OK) return r;
    if ((r = check_model(h, model)) != PES_OK) return r;
    if ((r = check_method(h, method, model)) != PES_OK) return r;
    if (!x_nom || !y || !F || !c || !Qp || !H || !d || !Rp) return fail(h, PES_ERR_INVALID_ARG, "NULL array");
    if (method != PES_IEKS && !P_nom) return fail(h, PES_ERR_INVALID_ARG, "sigma-point methods need P_nom");
    cudaStream_t st = (cudaStream_t)stream;
    PES_CUDA(h, launch_validate_offsets(offsets, B, N, h->status, st));
    const int lin = lin_of(method);
    if (prec == PES_FP64) {
        KParams<double> p{};
        p.N = N; p.offsets = offsets; p.B = B;
        if ((r = device_model<double>(h, *model, B, st, p.model, method)) != PES_OK) return r;
        p.x = (double*)x_nom; p.P = (double*)P_nom; p.y = (const double*)y; p.status = h->status; p.cs = N;
        PES_CUDA(h, launch_linearize<double>(p, lin, (double*)F, (double*)c, (double*)Qp, (double*)H, (double*)d,
                                             (double*)Rp, (double*)y_used, st));
    } else {
        KParams<float> p{};
        p.N = N; p.offsets = offsets; p.B = B;
        if ((r = device_model<float>(h, *model, B, st, p.model, method)) != PES_OK) return r;
        p.x = (float*)x_nom; p.P = (float*)P_nom; p.y = (const float*)y; p.status = h->status; p.cs = N;
        PES_CUDA(h, launch_linearize<float>(p, lin, (float*)F, (float*)c, (float*)Qp, (float*)H, (float*)d,
                                            (float*)Rp, (float*)y_used, st));
    }
    return PES_OK;
}


pes_status pes_filter_scan(pes_handle* h, pes_precision prec, const void* F, const void* c, const void* Qp,
                           const void* H, const void* d, const void* Rp, const void* y, const void* m0,
                           const void* P0, const int64_t* offsets, int32_t B, int64_t N, void* xf, void* Pf,
                           void* stream)
{
    pes::TraceRange trace_("pes_filter_scan");
    pes_status r = check_common(h, prec, offsets, B, N);
    if (r != PES_OK) return r;
    if (!F || !c || !Qp || !H || !d || !Rp || !y || !m0 || !P0 || !xf || !Pf)
        return fail(h, PES_ERR_INVALID_ARG, "NULL array");
    cudaStream_t st = (cudaStream_t)stream;
    PES_CUDA(h, launch_validate_offsets(offsets, B, N, h->status, st));
    if (prec == PES_FP64) return filter_scan_t<double>(h, F, c, Qp, H, d, Rp, y, m0, P0, offsets, B, N, xf, Pf, prec, st);
    return filter_scan_t<float>(h, F, c, Qp, H, d, Rp, y, m0, P0, offsets, B, N, xf, Pf, prec, st);
}


pes_status pes_filter_loglik(pes_handle* h, pes_precision prec, const void* F, const void* c, const void* Qp,
                             const void* H, const void* d, const void* Rp, const void* y, const void* m0,
                             const void* P0, const int64_t* offsets, int32_t B, int64_t N, void* xf, void* Pf,
                             double* loglik, void* stream)
{
    pes::TraceRange trace_("pes_filter_loglik");
    pes_status r = check_common(h, prec, offsets, B, N);
    if (r != PES_OK) return r;
    if (!F || !c || !Qp || !H || !d || !Rp || !y || !m0 || !P0 || !xf || !Pf || !loglik)
        return fail(h, PES_ERR_INVALID_ARG, "NULL array");
    cudaStream_t st = (cudaStream_t)stream;
    PES_CUDA(h, launch_validate_offsets(offsets, B, N, h->status, st));
    if (prec == PES_FP64)
        return filter_scan_t<double>(h, F, c, Qp, H, d, Rp, y, m0, P0, offsets, B, N, xf, Pf, prec, st, loglik);
    return filter_scan_t<float>(h, F, c, Qp, H, d, Rp, y, m0, P0, offsets, B, N, xf, Pf, prec, st, loglik);
}

pes_status pes_smooth_scan(pes_handle* h, pes_precision prec, const void* F, const void* c, const void* Qp,
                           const void* xf, const void* Pf, const int64_t* offsets, int32_t B, int64_t N, void* xs,
                           void* Ps, void* stream)
{
    pes::TraceRange trace_("pes_smooth_scan");
    pes_status r = check_common(h, prec, offsets, B, N);
    if (r != PES_OK) return r;
    if (!F || !c || !Qp || !xf || !Pf || !xs || !Ps) return fail(h, PES_ERR_INVALID_ARG, "NULL array");
    cudaStream_t st = (cudaStream_t)stream;
    PES_CUDA(h, launch_validate_offsets(offsets, B, N, h->status, st));
    if (prec == PES_FP64) return smooth_scan_t<double>(h, F, c, Qp, xf, Pf, offsets, B, N, xs, Ps, prec, st);
    return smooth_scan_t<float>(h, F, c, Qp, xf, Pf, offsets, B, N, xs, Ps, prec, st);
}


pes_status pes_ieks_run(pes_handle* h, const pes_model* model, pes_method method, pes_precision prec, const void* y,
                        const int64_t* offsets, int32_t B, int64_t N, const void* m0, const void* P0,
                        const void* x_init, const void* P_init, int32_t max_iters, double tol, void* x_out,
                        void* P_out, int32_t* iters_used, void* stream)
{
    pes::TraceRange trace_("pes_ieks_run");
    pes_status r = check_common(h, prec, offsets, B, N, true);
    if (r != PES_OK) return r;
    if ((r = check_model(h, model)) != PES_OK) return r;
    if ((r = check_method(h, method, model)) != PES_OK) return r;
    if (!y || !m0 || !P0 || !x_out || !P_out) return fail(h, PES_ERR_INVALID_ARG, "NULL array");
    if (max_iters < 1) return fail(h, PES_ERR_INVALID_ARG, "max_iters must be >= 1");
    if (!(tol == tol)) return fail(h, PES_ERR_INVALID_ARG, "tol is NaN");
    cudaStream_t st = (cudaStream_t)stream;
    PES_CUDA(h, launch_validate_offsets(offsets, B, N, h->status, st));
    if (prec == PES_MIXED)
        return ieks_run_mixed(h, model, method, y, offsets, B, N, m0, P0, x_init, P_init, max_iters, tol, x_out, P_out,
                              iters_used, st);
    if (prec == PES_REFINED)
        return ieks_run_refined(h, model, method, y, offsets, B, N, m0, P0, x_init, P_init, max_iters, tol, x_out,
                                P_out, iters_used, st);
    if (prec == PES_FP64)
        return ieks_run_t<double>(h, model, method, prec, y, offsets, B, N, m0, P0, x_init, P_init, max_iters, tol,
                                  x_out, P_out, iters_used, st);
    return ieks_run_t<float>(h, model, method, prec, y, offsets, B, N, m0, P0, x_init, P_init, max_iters, tol, x_out,
                             P_out, iters_used, st);
}

pes_status pes_ieks_run_lm(pes_handle* h, const pes_model* model, pes_precision prec, const void* y,
                           const int64_t* offsets, int32_t B, int64_t N, const void* m0, const void* P0,
                           const void* x_init, int32_t max_iters, double tol, double lambda0, double nu,
                           void* x_out, void* P_out, int32_t* iters_used, double* lambda_out,
                           int32_t* accepted_out, int32_t* conv_iter_out, void* stream)
{
    pes::TraceRange trace_("pes_ieks_run_lm");
    pes_status r = check_common(h, prec, offsets, B, N);
    if (r != PES_OK) return r;
    if ((r = check_model(h, model)) != PES_OK) return r;
    if (!y || !m0 || !P0 || !x_out || !P_out) return fail(h, PES_ERR_INVALID_ARG, "NULL array");
    if (max_iters < 1) return fail(h, PES_ERR_INVALID_ARG, "max_iters must be >= 1");
    if (!(lambda0 > 0.0) || !std::isfinite(lambda0) || !(nu > 1.0) || !std::isfinite(nu) || !(tol == tol))
        return fail(h, PES_ERR_INVALID_ARG, "lambda0 > 0 and nu > 1 (finite), tol not NaN");
    if (model->lm_lambda != 0.0) return fail(h, PES_ERR_INVALID_ARG, "the damping is adaptive here: lm_lambda must be 0");
    cudaStream_t st = (cudaStream_t)stream;
    PES_CUDA(h, launch_validate_offsets(offsets, B, N, h->status, st));
    if (prec == PES_FP64)
        return ieks_run_lm_t<double>(h, model, prec, y, offsets, B, N, m0, P0, x_init, max_iters, tol, lambda0, nu,
                                     x_out, P_out, iters_used, lambda_out, accepted_out, conv_iter_out, st);
    return ieks_run_lm_t<float>(h, model, prec, y, offsets, B, N, m0, P0, x_init, max_iters, tol, lambda0, nu, x_out,
                                P_out, iters_used, lambda_out, accepted_out, conv_iter_out, st);
}

pes_status pes_ieks_run_sequential(pes_handle* h, const pes_model* model, pes_method method, pes_precision prec,
                                   const void* y, const int64_t* offsets, int32_t B, int64_t N, const void* m0,
                                   const void* P0, const void* x_init, const void* P_init, int32_t max_iters,
                                   double tol, void* x_out, void* P_out, int32_t* iters_used, void* stream)
{
    pes::TraceRange trace_("pes_ieks_run_sequential");
    pes_status r = check_common(h, prec, offsets, B, N);
    if (r != PES_OK) return r;
    if ((r = check_model(h, model)) != PES_OK) return r;
    if ((r = check_method(h, method, model)) != PES_OK) return r;
    if (!y || !m0 || !P0 || !x_out || !P_out) return fail(h, PES_ERR_INVALID_ARG, "NULL array");
    if (max_iters < 1) return fail(h, PES_ERR_INVALID_ARG, "max_iters must be >= 1");
    if (!(tol == tol)) return fail(h, PES_ERR_INVALID_ARG, "tol is NaN");
    cudaStream_t st = (cudaStream_t)stream;
    PES_CUDA(h, launch_validate_offsets(offsets, B, N, h->status, st));
    if (prec == PES_FP64)
        return ieks_run_sequential_t<double>(h, model, method, y, offsets, B, N, m0, P0, x_init, P_init, max_iters,
                                             tol, x_out, P_out, iters_used, st);
    return ieks_run_sequential_t<float>(h, model, method, y, offsets, B, N, m0, P0, x_init, P_init, max_iters, tol,
                                        x_out, P_out, iters_used, st);
}

pes_status pes_traj_iterations(pes_handle* h, int32_t* iters, int32_t B, void* stream)
{
    if (!h || !iters) return fail(h, PES_ERR_INVALID_ARG, "NULL argument");
    if (B != h->traj_iters_B || B < 1)
        return fail(h, PES_ERR_INVALID_ARG, "no tolerance-mode run over %d trajectories was recorded", (int)B);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    PES_CUDA(h, cudaMemcpyAsync(iters, h->traj_iters, sizeof(int32_t) * B, cudaMemcpyDeviceToHost, st));
    PES_CUDA(h, cudaStreamSynchronize(st));
    return PES_OK;
}

pes_status pes_ieks_run_host(pes_handle* h, const pes_model* model, pes_method method, pes_precision prec,
                             const void* y, const int64_t* offsets, int32_t B, int64_t N, const void* m0,
                             const void* P0, const void* x_init, const void* P_init, int32_t max_iters, double tol,
                             void* x_out, void* P_out, int32_t* iters_used, void* stream)
{
    pes::TraceRange trace_("pes_ieks_run_host");
    if (!h) return PES_ERR_INVALID_ARG;
    if (prec != PES_FP32 && prec != PES_FP64 && prec != PES_MIXED && prec != PES_REFINED)
        return fail(h, PES_ERR_INVALID_ARG, "unknown precision");
    if (!model || !y || !offsets || !m0 || !P0 || !x_out || !P_out) return fail(h, PES_ERR_INVALID_ARG, "NULL array");
    if (B < 1 || N < B || N > h->max_states || B > h->max_batch)
        return fail(h, PES_ERR_INVALID_ARG, "sizes out of range (N %lld, B %d)", (long long)N, (int)B);
    // host-side offsets check (they are host memory here)
    if (offsets[0] != 0 || offsets[B] != N) return fail(h, PES_ERR_INVALID_ARG, "offsets must start at 0 and end at N");
    for (int32_t b = 0; b < B; ++b)
        if (offsets[b + 1] <= offsets[b]) return fail(h, PES_ERR_INVALID_ARG, "offsets must increase strictly");
    const size_t ts = scalar_size(prec);
    const size_t Nmax = (size_t)h->max_states, Bmax = (size_t)h->max_batch;
    if (!h->hy) {
        cudaError_t e = cudaMalloc(&h->hy, sizeof(double) * 2 * Nmax);
        if (e == cudaSuccess) e = cudaMalloc((void**)&h->hoff, sizeof(int64_t) * (Bmax + 1));
        if (e == cudaSuccess) e = cudaMalloc(&h->hm0, sizeof(double) * 5 * Bmax);
        if (e == cudaSuccess) e = cudaMalloc(&h->hP0, sizeof(double) * 15 * Bmax);
        if (e == cudaSuccess) e = cudaMalloc(&h->hx, sizeof(double) * 5 * Nmax);
        if (e == cudaSuccess) e = cudaMalloc(&h->hP, sizeof(double) * 15 * Nmax);
        if (e == cudaSuccess) e = cudaMalloc((void**)&h->hsens, sizeof(double) * 4 * Bmax);
        if (e != cudaSuccess) {
            // leave none of them set, so that a later call allocates them all again
            void** bufs[] = {&h->hy, (void**)&h->hoff, &h->hm0, &h->hP0, &h->hx, &h->hP, (void**)&h->hsens};
            for (void** b : bufs) {
                if (*b) cudaFree(*b);
                *b = nullptr;
            }
            return cuda_fail(h, e, "allocating the host-path buffers");
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    pes_model dm = *model;
    if (model->kind == PES_MODEL_CT_BEARINGS) {
        if (!model->sensors) return fail(h, PES_ERR_INVALID_ARG, "model.sensors is NULL");
        const size_t ns = model->sensors_per_traj ? (size_t)B : 1;
        PES_CUDA(h, cudaMemcpyAsync(h->hsens, model->sensors, sizeof(double) * 4 * ns, cudaMemcpyHostToDevice, st));
        dm.sensors = h->hsens;
    }
    {
        pes::TraceRange trace_in_("copies in");
        PES_CUDA(h, cudaMemcpyAsync(h->hy, y, ts * 2 * N, cudaMemcpyHostToDevice, st));
        PES_CUDA(h, cudaMemcpyAsync(h->hoff, offsets, sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice, st));
        PES_CUDA(h, cudaMemcpyAsync(h->hm0, m0, ts * 5 * B, cudaMemcpyHostToDevice, st));
        PES_CUDA(h, cudaMemcpyAsync(h->hP0, P0, ts * 15 * B, cudaMemcpyHostToDevice, st));
        if (x_init) PES_CUDA(h, cudaMemcpyAsync(h->hx, x_init, ts * 5 * N, cudaMemcpyHostToDevice, st));
        if (P_init && method != PES_IEKS)
            PES_CUDA(h, cudaMemcpyAsync(h->hP, P_init, ts * 15 * N, cudaMemcpyHostToDevice, st));
    }
    int32_t it = 0;
    pes_status r = pes_ieks_run(h, &dm, method, prec, h->hy, h->hoff, B, N, h->hm0, h->hP0, x_init ? h->hx : nullptr,
                                (P_init && method != PES_IEKS) ? h->hP : nullptr, max_iters, tol, h->hx, h->hP,
                                &it, stream);
    if (iters_used) *iters_used = it;
    if (r != PES_OK && r != PES_ERR_NOT_CONVERGED) return r;
    pes::TraceRange trace_out_("copies out");
    PES_CUDA(h, cudaMemcpyAsync(x_out, h->hx, ts * 5 * N, cudaMemcpyDeviceToHost, st));
    PES_CUDA(h, cudaMemcpyAsync(P_out, h->hP, ts * 15 * N, cudaMemcpyDeviceToHost, st));
    PES_CUDA(h, cudaStreamSynchronize(st));
    return r;
}

}  // extern "C"
