/*
 * pes.h — C ABI of the GB300 (sm_103a) parallel iterated extended (IEKS) and
 * cubature sigma-point (IPLS) Kalman smoother.
 *
 * Method: Yaghoobi, Corenflos, Hassan, Sarkka, "Parallel Iterated Extended and
 * Sigma-Point Kalman Smoothers" (ICASSP 2021). One iteration linearises every
 * step about the previous smoothed trajectory (Eq. 10 for IEKS, Eqs. 7-9 for
 * the cubature IPLS), runs the associative filtering scan over the elements
 * of Eqs. 13-14 with the operator of Eq. 15, then the associative smoothing
 * scan over the elements of Eqs. 17-18 with the operator of Eq. 19 (Sec. 4);
 * the iteration of Sec. 3 repeats this about the new smoothed means.
 *
 * Conventions shared by every entry point
 * -----------------------------------------
 * State dimension n_x = 5 (x = [px, py, vx, vy, omega] for the coordinated-turn
 * model), measurement dimension n_y = 2.
 *
 * Trajectories. B trajectories are concatenated. offsets[B+1] (int64, DEVICE
 * memory) gives the state ranges: trajectory b owns states
 * offsets[b] .. offsets[b+1]-1, offsets[0] = 0, offsets[B] = N, strictly
 * increasing. State offsets[b] is that trajectory's x_0 (prior N(m0_b, P0_b),
 * no measurement); states offsets[b]+1 .. offsets[b+1]-1 are x_1 .. x_{T_b},
 * each with a measurement y_k (Eq. 4). A trajectory may have T_b = 0.
 *
 * Layout. Per-state arrays are structure-of-arrays, component-major:
 * comp c of state k is at ptr[c * N + k]. Symmetric matrices are packed
 * upper-triangular row-major: 5x5 -> 15 components (00,01,02,03,04,11,12,13,
 * 14,22,23,24,33,34,44), 2x2 -> 3 components (00,01,11). General matrices
 * are row-major: F (5x5) -> 25 components, H (2x5) -> 10 components.
 * y is [2][N]; the entries at the x_0 slots are ignored.
 * Per-trajectory priors: m0 [B][5], P0 [B][15] (packed), row-major.
 * Transitions are indexed by their source state: F[:, k], c[:, k], Qp[:, k]
 * describe x_{k+1} = F_k x_k + c_k + q, q ~ N(0, Qp_k) (Eq. 11; entries at the
 * last state of a trajectory are ignored). Observations by their own state:
 * y_k = H_k x_k + d_k + r, r ~ N(0, Rp_k).
 *
 * Precision. PES_FP64: every floating-point array is double. PES_FP32: every
 * floating-point array (except the model's sensors) is float.
 * PES_MIXED (pes_ieks_run only; arrays are float): the first max_iters - 1
 * iterations run in FP32, the final iteration — the one whose means and
 * smoother covariances are returned — in FP64 from the FP32 nominal. Its first
 * call on a handle allocates the FP64 copies (22 doubles per state).
 * PES_REFINED (pes_ieks_run only; arrays are float; IEKS and the symmetric
 * sigma-point rules, no Levenberg-Marquardt damping): the first max_iters - 1
 * iterations run in FP32; the final iteration runs in FP32 and is then
 * refined by one Newton step on its filter and RTS recursions (the Kalman
 * and Rauch-Tung-Striebel steps of the affine model of Eq. 11, i.e. the
 * smoother that Sec. 4's operators compute): residuals of every step in
 * float-float arithmetic (about 48 significant bits on the FP32 pipe), the
 * cubature transition's regression slope (Eq. 9) recomputed in float-float,
 * corrections by FP32 associative scans. The returned moments are those of
 * the exact smoother of the final linearisation to about 1e-6 relative,
 * at about a quarter of the cost of an FP64 iteration on this GPU. Its first
 * call on a handle allocates its workspace (155 floats per state). In
 * tolerance mode the FP32 iterations stop at tol (at most max_iters - 1) and
 * the refined iteration follows; *iters_used counts both.
 * Other entry points return PES_ERR_UNSUPPORTED for PES_MIXED and PES_REFINED.
 *
 * Memory and ownership. Unless stated otherwise every pointer is DEVICE memory
 * owned by the caller and must stay valid until the work on `stream` has
 * completed. The handle owns only its workspace. `stream` is a cudaStream_t
 * passed as void* (NULL = the legacy default stream).
 *
 * Execution and errors. Arguments are validated on the host before anything
 * is launched (PES_ERR_INVALID_ARG, nothing launched). Entry points enqueue
 * their kernels on `stream` and return; faults found on the device (a
 * covariance that is not positive definite, a non-finite result, malformed
 * offsets, an internal wait that ran out of time) are recorded in the
 * handle's device status word and returned by the next pes_sync(), or by an
 * entry point that synchronises (documented per call). pes_last_error()
 * describes the most recent failure. No exception crosses this interface.
 * Calls on one handle must not overlap in time (they share the workspace).
 */
#ifndef PES_H
#define PES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PES_OK = 0,
    PES_ERR_INVALID_ARG = 1,
    PES_ERR_NOT_PD = 2,        /* a covariance / innovation matrix was not positive definite */
    PES_ERR_NONFINITE = 3,     /* a non-finite smoothed mean was produced */
    PES_ERR_NOT_CONVERGED = 4, /* tolerance mode: max_iters reached first */
    PES_ERR_CUDA = 5,          /* a CUDA runtime call failed */
    PES_ERR_UNSUPPORTED = 6,
    PES_ERR_TIMEOUT = 7        /* an internal grid-wide wait exceeded its time limit */
} pes_status;

/* Linearisation of Sec. 3: PES_IEKS, first-order Taylor expansion (Eq. 10);
 * PES_CUBATURE, statistical linear regression (Eqs. 7-9) over the third-degree
 * spherical-radial cubature points xbar +- sqrt(n) chol(Pbar) e_i, weights
 * 1/(2n); PES_UNSCENTED, the same regression over the unscented points of
 * parameters (ut_alpha, ut_beta, ut_kappa) of pes_model: lambda =
 * alpha^2 (n + kappa) - n, points xbar and xbar +- sqrt(n + lambda) chol(Pbar) e_i,
 * mean weights lambda/(n + lambda) (centre) and 1/(2(n + lambda)), the
 * centre's covariance weight lambda/(n + lambda) + 1 - alpha^2 + beta
 * (n + lambda > 0 required); PES_GAUSS_HERMITE, the same regression over the
 * third-order Gauss-Hermite product rule: the 3^5 points
 * xbar + chol(Pbar) xi, xi in {-sqrt 3, 0, sqrt 3}^5, weights the products of
 * 1/6, 2/3, 1/6 (exact for polynomials of degree 5 in each coordinate; about
 * 25x the cubature rule's arithmetic per transition). The paper names
 * sigma-point rules generally (Sec. 3); these are three of them. */
typedef enum { PES_IEKS = 0, PES_CUBATURE = 1, PES_UNSCENTED = 2, PES_GAUSS_HERMITE = 3 } pes_method;
typedef enum { PES_FP64 = 0, PES_FP32 = 1, PES_MIXED = 2, PES_REFINED = 3 } pes_precision;
typedef enum { PES_MODEL_CT_BEARINGS = 0, PES_MODEL_LINEAR = 1 } pes_model_kind;

/*
 * The state-space model of Eq. 4 with additive Gaussian noise.
 *
 * PES_MODEL_CT_BEARINGS (the simulated experiment of Sec. 5): coordinated
 * turn with sampling period dt,
 *   px' = px + sin(w dt)/w vx - (1-cos(w dt))/w vy,  py' = py + (1-cos(w dt))/w vx + sin(w dt)/w vy,
 *   vx' = cos(w dt) vx - sin(w dt) vy,  vy' = sin(w dt) vx + cos(w dt) vy,  w' = w,
 * process noise q_form 0: Q = diag(0, 0, q_c dt, q_c dt, q_w dt); q_form 1:
 * q_c [[dt^3/3, dt^2/2], [dt^2/2, dt]] on each (position, velocity) axis pair
 * and q_w dt on w. Measurements: the bearings atan2(py - s_y, px - s_x) from two
 * sensors, R = r_std^2 I. Bearings are unwrapped to the branch nearest the
 * nominal's predicted bearing. `sensors` is a DEVICE array of doubles
 * [n][4] = (s1x, s1y, s2x, s2y), n = 1 (sensors_per_traj = 0) or B (1).
 *
 * PES_MODEL_LINEAR: x' = F x + c + q, y = H x + d + r with q ~ N(0, Q),
 * r ~ N(0, R); F, c, Q (packed), H, d, R (packed) are given here by value.
 */
typedef struct {
    int32_t kind;
    int32_t q_form;
    double dt;
    double q_c;
    double q_w;
    double r_std;
    const double* sensors;
    int32_t sensors_per_traj;
    double F[25];
    double c[5];
    double Q[15];
    double H[10];
    double d[2];
    double R[3];
    double ut_alpha;   /* PES_UNSCENTED only: spread, prior-knowledge and secondary scaling parameters */
    double ut_beta;
    double ut_kappa;
    /* Levenberg-Marquardt damping of the iteration (Sec. 3 names it as a
     * variant; 0 = none): each iteration adds at every state the
     * pseudo-measurement xbar_k = x_k + e, e ~ N(0, I / lm_lambda), of the
     * previous nominal, which turns the Gauss-Newton step of the IEKS into a
     * Levenberg-Marquardt step (any method; pes_ieks_run and its variants). */
    double lm_lambda;
} pes_model;

/* A handle owns its workspace and nothing else that is shared: handles are
 * independent, so several host threads may each drive their own handle (on
 * their own streams) at the same time. One handle serves one call at a time. */
typedef struct pes_handle pes_handle;

/* Create a handle on the current CUDA device with workspace for up to
 * max_states concatenated states and max_batch trajectories. Allocates device
 * memory once; later calls with N <= max_states and B <= max_batch allocate
 * nothing on the device (except pes_ieks_run_host, see there). */
pes_status pes_create(pes_handle** out, int64_t max_states, int32_t max_batch);

/* Free the handle and its workspace (synchronises the device first). */
pes_status pes_destroy(pes_handle* h);

/* Human-readable description of the handle's most recent failure ("" if none).
 * The string is owned by the handle. */
const char* pes_last_error(const pes_handle* h);

/* Wait for `stream` and report (then clear) the device status of prior calls. */
pes_status pes_sync(pes_handle* h, void* stream);

/*
 * Linearisation of every step about a nominal trajectory (Sec. 3):
 *   PES_IEKS: Taylor expansion, Eq. 10 (Lambda = Omega = 0): F_k = grad f(xbar_k),
 *             c_k = f(xbar_k) - F_k xbar_k, H_k = grad h(xbar_k), d_k = h(xbar_k) - H_k xbar_k;
 *   PES_CUBATURE: statistical linear regression with the 3rd-degree cubature
 *             rule (2 n_x points xbar +- sqrt(n_x) chol(Pbar) e_i), Eqs. 7-9.
 * Outputs Qp = Q + Lambda, Rp = R + Omega (Eq. 11) and y_used, the measurement
 * unwrapped to the branch nearest h(xbar_k) (copied unchanged for the linear
 * model). Inputs: x_nom [5][N], P_nom [15][N] (cubature only; may be NULL for
 * IEKS), y [2][N]. Outputs: F [25][N], c [5][N], Qp [15][N], H [10][N],
 * d [2][N], Rp [3][N], y_used [2][N] (y_used may be NULL). Entries that do not
 * exist (transition of a last state, observation of an x_0) are set to 0.
 */
pes_status pes_linearize(pes_handle* h, const pes_model* model, pes_method method, pes_precision prec,
                         const void* x_nom, const void* P_nom, const void* y,
                         const int64_t* offsets, int32_t B, int64_t N,
                         void* F, void* c, void* Qp, void* H, void* d, void* Rp, void* y_used,
                         void* stream);

/*
 * Filtering by the associative scan of Sec. 4 (elements Eqs. 13-14, operator
 * Eq. 15, prefix products as in Sec. 2) for given linearisation parameters:
 * the filtered means xf [5][N] and covariances Pf [15][N] of every state,
 * x_0 included (its prior).
 */
pes_status pes_filter_scan(pes_handle* h, pes_precision prec,
                           const void* F, const void* c, const void* Qp,
                           const void* H, const void* d, const void* Rp, const void* y,
                           const void* m0, const void* P0, const int64_t* offsets, int32_t B, int64_t N,
                           void* xf, void* Pf, void* stream);

/*
 * pes_filter_scan plus the log-likelihood of each trajectory's measurements
 * under the affine model, loglik[b] = log p(y_1..y_{T_b}) (DEVICE double [B];
 * 0 for a trajectory without measurements). The paper notes (Sec. 2) that the
 * filtering elements can carry this marginal likelihood; here it comes from
 * the same pass, as the sum over steps of log N(y_k; H_k m_k^- + d_k, S_k),
 * with m_k^-, S_k the exact one-step predictions that the scan's re-run
 * produces, terms accumulated in double for either precision.
 */
pes_status pes_filter_loglik(pes_handle* h, pes_precision prec,
                             const void* F, const void* c, const void* Qp,
                             const void* H, const void* d, const void* Rp, const void* y,
                             const void* m0, const void* P0, const int64_t* offsets, int32_t B, int64_t N,
                             void* xf, void* Pf, double* loglik, void* stream);

/*
 * Smoothing by the reverse associative scan of Sec. 4 (elements Eqs. 17-18,
 * operator Eq. 19, suffix products as in Sec. 2) from filtered moments
 * xf [5][N], Pf [15][N] and the transitions F, c, Qp: smoothed means
 * xs [5][N] and covariances Ps [15][N].
 */
pes_status pes_smooth_scan(pes_handle* h, pes_precision prec,
                           const void* F, const void* c, const void* Qp,
                           const void* xf, const void* Pf, const int64_t* offsets, int32_t B, int64_t N,
                           void* xs, void* Ps, void* stream);

/*
 * The iterated smoother (Sec. 3 with the parallel filter and smoother of
 * Sec. 4), all iterations in one persistent launch:
 *   nominal^(0): x_init [5][N] (NULL: every state of trajectory b at m0_b),
 *                P_init [15][N] (cubature only; NULL: P0_b);
 *   iteration i: linearise about nominal^(i-1), filter, smooth; nominal^(i) =
 *                the smoothed moments.
 * max_iters >= 1. tol <= 0: exactly max_iters iterations. tol > 0: stop after
 * the first iteration whose relative update norm
 * ||X^(i) - X^(i-1)||_F / ||X^(i)||_F (per trajectory, worst trajectory) is
 * <= tol; PES_ERR_NOT_CONVERGED if max_iters iterations did not reach it
 * (outputs still hold the last iterate).
 * Outputs: x_out [5][N] smoothed means, P_out [15][N] smoothed covariances of
 * the last iteration. x_out / P_out may equal x_init / P_init.
 * iters_used: HOST int* (may be NULL) receiving the number of iterations run.
 * Synchronises `stream` (and returns device status) when tol > 0 or
 * iters_used != NULL; otherwise it is asynchronous (status via pes_sync).
 */
pes_status pes_ieks_run(pes_handle* h, const pes_model* model, pes_method method, pes_precision prec,
                        const void* y, const int64_t* offsets, int32_t B, int64_t N,
                        const void* m0, const void* P0, const void* x_init, const void* P_init,
                        int32_t max_iters, double tol, void* x_out, void* P_out, int32_t* iters_used,
                        void* stream);

/*
 * pes_ieks_run with HOST buffers: y, offsets, m0, P0, x_init, P_init, the
 * model's sensors, x_out and P_out are HOST memory (pinned memory gives the
 * fastest copies). Copies the inputs to the device, runs, copies the outputs
 * back and synchronises `stream`. Device buffers for these copies are
 * allocated by the first call on the handle (sized for max_states / max_batch)
 * and reused afterwards.
 */
pes_status pes_ieks_run_host(pes_handle* h, const pes_model* model, pes_method method, pes_precision prec,
                             const void* y, const int64_t* offsets, int32_t B, int64_t N,
                             const void* m0, const void* P0, const void* x_init, const void* P_init,
                             int32_t max_iters, double tol, void* x_out, void* P_out, int32_t* iters_used,
                             void* stream);

/*
 * The sequential counterpart of pes_ieks_run on the GPU, with the same
 * arguments, layouts and results: one thread per trajectory runs the extended
 * (PES_IEKS) or cubature (PES_CUBATURE) Kalman filter and RTS smoother of the
 * Sec. 3 iteration over its whole trajectory, the form the paper's parallel
 * method is measured against. It suits many short trajectories; with few
 * trajectories most of the GPU idles. In tolerance mode each trajectory stops
 * at its own first iteration whose relative update is <= tol (recorded for
 * pes_traj_iterations), and *iters_used is the largest count. Uses the
 * handle's workspace; PES_MIXED returns PES_ERR_UNSUPPORTED. x_out / P_out
 * hold the nominal between iterations (they may equal x_init / P_init).
 */
pes_status pes_ieks_run_sequential(pes_handle* h, const pes_model* model, pes_method method, pes_precision prec,
                                   const void* y, const int64_t* offsets, int32_t B, int64_t N,
                                   const void* m0, const void* P0, const void* x_init, const void* P_init,
                                   int32_t max_iters, double tol, void* x_out, void* P_out, int32_t* iters_used,
                                   void* stream);

/*
 * The IEKS with Levenberg-Marquardt steps whose damping adapts per trajectory
 * (Sec. 3 names the Levenberg-Marquardt variant of the iteration). A step is
 * one IEKS iteration about the current nominal with the damping of
 * pes_model.lm_lambda taken per trajectory (the pseudo-measurement
 * xbar_k = x_k + e, e ~ N(0, I / lambda_b), at every state): it is kept if it
 * lowers the trajectory's MAP objective
 *   J = 1/2 |x_0 - m0|^2_{P0^-1} + 1/2 sum_k |x_k - f(x_{k-1})|^2_{Q^-1}
 *       + 1/2 sum_k |y_k - h(x_k)|^2_{R^-1}
 * (bearing residuals on the branch nearest zero; evaluated in FP64), and then
 * lambda_b <- lambda_b / nu; otherwise the trajectory's nominal and
 * covariances stay and lambda_b <- lambda_b * nu. Every trajectory starts at
 * lambda0 (> 0), nu > 1. The objective needs a positive definite Q and R
 * (q_form 1, or a linear model with them): otherwise PES_ERR_UNSUPPORTED.
 * Convergence: a trajectory has converged at the first iteration whose step,
 * kept or not, has a relative size ||x_step - x_nom||_F / ||x_step||_F <= tol;
 * with tol > 0 the iteration stops once all have (PES_ERR_NOT_CONVERGED if
 * max_iters come first; the call then synchronises every iteration), with
 * tol <= 0 it runs max_iters iterations. pes_model.lm_lambda must be 0.
 * Arguments and layouts as pes_ieks_run (PES_FP64 or PES_FP32; x_init may be
 * NULL for the prior start). Outputs: x_out [5][N] the kept nominal, P_out
 * [15][N] the damped smoother's covariances of each trajectory's last kept
 * step (its prior P0 if none was kept); HOST, each may be NULL:
 * *iters_used, lambda_out [B] the final dampings, accepted_out [B] the steps
 * kept, conv_iter_out [B] the converged iteration (0: none). Synchronises
 * `stream` before returning.
 */
pes_status pes_ieks_run_lm(pes_handle* h, const pes_model* model, pes_precision prec, const void* y,
                           const int64_t* offsets, int32_t B, int64_t N, const void* m0, const void* P0,
                           const void* x_init, int32_t max_iters, double tol, double lambda0, double nu,
                           void* x_out, void* P_out, int32_t* iters_used, double* lambda_out,
                           int32_t* accepted_out, int32_t* conv_iter_out, void* stream);

/*
 * Per-trajectory iteration counts of the last pes_ieks_run,
 * pes_ieks_run_host or pes_ieks_run_sequential call on this handle that ran in
 * tolerance mode (tol > 0) with PES_FP32 or PES_FP64: iters[b] (HOST int32 [B]) is the first iteration
 * after which trajectory b's relative update norm (Sec. 3 iteration; the
 * measure of the tolerance) was <= tol, or 0 if it never was within the
 * iterations run. The run continues until every trajectory meets tol or
 * max_iters is reached, so trajectories that met it early keep iterating.
 * B must equal that call's batch size (PES_ERR_INVALID_ARG otherwise).
 * Waits for the work on `stream`.
 */
pes_status pes_traj_iterations(pes_handle* h, int32_t* iters, int32_t B, void* stream);

/*
 * pes_ieks_run without a handle and without allocating device memory. The
 * paper has no counterpart: this is a deployment variant of pes_ieks_run.
 *
 * Some callers cannot create a handle, because pes_create allocates device
 * memory: code whose memory plan is fixed once the process has started (a
 * real-time loop, a service with a pre-reserved budget), code inside a
 * framework that routes every device allocation through its own pool, and
 * latency-critical code that cannot afford an allocation, which may
 * synchronise the device. This entry point calls no cudaMalloc, cudaFree or
 * other allocating routine. Its scratch is one fixed array in the library's
 * device memory, about 11 MB, which every GPU that loads the library holds
 * until the process exits.
 *
 * Arguments, layouts and results are those of pes_ieks_run (DEVICE pointers),
 * for PES_FP64 and PES_FP32; PES_MIXED and PES_REFINED, whose FP64 copies or
 * refinement workspace pes_ieks_run allocates, return PES_ERR_UNSUPPORTED.
 * Per-trajectory iteration counts (pes_traj_iterations) are not kept, and only
 * the status code reports a failure (there is no handle to hold its text).
 * Grid-wide waits honour PES_BARRIER_TIMEOUT_MS as pes_create does. Limits: N <= PES_NOALLOC_MAX_STATES and B <= PES_NOALLOC_MAX_BATCH; larger
 * sizes return PES_ERR_INVALID_ARG before anything is launched.
 * The first call on a device sets the scratch up (it looks up the array's
 * device address and clears its counters), so make that first call before
 * any stream capture. Every call waits for its work on `stream` and returns
 * the device status. All calls on a device share the one scratch array, which
 * keeps the last call's contents; calls that overlap in time on the GPU (for
 * instance from two host threads, or on two streams) race on it and must not
 * be issued.
 */
#define PES_NOALLOC_MAX_STATES 8192
#define PES_NOALLOC_MAX_BATCH 64
pes_status pes_ieks_run_noalloc(const pes_model* model, pes_method method, pes_precision prec,
                                const void* y, const int64_t* offsets, int32_t B, int64_t N,
                                const void* m0, const void* P0, const void* x_init, const void* P_init,
                                int32_t max_iters, double tol, void* x_out, void* P_out, int32_t* iters_used,
                                void* stream);

/*
 * A pes_ieks_run of fixed arguments (fixed iterations: no tolerance, no
 * iteration count read back) captured once into a CUDA graph: offsets
 * validation, sensor conversion, the layout transposes, the nominal
 * initialisation and the persistent launch that runs every iteration. The
 * graph keeps the pointers; replay it with pes_graph_launch after changing the
 * arrays' contents (not their addresses or sizes). Replays use the handle's
 * workspace, so they must not overlap other calls on the handle; device-side
 * faults reach the handle's status word (pes_sync). PES_MIXED synchronises and
 * returns PES_ERR_UNSUPPORTED.
 */
typedef struct pes_graph pes_graph;
pes_status pes_ieks_graph_create(pes_handle* h, const pes_model* model, pes_method method, pes_precision prec,
                                 const void* y, const int64_t* offsets, int32_t B, int64_t N, const void* m0,
                                 const void* P0, const void* x_init, const void* P_init, int32_t iters,
                                 void* x_out, void* P_out, pes_graph** out);
pes_status pes_graph_launch(pes_graph* g, void* stream);
pes_status pes_graph_destroy(pes_graph* g);

/*
 * Autotuner of the launch shape (the paper runs its scans through JAX; here
 * the shape is this library's choice): times pes_ieks_run of the given
 * workload with `iters` iterations for every distinct launch the candidates
 * give (threads per block 128 or 256 for FP32, 128 for FP64; at least
 * 4 .. 128 steps per lane, which sets the number of blocks when N is small)
 * and keeps the fastest for this handle, method and precision: later calls
 * of any size use it (pes_launch_shape reports it). x_scratch [5][N] and
 * P_scratch [15][N] (DEVICE, the precision's type) receive the runs' outputs.
 * Outputs (HOST, may be NULL): the chosen threads per block and minimum
 * steps per lane, and its time per run in ms. Synchronous; on an error the
 * previous choice stays.
 */
pes_status pes_autotune(pes_handle* h, const pes_model* model, pes_method method, pes_precision prec,
                        const void* y, const int64_t* offsets, int32_t B, int64_t N, const void* m0,
                        const void* P0, int32_t iters, void* x_scratch, void* P_scratch, int32_t* threads,
                        int32_t* min_steps, float* ms_per_run, void* stream);

/* Set the launch shape that pes_autotune would keep for (method, precision)
 * without timing anything: a choice recorded by an earlier pes_autotune (for
 * example one cached on disk for this GPU). threads: a compiled block size
 * (128 or 256 for PES_FP32, 128 for PES_FP64), or 0 with min_steps 0 for the
 * defaults; min_steps: at least 1, the minimum steps per lane. prec PES_FP32
 * also sets the shape of PES_MIXED's and PES_REFINED's FP32 iterations.
 * PES_ERR_INVALID_ARG for anything else; the previous choice then stays. */
pes_status pes_set_launch_shape(pes_handle* h, pes_method method, pes_precision prec, int32_t threads,
                                int32_t min_steps);

/* Launch shape the next call of the given kind would use (for tests and the
 * benchmark): blocks, threads per block, steps per thread. */
pes_status pes_launch_shape(pes_handle* h, pes_method method, pes_precision prec, int64_t N,
                            int32_t* blocks, int32_t* threads, int32_t* steps_per_thread);

/* Diagnostic: per-phase durations of the first iteration of the last
 * persistent launch, when the handle was created with the environment variable
 * PES_PHASE_TIMES=1 (else PES_ERR_UNSUPPORTED). mean_ns[i] / max_ns[i] (max_ns
 * may be NULL) receive the mean / maximum over blocks of the time between
 * phase boundaries i and i+1: 0 fold, 1 filter up-sweep, 2 barrier, 3 filter
 * top level, 4 filter down-sweep, 5 filter re-run, 6 between the passes,
 * 7 smoother up-sweep, 8 barrier, 9 smoother top level, 10 smoother
 * down-sweep, 11 RTS re-run, 12 end-of-iteration barrier; -1 where not
 * recorded.
 * Synchronises the device. */
pes_status pes_debug_phase_times(pes_handle* h, double* mean_ns, double* max_ns, int32_t n);

/* Measured arithmetic throughput of this device's CUDA cores (a diagnostic for
 * roofline accounting, not part of the method): a dependent-chain-free FMA
 * loop over all SMs, timed with CUDA events. Outputs in GFLOP/s (2 flops per
 * FMA) for fp32 and fp64; either pointer may be NULL. Synchronises the device. */
pes_status pes_measure_fma_peak(double* fp32_gflops, double* fp64_gflops);

#ifdef __cplusplus
}
#endif

#endif /* PES_H */
