// The persistent smoother kernel: one cooperative launch runs M iterations of
//   (a) linearisation of every step about the nominal (Eq. 10 or Eqs. 7-9),
//   (b) the forward associative scan of filtering elements (Eqs. 13-15),
//   (c) the reverse associative scan of smoothing elements (Eqs. 17-19),
// and re-linearises about the smoothed means between iterations (Sec. 3).
//
// Scan layout. The N states are split into NB x NT contiguous chunks of L
// steps, one per thread ("lane"). Each scan is a three-level reduce-then-scan:
//   1. every lane folds its chunk into one element (sequentially, exact);
//   2. a Blelloch up-sweep over the NT lane elements of a block in shared
//      memory gives the block's element, published to global memory;
//   3. after a grid barrier every block reduces the elements of the blocks
//      before it (filtering) or after it (smoothing) with a tree in shared
//      memory; since the sequence starts with a prior element and ends with
//      a last-state element, that reduction is a Gaussian;
//   4. a Blelloch down-sweep pushes that Gaussian through the lane tree, so
//      every lane gets the Gaussian of the state just before (filtering) or
//      after (smoothing) its chunk, and
//   5. each lane re-runs its chunk sequentially from it, which yields the
//      filtered (smoothed) moments of every state in the chunk.
// The filtering re-run also builds the smoothing elements of its chunk and
// folds them, so the smoothing pass starts at level 2.
//
// Grid barriers spin on a global counter with a wall-clock limit; on timeout
// they set ST_TIMEOUT and return, so the kernel always terminates.
#pragma once

#include "pes_async.cuh"
#include "pes_ops.cuh"

namespace pes {

enum { MODE_FILTER = 0, MODE_SMOOTH = 1, MODE_RUN = 2 };

constexpr int FE = sizeof(FElem<double>) / sizeof(double);   // 70
constexpr int SE = sizeof(SElem<double>) / sizeof(double);   // 50
constexpr int GE = sizeof(Gauss<double>) / sizeof(double);   // 20
constexpr int HAND = 50;                                      // handoff scalars per state: one SElem
constexpr int LINS = 65;                                      // stored linearisation scalars per state

template <typename T>
struct KParams {
    int64_t N;
    const int64_t* offsets;   // [B+1], device
    int B;
    int mode;
    int iters;                // RUN: maximum iterations; otherwise 1
    double tol;               // RUN: relative update-norm tolerance (<= 0: fixed iterations)
    int write_P_every_iter;   // RUN: write smoothed covariances in every iteration
    DevModel<T> model;
    const T* y;               // [2][N] (slot of each x_0 ignored)
    const T* m0;              // [B][5]
    const T* P0;              // [B][15]
    // linearisation arrays (MODE_FILTER / MODE_SMOOTH), SoA [ncomp][N]
    const T* F;
    const T* c;
    const T* Qp;
    const T* H;
    const T* d;
    const T* Rp;
    // filtered moments (MODE_FILTER output, MODE_SMOOTH input), SoA
    T* xf;
    T* Pf;
    // smoothed moments: MODE_SMOOTH output; MODE_RUN nominal (in place) and output
    T* x;
    T* P;
    // MODE_RUN: the filtered moments of every state, [20][cs] in the layout of
    // x and P (means then packed covariances), or NULL (not stored)
    T* fstore;
    // workspace
    T* hand;           // MODE_RUN handoff of smoothing elements: [warp][s][c][32 lanes]
    T* lin;            // MODE_RUN cubature linearisation handed from the fold to the re-run: [warp][s][LINS][32]
    T* aggF;           // [NB][FE]
    T* aggS;           // [NB][SE]
    unsigned* bar;     // grid barrier counter, zero at launch
    int* status;       // ST_* bits
    double* conv;      // [2][B][2] update-norm accumulators, zero at launch
    int* iters_done;
    int* traj_iters;   // RUN with tol > 0: [B], the first iteration whose update met tol (0: none); or NULL
    double* loglik;    // FILTER: [B] log p(y_{1:T_b}) accumulated (zero at launch), or NULL
    int L;             // steps per lane
    int NL;            // lanes = NB * NT
    int lanes_layout;  // x, P, y use the kernel's lane-major layout (MODE_RUN)
    int64_t cs;        // component stride of x, P, y
    long long timeout_ns;
    long long* ptime;  // optional per-block phase timestamps of the first iteration (NULL: off)
};

constexpr int NPHASE = 16;
// Phase timestamps: thread 0 of every block records %globaltimer at the phase
// boundaries of the first iteration when p.ptime is set.
#define PES_PHASE(p, it, i)                                                        \
    do {                                                                           \
        if ((p).ptime && (it) == 0 && threadIdx.x == 0)                            \
            (p).ptime[(size_t)blockIdx.x * NPHASE + (i)] = globaltimer_ns();      \
    } while (0)

// ---- small device utilities ------------------------------------------------

PES_DEV long long globaltimer_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

PES_DEV unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).
template <typename T>
PES_DEV void grid_barrier(const KParams<T>& p, unsigned& gen)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        ++gen;
        const unsigned target = gen * gridDim.x;
        __threadfence();
        atomicAdd(p.bar, 1u);
        const long long t0 = globaltimer_ns();
        unsigned polls = 0;
        while (ld_acquire(p.bar) < target) {
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

// Trajectory cursor over the CSR offsets.
struct SegCursor {
    const int64_t* off;
    int b;
    int64_t head, next;
    PES_DEV void init(const int64_t* o, int B, int64_t k)
    {
        off = o;
        int lo = 0, hi = B - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(o + mid) <= k) lo = mid;
            else hi = mid - 1;
        }
        b = lo;
        head = __ldg(o + b);
        next = __ldg(o + b + 1);
    }
    PES_DEV void forward(int64_t k)
    {
        while (k >= next) {
            ++b;
            head = next;
            next = __ldg(off + b + 1);
        }
    }
    PES_DEV void backward(int64_t k)
    {
        while (k < head) {
            --b;
            next = head;
            head = __ldg(off + b);
        }
    }
    PES_DEV bool is_head(int64_t k) const { return k == head; }
    PES_DEV bool is_tail(int64_t k) const { return k == next - 1; }
};

template <typename T>
PES_DEV void load_prior(const KParams<T>& p, int b, T* m0, T* P0)
{
#pragma unroll
    for (int i = 0; i < 5; ++i) m0[i] = __ldg(p.m0 + 5 * b + i);
#pragma unroll
    for (int i = 0; i < 15; ++i) P0[i] = __ldg(p.P0 + 15 * b + i);
}

// The nominal trajectory is rewritten by every iteration. Reads of it (and of
// other data written earlier in the same launch) are plain L1-cached loads:
// every such read follows a grid barrier, whose gpu-scope acquire and fence
// make the other blocks' writes visible, and consecutive steps of a lane share
// cache sectors.
template <typename T>
PES_DEV void load_nominal(const KParams<T>& p, int64_t ix, T* x)
{
#pragma unroll
    for (int i = 0; i < 5; ++i) x[i] = p.x[i * p.cs + ix];
}

template <typename T>
PES_DEV void load_nominal_cov(const KParams<T>& p, int64_t ix, T* P)
{
#pragma unroll
    for (int i = 0; i < 15; ++i) P[i] = p.P[i * p.cs + ix];
}

template <typename T>
PES_DEV void load_y(const KParams<T>& p, int64_t ix, T* y)
{
    y[0] = __ldg(p.y + ix);
    y[1] = __ldg(p.y + p.cs + ix);
}

// Index of state k of the chunk [a, e) of `lane` in the per-state arrays the
// kernel reads and writes (x, P, y): in MODE_RUN the kernel's lane-major
// layout [component][step][lane], in which a warp's accesses at one step are
// contiguous; otherwise the caller's [component][N] layout.
template <typename T>
PES_DEV int64_t state_ix(const KParams<T>& p, int64_t k, int64_t a, int lane)
{
    return p.lanes_layout ? (k - a) * p.NL + lane : k;
}

// Index of the state just before the chunk (k = a - 1): the last state of the
// previous lane's chunk, which is full.
template <typename T>
PES_DEV int64_t prev_ix(const KParams<T>& p, int64_t a, int lane)
{
    return p.lanes_layout ? (int64_t)(p.L - 1) * p.NL + (lane - 1) : a - 1;
}

// ---- linearisation of one step ------------------------------------------------

// Per-state inputs of the linearisation, loaded one step ahead of their use
// so that the loads overlap the previous step's arithmetic.
template <typename T, int LIN>
struct StateIn {
    T x[5];    // nominal mean (IEKS, cubature)
    T P[15];   // nominal covariance (cubature)
    T y[2];    // measurement
};

template <typename T, int LIN>
PES_DEV void load_state(const KParams<T>& p, int64_t ix, StateIn<T, LIN>& s)
{
    if (LIN != LIN_ARRAYS) load_nominal(p, ix, s.x);
    if (kSigma<LIN>) load_nominal_cov(p, ix, s.P);
    load_y(p, ix, s.y);
}

// Sigma-point factor of the state's nominal covariance (cubature only).
template <typename T, int LIN>
struct Factor {
    T L[kSigma<LIN> ? 25 : 1];
    T rd[kSigma<LIN> ? 5 : 1];
};

template <typename T, int LIN>
PES_DEV bool factor_state(const StateIn<T, LIN>& s, Factor<T, LIN>& f)
{
    if (kSigma<LIN>) return cub_factor(s.P, f.L, f.rd);
    return true;
}

// Transition k -> k+1 (Eq. 10 or Eq. 7).
template <typename T, int LIN>
PES_DEV void lin_trans(const KParams<T>& p, int64_t k, const StateIn<T, LIN>& s, const Factor<T, LIN>& f,
                       Trans<T>& tr)
{
    if (LIN == LIN_ARRAYS) {
#pragma unroll
        for (int i = 0; i < 25; ++i) tr.F[i] = __ldg(p.F + i * p.N + k);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            tr.fx[i] = __ldg(p.c + i * p.N + k);
            tr.xn[i] = T(0);
        }
#pragma unroll
        for (int i = 0; i < 15; ++i) tr.Q[i] = __ldg(p.Qp + i * p.N + k);
    } else if (LIN == LIN_IEKS) {
        lin_trans_taylor(p.model, s.x, tr);
    } else if (LIN == LIN_GH) {
        lin_trans_gh(p.model, s.x, f.L, f.rd, tr);
    } else {
        lin_trans_cubature(p.model, s.x, f.L, f.rd, tr);
    }
}

// Observation at k (Eq. 10 or Eq. 9).
template <typename T, int LIN>
PES_DEV void lin_obs(const KParams<T>& p, int64_t k, int b, const StateIn<T, LIN>& s, const Factor<T, LIN>& f,
                     Obs<T>& ob)
{
    if (LIN == LIN_ARRAYS) {
#pragma unroll
        for (int i = 0; i < 10; ++i) ob.H[i] = __ldg(p.H + i * p.N + k);
        ob.r[0] = s.y[0] - __ldg(p.d + k);
        ob.r[1] = s.y[1] - __ldg(p.d + p.N + k);
#pragma unroll
        for (int i = 0; i < 5; ++i) ob.xn[i] = T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) ob.R[i] = __ldg(p.Rp + i * p.N + k);
    } else if (LIN == LIN_IEKS) {
        lin_obs_taylor(p.model, b, s.x, s.y, ob);
    } else if (LIN == LIN_GH) {
        lin_obs_gh(p.model, b, s.x, f.L, f.rd, s.y, ob);
    } else {
        lin_obs_cubature(p.model, b, s.x, f.L, f.rd, s.y, ob);
    }
}

// One-shot forms used by the stand-alone linearisation kernel.
template <typename T, int LIN>
PES_DEV bool get_trans(const KParams<T>& p, int64_t k, int64_t ix, Trans<T>& tr)
{
    StateIn<T, LIN> s;
    load_state(p, ix, s);
    Factor<T, LIN> f;
    const bool ok = factor_state(s, f);
    lin_trans(p, k, s, f, tr);
    return ok;
}

template <typename T, int LIN>
PES_DEV bool get_obs(const KParams<T>& p, int64_t k, int64_t ix, int b, Obs<T>& ob)
{
    StateIn<T, LIN> s;
    load_state(p, ix, s);
    Factor<T, LIN> f;
    const bool ok = factor_state(s, f);
    lin_obs(p, k, b, s, f, ob);
    return ok;
}

// ---- lane-level passes -------------------------------------------------------------

// Whether the fold hands its linearisation of every state to the filtering
// re-run (65 scalars per state) instead of the re-run linearising again. The
// cubature linearisation (2 n_x sigma points through f and h) costs far more
// than the traffic; the Taylor one does not.
template <int LIN>
constexpr bool kStoreLin = kSigma<LIN>;

// Layout [warp][s][LINS][32 lanes]; per state: H (10), r (2), R' (3), xn (5),
// F (25), fx (5), Q' (15).
template <typename T>
PES_DEV T* lin_slot(const KParams<T>& p, int s, int lane)
{
    return p.lin + ((size_t)(lane >> 5) * p.L + s) * (LINS * 32) + (lane & 31);
}

template <typename T>
PES_DEV void store_lin_obs(const KParams<T>& p, int s, int lane, const Obs<T>& ob)
{
    T* h = lin_slot(p, s, lane);
#pragma unroll
    for (int i = 0; i < 5; ++i) h[(15 + i) * 32] = ob.xn[i];
#pragma unroll
    for (int i = 0; i < 10; ++i) h[i * 32] = ob.H[i];
    h[10 * 32] = ob.r[0];
    h[11 * 32] = ob.r[1];
#pragma unroll
    for (int i = 0; i < 3; ++i) h[(12 + i) * 32] = ob.R[i];
}

template <typename T>
PES_DEV void store_lin_trans(const KParams<T>& p, int s, int lane, const Trans<T>& tr)
{
    T* h = lin_slot(p, s, lane);
#pragma unroll
    for (int i = 0; i < 5; ++i) h[(15 + i) * 32] = tr.xn[i];
#pragma unroll
    for (int i = 0; i < 25; ++i) h[(20 + i) * 32] = tr.F[i];
#pragma unroll
    for (int i = 0; i < 5; ++i) h[(45 + i) * 32] = tr.fx[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) h[(50 + i) * 32] = tr.Q[i];
}

template <typename T>
PES_DEV void load_lin_obs(const KParams<T>& p, int s, int lane, Obs<T>& ob)
{
    const T* h = lin_slot(p, s, lane);
#pragma unroll
    for (int i = 0; i < 10; ++i) ob.H[i] = h[i * 32];
    ob.r[0] = h[10 * 32];
    ob.r[1] = h[11 * 32];
#pragma unroll
    for (int i = 0; i < 3; ++i) ob.R[i] = h[(12 + i) * 32];
#pragma unroll
    for (int i = 0; i < 5; ++i) ob.xn[i] = h[(15 + i) * 32];
}

template <typename T>
PES_DEV void load_lin_trans(const KParams<T>& p, int s, int lane, Trans<T>& tr)
{
    const T* h = lin_slot(p, s, lane);
#pragma unroll
    for (int i = 0; i < 5; ++i) tr.xn[i] = h[(15 + i) * 32];
#pragma unroll
    for (int i = 0; i < 25; ++i) tr.F[i] = h[(20 + i) * 32];
#pragma unroll
    for (int i = 0; i < 5; ++i) tr.fx[i] = h[(45 + i) * 32];
#pragma unroll
    for (int i = 0; i < 15; ++i) tr.Q[i] = h[(50 + i) * 32];
}

// Per-thread asynchronous prefetch of the next state's inputs (nominal mean
// and covariance, measurement: 22 scalars) into shared memory, for the
// sigma-point folds, whose register pressure rules out a register prefetch.
// Each thread copies its own scalars with cp.async (L1-allocating, like the
// plain loads it replaces; every read of the nominal follows a grid barrier's
// acquire) into one of two stages and reads only its own stage back after
// cp.async.wait_group, so no block synchronisation is involved. Element c of
// stage s sits at base[(s * NS + c) * stride] (thread-contiguous columns).
template <typename T>
struct StatePrefetch {
    static constexpr int NS = 22;
    T* base;
    int stride;
    PES_DEV void copy(T* dst, const T* src) const
    {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(sizeof(T))
                     : "memory");
    }
    PES_DEV void issue(const KParams<T>& p, int64_t ix, int s) const
    {
        T* d = base + (size_t)s * NS * stride;
#pragma unroll
        for (int i = 0; i < 5; ++i) copy(d + i * stride, p.x + i * p.cs + ix);
#pragma unroll
        for (int i = 0; i < 15; ++i) copy(d + (5 + i) * stride, p.P + i * p.cs + ix);
        copy(d + 20 * stride, p.y + ix);
        copy(d + 21 * stride, p.y + p.cs + ix);
    }
    PES_DEV static void commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
    // all but the most recent group complete
    PES_DEV static void wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
    template <int LIN>
    PES_DEV void take(int s, StateIn<T, LIN>& st) const
    {
        const T* d = base + (size_t)s * NS * stride;
#pragma unroll
        for (int i = 0; i < 5; ++i) st.x[i] = d[i * stride];
#pragma unroll
        for (int i = 0; i < 15; ++i) st.P[i] = d[(5 + i) * stride];
        st.y[0] = d[20 * stride];
        st.y[1] = d[21 * stride];
    }
};

// Filtering, level 1: fold the lane's chunk [a, e) into one element. Step k
// folds the update with its own observation and then the prediction through
// its outgoing transition (k -> k+1), both linearised about the nominal of k,
// so the state's sigma-point factor serves both and no earlier state's inputs
// stay live. The transition into the chunk's first state is linearised once
// before the loop; the outgoing transition of the chunk's last state is
// linearised only to be stored for the re-run (the next lane folds it itself).
// With a stored linearisation (MODE_RUN, cubature) both are kept for the
// re-run, the transition at the slot of its source state.
template <typename T, int LIN>
PES_DEV bool fold_filter_chunk(const KParams<T>& p, int64_t a, int64_t e, int lane, FElem<T>& acc,
                               const StatePrefetch<T>* pf = nullptr)
{
    bool ok = true;
    T zero[5] = {T(0), T(0), T(0), T(0), T(0)};
    felem_identity(acc, zero);
    if (a >= e) return ok;
    const bool store_lin = kStoreLin<LIN> && p.mode == MODE_RUN;
    SegCursor cur;
    cur.init(p.offsets, p.B, a);
    const int64_t dix = p.lanes_layout ? p.NL : 1;
    int64_t ix = state_ix(p, a, a, lane);
    StateIn<T, LIN> sc, sn;   // inputs of states k, k+1
    if (!cur.is_head(a)) {
        StateIn<T, LIN> sp;
        load_state(p, prev_ix(p, a, lane), sp);
        Trans<T> tr;
        Factor<T, LIN> fp;
        ok &= factor_state(sp, fp);
        lin_trans(p, a - 1, sp, fp, tr);
        felem_identity(acc, tr.xn);
        fold_predict(acc, tr);
    }
    // the next state's inputs are loaded a step ahead: into registers for
    // the Taylor linearisation; for the sigma-point ones, whose register
    // pressure makes a register prefetch cost more in spills than it hides
    // (measured: fold 202 -> 194 us per iteration at T = 2^20 without it),
    // into shared memory by cp.async when the caller provides the stages
    constexpr bool prefetch = !kSigma<LIN>;
    const bool async_pf = kSigma<LIN> && pf != nullptr;
    if (prefetch) load_state(p, ix, sc);
    if (async_pf) {
        pf->issue(p, ix, 0);
        StatePrefetch<T>::commit();
    }
#pragma unroll 1
    for (int64_t k = a; k < e; ++k, ix += dix) {
        cur.forward(k);
        const int s = (int)(k - a);
        if (prefetch) {
            if (k + 1 < e) load_state(p, ix + dix, sn);
        } else if (async_pf) {
            if (k + 1 < e) pf->issue(p, ix + dix, (s + 1) & 1);
            StatePrefetch<T>::commit();
            StatePrefetch<T>::wait_prev();
            pf->take(s & 1, sc);
        } else {
            load_state(p, ix, sc);
        }
        Factor<T, LIN> fc;
        ok &= factor_state(sc, fc);
        if (cur.is_head(k)) {
            T m0[5], P0[15];
            load_prior(p, cur.b, m0, P0);
            felem_apply_prior(acc, m0, P0);
        } else {
            Obs<T> ob;
            lin_obs(p, k, cur.b, sc, fc, ob);
            if (store_lin) store_lin_obs(p, s, lane, ob);
            ok &= fold_update(acc, ob);
        }
        if (LIN != LIN_ARRAYS && lm_of(p.model, cur.b) > T(0)) {
            // Levenberg-Marquardt pseudo-measurement of this state's nominal
            FElem<T> dmp;
            felem_damping(dmp, sc.x, lm_of(p.model, cur.b));
            combine_filter(acc, dmp, acc);
        }
        if (!cur.is_tail(k) && (k + 1 < e || store_lin)) {
            Trans<T> tr;
            lin_trans(p, k, sc, fc, tr);
            if (store_lin) store_lin_trans(p, s, lane, tr);
            if (k + 1 < e) fold_predict(acc, tr);
        }
        if (prefetch) sc = sn;
    }
    return ok;
}

// Filtered moments in the caller's arrays (MODE_FILTER output, MODE_SMOOTH input).
template <typename T>
PES_DEV void store_filtered(const KParams<T>& p, int64_t k, const T* m, const T* P)
{
#pragma unroll
    for (int i = 0; i < 5; ++i) p.xf[i * p.N + k] = m[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) p.Pf[i * p.N + k] = P[i];
}

template <typename T>
PES_DEV void load_filtered(const KParams<T>& p, int64_t k, T* m, T* P)
{
#pragma unroll
    for (int i = 0; i < 5; ++i) m[i] = __ldg(p.xf + i * p.N + k);
#pragma unroll
    for (int i = 0; i < 15; ++i) P[i] = __ldg(p.Pf + i * p.N + k);
}

// MODE_RUN: the smoothing element of state a + s of a lane, kept between the
// filtering re-run that builds it and the RTS pass that applies it. Layout
// [warp][s][component][32 lanes]: a warp's accesses for one step are one
// contiguous, coalesced run, and its consecutive steps are adjacent.
template <typename T>
PES_DEV T* selem_slot(const KParams<T>& p, int s, int lane)
{
    return p.hand + ((size_t)(lane >> 5) * p.L + s) * (HAND * 32) + (lane & 31);
}

template <typename T>
PES_DEV void store_selem(const KParams<T>& p, int s, int lane, const SElem<T>& el)
{
    T* h = selem_slot(p, s, lane);
    const T* src = reinterpret_cast<const T*>(&el);
#pragma unroll
    for (int i = 0; i < HAND; ++i) h[i * 32] = src[i];
}

template <typename T>
PES_DEV void load_selem(const KParams<T>& p, int s, int lane, SElem<T>& el)
{
    const T* h = selem_slot(p, s, lane);
    T* dst = reinterpret_cast<T*>(&el);
#pragma unroll
    for (int i = 0; i < HAND; ++i) dst[i] = h[i * 32];
}

// MODE_RUN handoff alternative: the filtered moments (x*, P*) of state a + s,
// from which the RTS pass rebuilds the smoothing element (same slot layout).
template <typename T>
PES_DEV void store_xP(const KParams<T>& p, int s, int lane, const T* m, const T* P)
{
    T* h = selem_slot(p, s, lane);
#pragma unroll
    for (int i = 0; i < 5; ++i) h[i * 32] = m[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) h[(5 + i) * 32] = P[i];
}

template <typename T>
PES_DEV void load_xP(const KParams<T>& p, int s, int lane, T* m, T* P)
{
    const T* h = selem_slot(p, s, lane);
#pragma unroll
    for (int i = 0; i < 5; ++i) m[i] = h[i * 32];
#pragma unroll
    for (int i = 0; i < 15; ++i) P[i] = h[(5 + i) * 32];
}

// Whether the filtering re-run hands the RTS pass finished smoothing elements
// (50 scalars per state) or the filtered moments (20 scalars per state) from
// which the RTS pass would rebuild them. The re-run builds every element
// anyway (it folds them for the smoother's tree), so handing them over saves
// the RTS pass a transition linearisation, a prediction and a Cholesky per
// step for 120 more bytes of traffic per state (measured: IEKS 326 -> 304 us
// per iteration at T = 2^20).
template <int LIN>
constexpr bool kStoreElements = (LIN != LIN_ARRAYS);

// Stored linearisation of step stage `i` of a lane-stream (layout of store_lin_*).
template <typename T, class S>
PES_DEV void obs_from_stage(const S& ws, int i, Obs<T>& ob)
{
#pragma unroll
    for (int c = 0; c < 10; ++c) ob.H[c] = ws.get(i, c);
    ob.r[0] = ws.get(i, 10);
    ob.r[1] = ws.get(i, 11);
#pragma unroll
    for (int c = 0; c < 3; ++c) ob.R[c] = ws.get(i, 12 + c);
#pragma unroll
    for (int c = 0; c < 5; ++c) ob.xn[c] = ws.get(i, 15 + c);
}

template <typename T, class S>
PES_DEV void trans_from_stage(const S& ws, int i, Trans<T>& tr)
{
#pragma unroll
    for (int c = 0; c < 5; ++c) tr.xn[c] = ws.get(i, 15 + c);
#pragma unroll
    for (int c = 0; c < 25; ++c) tr.F[c] = ws.get(i, 20 + c);
#pragma unroll
    for (int c = 0; c < 5; ++c) tr.fx[c] = ws.get(i, 45 + c);
#pragma unroll
    for (int c = 0; c < 15; ++c) tr.Q[c] = ws.get(i, 50 + c);
}

// Filtering, level 5: re-run the chunk from the Gaussian of the state before it,
// storing filtered moments; in MODE_RUN also build and fold the chunk's
// smoothing elements (Eqs. 17-18) into accS. The loop runs over the L steps
// of the chunk in every lane of the warp (lanes whose chunk is shorter idle),
// so that a warp stream can feed it the stored linearisation: step s reads
// the transition into state s from the previous step's stage, then releases
// that stage for the copy of step s + 1, then reads its observation.
template <typename T, int LIN>
PES_DEV bool rerun_filter_chunk(const KParams<T>& p, int64_t a, int64_t e, int lane, const Gauss<T>& G,
                                SElem<T>& accS, T* wstage, uint64_t* wbar, uint32_t& wpar)
{
    bool ok = true;
    selem_identity(accS);
    const bool smooth = (p.mode == MODE_RUN);
    double ll = 0.0;   // log-likelihood terms of trajectory llb (filter scan with given arrays only)
    int llb = -1;
    const bool any = a < e;
    constexpr bool stored_lin = kStoreLin<LIN>;
    const bool use_lin = stored_lin && smooth;
    SegCursor cur;
    if (any) cur.init(p.offsets, p.B, a);
    T m[5], P[15];
#pragma unroll
    for (int i = 0; i < 5; ++i) m[i] = G.m[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) P[i] = G.P[i];
    const int64_t dix = p.lanes_layout ? p.NL : 1;
    int64_t ix = state_ix(p, a, a, lane);
    StateIn<T, LIN> sp, sc, sn;   // inputs of states k-1, k, k+1 (when linearising here)
    if (!use_lin && any) {
        if (!cur.is_head(a)) load_state(p, prev_ix(p, a, lane), sp);
        load_state(p, ix, sc);
    }
    WarpStream<T, LINS, LINS> ws;
    if (use_lin) {
        ws.init(p.lin + (size_t)(lane >> 5) * p.L * (LINS * 32), wstage, wbar, wpar);
        ws.issue(0, 0);
    }
#pragma unroll 1
    for (int s = 0; s < p.L; ++s, ix += dix) {
        const int64_t k = a + s;
        const bool act = k < e;
        if (use_lin) ws.wait(s & 1, p.status);
        T mp[5], Pp[15];
        bool head = false;
        if (act) {
            cur.forward(k);
            if (!use_lin && k + 1 < e) load_state(p, ix + dix, sn);
            head = cur.is_head(k);
            if (head) {
                if (smooth && k > a) {
                    SElem<T> el;
                    selem_last(el, m, P);
                    combine_smoother(accS, el, accS);
                    if (kStoreElements<LIN>) store_selem(p, s - 1, lane, el);
                }
            } else {
                Trans<T> tr;
                if (use_lin) {
                    if (s == 0) load_lin_trans(p, p.L - 1, lane - 1, tr);
                    else trans_from_stage<T>(ws, (s - 1) & 1, tr);
                } else {
                    Factor<T, LIN> fp;
                    ok &= factor_state(sp, fp);
                    lin_trans(p, k - 1, sp, fp, tr);
                }
                T FP[25];
                predict(tr, m, P, mp, FP, Pp);
                if (smooth && k > a) {
                    SElem<T> el;
                    ok &= selem_from_prediction(m, P, FP, Pp, mp, el);
                    combine_smoother(accS, el, accS);
                    if (kStoreElements<LIN>) store_selem(p, s - 1, lane, el);
                }
            }
        }
        if (use_lin) {
            // every lane is done with the previous step's stage: refill it
            __syncwarp();
            if (s + 1 < p.L) ws.issue(s + 1, (s + 1) & 1);
        }
        if (act) {
            if (head) {
                load_prior(p, cur.b, m, P);
            } else {
                Obs<T> ob;
                if (use_lin) {
                    obs_from_stage<T>(ws, s & 1, ob);
                } else {
                    Factor<T, LIN> fc;
                    ok &= factor_state(sc, fc);
                    lin_obs(p, k, cur.b, sc, fc, ob);
                }
                if constexpr (LIN == LIN_ARRAYS) {
                    if (p.loglik) {
                        double term;
                        ok &= kf_update(ob, mp, Pp, m, P, &term);
                        if (cur.b != llb) {
                            if (llb >= 0) atomicAdd(p.loglik + llb, ll);
                            ll = 0.0;
                            llb = cur.b;
                        }
                        ll += term;
                    } else {
                        ok &= kf_update(ob, mp, Pp, m, P);
                    }
                } else {
                    ok &= kf_update(ob, mp, Pp, m, P);
                }
            }
            if (LIN != LIN_ARRAYS && lm_of(p.model, cur.b) > T(0)) {
                // Levenberg-Marquardt pseudo-measurement of this state's nominal
                T xb[5];
                load_nominal(p, ix, xb);
                FElem<T> dmp;
                felem_damping(dmp, xb, lm_of(p.model, cur.b));
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
            if (!smooth) store_filtered(p, k, m, P);
            else if (!kStoreElements<LIN>) store_xP(p, s, lane, m, P);
            if (p.fstore) {
#pragma unroll
                for (int i = 0; i < 5; ++i) p.fstore[i * p.cs + ix] = m[i];
#pragma unroll
                for (int i = 0; i < 15; ++i) p.fstore[(5 + i) * p.cs + ix] = P[i];
            }
            if (!use_lin) {
                sp = sc;
                sc = sn;
            }
        }
    }
    if (use_lin) wpar = ws.parity;
    if (llb >= 0) atomicAdd(p.loglik + llb, ll);
    if (smooth && any) {
        // smoothing element of the chunk's last state: the transition out of the
        // chunk is linearised about the last state's nominal
        SElem<T> el;
        if (cur.is_tail(e - 1)) {
            selem_last(el, m, P);
        } else {
            Trans<T> tr;
            if (use_lin) {
                trans_from_stage<T>(ws, (p.L - 1) & 1, tr);
            } else {
                Factor<T, LIN> fp;
                ok &= factor_state(sp, fp);
                lin_trans(p, e - 1, sp, fp, tr);
            }
            T mp[5], FP[25], Pp[15];
            predict(tr, m, P, mp, FP, Pp);
            ok &= selem_from_prediction(m, P, FP, Pp, mp, el);
        }
        combine_smoother(accS, el, accS);
        if (kStoreElements<LIN>) store_selem(p, (int)(e - 1 - a), lane, el);
    }
    return ok;
}

// Smoothing, level 1 in MODE_SMOOTH: fold the chunk's smoothing elements from
// the given filtered moments and transitions.
template <typename T, int LIN>
PES_DEV bool fold_smoother_chunk(const KParams<T>& p, int64_t a, int64_t e, int lane, SElem<T>& accS)
{
    bool ok = true;
    selem_identity(accS);
    if (a >= e) return ok;
    SegCursor cur;
    cur.init(p.offsets, p.B, a);
#pragma unroll 1
    for (int64_t k = a; k < e; ++k) {
        cur.forward(k);
        T m[5], P[15];
        load_filtered(p, k, m, P);
        SElem<T> el;
        if (cur.is_tail(k)) {
            selem_last(el, m, P);
        } else {
            Trans<T> tr;
            ok &= get_trans<T, LIN>(p, k, k, tr);
            T mp[5], FP[25], Pp[15];
            predict(tr, m, P, mp, FP, Pp);
            ok &= selem_from_prediction(m, P, FP, Pp, mp, el);
        }
        combine_smoother(accS, el, accS);
    }
    return ok;
}

// Smoothing, level 5: Rauch-Tung-Striebel re-run backwards from the Gaussian of
// the state after the chunk: x_k ~ E_k (x_{k+1} - xr_k) + g_k with covariance
// E P E^T + L (a last state has E = 0). In MODE_RUN the stored elements (or
// the stored filtered moments, from which the elements are rebuilt) arrive
// through a warp stream and the smoothed moments replace the nominal in
// place; in MODE_SMOOTH the elements are rebuilt from the given arrays.
template <typename T, int LIN>
PES_DEV bool rts_chunk(const KParams<T>& p, int64_t a, int64_t e, int lane, const Gauss<T>& G, bool write_P,
                       bool want_norm, double* conv, int& nb, double& num, double& den, T* wstage, uint64_t* wbar,
                       uint32_t& wpar)
{
    bool ok = true;
    const bool any = a < e;
    SegCursor cur;
    if (any) cur.init(p.offsets, p.B, e - 1);
    Gauss<T> s = G;
    const bool run = (p.mode == MODE_RUN);
    const bool stored = run && kStoreElements<LIN>;
    const T* wbase = p.hand + (size_t)(lane >> 5) * p.L * (HAND * 32);
    WarpStream<T, HAND, HAND> we;   // stored smoothing elements
    WarpStream<T, 20, HAND> wx;     // stored filtered moments
    if (run) {
        if (stored) {
            we.init(wbase, wstage, wbar, wpar);
            we.issue(p.L - 1, 0);
        } else {
            wx.init(wbase, wstage, wbar, wpar);
            wx.issue(p.L - 1, 0);
        }
    }
#pragma unroll 1
    for (int it = 0; it < p.L; ++it) {
        const int sidx = p.L - 1 - it;
        const int64_t k = a + sidx;
        const int st = it & 1;
        if (run) {
            if (stored) {
                if (it + 1 < p.L) we.issue(sidx - 1, st ^ 1);
                we.wait(st, p.status);
            } else {
                if (it + 1 < p.L) wx.issue(sidx - 1, st ^ 1);
                wx.wait(st, p.status);
            }
        }
        if (k < e) {
            cur.backward(k);
            SElem<T> ec;
            if (stored) {
                T* dst = reinterpret_cast<T*>(&ec);
#pragma unroll
                for (int c = 0; c < HAND; ++c) dst[c] = we.get(st, c);
            } else {
                T m[5], P[15];
                if (run) {
#pragma unroll
                    for (int c = 0; c < 5; ++c) m[c] = wx.get(st, c);
#pragma unroll
                    for (int c = 0; c < 15; ++c) P[c] = wx.get(st, 5 + c);
                } else {
                    load_filtered(p, k, m, P);
                }
                if (cur.is_tail(k)) {
                    selem_last(ec, m, P);
                } else {
                    Trans<T> tr;
                    ok &= get_trans<T, LIN>(p, k, state_ix(p, k, a, lane), tr);
                    T mp[5], FP[25], Pp[15];
                    predict(tr, m, P, mp, FP, Pp);
                    ok &= selem_from_prediction(m, P, FP, Pp, mp, ec);
                }
            }
            apply_smoother(ec, s, s);
            const int64_t ix = state_ix(p, k, a, lane);
            T xold[5];
            if (want_norm) load_nominal(p, ix, xold);
            bool finite = true;
#pragma unroll
            for (int i = 0; i < 5; ++i) {
                finite = finite && isfinite(s.m[i]);
                p.x[i * p.cs + ix] = s.m[i];
            }
            if (!finite) atomicOr(p.status, ST_NONFINITE);
            if (write_P) {
#pragma unroll
                for (int i = 0; i < 15; ++i) p.P[i * p.cs + ix] = s.P[i];
            }
            if (want_norm) {
                if (cur.b != nb) {
                    if (nb >= 0) {
                        atomicAdd(conv + 2 * nb, num);
                        atomicAdd(conv + 2 * nb + 1, den);
                    }
                    nb = cur.b;
                    num = 0.0;
                    den = 0.0;
                }
#pragma unroll
                for (int i = 0; i < 5; ++i) {
                    const double dv = double(s.m[i]) - double(xold[i]);
                    num += dv * dv;
                    den += double(s.m[i]) * double(s.m[i]);
                }
            }
        }
        if (run) __syncwarp();
    }
    if (run) wpar = stored ? we.parity : wx.parity;
    return ok;
}

// ---- block and grid levels -------------------------------------------------------------

// The filtering operator of the tree levels as one out-of-line function: the
// lane and top-level trees then run the same copy of its ~2,000 instructions,
// which stays in the instruction cache from level to level, where two inlined
// copies were each fetched afresh (the smaller operators stay inline).
template <typename T>
__device__ __noinline__ void tree_combine_filter(const FElem<T>& a, const FElem<T>& b, FElem<T>& o)
{
    combine_filter(a, b, o);
}

template <typename T, int NE>
PES_DEV void copy_elem_to_global(const T* src, T* dst)
{
    for (int i = threadIdx.x; i < NE; i += blockDim.x) dst[i] = src[i];
}

// n blocks' aggregates (NE scalars each) from global into shared memory, eight
// loads in flight per thread before their stores (one L2 round trip per eight
// scalars instead of one per scalar).
template <typename T, int NT, int NE>
PES_DEV void load_aggregates(const T* src, T* dst, int n)
{
    constexpr int U = 8;
    const int total = n * NE;
#pragma unroll 1
    for (int i0 = threadIdx.x; i0 < total; i0 += U * NT) {
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * NT;
            v[u] = i < total ? src[i] : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * NT;
            if (i < total) dst[i] = v[u];
        }
    }
}

// Filtering levels 2-4. elem[t] holds lane t's folded element on entry; returns
// the Gaussian of the state before lane t's chunk.
//
// The operators of a tree level are issue-bound, one thread's instruction
// stream each: a level costs one operator's time only while no SM
// sub-partition runs two warps of it. So the operator at element 2t + 1 (or
// 2t) runs on thread t < NT / 2: a level's active threads then sit in at most
// NT / 64 warps, one per sub-partition, where the element's own thread would
// spread them over all NT / 32 warps.
template <typename T, int NT>
PES_DEV void filter_block_scan(const KParams<T>& p, FElem<T>* elem, FElem<T>* top, Gauss<T>* gs,
                               Gauss<T>* gblock, unsigned& gen, Gauss<T>& out, int it)
{
    const int t = threadIdx.x;
    const bool half = t < NT / 2;
    const int to = 2 * t + 1, te = 2 * t;   // the odd and the even element of thread t
    __syncthreads();
    PES_PHASE(p, it, 1);
#pragma unroll 1
    for (int s = 1; s < NT; s <<= 1) {
        if (half && ((to + 1) & (2 * s - 1)) == 0) tree_combine_filter(elem[to - s], elem[to], elem[to]);
        __syncthreads();
    }
    copy_elem_to_global<T, FE>(reinterpret_cast<const T*>(&elem[NT - 1]), p.aggF + (size_t)blockIdx.x * FE);
    PES_PHASE(p, it, 2);
    grid_barrier(p, gen);
    PES_PHASE(p, it, 3);
    // level 3: Gaussian of the state before this block = product of blocks [0, blockIdx)
    if (t == 0) {
#pragma unroll
        for (int i = 0; i < 5; ++i) gblock->m[i] = T(0);
#pragma unroll
        for (int i = 0; i < 15; ++i) gblock->P[i] = T(0);
    }
    const int j = blockIdx.x;
#pragma unroll 1
    for (int c0 = 0; c0 < j; c0 += NT) {
        const int n = min(NT, j - c0);
        __syncthreads();
        load_aggregates<T, NT, FE>(p.aggF + (size_t)c0 * FE, reinterpret_cast<T*>(top), n);
        __syncthreads();
#pragma unroll 1
        for (int s = 1; s < n; s <<= 1) {
            if (half && (te & (2 * s - 1)) == 0 && te + s < n) tree_combine_filter(top[te], top[te + s], top[te]);
            __syncthreads();
        }
        if (t == 0) apply_filter(*gblock, top[0], *gblock);
    }
    __syncthreads();
    PES_PHASE(p, it, 4);
    // level 4: down-sweep
    if (t == NT - 1) gs[NT - 1] = *gblock;
    __syncthreads();
#pragma unroll 1
    for (int s = NT / 2; s >= 1; s >>= 1) {
        if (half && ((to + 1) & (2 * s - 1)) == 0) {
            const Gauss<T> gin = gs[to];
            Gauss<T> gr;
            apply_filter(gin, elem[to - s], gr);
            gs[to - s] = gin;
            gs[to] = gr;
        }
        __syncthreads();
    }
    out = gs[t];
    __syncthreads();
    PES_PHASE(p, it, 5);
}

// Smoothing levels 2-4 (mirrored: subtrees accumulate at their left end).
// Returns the Gaussian of the state after lane t's chunk.
template <typename T, int NT>
PES_DEV void smoother_block_scan(const KParams<T>& p, SElem<T>* elem, SElem<T>* top, Gauss<T>* gs,
                                 Gauss<T>* gblock, unsigned& gen, Gauss<T>& out, int it)
{
    const int t = threadIdx.x;
    const bool half = t < NT / 2;
    const int te = 2 * t;   // the operators run as in filter_block_scan
    __syncthreads();
    PES_PHASE(p, it, 7);
#pragma unroll 1
    for (int s = 1; s < NT; s <<= 1) {
        if (half && (te & (2 * s - 1)) == 0) combine_smoother(elem[te], elem[te + s], elem[te]);
        __syncthreads();
    }
    copy_elem_to_global<T, SE>(reinterpret_cast<const T*>(&elem[0]), p.aggS + (size_t)blockIdx.x * SE);
    PES_PHASE(p, it, 8);
    grid_barrier(p, gen);
    PES_PHASE(p, it, 9);
    if (t == 0) {
#pragma unroll
        for (int i = 0; i < 5; ++i) gblock->m[i] = T(0);
#pragma unroll
        for (int i = 0; i < 15; ++i) gblock->P[i] = T(0);
    }
    const int j = blockIdx.x;
    const int nb = gridDim.x;
#pragma unroll 1
    for (int c1 = nb; c1 > j + 1;) {
        const int n = min(NT, c1 - (j + 1));
        const int c0 = c1 - n;
        __syncthreads();
        load_aggregates<T, NT, SE>(p.aggS + (size_t)c0 * SE, reinterpret_cast<T*>(top), n);
        __syncthreads();
#pragma unroll 1
        for (int s = 1; s < n; s <<= 1) {
            if (half && (te & (2 * s - 1)) == 0 && te + s < n) combine_smoother(top[te], top[te + s], top[te]);
            __syncthreads();
        }
        if (t == 0) apply_smoother(top[0], *gblock, *gblock);
        c1 = c0;
    }
    __syncthreads();
    PES_PHASE(p, it, 10);
    if (t == 0) gs[0] = *gblock;
    __syncthreads();
#pragma unroll 1
    for (int s = NT / 2; s >= 1; s >>= 1) {
        if (half && (te & (2 * s - 1)) == 0) {
            const Gauss<T> gin = gs[te];
            Gauss<T> gl;
            apply_smoother(elem[te + s], gin, gl);
            gs[te + s] = gin;
            gs[te] = gl;
        }
        __syncthreads();
    }
    out = gs[t];
    __syncthreads();
    PES_PHASE(p, it, 11);
}

template <int NT>
constexpr size_t smem_bytes_for(size_t scalar)
{
    // lane tree (filtering elements; smoothing elements alias it), top-level
    // buffer, down-sweep Gaussians, one block Gaussian; the per-warp stream
    // stages (2 x LINS x 32 scalars per warp) reuse this memory
    static_assert(size_t(NT) * FE * 2 + size_t(NT) * GE + GE >= size_t(NT) * 2 * LINS, "stream stages must fit");
    static_assert(FE >= 2 * StatePrefetch<double>::NS, "the fold's prefetch stages fit the top-level buffer");
    return scalar * (size_t(NT) * FE * 2 + size_t(NT) * GE + GE);
}

template <typename T, int LIN, int NT>
__global__ void __launch_bounds__(NT, 1) pes_persistent_kernel(const KParams<T> p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FElem<T>* elemF = reinterpret_cast<FElem<T>*>(smem_raw);
    SElem<T>* elemS = reinterpret_cast<SElem<T>*>(smem_raw);
    FElem<T>* topF = elemF + NT;
    SElem<T>* topS = reinterpret_cast<SElem<T>*>(topF);
    Gauss<T>* gs = reinterpret_cast<Gauss<T>*>(topF + NT);
    Gauss<T>* gblock = gs + NT;
    __shared__ int s_flag;
    __shared__ double s_red[NT];
    // per-warp stream stages reuse the tree memory during the sequential passes
    __shared__ __align__(8) uint64_t s_bar[2 * (NT / 32)];
    T* wstage = reinterpret_cast<T*>(smem_raw) + (size_t)(threadIdx.x >> 5) * 2 * LINS * 32;
    uint64_t* wbar = s_bar + 2 * (threadIdx.x >> 5);
    uint32_t wpar = 0;
    if ((threadIdx.x & 31) == 0) {
        mbar_init(wbar, 1);
        mbar_init(wbar + 1, 1);
    }
    mbar_init_fence();
    __syncthreads();

    const int t = threadIdx.x;
    const int lane = blockIdx.x * NT + t;
    const int64_t a = min((int64_t)lane * p.L, p.N);
    const int64_t e = min(a + (int64_t)p.L, p.N);
    unsigned gen = 0;
    bool ok = true;

    const bool do_filter = (p.mode != MODE_SMOOTH);
    const bool do_smooth = (p.mode != MODE_FILTER);
    const bool track = (p.mode == MODE_RUN) && (p.tol > 0.0);

    int it = 0;
    bool converged = false;
#pragma unroll 1
    for (it = 0; it < p.iters; ++it) {
        if (*(volatile int*)p.status & (ST_TIMEOUT | ST_BADARG)) break;
        const bool last = (it == p.iters - 1);
        SElem<T> accS;
        PES_PHASE(p, it, 0);
        if (do_filter) {
            FElem<T> acc;
            // the sigma-point folds prefetch each next state into the
            // top-level tree's memory, idle until after the block up-sweep
            StatePrefetch<T> pf;
            pf.base = reinterpret_cast<T*>(topF) + t;
            pf.stride = NT;
            ok &= fold_filter_chunk<T, LIN>(p, a, e, lane, acc, &pf);
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            elemF[t] = acc;
            Gauss<T> G;
            filter_block_scan<T, NT>(p, elemF, topF, gs, gblock, gen, G, it);
            ok &= rerun_filter_chunk<T, LIN>(p, a, e, lane, G, accS, wstage, wbar, wpar);
            __syncthreads();   // the stream stages overlap the smoothing lane tree
            PES_PHASE(p, it, 6);
            if (track && blockIdx.x == 0) {
                // the accumulators of the next iteration were last read before
                // this iteration's first barrier; clear them for reuse
                double* nxt = p.conv + (size_t)((it + 1) & 1) * 2 * p.B;
                for (int i = t; i < 2 * p.B; i += NT) nxt[i] = 0.0;
            }
        } else {
            ok &= fold_smoother_chunk<T, LIN>(p, a, e, lane, accS);
        }
        if (do_smooth) {
            elemS[t] = accS;
            Gauss<T> Gs;
            smoother_block_scan<T, NT>(p, elemS, topS, gs, gblock, gen, Gs, it);
            const bool write_P = (p.mode != MODE_RUN) || kSigma<LIN> || last || p.write_P_every_iter;
            int nb = -1;
            double num = 0.0, den = 0.0;
            double* conv = p.conv + (size_t)(it & 1) * 2 * p.B;
            ok &= rts_chunk<T, LIN>(p, a, e, lane, Gs, write_P, track, conv, nb, num, den, wstage, wbar, wpar);
            __syncthreads();
            PES_PHASE(p, it, 12);
            if (track && nb >= 0) {
                atomicAdd(conv + 2 * nb, num);
                atomicAdd(conv + 2 * nb + 1, den);
            }
        }
        if (p.mode == MODE_RUN && (!last || track)) {
            grid_barrier(p, gen);
            PES_PHASE(p, it, 13);
            if (track) {
                // worst relative update norm over trajectories, identical in every block
                const double* conv = p.conv + (size_t)(it & 1) * 2 * p.B;
                double worst = 0.0;
                for (int b = t; b < p.B; b += NT) {
                    const double num = __ldcg(conv + 2 * b), den = __ldcg(conv + 2 * b + 1);
                    const double r = den > 0.0 ? sqrt(num / den) : sqrt(num);
                    worst = fmax(worst, r);
                    if (p.traj_iters && blockIdx.x == 0 && r <= p.tol && p.traj_iters[b] == 0) p.traj_iters[b] = it + 1;
                }
                s_red[t] = worst;
                __syncthreads();
                for (int s = NT / 2; s > 0; s >>= 1) {
                    if (t < s) s_red[t] = fmax(s_red[t], s_red[t + s]);
                    __syncthreads();
                }
                if (t == 0) s_flag = (s_red[0] <= p.tol) ? 1 : 0;
                __syncthreads();
                const int done = s_flag;
                __syncthreads();
                if (done) {
                    converged = true;
                    ++it;
                    break;
                }
            }
        }
    }
    if (!ok) atomicOr(p.status, ST_NOT_PD);
    if (blockIdx.x == 0 && t == 0) {
        if (p.iters_done) *p.iters_done = it;
        if (track && !converged) atomicOr(p.status, ST_NOT_CONVERGED);
    }
}

}  // namespace pes
