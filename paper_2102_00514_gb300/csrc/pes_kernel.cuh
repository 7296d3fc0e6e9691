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

#include "pes_ops.cuh"

namespace pes {

enum { MODE_FILTER = 0, MODE_SMOOTH = 1, MODE_RUN = 2 };

constexpr int FE = sizeof(FElem<double>) / sizeof(double);   // 70
constexpr int SE = sizeof(SElem<double>) / sizeof(double);   // 50
constexpr int GE = sizeof(Gauss<double>) / sizeof(double);   // 20
constexpr int HAND = 20;                                      // handoff scalars per state

template <typename T>
struct KParams {
    int64_t N;
    const int64_t* offsets;   // [B+1], device
    int B;
    int mode;
    int iters;                // RUN: maximum iterations; otherwise 1
    double tol;               // RUN: relative update-norm tolerance (<= 0: fixed iterations)
    int write_P_every_iter;   // RUN: write smoothed covariances in every iteration
    DevModel model;
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
    // workspace
    T* hand;           // MODE_RUN handoff: [(s * HAND + c) * NL + lane]
    T* aggF;           // [NB][FE]
    T* aggS;           // [NB][SE]
    unsigned* bar;     // grid barrier counter, zero at launch
    int* status;       // ST_* bits
    double* conv;      // [2][B][2] update-norm accumulators, zero at launch
    int* iters_done;
    int L;             // steps per lane
    int NL;            // lanes = NB * NT
    long long timeout_ns;
};

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

template <typename T>
PES_DEV void load_nominal(const KParams<T>& p, int64_t k, T* x)
{
#pragma unroll
    for (int i = 0; i < 5; ++i) x[i] = __ldcg(p.x + i * p.N + k);
}

template <typename T>
PES_DEV void load_nominal_cov(const KParams<T>& p, int64_t k, T* P)
{
#pragma unroll
    for (int i = 0; i < 15; ++i) P[i] = __ldcg(p.P + i * p.N + k);
}

template <typename T>
PES_DEV void load_y(const KParams<T>& p, int64_t k, T* y)
{
    y[0] = __ldg(p.y + k);
    y[1] = __ldg(p.y + p.N + k);
}

// ---- linearisation of one step ------------------------------------------------

// Transition k -> k+1.
template <typename T, int LIN>
PES_DEV bool get_trans(const KParams<T>& p, int64_t k, Trans<T>& tr)
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
        return true;
    } else if (LIN == LIN_IEKS) {
        T xn[5];
        load_nominal(p, k, xn);
        lin_trans_taylor(p.model, xn, tr);
        return true;
    } else {
        T xn[5], Pn[15], L[25], rd[5];
        load_nominal(p, k, xn);
        load_nominal_cov(p, k, Pn);
        const bool ok = cub_factor(Pn, L, rd);
        lin_trans_cubature(p.model, xn, L, rd, tr);
        return ok;
    }
}

// Observation at k (optionally also the transition k -> k+1, which shares
// the nominal and, for cubature, the sigma points' factor).
template <typename T, int LIN>
PES_DEV bool get_obs(const KParams<T>& p, int64_t k, int b, Obs<T>& ob, bool want_trans, Trans<T>& tr)
{
    T y[2];
    load_y(p, k, y);
    if (LIN == LIN_ARRAYS) {
#pragma unroll
        for (int i = 0; i < 10; ++i) ob.H[i] = __ldg(p.H + i * p.N + k);
        ob.r[0] = y[0] - __ldg(p.d + k);
        ob.r[1] = y[1] - __ldg(p.d + p.N + k);
#pragma unroll
        for (int i = 0; i < 5; ++i) ob.xn[i] = T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i) ob.R[i] = __ldg(p.Rp + i * p.N + k);
        if (want_trans) get_trans<T, LIN>(p, k, tr);
        return true;
    } else if (LIN == LIN_IEKS) {
        T xn[5];
        load_nominal(p, k, xn);
        lin_obs_taylor(p.model, b, xn, y, ob);
        if (want_trans) lin_trans_taylor(p.model, xn, tr);
        return true;
    } else {
        T xn[5], Pn[15], L[25], rd[5];
        load_nominal(p, k, xn);
        load_nominal_cov(p, k, Pn);
        const bool ok = cub_factor(Pn, L, rd);
        lin_obs_cubature(p.model, b, xn, L, rd, y, ob);
        if (want_trans) lin_trans_cubature(p.model, xn, L, rd, tr);
        return ok;
    }
}

// ---- lane-level passes -------------------------------------------------------------

// Filtering, level 1: fold the lane's chunk [a, e) into one element.
template <typename T, int LIN>
PES_DEV bool fold_filter_chunk(const KParams<T>& p, int64_t a, int64_t e, FElem<T>& acc)
{
    bool ok = true;
    T zero[5] = {T(0), T(0), T(0), T(0), T(0)};
    if (a >= e) {
        felem_identity(acc, zero);
        return ok;
    }
    SegCursor cur;
    cur.init(p.offsets, p.B, a);
    Trans<T> tr;
    if (!cur.is_head(a)) {
        ok &= get_trans<T, LIN>(p, a - 1, tr);
        felem_identity(acc, tr.xn);
    } else {
        felem_identity(acc, zero);
    }
    for (int64_t k = a; k < e; ++k) {
        cur.forward(k);
        const bool want_trans = (k + 1 < e) && !cur.is_tail(k);
        if (cur.is_head(k)) {
            T m0[5], P0[15];
            load_prior(p, cur.b, m0, P0);
            felem_apply_prior(acc, m0, P0);
            if (want_trans) ok &= get_trans<T, LIN>(p, k, tr);
        } else {
            Obs<T> ob;
            Trans<T> trn;
            ok &= get_obs<T, LIN>(p, k, cur.b, ob, want_trans, trn);
            ok &= fold_filter_step(acc, tr, ob);
            if (want_trans) tr = trn;
        }
    }
    return ok;
}

template <typename T>
PES_DEV void store_filtered(const KParams<T>& p, int64_t k, int s, int lane, const T* m, const T* P)
{
    if (p.mode == MODE_RUN) {
        T* h = p.hand + (size_t)s * HAND * p.NL + lane;
#pragma unroll
        for (int i = 0; i < 5; ++i) h[(size_t)i * p.NL] = m[i];
#pragma unroll
        for (int i = 0; i < 15; ++i) h[(size_t)(5 + i) * p.NL] = P[i];
    } else {
#pragma unroll
        for (int i = 0; i < 5; ++i) p.xf[i * p.N + k] = m[i];
#pragma unroll
        for (int i = 0; i < 15; ++i) p.Pf[i * p.N + k] = P[i];
    }
}

template <typename T>
PES_DEV void load_filtered(const KParams<T>& p, int64_t k, int s, int lane, T* m, T* P)
{
    if (p.mode == MODE_RUN) {
        const T* h = p.hand + (size_t)s * HAND * p.NL + lane;
#pragma unroll
        for (int i = 0; i < 5; ++i) m[i] = h[(size_t)i * p.NL];
#pragma unroll
        for (int i = 0; i < 15; ++i) P[i] = h[(size_t)(5 + i) * p.NL];
    } else {
#pragma unroll
        for (int i = 0; i < 5; ++i) m[i] = __ldg(p.xf + i * p.N + k);
#pragma unroll
        for (int i = 0; i < 15; ++i) P[i] = __ldg(p.Pf + i * p.N + k);
    }
}

// Filtering, level 5: re-run the chunk from the Gaussian of the state before it,
// storing filtered moments; in MODE_RUN also build and fold the chunk's
// smoothing elements (Eqs. 17-18) into accS.
template <typename T, int LIN>
PES_DEV bool rerun_filter_chunk(const KParams<T>& p, int64_t a, int64_t e, int lane, const Gauss<T>& G,
                                SElem<T>& accS)
{
    bool ok = true;
    selem_identity(accS);
    if (a >= e) return ok;
    const bool smooth = (p.mode == MODE_RUN);
    SegCursor cur;
    cur.init(p.offsets, p.B, a);
    T m[5], P[15];
#pragma unroll
    for (int i = 0; i < 5; ++i) m[i] = G.m[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) P[i] = G.P[i];
    Trans<T> tr;
    if (!cur.is_head(a)) ok &= get_trans<T, LIN>(p, a - 1, tr);
    for (int64_t k = a; k < e; ++k) {
        cur.forward(k);
        const bool want_trans = !cur.is_tail(k) && (k + 1 < p.N);
        if (cur.is_head(k)) {
            if (smooth && k > a) {
                SElem<T> el;
                selem_last(el, m, P);
                combine_smoother(accS, el, accS);
            }
            load_prior(p, cur.b, m, P);
            if (want_trans) ok &= get_trans<T, LIN>(p, k, tr);
        } else {
            T mp[5], FP[25], Pp[15];
            predict(tr, m, P, mp, FP, Pp);
            if (smooth && k > a) {
                SElem<T> el;
                ok &= selem_from_prediction(m, P, FP, Pp, mp, el);
                combine_smoother(accS, el, accS);
            }
            Obs<T> ob;
            Trans<T> trn;
            ok &= get_obs<T, LIN>(p, k, cur.b, ob, want_trans, trn);
            ok &= kf_update(ob, mp, Pp, m, P);
            if (want_trans) tr = trn;
        }
        store_filtered(p, k, (int)(k - a), lane, m, P);
    }
    if (smooth) {
        // smoothing element of the chunk's last state
        SElem<T> el;
        if (cur.is_tail(e - 1)) {
            selem_last(el, m, P);
        } else {
            T mp[5], FP[25], Pp[15];
            predict(tr, m, P, mp, FP, Pp);
            ok &= selem_from_prediction(m, P, FP, Pp, mp, el);
        }
        combine_smoother(accS, el, accS);
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
    for (int64_t k = a; k < e; ++k) {
        cur.forward(k);
        T m[5], P[15];
        load_filtered(p, k, (int)(k - a), lane, m, P);
        SElem<T> el;
        if (cur.is_tail(k)) {
            selem_last(el, m, P);
        } else {
            Trans<T> tr;
            ok &= get_trans<T, LIN>(p, k, tr);
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
// E P E^T + L. Writes the smoothed moments; in MODE_RUN they replace the
// nominal in place (each state's nominal is read before it is overwritten).
template <typename T, int LIN>
PES_DEV bool rts_chunk(const KParams<T>& p, int64_t a, int64_t e, int lane, const Gauss<T>& G, bool write_P,
                       bool want_norm, double* conv, int& nb, double& num, double& den)
{
    bool ok = true;
    if (a >= e) return ok;
    SegCursor cur;
    cur.init(p.offsets, p.B, e - 1);
    Gauss<T> s = G;
    for (int64_t k = e - 1; k >= a; --k) {
        cur.backward(k);
        T m[5], P[15];
        load_filtered(p, k, (int)(k - a), lane, m, P);
        T xold[5];
        if (cur.is_tail(k)) {
#pragma unroll
            for (int i = 0; i < 5; ++i) s.m[i] = m[i];
#pragma unroll
            for (int i = 0; i < 15; ++i) s.P[i] = P[i];
            if (want_norm) load_nominal(p, k, xold);
        } else {
            Trans<T> tr;
            ok &= get_trans<T, LIN>(p, k, tr);
            if (want_norm) {
#pragma unroll
                for (int i = 0; i < 5; ++i) xold[i] = tr.xn[i];
            }
            T mp[5], FP[25], Pp[15];
            predict(tr, m, P, mp, FP, Pp);
            SElem<T> el;
            ok &= selem_from_prediction(m, P, FP, Pp, mp, el);
            apply_smoother(el, s, s);
        }
        bool finite = true;
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            finite = finite && isfinite(s.m[i]);
            p.x[i * p.N + k] = s.m[i];
        }
        if (!finite) atomicOr(p.status, ST_NONFINITE);
        if (write_P) {
#pragma unroll
            for (int i = 0; i < 15; ++i) p.P[i * p.N + k] = s.P[i];
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
    return ok;
}

// ---- block and grid levels -------------------------------------------------------------

template <typename T, int NE>
PES_DEV void copy_elem_to_global(const T* src, T* dst)
{
    for (int i = threadIdx.x; i < NE; i += blockDim.x) dst[i] = src[i];
}

// Filtering levels 2-4. elem[t] holds lane t's folded element on entry; returns
// the Gaussian of the state before lane t's chunk.
template <typename T, int NT>
PES_DEV void filter_block_scan(const KParams<T>& p, FElem<T>* elem, FElem<T>* top, Gauss<T>* gs,
                               Gauss<T>* gblock, unsigned& gen, Gauss<T>& out)
{
    const int t = threadIdx.x;
    __syncthreads();
#pragma unroll 1
    for (int s = 1; s < NT; s <<= 1) {
        if (((t + 1) & (2 * s - 1)) == 0) combine_filter(elem[t - s], elem[t], elem[t]);
        __syncthreads();
    }
    copy_elem_to_global<T, FE>(reinterpret_cast<const T*>(&elem[NT - 1]), p.aggF + (size_t)blockIdx.x * FE);
    grid_barrier(p, gen);
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
        for (int i = t; i < n * FE; i += NT)
            reinterpret_cast<T*>(top)[i] = __ldcg(p.aggF + (size_t)c0 * FE + i);
        __syncthreads();
#pragma unroll 1
        for (int s = 1; s < n; s <<= 1) {
            if ((t & (2 * s - 1)) == 0 && t + s < n) combine_filter(top[t], top[t + s], top[t]);
            __syncthreads();
        }
        if (t == 0) apply_filter(*gblock, top[0], *gblock);
    }
    __syncthreads();
    // level 4: down-sweep
    if (t == NT - 1) gs[NT - 1] = *gblock;
    __syncthreads();
#pragma unroll 1
    for (int s = NT / 2; s >= 1; s >>= 1) {
        if (((t + 1) & (2 * s - 1)) == 0) {
            const Gauss<T> gin = gs[t];
            Gauss<T> gr;
            apply_filter(gin, elem[t - s], gr);
            gs[t - s] = gin;
            gs[t] = gr;
        }
        __syncthreads();
    }
    out = gs[t];
    __syncthreads();
}

// Smoothing levels 2-4 (mirrored: subtrees accumulate at their left end).
// Returns the Gaussian of the state after lane t's chunk.
template <typename T, int NT>
PES_DEV void smoother_block_scan(const KParams<T>& p, SElem<T>* elem, SElem<T>* top, Gauss<T>* gs,
                                 Gauss<T>* gblock, unsigned& gen, Gauss<T>& out)
{
    const int t = threadIdx.x;
    __syncthreads();
#pragma unroll 1
    for (int s = 1; s < NT; s <<= 1) {
        if ((t & (2 * s - 1)) == 0) combine_smoother(elem[t], elem[t + s], elem[t]);
        __syncthreads();
    }
    copy_elem_to_global<T, SE>(reinterpret_cast<const T*>(&elem[0]), p.aggS + (size_t)blockIdx.x * SE);
    grid_barrier(p, gen);
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
        for (int i = t; i < n * SE; i += NT)
            reinterpret_cast<T*>(top)[i] = __ldcg(p.aggS + (size_t)c0 * SE + i);
        __syncthreads();
#pragma unroll 1
        for (int s = 1; s < n; s <<= 1) {
            if ((t & (2 * s - 1)) == 0 && t + s < n) combine_smoother(top[t], top[t + s], top[t]);
            __syncthreads();
        }
        if (t == 0) apply_smoother(top[0], *gblock, *gblock);
        c1 = c0;
    }
    __syncthreads();
    if (t == 0) gs[0] = *gblock;
    __syncthreads();
#pragma unroll 1
    for (int s = NT / 2; s >= 1; s >>= 1) {
        if ((t & (2 * s - 1)) == 0) {
            const Gauss<T> gin = gs[t];
            Gauss<T> gl;
            apply_smoother(elem[t + s], gin, gl);
            gs[t + s] = gin;
            gs[t] = gl;
        }
        __syncthreads();
    }
    out = gs[t];
    __syncthreads();
}

template <int NT>
constexpr size_t smem_bytes_for(size_t scalar)
{
    // lane tree (filtering elements; smoothing elements alias it), top-level
    // buffer, down-sweep Gaussians, one block Gaussian
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
        if (do_filter) {
            FElem<T> acc;
            ok &= fold_filter_chunk<T, LIN>(p, a, e, acc);
            elemF[t] = acc;
            Gauss<T> G;
            filter_block_scan<T, NT>(p, elemF, topF, gs, gblock, gen, G);
            ok &= rerun_filter_chunk<T, LIN>(p, a, e, lane, G, accS);
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
            smoother_block_scan<T, NT>(p, elemS, topS, gs, gblock, gen, Gs);
            const bool write_P = (p.mode != MODE_RUN) || (LIN == LIN_CUBATURE) || last || p.write_P_every_iter;
            int nb = -1;
            double num = 0.0, den = 0.0;
            double* conv = p.conv + (size_t)(it & 1) * 2 * p.B;
            ok &= rts_chunk<T, LIN>(p, a, e, lane, Gs, write_P, track, conv, nb, num, den);
            if (track && nb >= 0) {
                atomicAdd(conv + 2 * nb, num);
                atomicAdd(conv + 2 * nb + 1, den);
            }
        }
        if (p.mode == MODE_RUN && (!last || track)) {
            grid_barrier(p, gen);
            if (track) {
                // worst relative update norm over trajectories, identical in every block
                const double* conv = p.conv + (size_t)(it & 1) * 2 * p.B;
                double worst = 0.0;
                for (int b = t; b < p.B; b += NT) {
                    const double num = __ldcg(conv + 2 * b), den = __ldcg(conv + 2 * b + 1);
                    const double r = den > 0.0 ? sqrt(num / den) : sqrt(num);
                    worst = fmax(worst, r);
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
