// Refinement of the final iteration: Newton's method on the Kalman filter and
// RTS recursions of the linearised model (Sec. 3 iteration, Eq. 11 model).
//
// Given one iteration's linearisation, the smoothed moments it defines are the
// solution of two recursions: the filter, (m_k, P_k) = Phi_k(m_{k-1}, P_{k-1})
// (predict through the transition k-1 -> k, update with y_k), and the RTS
// smoother, (m^s_k, P^s_k) = Psi_k(m^s_{k+1}, P^s_{k+1}; m_k, P_k). The FP32
// scan solves them to about 1e-4 relative on long, ill-conditioned
// trajectories. Newton's method on the stacked equations takes that solution
// to full accuracy in one step:
//   * residuals: the exact-arithmetic image of each step, evaluated in
//     float-float from the FP32 solution at the step's input, minus the FP32
//     solution at its output: s_k, r_k (means, covariances);
//   * the step's derivative: for the filter, the covariance recursion's is
//     dP -> Abar dP Abar^T with the closed-loop matrix Abar = (I - K H) F, and
//     the mean's is dm -> Abar (dm + dP w) with w = F^T H^T S^{-1} v (v the
//     innovation: the gain moves with the covariance); for the RTS step, which
//     is affine in the later state, dm -> G dm, dP -> G dP G^T;
//   * the correction: the linear recursion delta_k = D_k(delta_{k-1}) + (s_k, r_k),
//     itself an associative scan over the elements (Abar, w, s, r), solved in
//     FP32 by the same three-level scan as the smoother (its values are the
//     small differences, so FP32 holds them to ~1e-4 of their size, ~1e-8 of
//     the moments').
// The filter's correction comes first (its second-order remainder is measured
// at ~1e-7 of the moments at T = 2^20); the RTS residuals then use the
// corrected filtered moments, as float-float pairs (FP32 value + FP32
// correction), and since the RTS step is affine in the later state its
// correction is exact up to rounding.
//
// The linearisation itself must be as accurate as the refined result: FP32
// rounding of F, c, Q', H, d, R' moves the smoother by ~6e-7 relative, but the
// FP32 cubature regression's slope F = Psi^T Pbar^{-1} carries ~2e-6 relative
// error (differences of f at sigma points, divided by the factor of an
// ill-conditioned Pbar), which moves the smoother by ~6e-5. The cubature
// transition's slope is therefore recomputed in float-float
// (cub_trans_slope_ff); every other linearisation quantity keeps its FP32 value.
#pragma once

#include "pes_ff.cuh"
#include "pes_kernel.cuh"

namespace pes {

constexpr int RE = 50;   // correction element: Abar (or G) 25, w 5, s 5, r 15
constexpr int RT = 45;   // stored transition: F 25, fx 5, Q' 15
constexpr int RD = 20;   // correction of one state: means 5, covariance 15

struct RefineParams {
    int64_t N;
    const int64_t* offsets;   // [B+1], device
    int B;
    int L, NL;                // lane-major geometry of every per-state array below
    int64_t cs;               // component stride: L * NL
    DevModel<float> model;
    const float* y;           // [2][cs]
    const float* m0;          // [B][5]
    const float* P0;          // [B][15]
    const float* nom;         // [20][cs]: the final iteration's nominal, means then covariances
    const float* filt;        // [20][cs]: the FP32 filtered moments of the final iteration
    float* xs;                // [20][cs]: the FP32 smoothed moments; refined in place
    float* elem;              // [RE][cs]
    float* trans;             // [RT][cs]
    float* dlt;               // [RD][cs]: the filter's correction
    float* agg;               // [blocks][RE]: block aggregates of the correction scan
    unsigned* bar;            // grid barrier counter, zero at launch
    int* status;
    long long timeout_ns;
};

struct RElem {
    float A[25];
    float w[5];
    float s[5];
    float r[15];
};

struct RState {
    float m[5];
    float P[15];
};

PES_DEV int64_t lane_index(int64_t k, int L, int NL) { return (k % L) * NL + k / L; }

PES_DEV int traj_of(const int64_t* off, int B, int64_t k)
{
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---- per-thread scratch -----------------------------------------------------------
//
// The float-float steps below keep the matrices that a rolled loop indexes by
// its counter in shared memory, one slice per thread: element e of the calling
// thread at p[e * NT] (a warp's accesses to one element fall in consecutive
// banks); a float-float value takes two consecutive elements. Rolling the outer
// loop of each matrix product keeps the code a few thousand instructions long,
// small enough for the instruction caches, where the fully unrolled form (about
// 9,000 per step) left most warps waiting for instructions.
constexpr int SCR_F = 0;     // F, 25 floats
constexpr int SCR_M = 25;    // a 5x5 float-float matrix (F P, then the gain), 50 floats
constexpr int SCR_S = 75;    // a packed symmetric float-float matrix (the prediction), 30 floats
constexpr int SCR_N = 105;   // floats per thread

template <int NT>
struct Scratch {
    float* p;
    PES_DEV float& operator[](int e) const { return p[e * NT]; }
    PES_DEV ff ld(int e) const { return ff{p[e * NT], p[(e + 1) * NT]}; }
    PES_DEV void st(int e, ff v) const
    {
        p[e * NT] = v.hi;
        p[(e + 1) * NT] = v.lo;
    }
};

// packed index of (i, j), i <= j, for a runtime i
PES_DEV int si_rt(int i, int j) { return i * 5 - (i * (i - 1)) / 2 + (j - i); }

// ---- the cubature transition slope in float-float -------------------------------
//
// The sigma points are xbar +- S e_i with S = fl(scale L), the FP32 factor
// scaled in FP32 (a point set whose covariance S S^T / scale^2 differs from
// Pbar by rounding only); for that point set the regression slope is exactly
// F = (1/2) D S^{-1} with D_i = f(xbar + S e_i) - f(xbar - S e_i), which is
// formed here with every operation in float-float. The turn angles
// (w +- S_4i) dt come by angle addition from the reference angle's sine and
// cosine (float-float series after reduction) and the offsets' (series).
// Writes F to the scratch (SCR_F); uses SCR_M .. SCR_M + 65 for S and D.
template <int NT>
PES_DEV void cub_trans_slope_ff(const DevModel<float>& m, const float* xbar, const float* L, Scratch<NT> sc)
{
    if (m.kind == MODEL_LINEAR) {
#pragma unroll
        for (int i = 0; i < 25; ++i) sc[SCR_F + i] = m.F[i];
        return;
    }
    constexpr int SS = SCR_M;        // S, 25 floats
    constexpr int SD = SCR_M + 25;   // D rows 0..3 by columns, float-float: 40 floats
    const float dt = m.dt;
#pragma unroll
    for (int i = 0; i < 25; ++i) sc[SS + i] = __fmul_rn(m.sp_scale, L[i]);
    ff s0, c0, o0;
    ff_sincos(two_prod(xbar[4], dt), &s0, &c0, &o0);
#pragma unroll 1
    for (int i = 0; i < 5; ++i) {
        const float Spx = sc[SS + i], Spy = sc[SS + 5 + i], Svx = sc[SS + 10 + i], Svy = sc[SS + 15 + i];
        const float Sw = sc[SS + 20 + i];
        ff se, ce, oe;
        ff_sincos(two_prod(Sw, dt), &se, &ce, &oe);
        const ff s0ce = ff_mul(s0, ce), c0se = ff_mul(c0, se), s0se = ff_mul(s0, se);
        const ff c0ce = ff_mul(c0, ce);
        const ff omc_base = ff_fma(c0, oe, o0);   // (1 - c0) + c0 (1 - ce)
        ff z[2][4];
#pragma unroll
        for (int sg = 0; sg < 2; ++sg) {
            const float sgn = sg == 0 ? 1.0f : -1.0f;
            // sin, cos and 1 - cos of the angle (w + sgn S_4i) dt
            const ff sn = sg == 0 ? ff_add(s0ce, c0se) : ff_sub(s0ce, c0se);
            const ff cs = sg == 0 ? ff_sub(c0ce, s0se) : ff_add(c0ce, s0se);
            const ff om = sg == 0 ? ff_add(omc_base, s0se) : ff_sub(omc_base, s0se);
            const ff w = two_sum(xbar[4], sgn * Sw);
            ff A1, A2;
            if (w.hi == 0.0f && w.lo == 0.0f) {
                A1 = ff_make(dt);
                A2 = ff_make(0.0f);
            } else {
                const ff iw = ff_rcp(w);
                A1 = ff_mul(sn, iw);
                A2 = ff_mul(om, iw);
            }
            const ff vx = two_sum(xbar[2], sgn * Svx);
            const ff vy = two_sum(xbar[3], sgn * Svy);
            // position increments and velocities of f at the point (the
            // positions themselves contribute 2 S_pi to D, added below)
            z[sg][0] = ff_sub(ff_mul(A1, vx), ff_mul(A2, vy));
            z[sg][1] = ff_add(ff_mul(A2, vx), ff_mul(A1, vy));
            z[sg][2] = ff_sub(ff_mul(cs, vx), ff_mul(sn, vy));
            z[sg][3] = ff_add(ff_mul(sn, vx), ff_mul(cs, vy));
        }
        sc.st(SD + 2 * (0 * 5 + i), ff_add_f(ff_sub(z[0][0], z[1][0]), 2.0f * Spx));
        sc.st(SD + 2 * (1 * 5 + i), ff_add_f(ff_sub(z[0][1], z[1][1]), 2.0f * Spy));
        sc.st(SD + 2 * (2 * 5 + i), ff_sub(z[0][2], z[1][2]));
        sc.st(SD + 2 * (3 * 5 + i), ff_sub(z[0][3], z[1][3]));
    }
    // rows g of F solve g S = D_r / 2 (S lower triangular), from the last column
    ff rs[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) rs[c] = ff_rcp(ff_make(sc[SS + c * 5 + c]));
#pragma unroll 1
    for (int r = 0; r < 4; ++r) {
        ff g[5];
#pragma unroll
        for (int c = 4; c >= 0; --c) {
            const ff dd = sc.ld(SD + 2 * (r * 5 + c));
            ffacc acc = acc_of(ff{0.5f * dd.hi, 0.5f * dd.lo});
#pragma unroll
            for (int l = c + 1; l < 5; ++l) acc_add(acc, g[l], -sc[SS + l * 5 + c]);
            g[c] = ff_mul(acc_done(acc), rs[c]);
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) sc[SCR_F + r * 5 + c] = g[c].hi;
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) sc[SCR_F + 20 + c] = c == 4 ? 1.0f : 0.0f;
}

// ---- residuals ---------------------------------------------------------------------

// One Kalman step in float-float from the FP32 filtered moments (m, P) of
// state k, through the transition (k -> k+1: F in the scratch at SCR_F, fx,
// Q', xn of tr) and the observation ob of state k+1: the step's
// exact-arithmetic image (mf, Pf), to about 1e-14 relative of the operands,
// and its derivatives Abar = (I - K H) F, w = F^T H^T S^{-1} v in FP32.
// Returns false if S is not positive definite.
template <int NT>
PES_DEV bool ff_kalman_step(const Trans<float>& tr, const Obs<float>& ob, const float* m, const float* P, ff* mf,
                            ff* Pf, float* Abar, float* w, Scratch<NT> sc)
{
    // F P by rows
#pragma unroll 1
    for (int i = 0; i < 5; ++i) {
        float Fi[5];
#pragma unroll
        for (int l = 0; l < 5; ++l) Fi[l] = sc[SCR_F + i * 5 + l];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            ffacc acc = acc_of(two_prod(Fi[0], P[si(0, j)]));
#pragma unroll
            for (int l = 1; l < 5; ++l) acc_add(acc, Fi[l], P[si(l, j)]);
            sc.st(SCR_M + 2 * (i * 5 + j), acc_done(acc));
        }
    }
    // (F P) F^T, upper triangle by rows
#pragma unroll 1
    for (int i = 0; i < 5; ++i) {
        ff FPi[5];
#pragma unroll
        for (int l = 0; l < 5; ++l) FPi[l] = sc.ld(SCR_M + 2 * (i * 5 + l));
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            if (j < i) continue;
            ffacc acc = acc_of(ff_mul_f(FPi[0], sc[SCR_F + j * 5]));
#pragma unroll
            for (int l = 1; l < 5; ++l) acc_add(acc, FPi[l], sc[SCR_F + j * 5 + l]);
            sc.st(SCR_S + 2 * si_rt(i, j), acc_done(acc));
        }
    }
    ff Pp[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) Pp[i] = ff_add_f(sc.ld(SCR_S + 2 * i), tr.Q[i]);
    ff mp[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        ffacc acc = acc_of_f(tr.fx[i]);
#pragma unroll
        for (int l = 0; l < 5; ++l) acc_add(acc, ff_diff_f(m[l], tr.xn[l]), sc[SCR_F + i * 5 + l]);
        mp[i] = acc_done(acc);
    }
    ff HP[10];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            ffacc acc = acc_of(ff_mul_f(Pp[si(0, j)], ob.H[r * 5]));
#pragma unroll
            for (int l = 1; l < 5; ++l) acc_add(acc, Pp[si(l, j)], ob.H[r * 5 + l]);
            HP[r * 5 + j] = acc_done(acc);
        }
    ff S[3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int q = r; q < 2; ++q) {
            ffacc acc = acc_of_f(ob.R[si2(r, q)]);
#pragma unroll
            for (int l = 0; l < 5; ++l) acc_add(acc, HP[r * 5 + l], ob.H[q * 5 + l]);
            S[si2(r, q)] = acc_done(acc);
        }
    const ff det = ff_sub(ff_mul(S[0], S[2]), ff_mul(S[1], S[1]));
    const bool ok = det.hi > 0.0f && S[0].hi > 0.0f;
    const ff rdet = ff_rcp(ok ? det : ff_make(1.0f));
    const ff Si[3] = {ff_mul(S[2], rdet), ff_neg(ff_mul(S[1], rdet)), ff_mul(S[0], rdet)};
    // K^T = S^{-1} H P-, innovation v = r - H (m- - xn)
    ff KT[10];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int j = 0; j < 5; ++j) KT[r * 5 + j] = ff_fma(Si[si2(r, 1)], HP[5 + j], ff_mul(Si[si2(r, 0)], HP[j]));
    ff v[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        ffacc acc = acc_of_f(ob.r[r]);
#pragma unroll
        for (int l = 0; l < 5; ++l) acc_add(acc, ff_add_f(mp[l], -ob.xn[l]), -ob.H[r * 5 + l]);
        v[r] = acc_done(acc);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        ffacc acc = acc_of(mp[i]);
        acc_add(acc, KT[i], v[0]);
        acc_add(acc, KT[5 + i], v[1]);
        mf[i] = acc_done(acc);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i; j < 5; ++j) {
            ffacc acc = acc_of(Pp[si(i, j)]);
            acc_add(acc, ff_neg(KT[i]), HP[j]);
            acc_add(acc, ff_neg(KT[5 + i]), HP[5 + j]);
            Pf[si(i, j)] = acc_done(acc);
        }
    // derivatives, FP32
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            float t = 0.0f;
#pragma unroll
            for (int l = 0; l < 5; ++l) {
                const float ikh = (i == l ? 1.0f : 0.0f) - KT[i].hi * ob.H[l] - KT[5 + i].hi * ob.H[5 + l];
                t = fmaf(ikh, sc[SCR_F + l * 5 + j], t);
            }
            Abar[i * 5 + j] = t;
        }
    const float Siv0 = Si[0].hi * v[0].hi + Si[1].hi * v[1].hi;
    const float Siv1 = Si[1].hi * v[0].hi + Si[2].hi * v[1].hi;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        float t = 0.0f;
#pragma unroll
        for (int l = 0; l < 5; ++l) t = fmaf(sc[SCR_F + l * 5 + i], ob.H[l] * Siv0 + ob.H[5 + l] * Siv1, t);
        w[i] = t;
    }
    return ok;
}

// One RTS step in float-float: from the refined filtered moments (mf, Pf) of
// state k, the transition out of k (F in the scratch at SCR_F, fx, Q', xn of
// tr) and the FP32 smoothed moments (xs1, Ps1) of state k+1. Leaves the gain
// transposed, G^T = (F Pf F^T + Q')^{-1} F Pf, in the scratch at SCR_M and
// returns the smoothed mean ms and dP = Ps1 - (F Pf F^T + Q'); the covariance
// rows Pf + G dP G^T are formed by rts_cov_row.
// Returns false if the predicted covariance is not positive definite.
template <int NT>
PES_DEV bool ff_rts_gain(const Trans<float>& tr, const ff* mf, const ff* Pf, const float* xs1, const float* Ps1,
                         ff* ms, ff* dP, Scratch<NT> sc)
{
    // F Pf by rows
#pragma unroll 1
    for (int i = 0; i < 5; ++i) {
        float Fi[5];
#pragma unroll
        for (int l = 0; l < 5; ++l) Fi[l] = sc[SCR_F + i * 5 + l];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            ffacc acc = acc_of(ff_mul_f(Pf[si(0, j)], Fi[0]));
#pragma unroll
            for (int l = 1; l < 5; ++l) acc_add(acc, Pf[si(l, j)], Fi[l]);
            sc.st(SCR_M + 2 * (i * 5 + j), acc_done(acc));
        }
    }
    // (F Pf) F^T, upper triangle by rows
#pragma unroll 1
    for (int i = 0; i < 5; ++i) {
        ff FPi[5];
#pragma unroll
        for (int l = 0; l < 5; ++l) FPi[l] = sc.ld(SCR_M + 2 * (i * 5 + l));
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            if (j < i) continue;
            ffacc acc = acc_of(ff_mul_f(FPi[0], sc[SCR_F + j * 5]));
#pragma unroll
            for (int l = 1; l < 5; ++l) acc_add(acc, FPi[l], sc[SCR_F + j * 5 + l]);
            sc.st(SCR_S + 2 * si_rt(i, j), acc_done(acc));
        }
    }
    ff Pp[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) Pp[i] = ff_add_f(sc.ld(SCR_S + 2 * i), tr.Q[i]);
    // Cholesky Pp = C C^T (C lower, in Pp's packed slots) with reciprocal diagonal rd
    ff C[15], rd[5];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        ffacc sj = acc_of(Pp[si(j, j)]);
#pragma unroll
        for (int l = 0; l < j; ++l) acc_add(sj, ff_neg(C[si(j, l)]), C[si(j, l)]);
        const ff sjj = acc_done(sj);
        ok = ok && sjj.hi > 0.0f;
        const ff d = ff_sqrt(sjj.hi > 0.0f ? sjj : ff_make(1.0f));
        C[si(j, j)] = d;
        rd[j] = ff_rcp(d);
#pragma unroll
        for (int i = j + 1; i < 5; ++i) {
            ffacc t = acc_of(Pp[si(i, j)]);
#pragma unroll
            for (int l = 0; l < j; ++l) acc_add(t, ff_neg(C[si(i, l)]), C[si(j, l)]);
            C[si(i, j)] = ff_mul(acc_done(t), rd[j]);
        }
    }
    // G^T = Pp^{-1} (F Pf), column by column in place
#pragma unroll 1
    for (int c = 0; c < 5; ++c) {
        ff x[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            ffacc t = acc_of(sc.ld(SCR_M + 2 * (i * 5 + c)));
#pragma unroll
            for (int l = 0; l < i; ++l) acc_add(t, ff_neg(C[si(i, l)]), x[l]);
            x[i] = ff_mul(acc_done(t), rd[i]);
        }
#pragma unroll
        for (int i = 4; i >= 0; --i) {
            ffacc t = acc_of(x[i]);
#pragma unroll
            for (int l = i + 1; l < 5; ++l) acc_add(t, ff_neg(C[si(l, i)]), x[l]);
            x[i] = ff_mul(acc_done(t), rd[i]);
        }
#pragma unroll
        for (int i = 0; i < 5; ++i) sc.st(SCR_M + 2 * (i * 5 + c), x[i]);
    }
    // ms = mf + G (xs1 - mp), mp = fx + F (mf - xn)
    ff e[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        ffacc acc = acc_of_f(tr.fx[i]);
#pragma unroll
        for (int l = 0; l < 5; ++l) acc_add(acc, ff_add_f(mf[l], -tr.xn[l]), sc[SCR_F + i * 5 + l]);
        e[i] = ff_add_f(ff_neg(acc_done(acc)), xs1[i]);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        ffacc acc = acc_of(mf[i]);
#pragma unroll
        for (int j = 0; j < 5; ++j) acc_add(acc, sc.ld(SCR_M + 2 * (j * 5 + i)), e[j]);
        ms[i] = acc_done(acc);
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) dP[i] = ff_add_f(ff_neg(Pp[i]), Ps1[i]);
    return ok;
}

// Row i of G (Ps1 - Pp) G^T: G_il = Gt_li from the scratch; dP = Ps1 - Pp.
// Writes the row's upper part (j >= i) through out(j, value).
template <int NT, class Out>
PES_DEV void rts_cov_row(int i, const ff* dP, Scratch<NT> sc, Out out)
{
    ff row[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        ffacc acc = acc_of(ff_mul(sc.ld(SCR_M + 2 * (0 * 5 + i)), dP[si(0, j)]));
#pragma unroll
        for (int l = 1; l < 5; ++l) acc_add(acc, sc.ld(SCR_M + 2 * (l * 5 + i)), dP[si(l, j)]);
        row[j] = acc_done(acc);
    }
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        if (j < i) continue;
        ffacc acc = acc_of(ff_mul(row[0], sc.ld(SCR_M + 2 * (0 * 5 + j))));
#pragma unroll
        for (int l = 1; l < 5; ++l) acc_add(acc, row[l], sc.ld(SCR_M + 2 * (l * 5 + j)));
        out(j, acc_done(acc));
    }
}

// ---- correction elements and their composition --------------------------------------
//
// An element maps the correction of the state before it (after it, for the
// RTS direction) to its own: dm' = A (dm + dP w) + s, dP' = A dP A^T + r.
// Composition (b after a) is again such a map:
//   A = A_b A_a,  w = w_a + A_a^T w_b,  s = A_b (s_a + r_a w_b) + s_b,
//   r = A_b r_a A_b^T + r_b.
// The RTS elements have w = 0.

// y = S x + add, S symmetric packed
PES_DEV void sv_sym_add(const float* S, const float* x, const float* add, float* y)
{
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        float t = add[i];
#pragma unroll
        for (int l = 0; l < 5; ++l) t = fmaf(S[si(i, l)], x[l], t);
        y[i] = t;
    }
}

PES_DEV void relem_identity(RElem& e)
{
    set_identity(e.A);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        e.w[i] = 0.0f;
        e.s[i] = 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) e.r[i] = 0.0f;
}

template <bool W>
PES_DEV void relem_compose(const RElem& b, const RElem& a, RElem& c)
{
    float sv[5];
    if (W) {
        sv_sym_add(a.r, b.w, a.s, sv);
    } else {
#pragma unroll
        for (int i = 0; i < 5; ++i) sv[i] = a.s[i];
    }
    float s[5];
    mv(b.A, sv, s);
    float w[5];
    if (W) {
        mtv(a.A, b.w, w);
#pragma unroll
        for (int i = 0; i < 5; ++i) w[i] += a.w[i];
    }
    float Ar[25], r[15], A[25];
    m_s(b.A, a.r, Ar);
    abt_sym_add(Ar, b.A, b.r, r);
    mm(b.A, a.A, A);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        c.s[i] = s[i] + b.s[i];
        c.w[i] = W ? w[i] : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < 25; ++i) c.A[i] = A[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) c.r[i] = r[i];
}

template <bool W>
PES_DEV void relem_apply(const RElem& e, const RState& d, RState& o)
{
    float u[5];
    if (W) {
        sv_sym_add(d.P, e.w, d.m, u);
    } else {
#pragma unroll
        for (int i = 0; i < 5; ++i) u[i] = d.m[i];
    }
    float m[5];
    mv(e.A, u, m);
    float AP[25], P[15];
    m_s(e.A, d.P, AP);
    abt_sym_add(AP, e.A, e.r, P);
#pragma unroll
    for (int i = 0; i < 5; ++i) o.m[i] = m[i] + e.s[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) o.P[i] = P[i];
}

}  // namespace pes
