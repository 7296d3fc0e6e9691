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

// ---- the cubature transition slope in float-float -------------------------------
//
// The sigma points are xbar +- S e_i with S = fl(scale L), the FP32 factor
// scaled in FP32 (a point set whose covariance S S^T / scale^2 differs from
// Pbar by rounding only); for that point set the regression slope is exactly
// F = (1/2) D S^{-1} with D_i = f(xbar + S e_i) - f(xbar - S e_i), which is
// formed here with every operation in float-float. The turn angles
// (w +- S_4i) dt come by angle addition from the reference angle's sine and
// cosine (float-float series after reduction) and the offsets' (series).
PES_DEV void cub_trans_slope_ff(const DevModel<float>& m, const float* xbar, const float* L, float* F)
{
    if (m.kind == MODEL_LINEAR) {
#pragma unroll
        for (int i = 0; i < 25; ++i) F[i] = m.F[i];
        return;
    }
    const float dt = m.dt;
    float S[25];
#pragma unroll
    for (int i = 0; i < 25; ++i) S[i] = __fmul_rn(m.sp_scale, L[i]);
    ff s0, c0, o0;
    ff_sincos(two_prod(xbar[4], dt), &s0, &c0, &o0);
    ff D[4][5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        ff se, ce, oe;
        ff_sincos(two_prod(S[20 + i], dt), &se, &ce, &oe);
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
            const ff w = two_sum(xbar[4], sgn * S[20 + i]);
            ff A1, A2;
            if (w.hi == 0.0f && w.lo == 0.0f) {
                A1 = ff_make(dt);
                A2 = ff_make(0.0f);
            } else {
                const ff iw = ff_rcp(w);
                A1 = ff_mul(sn, iw);
                A2 = ff_mul(om, iw);
            }
            const ff vx = two_sum(xbar[2], sgn * S[10 + i]);
            const ff vy = two_sum(xbar[3], sgn * S[15 + i]);
            // position increments and velocities of f at the point (the
            // positions themselves contribute 2 S_pi to D, added below)
            z[sg][0] = ff_sub(ff_mul(A1, vx), ff_mul(A2, vy));
            z[sg][1] = ff_add(ff_mul(A2, vx), ff_mul(A1, vy));
            z[sg][2] = ff_sub(ff_mul(cs, vx), ff_mul(sn, vy));
            z[sg][3] = ff_add(ff_mul(sn, vx), ff_mul(cs, vy));
        }
        D[0][i] = ff_add_f(ff_sub(z[0][0], z[1][0]), 2.0f * S[i]);
        D[1][i] = ff_add_f(ff_sub(z[0][1], z[1][1]), 2.0f * S[5 + i]);
        D[2][i] = ff_sub(z[0][2], z[1][2]);
        D[3][i] = ff_sub(z[0][3], z[1][3]);
    }
    // rows g of F solve g S = D_r / 2 (S lower triangular), from the last column
    ff rs[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) rs[c] = ff_rcp(ff_make(S[c * 5 + c]));
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        ff g[5];
#pragma unroll
        for (int c = 4; c >= 0; --c) {
            ff acc = ff{0.5f * D[r][c].hi, 0.5f * D[r][c].lo};
#pragma unroll
            for (int l = c + 1; l < 5; ++l) acc = ff_fma_f(g[l], -S[l * 5 + c], acc);
            g[c] = ff_mul(acc, rs[c]);
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) F[r * 5 + c] = g[c].hi;
    }
    F[20] = F[21] = F[22] = F[23] = 0.0f;
    F[24] = 1.0f;
}

// ---- residuals ---------------------------------------------------------------------

// One Kalman step in float-float from the FP32 filtered moments (m, P) of
// state k, through the transition tr (k -> k+1) and the observation ob of
// state k+1: the step's exact-arithmetic image (mf, Pf), to about 1e-14
// relative of the operands, and its derivatives Abar = (I - K H) F,
// w = F^T H^T S^{-1} v in FP32. Returns false if S is not positive definite.
PES_DEV bool ff_kalman_step(const Trans<float>& tr, const Obs<float>& ob, const float* m, const float* P, ff* mf,
                            ff* Pf, float* Abar, float* w)
{
    ff mp[5];
    {
        ff dx[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) dx[i] = ff_diff_f(m[i], tr.xn[i]);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            ff acc = ff_make(tr.fx[i]);
#pragma unroll
            for (int l = 0; l < 5; ++l) acc = ff_fma_f(dx[l], tr.F[i * 5 + l], acc);
            mp[i] = acc;
        }
    }
    ff Pp[15];
    {
        ff FP[25];
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                ff acc = two_prod(tr.F[i * 5], P[si(0, j)]);
#pragma unroll
                for (int l = 1; l < 5; ++l) acc = ff_fma_ff(tr.F[i * 5 + l], P[si(l, j)], acc);
                FP[i * 5 + j] = acc;
            }
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = i; j < 5; ++j) {
                ff acc = ff_make(tr.Q[si(i, j)]);
#pragma unroll
                for (int l = 0; l < 5; ++l) acc = ff_fma_f(FP[i * 5 + l], tr.F[j * 5 + l], acc);
                Pp[si(i, j)] = acc;
            }
    }
    ff HP[10];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            ff acc = ff_mul_f(Pp[si(0, j)], ob.H[r * 5]);
#pragma unroll
            for (int l = 1; l < 5; ++l) acc = ff_fma_f(Pp[si(l, j)], ob.H[r * 5 + l], acc);
            HP[r * 5 + j] = acc;
        }
    ff S[3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int q = r; q < 2; ++q) {
            ff acc = ff_make(ob.R[si2(r, q)]);
#pragma unroll
            for (int l = 0; l < 5; ++l) acc = ff_fma_f(HP[r * 5 + l], ob.H[q * 5 + l], acc);
            S[si2(r, q)] = acc;
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
        ff acc = ff_make(ob.r[r]);
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = ff_fma_f(ff_add_f(mp[l], -ob.xn[l]), -ob.H[r * 5 + l], acc);
        v[r] = acc;
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) mf[i] = ff_fma(KT[5 + i], v[1], ff_fma(KT[i], v[0], mp[i]));
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i; j < 5; ++j)
            Pf[si(i, j)] = ff_fma(ff_neg(KT[5 + i]), HP[5 + j], ff_fma(ff_neg(KT[i]), HP[j], Pp[si(i, j)]));
    // derivatives, FP32
    float IKH[25];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int l = 0; l < 5; ++l)
            IKH[i * 5 + l] = (i == l ? 1.0f : 0.0f) - KT[i].hi * ob.H[l] - KT[5 + i].hi * ob.H[5 + l];
    mm(IKH, tr.F, Abar);
    const float Siv0 = Si[0].hi * v[0].hi + Si[1].hi * v[1].hi;
    const float Siv1 = Si[1].hi * v[0].hi + Si[2].hi * v[1].hi;
    float hs[5];
#pragma unroll
    for (int l = 0; l < 5; ++l) hs[l] = ob.H[l] * Siv0 + ob.H[5 + l] * Siv1;
    mtv(tr.F, hs, w);
    return ok;
}

// One RTS step in float-float: from the refined filtered moments (mf, Pf) of
// state k, the transition tr out of k, and the FP32 smoothed moments
// (xs1, Ps1) of state k+1: the step's exact-arithmetic image (ms, Ps) and its
// gain G = Pf F^T (F Pf F^T + Q')^{-1} in FP32. Returns false if the predicted
// covariance is not positive definite.
PES_DEV bool ff_rts_step(const Trans<float>& tr, const ff* mf, const ff* Pf, const float* xs1, const float* Ps1,
                         ff* ms, ff* Ps, float* G)
{
    ff mp[5];
    {
        ff dx[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) dx[i] = ff_add_f(mf[i], -tr.xn[i]);
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            ff acc = ff_make(tr.fx[i]);
#pragma unroll
            for (int l = 0; l < 5; ++l) acc = ff_fma_f(dx[l], tr.F[i * 5 + l], acc);
            mp[i] = acc;
        }
    }
    // Gt = (F Pf F^T + Q')^{-1} F Pf, formed in place of F Pf
    ff Gt[25];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            ff acc = ff_mul_f(Pf[si(0, j)], tr.F[i * 5]);
#pragma unroll
            for (int l = 1; l < 5; ++l) acc = ff_fma_f(Pf[si(l, j)], tr.F[i * 5 + l], acc);
            Gt[i * 5 + j] = acc;
        }
    ff Pp[15];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i; j < 5; ++j) {
            ff acc = ff_make(tr.Q[si(i, j)]);
#pragma unroll
            for (int l = 0; l < 5; ++l) acc = ff_fma_f(Gt[i * 5 + l], tr.F[j * 5 + l], acc);
            Pp[si(i, j)] = acc;
        }
    // Cholesky Pp = C C^T (C lower, packed by rows into Pp's slots) with
    // reciprocal diagonal rd
    ff C[15], rd[5];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        ff sjj = Pp[si(j, j)];
#pragma unroll
        for (int l = 0; l < j; ++l) sjj = ff_fma(ff_neg(C[si(j, l)]), C[si(j, l)], sjj);
        ok = ok && sjj.hi > 0.0f;
        const ff d = ff_sqrt(sjj.hi > 0.0f ? sjj : ff_make(1.0f));
        C[si(j, j)] = d;
        rd[j] = ff_rcp(d);
#pragma unroll
        for (int i = j + 1; i < 5; ++i) {
            ff t = Pp[si(i, j)];
#pragma unroll
            for (int l = 0; l < j; ++l) t = ff_fma(ff_neg(C[si(i, l)]), C[si(j, l)], t);
            C[si(i, j)] = ff_mul(t, rd[j]);
        }
    }
    // solve C C^T X = Gt column by column
#pragma unroll
    for (int c = 0; c < 5; ++c) {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            ff t = Gt[i * 5 + c];
#pragma unroll
            for (int l = 0; l < i; ++l) t = ff_fma(ff_neg(C[si(i, l)]), Gt[l * 5 + c], t);
            Gt[i * 5 + c] = ff_mul(t, rd[i]);
        }
#pragma unroll
        for (int i = 4; i >= 0; --i) {
            ff t = Gt[i * 5 + c];
#pragma unroll
            for (int l = i + 1; l < 5; ++l) t = ff_fma(ff_neg(C[si(l, i)]), Gt[l * 5 + c], t);
            Gt[i * 5 + c] = ff_mul(t, rd[i]);
        }
    }
    // G_ij = Gt_ji
    ff e[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) e[j] = ff_add_f(ff_neg(mp[j]), xs1[j]);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        ff acc = mf[i];
#pragma unroll
        for (int j = 0; j < 5; ++j) acc = ff_fma(Gt[j * 5 + i], e[j], acc);
        ms[i] = acc;
    }
    // Ps = Pf + G (Ps1 - Pp) G^T, one row of G (Ps1 - Pp) at a time
    ff dP[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) dP[i] = ff_add_f(ff_neg(Pp[i]), Ps1[i]);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        ff row[5];
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            ff acc = ff_mul(Gt[i], dP[si(0, j)]);
#pragma unroll
            for (int l = 1; l < 5; ++l) acc = ff_fma(Gt[l * 5 + i], dP[si(l, j)], acc);
            row[j] = acc;
        }
#pragma unroll
        for (int j = i; j < 5; ++j) {
            ff acc = Pf[si(i, j)];
#pragma unroll
            for (int l = 0; l < 5; ++l) acc = ff_fma(row[l], Gt[l * 5 + j], acc);
            Ps[si(i, j)] = acc;
        }
    }
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) G[i * 5 + j] = Gt[j * 5 + i].hi;
    return ok;
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
