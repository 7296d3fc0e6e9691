// Filtering and smoothing elements and their associative operators (Sec. 4).
//
// Filtering element (Eqs. 12-14): the conditional density
//   p(x_k | y, x_in) = N(A (x_in - xr) + b, C)
// and the likelihood of the data given the input state in information form,
//   p(y | x_in) ∝ exp(-1/2 d^T J d + eta^T d),  d = x_in - xr.
// The input is measured from a reference point xr (the nominal state the
// element starts from); with xr = 0 this is exactly the paper's (A, b, C, eta, J).
//
// Smoothing element (Eqs. 16-18): p(x_k | y_{1:k}, x_next) = N(E (x_next - xr) + g, L).
//
// Operators: Eq. 15 (filtering) and Eq. 19 (smoothing). Eq. 15 is evaluated
// through the symmetric matrix D = (I + C_i J_j)^{-1} C_i = (C_i^{-1} + J_j)^{-1}
// (see info_update_cov), using (I + C_i J_j)^{-1} = I - D J_j and
// (I + J_j C_i)^{-1} = I - J_j D.
#pragma once

#include "pes_model.cuh"

namespace pes {

template <typename T>
struct FElem {
    T A[25];
    T b[5];
    T C[15];
    T eta[5];
    T J[15];
    T xr[5];
};

template <typename T>
struct SElem {
    T E[25];
    T g[5];
    T L[15];
    T xr[5];
};

template <typename T>
struct Gauss {
    T m[5];
    T P[15];
};

// Identity of Eq. 15 with input reference xr: (A = I, b = xr, C = 0, eta = 0, J = 0).
template <typename T>
PES_DEV void felem_identity(FElem<T>& a, const T* xr)
{
    set_identity(a.A);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        a.b[i] = xr[i];
        a.eta[i] = T(0);
        a.xr[i] = xr[i];
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) {
        a.C[i] = T(0);
        a.J[i] = T(0);
    }
}

// The Levenberg-Marquardt damping of state k as a filtering element: the
// pseudo-measurement xbar = x_k + e, e ~ N(0, I / lambda), through an identity
// transition, about the reference xr = xbar: A = I, b = xbar, C = 0, eta = 0,
// J = lambda I. acc (x) damping adds the damping to the state acc ends at.
template <typename T>
PES_DEV void felem_damping(FElem<T>& a, const T* xbar, T lambda)
{
    set_identity(a.A);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        a.b[i] = xbar[i];
        a.eta[i] = T(0);
        a.xr[i] = xbar[i];
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) {
        a.C[i] = T(0);
        a.J[i] = T(0);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) a.J[si(i, i)] = lambda;
}

// a (x) a_0 where a_0 is the prior element (A = 0, b = m0, C = P0, eta = J = 0):
// the conditional density forgets its input; the likelihood stays.
template <typename T>
PES_DEV void felem_apply_prior(FElem<T>& a, const T* m0, const T* P0)
{
#pragma unroll
    for (int i = 0; i < 25; ++i) a.A[i] = T(0);
#pragma unroll
    for (int i = 0; i < 5; ++i) a.b[i] = m0[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) a.C[i] = P0[i];
}

// acc <- acc (x) a_k for the single-step element a_k of Eqs. 13-14 built from
// the transition (k-1 -> k) and the observation at k.
//
// a_k's J_k = G^T S^{-1} G has rank n_y, so the Woodbury identity turns the
// 5x5 inverse (I + C J_k)^{-1} of Eq. 15 into the 2x2 S^{-1}: the product is a
// Kalman predict + update of the affine conditional acc. Predict
//   A- = F A,  b- = fx + F (b - xn),  C- = F C F^T + Q',
// update with S = H C- H^T + R', K = C- H^T S^{-1}, G = H A-, v = r - H (b- - xn_k):
//   A = A- - K G,  b = b- + K v,  C = C- - K H C-,
// and the likelihood of y_k given the input accumulates
//   J += G^T S^{-1} G,  eta += G^T S^{-1} v.
// The two halves of fold_filter_step: the prediction through the transition,
// after which a describes x_k given the input, then the update with the
// observation at k. Folding them separately keeps the transition and the
// observation from being live together.
template <typename T>
PES_DEV void fold_predict(FElem<T>& a, const Trans<T>& tr)
{
    T Am[25];
    mm(tr.F, a.A, Am);
    T dv[5], bm[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) dv[i] = a.b[i] - tr.xn[i];
    mv(tr.F, dv, bm);
#pragma unroll
    for (int i = 0; i < 5; ++i) bm[i] += tr.fx[i];
    T FC[25], Cm[15];
    m_s(tr.F, a.C, FC);
    abt_sym_add(FC, tr.F, tr.Q, Cm);
#pragma unroll
    for (int i = 0; i < 25; ++i) a.A[i] = Am[i];
#pragma unroll
    for (int i = 0; i < 5; ++i) a.b[i] = bm[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) a.C[i] = Cm[i];
}

template <typename T>
PES_DEV bool fold_update(FElem<T>& a, const Obs<T>& ob)
{
    const T* Am = a.A;
    const T* bm = a.b;
    const T* Cm = a.C;
    // H C-
    T HC[10];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            T s = ob.H[r * 5] * Cm[si(0, j)];
#pragma unroll
            for (int l = 1; l < 5; ++l) s = fma(ob.H[r * 5 + l], Cm[si(l, j)], s);
            HC[r * 5 + j] = s;
        }
    T S[3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int q = r; q < 2; ++q) {
            T s = ob.R[si2(r, q)];
#pragma unroll
            for (int l = 0; l < 5; ++l) s = fma(HC[r * 5 + l], ob.H[q * 5 + l], s);
            S[si2(r, q)] = s;
        }
    T Si[3];
    const bool ok = inv2_spd(S, Si);
    // K^T = S^{-1} H C-,  G = H A-,  v
    T KT[10], G[10], v[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            KT[r * 5 + j] = Si[si2(r, 0)] * HC[j] + Si[si2(r, 1)] * HC[5 + j];
            T s = ob.H[r * 5] * Am[j];
#pragma unroll
            for (int l = 1; l < 5; ++l) s = fma(ob.H[r * 5 + l], Am[l * 5 + j], s);
            G[r * 5 + j] = s;
        }
        T hv = ob.r[r];
#pragma unroll
        for (int l = 0; l < 5; ++l) hv = fma(-ob.H[r * 5 + l], bm[l] - ob.xn[l], hv);
        v[r] = hv;
    }
    T Anew[25], bnew[5], Cnew[15];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
#pragma unroll
        for (int j = 0; j < 5; ++j)
            Anew[i * 5 + j] = fma(-KT[5 + i], G[5 + j], fma(-KT[i], G[j], Am[i * 5 + j]));
        bnew[i] = fma(KT[5 + i], v[1], fma(KT[i], v[0], bm[i]));
    }
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i; j < 5; ++j)
            Cnew[si(i, j)] = fma(-KT[5 + i], HC[5 + j], fma(-KT[i], HC[j], Cm[si(i, j)]));
#pragma unroll
    for (int i = 0; i < 25; ++i) a.A[i] = Anew[i];
#pragma unroll
    for (int i = 0; i < 5; ++i) a.b[i] = bnew[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) a.C[i] = Cnew[i];
    // likelihood of y_k given the input
    T SiG[10], Siv[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
#pragma unroll
        for (int j = 0; j < 5; ++j) SiG[r * 5 + j] = Si[si2(r, 0)] * G[j] + Si[si2(r, 1)] * G[5 + j];
        Siv[r] = Si[si2(r, 0)] * v[0] + Si[si2(r, 1)] * v[1];
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
#pragma unroll
        for (int j = i; j < 5; ++j)
            a.J[si(i, j)] = fma(G[5 + i], SiG[5 + j], fma(G[i], SiG[j], a.J[si(i, j)]));
        a.eta[i] = fma(G[5 + i], Siv[1], fma(G[i], Siv[0], a.eta[i]));
    }
    return ok;
}

template <typename T>
PES_DEV bool fold_filter_step(FElem<T>& a, const Trans<T>& tr, const Obs<T>& ob)
{
    fold_predict(a, tr);
    return fold_update(a, ob);
}

// out = ai (x) aj, Eq. 15 (ai earlier in time). aj's input reference is the
// point where ai's output is measured from.
template <typename T>
PES_DEV void combine_filter(const FElem<T>& ai, const FElem<T>& aj, FElem<T>& out)
{
    T bt[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) bt[i] = ai.b[i] - aj.xr[i];
    T D[15];
    info_update_cov(ai.C, aj.J, D);
    T AD[25];
    m_s(aj.A, D, AD);
    // W = A_j (I + C_i J_j)^{-1} = A_j - (A_j D) J_j
    T W[25];
    m_s(AD, aj.J, W);
#pragma unroll
    for (int i = 0; i < 25; ++i) W[i] = aj.A[i] - W[i];
    // mean: A_j (I + C_i J_j)^{-1} (bt + C_i eta_j) + b_j = A_j (bt + D u) + b_j, u = eta_j - J_j bt
    T u[5], Du[5], w[5], Aw[5];
    sv(aj.J, bt, u);
#pragma unroll
    for (int i = 0; i < 5; ++i) u[i] = aj.eta[i] - u[i];
    sv(D, u, Du);
#pragma unroll
    for (int i = 0; i < 5; ++i) w[i] = bt[i] + Du[i];
    mv(aj.A, w, Aw);
    // likelihood: A_i^T (I - J_j D) u + eta_i
    T JDu[5], z[5], Az[5];
    sv(aj.J, Du, JDu);
#pragma unroll
    for (int i = 0; i < 5; ++i) z[i] = u[i] - JDu[i];
    mtv(ai.A, z, Az);
    // K2 = J_j - J_j D J_j
    T JD[25], K2[15];
    {
        T Df[25];
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j < 5; ++j) Df[i * 5 + j] = D[si(i, j)];
        s_m(aj.J, Df, JD);
    }
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i; j < 5; ++j) {
            T s = aj.J[si(i, j)];
#pragma unroll
            for (int l = 0; l < 5; ++l) s = fma(-JD[i * 5 + l], aj.J[si(l, j)], s);
            K2[si(i, j)] = s;
        }
    T K2A[25];
    {
        T K2f[25];
#pragma unroll
        for (int i = 0; i < 5; ++i)
#pragma unroll
            for (int j = 0; j < 5; ++j) K2f[i * 5 + j] = K2[si(i, j)];
        mm(K2f, ai.A, K2A);
    }
    // outputs are written last, so out may alias either input
    T Anew[25];
    mm(W, ai.A, Anew);
    T Cnew[15];
    abt_sym_add(AD, aj.A, aj.C, Cnew);
    T Jnew[15];
    atb_sym_add(ai.A, K2A, ai.J, Jnew);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        out.b[i] = Aw[i] + aj.b[i];
        out.eta[i] = Az[i] + ai.eta[i];
        out.xr[i] = ai.xr[i];
    }
#pragma unroll
    for (int i = 0; i < 25; ++i) out.A[i] = Anew[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) {
        out.C[i] = Cnew[i];
        out.J[i] = Jnew[i];
    }
}

// (m, P) (x) a: a Gaussian state before a's span, pushed through a. This is
// Eq. 15 with a left operand whose A, eta, J vanish (a filtering prefix that
// starts at a prior element): the Gaussian is conditioned on a's likelihood,
// D = (P^{-1} + J)^{-1}, mean m + D (eta - J m), then mapped by (A, b, C).
template <typename T>
PES_DEV void apply_filter(const Gauss<T>& g, const FElem<T>& a, Gauss<T>& out)
{
    T dm[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) dm[i] = g.m[i] - a.xr[i];
    T D[15];
    info_update_cov(g.P, a.J, D);
    T u[5], Du[5], w[5], Aw[5];
    sv(a.J, dm, u);
#pragma unroll
    for (int i = 0; i < 5; ++i) u[i] = a.eta[i] - u[i];
    sv(D, u, Du);
#pragma unroll
    for (int i = 0; i < 5; ++i) w[i] = dm[i] + Du[i];
    mv(a.A, w, Aw);
    T AD[25];
    m_s(a.A, D, AD);
    T Pn[15];
    abt_sym_add(AD, a.A, a.C, Pn);
#pragma unroll
    for (int i = 0; i < 5; ++i) out.m[i] = Aw[i] + a.b[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) out.P[i] = Pn[i];
}

// ---- smoothing --------------------------------------------------------------------

template <typename T>
PES_DEV void selem_identity(SElem<T>& a)
{
    set_identity(a.E);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        a.g[i] = T(0);
        a.xr[i] = T(0);
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) a.L[i] = T(0);
}

// Eq. 18: the last state of a trajectory, E = 0, g = x*, L = P*.
template <typename T>
PES_DEV void selem_last(SElem<T>& a, const T* xf, const T* Pf)
{
#pragma unroll
    for (int i = 0; i < 25; ++i) a.E[i] = T(0);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        a.g[i] = xf[i];
        a.xr[i] = T(0);
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) a.L[i] = Pf[i];
}

// Eq. 17 from the predicted moments of x_{k+1}: FP = F_k P*_k, Pp = FP F^T + Q'_k,
// mp = F-prediction of x*_k:
//   E = P* F^T Pp^{-1},  L = P* - E F P*,
// and g = x*_k - E mp is kept as (g = x*_k, xr = mp), i.e. the element maps
// x_{k+1} to E (x_{k+1} - mp) + x*_k.
template <typename T>
PES_DEV bool selem_from_prediction(const T* xf, const T* Pf, const T* FP, const T* Pp, const T* mp, SElem<T>& a)
{
    T Lc[25], rd[5];
    const bool ok = chol_pd(Pp, Lc, rd);
    T Et[25];
#pragma unroll
    for (int i = 0; i < 25; ++i) Et[i] = FP[i];
    chol_solve_cols(Lc, rd, Et);   // Et = Pp^{-1} F P* = E^T
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j < 5; ++j) a.E[i * 5 + j] = Et[j * 5 + i];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i; j < 5; ++j) {
            T s = Pf[si(i, j)];
#pragma unroll
            for (int l = 0; l < 5; ++l) s = fma(-Et[l * 5 + i], FP[l * 5 + j], s);
            a.L[si(i, j)] = s;
        }
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        a.g[i] = xf[i];
        a.xr[i] = mp[i];
    }
    return ok;
}

// Predicted moments of the transition tr applied to (m, P): mp, FP = F P, Pp.
template <typename T>
PES_DEV void predict(const Trans<T>& tr, const T* m, const T* P, T* mp, T* FP, T* Pp)
{
    T dx[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) dx[i] = m[i] - tr.xn[i];
    mv(tr.F, dx, mp);
#pragma unroll
    for (int i = 0; i < 5; ++i) mp[i] += tr.fx[i];
    m_s(tr.F, P, FP);
    abt_sym_add(FP, tr.F, tr.Q, Pp);
}

// Kalman update of (mp, Pp) with the observation ob: (m, P).
template <typename T>
PES_DEV bool kf_update(const Obs<T>& ob, const T* mp, const T* Pp, T* m, T* P, double* loglik_term = nullptr)
{
    T HP[10];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            T s = ob.H[r * 5] * Pp[si(0, j)];
#pragma unroll
            for (int l = 1; l < 5; ++l) s = fma(ob.H[r * 5 + l], Pp[si(l, j)], s);
            HP[r * 5 + j] = s;
        }
    T S[3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int q = r; q < 2; ++q) {
            T s = ob.R[si2(r, q)];
#pragma unroll
            for (int l = 0; l < 5; ++l) s = fma(HP[r * 5 + l], ob.H[q * 5 + l], s);
            S[si2(r, q)] = s;
        }
    T Si[3];
    const bool ok = inv2_spd(S, Si);
    T KT[10], v[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
#pragma unroll
        for (int j = 0; j < 5; ++j) KT[r * 5 + j] = Si[si2(r, 0)] * HP[j] + Si[si2(r, 1)] * HP[5 + j];
        T hv = ob.r[r];
#pragma unroll
        for (int l = 0; l < 5; ++l) hv = fma(-ob.H[r * 5 + l], mp[l] - ob.xn[l], hv);
        v[r] = hv;
    }
    if (loglik_term) {
        // log N(v; 0, S): the term of step k in log p(y_{1:T}) = sum_k log p(y_k | y_{1:k-1})
        const double s00 = S[si2(0, 0)], s01 = S[si2(0, 1)], s11 = S[si2(1, 1)];
        const double det = s00 * s11 - s01 * s01;
        const double v0 = v[0], v1 = v[1];
        const double q = (s11 * v0 * v0 - 2.0 * s01 * v0 * v1 + s00 * v1 * v1) / det;
        *loglik_term = -0.5 * (q + log(det)) - 1.8378770664093454836;   // log(2 pi)
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) m[i] = fma(KT[5 + i], v[1], fma(KT[i], v[0], mp[i]));
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = i; j < 5; ++j)
            P[si(i, j)] = fma(-KT[5 + i], HP[5 + j], fma(-KT[i], HP[j], Pp[si(i, j)]));
    return ok;
}

// out = ai (x) aj, Eq. 19 (ai earlier in time):
// E = E_i E_j, g = E_i (g_j - xr_i) + g_i, L = E_i L_j E_i^T + L_i, xr = xr_j.
template <typename T>
PES_DEV void combine_smoother(const SElem<T>& ai, const SElem<T>& aj, SElem<T>& out)
{
    T dg[5], Eg[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) dg[i] = aj.g[i] - ai.xr[i];
    mv(ai.E, dg, Eg);
    T EL[25];
    m_s(ai.E, aj.L, EL);
    T Ln[15];
    abt_sym_add(EL, ai.E, ai.L, Ln);
    T En[25];
    mm(ai.E, aj.E, En);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        out.g[i] = Eg[i] + ai.g[i];
        out.xr[i] = aj.xr[i];
    }
#pragma unroll
    for (int i = 0; i < 25; ++i) out.E[i] = En[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) out.L[i] = Ln[i];
}

// a (x) (m, P): the smoothing distribution of the state after a's span pushed
// back through a: m' = E (m - xr) + g, P' = E P E^T + L.
template <typename T>
PES_DEV void apply_smoother(const SElem<T>& a, const Gauss<T>& g, Gauss<T>& out)
{
    T dm[5], Em[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) dm[i] = g.m[i] - a.xr[i];
    mv(a.E, dm, Em);
    T EP[25];
    m_s(a.E, g.P, EP);
    T Pn[15];
    abt_sym_add(EP, a.E, a.L, Pn);
#pragma unroll
    for (int i = 0; i < 5; ++i) out.m[i] = Em[i] + a.g[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) out.P[i] = Pn[i];
}

}  // namespace pes
