// State-space model (Eq. 4) and its linearisation (Eqs. 7-10) on the device.
//
// Model: coordinated turn, x = [px, py, vx, vy, omega], with bearings from two
// sensors (the experiment of Sec. 5), or a linear-Gaussian model.
//
// Linearisations are kept *about the nominal*: the affine approximation
// f(x) ~ F x + c of Eq. 5 is stored as f(x) ~ fx + F (x - xn) with xn the
// nominal state, fx = F xn + c; likewise h(x) ~ hx + H (x - xn) with the
// measurement residual r = y - hx. This is the same affine map; it keeps
// single precision accurate when states are large (positions of thousands
// of units) because c = f(xn) - F xn cancels there.
#pragma once

#include "pes_math.cuh"

namespace pes {

enum { MODEL_CT_BEARINGS = 0, MODEL_LINEAR = 1 };
enum { LIN_ARRAYS = 0, LIN_IEKS = 1, LIN_CUBATURE = 2, LIN_GH = 3 };

// Linearisations by statistical linear regression over sigma points (Eqs. 7-9),
// which need the nominal covariance and its factor.
template <int LIN>
constexpr bool kSigma = (LIN == LIN_CUBATURE || LIN == LIN_GH);
enum { ST_NOT_PD = 1, ST_NONFINITE = 2, ST_TIMEOUT = 4, ST_NOT_CONVERGED = 8, ST_BADARG = 16 };

// Model parameters as passed to the kernels, already in the kernel's
// precision (no conversions on the device). Q and R are packed (upper).
template <typename T>
struct DevModel {
    int kind;
    int sensors_per_traj;
    T dt;
    const T* sensors;   // device, [1 or B][4]
    T Q[15];
    T R[3];
    T F[25], c[5], H[10], d[2];   // linear model
    // sigma-point rule of the regression (Eqs. 7-9) over symmetric points
    // xbar +- sp_scale chol(Pbar) e_i: sp_w = 1 / sp_scale^2 is twice a side
    // point's weight, sp_w0c the centre's covariance weight (cubature:
    // sqrt(n), 1/n, 0)
    T sp_scale, sp_w, sp_w0c;
    T lm;   // Levenberg-Marquardt damping lambda (0: none)
    const T* lm_traj;   // per-trajectory damping [B] (device), overriding lm; or NULL
};

// The Levenberg-Marquardt damping of trajectory b.
template <typename T>
PES_DEV T lm_of(const DevModel<T>& m, int b)
{
    return m.lm_traj ? __ldg(m.lm_traj + b) : m.lm;
}

// Transition k -> k+1 linearised about xn = xbar_k: x_{k+1} ~ fx + F (x_k - xn) + N(0, Q')
template <typename T>
struct Trans {
    T F[25];
    T fx[5];
    T xn[5];
    T Q[15];
};

// Observation at k linearised about xn = xbar_k: y_k - hx ~ r-form, i.e. the
// innovation of a state x is  r - H (x - xn),  noise N(0, R')
template <typename T>
struct Obs {
    T H[10];
    T xn[5];
    T r[2];
    T R[3];
};

template <typename T> PES_DEV void tsincos(T a, T* s, T* c);
template <> PES_DEV void tsincos<float>(float a, float* s, float* c) { sincosf(a, s, c); }
template <> PES_DEV void tsincos<double>(double a, double* s, double* c) { sincos(a, s, c); }
template <typename T> PES_DEV T tatan2(T y, T x);
template <> PES_DEV float tatan2<float>(float y, float x) { return atan2f(y, x); }
template <> PES_DEV double tatan2<double>(double y, double x) { return atan2(y, x); }
template <typename T> PES_DEV T tfloor(T x);
template <> PES_DEV float tfloor<float>(float x) { return floorf(x); }
template <> PES_DEV double tfloor<double>(double x) { return floor(x); }

template <typename T>
PES_DEV T wrap_angle(T a)
{
    const T pi = T(3.14159265358979323846);
    const T two_pi = T(6.28318530717958647692);
    return a - two_pi * tfloor((a + pi) / two_pi);
}

// ---- coordinated turn --------------------------------------------------------
// With a = omega dt:  A1 = sin(a)/omega,  A2 = (1 - cos a)/omega  and their
// omega-derivatives. Below |a| < thr their Taylor series in a are used.
template <typename T>
struct CTCoef {
    T s, c, A1, A2, dA1, dA2;
};

template <typename T>
PES_DEV CTCoef<T> ct_coef(T w, T dt)
{
    CTCoef<T> k;
    const T a = w * dt;
    tsincos(a, &k.s, &k.c);
    const T thr = sizeof(T) == 4 ? T(0.05) : T(0.01);
    if (fabs(a) < thr) {
        const T a2 = a * a;
        k.A1 = dt * (T(1) - a2 * (T(1) / T(6)) + a2 * a2 * (T(1) / T(120)));
        k.A2 = dt * a * (T(0.5) - a2 * (T(1) / T(24)) + a2 * a2 * (T(1) / T(720)));
        k.dA1 = dt * dt * a * (-T(1) / T(3) + a2 * (T(1) / T(30)) - a2 * a2 * (T(1) / T(840)));
        k.dA2 = dt * dt * (T(0.5) - a2 * T(0.125) + a2 * a2 * (T(1) / T(144)));
    } else {
        // 1 - cos a without cancellation for cos a > 0
        const T omc = (k.c > T(0)) ? k.s * k.s * trcp(T(1) + k.c) : T(1) - k.c;
        const T iw = trcp(w);
        k.A1 = k.s * iw;
        k.A2 = omc * iw;
        k.dA1 = (a * k.c - k.s) * iw * iw;
        k.dA2 = (a * k.s - omc) * iw * iw;
    }
    return k;
}

// f(x) split as position increment and the rest:
//   out = [A1 vx - A2 vy, A2 vx + A1 vy, c vx - s vy, s vx + c vy, omega]
// so that f(x) = out + [px, py, 0, 0, 0].
template <typename T>
PES_DEV void ct_increment(const T* x, const CTCoef<T>& k, T* out)
{
    out[0] = k.A1 * x[2] - k.A2 * x[3];
    out[1] = k.A2 * x[2] + k.A1 * x[3];
    out[2] = k.c * x[2] - k.s * x[3];
    out[3] = k.s * x[2] + k.c * x[3];
    out[4] = x[4];
}

template <typename T>
PES_DEV void ct_jacobian(const T* x, const CTCoef<T>& k, T dt, T* F)
{
#pragma unroll
    for (int i = 0; i < 25; ++i) F[i] = T(0);
    F[0] = T(1);
    F[2] = k.A1;
    F[3] = -k.A2;
    F[4] = k.dA1 * x[2] - k.dA2 * x[3];
    F[6] = T(1);
    F[7] = k.A2;
    F[8] = k.A1;
    F[9] = k.dA2 * x[2] + k.dA1 * x[3];
    F[12] = k.c;
    F[13] = -k.s;
    F[14] = -dt * (k.s * x[2] + k.c * x[3]);
    F[17] = k.s;
    F[18] = k.c;
    F[19] = dt * (k.c * x[2] - k.s * x[3]);
    F[24] = T(1);
}

template <typename T>
PES_DEV void load_sensors(const DevModel<T>& m, int b, T* s)
{
    const T* p = m.sensors + (m.sensors_per_traj ? 4 * b : 0);
#pragma unroll
    for (int i = 0; i < 4; ++i) s[i] = __ldg(p + i);
}

template <typename T>
PES_DEV void bearings(const T* x, const T* s, T* out)
{
    out[0] = tatan2(x[1] - s[1], x[0] - s[0]);
    out[1] = tatan2(x[1] - s[3], x[0] - s[2]);
}

template <typename T>
PES_DEV void bearings_jacobian(const T* x, const T* s, T* H)
{
#pragma unroll
    for (int i = 0; i < 10; ++i) H[i] = T(0);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const T dx = x[0] - s[2 * r], dy = x[1] - s[2 * r + 1];
        const T ir2 = trcp(dx * dx + dy * dy);
        H[r * 5 + 0] = -dy * ir2;
        H[r * 5 + 1] = dx * ir2;
    }
}

// ---- Taylor linearisation (IEKS, Eq. 10) ---------------------------------------

template <typename T>
PES_DEV void lin_trans_taylor(const DevModel<T>& m, const T* xn, Trans<T>& tr)
{
#pragma unroll
    for (int i = 0; i < 5; ++i) tr.xn[i] = xn[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) tr.Q[i] = m.Q[i];
    if (m.kind == MODEL_LINEAR) {
#pragma unroll
        for (int i = 0; i < 25; ++i) tr.F[i] = m.F[i];
        T Fx[5];
        mv(tr.F, xn, Fx);
#pragma unroll
        for (int i = 0; i < 5; ++i) tr.fx[i] = Fx[i] + m.c[i];
    } else {
        const T dt = m.dt;
        const CTCoef<T> k = ct_coef(xn[4], dt);
        ct_jacobian(xn, k, dt, tr.F);
        T inc[5];
        ct_increment(xn, k, inc);
        tr.fx[0] = xn[0] + inc[0];
        tr.fx[1] = xn[1] + inc[1];
        tr.fx[2] = inc[2];
        tr.fx[3] = inc[3];
        tr.fx[4] = inc[4];
    }
}

template <typename T>
PES_DEV void lin_obs_taylor(const DevModel<T>& m, int b, const T* xn, const T* y, Obs<T>& ob)
{
#pragma unroll
    for (int i = 0; i < 5; ++i) ob.xn[i] = xn[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) ob.R[i] = m.R[i];
    if (m.kind == MODEL_LINEAR) {
#pragma unroll
        for (int i = 0; i < 10; ++i) ob.H[i] = m.H[i];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            T hx = m.d[r];
#pragma unroll
            for (int l = 0; l < 5; ++l) hx = fma(ob.H[r * 5 + l], xn[l], hx);
            ob.r[r] = y[r] - hx;
        }
    } else {
        T s[4];
        load_sensors(m, b, s);
        bearings_jacobian(xn, s, ob.H);
        T hx[2];
        bearings(xn, s, hx);
        ob.r[0] = wrap_angle(y[0] - hx[0]);
        ob.r[1] = wrap_angle(y[1] - hx[1]);
    }
}

// ---- cubature statistical linear regression (IPLS, Eqs. 7-9) -------------------
//
// Sigma points X_{i+-} = xbar +- sqrt(n) L e_i (P = L L^T, weights 1/(2n)).
// With D_i = Z_{i+} - Z_{i-} and u_i = (Z_{i+} + Z_{i-})/2 - zbar, the moments of
// Eq. 8 give, exactly for this symmetric point set,
//     F = Psi^T P^{-1} = D L^{-1} / (2 sqrt(n)),     Lambda = Phi - F P F^T = (1/n) sum_i u_i u_i^T,
// the second being positive semi-definite by construction. Deviations
// Z - f(xbar) are formed directly (position increments, wrapped bearings).

// Deviations of the transition for the pair of sigma points xbar +- sg:
// zp = f(xbar + sg) - f(xbar), zm = f(xbar - sg) - f(xbar). For the
// coordinated turn the two turn angles a +- d (a = omega dt, d = sg_omega dt)
// come from one sincos of d by angle addition with the reference's (s, c);
// 1 - cos is formed without cancellation. inc_ref = f(xbar) - [px, py, 0, 0, 0].
template <typename T>
PES_DEV void dev_f_pair(const DevModel<T>& m, const T* xbar, const CTCoef<T>& kr, const T* inc_ref, const T* sg,
                        T* zp, T* zm)
{
    if (m.kind == MODEL_LINEAR) {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            T s = T(0);
#pragma unroll
            for (int l = 0; l < 5; ++l) s = fma(m.F[i * 5 + l], sg[l], s);
            zp[i] = s;
            zm[i] = -s;
        }
        return;
    }
    const T dt = m.dt;
    const T thr = sizeof(T) == 4 ? T(0.05) : T(0.01);
    // the turn-angle offset d = sg_omega dt of a sigma point is small: below
    // 0.05 its sine and 1 - cos by their Taylor series through d^7 and d^8
    // (remainders below d^9/9! < 6e-18), else by sincos
    T sd, cd, omcd;
    const T d = sg[4] * dt;
    if (fabs(d) < T(0.05)) {
        const T d2 = d * d;
        sd = d * (T(1) - d2 * (T(1) / T(6)) * (T(1) - d2 * (T(1) / T(20)) * (T(1) - d2 * (T(1) / T(42)))));
        omcd = d2 * T(0.5) * (T(1) - d2 * (T(1) / T(12)) * (T(1) - d2 * (T(1) / T(30)) * (T(1) - d2 * (T(1) / T(56)))));
        cd = T(1) - omcd;
    } else {
        tsincos(d, &sd, &cd);
        omcd = sd * sd * trcp(T(1) + cd);
    }
    const T omcr = (kr.c > T(0)) ? kr.s * kr.s * trcp(T(1) + kr.c) : T(1) - kr.c;
#pragma unroll
    for (int sign = 0; sign < 2; ++sign) {
        const T sgn = sign == 0 ? T(1) : T(-1);
        const T w = xbar[4] + sgn * sg[4];
        const T a = w * dt;
        const T s = kr.s * cd + sgn * kr.c * sd;
        const T c = kr.c * cd - sgn * kr.s * sd;
        T A1, A2;
        if (fabs(a) < thr) {
            const T a2 = a * a;
            A1 = dt * (T(1) - a2 * (T(1) / T(6)) + a2 * a2 * (T(1) / T(120)));
            A2 = dt * a * (T(0.5) - a2 * (T(1) / T(24)) + a2 * a2 * (T(1) / T(720)));
        } else {
            const T omc = omcr + kr.c * omcd + sgn * kr.s * sd;
            const T iw = trcp(w);
            A1 = s * iw;
            A2 = omc * iw;
        }
        const T vx = xbar[2] + sgn * sg[2], vy = xbar[3] + sgn * sg[3];
        T* z = sign == 0 ? zp : zm;
        z[0] = sgn * sg[0] + ((A1 * vx - A2 * vy) - inc_ref[0]);
        z[1] = sgn * sg[1] + ((A2 * vx + A1 * vy) - inc_ref[1]);
        z[2] = (c * vx - s * vy) - inc_ref[2];
        z[3] = (s * vx + c * vy) - inc_ref[3];
        z[4] = sgn * sg[4];
    }
}

// Deviation of the observation for the pair xbar +- sg. For bearings the angle
// from the reference direction r = p - s to r +- sg_p is
// atan2(+-(r x sg_p), |r|^2 +- r . sg_p): already the branch nearest h(xbar),
// and free of cancellation for small deviations.
template <typename T>
PES_DEV void dev_h_pair(const DevModel<T>& m, const T* xbar, const T* s, const T* sg, T* zp, T* zm)
{
    if (m.kind == MODEL_LINEAR) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            T v = T(0);
#pragma unroll
            for (int l = 0; l < 5; ++l) v = fma(m.H[r * 5 + l], sg[l], v);
            zp[r] = v;
            zm[r] = -v;
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const T rx = xbar[0] - s[2 * r], ry = xbar[1] - s[2 * r + 1];
        const T cross = rx * sg[1] - ry * sg[0];
        const T rr = rx * rx + ry * ry;
        const T rs = rx * sg[0] + ry * sg[1];
        zp[r] = tatan2(cross, rr + rs);
        zm[r] = tatan2(-cross, rr - rs);
    }
}

// Solve G L = Dsc (row vectors) for G: each row g satisfies sum_{l>=c} g_l L_{lc} = Dsc_c.
template <typename T, int NZ>
PES_DEV void solve_rows_lower_t(const T* L, const T* rdiag, const T* Dsc, T* G)
{
#pragma unroll
    for (int r = 0; r < NZ; ++r)
#pragma unroll
        for (int c = NX - 1; c >= 0; --c) {
            T s = Dsc[r * NX + c];
#pragma unroll
            for (int l = c + 1; l < NX; ++l) s = fma(-G[r * NX + l], L[l * NX + c], s);
            G[r * NX + c] = s * rdiag[c];
        }
}

// Cubature factor of Pbar; false if Pbar is not positive definite.
template <typename T>
PES_DEV bool cub_factor(const T* Pbar, T* L, T* rdiag)
{
    return chol_pd(Pbar, L, rdiag);
}

template <typename T>
PES_DEV void lin_trans_cubature(const DevModel<T>& m, const T* xbar, const T* L, const T* rdiag, Trans<T>& tr)
{
    const T sq = m.sp_scale;
    T inc_ref[5];
    CTCoef<T> kr;
    if (m.kind == MODEL_LINEAR) {
#pragma unroll
        for (int i = 0; i < 5; ++i) inc_ref[i] = T(0);
        kr.s = kr.c = kr.A1 = kr.A2 = kr.dA1 = kr.dA2 = T(0);
    } else {
        kr = ct_coef(xbar[4], m.dt);
        ct_increment(xbar, kr, inc_ref);
    }
    T Dm[25];       // columns D_i (row-major: Dm[r*5 + i])
    T U[25];        // columns u_i + zdev (before centring)
    T zdev[5] = {T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int i = 0; i < NX; ++i) {
        T sg[5], zp[5], zm[5];
#pragma unroll
        for (int r = 0; r < 5; ++r) sg[r] = sq * L[r * NX + i];
        dev_f_pair(m, xbar, kr, inc_ref, sg, zp, zm);
#pragma unroll
        for (int r = 0; r < 5; ++r) {
            Dm[r * NX + i] = zp[r] - zm[r];
            const T h = T(0.5) * (zp[r] + zm[r]);
            U[r * NX + i] = h;
            zdev[r] += h;
        }
    }
    // zbar - f(xbar): the side points' mean deviation (the centre's is zero)
#pragma unroll
    for (int r = 0; r < 5; ++r) zdev[r] *= m.sp_w;
    // F = D L^{-1} / (2 scale)
    const T sc = T(0.5) * trcp(sq);
#pragma unroll
    for (int i = 0; i < 25; ++i) Dm[i] *= sc;
    solve_rows_lower_t<T, 5>(L, rdiag, Dm, tr.F);
    // Lambda = w sum_i u_i u_i^T + w0c zdev zdev^T with u_i = U_i - zdev (the
    // side points' D D^T part cancels against F Pbar F^T)
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int i = 0; i < NX; ++i) U[r * NX + i] -= zdev[r];
#pragma unroll
    for (int r = 0; r < 5; ++r)
#pragma unroll
        for (int q = r; q < 5; ++q) {
            T s = T(0);
#pragma unroll
            for (int i = 0; i < NX; ++i) s = fma(U[r * NX + i], U[q * NX + i], s);
            tr.Q[si(r, q)] = m.Q[si(r, q)] + s * m.sp_w + m.sp_w0c * zdev[r] * zdev[q];
        }
    // fx = zbar = f(xbar) + zdev
    if (m.kind == MODEL_LINEAR) {
        T Fx[5];
        T Fm[25];
#pragma unroll
        for (int i = 0; i < 25; ++i) Fm[i] = m.F[i];
        mv(Fm, xbar, Fx);
#pragma unroll
        for (int r = 0; r < 5; ++r) tr.fx[r] = Fx[r] + m.c[r] + zdev[r];
    } else {
        tr.fx[0] = xbar[0] + inc_ref[0] + zdev[0];
        tr.fx[1] = xbar[1] + inc_ref[1] + zdev[1];
        tr.fx[2] = inc_ref[2] + zdev[2];
        tr.fx[3] = inc_ref[3] + zdev[3];
        tr.fx[4] = inc_ref[4] + zdev[4];
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) tr.xn[i] = xbar[i];
}

template <typename T>
PES_DEV void lin_obs_cubature(const DevModel<T>& m, int b, const T* xbar, const T* L, const T* rdiag, const T* y,
                              Obs<T>& ob)
{
    const T sq = m.sp_scale;
    T s[4] = {T(0), T(0), T(0), T(0)};
    T h_ref[2];
    const bool lin = (m.kind == MODEL_LINEAR);
    if (lin) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            T v = m.d[r];
#pragma unroll
            for (int l = 0; l < 5; ++l) v = fma(m.H[r * 5 + l], xbar[l], v);
            h_ref[r] = v;
        }
    } else {
        load_sensors(m, b, s);
        bearings(xbar, s, h_ref);
    }
    T Dm[10], U[10];
    T zdev[2] = {T(0), T(0)};
#pragma unroll
    for (int i = 0; i < NX; ++i) {
        T zp[2] = {T(0), T(0)}, zm[2] = {T(0), T(0)};
        // bearings see only the position; chol(Pbar) is lower triangular, so
        // sigma directions i >= 2 leave the position (and the bearing) unchanged
        if (lin || i < 2) {
            T sg[5];
#pragma unroll
            for (int r = 0; r < 5; ++r) sg[r] = sq * L[r * NX + i];
            dev_h_pair(m, xbar, s, sg, zp, zm);
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            Dm[r * NX + i] = zp[r] - zm[r];
            const T h = T(0.5) * (zp[r] + zm[r]);
            U[r * NX + i] = h;
            zdev[r] += h;
        }
    }
#pragma unroll
    for (int r = 0; r < 2; ++r) zdev[r] *= m.sp_w;
    const T sc = T(0.5) * trcp(sq);
#pragma unroll
    for (int i = 0; i < 10; ++i) Dm[i] *= sc;
    solve_rows_lower_t<T, 2>(L, rdiag, Dm, ob.H);
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int i = 0; i < NX; ++i) U[r * NX + i] -= zdev[r];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int q = r; q < 2; ++q) {
            T v = T(0);
#pragma unroll
            for (int i = 0; i < NX; ++i) v = fma(U[r * NX + i], U[q * NX + i], v);
            ob.R[si2(r, q)] = m.R[si2(r, q)] + v * m.sp_w + m.sp_w0c * zdev[r] * zdev[q];
        }
    // residual about zbar = h(xbar) + zdev, measurement unwrapped nearest h(xbar)
    if (lin) {
        ob.r[0] = y[0] - h_ref[0] - zdev[0];
        ob.r[1] = y[1] - h_ref[1] - zdev[1];
    } else {
        ob.r[0] = wrap_angle(y[0] - h_ref[0]) - zdev[0];
        ob.r[1] = wrap_angle(y[1] - h_ref[1]) - zdev[1];
    }
#pragma unroll
    for (int i = 0; i < 5; ++i) ob.xn[i] = xbar[i];
}

// ---- third-order Gauss-Hermite product rule -------------------------------------
//
// The regression of Eqs. 7-9 over the 3^5 points xbar + L xi, L = chol(Pbar),
// xi in {-sqrt 3, 0, sqrt 3}^5, weights the products of 1/6, 2/3, 1/6. With the
// deviations dz = g(xbar + L xi) - g(xbar) and sum_i w_i xi_i = 0:
//   zbar - g(xbar) = sum w dz,   G = sum w dz xi^T,   F = Psi^T Pbar^{-1} = G L^{-1},
//   Lambda = sum w dz dz^T - (zbar - g)(zbar - g)^T - G G^T.

// Node and weight of digit q (0, 1, 2) of the product rule.
template <typename T>
PES_DEV void gh_node(int q, T& xi, T& w)
{
    const T r3 = T(1.7320508075688772935);
    xi = q == 0 ? -r3 : (q == 1 ? T(0) : r3);
    w = q == 1 ? T(2) / T(3) : T(1) / T(6);
}

// f(xbar + dx) - f(xbar) of the coordinated turn (the one-sided form of
// dev_f_pair).
template <typename T>
PES_DEV void ct_deviation(const DevModel<T>& m, const T* xbar, const CTCoef<T>& kr, const T* inc_ref, const T* dx,
                          T* dz)
{
    const T dt = m.dt;
    const T thr = sizeof(T) == 4 ? T(0.05) : T(0.01);
    T sd, cd, omcd;
    const T d = dx[4] * dt;
    if (fabs(d) < T(0.05)) {
        const T d2 = d * d;
        sd = d * (T(1) - d2 * (T(1) / T(6)) * (T(1) - d2 * (T(1) / T(20)) * (T(1) - d2 * (T(1) / T(42)))));
        omcd = d2 * T(0.5) * (T(1) - d2 * (T(1) / T(12)) * (T(1) - d2 * (T(1) / T(30)) * (T(1) - d2 * (T(1) / T(56)))));
        cd = T(1) - omcd;
    } else {
        tsincos(d, &sd, &cd);
        omcd = sd * sd * trcp(T(1) + cd);
    }
    const T omcr = (kr.c > T(0)) ? kr.s * kr.s * trcp(T(1) + kr.c) : T(1) - kr.c;
    const T w = xbar[4] + dx[4];
    const T a = w * dt;
    const T sn = kr.s * cd + kr.c * sd;
    const T cs = kr.c * cd - kr.s * sd;
    T A1, A2;
    if (fabs(a) < thr) {
        const T a2 = a * a;
        A1 = dt * (T(1) - a2 * (T(1) / T(6)) + a2 * a2 * (T(1) / T(120)));
        A2 = dt * a * (T(0.5) - a2 * (T(1) / T(24)) + a2 * a2 * (T(1) / T(720)));
    } else {
        const T omc = omcr + kr.c * omcd + kr.s * sd;
        const T iw = trcp(w);
        A1 = sn * iw;
        A2 = omc * iw;
    }
    const T vx = xbar[2] + dx[2], vy = xbar[3] + dx[3];
    dz[0] = dx[0] + ((A1 * vx - A2 * vy) - inc_ref[0]);
    dz[1] = dx[1] + ((A2 * vx + A1 * vy) - inc_ref[1]);
    dz[2] = (cs * vx - sn * vy) - inc_ref[2];
    dz[3] = (sn * vx + cs * vy) - inc_ref[3];
    dz[4] = dx[4];
}

// The point xbar + L xi of index pnt (base-3 digits) and its weight.
template <typename T>
PES_DEV T gh_point(int pnt, const T* L, T* xi, T* dx)
{
    T w = T(1);
    int q = pnt;
#pragma unroll
    for (int d = 0; d < 5; ++d) {
        T wd;
        gh_node<T>(q % 3, xi[d], wd);
        w *= wd;
        q /= 3;
    }
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        T v = T(0);
#pragma unroll
        for (int d = 0; d <= r; ++d) v = fma(L[r * NX + d], xi[d], v);
        dx[r] = v;
    }
    return w;
}

// Two passes over the points: the first sums zbar - f(xbar) and G; the second
// sums Lambda as the weighted second moment of the regression's residuals
// dz - (zbar - f) - G xi, which equals the moment form above without its
// cancellation (the residuals are the small, nonlinear part).
template <typename T>
PES_DEV void lin_trans_gh(const DevModel<T>& m, const T* xbar, const T* L, const T* rdiag, Trans<T>& tr)
{
    if (m.kind == MODEL_LINEAR) {   // the regression of an affine map is the map
        lin_trans_taylor(m, xbar, tr);
        return;
    }
    const CTCoef<T> kr = ct_coef(xbar[4], m.dt);
    T inc_ref[5];
    ct_increment(xbar, kr, inc_ref);
    T zd[5] = {T(0), T(0), T(0), T(0), T(0)}, G[25];
#pragma unroll
    for (int i = 0; i < 25; ++i) G[i] = T(0);
#pragma unroll 1
    for (int pnt = 0; pnt < 243; ++pnt) {
        T xi[5], dx[5], dz[5];
        const T w = gh_point(pnt, L, xi, dx);
        ct_deviation(m, xbar, kr, inc_ref, dx, dz);
#pragma unroll
        for (int r = 0; r < 5; ++r) {
            const T wz = w * dz[r];
            zd[r] += wz;
#pragma unroll
            for (int d = 0; d < 5; ++d) G[r * 5 + d] = fma(wz, xi[d], G[r * 5 + d]);
        }
    }
    T Lam[15];
#pragma unroll
    for (int i = 0; i < 15; ++i) Lam[i] = T(0);
#pragma unroll 1
    for (int pnt = 0; pnt < 243; ++pnt) {
        T xi[5], dx[5], dz[5];
        const T w = gh_point(pnt, L, xi, dx);
        ct_deviation(m, xbar, kr, inc_ref, dx, dz);
        T e[5];
#pragma unroll
        for (int r = 0; r < 5; ++r) {
            T v = dz[r] - zd[r];
#pragma unroll
            for (int d = 0; d < 5; ++d) v = fma(-G[r * 5 + d], xi[d], v);
            e[r] = v;
        }
#pragma unroll
        for (int r = 0; r < 5; ++r)
#pragma unroll
            for (int c = r; c < 5; ++c) Lam[si(r, c)] = fma(w * e[r], e[c], Lam[si(r, c)]);
    }
    solve_rows_lower_t<T, 5>(L, rdiag, G, tr.F);
#pragma unroll
    for (int i = 0; i < 15; ++i) tr.Q[i] = m.Q[i] + Lam[i];
    tr.fx[0] = xbar[0] + inc_ref[0] + zd[0];
    tr.fx[1] = xbar[1] + inc_ref[1] + zd[1];
    tr.fx[2] = inc_ref[2] + zd[2];
    tr.fx[3] = inc_ref[3] + zd[3];
    tr.fx[4] = inc_ref[4] + zd[4];
#pragma unroll
    for (int i = 0; i < 5; ++i) tr.xn[i] = xbar[i];
}

// Bearings see only the position, and with L lower triangular the position of
// xbar + L xi depends on xi_0 and xi_1 alone: the 243-point rule reduces to
// the 9 points of (xi_0, xi_1), the other coordinates' weights summing to 1.
template <typename T>
PES_DEV void lin_obs_gh(const DevModel<T>& m, int b, const T* xbar, const T* L, const T* rdiag, const T* y,
                        Obs<T>& ob)
{
    if (m.kind == MODEL_LINEAR) {
        lin_obs_taylor(m, b, xbar, y, ob);
        return;
    }
    T s[4];
    load_sensors(m, b, s);
    T h_ref[2];
    bearings(xbar, s, h_ref);
    T dzs[9][2], xs[9][2], ws[9];
    T zd[2] = {T(0), T(0)}, G[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) G[i] = T(0);
#pragma unroll
    for (int q0 = 0; q0 < 3; ++q0)
#pragma unroll
        for (int q1 = 0; q1 < 3; ++q1) {
            const int j = q0 * 3 + q1;
            T x0, w0, x1, w1;
            gh_node<T>(q0, x0, w0);
            gh_node<T>(q1, x1, w1);
            ws[j] = w0 * w1;
            xs[j][0] = x0;
            xs[j][1] = x1;
            const T dpx = L[0] * x0, dpy = L[NX] * x0 + L[NX + 1] * x1;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const T rx = xbar[0] - s[2 * r], ry = xbar[1] - s[2 * r + 1];
                const T cross = rx * dpy - ry * dpx;
                const T rr = rx * rx + ry * ry;
                const T rs = rx * dpx + ry * dpy;
                dzs[j][r] = tatan2(cross, rr + rs);
                const T wz = ws[j] * dzs[j][r];
                zd[r] += wz;
                G[r * 5 + 0] = fma(wz, x0, G[r * 5 + 0]);
                G[r * 5 + 1] = fma(wz, x1, G[r * 5 + 1]);
            }
        }
    T Om[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        T e[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) e[r] = dzs[j][r] - zd[r] - G[r * 5] * xs[j][0] - G[r * 5 + 1] * xs[j][1];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = r; c < 2; ++c) Om[si2(r, c)] = fma(ws[j] * e[r], e[c], Om[si2(r, c)]);
    }
    solve_rows_lower_t<T, 2>(L, rdiag, G, ob.H);
#pragma unroll
    for (int i = 0; i < 3; ++i) ob.R[i] = m.R[i] + Om[i];
    ob.r[0] = wrap_angle(y[0] - h_ref[0]) - zd[0];
    ob.r[1] = wrap_angle(y[1] - h_ref[1]) - zd[1];
#pragma unroll
    for (int i = 0; i < 5; ++i) ob.xn[i] = xbar[i];
}

}  // namespace pes
