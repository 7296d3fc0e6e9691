/*
 * CPU FP64 oracle of the parallel iterated extended (IEKS) and cubature
 * sigma-point (IPLS) Kalman smoothers.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline / reference arm of the benchmark load this library. The product
 * (the CUDA library and its binding) never includes, links or calls it, and it
 * shares no code with the product.
 *
 * What it computes.
 *  - Given linearisation parameters (Eq. 6), the smoothing distribution of the
 *    affine-Gaussian model of Eq. 11 is exactly what a Kalman filter followed
 *    by a Rauch-Tung-Striebel smoother produces; the parallel formulation of
 *    Sec. 4 (elements Eqs. 13-14 and 17-18, operators Eqs. 15 and 19, applied
 *    by a prefix/suffix scan) reaches the same result in another order. So the
 *    definition written here is the plain sequential filter/smoother
 *    (orc_kf_rts).
 *  - Linearisation: Taylor expansion for IEKS (Eq. 10) and cubature
 *    statistical linear regression for IPLS (Eqs. 7-9), about the previous
 *    smoothed moments; the whole thing is iterated (Sec. 3).
 *  - A literal implementation of the paper's filtering and smoothing elements
 *    and associative operators (Eqs. 13-19) is kept beside the definition
 *    (orc_filter_element .. orc_smoother_by_elements) so that tests can check
 *    the readings of those equations against the definition.
 *
 * Readings of the paper (where it is garbled or silent):
 *  - Eq. 10: the transition offset is c_{k-1} = f(xbar_{k-1}) - F_{k-1} xbar_{k-1}.
 *  - Eq. 13: b_k uses d_k (the offset of h_k), not d_{k-1}.
 *  - Eq. 14: eta_k = (H_k F_{k-1})^T S_k^{-1} (y_k - H_k c_{k-1} - d_k), without
 *    the extra H_k printed before the residual.
 *  - Eq. 17: E_k = P*_k F_k^T (F_k P*_k F_k^T + Q'_k)^{-1} (filtered covariance
 *    in front, Q'_k of the transition k -> k+1).
 *  - Eqs. 3/13 at k = 1: a prior element a_0 = (A=0, b=m_0, C=P_0, eta=0, J=0) is
 *    placed before a_1, so every k >= 1 uses the generic element and x_0 is
 *    estimated too.
 *  - Iteration 0 linearises about the prior: xbar_k = m_0, Pbar_k = P_0.
 *  - Cubature rule: 2 n_x points xbar +/- sqrt(n_x) chol(Pbar) e_i, weights 1/(2 n_x).
 *  - Bearings are unwrapped to the branch nearest h(xbar_k): the measurement
 *    y_k and every transformed sigma point.
 *
 * Layouts are state-major (array of structures): x[k*5+i], full symmetric
 * 5x5 matrices P[k*25 + 5*i + j], H[k*10 + 5*r + j], y[k*2 + r], R[k*4 + 2*r + s].
 * Index k = offsets[b] is the x_0 of trajectory b; transitions are stored at
 * their source state (F_k maps x_k to x_{k+1}); observations at their state.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NX 5
#define NY 2
#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* small dense linear algebra, row-major                                      */
/* ------------------------------------------------------------------------- */

/* C (n x p) = A (n x m) B (m x p) */
static void mm(int n, int m, int p, const double* A, const double* B, double* C)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < p; ++j) {
            double s = 0.0;
            for (int l = 0; l < m; ++l) s += A[i * m + l] * B[l * p + j];
            C[i * p + j] = s;
        }
}

/* C (n x p) = A (n x m) B^T, B is (p x m) */
static void mmt(int n, int m, int p, const double* A, const double* B, double* C)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < p; ++j) {
            double s = 0.0;
            for (int l = 0; l < m; ++l) s += A[i * m + l] * B[j * m + l];
            C[i * p + j] = s;
        }
}

/* C (n x p) = A^T B, A is (m x n), B is (m x p) */
static void mtm(int n, int m, int p, const double* A, const double* B, double* C)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < p; ++j) {
            double s = 0.0;
            for (int l = 0; l < m; ++l) s += A[l * n + i] * B[l * p + j];
            C[i * p + j] = s;
        }
}

/* y (n) = A (n x m) x */
static void mv(int n, int m, const double* A, const double* x, double* y)
{
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int l = 0; l < m; ++l) s += A[i * m + l] * x[l];
        y[i] = s;
    }
}

/* y (n) = A^T x, A is (m x n) */
static void mtv(int n, int m, const double* A, const double* x, double* y)
{
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int l = 0; l < m; ++l) s += A[l * n + i] * x[l];
        y[i] = s;
    }
}

static void symmetrize(int n, double* A)
{
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double v = 0.5 * (A[i * n + j] + A[j * n + i]);
            A[i * n + j] = v;
            A[j * n + i] = v;
        }
}

static void eye(int n, double* A)
{
    memset(A, 0, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i) A[i * n + i] = 1.0;
}

/* Cholesky A = L L^T (L lower, row-major). Returns 0 if A is not positive definite. */
static int cholesky(int n, const double* A, double* L)
{
    memset(L, 0, sizeof(double) * n * n);
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int l = 0; l < j; ++l) s -= L[j * n + l] * L[j * n + l];
        if (!(s > 0.0)) return 0;
        double d = sqrt(s);
        L[j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int l = 0; l < j; ++l) t -= L[i * n + l] * L[j * n + l];
            L[i * n + j] = t / d;
        }
    }
    return 1;
}

/* Solve (L L^T) X = B for X (n x r) given the Cholesky factor L. */
static void chol_solve(int n, int r, const double* L, const double* B, double* X)
{
    double* Y = (double*)malloc(sizeof(double) * n * r);
    for (int c = 0; c < r; ++c) {
        for (int i = 0; i < n; ++i) {
            double s = B[i * r + c];
            for (int l = 0; l < i; ++l) s -= L[i * n + l] * Y[l * r + c];
            Y[i * r + c] = s / L[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = Y[i * r + c];
            for (int l = i + 1; l < n; ++l) s -= L[l * n + i] * X[l * r + c];
            X[i * r + c] = s / L[i * n + i];
        }
    }
    free(Y);
}

/* Inverse by Gauss-Jordan elimination with partial pivoting. Returns 0 if singular. */
static int inverse(int n, const double* A, double* Ainv)
{
    double M[2 * NX * NX * 2];
    int w = 2 * n;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < w; ++j)
            M[i * w + j] = (j < n) ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int i = col + 1; i < n; ++i)
            if (fabs(M[i * w + col]) > fabs(M[piv * w + col])) piv = i;
        if (M[piv * w + col] == 0.0) return 0;
        if (piv != col)
            for (int j = 0; j < w; ++j) {
                double t = M[col * w + j];
                M[col * w + j] = M[piv * w + j];
                M[piv * w + j] = t;
            }
        double p = M[col * w + col];
        for (int j = 0; j < w; ++j) M[col * w + j] /= p;
        for (int i = 0; i < n; ++i) {
            if (i == col) continue;
            double f = M[i * w + col];
            if (f == 0.0) continue;
            for (int j = 0; j < w; ++j) M[i * w + j] -= f * M[col * w + j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ainv[i * n + j] = M[i * w + n + j];
    return 1;
}

/* ------------------------------------------------------------------------- */
/* model: coordinated turn (state [px, py, vx, vy, omega]) and bearings       */
/* ------------------------------------------------------------------------- */

double orc_wrap(double a)
{
    /* into [-pi, pi) */
    return a - 2.0 * ORC_PI * floor((a + ORC_PI) / (2.0 * ORC_PI));
}

/* sin(w dt)/w, (1-cos(w dt))/w and their derivatives in w; a series in
 * a = w dt below |a| < ORC_CT_SERIES where the closed forms lose accuracy. */
static void ct_coeffs(double w, double dt, double* A1, double* A2, double* dA1, double* dA2)
{
    double a = w * dt;
    if (fabs(a) < ORC_CT_SERIES) {
        double a2 = a * a;
        *A1 = dt * (1.0 - a2 / 6.0 + a2 * a2 / 120.0);
        *A2 = dt * a * (0.5 - a2 / 24.0 + a2 * a2 / 720.0);
        *dA1 = dt * dt * a * (-1.0 / 3.0 + a2 / 30.0 - a2 * a2 / 840.0);
        *dA2 = dt * dt * (0.5 - a2 / 8.0 + a2 * a2 / 144.0);
    } else {
        double s = sin(a), c = cos(a);
        *A1 = s / w;
        *A2 = (1.0 - c) / w;
        *dA1 = (a * c - s) / (w * w);
        *dA2 = (a * s - (1.0 - c)) / (w * w);
    }
}

void orc_ct_f(const double x[5], double dt, double out[5])
{
    double A1, A2, dA1, dA2;
    ct_coeffs(x[4], dt, &A1, &A2, &dA1, &dA2);
    double s = sin(x[4] * dt), c = cos(x[4] * dt);
    out[0] = x[0] + A1 * x[2] - A2 * x[3];
    out[1] = x[1] + A2 * x[2] + A1 * x[3];
    out[2] = c * x[2] - s * x[3];
    out[3] = s * x[2] + c * x[3];
    out[4] = x[4];
}

void orc_ct_jacobian(const double x[5], double dt, double F[25])
{
    double A1, A2, dA1, dA2;
    ct_coeffs(x[4], dt, &A1, &A2, &dA1, &dA2);
    double s = sin(x[4] * dt), c = cos(x[4] * dt);
    memset(F, 0, sizeof(double) * 25);
    F[0 * 5 + 0] = 1.0;
    F[0 * 5 + 2] = A1;
    F[0 * 5 + 3] = -A2;
    F[0 * 5 + 4] = dA1 * x[2] - dA2 * x[3];
    F[1 * 5 + 1] = 1.0;
    F[1 * 5 + 2] = A2;
    F[1 * 5 + 3] = A1;
    F[1 * 5 + 4] = dA2 * x[2] + dA1 * x[3];
    F[2 * 5 + 2] = c;
    F[2 * 5 + 3] = -s;
    F[2 * 5 + 4] = -dt * s * x[2] - dt * c * x[3];
    F[3 * 5 + 2] = s;
    F[3 * 5 + 3] = c;
    F[3 * 5 + 4] = dt * c * x[2] - dt * s * x[3];
    F[4 * 5 + 4] = 1.0;
}

void orc_bearings_h(const double x[5], const double s[4], double out[2])
{
    for (int r = 0; r < 2; ++r) out[r] = atan2(x[1] - s[2 * r + 1], x[0] - s[2 * r]);
}

void orc_bearings_jacobian(const double x[5], const double s[4], double H[10])
{
    memset(H, 0, sizeof(double) * 10);
    for (int r = 0; r < 2; ++r) {
        double dx = x[0] - s[2 * r], dy = x[1] - s[2 * r + 1];
        double rho2 = dx * dx + dy * dy;
        H[r * 5 + 0] = -dy / rho2;
        H[r * 5 + 1] = dx / rho2;
    }
}

void orc_process_noise(const orc_model* m, double Q[25])
{
    memset(Q, 0, sizeof(double) * 25);
    if (m->kind == ORC_MODEL_LINEAR) {
        memcpy(Q, m->Q, sizeof(double) * 25);
        return;
    }
    double dt = m->dt;
    if (m->q_form == 1) {
        for (int ax = 0; ax < 2; ++ax) {
            int p = ax, v = ax + 2;
            Q[p * 5 + p] = m->q_c * dt * dt * dt / 3.0;
            Q[p * 5 + v] = m->q_c * dt * dt / 2.0;
            Q[v * 5 + p] = m->q_c * dt * dt / 2.0;
            Q[v * 5 + v] = m->q_c * dt;
        }
    } else {
        Q[2 * 5 + 2] = m->q_c * dt;
        Q[3 * 5 + 3] = m->q_c * dt;
    }
    Q[4 * 5 + 4] = m->q_w * dt;
}

void orc_measurement_noise(const orc_model* m, double R[4])
{
    if (m->kind == ORC_MODEL_LINEAR) {
        memcpy(R, m->R, sizeof(double) * 4);
        return;
    }
    R[0] = m->r_std * m->r_std;
    R[1] = 0.0;
    R[2] = 0.0;
    R[3] = R[0];
}

static const double* sensors_of(const orc_model* m, int64_t b)
{
    return m->sensors + (m->sensors_per_traj ? 4 * b : 0);
}

static void model_f(const orc_model* m, const double* x, double* out)
{
    if (m->kind == ORC_MODEL_LINEAR) {
        mv(NX, NX, m->F, x, out);
        for (int i = 0; i < NX; ++i) out[i] += m->c[i];
    } else {
        orc_ct_f(x, m->dt, out);
    }
}

static void model_f_jac(const orc_model* m, const double* x, double* F)
{
    if (m->kind == ORC_MODEL_LINEAR)
        memcpy(F, m->F, sizeof(double) * 25);
    else
        orc_ct_jacobian(x, m->dt, F);
}

static void model_h(const orc_model* m, int64_t b, const double* x, double* out)
{
    if (m->kind == ORC_MODEL_LINEAR) {
        mv(NY, NX, m->H, x, out);
        for (int r = 0; r < NY; ++r) out[r] += m->d[r];
    } else {
        orc_bearings_h(x, sensors_of(m, b), out);
    }
}

static void model_h_jac(const orc_model* m, int64_t b, const double* x, double* H)
{
    if (m->kind == ORC_MODEL_LINEAR)
        memcpy(H, m->H, sizeof(double) * 10);
    else
        orc_bearings_jacobian(x, sensors_of(m, b), H);
}

/* measurements are angles (to be unwrapped) only for the bearings model */
static int angles(const orc_model* m) { return m->kind != ORC_MODEL_LINEAR; }

/* ------------------------------------------------------------------------- */
/* linearisation (Eqs. 7-10)                                                  */
/* ------------------------------------------------------------------------- */

/* Cubature statistical linear regression of z = g(x) about N(xbar, Pbar),
 * Eqs. 7-9: sigma points, the moments zbar, Psi, Phi of Eq. 8, then
 * G = Psi^T Pbar^{-1}, offset = zbar - G xbar, Lam = Phi - G Pbar G^T.
 * `which` 0: g = f (nz = 5); 1: g = h of trajectory b (nz = 2). */
int orc_slr(const orc_model* m, int which, int64_t b, const double xbar[5], const double Pbar[25],
            double* G, double* offset, double* Lam)
{
    const int nz = which == 0 ? NX : NY;
    double Lc[25];
    if (!cholesky(NX, Pbar, Lc)) return ORC_NOT_PD;
    double X[2 * NX][NX], Z[2 * NX][NX];
    const double scale = sqrt((double)NX);
    for (int i = 0; i < NX; ++i)
        for (int r = 0; r < NX; ++r) {
            X[i][r] = xbar[r] + scale * Lc[r * NX + i];
            X[i + NX][r] = xbar[r] - scale * Lc[r * NX + i];
        }
    double ref[NX];
    for (int j = 0; j < 2 * NX; ++j) {
        if (which == 0) model_f(m, X[j], Z[j]);
        else model_h(m, b, X[j], Z[j]);
    }
    if (which == 1 && angles(m)) {
        model_h(m, b, xbar, ref);
        for (int j = 0; j < 2 * NX; ++j)
            for (int r = 0; r < nz; ++r) Z[j][r] = ref[r] + orc_wrap(Z[j][r] - ref[r]);
    }
    const double w = 1.0 / (2.0 * NX);
    double zbar[NX] = {0};
    for (int j = 0; j < 2 * NX; ++j)
        for (int r = 0; r < nz; ++r) zbar[r] += w * Z[j][r];
    double Psi[NX * NX] = {0}; /* NX x nz */
    double Phi[NX * NX] = {0}; /* nz x nz */
    for (int j = 0; j < 2 * NX; ++j) {
        for (int i = 0; i < NX; ++i)
            for (int r = 0; r < nz; ++r)
                Psi[i * nz + r] += w * (X[j][i] - xbar[i]) * (Z[j][r] - zbar[r]);
        for (int r = 0; r < nz; ++r)
            for (int s = 0; s < nz; ++s)
                Phi[r * nz + s] += w * (Z[j][r] - zbar[r]) * (Z[j][s] - zbar[s]);
    }
    /* G^T = Pbar^{-1} Psi  (NX x nz) */
    double Gt[NX * NX];
    chol_solve(NX, nz, Lc, Psi, Gt);
    for (int r = 0; r < nz; ++r)
        for (int i = 0; i < NX; ++i) G[r * NX + i] = Gt[i * nz + r];
    double Gx[NX];
    mv(nz, NX, G, xbar, Gx);
    for (int r = 0; r < nz; ++r) offset[r] = zbar[r] - Gx[r];
    double GP[NX * NX], GPG[NX * NX];
    mm(nz, NX, NX, G, Pbar, GP);
    mmt(nz, NX, nz, GP, G, GPG);
    for (int r = 0; r < nz * nz; ++r) Lam[r] = Phi[r] - GPG[r];
    symmetrize(nz, Lam);
    return ORC_OK;
}

int orc_slr_unscented(const orc_model* m, int which, int64_t b, const double xbar[5], const double Pbar[25],
                      double* G, double* offset, double* Lam)
{
    const int nz = which == 0 ? NX : NY;
    const double a = m->ut_alpha, n = (double)NX;
    const double lambda = a * a * (n + m->ut_kappa) - n;
    if (!(n + lambda > 0.0)) return ORC_NOT_PD;
    double Lc[25];
    if (!cholesky(NX, Pbar, Lc)) return ORC_NOT_PD;
    /* point 0 is the centre; points 1..n and n+1..2n the two sides */
    double X[2 * NX + 1][NX], Z[2 * NX + 1][NX], Wm[2 * NX + 1], Wc[2 * NX + 1];
    const double scale = sqrt(n + lambda);
    for (int r = 0; r < NX; ++r) X[0][r] = xbar[r];
    for (int i = 0; i < NX; ++i)
        for (int r = 0; r < NX; ++r) {
            X[1 + i][r] = xbar[r] + scale * Lc[r * NX + i];
            X[1 + NX + i][r] = xbar[r] - scale * Lc[r * NX + i];
        }
    Wm[0] = lambda / (n + lambda);
    Wc[0] = Wm[0] + 1.0 - a * a + m->ut_beta;
    for (int j = 1; j < 2 * NX + 1; ++j) Wm[j] = Wc[j] = 1.0 / (2.0 * (n + lambda));
    double ref[NX];
    for (int j = 0; j < 2 * NX + 1; ++j) {
        if (which == 0) model_f(m, X[j], Z[j]);
        else model_h(m, b, X[j], Z[j]);
    }
    if (which == 1 && angles(m)) {
        model_h(m, b, xbar, ref);
        for (int j = 0; j < 2 * NX + 1; ++j)
            for (int r = 0; r < nz; ++r) Z[j][r] = ref[r] + orc_wrap(Z[j][r] - ref[r]);
    }
    double zbar[NX] = {0};
    for (int j = 0; j < 2 * NX + 1; ++j)
        for (int r = 0; r < nz; ++r) zbar[r] += Wm[j] * Z[j][r];
    double Psi[NX * NX] = {0}; /* NX x nz */
    double Phi[NX * NX] = {0}; /* nz x nz */
    for (int j = 0; j < 2 * NX + 1; ++j) {
        for (int i = 0; i < NX; ++i)
            for (int r = 0; r < nz; ++r)
                Psi[i * nz + r] += Wc[j] * (X[j][i] - xbar[i]) * (Z[j][r] - zbar[r]);
        for (int r = 0; r < nz; ++r)
            for (int s = 0; s < nz; ++s)
                Phi[r * nz + s] += Wc[j] * (Z[j][r] - zbar[r]) * (Z[j][s] - zbar[s]);
    }
    double Gt[NX * NX];
    chol_solve(NX, nz, Lc, Psi, Gt);
    for (int r = 0; r < nz; ++r)
        for (int i = 0; i < NX; ++i) G[r * NX + i] = Gt[i * nz + r];
    double Gx[NX];
    mv(nz, NX, G, xbar, Gx);
    for (int r = 0; r < nz; ++r) offset[r] = zbar[r] - Gx[r];
    double GP[NX * NX], GPG[NX * NX];
    mm(nz, NX, NX, G, Pbar, GP);
    mmt(nz, NX, nz, GP, G, GPG);
    for (int r = 0; r < nz * nz; ++r) Lam[r] = Phi[r] - GPG[r];
    symmetrize(nz, Lam);
    return ORC_OK;
}

int orc_slr_gauss_hermite(const orc_model* m, int which, int64_t b, const double xbar[5], const double Pbar[25],
                          double* G, double* offset, double* Lam)
{
    const int nz = which == 0 ? NX : NY;
    double Lc[25];
    if (!cholesky(NX, Pbar, Lc)) return ORC_NOT_PD;
    const double node[3] = {-sqrt(3.0), 0.0, sqrt(3.0)};
    const double wt[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
    enum { NP = 243 };   /* 3^5 */
    static __thread double X[NP][NX], Z[NP][NX], W[NP];
    for (int p = 0; p < NP; ++p) {
        double xi[NX];
        int q = p;
        W[p] = 1.0;
        for (int d = 0; d < NX; ++d) {
            xi[d] = node[q % 3];
            W[p] *= wt[q % 3];
            q /= 3;
        }
        for (int r = 0; r < NX; ++r) {
            double v = xbar[r];
            for (int d = 0; d < NX; ++d) v += Lc[r * NX + d] * xi[d];
            X[p][r] = v;
        }
        if (which == 0) model_f(m, X[p], Z[p]);
        else model_h(m, b, X[p], Z[p]);
    }
    if (which == 1 && angles(m)) {
        double ref[NX];
        model_h(m, b, xbar, ref);
        for (int p = 0; p < NP; ++p)
            for (int r = 0; r < nz; ++r) Z[p][r] = ref[r] + orc_wrap(Z[p][r] - ref[r]);
    }
    double zbar[NX] = {0};
    for (int p = 0; p < NP; ++p)
        for (int r = 0; r < nz; ++r) zbar[r] += W[p] * Z[p][r];
    double Psi[NX * NX] = {0}; /* NX x nz */
    double Phi[NX * NX] = {0}; /* nz x nz */
    for (int p = 0; p < NP; ++p) {
        for (int i = 0; i < NX; ++i)
            for (int r = 0; r < nz; ++r) Psi[i * nz + r] += W[p] * (X[p][i] - xbar[i]) * (Z[p][r] - zbar[r]);
        for (int r = 0; r < nz; ++r)
            for (int t = 0; t < nz; ++t) Phi[r * nz + t] += W[p] * (Z[p][r] - zbar[r]) * (Z[p][t] - zbar[t]);
    }
    double Gt[NX * NX];
    chol_solve(NX, nz, Lc, Psi, Gt);
    for (int r = 0; r < nz; ++r)
        for (int i = 0; i < NX; ++i) G[r * NX + i] = Gt[i * nz + r];
    double Gx[NX];
    mv(nz, NX, G, xbar, Gx);
    for (int r = 0; r < nz; ++r) offset[r] = zbar[r] - Gx[r];
    double GP[NX * NX], GPG[NX * NX];
    mm(nz, NX, NX, G, Pbar, GP);
    mmt(nz, NX, nz, GP, G, GPG);
    for (int r = 0; r < nz * nz; ++r) Lam[r] = Phi[r] - GPG[r];
    symmetrize(nz, Lam);
    return ORC_OK;
}

int orc_linearize(const orc_model* m, int method, int64_t N, const int64_t* offsets, int64_t B,
                  const double* xbar, const double* Pbar, const double* y,
                  double* F, double* c, double* Qp, double* H, double* d, double* Rp, double* y_used)
{
    double Q[25], R[4];
    orc_process_noise(m, Q);
    orc_measurement_noise(m, R);
    (void)N;
    for (int64_t b = 0; b < B; ++b) {
        for (int64_t k = offsets[b]; k < offsets[b + 1]; ++k) {
            const double* xk = xbar + 5 * k;
            int has_next = (k + 1 < offsets[b + 1]);
            int has_obs = (k > offsets[b]);
            /* transition k -> k+1 (Eq. 10 or Eq. 7) */
            if (has_next) {
                if (method == ORC_IEKS) {
                    double fx[NX], Fx[NX];
                    model_f_jac(m, xk, F + 25 * k);
                    model_f(m, xk, fx);
                    mv(NX, NX, F + 25 * k, xk, Fx);
                    for (int i = 0; i < NX; ++i) c[5 * k + i] = fx[i] - Fx[i];
                    memcpy(Qp + 25 * k, Q, sizeof(Q));
                } else {
                    double Lam[25];
                    int st = method == ORC_UNSCENTED
                                 ? orc_slr_unscented(m, 0, b, xk, Pbar + 25 * k, F + 25 * k, c + 5 * k, Lam)
                             : method == ORC_GAUSS_HERMITE
                                 ? orc_slr_gauss_hermite(m, 0, b, xk, Pbar + 25 * k, F + 25 * k, c + 5 * k, Lam)
                                 : orc_slr(m, 0, b, xk, Pbar + 25 * k, F + 25 * k, c + 5 * k, Lam);
                    if (st != ORC_OK) return st;
                    for (int i = 0; i < 25; ++i) Qp[25 * k + i] = Q[i] + Lam[i];
                }
            } else {
                memset(F + 25 * k, 0, sizeof(double) * 25);
                memset(c + 5 * k, 0, sizeof(double) * 5);
                memset(Qp + 25 * k, 0, sizeof(double) * 25);
            }
            /* observation at k (Eq. 10 or Eq. 9) */
            if (has_obs) {
                double hx[NY];
                model_h(m, b, xk, hx);
                if (method == ORC_IEKS) {
                    double Hx[NY];
                    model_h_jac(m, b, xk, H + 10 * k);
                    mv(NY, NX, H + 10 * k, xk, Hx);
                    for (int r = 0; r < NY; ++r) d[2 * k + r] = hx[r] - Hx[r];
                    memcpy(Rp + 4 * k, R, sizeof(R));
                } else {
                    double Om[4];
                    int st = method == ORC_UNSCENTED
                                 ? orc_slr_unscented(m, 1, b, xk, Pbar + 25 * k, H + 10 * k, d + 2 * k, Om)
                             : method == ORC_GAUSS_HERMITE
                                 ? orc_slr_gauss_hermite(m, 1, b, xk, Pbar + 25 * k, H + 10 * k, d + 2 * k, Om)
                                 : orc_slr(m, 1, b, xk, Pbar + 25 * k, H + 10 * k, d + 2 * k, Om);
                    if (st != ORC_OK) return st;
                    for (int i = 0; i < 4; ++i) Rp[4 * k + i] = R[i] + Om[i];
                }
                for (int r = 0; r < NY; ++r)
                    y_used[2 * k + r] = angles(m) ? hx[r] + orc_wrap(y[2 * k + r] - hx[r]) : y[2 * k + r];
            } else {
                memset(H + 10 * k, 0, sizeof(double) * 10);
                memset(d + 2 * k, 0, sizeof(double) * 2);
                memset(Rp + 4 * k, 0, sizeof(double) * 4);
                y_used[2 * k] = 0.0;
                y_used[2 * k + 1] = 0.0;
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* the definition: sequential Kalman filter + RTS smoother of Eq. 11          */
/* ------------------------------------------------------------------------- */

/* The Levenberg-Marquardt pseudo-measurement of state k: a Kalman update of
 * (m, P) with H = I, R = I / lambda and measurement xbar_k. */
static int damp_update(double* m, double* P, const double* xbar, double lambda)
{
    double S[25], Sinv[25], K[25], KP[25];
    memcpy(S, P, sizeof S);
    for (int i = 0; i < NX; ++i) S[i * NX + i] += 1.0 / lambda;
    if (!inverse(NX, S, Sinv)) return ORC_NOT_PD;
    mm(NX, NX, NX, P, Sinv, K);
    double v[NX], Kv[NX];
    for (int i = 0; i < NX; ++i) v[i] = xbar[i] - m[i];
    mv(NX, NX, K, v, Kv);
    for (int i = 0; i < NX; ++i) m[i] += Kv[i];
    mm(NX, NX, NX, K, P, KP);
    for (int i = 0; i < 25; ++i) P[i] -= KP[i];
    symmetrize(NX, P);
    return ORC_OK;
}

int orc_kf_rts(int64_t N, const int64_t* offsets, int64_t B,
               const double* F, const double* c, const double* Qp,
               const double* H, const double* d, const double* Rp, const double* y,
               const double* m0, const double* P0,
               double* xf, double* Pf, double* xs, double* Ps)
{
    return orc_kf_rts_damped(N, offsets, B, F, c, Qp, H, d, Rp, y, m0, P0, NULL, 0.0, xf, Pf, xs, Ps);
}

int orc_kf_rts_damped(int64_t N, const int64_t* offsets, int64_t B,
                      const double* F, const double* c, const double* Qp,
                      const double* H, const double* d, const double* Rp, const double* y,
                      const double* m0, const double* P0, const double* xbar, double lambda,
                      double* xf, double* Pf, double* xs, double* Ps)
{
    double* xp = (double*)malloc(sizeof(double) * 5 * N);
    double* Pp = (double*)malloc(sizeof(double) * 25 * N);
    int status = ORC_OK;
    for (int64_t b = 0; b < B && status == ORC_OK; ++b) {
        int64_t k0 = offsets[b], k1 = offsets[b + 1];
        memcpy(xf + 5 * k0, m0 + 5 * b, sizeof(double) * 5);
        memcpy(Pf + 25 * k0, P0 + 25 * b, sizeof(double) * 25);
        if (lambda > 0.0 && (status = damp_update(xf + 5 * k0, Pf + 25 * k0, xbar + 5 * k0, lambda)) != ORC_OK) break;
        for (int64_t k = k0 + 1; k < k1; ++k) {
            /* predict with the transition k-1 -> k */
            const double* Fk = F + 25 * (k - 1);
            double* mp = xp + 5 * k;
            double* P_ = Pp + 25 * k;
            mv(NX, NX, Fk, xf + 5 * (k - 1), mp);
            for (int i = 0; i < NX; ++i) mp[i] += c[5 * (k - 1) + i];
            double FP[25];
            mm(NX, NX, NX, Fk, Pf + 25 * (k - 1), FP);
            mmt(NX, NX, NX, FP, Fk, P_);
            for (int i = 0; i < 25; ++i) P_[i] += Qp[25 * (k - 1) + i];
            symmetrize(NX, P_);
            /* update with y_k */
            const double* Hk = H + 10 * k;
            double HP[10], S[4], Sinv[4], K[10], PHt[10];
            mm(NY, NX, NX, Hk, P_, HP);
            mmt(NY, NX, NY, HP, Hk, S);
            for (int i = 0; i < 4; ++i) S[i] += Rp[4 * k + i];
            if (!inverse(NY, S, Sinv)) { status = ORC_NOT_PD; break; }
            mmt(NX, NX, NY, P_, Hk, PHt);
            mm(NX, NY, NY, PHt, Sinv, K);
            double Hm[NY], v[NY];
            mv(NY, NX, Hk, mp, Hm);
            for (int r = 0; r < NY; ++r) v[r] = y[2 * k + r] - Hm[r] - d[2 * k + r];
            double Kv[NX];
            mv(NX, NY, K, v, Kv);
            for (int i = 0; i < NX; ++i) xf[5 * k + i] = mp[i] + Kv[i];
            double KS[10], KSK[25];
            mm(NX, NY, NY, K, S, KS);
            mmt(NX, NY, NX, KS, K, KSK);
            for (int i = 0; i < 25; ++i) Pf[25 * k + i] = P_[i] - KSK[i];
            symmetrize(NX, Pf + 25 * k);
            if (lambda > 0.0 && (status = damp_update(xf + 5 * k, Pf + 25 * k, xbar + 5 * k, lambda)) != ORC_OK) break;
        }
        if (status != ORC_OK) break;
        /* Rauch-Tung-Striebel backward pass */
        memcpy(xs + 5 * (k1 - 1), xf + 5 * (k1 - 1), sizeof(double) * 5);
        memcpy(Ps + 25 * (k1 - 1), Pf + 25 * (k1 - 1), sizeof(double) * 25);
        for (int64_t k = k1 - 2; k >= k0; --k) {
            double L[25];
            if (!cholesky(NX, Pp + 25 * (k + 1), L)) { status = ORC_NOT_PD; break; }
            /* G = Pf_k F_k^T Pp_{k+1}^{-1}  <=>  Pp_{k+1} G^T = F_k Pf_k */
            double FP[25], Gt[25], G[25];
            mm(NX, NX, NX, F + 25 * k, Pf + 25 * k, FP);
            chol_solve(NX, NX, L, FP, Gt);
            for (int i = 0; i < NX; ++i)
                for (int j = 0; j < NX; ++j) G[i * 5 + j] = Gt[j * 5 + i];
            double dm[NX], Gdm[NX];
            for (int i = 0; i < NX; ++i) dm[i] = xs[5 * (k + 1) + i] - xp[5 * (k + 1) + i];
            mv(NX, NX, G, dm, Gdm);
            for (int i = 0; i < NX; ++i) xs[5 * k + i] = xf[5 * k + i] + Gdm[i];
            double dP[25], GdP[25], GdPG[25];
            for (int i = 0; i < 25; ++i) dP[i] = Ps[25 * (k + 1) + i] - Pp[25 * (k + 1) + i];
            mm(NX, NX, NX, G, dP, GdP);
            mmt(NX, NX, NX, GdP, G, GdPG);
            for (int i = 0; i < 25; ++i) Ps[25 * k + i] = Pf[25 * k + i] + GdPG[i];
            symmetrize(NX, Ps + 25 * k);
        }
    }
    free(xp);
    free(Pp);
    return status;
}

/* ------------------------------------------------------------------------- */
/* the iteration (Sec. 3): re-linearise about the previous smoothed moments   */
/* ------------------------------------------------------------------------- */

int orc_kf_loglik(int64_t N, const int64_t* offsets, int64_t B,
                  const double* F, const double* c, const double* Qp,
                  const double* H, const double* d, const double* Rp, const double* y,
                  const double* m0, const double* P0, double* loglik)
{
    (void)N;
    const double log_2pi = log(2.0 * 3.14159265358979323846);
    for (int64_t b = 0; b < B; ++b) {
        double m[5], P[25];
        memcpy(m, m0 + 5 * b, sizeof m);
        memcpy(P, P0 + 25 * b, sizeof P);
        double ll = 0.0;
        for (int64_t k = offsets[b] + 1; k < offsets[b + 1]; ++k) {
            /* one-step prediction of x_k and of y_k */
            double mp[5], FP[25], Pp[25];
            mv(NX, NX, F + 25 * (k - 1), m, mp);
            for (int i = 0; i < NX; ++i) mp[i] += c[5 * (k - 1) + i];
            mm(NX, NX, NX, F + 25 * (k - 1), P, FP);
            mmt(NX, NX, NX, FP, F + 25 * (k - 1), Pp);
            for (int i = 0; i < 25; ++i) Pp[i] += Qp[25 * (k - 1) + i];
            const double* Hk = H + 10 * k;
            double HP[10], S[4], Sinv[4], Hm[2], v[2];
            mm(NY, NX, NX, Hk, Pp, HP);
            mmt(NY, NX, NY, HP, Hk, S);
            for (int i = 0; i < 4; ++i) S[i] += Rp[4 * k + i];
            if (!inverse(NY, S, Sinv)) return ORC_NOT_PD;
            const double det = S[0] * S[3] - S[1] * S[2];
            if (!(det > 0.0)) return ORC_NOT_PD;
            mv(NY, NX, Hk, mp, Hm);
            for (int r = 0; r < NY; ++r) v[r] = y[2 * k + r] - Hm[r] - d[2 * k + r];
            double q = 0.0;
            for (int r = 0; r < NY; ++r)
                for (int s = 0; s < NY; ++s) q += v[r] * Sinv[r * 2 + s] * v[s];
            ll += -0.5 * (q + log(det)) - 0.5 * NY * log_2pi;
            /* the update, as in the filter */
            double PHt[10], K[10], Kv[5], KS[10], KSK[25];
            mmt(NX, NX, NY, Pp, Hk, PHt);
            mm(NX, NY, NY, PHt, Sinv, K);
            mv(NX, NY, K, v, Kv);
            for (int i = 0; i < NX; ++i) m[i] = mp[i] + Kv[i];
            mm(NX, NY, NY, K, S, KS);
            mmt(NX, NY, NX, KS, K, KSK);
            for (int i = 0; i < 25; ++i) P[i] = Pp[i] - KSK[i];
            symmetrize(NX, P);
        }
        loglik[b] = ll;
    }
    return ORC_OK;
}

int orc_iterated_smoother(const orc_model* m, int method, int64_t N, const int64_t* offsets, int64_t B,
                          const double* y, const double* m0, const double* P0,
                          const double* x_init, const double* P_init, int max_iters, double tol,
                          double* x_out, double* P_out, int* iters_used, double* rel_history)
{
    double* F = (double*)malloc(sizeof(double) * 25 * N);
    double* c = (double*)malloc(sizeof(double) * 5 * N);
    double* Qp = (double*)malloc(sizeof(double) * 25 * N);
    double* H = (double*)malloc(sizeof(double) * 10 * N);
    double* d = (double*)malloc(sizeof(double) * 2 * N);
    double* Rp = (double*)malloc(sizeof(double) * 4 * N);
    double* yu = (double*)malloc(sizeof(double) * 2 * N);
    double* xf = (double*)malloc(sizeof(double) * 5 * N);
    double* Pf = (double*)malloc(sizeof(double) * 25 * N);
    double* xs = (double*)malloc(sizeof(double) * 5 * N);
    double* Ps = (double*)malloc(sizeof(double) * 25 * N);
    /* nominal trajectory: x_out / P_out hold it between iterations */
    for (int64_t b = 0; b < B; ++b)
        for (int64_t k = offsets[b]; k < offsets[b + 1]; ++k) {
            if (x_init) memcpy(x_out + 5 * k, x_init + 5 * k, sizeof(double) * 5);
            else memcpy(x_out + 5 * k, m0 + 5 * b, sizeof(double) * 5);
            if (P_init) memcpy(P_out + 25 * k, P_init + 25 * k, sizeof(double) * 25);
            else memcpy(P_out + 25 * k, P0 + 25 * b, sizeof(double) * 25);
        }
    int status = ORC_OK;
    int it = 0;
    int converged = 0;
    for (it = 1; it <= max_iters; ++it) {
        status = orc_linearize(m, method, N, offsets, B, x_out, P_out, y, F, c, Qp, H, d, Rp, yu);
        if (status != ORC_OK) break;
        status = orc_kf_rts_damped(N, offsets, B, F, c, Qp, H, d, Rp, yu, m0, P0, x_out, m->lm_lambda, xf, Pf, xs,
                                   Ps);
        if (status != ORC_OK) break;
        /* relative update norm, worst trajectory */
        double rel = 0.0;
        for (int64_t b = 0; b < B; ++b) {
            double num = 0.0, den = 0.0;
            for (int64_t k = offsets[b]; k < offsets[b + 1]; ++k)
                for (int i = 0; i < 5; ++i) {
                    double dv = xs[5 * k + i] - x_out[5 * k + i];
                    num += dv * dv;
                    den += xs[5 * k + i] * xs[5 * k + i];
                }
            double r = den > 0.0 ? sqrt(num / den) : sqrt(num);
            if (r > rel) rel = r;
        }
        if (rel_history) rel_history[it - 1] = rel;
        memcpy(x_out, xs, sizeof(double) * 5 * N);
        memcpy(P_out, Ps, sizeof(double) * 25 * N);
        if (tol > 0.0 && rel <= tol) {
            converged = 1;
            break;
        }
    }
    if (it > max_iters) it = max_iters;
    if (iters_used) *iters_used = it;
    if (status == ORC_OK && tol > 0.0 && !converged) status = ORC_NOT_CONVERGED;
    free(F); free(c); free(Qp); free(H); free(d); free(Rp); free(yu);
    free(xf); free(Pf); free(xs); free(Ps);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Levenberg-Marquardt with an adaptive damping (Sec. 3 names the LM variant)  */
/* ------------------------------------------------------------------------- */

/* The MAP objective of Eq. 4 that the IEKS minimises by Gauss-Newton steps
 * (Sec. 3), per trajectory, for a positive definite Q:
 *   J = 1/2 |x_0 - m0|^2_{P0^-1} + 1/2 sum_k |x_k - f(x_{k-1})|^2_{Q^-1}
 *       + 1/2 sum_k |y_k - h(x_k)|^2_{R^-1},
 * the bearing residuals taken on the branch nearest zero. Returns ORC_NOT_PD
 * if Q, R or P0 is not positive definite. */
int orc_map_cost(const orc_model* m, int64_t N, const int64_t* offsets, int64_t B, const double* y,
                 const double* m0, const double* P0, const double* x, double* cost)
{
    (void)N;
    double Q[25], R[4], Qi[25], Ri[4];
    orc_process_noise(m, Q);
    orc_measurement_noise(m, R);
    double LQ[25];
    if (!cholesky(NX, Q, LQ) || !inverse(NX, Q, Qi) || !inverse(NY, R, Ri) || R[0] <= 0.0) return ORC_NOT_PD;
    for (int64_t b = 0; b < B; ++b) {
        const int64_t k0 = offsets[b], k1 = offsets[b + 1];
        double P0i[25], L0[25];
        if (!cholesky(NX, P0 + 25 * b, L0) || !inverse(NX, P0 + 25 * b, P0i)) return ORC_NOT_PD;
        double J = 0.0, e[NX], t[NX];
        for (int i = 0; i < NX; ++i) e[i] = x[5 * k0 + i] - m0[5 * b + i];
        mv(NX, NX, P0i, e, t);
        for (int i = 0; i < NX; ++i) J += 0.5 * e[i] * t[i];
        for (int64_t k = k0 + 1; k < k1; ++k) {
            double fx[NX];
            model_f(m, x + 5 * (k - 1), fx);
            for (int i = 0; i < NX; ++i) e[i] = x[5 * k + i] - fx[i];
            mv(NX, NX, Qi, e, t);
            for (int i = 0; i < NX; ++i) J += 0.5 * e[i] * t[i];
            double hx[NY], r[NY], u[NY];
            model_h(m, b, x + 5 * k, hx);
            for (int i = 0; i < NY; ++i) {
                r[i] = y[2 * k + i] - hx[i];
                if (angles(m)) r[i] = orc_wrap(r[i]);
            }
            mv(NY, NY, Ri, r, u);
            for (int i = 0; i < NY; ++i) J += 0.5 * r[i] * u[i];
        }
        cost[b] = J;
    }
    return ORC_OK;
}

/* The IEKS with Levenberg-Marquardt steps and an adaptive damping, per
 * trajectory b: the step of iteration i is the IEKS iteration about the
 * current nominal with the pseudo-measurement damping lambda_b (the smoother
 * of orc_kf_rts_damped); it is accepted if it lowers the MAP cost
 * (orc_map_cost), and then lambda_b <- lambda_b / nu; otherwise the nominal
 * stays and lambda_b <- lambda_b * nu. Every trajectory starts at lambda0.
 * A trajectory has converged at the first iteration whose step (accepted or
 * not: near the optimum the cost no longer separates a step from the nominal)
 * has a relative size ||x_step - x_nom||_F / ||x_step||_F <= tol; with tol > 0
 * the iteration stops
 * once every trajectory has (ORC_NOT_CONVERGED if max_iters come first), with
 * tol <= 0 it runs max_iters iterations. Outputs: the accepted nominal x_out
 * [N][5], the damped smoother's covariances of each trajectory's last
 * accepted step P_out [N][25] (the prior covariance P0 until one is accepted),
 * iterations run, and per trajectory (each may be NULL) the final damping,
 * the first converged iteration (0: none) and the number of accepted steps. */
int orc_iterated_smoother_lm(const orc_model* m, int64_t N, const int64_t* offsets, int64_t B, const double* y,
                             const double* m0, const double* P0, const double* x_init, int max_iters, double tol,
                             double lambda0, double nu, double* x_out, double* P_out, int* iters_used,
                             double* lambda_out, int* conv_iter, int* accepted)
{
    double* F = (double*)malloc(sizeof(double) * 25 * N);
    double* c = (double*)malloc(sizeof(double) * 5 * N);
    double* Qp = (double*)malloc(sizeof(double) * 25 * N);
    double* H = (double*)malloc(sizeof(double) * 10 * N);
    double* d = (double*)malloc(sizeof(double) * 2 * N);
    double* Rp = (double*)malloc(sizeof(double) * 4 * N);
    double* yu = (double*)malloc(sizeof(double) * 2 * N);
    double* xf = (double*)malloc(sizeof(double) * 5 * N);
    double* Pf = (double*)malloc(sizeof(double) * 25 * N);
    double* xs = (double*)malloc(sizeof(double) * 5 * N);
    double* Ps = (double*)malloc(sizeof(double) * 25 * N);
    double* lam = (double*)malloc(sizeof(double) * B);
    double* Jcur = (double*)malloc(sizeof(double) * B);
    double* Jnew = (double*)malloc(sizeof(double) * B);
    int* conv = (int*)calloc((size_t)B, sizeof(int));
    int* acc = (int*)calloc((size_t)B, sizeof(int));
    for (int64_t b = 0; b < B; ++b) {
        lam[b] = lambda0;
        for (int64_t k = offsets[b]; k < offsets[b + 1]; ++k) {
            if (x_init) memcpy(x_out + 5 * k, x_init + 5 * k, sizeof(double) * 5);
            else memcpy(x_out + 5 * k, m0 + 5 * b, sizeof(double) * 5);
            memcpy(P_out + 25 * k, P0 + 25 * b, sizeof(double) * 25);
        }
    }
    int status = orc_map_cost(m, N, offsets, B, y, m0, P0, x_out, Jcur);
    int it = 0, all = 0;
    for (it = 1; it <= max_iters && status == ORC_OK; ++it) {
        status = orc_linearize(m, ORC_IEKS, N, offsets, B, x_out, NULL, y, F, c, Qp, H, d, Rp, yu);
        if (status != ORC_OK) break;
        /* each trajectory's damped step with its own lambda */
        for (int64_t b = 0; b < B && status == ORC_OK; ++b) {
            const int64_t k0 = offsets[b], n = offsets[b + 1] - k0;
            const int64_t o1[2] = {0, n};
            status = orc_kf_rts_damped(n, o1, 1, F + 25 * k0, c + 5 * k0, Qp + 25 * k0, H + 10 * k0, d + 2 * k0,
                                       Rp + 4 * k0, yu + 2 * k0, m0 + 5 * b, P0 + 25 * b, x_out + 5 * k0, lam[b],
                                       xf + 5 * k0, Pf + 25 * k0, xs + 5 * k0, Ps + 25 * k0);
        }
        if (status != ORC_OK) break;
        status = orc_map_cost(m, N, offsets, B, y, m0, P0, xs, Jnew);
        if (status != ORC_OK) break;
        all = 1;
        for (int64_t b = 0; b < B; ++b) {
            const int64_t k0 = offsets[b], k1 = offsets[b + 1];
            double num = 0.0, den = 0.0;
            for (int64_t k = k0; k < k1; ++k)
                for (int i = 0; i < 5; ++i) {
                    const double dv = xs[5 * k + i] - x_out[5 * k + i];
                    num += dv * dv;
                    den += xs[5 * k + i] * xs[5 * k + i];
                }
            const double rel = den > 0.0 ? sqrt(num / den) : sqrt(num);
            if (Jnew[b] < Jcur[b]) {
                memcpy(x_out + 5 * k0, xs + 5 * k0, sizeof(double) * 5 * (k1 - k0));
                memcpy(P_out + 25 * k0, Ps + 25 * k0, sizeof(double) * 25 * (k1 - k0));
                Jcur[b] = Jnew[b];
                lam[b] /= nu;
                ++acc[b];
            } else {
                lam[b] *= nu;
            }
            if (!conv[b] && tol > 0.0 && rel <= tol) conv[b] = it;
            all = all && conv[b];
        }
        if (tol > 0.0 && all) break;
    }
    if (it > max_iters) it = max_iters;
    if (iters_used) *iters_used = it;
    if (status == ORC_OK && tol > 0.0 && !all) status = ORC_NOT_CONVERGED;
    for (int64_t b = 0; b < B; ++b) {
        if (lambda_out) lambda_out[b] = lam[b];
        if (conv_iter) conv_iter[b] = conv[b];
        if (accepted) accepted[b] = acc[b];
    }
    free(F); free(c); free(Qp); free(H); free(d); free(Rp); free(yu);
    free(xf); free(Pf); free(xs); free(Ps); free(lam); free(Jcur); free(Jnew); free(conv); free(acc);
    return status;
}

/* ------------------------------------------------------------------------- */
/* the paper's parallel-form elements and operators, written literally        */
/* ------------------------------------------------------------------------- */

/* Filtering element a_k = (A_k, b_k, C_k, eta_k, J_k), Eqs. 13-14, from the
 * transition (F, c, Q') of k-1 -> k and the observation (H, d, R', y) of k. */
int orc_filter_element(const double F[25], const double c[5], const double Qp[25],
                       const double H[10], const double d[2], const double Rp[4], const double y[2],
                       orc_felem* e)
{
    double HQ[10], S[4], Sinv[4], QHt[10], K[10];
    mm(NY, NX, NX, H, Qp, HQ);
    mmt(NY, NX, NY, HQ, H, S);
    for (int i = 0; i < 4; ++i) S[i] += Rp[i];
    if (!inverse(NY, S, Sinv)) return ORC_NOT_PD;
    mmt(NX, NX, NY, Qp, H, QHt);
    mm(NX, NY, NY, QHt, Sinv, K);
    double KH[25], IKH[25];
    mm(NX, NY, NX, K, H, KH);
    eye(NX, IKH);
    for (int i = 0; i < 25; ++i) IKH[i] -= KH[i];
    mm(NX, NX, NX, IKH, F, e->A);
    double Hc[NY], v[NY], Kv[NX];
    mv(NY, NX, H, c, Hc);
    for (int r = 0; r < NY; ++r) v[r] = y[r] - Hc[r] - d[r];
    mv(NX, NY, K, v, Kv);
    for (int i = 0; i < NX; ++i) e->b[i] = c[i] + Kv[i];
    mm(NX, NX, NX, IKH, Qp, e->C);
    symmetrize(NX, e->C);
    double HF[10], SiHF[10], Siv[2];
    mm(NY, NX, NX, H, F, HF);
    mm(NY, NY, NX, Sinv, HF, SiHF);
    mtm(NX, NY, NX, HF, SiHF, e->J);
    symmetrize(NX, e->J);
    mv(NY, NY, Sinv, v, Siv);
    mtv(NX, NY, HF, Siv, e->eta);
    return ORC_OK;
}

void orc_filter_prior_element(const double m0[5], const double P0[25], orc_felem* e)
{
    memset(e, 0, sizeof(*e));
    memcpy(e->b, m0, sizeof(double) * 5);
    memcpy(e->C, P0, sizeof(double) * 25);
}

/* a_i (x) a_j, Eq. 15. */
int orc_filter_combine(const orc_felem* ei, const orc_felem* ej, orc_felem* out)
{
    double CJ[25], M[25], Minv[25], JC[25], Mt[25], Mtinv[25];
    mm(NX, NX, NX, ei->C, ej->J, CJ);
    mm(NX, NX, NX, ej->J, ei->C, JC);
    eye(NX, M);
    eye(NX, Mt);
    for (int i = 0; i < 25; ++i) {
        M[i] += CJ[i];
        Mt[i] += JC[i];
    }
    if (!inverse(NX, M, Minv)) return ORC_NOT_PD;
    if (!inverse(NX, Mt, Mtinv)) return ORC_NOT_PD;
    orc_felem r;
    double AjM[25], t1[NX], t2[NX], t3[NX];
    mm(NX, NX, NX, ej->A, Minv, AjM);
    mm(NX, NX, NX, AjM, ei->A, r.A);
    mv(NX, NX, ei->C, ej->eta, t1);
    for (int i = 0; i < NX; ++i) t1[i] += ei->b[i];
    mv(NX, NX, AjM, t1, t2);
    for (int i = 0; i < NX; ++i) r.b[i] = t2[i] + ej->b[i];
    double AjMC[25], AjMCAt[25];
    mm(NX, NX, NX, AjM, ei->C, AjMC);
    mmt(NX, NX, NX, AjMC, ej->A, AjMCAt);
    for (int i = 0; i < 25; ++i) r.C[i] = AjMCAt[i] + ej->C[i];
    symmetrize(NX, r.C);
    double AitMt[25];
    mtm(NX, NX, NX, ei->A, Mtinv, AitMt);
    mv(NX, NX, ej->J, ei->b, t1);
    for (int i = 0; i < NX; ++i) t1[i] = ej->eta[i] - t1[i];
    mv(NX, NX, AitMt, t1, t3);
    for (int i = 0; i < NX; ++i) r.eta[i] = t3[i] + ei->eta[i];
    double AitMtJ[25], AitMtJA[25];
    mm(NX, NX, NX, AitMt, ej->J, AitMtJ);
    mm(NX, NX, NX, AitMtJ, ei->A, AitMtJA);
    for (int i = 0; i < 25; ++i) r.J[i] = AitMtJA[i] + ei->J[i];
    symmetrize(NX, r.J);
    *out = r;
    return ORC_OK;
}

/* Smoothing element a_k = (E_k, g_k, L_k) for k < n, Eq. 17. */
int orc_smoother_element(const double xf[5], const double Pf[25], const double F[25], const double c[5],
                         const double Qp[25], orc_selem* e)
{
    double FP[25], Pp[25], L[25], Et[25];
    mm(NX, NX, NX, F, Pf, FP);
    mmt(NX, NX, NX, FP, F, Pp);
    for (int i = 0; i < 25; ++i) Pp[i] += Qp[i];
    symmetrize(NX, Pp);
    if (!cholesky(NX, Pp, L)) return ORC_NOT_PD;
    /* E^T = Pp^{-1} F Pf */
    chol_solve(NX, NX, L, FP, Et);
    for (int i = 0; i < NX; ++i)
        for (int j = 0; j < NX; ++j) e->E[i * 5 + j] = Et[j * 5 + i];
    double mp[NX], Em[NX];
    mv(NX, NX, F, xf, mp);
    for (int i = 0; i < NX; ++i) mp[i] += c[i];
    mv(NX, NX, e->E, mp, Em);
    for (int i = 0; i < NX; ++i) e->g[i] = xf[i] - Em[i];
    double EFP[25];
    mm(NX, NX, NX, e->E, FP, EFP);
    for (int i = 0; i < 25; ++i) e->L[i] = Pf[i] - EFP[i];
    symmetrize(NX, e->L);
    return ORC_OK;
}

/* Eq. 18 */
void orc_smoother_last_element(const double xf[5], const double Pf[25], orc_selem* e)
{
    memset(e->E, 0, sizeof(e->E));
    memcpy(e->g, xf, sizeof(double) * 5);
    memcpy(e->L, Pf, sizeof(double) * 25);
}

/* a_i (x) a_j, Eq. 19. */
void orc_smoother_combine(const orc_selem* ei, const orc_selem* ej, orc_selem* out)
{
    orc_selem r;
    mm(NX, NX, NX, ei->E, ej->E, r.E);
    double Eg[NX];
    mv(NX, NX, ei->E, ej->g, Eg);
    for (int i = 0; i < NX; ++i) r.g[i] = Eg[i] + ei->g[i];
    double EL[25], ELE[25];
    mm(NX, NX, NX, ei->E, ej->L, EL);
    mmt(NX, NX, NX, EL, ei->E, ELE);
    for (int i = 0; i < 25; ++i) r.L[i] = ELE[i] + ei->L[i];
    symmetrize(NX, r.L);
    *out = r;
}

/* Filtering means/covariances as the prefix products a_0 (x) a_1 (x) ... (x) a_k
 * (Eq. 3 and Sec. 2), evaluated by a sequential left fold. */
int orc_filter_by_elements(int64_t N, const int64_t* offsets, int64_t B,
                           const double* F, const double* c, const double* Qp,
                           const double* H, const double* d, const double* Rp, const double* y,
                           const double* m0, const double* P0, double* xf, double* Pf)
{
    (void)N;
    for (int64_t b = 0; b < B; ++b) {
        int64_t k0 = offsets[b], k1 = offsets[b + 1];
        orc_felem acc, e;
        orc_filter_prior_element(m0 + 5 * b, P0 + 25 * b, &acc);
        memcpy(xf + 5 * k0, acc.b, sizeof(double) * 5);
        memcpy(Pf + 25 * k0, acc.C, sizeof(double) * 25);
        for (int64_t k = k0 + 1; k < k1; ++k) {
            int st = orc_filter_element(F + 25 * (k - 1), c + 5 * (k - 1), Qp + 25 * (k - 1),
                                        H + 10 * k, d + 2 * k, Rp + 4 * k, y + 2 * k, &e);
            if (st != ORC_OK) return st;
            st = orc_filter_combine(&acc, &e, &acc);
            if (st != ORC_OK) return st;
            memcpy(xf + 5 * k, acc.b, sizeof(double) * 5);
            memcpy(Pf + 25 * k, acc.C, sizeof(double) * 25);
        }
    }
    return ORC_OK;
}

/* Smoothing means/covariances as the suffix products a_k (x) ... (x) a_n
 * (Sec. 2), evaluated by a sequential right fold. */
int orc_smoother_by_elements(int64_t N, const int64_t* offsets, int64_t B,
                             const double* F, const double* c, const double* Qp,
                             const double* xf, const double* Pf, double* xs, double* Ps)
{
    (void)N;
    for (int64_t b = 0; b < B; ++b) {
        int64_t k0 = offsets[b], k1 = offsets[b + 1];
        orc_selem acc, e;
        orc_smoother_last_element(xf + 5 * (k1 - 1), Pf + 25 * (k1 - 1), &acc);
        memcpy(xs + 5 * (k1 - 1), acc.g, sizeof(double) * 5);
        memcpy(Ps + 25 * (k1 - 1), acc.L, sizeof(double) * 25);
        for (int64_t k = k1 - 2; k >= k0; --k) {
            int st = orc_smoother_element(xf + 5 * k, Pf + 25 * k, F + 25 * k, c + 5 * k, Qp + 25 * k, &e);
            if (st != ORC_OK) return st;
            orc_smoother_combine(&e, &acc, &acc);
            memcpy(xs + 5 * k, acc.g, sizeof(double) * 5);
            memcpy(Ps + 25 * k, acc.L, sizeof(double) * 25);
        }
    }
    return ORC_OK;
}
