/*
 * CPU FP64 oracle of the parallel iterated extended / cubature Kalman smoothers.
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline of the benchmark, never by the product library. See oracle.c.
 */
#ifndef PES_ORACLE_H
#define PES_ORACLE_H

#include <stdint.h>

#define ORC_OK 0
#define ORC_NOT_PD 2
#define ORC_NOT_CONVERGED 4

#define ORC_IEKS 0
#define ORC_CUBATURE 1
#define ORC_UNSCENTED 2
#define ORC_GAUSS_HERMITE 3

#define ORC_MODEL_CT_BEARINGS 0
#define ORC_MODEL_LINEAR 1

/* |omega dt| below which the coordinated-turn coefficients use their series
 * (kept through a^4: truncation below 2e-16 relative up to here, whereas the
 * closed forms lose up to ~1e-8 relative to cancellation near 1e-4) */
#define ORC_CT_SERIES 1e-2

typedef struct {
    int kind;       /* ORC_MODEL_CT_BEARINGS or ORC_MODEL_LINEAR */
    int q_form;     /* CT: 0 = diag(0,0,q_c dt,q_c dt,q_w dt); 1 = continuous white acceleration */
    double dt, q_c, q_w, r_std;
    const double* sensors; /* [1 or B][4] = s1x, s1y, s2x, s2y */
    int sensors_per_traj;
    /* linear model x' = F x + c + q, y = H x + d + r (full matrices, row-major) */
    double F[25], c[5], Q[25], H[10], d[2], R[4];
    /* unscented rule (ORC_UNSCENTED): spread alpha, prior-knowledge beta, kappa */
    double ut_alpha, ut_beta, ut_kappa;
    /* Levenberg-Marquardt damping of the iteration (0: none): every state gets
     * the pseudo-measurement xbar_k = x_k + e, e ~ N(0, I / lm_lambda) */
    double lm_lambda;
} orc_model;

typedef struct { double A[25], b[5], C[25], eta[5], J[25]; } orc_felem;
typedef struct { double E[25], g[5], L[25]; } orc_selem;

double orc_wrap(double a);
void orc_ct_f(const double x[5], double dt, double out[5]);
void orc_ct_jacobian(const double x[5], double dt, double F[25]);
void orc_bearings_h(const double x[5], const double s[4], double out[2]);
void orc_bearings_jacobian(const double x[5], const double s[4], double H[10]);
void orc_process_noise(const orc_model* m, double Q[25]);
void orc_measurement_noise(const orc_model* m, double R[4]);

int orc_slr(const orc_model* m, int which, int64_t b, const double xbar[5], const double Pbar[25],
            double* G, double* offset, double* Lam);
/* The same regression with the unscented rule of parameters (alpha, beta,
 * kappa): lambda = alpha^2 (n + kappa) - n, points xbar and
 * xbar +- sqrt(n + lambda) (chol Pbar) e_i, mean weights lambda / (n + lambda)
 * (centre) and 1 / (2 (n + lambda)), covariance weights the same except
 * lambda / (n + lambda) + 1 - alpha^2 + beta at the centre. */
int orc_slr_unscented(const orc_model* m, int which, int64_t b, const double xbar[5], const double Pbar[25],
                      double* G, double* offset, double* Lam);
/* The same regression with the third-order Gauss-Hermite product rule:
 * 3^n points xbar + chol(Pbar) xi, xi in {-sqrt 3, 0, sqrt 3}^n, weights the
 * products of 1/6, 2/3, 1/6 (exact for polynomials of degree 5 in each
 * coordinate of a standard Gaussian). */
int orc_slr_gauss_hermite(const orc_model* m, int which, int64_t b, const double xbar[5], const double Pbar[25],
                          double* G, double* offset, double* Lam);
int orc_linearize(const orc_model* m, int method, int64_t N, const int64_t* offsets, int64_t B,
                  const double* xbar, const double* Pbar, const double* y,
                  double* F, double* c, double* Qp, double* H, double* d, double* Rp, double* y_used);
int orc_kf_rts(int64_t N, const int64_t* offsets, int64_t B,
               const double* F, const double* c, const double* Qp,
               const double* H, const double* d, const double* Rp, const double* y,
               const double* m0, const double* P0,
               double* xf, double* Pf, double* xs, double* Ps);
/* log p(y_1..y_T) of each trajectory under the affine model (Sec. 2: the
 * marginal likelihood the filtering recursion carries), by the prediction
 * error decomposition: sum over k of log N(y_k; H_k m_k^- + d_k, S_k). */
int orc_kf_loglik(int64_t N, const int64_t* offsets, int64_t B,
                  const double* F, const double* c, const double* Qp,
                  const double* H, const double* d, const double* Rp, const double* y,
                  const double* m0, const double* P0, double* loglik);
/* orc_kf_rts with the Levenberg-Marquardt pseudo-measurements of the nominal
 * xbar [N][5] (covariance I / lambda) applied after each state's update
 * (lambda = 0: orc_kf_rts). */
int orc_kf_rts_damped(int64_t N, const int64_t* offsets, int64_t B,
                      const double* F, const double* c, const double* Qp,
                      const double* H, const double* d, const double* Rp, const double* y,
                      const double* m0, const double* P0, const double* xbar, double lambda,
                      double* xf, double* Pf, double* xs, double* Ps);
int orc_iterated_smoother(const orc_model* m, int method, int64_t N, const int64_t* offsets, int64_t B,
                          const double* y, const double* m0, const double* P0,
                          const double* x_init, const double* P_init, int max_iters, double tol,
                          double* x_out, double* P_out, int* iters_used, double* rel_history);

/* MAP objective of Eq. 4 per trajectory (positive definite Q), and the IEKS
 * with Levenberg-Marquardt steps whose damping adapts per trajectory (Sec. 3):
 * see oracle.c. */
int orc_map_cost(const orc_model* m, int64_t N, const int64_t* offsets, int64_t B, const double* y,
                 const double* m0, const double* P0, const double* x, double* cost);
int orc_iterated_smoother_lm(const orc_model* m, int64_t N, const int64_t* offsets, int64_t B, const double* y,
                             const double* m0, const double* P0, const double* x_init, int max_iters, double tol,
                             double lambda0, double nu, double* x_out, double* P_out, int* iters_used,
                             double* lambda_out, int* conv_iter, int* accepted);

int orc_filter_element(const double F[25], const double c[5], const double Qp[25],
                       const double H[10], const double d[2], const double Rp[4], const double y[2],
                       orc_felem* e);
void orc_filter_prior_element(const double m0[5], const double P0[25], orc_felem* e);
int orc_filter_combine(const orc_felem* ei, const orc_felem* ej, orc_felem* out);
int orc_smoother_element(const double xf[5], const double Pf[25], const double F[25], const double c[5],
                         const double Qp[25], orc_selem* e);
void orc_smoother_last_element(const double xf[5], const double Pf[25], orc_selem* e);
void orc_smoother_combine(const orc_selem* ei, const orc_selem* ej, orc_selem* out);
int orc_filter_by_elements(int64_t N, const int64_t* offsets, int64_t B,
                           const double* F, const double* c, const double* Qp,
                           const double* H, const double* d, const double* Rp, const double* y,
                           const double* m0, const double* P0, double* xf, double* Pf);
int orc_smoother_by_elements(int64_t N, const int64_t* offsets, int64_t B,
                             const double* F, const double* c, const double* Qp,
                             const double* xf, const double* Pf, double* xs, double* Ps);

#endif
