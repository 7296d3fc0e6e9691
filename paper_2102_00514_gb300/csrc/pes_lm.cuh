// Parameters of the Levenberg-Marquardt kernels (pes_lm.cu): the model in
// FP64 (the objective is evaluated in FP64 for either precision), the
// lane-major geometry of the smoother kernel, and per-trajectory accumulators.
#pragma once

#include "pes_model.cuh"

namespace pes {

struct LMParams {
    int64_t N;
    const int64_t* offsets;
    int B;
    int L, NL;
    int64_t cs;
    int kind;
    int sensors_per_traj;
    double dt;
    const double* sensors;   // device [1 or B][4]
    double F[25], c[5], H[10], d[2];   // linear model
    double Qi[15], Ri[3];              // inverses of Q and R (packed)
    double* cost;       // [B] objective at the nominal
    double* cost_new;   // [B] objective at the step
    double* num;        // [B] squared step
    double* den;        // [B] squared nominal
    int* reject;        // [B]
    int* accepted;      // [B] steps accepted so far
    int* conv_iter;     // [B] first converged iteration (0: none)
    int* unconv;        // trajectories not yet converged
};

// The objective of every trajectory at x, added into cost_out [B]; with xold
// also the squared step and squared nominal into p.num, p.den.
template <typename T>
cudaError_t launch_lm_cost(const LMParams& p, double* cost_out, const T* x, const T* xold, const T* y, const T* m0,
                           const T* P0, cudaStream_t st);
template <typename T>
cudaError_t launch_lm_decide(const LMParams& p, T* lam, int it, double tol, double nu, cudaStream_t st);
template <typename T>
cudaError_t launch_lm_restore(const LMParams& p, T* x, T* P, const T* xold, const T* Pold, cudaStream_t st);
template <typename T>
cudaError_t launch_lm_fill(T* lam, int B, double v, cudaStream_t st);

}  // namespace pes
