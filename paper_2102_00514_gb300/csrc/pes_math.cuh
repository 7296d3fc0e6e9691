// Register-resident small dense linear algebra for n_x = 5, n_y = 2.
//
// Every routine is fully unrolled over compile-time bounds so that the arrays
// below live in registers. Matrices are row-major (5x5: 25 scalars, 2x5: 10);
// symmetric matrices are packed upper-triangular row-major (5x5: 15, 2x2: 3).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define PES_DEV __device__ __forceinline__

namespace pes {

constexpr int NX = 5;
constexpr int NY = 2;
constexpr int NS = 15;   // packed 5x5 symmetric
constexpr int NS2 = 3;   // packed 2x2 symmetric

// packed upper index of entry (i, j) of a symmetric 5x5 matrix
__host__ __device__ constexpr int si(int i, int j)
{
    return (i <= j) ? (i * NX - i * (i - 1) / 2 + (j - i)) : (j * NX - j * (j - 1) / 2 + (i - j));
}
// packed index of a symmetric 2x2 matrix
__host__ __device__ constexpr int si2(int i, int j) { return i + j; }

template <typename T> PES_DEV T tsqrt(T x);
template <> PES_DEV float tsqrt<float>(float x) { return sqrtf(x); }
template <> PES_DEV double tsqrt<double>(double x) { return sqrt(x); }

// Reciprocal square root and reciprocal on the pivot chains of the
// factorisations: FP32 takes the hardware approximations (rsqrtf, and
// __fdividef for the reciprocal: a few ulp), FP64 the correctly rounded forms.
template <typename T> PES_DEV T trsqrt(T x);
template <> PES_DEV float trsqrt<float>(float x) { return rsqrtf(x); }
template <> PES_DEV double trsqrt<double>(double x) { return 1.0 / sqrt(x); }
template <typename T> PES_DEV T trcp(T x);
template <> PES_DEV float trcp<float>(float x) { return __fdividef(1.0f, x); }
template <> PES_DEV double trcp<double>(double x) { return 1.0 / x; }

// ---- products -------------------------------------------------------------

// C = A B (5x5)
template <typename T>
PES_DEV void mm(const T* A, const T* B, T* C)
{
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
        for (int j = 0; j < NX; ++j) {
            T s = A[i * NX] * B[j];
#pragma unroll
            for (int l = 1; l < NX; ++l) s = fma(A[i * NX + l], B[l * NX + j], s);
            C[i * NX + j] = s;
        }
}

// C = A S with S symmetric packed
template <typename T>
PES_DEV void m_s(const T* A, const T* S, T* C)
{
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
        for (int j = 0; j < NX; ++j) {
            T s = A[i * NX] * S[si(0, j)];
#pragma unroll
            for (int l = 1; l < NX; ++l) s = fma(A[i * NX + l], S[si(l, j)], s);
            C[i * NX + j] = s;
        }
}

// C = S A with S symmetric packed
template <typename T>
PES_DEV void s_m(const T* S, const T* A, T* C)
{
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
        for (int j = 0; j < NX; ++j) {
            T s = S[si(i, 0)] * A[j];
#pragma unroll
            for (int l = 1; l < NX; ++l) s = fma(S[si(i, l)], A[l * NX + j], s);
            C[i * NX + j] = s;
        }
}

// Out (sym) = A B^T + Add (sym), where the product is known to be symmetric;
// only the upper triangle is formed.
template <typename T>
PES_DEV void abt_sym_add(const T* A, const T* B, const T* Add, T* Out)
{
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
        for (int j = i; j < NX; ++j) {
            T s = Add[si(i, j)];
#pragma unroll
            for (int l = 0; l < NX; ++l) s = fma(A[i * NX + l], B[j * NX + l], s);
            Out[si(i, j)] = s;
        }
}

// Out (sym) = A^T B + Add (sym), product known to be symmetric
template <typename T>
PES_DEV void atb_sym_add(const T* A, const T* B, const T* Add, T* Out)
{
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
        for (int j = i; j < NX; ++j) {
            T s = Add[si(i, j)];
#pragma unroll
            for (int l = 0; l < NX; ++l) s = fma(A[l * NX + i], B[l * NX + j], s);
            Out[si(i, j)] = s;
        }
}

// y = A x (5x5)
template <typename T>
PES_DEV void mv(const T* A, const T* x, T* y)
{
#pragma unroll
    for (int i = 0; i < NX; ++i) {
        T s = A[i * NX] * x[0];
#pragma unroll
        for (int l = 1; l < NX; ++l) s = fma(A[i * NX + l], x[l], s);
        y[i] = s;
    }
}

// y = A^T x (5x5)
template <typename T>
PES_DEV void mtv(const T* A, const T* x, T* y)
{
#pragma unroll
    for (int i = 0; i < NX; ++i) {
        T s = A[i] * x[0];
#pragma unroll
        for (int l = 1; l < NX; ++l) s = fma(A[l * NX + i], x[l], s);
        y[i] = s;
    }
}

// y = S x (S symmetric packed)
template <typename T>
PES_DEV void sv(const T* S, const T* x, T* y)
{
#pragma unroll
    for (int i = 0; i < NX; ++i) {
        T s = S[si(i, 0)] * x[0];
#pragma unroll
        for (int l = 1; l < NX; ++l) s = fma(S[si(i, l)], x[l], s);
        y[i] = s;
    }
}

template <typename T>
PES_DEV void set_identity(T* A)
{
#pragma unroll
    for (int i = 0; i < NX * NX; ++i) A[i] = (i % (NX + 1) == 0) ? T(1) : T(0);
}

template <typename T>
PES_DEV void set_zero(T* a, int n)
{
    for (int i = 0; i < n; ++i) a[i] = T(0);
}

// ---- factorisations --------------------------------------------------------

// Semi-definite Cholesky S = L L^T (L lower, row-major 5x5, zeros above the
// diagonal). A pivot that is not positive (a singular or rounding-indefinite
// direction) leaves a zero column. Returns the number of such pivots.
template <typename T>
PES_DEV int chol_psd(const T* S, T* L)
{
    int zero_pivots = 0;
#pragma unroll
    for (int i = 0; i < NX * NX; ++i) L[i] = T(0);
#pragma unroll
    for (int j = 0; j < NX; ++j) {
        T s = S[si(j, j)];
#pragma unroll
        for (int l = 0; l < j; ++l) s = fma(-L[j * NX + l], L[j * NX + l], s);
        const bool ok = s > T(0);
        zero_pivots += ok ? 0 : 1;
        const T inv = ok ? trsqrt(s) : T(0);
        const T d = s * inv;
        L[j * NX + j] = d;
#pragma unroll
        for (int i = j + 1; i < NX; ++i) {
            T t = S[si(i, j)];
#pragma unroll
            for (int l = 0; l < j; ++l) t = fma(-L[i * NX + l], L[j * NX + l], t);
            L[i * NX + j] = t * inv;
        }
    }
    return zero_pivots;
}

// Cholesky of a matrix known to be positive definite: S = L L^T. Returns false
// when a pivot is not positive. Also returns the reciprocal diagonal.
template <typename T>
PES_DEV bool chol_pd(const T* S, T* L, T* rdiag)
{
    bool ok_all = true;
#pragma unroll
    for (int i = 0; i < NX * NX; ++i) L[i] = T(0);
#pragma unroll
    for (int j = 0; j < NX; ++j) {
        T s = S[si(j, j)];
#pragma unroll
        for (int l = 0; l < j; ++l) s = fma(-L[j * NX + l], L[j * NX + l], s);
        const bool ok = s > T(0);
        ok_all = ok_all && ok;
        const T inv = ok ? trsqrt(s) : T(1);
        const T d = ok ? s * inv : T(1);
        L[j * NX + j] = d;
        rdiag[j] = inv;
#pragma unroll
        for (int i = j + 1; i < NX; ++i) {
            T t = S[si(i, j)];
#pragma unroll
            for (int l = 0; l < j; ++l) t = fma(-L[i * NX + l], L[j * NX + l], t);
            L[i * NX + j] = t * inv;
        }
    }
    return ok_all;
}

// Solve (L L^T) X = B in place for 5 right-hand-side columns of B (5x5).
template <typename T>
PES_DEV void chol_solve_cols(const T* L, const T* rdiag, T* B)
{
#pragma unroll
    for (int c = 0; c < NX; ++c) {
#pragma unroll
        for (int i = 0; i < NX; ++i) {
            T s = B[i * NX + c];
#pragma unroll
            for (int l = 0; l < i; ++l) s = fma(-L[i * NX + l], B[l * NX + c], s);
            B[i * NX + c] = s * rdiag[i];
        }
#pragma unroll
        for (int i = NX - 1; i >= 0; --i) {
            T s = B[i * NX + c];
#pragma unroll
            for (int l = i + 1; l < NX; ++l) s = fma(-L[l * NX + i], B[l * NX + c], s);
            B[i * NX + c] = s * rdiag[i];
        }
    }
}

// D = (P^{-1} + J)^{-1} = L (I + L^T J L)^{-1} L^T with P = L L^T, for
// symmetric positive semi-definite P and J (both packed). The middle matrix
// has eigenvalues >= 1, so its Cholesky needs no pivoting; a singular P is
// handled by its semi-definite factor. This is the symmetric form of
// (I + P J)^{-1} P used by both associative operators.
template <typename T>
PES_DEV void info_update_cov(const T* P, const T* J, T* D)
{
    T L[NX * NX];
    chol_psd(P, L);
    // K = I + L^T J L  (symmetric)
    T JL[NX * NX];
    s_m(J, L, JL);
    T K[NS];
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
        for (int j = i; j < NX; ++j) {
            T s = (i == j) ? T(1) : T(0);
#pragma unroll
            for (int l = i; l < NX; ++l) s = fma(L[l * NX + i], JL[l * NX + j], s);
            K[si(i, j)] = s;
        }
    // K = U U^T (U lower); V = L U^{-T} solves V U^T = L row by row
    T U[NX * NX], ru[NX];
    chol_pd(K, U, ru);
    T V[NX * NX];
#pragma unroll
    for (int r = 0; r < NX; ++r)
#pragma unroll
        for (int j = 0; j < NX; ++j) {
            // V[r][j] = (L[r][j] - sum_{l<j} V[r][l] U[j][l]) / U[j][j]
            T s = L[r * NX + j];
#pragma unroll
            for (int l = 0; l < j; ++l) s = fma(-V[r * NX + l], U[j * NX + l], s);
            V[r * NX + j] = s * ru[j];
        }
    // D = V V^T
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
        for (int j = i; j < NX; ++j) {
            T s = T(0);
#pragma unroll
            for (int l = 0; l < NX; ++l) s = fma(V[i * NX + l], V[j * NX + l], s);
            D[si(i, j)] = s;
        }
}

// inverse of a symmetric 2x2 (packed); returns false if not positive definite
template <typename T>
PES_DEV bool inv2_spd(const T* S, T* Si)
{
    const T det = S[0] * S[2] - S[1] * S[1];
    const bool ok = (det > T(0)) && (S[0] > T(0));
    const T r = ok ? trcp(det) : T(0);
    Si[0] = S[2] * r;
    Si[1] = -S[1] * r;
    Si[2] = S[0] * r;
    return ok;
}

}  // namespace pes
