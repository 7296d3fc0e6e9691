// Team-parallel forms of the associative operators for the narrow levels of
// the scan trees.
//
// A team is tau consecutive lanes of one warp (tau in {2, 4, 8, 16, 32}).
// The team applies one operator with all operands in shared memory: output
// entries of each 5x5 product are spread round-robin over the team, the small
// sequential factorisations run on the team's first lane, and __syncwarp
// orders the steps. Results go to team scratch first and are copied out at
// the end, so the output may alias either operand. The arithmetic is the same
// as the single-thread operators of pes_ops.cuh (Eq. 15 through
// D = (C_i^{-1} + J_j)^{-1}, Eq. 19), evaluated in a different order.
#pragma once

#include "pes_ops.cuh"

namespace pes {

// Scratch of one team, in shared memory.
template <typename T>
struct TeamScratch {
    T L[25], U[25], V[25], ru[5];
    T JL[25], K[15], D[15];
    T AD[25], W[25], JD[25], K2[15], K2A[25];
    T bt[5], u[5], Du[5], z[5];
    T oA[25], oC[15], oJ[15], ob[5], oeta[5];
};

struct Team {
    int r;          // rank in the team
    int tau;        // team size
    unsigned mask;  // the team's lanes in the warp
    PES_DEV void sync() const { __syncwarp(mask); }
};

PES_DEV Team make_team(int tau)
{
    Team tm;
    const int lane = threadIdx.x & 31;
    tm.tau = tau;
    tm.r = lane % tau;
    const unsigned base = (tau == 32) ? 0xffffffffu : ((1u << tau) - 1u);
    tm.mask = (tau == 32) ? 0xffffffffu : (base << (lane - tm.r));
    return tm;
}

// full-matrix entry (i, j) of a packed symmetric 5x5
template <typename T>
PES_DEV T sym_at(const T* S, int i, int j)
{
    return S[i <= j ? (i * 5 - i * (i - 1) / 2 + (j - i)) : (j * 5 - j * (j - 1) / 2 + (i - j))];
}

// packed (row, col) of packed index e, row <= col
PES_DEV void packed_rc(int e, int& i, int& j)
{
    // rows start at 0, 5, 9, 12, 14
    i = (e >= 5) + (e >= 9) + (e >= 12) + (e >= 14);
    const int start = i * 5 - i * (i - 1) / 2;
    j = i + (e - start);
}

// Team form of info_update_cov: D = (P^{-1} + J)^{-1} = L (I + L^T J L)^{-1} L^T.
template <typename T>
PES_DEV void team_info_update_cov(const T* P, const T* J, TeamScratch<T>& s, const Team& tm)
{
    if (tm.r == 0) chol_psd(P, s.L);
    tm.sync();
    for (int e = tm.r; e < 25; e += tm.tau) {   // JL = J L
        const int i = e / 5, j = e % 5;
        T acc = T(0);
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(sym_at(J, i, l), s.L[l * 5 + j], acc);
        s.JL[e] = acc;
    }
    tm.sync();
    for (int e = tm.r; e < 15; e += tm.tau) {   // K = I + L^T J L
        int i, j;
        packed_rc(e, i, j);
        T acc = (i == j) ? T(1) : T(0);
        for (int l = i; l < 5; ++l) acc = fma(s.L[l * 5 + i], s.JL[l * 5 + j], acc);
        s.K[e] = acc;
    }
    tm.sync();
    if (tm.r == 0) chol_pd(s.K, s.U, s.ru);
    tm.sync();
    for (int row = tm.r; row < 5; row += tm.tau) {   // V = L U^{-T}, row by row
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            T acc = s.L[row * 5 + j];
            for (int l = 0; l < j; ++l) acc = fma(-s.V[row * 5 + l], s.U[j * 5 + l], acc);
            s.V[row * 5 + j] = acc * s.ru[j];
        }
    }
    tm.sync();
    for (int e = tm.r; e < 15; e += tm.tau) {   // D = V V^T
        int i, j;
        packed_rc(e, i, j);
        T acc = T(0);
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(s.V[i * 5 + l], s.V[j * 5 + l], acc);
        s.D[e] = acc;
    }
    tm.sync();
}

// out = ai (x) aj, Eq. 15, by a team.
template <typename T>
PES_DEV void team_combine_filter(const FElem<T>& ai, const FElem<T>& aj, FElem<T>& out, TeamScratch<T>& s,
                                 const Team& tm)
{
    for (int i = tm.r; i < 5; i += tm.tau) s.bt[i] = ai.b[i] - aj.xr[i];
    team_info_update_cov(ai.C, aj.J, s, tm);
    for (int e = tm.r; e < 25; e += tm.tau) {   // AD = A_j D, JD = J_j D
        const int i = e / 5, j = e % 5;
        T a1 = T(0), a2 = T(0);
#pragma unroll
        for (int l = 0; l < 5; ++l) {
            a1 = fma(aj.A[i * 5 + l], sym_at(s.D, l, j), a1);
            a2 = fma(sym_at(aj.J, i, l), sym_at(s.D, l, j), a2);
        }
        s.AD[e] = a1;
        s.JD[e] = a2;
    }
    for (int i = tm.r; i < 5; i += tm.tau) {   // u = eta_j - J_j bt
        T acc = aj.eta[i];
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(-sym_at(aj.J, i, l), s.bt[l], acc);
        s.u[i] = acc;
    }
    tm.sync();
    for (int e = tm.r; e < 25; e += tm.tau) {   // W = A_j - (A_j D) J_j
        const int i = e / 5, j = e % 5;
        T acc = aj.A[e];
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(-s.AD[i * 5 + l], sym_at(aj.J, l, j), acc);
        s.W[e] = acc;
    }
    for (int e = tm.r; e < 15; e += tm.tau) {   // K2 = J_j - (J_j D) J_j ; C_ij = (A_j D) A_j^T + C_j
        int i, j;
        packed_rc(e, i, j);
        T k2 = aj.J[e], c = aj.C[e];
#pragma unroll
        for (int l = 0; l < 5; ++l) {
            k2 = fma(-s.JD[i * 5 + l], sym_at(aj.J, l, j), k2);
            c = fma(s.AD[i * 5 + l], aj.A[j * 5 + l], c);
        }
        s.K2[e] = k2;
        s.oC[e] = c;
    }
    for (int i = tm.r; i < 5; i += tm.tau) {   // Du = D u
        T acc = T(0);
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(sym_at(s.D, i, l), s.u[l], acc);
        s.Du[i] = acc;
    }
    tm.sync();
    for (int e = tm.r; e < 25; e += tm.tau) {   // A_ij = W A_i ; K2A = K2 A_i
        const int i = e / 5, j = e % 5;
        T a1 = T(0), a2 = T(0);
#pragma unroll
        for (int l = 0; l < 5; ++l) {
            a1 = fma(s.W[i * 5 + l], ai.A[l * 5 + j], a1);
            a2 = fma(sym_at(s.K2, i, l), ai.A[l * 5 + j], a2);
        }
        s.oA[e] = a1;
        s.K2A[e] = a2;
    }
    for (int i = tm.r; i < 5; i += tm.tau) {   // z = u - J_j D u ; b_ij = A_j (bt + D u) + b_j
        T jdu = T(0), ab = aj.b[i];
#pragma unroll
        for (int l = 0; l < 5; ++l) {
            jdu = fma(sym_at(aj.J, i, l), s.Du[l], jdu);
            ab = fma(aj.A[i * 5 + l], s.bt[l] + s.Du[l], ab);
        }
        s.z[i] = s.u[i] - jdu;
        s.ob[i] = ab;
    }
    tm.sync();
    for (int e = tm.r; e < 15; e += tm.tau) {   // J_ij = A_i^T K2A + J_i
        int i, j;
        packed_rc(e, i, j);
        T acc = ai.J[e];
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(ai.A[l * 5 + i], s.K2A[l * 5 + j], acc);
        s.oJ[e] = acc;
    }
    for (int i = tm.r; i < 5; i += tm.tau) {   // eta_ij = A_i^T z + eta_i
        T acc = ai.eta[i];
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(ai.A[l * 5 + i], s.z[l], acc);
        s.oeta[i] = acc;
    }
    tm.sync();
    // copy out (out may alias ai or aj; every read of them is done)
    for (int e = tm.r; e < 25; e += tm.tau) out.A[e] = s.oA[e];
    for (int e = tm.r; e < 15; e += tm.tau) {
        out.C[e] = s.oC[e];
        out.J[e] = s.oJ[e];
    }
    for (int i = tm.r; i < 5; i += tm.tau) {
        out.b[i] = s.ob[i];
        out.eta[i] = s.oeta[i];
        out.xr[i] = ai.xr[i];
    }
    tm.sync();
}

// out = (m, P) (x) a by a team (see apply_filter).
template <typename T>
PES_DEV void team_apply_filter(const Gauss<T>& g, const FElem<T>& a, Gauss<T>& out, TeamScratch<T>& s,
                               const Team& tm)
{
    for (int i = tm.r; i < 5; i += tm.tau) s.bt[i] = g.m[i] - a.xr[i];
    team_info_update_cov(g.P, a.J, s, tm);
    for (int e = tm.r; e < 25; e += tm.tau) {   // AD = A D
        const int i = e / 5, j = e % 5;
        T acc = T(0);
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(a.A[i * 5 + l], sym_at(s.D, l, j), acc);
        s.AD[e] = acc;
    }
    for (int i = tm.r; i < 5; i += tm.tau) {   // u = eta - J dm
        T acc = a.eta[i];
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(-sym_at(a.J, i, l), s.bt[l], acc);
        s.u[i] = acc;
    }
    tm.sync();
    for (int i = tm.r; i < 5; i += tm.tau) {   // w = dm + D u
        T acc = s.bt[i];
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(sym_at(s.D, i, l), s.u[l], acc);
        s.Du[i] = acc;
    }
    for (int e = tm.r; e < 15; e += tm.tau) {   // P' = (A D) A^T + C
        int i, j;
        packed_rc(e, i, j);
        T acc = a.C[e];
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(s.AD[i * 5 + l], a.A[j * 5 + l], acc);
        s.oC[e] = acc;
    }
    tm.sync();
    for (int i = tm.r; i < 5; i += tm.tau) {   // m' = A w + b
        T acc = a.b[i];
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(a.A[i * 5 + l], s.Du[l], acc);
        s.ob[i] = acc;
    }
    tm.sync();
    for (int e = tm.r; e < 15; e += tm.tau) out.P[e] = s.oC[e];
    for (int i = tm.r; i < 5; i += tm.tau) out.m[i] = s.ob[i];
    tm.sync();
}

// out = ai (x) aj, Eq. 19, by a team.
template <typename T>
PES_DEV void team_combine_smoother(const SElem<T>& ai, const SElem<T>& aj, SElem<T>& out, TeamScratch<T>& s,
                                   const Team& tm)
{
    for (int e = tm.r; e < 25; e += tm.tau) {   // E = E_i E_j ; EL = E_i L_j
        const int i = e / 5, j = e % 5;
        T a1 = T(0), a2 = T(0);
#pragma unroll
        for (int l = 0; l < 5; ++l) {
            a1 = fma(ai.E[i * 5 + l], aj.E[l * 5 + j], a1);
            a2 = fma(ai.E[i * 5 + l], sym_at(aj.L, l, j), a2);
        }
        s.oA[e] = a1;
        s.AD[e] = a2;
    }
    for (int i = tm.r; i < 5; i += tm.tau) {   // g = E_i (g_j - xr_i) + g_i
        T acc = ai.g[i];
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(ai.E[i * 5 + l], aj.g[l] - ai.xr[l], acc);
        s.ob[i] = acc;
    }
    tm.sync();
    for (int e = tm.r; e < 15; e += tm.tau) {   // L = (E_i L_j) E_i^T + L_i
        int i, j;
        packed_rc(e, i, j);
        T acc = ai.L[e];
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(s.AD[i * 5 + l], ai.E[j * 5 + l], acc);
        s.oC[e] = acc;
    }
    tm.sync();
    for (int e = tm.r; e < 25; e += tm.tau) out.E[e] = s.oA[e];
    for (int e = tm.r; e < 15; e += tm.tau) out.L[e] = s.oC[e];
    for (int i = tm.r; i < 5; i += tm.tau) {
        out.g[i] = s.ob[i];
        out.xr[i] = aj.xr[i];
    }
    tm.sync();
}

// out = a (x) (m, P), Eq. 19 with a Gaussian right operand, by a team.
template <typename T>
PES_DEV void team_apply_smoother(const SElem<T>& a, const Gauss<T>& g, Gauss<T>& out, TeamScratch<T>& s,
                                 const Team& tm)
{
    for (int e = tm.r; e < 25; e += tm.tau) {   // EP = E P
        const int i = e / 5, j = e % 5;
        T acc = T(0);
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(a.E[i * 5 + l], sym_at(g.P, l, j), acc);
        s.AD[e] = acc;
    }
    for (int i = tm.r; i < 5; i += tm.tau) {   // m' = E (m - xr) + g
        T acc = a.g[i];
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(a.E[i * 5 + l], g.m[l] - a.xr[l], acc);
        s.ob[i] = acc;
    }
    tm.sync();
    for (int e = tm.r; e < 15; e += tm.tau) {   // P' = (E P) E^T + L
        int i, j;
        packed_rc(e, i, j);
        T acc = a.L[e];
#pragma unroll
        for (int l = 0; l < 5; ++l) acc = fma(s.AD[i * 5 + l], a.E[j * 5 + l], acc);
        s.oC[e] = acc;
    }
    tm.sync();
    for (int e = tm.r; e < 15; e += tm.tau) out.P[e] = s.oC[e];
    for (int i = tm.r; i < 5; i += tm.tau) out.m[i] = s.ob[i];
    tm.sync();
}

}  // namespace pes
