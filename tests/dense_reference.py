"""Brute-force dense references used to pin the oracle (test infrastructure).

These are textbook computations on the stacked (batch) form of a short
trajectory. They are independent of the oracle's sequential filter/smoother
and of the CUDA path:

* Gaussian conditioning of the stacked affine model (exact smoothing and
  filtering distributions for given linearisation parameters, Eq. 11);
* one Gauss-Newton step of the MAP problem (the IEKS iteration, Sec. 3).
"""
from __future__ import annotations

import numpy as np


def stacked_prior(F, c, Qp, m0, P0):
    """Prior mean/covariance of x_{0:T} for x_k = F_{k-1} x_{k-1} + c_{k-1} + q,
    q ~ N(0, Qp_{k-1}), x_0 ~ N(m0, P0). F: [T][5][5] (F[k] maps k -> k+1)."""
    T = len(F)
    n = 5
    mu = np.zeros((T + 1) * n)
    S = np.zeros(((T + 1) * n, (T + 1) * n))
    mu[:n] = m0
    S[:n, :n] = P0
    for k in range(1, T + 1):
        Fk = F[k - 1]
        sl, pl = slice(k * n, (k + 1) * n), slice((k - 1) * n, k * n)
        mu[sl] = Fk @ mu[pl] + c[k - 1]
        # Cov(x_k, x_j) = F Cov(x_{k-1}, x_j) for j < k
        S[sl, :k * n] = Fk @ S[pl, :k * n]
        S[:k * n, sl] = S[sl, :k * n].T
        S[sl, sl] = Fk @ S[pl, pl] @ Fk.T + Qp[k - 1]
    return mu, S


def condition(mu, S, H, d, R, y, upto=None):
    """Condition N(mu, S) of the stacked x_{0:T} on y_k = H_k x_k + d_k + r,
    r ~ N(0, R_k), k = 1..upto (default all). H: [T+1][2][5] (index 0 unused)."""
    n, m = 5, 2
    T = len(H) - 1
    upto = T if upto is None else upto
    if upto == 0:
        return mu.copy(), S.copy()
    Hs = np.zeros((upto * m, (T + 1) * n))
    ds = np.zeros(upto * m)
    ys = np.zeros(upto * m)
    Rs = np.zeros((upto * m, upto * m))
    for k in range(1, upto + 1):
        r = slice((k - 1) * m, k * m)
        Hs[r, k * n:(k + 1) * n] = H[k]
        ds[r] = d[k]
        ys[r] = y[k]
        Rs[r, r] = R[k]
    G = Hs @ S @ Hs.T + Rs
    K = np.linalg.solve(G, Hs @ S).T
    mpost = mu + K @ (ys - Hs @ mu - ds)
    Spost = S - K @ Hs @ S
    return mpost, 0.5 * (Spost + Spost.T)


def dense_log_evidence(F, c, Qp, H, d, R, y, m0, P0):
    """log p(y_1..y_T) of the stacked affine model: y stacked is Gaussian with
    mean Hs mu + ds and covariance Hs S Hs^T + Rs."""
    mu, S = stacked_prior(F, c, Qp, m0, P0)
    n, m = 5, 2
    T = len(H) - 1
    if T == 0:
        return 0.0
    Hs = np.zeros((T * m, (T + 1) * n))
    ds = np.zeros(T * m)
    ys = np.zeros(T * m)
    Rs = np.zeros((T * m, T * m))
    for k in range(1, T + 1):
        r = slice((k - 1) * m, k * m)
        Hs[r, k * n:(k + 1) * n] = H[k]
        ds[r] = d[k]
        ys[r] = y[k]
        Rs[r, r] = R[k]
    G = Hs @ S @ Hs.T + Rs
    e = ys - Hs @ mu - ds
    sign, logdet = np.linalg.slogdet(G)
    assert sign > 0
    return float(-0.5 * (e @ np.linalg.solve(G, e) + logdet + T * m * np.log(2 * np.pi)))


def dense_smoother(F, c, Qp, H, d, R, y, m0, P0):
    """Smoothed means [T+1][5] and covariances [T+1][5][5]."""
    mu, S = stacked_prior(F, c, Qp, m0, P0)
    mp, Sp = condition(mu, S, H, d, R, y)
    T = len(F)
    xs = mp.reshape(T + 1, 5)
    Ps = np.stack([Sp[k * 5:(k + 1) * 5, k * 5:(k + 1) * 5] for k in range(T + 1)])
    return xs, Ps


def dense_filter(F, c, Qp, H, d, R, y, m0, P0):
    """Filtered means/covariances: marginal of x_k given y_{1:k}."""
    mu, S = stacked_prior(F, c, Qp, m0, P0)
    T = len(F)
    xf = np.zeros((T + 1, 5))
    Pf = np.zeros((T + 1, 5, 5))
    for k in range(T + 1):
        mp, Sp = condition(mu, S, H, d, R, y, upto=k)
        xf[k] = mp[k * 5:(k + 1) * 5]
        Pf[k] = Sp[k * 5:(k + 1) * 5, k * 5:(k + 1) * 5]
    return xf, Pf


def gauss_newton_step(x, f, fjac, h, hjac, Q, R, y, m0, P0, damping=0.0):
    """One Gauss-Newton step of the MAP problem
        |x_0 - m0|^2_{P0^-1} + sum_k |x_k - f(x_{k-1})|^2_{Q^-1} + sum_k |y_k - h(x_k)|^2_{R^-1}
    about the trajectory x [T+1][5] (Q positive definite); with damping > 0 the
    Levenberg-Marquardt step (J^T W J + damping I) dx = -J^T W r. Returns the
    new trajectory and the gradient of the objective at x."""
    T = len(x) - 1
    n, m = 5, 2
    nv = (T + 1) * n
    rows = []
    res = []
    Wb = []
    # prior
    Jp = np.zeros((n, nv)); Jp[:, :n] = np.eye(n)
    rows.append(Jp); res.append(x[0] - m0); Wb.append(np.linalg.inv(P0))
    Qi = np.linalg.inv(Q)
    Ri = np.linalg.inv(R)
    for k in range(1, T + 1):
        J = np.zeros((n, nv))
        J[:, k * n:(k + 1) * n] = np.eye(n)
        J[:, (k - 1) * n:k * n] = -fjac(x[k - 1])
        rows.append(J); res.append(x[k] - f(x[k - 1])); Wb.append(Qi)
    for k in range(1, T + 1):
        J = np.zeros((m, nv))
        J[:, k * n:(k + 1) * n] = -hjac(x[k])
        rows.append(J); res.append(y[k] - h(x[k])); Wb.append(Ri)
    Jm = np.vstack(rows)
    r = np.concatenate(res)
    W = np.zeros((len(r), len(r)))
    o = 0
    for w in Wb:
        s = w.shape[0]
        W[o:o + s, o:o + s] = w
        o += s
    A = Jm.T @ W @ Jm
    g = Jm.T @ W @ r
    dx = -np.linalg.solve(A + damping * np.eye(nv), g)
    return x + dx.reshape(T + 1, n), 2.0 * g


def map_objective(x, f, h, Q, R, y, m0, P0):
    """The MAP objective of the model (without the factor 1/2):
        |x_0 - m0|^2_{P0^-1} + sum_k |x_k - f(x_{k-1})|^2_{Q^-1} + sum_k |y_k - h(x_k)|^2_{R^-1}
    for a trajectory x [T+1][5] (Q positive definite)."""
    T = len(x) - 1
    e0 = x[0] - m0
    J = float(e0 @ np.linalg.solve(P0, e0))
    for k in range(1, T + 1):
        e = x[k] - f(x[k - 1])
        J += float(e @ np.linalg.solve(Q, e))
        r = y[k] - h(x[k])
        J += float(r @ np.linalg.solve(R, r))
    return J
