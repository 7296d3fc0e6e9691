"""Pins for the oracle's filter/smoother, elements and operators.

* The sequential KF + RTS (the definition) equals dense Gaussian conditioning
  of the stacked affine model (Eq. 11), also with a singular Q.
* A scalar random walk reaches the closed-form steady-state Riccati variance.
* The paper's elements and operators (Eqs. 13-19), folded sequentially, equal
  the definition; the operators are associative and have identities.
* For a linear-Gaussian model one iteration is exact and a second changes nothing.
* The filter's log-likelihood equals the log-density of the stacked measurement
  vector (brute force), and its increments are the one-step predictive densities.
"""
import numpy as np
import pytest

import oracle
from tests.dense_reference import dense_filter, dense_log_evidence, dense_smoother

RNG = np.random.default_rng(20210201)


def rand_spd(n, rng, scale=1.0, rank=None):
    rank = n if rank is None else rank
    A = rng.standard_normal((n, rank))
    return scale * (A @ A.T + (1e-3 * np.eye(n) if rank == n else 0))


def random_linear_lin(T, rng, singular_q=False):
    """Random per-step affine parameters in the oracle's SoA layout (packed)."""
    N = T + 1
    F = np.zeros((N, 5, 5)); c = np.zeros((N, 5)); Q = np.zeros((N, 5, 5))
    H = np.zeros((N, 2, 5)); d = np.zeros((N, 2)); R = np.zeros((N, 2, 2))
    for k in range(N):
        if k < T:
            F[k] = np.eye(5) + 0.3 * rng.standard_normal((5, 5))
            c[k] = rng.standard_normal(5)
            Q[k] = rand_spd(5, rng, 0.1, rank=3 if singular_q else None)
        if k > 0:
            H[k] = rng.standard_normal((2, 5))
            d[k] = rng.standard_normal(2)
            R[k] = rand_spd(2, rng, 0.2)
    y = np.zeros((N, 2))
    y[1:] = rng.standard_normal((T, 2))
    lin = dict(F=F.reshape(N, 25).T.copy(), c=c.T.copy(), Qp=oracle.sym_packed(Q).T.copy(),
               H=H.reshape(N, 10).T.copy(), d=d.T.copy(), Rp=oracle.sym_packed(R).T.copy())
    m0 = rng.standard_normal((1, 5))
    P0 = oracle.sym_packed(rand_spd(5, rng))[None]
    return lin, y.T.copy(), m0, P0, (F, c, Q, H, d, R, y)


@pytest.mark.parametrize("singular_q", [False, True])
@pytest.mark.parametrize("T", [1, 2, 7, 25])
def test_kf_rts_equals_dense_conditioning(T, singular_q):
    lin, y, m0, P0, (F, c, Q, H, d, R, yy) = random_linear_lin(T, RNG, singular_q)
    off = np.array([0, T + 1])
    out = oracle.kf_rts(off, lin, y, m0, P0)
    P0f = oracle.sym_full(P0[0], 5)
    xs, Ps = dense_smoother(F[:T], c[:T], Q[:T], H, d, R, yy, m0[0], P0f)
    xf, Pf = dense_filter(F[:T], c[:T], Q[:T], H, d, R, yy, m0[0], P0f)
    np.testing.assert_allclose(out["xs"].T, xs, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(oracle.sym_full(out["Ps"].T, 5), Ps, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(out["xf"].T, xf, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(oracle.sym_full(out["Pf"].T, 5), Pf, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("singular_q", [False, True])
@pytest.mark.parametrize("T", [1, 2, 7, 25])
def test_loglik_equals_dense_log_evidence(T, singular_q):
    lin, y, m0, P0, (F, c, Q, H, d, R, yy) = random_linear_lin(T, RNG, singular_q)
    ll = oracle.kf_loglik(np.array([0, T + 1]), lin, y, m0, P0)
    ref = dense_log_evidence(F[:T], c[:T], Q[:T], H, d, R, yy, m0[0], oracle.sym_full(P0[0], 5))
    assert abs(ll[0] - ref) < 1e-9 * max(1.0, abs(ref))


def test_loglik_increment_is_the_predictive_density():
    # log p(y_{1:T}) - log p(y_{1:T-1}) = log N(y_T; H m_T^- + d, H P_T^- H^T + R)
    T = 9
    lin, y, m0, P0, (F, c, Q, H, d, R, yy) = random_linear_lin(T, RNG)
    full = oracle.kf_loglik(np.array([0, T + 1]), lin, y, m0, P0)[0]
    cut = {k: v[:, :T].copy() for k, v in lin.items()}
    short = oracle.kf_loglik(np.array([0, T]), cut, y[:, :T].copy(), m0, P0)[0]
    out = oracle.kf_rts(np.array([0, T]), cut, y[:, :T].copy(), m0, P0)
    m = out["xf"][:, T - 1]
    P = oracle.sym_full(out["Pf"][:, T - 1], 5)
    mp = F[T - 1] @ m + c[T - 1]
    Pp = F[T - 1] @ P @ F[T - 1].T + Q[T - 1]
    S = H[T] @ Pp @ H[T].T + R[T]
    e = yy[T] - H[T] @ mp - d[T]
    dens = -0.5 * (e @ np.linalg.solve(S, e) + np.log(np.linalg.det(S)) + 2 * np.log(2 * np.pi))
    assert abs((full - short) - dens) < 1e-10 * max(1.0, abs(dens))


def test_loglik_of_a_batch_is_per_trajectory():
    parts = [random_linear_lin(T, RNG) for T in (3, 1, 6)]
    lls = [oracle.kf_loglik(np.array([0, T + 1]), p[0], p[1], p[2], p[3])[0] for T, p in zip((3, 1, 6), parts)]
    lin = {k: np.concatenate([p[0][k] for p in parts], axis=1) for k in parts[0][0]}
    y = np.concatenate([p[1] for p in parts], axis=1)
    m0 = np.concatenate([p[2] for p in parts])
    P0 = np.concatenate([p[3] for p in parts])
    got = oracle.kf_loglik(np.array([0, 4, 6, 13]), lin, y, m0, P0)
    np.testing.assert_allclose(got, lls, rtol=1e-13)


@pytest.mark.parametrize("singular_q", [False, True])
def test_elements_fold_equals_definition(singular_q):
    """Eqs. 13-15 (prefix) and 17-19 (suffix) against the sequential KF/RTS."""
    T = 40
    lin, y, m0, P0, _ = random_linear_lin(T, RNG, singular_q)
    off = np.array([0, T + 1])
    a = oracle.kf_rts(off, lin, y, m0, P0)
    b = oracle.by_elements(off, lin, y, m0, P0)
    for key in ("xf", "Pf", "xs", "Ps"):
        np.testing.assert_allclose(b[key], a[key], rtol=1e-9, atol=1e-10, err_msg=key)


def test_scalar_random_walk_reaches_riccati_steady_state():
    """Decoupled random walks observed directly: the filtered variance tends to
    P = (-q + sqrt(q^2 + 4 q r)) / 2, the positive root of P^2 + q P - q r = 0."""
    T = 400
    N = T + 1
    q, r = 0.3, 0.7
    F = np.tile(np.eye(5).reshape(25, 1), (1, N))
    c = np.zeros((5, N))
    Qp = np.tile(oracle.sym_packed(q * np.eye(5))[:, None], (1, N))
    Hm = np.zeros((2, 5)); Hm[0, 0] = 1; Hm[1, 1] = 1
    H = np.tile(Hm.reshape(10, 1), (1, N)); H[:, 0] = 0
    d = np.zeros((2, N))
    Rp = np.tile(oracle.sym_packed(r * np.eye(2))[:, None], (1, N))
    y = RNG.standard_normal((2, N)); y[:, 0] = 0
    lin = dict(F=F, c=c, Qp=Qp, H=H, d=d, Rp=Rp)
    out = oracle.kf_rts(np.array([0, N]), lin, y, np.zeros((1, 5)), oracle.sym_packed(np.eye(5))[None])
    P_inf = (-q + np.sqrt(q * q + 4 * q * r)) / 2
    Pf = oracle.sym_full(out["Pf"][:, T], 5)
    assert abs(Pf[0, 0] - P_inf) < 1e-12 and abs(Pf[1, 1] - P_inf) < 1e-12
    # unobserved coordinates grow by q each step: 1 + T q
    assert abs(Pf[4, 4] - (1 + T * q)) < 1e-9
    # smoothed steady state in the middle: Ps = P - G^2 (P+q) + G^2 Ps with G = P/(P+q)
    G = P_inf / (P_inf + q)
    Ps_inf = (P_inf - G * G * (P_inf + q)) / (1 - G * G)
    Ps = oracle.sym_full(out["Ps"][:, T // 2], 5)
    assert abs(Ps[0, 0] - Ps_inf) < 1e-12


def random_felem(rng):
    A = 0.5 * rng.standard_normal((5, 5))
    return oracle.FElem.from_arrays(A, rng.standard_normal(5), rand_spd(5, rng, 0.5),
                                    rng.standard_normal(5), rand_spd(5, rng, 0.5))


def random_selem(rng):
    return oracle.SElem.from_arrays(0.5 * rng.standard_normal((5, 5)), rng.standard_normal(5),
                                    rand_spd(5, rng, 0.5))


def _close(d1, d2, tol):
    for k in d1:
        np.testing.assert_allclose(d1[k], d2[k], rtol=tol, atol=tol, err_msg=k)


def test_filter_operator_associative():
    for _ in range(20):
        a, b, c = random_felem(RNG), random_felem(RNG), random_felem(RNG)
        left = oracle.filter_combine(oracle.filter_combine(a, b), c)
        right = oracle.filter_combine(a, oracle.filter_combine(b, c))
        _close(left.as_dict(), right.as_dict(), 1e-11)


def test_smoother_operator_associative():
    for _ in range(20):
        a, b, c = random_selem(RNG), random_selem(RNG), random_selem(RNG)
        left = oracle.smoother_combine(oracle.smoother_combine(a, b), c)
        right = oracle.smoother_combine(a, oracle.smoother_combine(b, c))
        _close(left.as_dict(), right.as_dict(), 1e-12)


def test_operator_identities():
    e = oracle.FElem.from_arrays(np.eye(5), np.zeros(5), np.zeros((5, 5)), np.zeros(5), np.zeros((5, 5)))
    a = random_felem(RNG)
    _close(oracle.filter_combine(e, a).as_dict(), a.as_dict(), 1e-14)
    _close(oracle.filter_combine(a, e).as_dict(), a.as_dict(), 1e-14)
    es = oracle.SElem.from_arrays(np.eye(5), np.zeros(5), np.zeros((5, 5)))
    s = random_selem(RNG)
    _close(oracle.smoother_combine(es, s).as_dict(), s.as_dict(), 1e-15)
    _close(oracle.smoother_combine(s, es).as_dict(), s.as_dict(), 1e-15)


def test_prior_element_times_first_element_is_one_kalman_step():
    """a_0 (x) a_1 = Kalman predict + update from (m0, P0), written out here."""
    F = np.eye(5) + 0.2 * RNG.standard_normal((5, 5)); c = RNG.standard_normal(5)
    Q = rand_spd(5, RNG, 0.1, rank=2); H = RNG.standard_normal((2, 5)); d = RNG.standard_normal(2)
    R = rand_spd(2, RNG, 0.3); y = RNG.standard_normal(2)
    m0 = RNG.standard_normal(5); P0 = rand_spd(5, RNG)
    a1 = oracle.filter_element(F, c, Q, H, d, R, y)
    a0 = oracle.filter_prior_element(m0, P0)
    r = oracle.filter_combine(a0, a1).as_dict()
    mp = F @ m0 + c
    Pp = F @ P0 @ F.T + Q
    S = H @ Pp @ H.T + R
    K = Pp @ H.T @ np.linalg.inv(S)
    np.testing.assert_allclose(r["b"], mp + K @ (y - H @ mp - d), rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["C"], Pp - K @ S @ K.T, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(r["A"], 0, atol=0)
    np.testing.assert_allclose(r["J"], 0, atol=0)


def test_linear_model_one_iteration_exact_and_fixed_point():
    rng = np.random.default_rng(7)
    F = np.eye(5) + 0.1 * rng.standard_normal((5, 5)); c = 0.1 * rng.standard_normal(5)
    Q = rand_spd(5, rng, 0.01); H = rng.standard_normal((2, 5)); d = rng.standard_normal(2)
    R = rand_spd(2, rng, 0.1)
    model = oracle.Model.linear(F, c, Q, H, d, R)
    T = 12
    off = np.array([0, T + 1])
    y = rng.standard_normal((2, T + 1)); y[:, 0] = 0
    m0 = rng.standard_normal((1, 5)); P0 = oracle.sym_packed(rand_spd(5, rng))[None]
    P0f = oracle.sym_full(P0[0], 5)
    Ht = np.stack([H] * (T + 1)); dt_ = np.stack([d] * (T + 1)); Rt = np.stack([R] * (T + 1))
    xs, Ps = dense_smoother([F] * T, [c] * T, [Q] * T, Ht, dt_, Rt, y.T, m0[0], P0f)
    for method in (oracle.IEKS, oracle.CUBATURE):
        out = oracle.iterated_smoother(model, method, off, y, m0, P0, iters=2)
        np.testing.assert_allclose(out["x"].T, xs, rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(oracle.sym_full(out["P"].T, 5), Ps, rtol=1e-9, atol=1e-10)
        assert out["rel_history"][1] < 1e-12


def test_batched_equals_separate():
    from paper_2102_00514_gb300 import synth
    wl = synth.ct_bearings([30, 1, 17], seed=5, sensor_jitter=0.2, omega0_halfwidth=1.0)
    model = oracle.Model.from_workload(wl)
    off = wl["offsets"]
    for method in (oracle.IEKS, oracle.CUBATURE):
        allb = oracle.iterated_smoother(model, method, off, wl["y"], wl["m0"], wl["P0"], iters=3)
        for b in range(3):
            sl = slice(off[b], off[b + 1])
            mb = oracle.Model.from_workload(dict(wl, sensors=wl["sensors"][b:b + 1]))
            one = oracle.iterated_smoother(mb, method, np.array([0, off[b + 1] - off[b]]), wl["y"][:, sl],
                                           wl["m0"][b:b + 1], wl["P0"][b:b + 1], iters=3)
            np.testing.assert_allclose(allb["x"][:, sl], one["x"], rtol=1e-13, atol=1e-13)
            np.testing.assert_allclose(allb["P"][:, sl], one["P"], rtol=1e-13, atol=1e-13)
