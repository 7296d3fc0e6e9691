"""Pins for the oracle's linearisation and iteration on the coordinated-turn /
bearings model (Secs. 3 and 5).

* Cubature SLR (Eqs. 7-9) is exact for affine functions, recovers the
  Jacobian of the coordinates in which f is affine, and tends to the Taylor
  linearisation (Eq. 10) as the covariance shrinks.
* The unscented rule with alpha = 1, beta = 0, kappa = 0 is the cubature rule
  (a separate code path); for other parameters it is exact for affine
  functions and gives the exact mean of quadratic functions.
* The Gauss-Hermite product rule is exact for affine functions and its mean is
  of higher order than the cubature rule's.
* Every IEKS iteration is one Gauss-Newton step of the MAP problem (checked
  against a dense Gauss-Newton solve, positive-definite Q), and at
  convergence the MAP gradient vanishes.
* Every iteration of either method equals dense Gaussian conditioning of the
  stacked affine model built from the oracle's own linearisation.
* Covariances are symmetric positive semi-definite; the last filtered and
  smoothed moments coincide.
"""
import numpy as np
import pytest

import oracle
from paper_2102_00514_gb300 import synth
from tests.dense_reference import dense_smoother, gauss_newton_step


def ct_model(q_form=0, sensors=None):
    s = np.array(synth.SENSORS if sensors is None else sensors)
    return oracle.Model.ct_bearings(synth.DT, synth.Q_C, synth.Q_W, synth.R_STD, s, q_form=q_form)


def test_slr_exact_for_linear_model():
    rng = np.random.default_rng(3)
    F = rng.standard_normal((5, 5)); c = rng.standard_normal(5)
    H = rng.standard_normal((2, 5)); d = rng.standard_normal(2)
    m = oracle.Model.linear(F, c, np.eye(5), H, d, np.eye(2))
    xbar = rng.standard_normal(5)
    A = rng.standard_normal((5, 5)); P = A @ A.T + np.eye(5)
    G, off, Lam = oracle.slr(m, 0, 0, xbar, P)
    np.testing.assert_allclose(G, F, atol=1e-12)
    np.testing.assert_allclose(off, c, atol=1e-12)
    np.testing.assert_allclose(Lam, 0, atol=1e-12)
    G, off, Om = oracle.slr(m, 1, 0, xbar, P)
    np.testing.assert_allclose(G, H, atol=1e-12)
    np.testing.assert_allclose(off, d, atol=1e-12)
    np.testing.assert_allclose(Om, 0, atol=1e-12)


def test_slr_exact_in_coordinates_where_ct_is_affine():
    """With (almost) no turn-rate uncertainty f is affine in (p, v): the SLR
    recovers the Jacobian there and Lambda vanishes."""
    m = ct_model()
    xbar = np.array([0.4, -0.2, 1.1, 0.3, 0.8])
    P = np.diag([0.5, 0.3, 0.2, 0.4, 1e-24])
    P[0, 2] = P[2, 0] = 0.1
    G, off, Lam = oracle.slr(m, 0, 0, xbar, P)
    J = oracle.ct_jacobian(xbar, synth.DT)
    np.testing.assert_allclose(G[:, :4], J[:, :4], atol=1e-12)
    np.testing.assert_allclose(off + G @ xbar, oracle.ct_f(xbar, synth.DT), atol=1e-12)
    np.testing.assert_allclose(Lam, 0, atol=1e-12)


@pytest.mark.parametrize("which", [0, 1])
def test_slr_small_covariance_tends_to_taylor(which):
    m = ct_model()
    xbar = np.array([0.4, -0.2, 1.1, 0.3, 0.8])
    J = oracle.ct_jacobian(xbar, synth.DT) if which == 0 else oracle.bearings_jacobian(xbar, synth.SENSORS)
    errs = []
    for eps in (1e-2, 1e-3, 1e-4):
        G, off, Lam = oracle.slr(m, which, 0, xbar, eps * eps * np.eye(5))
        errs.append(np.abs(G - J).max())
        assert np.all(np.linalg.eigvalsh(Lam) > -1e-15)
    # second-order convergence in the sigma-point spread
    assert errs[1] < 0.02 * errs[0] + 1e-12 and errs[2] < 0.02 * errs[1] + 1e-12


UT_PARAMS = [(1.0, 2.0, 1.0), (0.8, 2.0, 0.5), (1.0, 0.0, -2.0)]


def test_unscented_with_cubature_parameters_is_the_cubature_rule():
    m = ct_model().unscented(1.0, 0.0, 0.0)
    xbar = np.array([0.4, -0.2, 1.1, 0.3, 0.8])
    A = np.random.default_rng(5).standard_normal((5, 5))
    P = 0.05 * (A @ A.T) + 0.01 * np.eye(5)
    for which in (0, 1):
        a = oracle.slr(m, which, 0, xbar, P, method=oracle.UNSCENTED)
        c = oracle.slr(m, which, 0, xbar, P, method=oracle.CUBATURE)
        for u, v in zip(a, c):
            np.testing.assert_allclose(u, v, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("alpha,beta,kappa", UT_PARAMS)
def test_unscented_exact_for_linear_model(alpha, beta, kappa):
    rng = np.random.default_rng(4)
    F = rng.standard_normal((5, 5)); c = rng.standard_normal(5)
    H = rng.standard_normal((2, 5)); d = rng.standard_normal(2)
    m = oracle.Model.linear(F, c, np.eye(5), H, d, np.eye(2)).unscented(alpha, beta, kappa)
    xbar = rng.standard_normal(5)
    A = rng.standard_normal((5, 5)); P = A @ A.T + np.eye(5)
    for which, (Gt, ot) in ((0, (F, c)), (1, (H, d))):
        G, off, Lam = oracle.slr(m, which, 0, xbar, P, method=oracle.UNSCENTED)
        np.testing.assert_allclose(G, Gt, atol=1e-11)
        np.testing.assert_allclose(off, ot, atol=1e-11)
        np.testing.assert_allclose(Lam, 0, atol=1e-11)


@pytest.mark.parametrize("alpha,beta,kappa", UT_PARAMS)
def test_unscented_mean_exact_for_quadratics(alpha, beta, kappa):
    """The symmetric rule integrates polynomials of degree 2 (and odd ones)
    exactly, so its mean of a function that is quadratic up to a tiny quartic
    remainder must match the Gaussian expectation: the coordinated turn with
    only the turn rate uncertain, N(0.8, 0.3^2), over dt = 0.01 (remainder of
    order (0.3 dt)^4). The expectation is integrated by 40-node Gauss-Hermite.
    A wrong centre or side weight moves the mean by O(1)."""
    m = ct_model().unscented(alpha, beta, kappa)
    xbar = np.array([0.4, -0.2, 1.1, 0.3, 0.8])
    P = np.diag([0.0, 0.0, 0.0, 0.0, 0.3 ** 2])
    P[:4, :4] = 1e-30 * np.eye(4)   # (p, v) fixed: f depends on omega alone
    G, off, Lam = oracle.slr(m, 0, 0, xbar, P, method=oracle.UNSCENTED)
    zbar = G @ xbar + off
    t, w = np.polynomial.hermite_e.hermegauss(40)
    exact = sum(wi * oracle.ct_f(xbar + np.array([0, 0, 0, 0, 0.3 * ti]), synth.DT) for ti, wi in zip(t, w))
    exact = exact / w.sum()
    np.testing.assert_allclose(zbar, exact, atol=1e-9)


def _residual_covariance_1d(f, x0, axis, sig, nodes=60):
    """The Gaussian SLR residual covariance Var(f) - Cov(f, u) Cov(f, u)^T / sig^2
    of f(x0 + u e_axis), u ~ N(0, sig^2), by Gauss-Hermite quadrature."""
    t, w = np.polynomial.hermite_e.hermegauss(nodes)
    w = w / w.sum()
    Z = np.array([f(x0 + sig * ti * np.eye(5)[axis]) for ti in t])
    zbar = w @ Z
    D = Z - zbar
    C = (w * sig * t) @ D
    return (D.T * w) @ D - np.outer(C, C) / sig ** 2


@pytest.mark.parametrize("alpha,beta,kappa,exact", [(1.0, 0.0, -2.0, True), (0.5, 2.0, -4.0, True),
                                                    (1.0, 2.0, 1.0, False)])
def test_unscented_residual_covariance_of_a_quadratic(alpha, beta, kappa, exact):
    """For a function of one Gaussian coordinate u ~ N(0, s^2) that is quadratic,
    a u^2 + b u, the rule's residual covariance is a^2 s^4 (alpha^2 (n + kappa - 1)
    + beta) (n = 5) against the true 2 a^2 s^4: exact when alpha^2 (n + kappa - 1)
    + beta = 2, as for kappa = 3 - n with beta = 0, or kappa = 1 - n with the
    Gaussian-optimal beta = 2 at any alpha. The coordinated turn with only the
    turn rate uncertain, N(0.8, 0.3^2) over dt = 0.01, is quadratic up to a
    relative remainder of order (0.3 dt)^2; the truth is integrated by
    60-node Gauss-Hermite. The centre point's covariance weight (beta) and
    the spread lambda enter only here."""
    m = ct_model().unscented(alpha, beta, kappa)
    xbar = np.array([0.4, -0.2, 1.1, 0.3, 0.8])
    P = np.diag([1e-30] * 4 + [0.3 ** 2])
    _, _, Lam = oracle.slr(m, 0, 0, xbar, P, method=oracle.UNSCENTED)
    true = _residual_covariance_1d(lambda v: oracle.ct_f(v, synth.DT), xbar, 4, 0.3)
    err = np.abs(Lam - true).max() / np.abs(true).max()
    if exact:
        assert err < 1e-3
    else:
        assert err > 1.0   # 3.5 times the truth: the check discriminates


def _residual_covariance_2d(f, x0, axes, sigs, nodes=24):
    """The Gaussian SLR residual covariance of f over two independent Gaussian
    coordinates (tensor-product Gauss-Hermite quadrature)."""
    t, w = np.polynomial.hermite_e.hermegauss(nodes)
    w = w / w.sum()
    U, Zs, W = [], [], []
    for ti, wi in zip(t, w):
        for tj, wj in zip(t, w):
            u = np.array([sigs[0] * ti, sigs[1] * tj])
            x = x0.copy()
            x[axes[0]] += u[0]
            x[axes[1]] += u[1]
            U.append(u); Zs.append(f(x)); W.append(wi * wj)
    U, Z, W = np.array(U), np.array(Zs), np.array(W)
    D = Z - W @ Z
    C = (U.T * W) @ D                       # Cov(u, z), 2 x nz
    return (D.T * W) @ D - C.T @ np.diag(1.0 / np.square(sigs)) @ C


def test_linearised_noise_adds_the_slr_residual_covariance():
    """Q' = Q + Lambda and R' = R + Omega (Eq. 10), with Lambda and Omega the
    residual covariances of the statistical linear regression: through the
    Gauss-Hermite rule, which integrates the quadratic part of f and h exactly,
    the linearisation's Q' - Q and R' - R must match the true residual
    covariances (tensor-product quadrature) of the coordinated turn with the
    turn rate and one velocity uncertain (the bilinear turn term) and of the
    bearings with the position uncertain."""
    m = ct_model()
    x0 = np.array([0.1, 0.2, 1.1, 0.3, 0.8])
    x1 = np.array([0.12, 0.19, 1.0, 0.4, 0.7])
    P0 = np.diag([1e-30, 1e-30, 1e-30, 0.5 ** 2, 2.0 ** 2])
    P1 = np.diag([0.05 ** 2, 0.04 ** 2, 1e-30, 1e-30, 1e-30])
    xbar = np.stack([x0, x1], axis=1)
    Pbar = np.stack([oracle.sym_packed(P0), oracle.sym_packed(P1)], axis=1)
    offsets = np.array([0, 2], dtype=np.int64)
    y = np.zeros((2, 2))
    lin = oracle.linearize(m, oracle.GAUSS_HERMITE, offsets, xbar, Pbar, y)
    Lam = oracle.sym_full(lin["Qp"][:, 0], 5) - m.Q()
    Om = oracle.sym_full(lin["Rp"][:, 1], 2) - m.R()
    Lt = _residual_covariance_2d(lambda v: oracle.ct_f(v, synth.DT), x0, (3, 4), (0.5, 2.0))
    Ot = _residual_covariance_2d(lambda v: oracle.bearings_h(v, np.array(synth.SENSORS)), x1, (0, 1), (0.05, 0.04))
    assert np.abs(Lt).max() > 1e-9 and np.abs(Ot).max() > 1e-9
    np.testing.assert_allclose(Lam, Lt, atol=1e-3 * np.abs(Lt).max())
    np.testing.assert_allclose(Om, Ot, atol=2e-2 * np.abs(Ot).max())


def test_gauss_hermite_exact_for_linear_model():
    rng = np.random.default_rng(6)
    F = rng.standard_normal((5, 5)); c = rng.standard_normal(5)
    H = rng.standard_normal((2, 5)); d = rng.standard_normal(2)
    m = oracle.Model.linear(F, c, np.eye(5), H, d, np.eye(2))
    xbar = rng.standard_normal(5)
    A = rng.standard_normal((5, 5)); P = A @ A.T + np.eye(5)
    for which, (Gt, ot) in ((0, (F, c)), (1, (H, d))):
        G, off, Lam = oracle.slr(m, which, 0, xbar, P, method=oracle.GAUSS_HERMITE)
        np.testing.assert_allclose(G, Gt, atol=1e-11)
        np.testing.assert_allclose(off, ot, atol=1e-11)
        np.testing.assert_allclose(Lam, 0, atol=1e-11)


@pytest.mark.parametrize("sig,gh_tol", [(0.3, 1e-13), (20.0, 2e-6)])
def test_gauss_hermite_mean_is_of_higher_order_than_cubature(sig, gh_tol):
    """The 3^n product rule integrates degree 5 per coordinate exactly, the
    cubature rule degree 3: for the coordinated turn with an uncertain turn
    rate the Gauss-Hermite mean stays within its degree-6 remainder of the
    Gaussian expectation (60-node Gauss-Hermite quadrature), far closer than
    the cubature mean once the turn-angle spread is not small."""
    m = ct_model()
    xbar = np.array([0.4, -0.2, 1.1, 0.3, 0.8])
    P = np.diag([1e-30] * 4 + [sig ** 2])
    t, w = np.polynomial.hermite_e.hermegauss(60)
    exact = sum(wi * oracle.ct_f(xbar + np.array([0, 0, 0, 0, sig * ti]), synth.DT) for ti, wi in zip(t, w))
    exact = exact / w.sum()
    errs = {}
    for meth in (oracle.CUBATURE, oracle.GAUSS_HERMITE):
        G, off, Lam = oracle.slr(m, 0, 0, xbar, P, method=meth)
        errs[meth] = np.abs(G @ xbar + off - exact).max()
        assert np.linalg.eigvalsh(Lam).min() > -1e-12 * max(1.0, np.abs(Lam).max())
    assert errs[oracle.GAUSS_HERMITE] < gh_tol
    if sig > 1:
        assert errs[oracle.GAUSS_HERMITE] < 0.01 * errs[oracle.CUBATURE]


def test_slr_unwraps_bearings_across_branch_cut():
    """A target just across the -pi/pi cut from a sensor: without unwrapping the
    sigma-point spread of atan2 would be ~2 pi."""
    s = np.array([0.0, 0.0, 5.0, 5.0])
    m = ct_model(sensors=s)
    xbar = np.array([-3.0, 1e-4, 1.0, 0.0, 0.0])
    G, off, Om = oracle.slr(m, 1, 0, xbar, 1e-4 * np.eye(5))
    J = oracle.bearings_jacobian(xbar, s)
    np.testing.assert_allclose(G, J, atol=1e-4)
    assert np.abs(Om).max() < 1e-6


def _ct_gn_damped(wl, model, x, lam):
    Q = model.Q(); R = model.R()
    s = wl["sensors"][0]
    return gauss_newton_step(
        x, lambda v: oracle.ct_f(v, wl["dt"]), lambda v: oracle.ct_jacobian(v, wl["dt"]),
        lambda v: oracle.bearings_h(v, s), lambda v: oracle.bearings_jacobian(v, s),
        Q, R, wl["y"].T, wl["m0"][0], oracle.sym_full(wl["P0"][0], 5), damping=lam)


def _ct_gn(wl, model, x):
    Q = model.Q(); R = model.R()
    s = wl["sensors"][0]
    return gauss_newton_step(
        x, lambda v: oracle.ct_f(v, wl["dt"]), lambda v: oracle.ct_jacobian(v, wl["dt"]),
        lambda v: oracle.bearings_h(v, s), lambda v: oracle.bearings_jacobian(v, s),
        Q, R, wl["y"].T, wl["m0"][0], oracle.sym_full(wl["P0"][0], 5))


@pytest.mark.parametrize("lam", [0.3, 5.0, 200.0])
def test_damped_iterations_are_levenberg_marquardt_steps(lam):
    """With damping lambda every IEKS iteration is the Levenberg-Marquardt
    step of the MAP problem about the current nominal (positive-definite Q;
    a trajectory whose bearings stay clear of the branch cut, which the dense
    step does not unwrap)."""
    wl = synth.ct_bearings([15], seed=11, q_form=1)
    model = oracle.Model.from_workload(wl)
    dm = model.damped(lam)
    x = np.tile(wl["m0"][0], (16, 1))
    for it in range(3):
        out = oracle.iterated_smoother(dm, oracle.IEKS, wl["offsets"], wl["y"], wl["m0"], wl["P0"], x_init=x.T,
                                       iters=1)
        x_gn, _ = _ct_gn_damped(wl, model, x, lam)
        np.testing.assert_allclose(out["x"].T, x_gn, rtol=1e-8, atol=1e-9)
        x = out["x"].T.copy()


def test_heavy_damping_shrinks_the_step():
    wl = synth.ct_bearings([15], seed=13, q_form=1)
    model = oracle.Model.from_workload(wl)
    x0 = np.tile(wl["m0"][0], (16, 1))
    steps = []
    # the step falls like 1 / lambda once lambda dominates the curvature
    # (Q^-1 of the positive-definite Q reaches ~1e8 here)
    for lam in (1e10, 1e12, 1e14):
        out = oracle.iterated_smoother(model.damped(lam), oracle.IEKS, wl["offsets"], wl["y"], wl["m0"], wl["P0"],
                                       x_init=x0.T, iters=1)
        steps.append(np.abs(out["x"].T - x0).max())
    assert 0.005 < steps[1] / steps[0] < 0.02 and 0.005 < steps[2] / steps[1] < 0.02


def test_ieks_iterations_are_gauss_newton_steps():
    wl = synth.ct_bearings([15], seed=11, q_form=1)
    model = oracle.Model.from_workload(wl)
    off = wl["offsets"]
    x = np.tile(wl["m0"][0], (16, 1))
    for it in range(1, 5):
        out = oracle.iterated_smoother(model, oracle.IEKS, off, wl["y"], wl["m0"], wl["P0"], iters=it)
        x, _ = _ct_gn(wl, model, x)
        np.testing.assert_allclose(out["x"].T, x, rtol=1e-8, atol=1e-9)


def test_ieks_fixed_point_zeroes_map_gradient():
    wl = synth.ct_bearings([20], seed=12, q_form=1)
    model = oracle.Model.from_workload(wl)
    out = oracle.iterated_smoother(model, oracle.IEKS, wl["offsets"], wl["y"], wl["m0"], wl["P0"], iters=50, tol=1e-12)
    assert out["status"] == oracle.OK
    x = out["x"].T
    x_next, grad = _ct_gn(wl, model, x)
    # the Gauss-Newton step from the fixed point vanishes (Newton decrement), and
    # the gradient is at rounding level for weights of order |Q^-1| ~ 1e8
    assert np.abs(x_next - x).max() < 1e-10
    assert np.abs(grad).max() < 1e-5


@pytest.mark.parametrize("method", [oracle.IEKS, oracle.CUBATURE])
def test_each_iteration_is_dense_conditioning(method):
    wl = synth.ct_bearings([18], seed=13)
    model = oracle.Model.from_workload(wl)
    off = wl["offsets"]
    N = 19
    xbar = np.tile(wl["m0"][0][:, None], (1, N))
    Pbar = np.tile(wl["P0"][0][:, None], (1, N))
    for it in range(3):
        lin = oracle.linearize(model, method, off, xbar, Pbar, wl["y"])
        F = oracle._aos(lin["F"]).reshape(N, 5, 5)[:N - 1]
        c = lin["c"].T[:N - 1]
        Q = oracle.sym_full(lin["Qp"].T, 5)[:N - 1]
        H = oracle._aos(lin["H"]).reshape(N, 2, 5)
        R = oracle.sym_full(lin["Rp"].T, 2)
        xs, Ps = dense_smoother(F, c, Q, H, lin["d"].T, R, lin["y_used"].T, wl["m0"][0],
                                oracle.sym_full(wl["P0"][0], 5))
        out = oracle.iterated_smoother(model, method, off, wl["y"], wl["m0"], wl["P0"],
                                       x_init=xbar, P_init=Pbar, iters=1)
        np.testing.assert_allclose(out["x"].T, xs, rtol=1e-8, atol=1e-9)
        np.testing.assert_allclose(oracle.sym_full(out["P"].T, 5), Ps, rtol=1e-8, atol=1e-9)
        xbar, Pbar = out["x"], out["P"]


@pytest.mark.parametrize("method", [oracle.IEKS, oracle.CUBATURE])
def test_covariance_invariants(method):
    wl = synth.workload("ieks_T500")
    model = oracle.Model.from_workload(wl)
    out = oracle.iterated_smoother(model, method, wl["offsets"], wl["y"], wl["m0"], wl["P0"], iters=5)
    P = oracle.sym_full(out["P"].T, 5)
    ev = np.linalg.eigvalsh(P)
    assert ev.min() > -1e-12 * ev.max()
    # the smoother's last state is the filter's last state
    N = wl["y"].shape[1]
    lin = oracle.linearize(model, method, wl["offsets"], out["x"], out["P"], wl["y"])
    kr = oracle.kf_rts(wl["offsets"], lin, lin["y_used"], wl["m0"], wl["P0"])
    np.testing.assert_array_equal(kr["xs"][:, N - 1], kr["xf"][:, N - 1])
    np.testing.assert_array_equal(kr["Ps"][:, N - 1], kr["Pf"][:, N - 1])


def test_tolerance_mode_reports_not_converged():
    wl = synth.workload("ieks_T500")
    model = oracle.Model.from_workload(wl)
    out = oracle.iterated_smoother(model, oracle.IEKS, wl["offsets"], wl["y"], wl["m0"], wl["P0"], iters=3, tol=1e-6)
    assert out["status"] == oracle.NOT_CONVERGED and out["iters_used"] == 3
    out = oracle.iterated_smoother(model, oracle.IEKS, wl["offsets"], wl["y"], wl["m0"], wl["P0"], iters=50, tol=1e-6)
    assert out["status"] == oracle.OK and out["iters_used"] < 50
    assert out["rel_history"][-1] <= 1e-6 < out["rel_history"][-2]
