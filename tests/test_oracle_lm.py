"""Pins of the oracle's Levenberg-Marquardt iteration with adaptive damping
(Sec. 3 names the LM variant of the IEKS) and of its MAP objective, against
the dense stacked form of the same problem (tests/dense_reference.py),
written independently of the oracle's sequential smoother."""
import numpy as np
import pytest

import oracle
from paper_2102_00514_gb300 import synth
from tests.dense_reference import gauss_newton_step, map_objective


def _dense(wl, model):
    s = wl["sensors"][0]
    f = lambda v: oracle.ct_f(v, wl["dt"])
    h = lambda v: oracle.bearings_h(v, s)
    fj = lambda v: oracle.ct_jacobian(v, wl["dt"])
    hj = lambda v: oracle.bearings_jacobian(v, s)
    Q, R = model.Q(), model.R()
    P0 = oracle.sym_full(wl["P0"][0], 5)
    return f, h, fj, hj, Q, R, wl["y"].T, wl["m0"][0], P0


def test_map_cost_is_half_the_dense_objective():
    wl = synth.ct_bearings([18], seed=21, q_form=1)
    model = oracle.Model.from_workload(wl)
    f, h, fj, hj, Q, R, y, m0, P0 = _dense(wl, model)
    rng = np.random.default_rng(0)
    for _ in range(3):
        x = wl["x_true"].T + 0.05 * rng.standard_normal((19, 5))
        got = oracle.map_cost(model, wl["offsets"], wl["y"], wl["m0"], wl["P0"], x.T)[0]
        assert got == pytest.approx(0.5 * map_objective(x, f, h, Q, R, y, m0, P0), rel=1e-12)


def test_map_cost_is_periodic_in_each_bearing():
    """A bearing and the same bearing plus or minus 2 pi are one measurement: the
    objective's angle residuals are taken on the branch nearest zero."""
    wl = synth.ct_bearings([12], seed=23, q_form=1)
    model = oracle.Model.from_workload(wl)
    x = wl["x_true"] + 0.02
    base = oracle.map_cost(model, wl["offsets"], wl["y"], wl["m0"], wl["P0"], x)[0]
    for k, r, turn in ((3, 0, 1), (7, 1, -1), (12, 0, 2)):
        y = wl["y"].copy()
        y[r, k] += 2 * np.pi * turn
        got = oracle.map_cost(model, wl["offsets"], y, wl["m0"], wl["P0"], x)[0]
        assert got == pytest.approx(base, rel=1e-9)


def test_map_cost_needs_positive_definite_q():
    wl = synth.ct_bearings([5], seed=22, q_form=0)   # diag(0, 0, ...): singular
    model = oracle.Model.from_workload(wl)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.map_cost(model, wl["offsets"], wl["y"], wl["m0"], wl["P0"], np.tile(wl["m0"][0], (6, 1)).T)


def _dense_lm(wl, model, iters, lam0, nu):
    """The adaptive rule on the dense problem: the damped Gauss-Newton step,
    accepted if it lowers the objective."""
    f, h, fj, hj, Q, R, y, m0, P0 = _dense(wl, model)
    x = np.tile(m0, (len(y), 1))
    lam = lam0
    J = map_objective(x, f, h, Q, R, y, m0, P0)
    hist = []
    for _ in range(iters):
        xn, _ = gauss_newton_step(x, f, fj, h, hj, Q, R, y, m0, P0, damping=lam)
        Jn = map_objective(xn, f, h, Q, R, y, m0, P0)
        if Jn < J:
            x, J, lam = xn, Jn, lam / nu
            hist.append(True)
        else:
            lam *= nu
            hist.append(False)
    return x, lam, hist


@pytest.mark.parametrize("lam0,nu", [(1e-3, 10.0), (1.0, 3.0), (50.0, 10.0)])
def test_adaptive_lm_iterations_match_the_dense_rule(lam0, nu):
    """Each iteration, from the oracle's own nominal and damping after the
    previous one: the dense damped Gauss-Newton step, kept if it lowers the
    dense objective (then lambda / nu), else the nominal kept (lambda nu).
    Step by step, so that the comparison does not carry the amplification of
    a nearly undamped iteration from one step to the next."""
    wl = synth.ct_bearings([15], seed=11, q_form=1)
    model = oracle.Model.from_workload(wl)
    f, h, fj, hj, Q, R, y, m0, P0 = _dense(wl, model)
    run = lambda n: oracle.iterated_smoother_lm(model, wl["offsets"], wl["y"], wl["m0"], wl["P0"], iters=n,
                                                lambda0=lam0, nu=nu)
    prev = None
    for it in range(1, 8):
        cur = run(it)
        x0 = np.tile(m0, (16, 1)) if prev is None else prev["x"].T
        lam = lam0 if prev is None else prev["lam"][0]
        xn, _ = gauss_newton_step(x0, f, fj, h, hj, Q, R, y, m0, P0, damping=lam)
        Jn, J0 = map_objective(xn, f, h, Q, R, y, m0, P0), map_objective(x0, f, h, Q, R, y, m0, P0)
        accept = Jn < J0
        if abs(Jn - J0) < 1e-12 * abs(J0):
            # converged: the two costs agree to rounding and either decision is right
            accept = cur["accepted"][0] > (0 if prev is None else prev["accepted"][0])
        np.testing.assert_allclose(cur["x"].T, xn if accept else x0, rtol=1e-8, atol=1e-9)
        assert cur["lam"][0] == pytest.approx(lam / nu if accept else lam * nu, rel=1e-12)
        assert cur["accepted"][0] == (0 if prev is None else prev["accepted"][0]) + int(accept)
        prev = cur


def test_adaptive_lm_rejects_a_step_that_raises_the_cost():
    """From a start off the truth (positions shifted by about a unit, turn
    rate by 0.74), the lightly damped steps overshoot and raise the MAP cost:
    the first four are rejected (the nominal stays, the damping grows tenfold
    each time) and the fifth, damped one is accepted; the dense rule gives the
    same sequence."""
    wl = synth.ct_bearings([15], seed=13, q_form=1)
    model = oracle.Model.from_workload(wl)
    x0 = wl["x_true"].T + np.array([0.048, -1.152, 0.0, 0.0, 0.741])
    f, h, fj, hj, Q, R, y, m0, P0 = _dense(wl, model)
    lam, hist, x = 1e-4, [], x0.copy()
    J = map_objective(x, f, h, Q, R, y, m0, P0)
    for _ in range(5):
        xn, _ = gauss_newton_step(x, f, fj, h, hj, Q, R, y, m0, P0, damping=lam)
        Jn = map_objective(xn, f, h, Q, R, y, m0, P0)
        hist.append(bool(Jn < J))
        if Jn < J:
            x, J, lam = xn, Jn, lam / 10.0
        else:
            lam *= 10.0
    assert hist == [False, False, False, False, True]
    run = lambda n: oracle.iterated_smoother_lm(model, wl["offsets"], wl["y"], wl["m0"], wl["P0"], x_init=x0.T,
                                                iters=n, lambda0=1e-4, nu=10.0)
    four, five = run(4), run(5)
    np.testing.assert_array_equal(four["x"], x0.T)
    assert four["lam"][0] == pytest.approx(1.0) and four["accepted"][0] == 0
    assert five["accepted"][0] == 1 and five["lam"][0] == pytest.approx(0.1)
    np.testing.assert_allclose(five["x"].T, x, rtol=1e-8, atol=1e-9)
    assert (oracle.map_cost(model, wl["offsets"], wl["y"], wl["m0"], wl["P0"], five["x"])[0] <
            oracle.map_cost(model, wl["offsets"], wl["y"], wl["m0"], wl["P0"], four["x"])[0])


def test_adaptive_lm_converges_to_a_stationary_point():
    wl = synth.ct_bearings([20], seed=12, q_form=1)
    model = oracle.Model.from_workload(wl)
    out = oracle.iterated_smoother_lm(model, wl["offsets"], wl["y"], wl["m0"], wl["P0"], iters=60, tol=1e-10,
                                      lambda0=1.0, nu=10.0)
    assert out["status"] == oracle.OK and out["conv_iter"][0] > 0
    f, h, fj, hj, Q, R, y, m0, P0 = _dense(wl, model)
    x = out["x"].T
    _, g = gauss_newton_step(x, f, fj, h, hj, Q, R, y, m0, P0)
    J = map_objective(x, f, h, Q, R, y, m0, P0)
    assert np.linalg.norm(g) < 1e-6 * max(1.0, J)


def test_adaptive_lm_batch_equals_separate_runs():
    wl = synth.ct_bearings([12, 30, 7], seed=13, q_form=1, sensor_jitter=0.2)
    model = oracle.Model.from_workload(wl)
    both = oracle.iterated_smoother_lm(model, wl["offsets"], wl["y"], wl["m0"], wl["P0"], iters=5, lambda0=1e-2,
                                       nu=10.0)
    off = wl["offsets"]
    for b in range(3):
        sl = slice(int(off[b]), int(off[b + 1]))
        one = dict(wl, offsets=np.array([0, off[b + 1] - off[b]]), y=wl["y"][:, sl], m0=wl["m0"][b:b + 1],
                   P0=wl["P0"][b:b + 1], sensors=wl["sensors"][b:b + 1])
        r = oracle.iterated_smoother_lm(oracle.Model.from_workload(one), one["offsets"], one["y"], one["m0"],
                                        one["P0"], iters=5, lambda0=1e-2, nu=10.0)
        np.testing.assert_allclose(both["x"][:, sl], r["x"], rtol=1e-12, atol=1e-12)
        assert both["lam"][b] == r["lam"][0] and both["accepted"][b] == r["accepted"][0]
