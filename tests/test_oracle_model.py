"""Pins for the oracle's model functions (coordinated turn, bearings, Sec. 5).

The coordinated-turn transition is the exact discretisation of the constant
turn-rate motion p' = v, v' = omega J v, omega' = 0; it is checked against a
fine Runge-Kutta integration of that ODE, against straight-line motion at
omega = 0, for continuity across its series threshold, and its Jacobian
against central differences. Bearings are checked on known geometry.
"""
import math

import numpy as np
import pytest

import oracle


def rk4_turn(x, dt, nsub=2000):
    """Integrate p' = v, v' = omega [[0,-1],[1,0]] v, omega' = 0 over dt."""
    def rhs(s):
        w = s[4]
        return np.array([s[2], s[3], -w * s[3], w * s[2], 0.0])
    s = np.array(x, dtype=float)
    h = dt / nsub
    for _ in range(nsub):
        k1 = rhs(s); k2 = rhs(s + 0.5 * h * k1); k3 = rhs(s + 0.5 * h * k2); k4 = rhs(s + h * k3)
        s = s + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return s


@pytest.mark.parametrize("w", [-3.0, -0.7, 0.05, 1.3, 11.0])
@pytest.mark.parametrize("dt", [0.01, 0.25])
def test_ct_is_exact_turn_discretisation(w, dt):
    x = np.array([0.3, -1.2, 1.1, -0.4, w])
    np.testing.assert_allclose(oracle.ct_f(x, dt), rk4_turn(x, dt), rtol=0, atol=1e-12)


def test_ct_straight_line_at_zero_turn_rate():
    x = np.array([0.3, -1.2, 1.1, -0.4, 0.0])
    dt = 0.01
    expect = np.array([0.3 + 1.1 * dt, -1.2 - 0.4 * dt, 1.1, -0.4, 0.0])
    np.testing.assert_allclose(oracle.ct_f(x, dt), expect, rtol=0, atol=1e-15)


def fd_jacobian(x, dt, h=1e-6):
    J = np.zeros((5, 5))
    for j in range(5):
        e = np.zeros(5); e[j] = h
        J[:, j] = (oracle.ct_f(x + e, dt) - oracle.ct_f(x - e, dt)) / (2 * h)
    return J


def test_ct_continuous_across_series_threshold():
    """Either side of |omega dt| = 1e-2 (series below, closed form above) the
    step in f matches the Jacobian's omega column times the step in omega, both
    sides match the integrated turn, and both Jacobians match differences."""
    dt = 0.01
    thr = 1e-2 / dt
    xa = np.array([0.3, -1.2, 1.1, -0.4, thr * (1 - 1e-9)])
    xb = np.array([0.3, -1.2, 1.1, -0.4, thr * (1 + 1e-9)])
    dw = xb[4] - xa[4]
    df = oracle.ct_f(xb, dt) - oracle.ct_f(xa, dt)
    J = 0.5 * (oracle.ct_jacobian(xa, dt) + oracle.ct_jacobian(xb, dt))
    # a wrong series coefficient would show as ~1e-8 here
    np.testing.assert_allclose(df, J[:, 4] * dw, rtol=0, atol=1e-15)
    for x in (xa, xb):
        np.testing.assert_allclose(oracle.ct_f(x, dt), rk4_turn(x, dt, nsub=200), rtol=0, atol=1e-13)
        np.testing.assert_allclose(oracle.ct_jacobian(x, dt), fd_jacobian(x, dt), rtol=0, atol=1e-9)


def test_ct_series_branch_matches_integration():
    dt = 0.01
    for w in (0.0, 1e-6, 3e-3, -0.5, 0.99):
        x = np.array([0.3, -1.2, 1.1, -0.4, w])
        # RK4 with 200 substeps: truncation ~1e-17, rounding ~1e-14
        np.testing.assert_allclose(oracle.ct_f(x, dt), rk4_turn(x, dt, nsub=200), rtol=0, atol=1e-13)


@pytest.mark.parametrize("w", [0.0, 2e-3, 0.02, 0.9, -4.0])
def test_ct_jacobian_central_differences(w):
    dt = 0.01
    x = np.array([0.3, -1.2, 1.1, -0.4, w])
    J = oracle.ct_jacobian(x, dt)
    h = 1e-6
    Jfd = np.zeros((5, 5))
    for j in range(5):
        e = np.zeros(5); e[j] = h
        Jfd[:, j] = (oracle.ct_f(x + e, dt) - oracle.ct_f(x - e, dt)) / (2 * h)
    np.testing.assert_allclose(J, Jfd, rtol=0, atol=1e-9)


def test_bearings_known_geometry():
    s = np.array([-1.5, 0.5, 1.0, 1.0])
    x = np.array([-1.5, 3.5, 0, 0, 0])          # due north of sensor 1
    y = oracle.bearings_h(x, s)
    assert abs(y[0] - math.pi / 2) < 1e-15
    assert abs(y[1] - math.atan2(2.5, -2.5)) < 1e-15  # 135 degrees from sensor 2
    assert abs(y[1] - 3 * math.pi / 4) < 1e-15


def test_bearings_jacobian_central_differences():
    s = np.array([-1.5, 0.5, 1.0, 1.0])
    x = np.array([0.7, -0.3, 1.0, 0.5, 0.2])
    J = oracle.bearings_jacobian(x, s)
    h = 1e-6
    Jfd = np.zeros((2, 5))
    for j in range(5):
        e = np.zeros(5); e[j] = h
        Jfd[:, j] = (oracle.bearings_h(x + e, s) - oracle.bearings_h(x - e, s)) / (2 * h)
    np.testing.assert_allclose(J, Jfd, rtol=0, atol=1e-8)


@pytest.mark.parametrize("a", [0.0, 1.0, -3.0, 3.2, 7.0, -9.5, 100.0])
def test_wrap_range_and_congruence(a):
    w = oracle.wrap(a)
    assert -math.pi <= w < math.pi
    k = (a - w) / (2 * math.pi)
    assert abs(k - round(k)) < 1e-12


def test_noise_covariances():
    m = oracle.Model.ct_bearings(0.01, 0.1, 0.01, 0.05, [-1.5, 0.5, 1.0, 1.0], q_form=0)
    np.testing.assert_allclose(np.diag(m.Q()), [0, 0, 1e-3, 1e-3, 1e-4], rtol=1e-15)
    assert np.count_nonzero(m.Q() - np.diag(np.diag(m.Q()))) == 0
    np.testing.assert_allclose(m.R(), 0.0025 * np.eye(2), rtol=1e-15)
    m1 = oracle.Model.ct_bearings(0.01, 0.1, 0.01, 0.05, [-1.5, 0.5, 1.0, 1.0], q_form=1)
    Q = m1.Q()
    assert np.all(np.linalg.eigvalsh(Q) > 0)  # positive definite variant
    # the white-acceleration block of one axis: q_c [[dt^3/3, dt^2/2], [dt^2/2, dt]]
    np.testing.assert_allclose(Q[np.ix_([0, 2], [0, 2])], 0.1 * np.array([[1e-6 / 3, 5e-5], [5e-5, 1e-2]]), rtol=1e-14)
