"""Pins for the oracle's LLG right-hand side (Eq. llg), RK4, Dormand-Prince
5(4) and Runge-Kutta-Fehlberg 4(5) integrators, the damping-only right-hand
side, renormalisation, energy decay and relax."""
import math

import numpy as np
import pytest

from oracle.constants import GAMMA, MU0
from oracle.llg import (DP_A, DP_B4, DP_B5, DP_C, RKF_A, RKF_B4, RKF_B5, RKF_C, Problem, dp45_attempt,
                        dp45_integrate, llg_rhs, normalize, relax, rk4_step, rkf45_attempt, rkf45_step)


def test_rhs_is_orthogonal_to_m_and_precesses():
    rng = np.random.default_rng(0)
    m = normalize(rng.normal(size=(3, 2, 1, 3)))
    h = rng.normal(size=(3, 2, 1, 3)) * 1e5
    f = llg_rhs(m, h, 0.3)
    assert np.max(np.abs(np.sum(f * m, axis=-1))) < 1e-9 * np.max(np.abs(f))
    # alpha = 0, m perpendicular to h: |dm/dt| = gamma |h|, dm/dt = -gamma m x h
    m1 = np.array([[[[1.0, 0.0, 0.0]]]])
    h1 = np.array([[[[0.0, 0.0, 2e4]]]])
    f1 = llg_rhs(m1, h1, 0.0)
    assert np.allclose(f1[0, 0, 0], [0.0, GAMMA * 2e4, 0.0], rtol=1e-15)


def _macrospin(alpha=0.1, H=8e4, precession=True):
    # one cubic cell: its demag field -M/3 is parallel to m and exerts no torque
    return Problem((1, 1, 1), (2e-9, 2e-9, 2e-9), Ms=8e5, A=1.3e-11, alpha=alpha,
                   h_ext=(0.0, 0.0, H), precession=precession)


def _exact(theta0, phi0, alpha, H, t):
    gp = GAMMA / (1 + alpha ** 2)
    th = 2 * math.atan(math.tan(theta0 / 2) * math.exp(-alpha * gp * H * t))
    ph = phi0 + gp * H * t
    return np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])


def _m0(theta0, phi0):
    return np.array([[[[math.sin(theta0) * math.cos(phi0), math.sin(theta0) * math.sin(phi0),
                        math.cos(theta0)]]]])


@pytest.mark.parametrize("renorm", [False, True])
def test_rk4_macrospin_fourth_order(renorm):
    alpha, H, T = 0.1, 8e4, 2e-10
    prob = _macrospin(alpha, H)
    th0, ph0 = 2.5, 0.3
    errs = []
    for nsteps in (50, 100, 200):
        dt = T / nsteps
        m = _m0(th0, ph0)
        for s in range(nsteps):
            m = rk4_step(prob, m, s * dt, dt, renorm=renorm)
        errs.append(np.max(np.abs(m[0, 0, 0] - _exact(th0, ph0, alpha, H, T))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13.0 < r1 < 19.0 and 13.0 < r2 < 19.0
    assert errs[2] < 1e-7


def test_dp45_tableau_order_conditions():
    c = np.array(DP_C)
    b5 = np.array(DP_B5)
    b4 = np.array(DP_B4)
    A = np.zeros((7, 7))
    for i, row in enumerate(DP_A):
        A[i, : len(row)] = row
    assert np.allclose(A.sum(axis=1), c, atol=1e-15)
    # quadrature conditions: exact for t^q, q <= 4 (fifth order), q <= 3 (fourth order)
    for q in range(5):
        assert abs(b5 @ c ** q - 1.0 / (q + 1)) < 1e-14
    for q in range(4):
        assert abs(b4 @ c ** q - 1.0 / (q + 1)) < 1e-14
    assert abs(b4 @ c ** 4 - 1.0 / 5) > 1e-6
    # a sample of the tree conditions of order 3..5
    assert abs(b5 @ (A @ c) - 1.0 / 6) < 1e-14
    assert abs(b5 @ (A @ c ** 2) - 1.0 / 12) < 1e-14
    assert abs(b5 @ (c * (A @ c)) - 1.0 / 8) < 1e-14
    assert abs(b5 @ (A @ (A @ c)) - 1.0 / 24) < 1e-14
    assert abs(b5 @ (A @ c ** 3) - 1.0 / 20) < 1e-14
    assert abs(b5 @ (A @ (A @ (A @ c))) - 1.0 / 120) < 1e-14
    assert abs(b5 @ (c * (A @ (A @ c))) - 1.0 / 30) < 1e-14
    assert abs(b5 @ ((A @ c) * (A @ c)) - 1.0 / 20) < 1e-14
    assert abs(b4 @ (A @ (A @ c)) - 1.0 / 24) < 1e-14
    # first same as last: the last row of A is the fifth-order weight vector
    assert np.allclose(A[6, :6], b5[:6]) and b5[6] == 0.0


def test_dp45_fixed_step_fifth_order():
    alpha, H, T = 0.1, 8e4, 2e-10
    prob = _macrospin(alpha, H)
    th0, ph0 = 2.5, 0.3
    errs = []
    for nsteps in (20, 40, 80):
        dt = T / nsteps
        m = _m0(th0, ph0)
        k1 = prob.rhs(m, 0.0)
        for s in range(nsteps):
            m, k1, _, _ = dp45_attempt(prob, m, s * dt, dt, k1, rtol=1e-5)
        errs.append(np.max(np.abs(m[0, 0, 0] - _exact(th0, ph0, alpha, H, T))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 26.0 < r1 < 38.0 and 26.0 < r2 < 38.0


def test_dp45_adaptive_meets_tolerance():
    alpha, H, T = 0.1, 8e4, 5e-10
    prob = _macrospin(alpha, H)
    th0, ph0 = 2.5, 0.3
    errs = {}
    for rtol in (1e-5, 1e-7):
        m, t, _, acc, rej = dp45_integrate(prob, _m0(th0, ph0), 0.0, T, dt0=1e-13, rtol=rtol)
        assert t == pytest.approx(T, rel=1e-15)
        errs[rtol] = np.max(np.abs(m[0, 0, 0] - _exact(th0, ph0, alpha, H, T)))
        assert errs[rtol] < 100 * rtol
    assert errs[1e-7] < errs[1e-5]


def _small_problem(alpha=0.5):
    n = (8, 6, 2)
    return Problem(n, (2.5e-9, 2.5e-9, 3e-9), Ms=8e5, A=1.3e-11, alpha=alpha,
                   Ku1=5e4, ku_axis=(0.0, 0.6, 0.8), h_ext=(0.01 / MU0, 0.0, 0.0))


def test_energy_decreases_under_damping_and_norm_is_kept():
    prob = _small_problem()
    rng = np.random.default_rng(7)
    m = normalize(rng.normal(size=prob.n + (3,)))
    E_prev = sum(prob.energies(m, 0.0))
    dt = 5e-14
    for s in range(40):
        m = rk4_step(prob, m, s * dt, dt)
        assert np.max(np.abs(np.linalg.norm(m, axis=-1) - 1.0)) < 1e-14
        E = sum(prob.energies(m, (s + 1) * dt))
        assert E <= E_prev + 1e-12 * abs(E_prev)
        E_prev = E


def test_relax_macrospin_aligns_with_field():
    prob = _macrospin(alpha=1.0, H=8e4)
    m, steps, tq, t = relax(prob, _m0(2.0, 0.1), tol=1e-3, max_steps=20000)
    assert tq < 1e-3
    assert steps > 0
    # the torque |m x h| / Ms < 1e-3 means sin(theta) < 1e-3 Ms / |h|
    hz = 8e4 - 8e5 / 3.0 * m[0, 0, 0, 2] + 8e5 / 3.0 * m[0, 0, 0, 2]
    assert math.sin(math.acos(min(1.0, m[0, 0, 0, 2]))) < 2e-3 * 8e5 / hz


def test_rkf45_tableau_order_conditions():
    c = np.array(RKF_C)
    b4 = np.array(RKF_B4)
    b5 = np.array(RKF_B5)
    A = np.zeros((6, 6))
    for i, row in enumerate(RKF_A):
        A[i, : len(row)] = row
    assert np.allclose(A.sum(axis=1), c, atol=1e-15)
    # the propagated weights are of order 4 (all eight conditions), not 5
    for q in range(4):
        assert abs(b4 @ c ** q - 1.0 / (q + 1)) < 1e-14
    assert abs(b4 @ (A @ c) - 1.0 / 6) < 1e-14
    assert abs(b4 @ (c * (A @ c)) - 1.0 / 8) < 1e-14
    assert abs(b4 @ (A @ c ** 2) - 1.0 / 12) < 1e-14
    assert abs(b4 @ (A @ (A @ c)) - 1.0 / 24) < 1e-14
    assert abs(b4 @ c ** 4 - 1.0 / 5) > 1e-6
    # the control weights are of order 5
    for q in range(5):
        assert abs(b5 @ c ** q - 1.0 / (q + 1)) < 1e-14
    assert abs(b5 @ (A @ c) - 1.0 / 6) < 1e-14
    assert abs(b5 @ (A @ (A @ c)) - 1.0 / 24) < 1e-14
    assert abs(b5 @ (A @ c ** 3) - 1.0 / 20) < 1e-14
    assert abs(b5 @ (c * (A @ (A @ c))) - 1.0 / 30) < 1e-14
    assert abs(b5 @ ((A @ c) * (A @ c)) - 1.0 / 20) < 1e-14
    assert abs(b5 @ (c ** 2 * (A @ c)) - 1.0 / 10) < 1e-14
    assert abs(b5 @ (A @ (A @ (A @ c))) - 1.0 / 120) < 1e-14


def test_rkf45_fixed_step_fourth_order():
    alpha, H, T = 0.1, 8e4, 2e-10
    prob = _macrospin(alpha, H)
    th0, ph0 = 2.5, 0.3
    errs = []
    for nsteps in (20, 40, 80):
        dt = T / nsteps
        m = _m0(th0, ph0)
        for s in range(nsteps):
            m, _ = rkf45_attempt(prob, m, s * dt, dt, prob.rhs(m, s * dt), rtol=1e-5)
        errs.append(np.max(np.abs(m[0, 0, 0] - _exact(th0, ph0, alpha, H, T))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13.0 < r1 < 19.0 and 13.0 < r2 < 19.0


def test_rkf45_adaptive_meets_tolerance():
    alpha, H, T = 0.1, 8e4, 5e-10
    prob = _macrospin(alpha, H)
    th0, ph0 = 2.5, 0.3
    errs = {}
    for rtol in (1e-5, 1e-7):
        m, t, dt = _m0(th0, ph0), 0.0, 1e-13
        while t < T:
            m, t, dt = rkf45_step(prob, m, t, min(dt, T - t), rtol)
        errs[rtol] = np.max(np.abs(m[0, 0, 0] - _exact(th0, ph0, alpha, H, T)))
        assert errs[rtol] < 100 * rtol
    assert errs[1e-7] < errs[1e-5]


def test_damping_only_macrospin_closed_form():
    """Without the precession term the azimuth stays fixed while the polar
    angle relaxes as tan(theta/2) = tan(theta0/2) exp(-alpha gamma' H t)."""
    alpha, H, T = 0.5, 8e4, 1e-10
    prob = _macrospin(alpha, H, precession=False)
    th0, ph0 = 2.5, 0.3
    m = _m0(th0, ph0)
    n = 400
    for s in range(n):
        m = rk4_step(prob, m, s * T / n, T / n)
    gp = GAMMA / (1 + alpha ** 2)
    th = 2 * math.atan(math.tan(th0 / 2) * math.exp(-alpha * gp * H * T))
    exact = np.array([math.sin(th) * math.cos(ph0), math.sin(th) * math.sin(ph0), math.cos(th)])
    assert np.max(np.abs(m[0, 0, 0] - exact)) < 1e-9
    # the right-hand side is the damping summand alone
    rng = np.random.default_rng(3)
    mm = normalize(rng.normal(size=(2, 2, 1, 3)))
    hh = rng.normal(size=(2, 2, 1, 3)) * 1e5
    full = llg_rhs(mm, hh, alpha)
    prec = -gp * np.cross(mm, hh)
    assert np.allclose(llg_rhs(mm, hh, alpha, precession=False), full - prec, rtol=1e-13, atol=0)


def test_rkf45_relax_without_precession_aligns():
    prob = _macrospin(alpha=1.0, H=8e4, precession=False)
    m, steps, tq, t = relax(prob, _m0(2.0, 0.1), tol=1e-3, max_steps=20000, method="rkf45")
    assert tq < 1e-3 and steps > 0
    # no precession: the azimuth of the initial state is kept
    assert abs(math.atan2(m[0, 0, 0, 1], m[0, 0, 0, 0]) - 0.1) < 1e-9
