"""Pins for the oracle's hand-derived adjoint: dot-product (transpose) tests of
the LLG right-hand side and of one RK4 step against their tangent-linear
maps by central differences, and the gradient of a short rollout with respect
to per-cell Ms against central finite differences (Sec. 5.2 computes the same
derivatives with autograd)."""
import numpy as np
import pytest

from oracle.adjoint import rhs_vjp, rk4_step_vjp, rollout_loss_and_grad
from oracle.constants import MU0
from oracle.llg import Problem, normalize, rk4_step


def _prob(Ms):
    return Problem((6, 5, 2), (3e-9, 3e-9, 3e-9), Ms=Ms, A=1.3e-11, alpha=0.3, Ku1=2e5,
                   ku_axis=(0.0, 0.6, 0.8), h_ext=(0.02 / MU0, 0.01 / MU0, 0.0))


def _state(seed, n=(6, 5, 2)):
    rng = np.random.default_rng(seed)
    return normalize(rng.normal(size=n + (3,)))


def test_rhs_vjp_matches_central_differences():
    rng = np.random.default_rng(1)
    Ms = rng.uniform(5e5, 1e6, size=(6, 5, 2))
    prob = _prob(Ms)
    m = _state(2)
    u = rng.normal(size=m.shape)
    dm = rng.normal(size=m.shape)
    lam, gMs = rhs_vjp(prob, m, 0.0, u)
    eps = 1e-6
    fd = (np.sum(u * prob.rhs(m + eps * dm, 0.0)) - np.sum(u * prob.rhs(m - eps * dm, 0.0))) / (2 * eps)
    assert abs(np.sum(lam * dm) - fd) < 1e-7 * abs(fd)
    dMs = rng.normal(size=Ms.shape) * 1e4
    p1, p2 = _prob(Ms + eps * dMs), _prob(Ms - eps * dMs)
    fd2 = (np.sum(u * p1.rhs(m, 0.0)) - np.sum(u * p2.rhs(m, 0.0))) / (2 * eps)
    assert abs(np.sum(gMs * dMs) - fd2) < 1e-7 * abs(fd2)


def test_rk4_step_vjp_matches_central_differences():
    rng = np.random.default_rng(3)
    Ms = rng.uniform(5e5, 1e6, size=(6, 5, 2))
    prob = _prob(Ms)
    m = _state(4)
    lam_next = rng.normal(size=m.shape)
    dm = rng.normal(size=m.shape)
    dt = 5e-14
    lam, gMs = rk4_step_vjp(prob, m, 0.0, dt, lam_next)
    eps = 1e-6
    fd = (np.sum(lam_next * rk4_step(prob, m + eps * dm, 0.0, dt))
          - np.sum(lam_next * rk4_step(prob, m - eps * dm, 0.0, dt))) / (2 * eps)
    assert abs(np.sum(lam * dm) - fd) < 1e-8 * max(abs(fd), 1.0)
    dMs = rng.normal(size=Ms.shape) * 1e4
    fd2 = (np.sum(lam_next * rk4_step(_prob(Ms + eps * dMs), m, 0.0, dt))
           - np.sum(lam_next * rk4_step(_prob(Ms - eps * dMs), m, 0.0, dt))) / (2 * eps)
    assert abs(np.sum(gMs * dMs) - fd2) < 1e-6 * abs(fd2)


def test_rollout_gradient_matches_finite_differences():
    n = (5, 4, 1)
    rng = np.random.default_rng(5)
    Ms0 = rng.uniform(5e5, 1e6, size=n)
    m0 = _state(6, n)
    weight = np.zeros(n + (3,))
    weight[3:, 2:, :, 1] = 1.0
    def factory(Ms):
        return Problem(n, (5e-9, 5e-9, 5e-9), Ms=Ms, A=1.3e-11, alpha=0.05,
                       h_ext=lambda t: np.array([0.0, 0.005 / MU0 * np.cos(3e10 * t), 0.0]))
    L, g = rollout_loss_and_grad(factory, Ms0, m0, 5e-14, 12, weight)
    eps = 1.0            # A/m on Ms ~ 1e6
    for idx in [(0, 0, 0), (2, 1, 0), (4, 3, 0)]:
        e = np.zeros(n)
        e[idx] = eps
        Lp, _ = rollout_loss_and_grad(factory, Ms0 + e, m0, 5e-14, 12, weight)
        Lm, _ = rollout_loss_and_grad(factory, Ms0 - e, m0, 5e-14, 12, weight)
        fd = (Lp - Lm) / (2 * eps)
        assert abs(g[idx] - fd) < 1e-5 * abs(fd) + 1e-18, (idx, g[idx], fd)


def _prob_dmi(Ms, D, kind, precession):
    return Problem((6, 5, 2), (3e-9, 3e-9, 3e-9), Ms=Ms, A=1.3e-11, alpha=0.3, Ku1=2e5,
                   ku_axis=(0.0, 0.6, 0.8), h_ext=(0.02 / MU0, 0.01 / MU0, 0.0), D=D, dmi=kind,
                   precession=precession)


@pytest.mark.parametrize("kind,precession", [("interface", True), ("bulk", True), ("d2d", False),
                                             ("interface", False)])
def test_rhs_and_step_vjp_with_dmi_and_precession_switch(kind, precession):
    """The adjoint with DMI (Sec. 4.3; per-cell D of both signs, so every branch
    of the link average of Eq. D_avg is differentiated) and with the LLG
    without its precession term (Sec. 3), against central differences of the
    oracle's own forward map: the right-hand side in m and in Ms, and one RK4
    step with renormalisation in m and in Ms."""
    rng = np.random.default_rng(11)
    n = (6, 5, 2)
    Ms = rng.uniform(5e5, 1e6, size=n)
    D = rng.uniform(-3e-3, 3e-3, size=n)
    prob = _prob_dmi(Ms, D, kind, precession)
    m = _state(12)
    u = rng.normal(size=m.shape)
    dm = rng.normal(size=m.shape)
    lam, gMs = rhs_vjp(prob, m, 0.0, u)
    eps = 1e-6
    fd = (np.sum(u * prob.rhs(m + eps * dm, 0.0)) - np.sum(u * prob.rhs(m - eps * dm, 0.0))) / (2 * eps)
    assert abs(np.sum(lam * dm) - fd) < 1e-7 * abs(fd)
    # Ms steps: eps_ms dMs is ~1 A/m, where the differences are no longer
    # rounding-dominated (relative agreement ~1e-9; ~1e-7 at 100x smaller steps)
    dMs = rng.normal(size=n) * 1e4
    e2 = 1e-4
    fd2 = (np.sum(u * _prob_dmi(Ms + e2 * dMs, D, kind, precession).rhs(m, 0.0))
           - np.sum(u * _prob_dmi(Ms - e2 * dMs, D, kind, precession).rhs(m, 0.0))) / (2 * e2)
    assert abs(np.sum(gMs * dMs) - fd2) < 1e-7 * abs(fd2)
    dt = 5e-14
    lam_next = rng.normal(size=m.shape)
    lam, gMs = rk4_step_vjp(prob, m, 0.0, dt, lam_next)
    fd = (np.sum(lam_next * rk4_step(prob, m + eps * dm, 0.0, dt))
          - np.sum(lam_next * rk4_step(prob, m - eps * dm, 0.0, dt))) / (2 * eps)
    assert abs(np.sum(lam * dm) - fd) < 1e-8 * max(abs(fd), 1.0)
    fd2 = (np.sum(lam_next * rk4_step(_prob_dmi(Ms + e2 * dMs, D, kind, precession), m, 0.0, dt))
           - np.sum(lam_next * rk4_step(_prob_dmi(Ms - e2 * dMs, D, kind, precession), m, 0.0, dt))) / (2 * e2)
    assert abs(np.sum(gMs * dMs) - fd2) < 1e-6 * abs(fd2)


def test_dmi_adjoint_term_is_needed():
    """A planted mistake -- the adjoint without its DMI term -- fails the
    central-difference check above by far (so that check sees the term)."""
    import oracle.adjoint as OA
    rng = np.random.default_rng(13)
    n = (6, 5, 2)
    Ms = rng.uniform(5e5, 1e6, size=n)
    D = rng.uniform(1e-3, 3e-3, size=n)
    prob = _prob_dmi(Ms, D, "bulk", True)
    m = _state(14)
    u = rng.normal(size=m.shape)
    dm = rng.normal(size=m.shape)
    eps = 1e-6
    fd = (np.sum(u * prob.rhs(m + eps * dm, 0.0)) - np.sum(u * prob.rhs(m - eps * dm, 0.0))) / (2 * eps)
    real = OA.dmi_field
    try:
        OA.dmi_field = lambda mm, *a, **k: np.zeros_like(mm)
        lam_wrong, _ = OA.rhs_vjp(prob, m, 0.0, u)
    finally:
        OA.dmi_field = real
    assert abs(np.sum(lam_wrong * dm) - fd) > 1e-4 * abs(fd)
