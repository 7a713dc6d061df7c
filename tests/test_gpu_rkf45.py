"""GPU parity of the Runge-Kutta-Fehlberg 4(5) integrator (the paper's
default solver, Sec. 3) and of the LLG without the precession term: accepted
step sizes and states against the oracle, relaxation without precession, the
fused FP32 RK4 path with the term switched off, and the adjoint without it."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, oracle_problem, rel, to_host

pytestmark = pytest.mark.gpu


def test_rkf45_steps_match_oracle():
    from oracle.llg import rkf45_step
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.workloads import from_soa
    w = W.thin_film(n=(64, 32, 1))
    s = setup_workload(w, "fp64")
    prob = oracle_problem(w)
    rtol = w.extra["rtol"]
    m, t, dt = w.m0.copy(), 0.0, 1e-13
    tg, dtg = 0.0, 1e-13
    for step in range(12):
        m, t, dt = rkf45_step(prob, m, t, dt, rtol)
        tg, dtg = s.step(dtg, tg, "rkf45", rtol)
        assert abs(tg - t) <= 1e-9 * t and abs(dtg - dt) <= 1e-6 * dt, (step, tg, t, dtg, dt)
    assert rel(from_soa(to_host(s.get_m())), m) < 1e-9
    s.close()


def test_rkf45_relax_without_precession_matches_oracle():
    """Relaxation without the precession term: the same number of accepted
    steps as the oracle, and the final torque, time and state within a bound
    measured from the oracle's own spread.  An adaptive run is a chaotic
    function of rounding (each accepted step sets the next from err^(-1/5),
    err a difference of two nearly equal solutions), so the oracle is rerun
    with rounding-level changes -- m0 perturbed by 1e-15 (three random-sign
    draws) and the Newell tensor evaluated with the cell size in nanometres --
    and the bounds are ten times the largest change seen (measured: 5e-8 in
    the relaxed time, 3e-9 in m, 5e-7 in the torque), never below 1e-9
    (time), 1e-8 (m) and 1e-6 (torque).  The step count must match exactly."""
    from oracle.llg import Problem, relax
    from oracle.newell import demag_tensor
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.workloads import Workload, from_soa
    rng = np.random.default_rng(31)
    n = (16, 8, 2)
    m0 = rng.normal(size=n + (3,))
    m0 /= np.linalg.norm(m0, axis=-1, keepdims=True)
    w = Workload("relax 16x8x2", n, (3e-9, 3e-9, 3e-9), Ms=8e5, A=1.3e-11, alpha=1.0, m0=m0)
    s = setup_workload(w, "fp64")
    s.set_llg_options(relax_method="rkf45", precession=False)
    steps, tq, t, _ = s.relax(tol=1e-3, max_steps=5000, rtol=1e-5)

    def oracle_relax(m_start, Nt=None):
        prob = Problem(n, w.dx, Ms=w.Ms, A=w.A, alpha=w.alpha, precession=False, Nt=Nt)
        return relax(prob, m_start, tol=1e-3, max_steps=5000, method="rkf45")

    mr, steps_r, tq_r, t_r = oracle_relax(m0)
    d_t = d_m = d_tq = 0.0
    variants = [m0 * (1.0 + 1e-15 * np.random.default_rng(100 + k).choice([-1.0, 1.0], size=m0.shape))
                for k in range(3)]
    runs = [oracle_relax(v) for v in variants]
    runs.append(oracle_relax(m0, demag_tensor(n, tuple(v * 1e9 for v in w.dx), 20)))
    for mv, steps_v, tq_v, t_v in runs:
        assert steps_v == steps_r
        d_t = max(d_t, abs(t_v - t_r) / t_r)
        d_m = max(d_m, rel(mv, mr))
        d_tq = max(d_tq, abs(tq_v - tq_r) / tq_r)
    assert steps == steps_r
    assert tq < 1e-3 and abs(tq - tq_r) <= max(1e-6, 10 * d_tq) * tq_r, (tq, tq_r, d_tq)
    assert abs(t - t_r) <= max(1e-9, 10 * d_t) * t_r, (t, t_r, d_t)
    assert rel(from_soa(to_host(s.get_m())), mr) < max(1e-8, 10 * d_m), d_m
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 5 * FP32_TOL)])
def test_rk4_without_precession(precision, tol):
    """FP32 runs the fused stage kernel, FP64 the separate passes."""
    from oracle.llg import Problem, rk4_step
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.workloads import from_soa
    w = W.plain_fp64()
    s = setup_workload(w, precision)
    s.set_llg_options(precession=False)
    prob = Problem(w.n, w.dx, Ms=w.Ms, A=w.A, alpha=w.alpha, h_ext=w.h_ext, precession=False)
    m, t = w.m0.copy(), 0.0
    for _ in range(5):
        m = rk4_step(prob, m, t, w.dt)
        t, _ = s.step(w.dt, t, "rk4")
    assert rel(from_soa(to_host(s.get_m())), m) < tol
    s.close()


def test_adjoint_without_precession_matches_oracle():
    """One RK4 step's adjoint with the precession term switched off, against
    the oracle's FP64 adjoint of the same right-hand side."""
    import torch
    from oracle.adjoint import rk4_step_vjp
    from oracle.constants import MU0
    from oracle.llg import Problem, normalize
    from paper_2302_08843_gb300.binding import State
    from paper_2302_08843_gb300.workloads import from_soa, to_soa
    n, d = (8, 6, 3), (3e-9, 2.5e-9, 3e-9)
    rng = np.random.default_rng(41)
    Ms = rng.uniform(5e5, 1e6, size=n)
    m = normalize(rng.normal(size=n + (3,)))
    lam1 = rng.normal(size=n + (3,))
    h = (0.02 / MU0, 0.01 / MU0, 0.0)
    prob = Problem(n, d, Ms=Ms, A=1.3e-11, alpha=0.3, Ku1=2e5, ku_axis=(0.0, 0.6, 0.8), h_ext=h, precession=False)
    dt, t = 5e-14, 0.0
    lam_ref, g_ref = rk4_step_vjp(prob, m, t, dt, lam1)
    s = State(n, d, "fp64")
    s.set_material(Ms=0.0, A=1.3e-11, alpha=0.3, Ku1=2e5, ku_axis=(0.0, 0.6, 0.8), Ms_cell=to_soa(Ms))
    s.set_zeeman(h=h)
    s.set_llg_options(precession=False)
    s.demag_setup(20)
    gMs = torch.zeros((n[2], n[1], n[0]), dtype=torch.float64, device="cuda")
    lam = s.step_adjoint(to_soa(m), to_soa(lam1), dt, t, grad_Ms=gMs)
    assert rel(from_soa(to_host(lam)), lam_ref) < 1e-9
    assert rel(from_soa(to_host(gMs)), g_ref) < 1e-9
    s.close()
