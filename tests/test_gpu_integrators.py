"""GPU parity of the integrators: RK4 trajectories (m and energies every
step) on the 32x32x4 plain workload, Dormand-Prince 5(4) steps (same
accepted step sizes), relaxation, and the invariants |m| = 1 and energy
decay under damping."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, oracle_problem, rel, to_host

pytestmark = pytest.mark.gpu


def _oracle_trajectory(prob, m0, steps, dt):
    from oracle.llg import rk4_step
    m, t, out = m0.copy(), 0.0, []
    for _ in range(steps):
        m = rk4_step(prob, m, t, dt)
        t += dt
        out.append((m.copy(), sum(prob.energies(m, t))))
    return out


def test_rk4_trajectory_fp64_matches_oracle_every_step():
    """m and the total energy after every one of the 200 RK4 steps, against
    the oracle.  The bound is max(1e-10, the oracle's own trajectory spread),
    the spread measured here two ways: m0 perturbed by 1e-15 (relative, random
    signs), and the Newell tensor evaluated with the cell size in nanometres
    instead of metres (the tensor is dimensionless, so the change is the
    rounding noise of Newell's 27-term sum carried through 800 field
    evaluations).  Measured: 1.4e-13 and 3.7e-10 in m; the library's own FP64
    tensor moves the oracle's trajectory by 1.6e-10."""
    from oracle.newell import demag_tensor
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.workloads import from_soa
    w = W.plain_fp64()
    prob = oracle_problem(w)
    base = _oracle_trajectory(prob, w.m0, w.steps, w.dt)
    rng = np.random.default_rng(99)
    m_pert = w.m0 * (1.0 + 1e-15 * rng.choice([-1.0, 1.0], size=w.m0.shape))
    pert = _oracle_trajectory(prob, m_pert, w.steps, w.dt)
    prob_nm = oracle_problem(w, Nt=demag_tensor(w.n, tuple(v * 1e9 for v in w.dx), 20))
    units = _oracle_trajectory(prob_nm, w.m0, w.steps, w.dt)
    spread_m = max(rel(a[0], b[0]) for other in (pert, units) for a, b in zip(other, base))
    spread_E = max(abs(a[1] - b[1]) / abs(b[1]) for other in (pert, units) for a, b in zip(other, base))
    tol_m, tol_E = max(1e-10, spread_m), max(1e-10, spread_E)
    s = setup_workload(w, "fp64")
    t = 0.0
    worst_m = worst_E = 0.0
    for step in range(w.steps):
        t, _ = s.step(w.dt, t, "rk4")
        mg = from_soa(to_host(s.get_m()))
        _, E = s.heff(t=t, energies=True)
        m_ref, E_ref = base[step]
        worst_m = max(worst_m, rel(mg, m_ref))
        worst_E = max(worst_E, abs(sum(E) - E_ref) / abs(E_ref))
    assert worst_m < tol_m, (worst_m, tol_m)
    assert worst_E < tol_E, (worst_E, tol_E)
    assert np.max(np.abs(np.linalg.norm(mg, axis=-1) - 1.0)) < 1e-14
    s.close()


def test_rk4_fp32_fields_error_vs_fp64_oracle():
    from oracle.llg import rk4_step
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.workloads import from_soa
    w = W.plain_fp64()
    s = setup_workload(w, "fp32")
    prob = oracle_problem(w)
    m = w.m0.copy()
    t = 0.0
    for step in range(20):
        t_new, _ = s.step(w.dt, t, "rk4")
        m = rk4_step(prob, m, t, w.dt)
        t = t_new
    mg = from_soa(to_host(s.get_m()))
    # state error after 20 FP32 steps (each field evaluation <= 1e-5)
    assert rel(mg, m) < 20 * FP32_TOL
    s.close()


def test_energy_decays_and_norm_kept_on_gpu():
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.workloads import from_soa
    w = W.bulk(crop=((0, 32), (0, 32), (0, 8)))
    for precision in ("fp64", "fp32"):
        s = setup_workload(w, precision)
        t = 0.0
        _, E0 = s.heff(t=t, energies=True)
        prev = sum(E0)
        for _ in range(30):
            t, _ = s.step(w.dt, t, "rk4")
            _, E = s.heff(t=t, energies=True)
            assert sum(E) <= prev + (1e-12 if precision == "fp64" else 1e-6) * abs(prev)
            prev = sum(E)
        m = from_soa(to_host(s.get_m()))
        assert np.max(np.abs(np.linalg.norm(m, axis=-1) - 1.0)) < (1e-14 if precision == "fp64" else 1e-6)
        s.close()


def test_dp45_steps_match_oracle():
    from oracle.llg import dp45_attempt, dp45_factor, normalize
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.workloads import from_soa
    w = W.thin_film(n=(64, 32, 1))
    s = setup_workload(w, "fp64")
    prob = oracle_problem(w)
    rtol = w.extra["rtol"]
    m = w.m0.copy()
    t, dt = 0.0, 1e-13
    k1 = prob.rhs(m, t)
    tg, dtg = 0.0, 1e-13
    for step in range(12):
        while True:
            y5, k7, _, err = dp45_attempt(prob, m, t, dt, k1, rtol)
            f = dp45_factor(err)
            if err <= 1.0:
                t += dt
                m = normalize(y5)
                k1 = k7
                dt *= f
                break
            dt *= f
        tg, dtg = s.step(dtg, tg, "dp45", rtol)
        assert abs(tg - t) <= 1e-9 * t and abs(dtg - dt) <= 1e-6 * dt, (tg, t, dtg, dt)
    mg = from_soa(to_host(s.get_m()))
    assert rel(mg, m) < 1e-9
    s.close()


def test_relax_matches_oracle():
    from oracle.llg import relax
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.workloads import Workload, from_soa
    rng = np.random.default_rng(9)
    n = (16, 8, 2)
    m0 = rng.normal(size=n + (3,))
    m0 /= np.linalg.norm(m0, axis=-1, keepdims=True)
    w = Workload("relax 16x8x2", n, (3e-9, 3e-9, 3e-9), Ms=8e5, A=1.3e-11, alpha=1.0, m0=m0)
    s = setup_workload(w, "fp64")
    steps, tq, t, _ = s.relax(tol=1e-3, max_steps=5000, rtol=1e-5)
    prob = oracle_problem(w)
    mr, steps_r, tq_r, t_r = relax(prob, m0, tol=1e-3, max_steps=5000)
    assert steps == steps_r
    assert tq < 1e-3 and abs(tq - tq_r) < 1e-6 * tq_r
    assert rel(from_soa(to_host(s.get_m())), mr) < 1e-8
    s.close()


def test_rk4_fp32_per_cell_materials_through_the_fused_kernel():
    """FP32 RK4 with per-cell Ms, A and Ku1 maps (including a cell with
    Ms = 0) runs the fused stage kernel (checked from the launch record);
    five steps against the oracle."""
    from oracle.llg import Problem, normalize, rk4_step
    from paper_2302_08843_gb300.binding import State
    from paper_2302_08843_gb300.workloads import from_soa, to_soa
    n, d = (32, 12, 6), (2.5e-9, 2.5e-9, 3e-9)
    rng = np.random.default_rng(51)
    Ms = rng.uniform(5e5, 1.1e6, size=n)
    Ms[3, 4, 2] = 0.0
    A = rng.uniform(0.8e-11, 1.6e-11, size=n)
    Ku = rng.uniform(0.0, 3e5, size=n)
    m0 = normalize(rng.normal(size=n + (3,)))
    h = (8000.0, 0.0, 2000.0)
    s = State(n, d, "fp32")
    s.set_material(Ms=0.0, A=0.0, alpha=0.2, Ku1=0.0, ku_axis=(0.0, 0.6, 0.8), Ms_cell=to_soa(Ms),
                   A_cell=to_soa(A), Ku1_cell=to_soa(Ku))
    s.set_zeeman(h=h)
    s.demag_setup(20)
    s.set_m(to_soa(m0))
    prob = Problem(n, d, Ms=Ms, A=A, alpha=0.2, Ku1=Ku, ku_axis=(0.0, 0.6, 0.8), h_ext=h)
    s.profile_enable(True)
    m, t, dt = m0.copy(), 0.0, 5e-14
    for _ in range(5):
        m = rk4_step(prob, m, t, dt)
        t, _ = s.step(dt, t, "rk4")
    prof = s.profile_read()
    s.profile_enable(False)
    assert "k5_fused" in prof and "stage_llg" not in prof, prof
    assert rel(from_soa(to_host(s.get_m())), m) < 5 * FP32_TOL
    s.close()


@pytest.mark.parametrize("n,variant", [((48, 20, 6), "uniform"), ((56, 12, 4), "cells"), ((100, 16, 2), "dmi")])
def test_rk4_fp32_mixed_radix_x_through_the_fused_kernel(n, variant):
    """FP32 RK4 on grids whose padded x line is a compiled mixed-radix length
    (96 = 3 2^5, 112 = 7 2^4, 200 = 25 2^3) runs the fused stage kernel on the
    mixed-radix engine (checked from the launch record): uniform material,
    per-cell maps, and uniform interface DMI; five steps against the oracle."""
    from oracle.llg import Problem, normalize, rk4_step
    from paper_2302_08843_gb300.binding import State, padded_extents
    from paper_2302_08843_gb300.workloads import from_soa, to_soa
    assert padded_extents(n)[0] in (96, 112, 200)
    d = (2.5e-9, 2.5e-9, 3e-9)
    rng = np.random.default_rng(52)
    m0 = normalize(rng.normal(size=n + (3,)))
    h = (8000.0, 0.0, 2000.0)
    s = State(n, d, "fp32")
    kw = dict(alpha=0.2, ku_axis=(0.0, 0.6, 0.8), h_ext=h)
    if variant == "cells":
        Ms = rng.uniform(5e5, 1.1e6, size=n)
        A = rng.uniform(0.8e-11, 1.6e-11, size=n)
        Ku = rng.uniform(0.0, 3e5, size=n)
        s.set_material(Ms=0.0, A=0.0, alpha=0.2, Ku1=0.0, ku_axis=(0.0, 0.6, 0.8), Ms_cell=to_soa(Ms),
                       A_cell=to_soa(A), Ku1_cell=to_soa(Ku))
        prob = Problem(n, d, Ms=Ms, A=A, Ku1=Ku, **kw)
    else:
        s.set_material(Ms=8e5, A=1.3e-11, alpha=0.2, Ku1=1e5, ku_axis=(0.0, 0.6, 0.8))
        D = 2e-3 if variant == "dmi" else 0.0
        if variant == "dmi":
            s.set_dmi("interface", D)
        prob = Problem(n, d, Ms=8e5, A=1.3e-11, Ku1=1e5, D=D, dmi="interface", **kw)
    s.set_zeeman(h=h)
    s.demag_setup(20)
    s.set_m(to_soa(m0))
    s.profile_enable(True)
    m, t, dt = m0.copy(), 0.0, 5e-14
    for _ in range(5):
        m = rk4_step(prob, m, t, dt)
        t, _ = s.step(dt, t, "rk4")
    prof = s.profile_read()
    s.profile_enable(False)
    assert "k5_fused" in prof and "stage_llg" not in prof, prof
    assert rel(from_soa(to_host(s.get_m())), m) < 5 * FP32_TOL
    s.close()
