"""GPU parity of the DMI term (Sec. 4.3): field and energy for the three DMI
types with uniform D and with a per-cell D of mixed signs (the link averaging
of Eq. D_avg), RK4 trajectories through the fused FP32 stage kernel and the
FP64 passes, and the adjoint of a step with DMI against the oracle's."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, rel, to_host

pytestmark = pytest.mark.gpu


def _setup(precision, kind, D, D_cell=None):
    from oracle.llg import Problem
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.workloads import to_soa
    w = W.plain_fp64()
    s = setup_workload(w, precision)
    s.set_dmi(kind, D, None if D_cell is None else to_soa(D_cell))
    prob = Problem(w.n, w.dx, Ms=w.Ms, A=w.A, alpha=w.alpha, h_ext=w.h_ext,
                   D=D if D_cell is None else D_cell, dmi=kind)
    return w, s, prob


def _tol(precision, w):
    from oracle.demag import magnetization, rounding_sensitivity
    if precision == "fp32":
        return FP32_TOL
    return max(1e-10, rounding_sensitivity(w.n, w.dx, 20, magnetization(w.m0, w.Ms)))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("kind", ["interface", "bulk", "d2d"])
@pytest.mark.parametrize("cellwise", [False, True])
def test_dmi_field_and_energy(kind, precision, cellwise):
    from paper_2302_08843_gb300.workloads import from_soa
    D_cell = None
    if cellwise:
        rng = np.random.default_rng(11)
        D_cell = rng.uniform(-3e-3, 3e-3, size=(32, 32, 4))
    w, s, prob = _setup(precision, kind, 3e-3, D_cell)
    t = 1.3e-11
    h, E = s.heff(t=t, energies=True)
    ref = prob.heff(w.m0, t)
    Eref = prob.energies(w.m0, t)
    tol = _tol(precision, w)
    assert rel(from_soa(to_host(h)), ref) < tol
    assert len(E) == 5 and abs(Eref[4]) > 0
    Escale = max(abs(e) for e in Eref)
    for a, b in zip(E, Eref):
        assert abs(a - b) < tol * Escale, (E, Eref)
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 5 * FP32_TOL)])
def test_rk4_with_dmi(precision, tol):
    """FP32 runs the fused stage kernel (uniform D), FP64 the separate passes."""
    from oracle.llg import rk4_step
    from paper_2302_08843_gb300.workloads import from_soa
    w, s, prob = _setup(precision, "interface", 3e-3)
    m, t = w.m0.copy(), 0.0
    for _ in range(5):
        m = rk4_step(prob, m, t, w.dt)
        t, _ = s.step(w.dt, t, "rk4")
    assert rel(from_soa(to_host(s.get_m())), m) < tol
    s.close()


@pytest.mark.parametrize("kind,n", [("interface", (16, 16, 1)), ("bulk", (8, 6, 3)), ("d2d", (8, 6, 3))])
def test_adjoint_with_dmi_matches_oracle(kind, n):
    """One RK4 step's adjoint (mm_llg_step_adjoint) with DMI and a per-cell D
    of both signs, against the oracle's FP64 adjoint (itself pinned by central
    differences): the cotangent of m and the Ms gradient, per cell."""
    import torch
    from oracle.adjoint import rk4_step_vjp
    from oracle.constants import MU0
    from oracle.llg import Problem, normalize
    from paper_2302_08843_gb300.binding import State
    from paper_2302_08843_gb300.workloads import from_soa, to_soa
    d = (3e-9, 2.5e-9, 3e-9)
    rng = np.random.default_rng(40)
    Ms = rng.uniform(5e5, 1e6, size=n)
    D = rng.uniform(-3e-3, 3e-3, size=n)
    m = normalize(rng.normal(size=n + (3,)))
    lam1 = rng.normal(size=n + (3,))
    h = (0.02 / MU0, 0.01 / MU0, 0.0)
    prob = Problem(n, d, Ms=Ms, A=1.3e-11, alpha=0.3, Ku1=2e5, ku_axis=(0.0, 0.6, 0.8), h_ext=h, D=D, dmi=kind)
    dt, t = 5e-14, 0.0
    lam_ref, g_ref = rk4_step_vjp(prob, m, t, dt, lam1)
    s = State(n, d, "fp64")
    s.set_material(Ms=0.0, A=1.3e-11, alpha=0.3, Ku1=2e5, ku_axis=(0.0, 0.6, 0.8), Ms_cell=to_soa(Ms))
    s.set_zeeman(h=h)
    s.set_dmi(kind, 0.0, to_soa(D))
    s.demag_setup(20)
    gMs = torch.zeros((n[2], n[1], n[0]), dtype=torch.float64, device="cuda")
    lam = s.step_adjoint(to_soa(m), to_soa(lam1), dt, t, grad_Ms=gMs)
    assert rel(from_soa(to_host(lam)), lam_ref) < 1e-9
    assert rel(from_soa(to_host(gMs)), g_ref) < 1e-9
    s.close()
