"""GPU parity of the DMI term (Sec. 4.3): field and energy for the three DMI
types with uniform D and with a per-cell D of mixed signs (the link averaging
of Eq. D_avg), RK4 trajectories through the fused FP32 stage kernel and the
FP64 passes, and the adjoint's refusal."""
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


def test_adjoint_refuses_dmi():
    import torch
    from paper_2302_08843_gb300.binding import MMError, STATUS_NAMES
    w, s, _ = _setup("fp64", "bulk", 2e-3)
    m = s.get_m().clone()
    with pytest.raises(MMError) as e:
        s.step_adjoint(m, torch.zeros_like(m), w.dt)
    assert STATUS_NAMES[e.value.status] == "MM_EINVAL"
    s.close()
