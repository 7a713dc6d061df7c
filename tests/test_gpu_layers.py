"""GPU parity of non-equidistant layers (Sec. 4.4): demag with the lateral
FFT and dense layer coupling, thickness-weighted exchange links and per-layer
cell volumes, against the oracle; RK4 trajectories; the full-size stack on
sampled cells; the reduction to the equidistant grid; RKF45 steps and relax
without precession; refusals."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, rel, to_host

pytestmark = pytest.mark.gpu

GRIDS = [(24, 20, 5), (33, 7, 3), (16, 1, 4), (40, 30, 2), (12, 9, 8)]


def _setup(n, precision, demag=True):
    from oracle.llg import Problem
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import State
    from paper_2302_08843_gb300.workloads import to_soa
    w = W.multilayer(n=n)
    h = w.extra["layers"]
    s = State(w.n, w.dx, precision)
    s.set_material(Ms=0.0, A=0.0, alpha=w.alpha, Ku1=0.0, ku_axis=w.ku_axis,
                   Ms_cell=to_soa(w.Ms), A_cell=to_soa(w.A), Ku1_cell=to_soa(w.Ku1))
    s.set_zeeman(h=w.h_ext)
    s.set_layers(h)
    if demag:
        s.demag_setup(20)
    else:
        s.demag_disable()
    s.set_m(to_soa(w.m0))
    prob = Problem(w.n, w.dx, Ms=w.Ms, A=w.A, alpha=w.alpha, Ku1=w.Ku1, ku_axis=w.ku_axis, h_ext=w.h_ext,
                   p=20, demag=demag, layers=h)
    return w, s, prob


def _tol(precision, w):
    from oracle.layers import layered_rounding_sensitivity
    if precision == "fp32":
        return FP32_TOL
    M = w.m0 * np.asarray(w.Ms)[..., None]
    return max(1e-10, layered_rounding_sensitivity(w.n, w.dx[0], w.dx[1], w.extra["layers"], 20, M))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n", GRIDS)
def test_layers_field_and_energy(n, precision):
    from paper_2302_08843_gb300.workloads import from_soa
    w, s, prob = _setup(n, precision)
    t = 2.0e-12
    h, E = s.heff(t=t, energies=True)
    ref = prob.heff(w.m0, t)
    Eref = prob.energies(w.m0, t)
    tol = _tol(precision, w)
    assert rel(from_soa(to_host(h)), ref) < tol
    Escale = max(abs(e) for e in Eref)
    for a, b in zip(E, Eref):
        assert abs(a - b) < tol * Escale, (E, Eref)
    s.close()


@pytest.mark.parametrize("n,precision", [((10, 6, 16), "fp64"), ((10, 6, 16), "fp32"), ((8, 5, 22), "fp32")])
def test_many_layers(n, precision):
    """Stacks whose tensor slice no longer fits one shared-memory copy (16
    layers in FP64, 22 in FP32) take the register-fed coupling kernel; 16
    layers in FP32 still the staged one."""
    from paper_2302_08843_gb300.workloads import from_soa
    w, s, prob = _setup(n, precision)
    h, E = s.heff(energies=True)
    assert rel(from_soa(to_host(h)), prob.heff(w.m0, 0.0)) < _tol(precision, w)
    Eref = prob.energies(w.m0, 0.0)
    Escale = max(abs(e) for e in Eref)
    for a, b in zip(E, Eref):
        assert abs(a - b) < _tol(precision, w) * Escale, (E, Eref)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_layers_demag_alone(precision):
    """Exchange, anisotropy and field off: the demag term alone (the coupling pass)."""
    from oracle.layers import layered_demag_fft, layered_tensor
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import State
    from paper_2302_08843_gb300.workloads import from_soa, to_soa
    w = W.multilayer(n=(20, 18, 6))
    hl = w.extra["layers"]
    s = State(w.n, w.dx, precision)
    s.set_material(Ms=0.0, A=0.0, alpha=0.1, Ms_cell=to_soa(w.Ms))
    s.set_layers(hl)
    s.demag_setup(20)
    s.set_m(to_soa(w.m0))
    h, _ = s.heff(energies=True)
    ref = layered_demag_fft(layered_tensor(w.n, w.dx[0], w.dx[1], hl, 20), w.m0 * w.Ms[..., None])
    assert rel(from_soa(to_host(h)), ref) < _tol(precision, w)
    s.close()


def test_layers_without_demag():
    from paper_2302_08843_gb300.workloads import from_soa
    w, s, prob = _setup((24, 20, 5), "fp64", demag=False)
    h, E = s.heff(energies=True)
    assert rel(from_soa(to_host(h)), prob.heff(w.m0, 0.0)) < 1e-12
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 5 * FP32_TOL)])
def test_layers_rk4_trajectory(precision, tol):
    from oracle.llg import rk4_step
    from paper_2302_08843_gb300.workloads import from_soa
    w, s, prob = _setup((24, 20, 5), precision)
    m, t = w.m0.copy(), 0.0
    for _ in range(5):
        m = rk4_step(prob, m, t, w.dt)
        t, _ = s.step(w.dt, t, "rk4")
    assert rel(from_soa(to_host(s.get_m())), m) < tol
    s.close()


def test_layers_rk4_fp32_through_the_fused_kernel():
    """FP32 RK4 on a stack with a power-of-two x line runs the fused stage
    kernel with per-cell materials and per-layer z links (checked from the
    launch record); five steps against the oracle."""
    from oracle.llg import rk4_step
    from paper_2302_08843_gb300.workloads import from_soa
    w, s, prob = _setup((32, 20, 5), "fp32")
    s.profile_enable(True)
    m, t = w.m0.copy(), 0.0
    for _ in range(5):
        m = rk4_step(prob, m, t, w.dt)
        t, _ = s.step(w.dt, t, "rk4")
    prof = s.profile_read()
    s.profile_enable(False)
    assert "k5_fused" in prof and "stage_llg" not in prof, prof
    assert rel(from_soa(to_host(s.get_m())), m) < 5 * FP32_TOL
    s.close()


def test_layers_dp45_steps():
    """Adaptive steps: the accepted times, step sizes and states follow the oracle."""
    from oracle.llg import dp45_attempt, dp45_factor, normalize
    from paper_2302_08843_gb300.workloads import from_soa
    w, s, prob = _setup((24, 20, 5), "fp64")
    rtol = 1e-5
    m, t, dt = w.m0.copy(), 0.0, 1e-14
    k1 = prob.rhs(m, t)
    tg, dtg = 0.0, 1e-14
    for _ in range(6):
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
    assert rel(from_soa(to_host(s.get_m())), m) < 1e-9
    s.close()


def test_equal_layers_equal_equidistant_grid():
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import State
    from paper_2302_08843_gb300.workloads import to_soa
    w = W.multilayer(n=(24, 20, 5))
    dz = 1.3e-9
    out = []
    for layered in (False, True):
        s = State(w.n, (w.dx[0], w.dx[1], dz), "fp64")
        s.set_material(Ms=0.0, A=0.0, alpha=0.1, Ku1=0.0, ku_axis=(0, 0, 1),
                       Ms_cell=to_soa(w.Ms), A_cell=to_soa(w.A), Ku1_cell=to_soa(w.Ku1))
        if layered:
            s.set_layers([dz] * 5)
        s.demag_setup(20)
        s.set_m(to_soa(w.m0))
        h, E = s.heff(energies=True)
        out.append((to_host(h), np.array(E)))
        s.close()
    assert rel(out[1][0], out[0][0]) < 1e-10
    assert np.max(np.abs(out[1][1] - out[0][1])) < 1e-10 * np.max(np.abs(out[0][1]))


def test_full_size_stack_sampled_cells():
    """The 256x256x8 stack in FP32 (as timed): demag alone at sampled cells
    against the oracle's direct sum over all 524288 source cells."""
    from oracle.layers import layered_demag_at
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import State
    from paper_2302_08843_gb300.workloads import from_soa, to_soa
    w = W.multilayer()
    hl = w.extra["layers"]
    s = State(w.n, w.dx, "fp32")
    s.set_material(Ms=0.0, A=0.0, alpha=0.1, Ms_cell=to_soa(w.Ms))
    s.set_layers(hl)
    s.demag_setup(20)
    s.set_m(to_soa(w.m0))
    h, _ = s.heff(energies=True)
    hg = from_soa(to_host(h))
    rng = np.random.default_rng(12)
    cells = [(0, 0, 0), (255, 255, 7), (128, 3, 2), (7, 200, 5)]
    cells += [tuple(int(v) for v in (rng.integers(256), rng.integers(256), rng.integers(8))) for _ in range(4)]
    ref = layered_demag_at(w.n, w.dx[0], w.dx[1], hl, w.m0 * w.Ms[..., None], cells, 20)
    got = np.array([hg[x, y, z] for (x, y, z) in cells])
    assert np.max(np.abs(got - ref)) < FP32_TOL * float(np.max(w.Ms)), (got, ref)
    s.close()


def test_layers_refusals():
    import torch
    from paper_2302_08843_gb300.binding import MMError, STATUS_NAMES
    w, s, _ = _setup((24, 20, 5), "fp64")

    def code(fn):
        with pytest.raises(MMError) as e:
            fn()
        return STATUS_NAMES[e.value.status]

    assert code(lambda: s.set_layers([1e-9] * 4)) == "MM_EINVAL"
    assert code(lambda: s.set_layers([1e-9, 1e-9, -1e-9, 1e-9, 1e-9])) == "MM_EINVAL"
    assert code(lambda: s.set_layers([1e-9, 1e-9, float("nan"), 1e-9, 1e-9])) == "MM_EINVAL"
    assert code(lambda: s.set_dmi("interface", 1e-3)) == "MM_EINVAL"
    m = s.get_m().clone()
    assert code(lambda: s.step_adjoint(m, torch.zeros_like(m), w.dt)) == "MM_EINVAL"
    # a new stack invalidates the tensor until demag_setup
    s.set_layers(w.extra["layers"][::-1].copy())
    assert code(lambda: s.heff()) == "MM_ENOTSETUP"
    s.set_layers(None)
    s.set_dmi("interface", 1e-3)
    assert code(lambda: s.set_layers(w.extra["layers"])) == "MM_EINVAL"
    s.close()


def test_layers_rkf45_steps():
    """RKF45 (the paper's default solver) on the stack: accepted times, step sizes, states."""
    from oracle.llg import rkf45_step
    from paper_2302_08843_gb300.workloads import from_soa
    w, s, prob = _setup((24, 20, 5), "fp64")
    rtol = 1e-5
    m, t, dt = w.m0.copy(), 0.0, 1e-14
    tg, dtg = 0.0, 1e-14
    for step in range(6):
        m, t, dt = rkf45_step(prob, m, t, dt, rtol)
        tg, dtg = s.step(dtg, tg, "rkf45", rtol)
        assert abs(tg - t) <= 1e-9 * t and abs(dtg - dt) <= 1e-6 * dt, (step, tg, t, dtg, dt)
    assert rel(from_soa(to_host(s.get_m())), m) < 1e-9
    s.close()


def test_layers_relax_without_precession():
    """Relax (RKF45, no precession term) of a small three-layer stack: step
    count, torque, time and state."""
    from oracle.llg import Problem, relax
    from paper_2302_08843_gb300.binding import State
    from paper_2302_08843_gb300.workloads import from_soa, to_soa
    rng = np.random.default_rng(33)
    n = (12, 8, 3)
    hl = [3e-9, 1.5e-9, 4e-9]
    m0 = rng.normal(size=n + (3,))
    m0 /= np.linalg.norm(m0, axis=-1, keepdims=True)
    s = State(n, (3e-9, 3e-9, 1e-9), "fp64")
    s.set_material(Ms=8e5, A=1.3e-11, alpha=1.0)
    s.set_layers(hl)
    s.demag_setup(20)
    s.set_m(to_soa(m0))
    s.set_llg_options(relax_method="rkf45", precession=False)
    steps, tq, t, _ = s.relax(tol=1e-3, max_steps=3000, rtol=1e-5)
    prob = Problem(n, (3e-9, 3e-9, 1e-9), Ms=8e5, A=1.3e-11, alpha=1.0, p=20, precession=False, layers=hl)
    mr, steps_r, tq_r, t_r = relax(prob, m0, tol=1e-3, max_steps=3000, method="rkf45")
    assert steps == steps_r
    assert tq < 1e-3 and abs(tq - tq_r) < 1e-6 * tq_r
    # each accepted step sets the next from err^(-1/5), err a difference of two
    # nearly equal solutions; the layered tensor's FP64 rounding floor is about 3x
    # the equidistant one (layered_rounding_sensitivity), and over ~1000 controller
    # updates the time and state agree to ~1e-8 (1e-9 on the equidistant grid)
    assert abs(t - t_r) <= 1e-7 * t_r
    assert rel(from_soa(to_host(s.get_m())), mr) < 1e-7
    s.close()
