"""Parity at the benchmark's full sizes and launch configurations: one RK4 step
of the bulk workload (256x256x64 cells, FP32 fields, the fused TMA path that
bench.py times) against one RK4 step of the FP64 oracle on the same inputs;
the FP32 field and stage derivative on the bulk grid and on the mixed-radix
192x192x48 grid.

The update m_{n+1} - m_n = dt * sum(b_s k_s) is compared relative to its own
size: each field evaluation carries <= 1e-5 relative error in FP32, and m is
stored in FP32 (6e-8 absolute)."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, oracle_problem, to_host

pytestmark = pytest.mark.gpu


def test_bulk_full_size_rk4_step_fp32():
    from oracle.llg import rk4_step
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.workloads import from_soa
    w = W.bulk()
    s = setup_workload(w, "fp32")
    m0_gpu = from_soa(to_host(s.get_m()))
    s.step(w.dt, 0.0, "rk4")
    mg = from_soa(to_host(s.get_m()))
    s.close()
    prob = oracle_problem(w)
    mr = rk4_step(prob, w.m0, 0.0, w.dt)
    inc = np.max(np.abs(mr - w.m0))
    err = np.max(np.abs(mg - mr))
    assert inc > 1e-4                      # the step does move m
    assert err < 2e-5 * inc + 2e-7, (err, inc)
    assert np.max(np.abs(np.linalg.norm(mg, axis=-1) - 1.0)) < 1e-6
    # the GPU's own FP32 copy of m0 differs from the FP64 input by rounding only
    assert np.max(np.abs(m0_gpu - w.m0)) < 1e-7


def test_bulk_full_size_field_fp32():
    """The FP32 effective field (mm_heff: demag, exchange, anisotropy on the
    64 grains, Zeeman) on the whole 256x256x64 bulk grid against the oracle's
    FP64 field of the same input, element by element: relative max-norm
    <= 1e-5.  The oracle evaluates the field at the GPU's own FP32 copy of m0,
    so the comparison measures the field arithmetic, not the input rounding."""
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.workloads import from_soa
    w = W.bulk()
    s = setup_workload(w, "fp32")
    m0_gpu = from_soa(to_host(s.get_m()))
    h = from_soa(to_host(s.heff(t=0.0)))
    s.close()
    ref = oracle_problem(w).heff(m0_gpu, 0.0)
    err = float(np.max(np.abs(h - ref)) / np.max(np.abs(ref)))
    assert err < FP32_TOL, err


def test_bulk_full_size_fused_stage_derivative_fp32():
    """The derivative the fused stage kernel forms (x-inverse of the demag
    spectrum + exchange + anisotropy + Zeeman + Eq. llg) at the bench's size
    and launch configuration, read back through mm_llg_rhs -- which on this
    FP32 uniform-material state runs the same kernels as the timed RK4 stages
    (checked from the launch record) -- against the oracle's FP64 llg_rhs of
    its own field, element by element: relative max-norm <= 1e-5."""
    from oracle.llg import llg_rhs
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.workloads import from_soa
    w = W.bulk()
    s = setup_workload(w, "fp32")
    m0_gpu = from_soa(to_host(s.get_m()))
    s.profile_enable(True)
    k = from_soa(to_host(s.llg_rhs(t=0.0)))
    prof = s.profile_read()
    s.profile_enable(False)
    s.close()
    assert "k5_fused" in prof and "stage_llg" not in prof, prof
    prob = oracle_problem(w)
    ref = llg_rhs(m0_gpu, prob.heff(m0_gpu, 0.0), w.alpha)
    err = float(np.max(np.abs(k - ref)) / np.max(np.abs(ref)))
    assert err < FP32_TOL, err


def test_thin_film_dp45_fp32_replayed_by_oracle():
    """FP32 Dormand-Prince steps on the thin-film workload; the oracle replays
    the step sizes the GPU accepted (the error norm itself is FP64 on both
    sides but its inputs differ by FP32 rounding, so the accept decisions are
    compared only where err is not within 1e-3 of the threshold)."""
    from oracle.llg import dp45_attempt, normalize
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.workloads import from_soa
    w = W.thin_film(n=(128, 32, 1))
    s = setup_workload(w, "fp32")
    prob = oracle_problem(w)
    m = w.m0.copy()
    t, dt = 0.0, 1e-13
    k1 = prob.rhs(m, t)
    for _ in range(10):
        t_new, dt = s.step(dt, t, "dp45", w.extra["rtol"])
        used = t_new - t
        y5, k7, _, err = dp45_attempt(prob, m, t, used, k1, w.extra["rtol"])
        assert err <= 1.0 + 1e-3
        m = normalize(y5)
        k1 = k7
        t = t_new
    mg = from_soa(to_host(s.get_m()))
    inc = np.max(np.abs(m - w.m0))
    assert np.max(np.abs(mg - m)) < 1e-4 * inc + 1e-6
    s.close()


def test_mixed_radix_full_size_stage_derivative_fp32():
    """The mixed-radix grid the bench times (the bulk construction on
    192x192x48, padded 384x384x96): the stage derivative read back through
    mm_llg_rhs runs the fused kernel on the 384-point 6 8 8 x lines (checked
    from the launch record), the classic 384-point y passes and the two-factor
    96-point z pass; against the oracle's FP64 llg_rhs of its own field,
    element by element, and the field of mm_heff likewise: relative max-norm
    <= 1e-5 for both."""
    from oracle.llg import llg_rhs
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import padded_extents, setup_workload
    from paper_2302_08843_gb300.workloads import from_soa
    w = W.bulk(n=(192, 192, 48))
    assert padded_extents(w.n) == (384, 384, 96)
    s = setup_workload(w, "fp32")
    m0_gpu = from_soa(to_host(s.get_m()))
    s.profile_enable(True)
    k = from_soa(to_host(s.llg_rhs(t=0.0)))
    prof = s.profile_read()
    s.profile_enable(False)
    h = from_soa(to_host(s.heff(t=0.0)))
    s.close()
    assert "k5_fused" in prof and "stage_llg" not in prof, prof
    href = oracle_problem(w).heff(m0_gpu, 0.0)
    ref = llg_rhs(m0_gpu, href, w.alpha)
    err_h = float(np.max(np.abs(h - href)) / np.max(np.abs(href)))
    err_k = float(np.max(np.abs(k - ref)) / np.max(np.abs(ref)))
    assert err_h < FP32_TOL, err_h
    assert err_k < FP32_TOL, err_k
