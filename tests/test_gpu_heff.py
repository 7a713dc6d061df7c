"""GPU parity of the full effective field (Sec. 4: demag + exchange +
uniaxial anisotropy + Zeeman) and the four energies, on the workloads'
material structure: constant material, Voronoi grains with per-grain easy
axes, per-cell Ms with a masked time-dependent Zeeman field."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, oracle_problem, rel, to_host

pytestmark = pytest.mark.gpu


def _workloads():
    from paper_2302_08843_gb300 import workloads as W
    return {
        "plain": W.plain_fp64(),
        "bulk_crop": W.bulk(crop=((0, 64), (0, 64), (0, 16))),
        "bulk_small_crop": W.bulk(crop=((10, 31), (5, 18), (3, 10))),
        "inverse": W.inverse_design(n=(48, 40, 1), strip=5, out_box=((30, 35), (20, 25))),
        "film": W.thin_film(n=(64, 32, 1)),
    }


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["plain", "bulk_crop", "bulk_small_crop", "inverse", "film"])
def test_heff_and_energies_match_oracle(name, precision):
    from oracle.demag import magnetization, rounding_sensitivity
    from paper_2302_08843_gb300.binding import setup_workload
    from paper_2302_08843_gb300.workloads import from_soa
    w = _workloads()[name]
    t = 3.1e-11
    s = setup_workload(w, precision)
    h, E, tq = s.heff(t=t, energies=True, torque=True)
    h = from_soa(to_host(h))
    prob = oracle_problem(w)
    ref = prob.heff(w.m0, t)
    Eref = prob.energies(w.m0, t)
    tq_ref = prob.max_torque(w.m0, ref)
    if precision == "fp64":
        tol = max(1e-10, rounding_sensitivity(w.n, w.dx, 20, magnetization(w.m0, w.Ms)))
    else:
        tol = FP32_TOL
    assert rel(h, ref) < tol
    Escale = max(abs(e) for e in Eref)
    for a, b in zip(E, Eref):
        assert abs(a - b) < tol * Escale, (E, Eref)
    assert abs(tq - tq_ref) < tol * tq_ref * 10
    s.close()
