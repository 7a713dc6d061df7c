"""GPU parity of the demag field (Sec. 4.4): the five FFT passes of libmm.so
against the oracle's convolution, element by element, FP64 and FP32, on grids
that cover one cell, 1-D and 2-D lines, ragged extents that pad beyond 2n,
every 5-smooth padded length of the mixed-radix passes (100, 200, 400, 800,
on each axis), several CTA tiles with ragged tails, and the largest padded
extent (4096)."""
import numpy as np
import pytest

from gpu_util import FP32_TOL, rel, to_host

pytestmark = pytest.mark.gpu

GRIDS = [
    ((1, 1, 1), (2e-9, 2e-9, 2e-9)),
    ((7, 5, 3), (2.5e-9, 3e-9, 2e-9)),
    ((4, 1, 1), (1e-9, 1e-9, 1e-9)),
    ((1, 6, 1), (1e-9, 2e-9, 1e-9)),
    ((1, 1, 5), (1e-9, 1e-9, 3e-9)),
    ((3, 4, 1), (2e-9, 2e-9, 1e-9)),
    ((2, 3, 2), (1e-9, 1e-9, 1e-9)),
    ((32, 32, 4), (2.5e-9, 2.5e-9, 3e-9)),
    ((16, 8, 8), (2e-9, 2e-9, 2e-9)),
    ((100, 3, 2), (3e-9, 3e-9, 3e-9)),
    ((33, 17, 9), (2e-9, 2.5e-9, 3e-9)),
    ((5, 70, 3), (2e-9, 2e-9, 2e-9)),
    ((6, 5, 40), (2e-9, 2e-9, 2e-9)),
    ((2048, 2, 1), (1e-9, 1e-9, 1e-9)),
    ((200, 6, 2), (2e-9, 2e-9, 2e-9)),          # x padded to 400
    ((300, 4, 1), (2e-9, 2e-9, 2e-9)),          # x padded to 800
    ((12, 150, 3), (2e-9, 2e-9, 3e-9)),         # y padded to 400
    ((10, 8, 48), (2e-9, 2e-9, 2e-9)),          # z padded to 100
    ((512, 3, 1), (2e-9, 2e-9, 2e-9)),          # x padded to 1024
    ((1024, 2, 1), (2e-9, 2e-9, 2e-9)),         # x padded to 2048
]


def test_padded_extents_rule():
    from paper_2302_08843_gb300.binding import padded_extents
    assert padded_extents((1, 2, 3)) == (1, 4, 8)
    assert padded_extents((50, 64, 100)) == (100, 128, 200)
    assert padded_extents((150, 200, 300)) == (400, 400, 800)
    assert padded_extents((401, 2048, 33)) == (1024, 4096, 100)


def _m(n, seed):
    rng = np.random.default_rng(seed)
    m = rng.normal(size=tuple(n) + (3,))
    return m / np.linalg.norm(m, axis=-1, keepdims=True)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,d", GRIDS)
def test_demag_matches_oracle(n, d, precision):
    from oracle.demag import demag_fft, magnetization, rounding_sensitivity
    from oracle.newell import demag_tensor
    from paper_2302_08843_gb300.binding import State
    from paper_2302_08843_gb300.workloads import from_soa, to_soa
    rng = np.random.default_rng(11)
    Ms = rng.uniform(4e5, 1.2e6, size=n)
    m = _m(n, 3)
    s = State(n, d, precision)
    s.set_material(Ms=0.0, A=0.0, alpha=0.1, Ms_cell=to_soa(Ms))
    s.demag_setup(20)
    h = from_soa(to_host(s.heff(m=to_soa(m))))
    M = magnetization(m, Ms)
    ref = demag_fft(demag_tensor(n, d, 20), M)
    err = rel(h, ref)
    if precision == "fp64":
        tol = max(1e-10, 2.0 * rounding_sensitivity(n, d, 20, M))
    else:
        tol = FP32_TOL
    assert err < tol, (err, tol)
    s.close()


def test_uniform_cube_cell_and_zero_ms():
    """One cube cell: h = -M/3 (the Newell self term); a cell with Ms = 0
    carries no field."""
    import torch
    from paper_2302_08843_gb300.binding import State
    s = State((1, 1, 1), (2e-9, 2e-9, 2e-9), "fp64")
    s.set_material(Ms=8e5, A=1e-11, alpha=0.1)
    s.demag_setup(20)
    m = torch.tensor([0.6, 0.0, 0.8], dtype=torch.float64, device="cuda").reshape(3, 1, 1, 1)
    h = to_host(s.heff(m=m)).reshape(3)
    assert np.allclose(h, -8e5 / 3.0 * np.array([0.6, 0.0, 0.8]), rtol=1e-14, atol=1e-9)
    s.set_material(Ms=0.0, A=1e-11, alpha=0.1)
    h0 = to_host(s.heff(m=m))
    assert np.all(h0 == 0.0)
    s.close()
