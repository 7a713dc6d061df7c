"""GPU parity of the demag field (Sec. 4.4): the five FFT passes of libmm.so
against the oracle's convolution, element by element, FP64 and FP32, on grids
that cover one cell, 1-D and 2-D lines, ragged extents, every compiled
mixed-radix padded length r 2^a (r = 3: 96 ... 768, r = 7: 112 ... 896,
r = 25: 100 ... 800) on at least one axis, runtime-plan 7-smooth lengths with
every radix (2, 3, 4, 5, 7) on every axis up to 3000, several CTA tiles with
ragged tails, and the largest padded extent (4096)."""
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
    ((380, 4, 1), (2e-9, 2e-9, 2e-9)),          # x padded to 768
    ((300, 4, 1), (2e-9, 2e-9, 2e-9)),          # x padded to 600 (runtime plan)
    ((12, 150, 3), (2e-9, 2e-9, 3e-9)),         # y padded to 300 (runtime plan)
    ((12, 190, 3), (2e-9, 2e-9, 3e-9)),         # y padded to 384
    ((10, 8, 48), (2e-9, 2e-9, 2e-9)),          # z padded to 96
    # the 96-point z line on the two-factor engine (8 x 12): odd and even nz,
    # several kx tiles with a ragged last tile
    ((40, 8, 47), (2e-9, 2.5e-9, 2e-9)),        # z 96, 3 tiles of 16 kx
    ((64, 12, 46), (2e-9, 2e-9, 3e-9)),         # z 96, 5 tiles (last one column)
    ((512, 3, 1), (2e-9, 2e-9, 2e-9)),          # x padded to 1024
    ((1024, 2, 1), (2e-9, 2e-9, 2e-9)),         # x padded to 2048
    # every mixed-radix length r 2^a (r = 3, 7, 25) on at least one axis
    ((50, 5, 3), (2e-9, 2e-9, 2e-9)),           # x 100
    ((3, 100, 2), (2e-9, 2e-9, 2e-9)),          # y 200
    ((5, 4, 50), (2e-9, 2e-9, 2e-9)),           # z 100
    ((400, 3, 1), (2e-9, 2e-9, 2e-9)),          # x 800
    ((56, 6, 3), (2e-9, 2.5e-9, 3e-9)),         # x 112
    ((4, 112, 2), (2e-9, 2e-9, 2e-9)),          # y 224
    ((4, 3, 56), (2e-9, 2e-9, 1e-9)),           # z 112
    ((224, 3, 2), (2e-9, 2e-9, 2e-9)),          # x 448
    ((448, 2, 1), (2e-9, 2e-9, 2e-9)),          # x 896
    ((3, 96, 2), (2e-9, 2e-9, 2e-9)),           # y 192
    ((6, 5, 96), (2e-9, 2e-9, 2e-9)),           # z 192
    ((3, 3, 112), (2e-9, 2e-9, 2e-9)),          # z 224
    ((2, 2, 192), (2e-9, 2e-9, 2e-9)),          # z 384
    ((2, 2, 224), (2e-9, 2e-9, 2e-9)),          # z 448
    ((2, 1, 384), (2e-9, 2e-9, 2e-9)),          # z 768
    ((2, 1, 400), (2e-9, 2e-9, 2e-9)),          # z 800
    ((2, 1, 448), (2e-9, 2e-9, 2e-9)),          # z 896
    # FP32 TMA z pass on 3 x 2^a lines (also as the 2-D path along y), and
    # TMA y tiles split into several boxes of uneven rows
    ((5, 40, 1), (2e-9, 2e-9, 2e-9)),           # y 80, 2-D (runtime plan)
    ((5, 48, 1), (2e-9, 2e-9, 2e-9)),           # y 96, 2-D
    ((4, 90, 1), (2e-9, 2e-9, 2e-9)),           # y 180, 2-D (runtime plan)
    ((4, 96, 1), (2e-9, 2e-9, 2e-9)),           # y 192, 2-D
    ((3, 300, 2), (2e-9, 2e-9, 2e-9)),          # y 600 (runtime plan)
    ((2, 450, 2), (2e-9, 2e-9, 2e-9)),          # y 900 (runtime plan)
    ((2, 510, 2), (2e-9, 2e-9, 2e-9)),          # y 1024: forward 2 boxes of 256 rows
    # 2-D grids whose padded y extent is above 256
    ((6, 250, 1), (2e-9, 2e-9, 2e-9)),          # y 500, 2-D
    ((6, 256, 1), (2e-9, 2e-9, 2e-9)),          # y 512, 2-D
    ((5, 180, 1), (2e-9, 2e-9, 2e-9)),          # y 360, 2-D
    ((3, 700, 1), (2e-9, 2e-9, 2e-9)),          # y 1400, 2-D
    # runtime-plan lengths (every 7-smooth length without a compiled engine), each radix
    ((35, 3, 2), (2e-9, 2e-9, 2e-9)),           # x 70 = 2 5 7
    ((3, 45, 2), (2e-9, 2e-9, 2e-9)),           # y 90 = 2 3^2 5
    ((4, 3, 27), (2e-9, 2e-9, 2e-9)),           # z 54 = 2 3^3
    ((5, 63, 1), (2e-9, 2e-9, 2e-9)),           # y 126 = 2 3^2 7, 2-D
    ((1500, 2, 1), (2e-9, 2e-9, 2e-9)),         # x 3000 = 2^3 3 5^3
    ((2, 2, 1400), (2e-9, 2e-9, 2e-9)),         # z 2800 = 2^4 5^2 7
    ((3, 1500, 1), (2e-9, 2e-9, 2e-9)),         # y 3000, 2-D through the y passes
]


def test_padded_extents_rule():
    """The smallest even 7-smooth length >= 2n (up to 3200; beyond that the next
    power of two), 1 for a single cell."""
    from paper_2302_08843_gb300.binding import padded_extents
    assert padded_extents((1, 2, 3)) == (1, 4, 6)
    assert padded_extents((50, 64, 100)) == (100, 128, 200)
    assert padded_extents((150, 200, 300)) == (300, 400, 600)
    assert padded_extents((401, 2048, 33)) == (810, 4096, 70)
    assert padded_extents((48, 56, 96)) == (96, 112, 192)
    assert padded_extents((49, 57, 97)) == (98, 120, 196)
    assert padded_extents((35, 45, 27)) == (70, 90, 54)
    assert padded_extents((65, 70, 5)) == (140, 140, 10)
    assert padded_extents((7, 1500, 1400)) == (14, 3000, 2800)
    assert padded_extents((1601, 1700, 2048)) == (4096, 4096, 4096)
    for n in range(2, 1601):
        L = padded_extents((n, 1, 1))[0]
        v = L
        for q in (2, 3, 5, 7):
            while v % q == 0:
                v //= q
        assert v == 1 and L % 2 == 0 and L >= 2 * n
        assert not any(_smooth(w) for w in range(2 * n, L, 2))


def _smooth(v):
    for q in (2, 3, 5, 7):
        while v % q == 0:
            v //= q
    return v == 1


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
        tol = max(1e-10, rounding_sensitivity(n, d, 20, M))
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
