"""Pins for the oracle's demag field (Sec. 4.4): the FFT convolution equals
the plain direct sum, the single-cell and uniform-box closed forms, the thin
film limit, and self-adjointness of the convolution."""
import numpy as np
import pytest

from oracle.demag import (demag_direct, demag_direct_c, demag_fft,
                          magnetization)
from oracle.newell import COMP_NAMES, demag_tensor, newell_component


def _rel(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def _rand_m(n, seed):
    rng = np.random.default_rng(seed)
    m = rng.normal(size=tuple(n) + (3,))
    return m / np.linalg.norm(m, axis=-1, keepdims=True)


@pytest.mark.parametrize("n", [(7, 5, 3), (1, 1, 1), (4, 1, 1), (1, 6, 1), (3, 4, 1), (2, 2, 5)])
def test_fft_equals_direct_sum_small(n):
    d = (2.5e-9, 3e-9, 2e-9)
    Nt = demag_tensor(n, d, p=20)
    rng = np.random.default_rng(1)
    Ms = rng.uniform(0.5e6, 1.5e6, size=n)
    M = magnetization(_rand_m(n, 2), Ms)
    hd = demag_direct(Nt, M)
    hf = demag_fft(Nt, M)
    assert _rel(hf, hd) < 1e-13


def test_c_direct_sum_equals_numpy_direct_sum():
    n = (6, 5, 3)
    Nt = demag_tensor(n, (1.0, 1.0, 1.0), p=2)
    M = _rand_m(n, 3)
    assert _rel(demag_direct_c(Nt, M), demag_direct(Nt, M)) < 1e-14


@pytest.mark.slow
@pytest.mark.parametrize("n,p", [((32, 32, 4), 20), ((48, 6, 2), 20)])
def test_fft_equals_direct_sum_config_sizes(n, p):
    d = (2.5e-9, 2.5e-9, 3e-9)
    Nt = demag_tensor(n, d, p=p)
    M = magnetization(_rand_m(n, 4), 8e5)
    assert _rel(demag_fft(Nt, M), demag_direct_c(Nt, M)) < 1e-13


def test_single_cube_cell():
    Nt = demag_tensor((1, 1, 1), (2e-9, 2e-9, 2e-9))
    M = np.array([[[[3.0, -1.0, 2.0]]]]) * 1e5
    h = demag_fft(Nt, M)
    assert np.allclose(h, -M / 3.0, rtol=1e-14, atol=0)


def test_uniform_box_average_equals_box_self_term():
    """Exactness of the cell average: the mean field of a uniformly magnetised
    box of cells is -N_box M with N_box the self term of one big cell."""
    n = (6, 4, 3)
    d = (1e-9, 1.5e-9, 2e-9)
    Nt = demag_tensor(n, d, p=None)
    for direction in np.eye(3):
        M = np.broadcast_to(direction * 7e5, n + (3,)).copy()
        hbar = demag_fft(Nt, M).reshape(-1, 3).mean(axis=0)
        D = (n[0] * d[0], n[1] * d[1], n[2] * d[2])
        T = np.zeros((3, 3))
        for c, name in enumerate(COMP_NAMES):
            p, q = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)][c]
            T[p, q] = T[q, p] = float(newell_component(name, 0.0, 0.0, 0.0, *D))
        assert np.allclose(hbar, -T @ (direction * 7e5), rtol=1e-12, atol=1e-9)


def test_thin_film_limit():
    """m = z on a wide film: h_z / Ms -> -1 at the centre as the film widens."""
    errs = []
    for L in (64, 128, 256):
        n = (L, L, 1)
        Nt = demag_tensor(n, (2e-9, 2e-9, 2e-9), p=20)
        M = np.zeros(n + (3,))
        M[..., 2] = 1.0
        h = demag_fft(Nt, M)
        errs.append(abs(h[L // 2, L // 2, 0, 2] + 1.0))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.02
    # error ~ thickness / width: halves when the width doubles
    assert 1.6 < errs[0] / errs[1] < 2.4 and 1.6 < errs[1] / errs[2] < 2.4


def test_convolution_is_self_adjoint():
    n = (9, 6, 4)
    Nt = demag_tensor(n, (1.0, 1.0, 2.0), p=3)
    rng = np.random.default_rng(5)
    u = rng.normal(size=n + (3,))
    v = rng.normal(size=n + (3,))
    Nv = demag_fft(Nt, v)
    a = np.sum(u * Nv)
    b = np.sum(demag_fft(Nt, u) * v)
    # rounding scale: the sum of the magnitudes of the terms of the inner product
    assert abs(a - b) < 1e-13 * np.sum(np.abs(u * Nv))


def test_inverse_design_gradient_sign_follows_analytic_boundary():
    """Sec. 5.2: for J = h_y at the cell (nx//2, 0, nz//2) of a 101x51x1 film of
    5 nm cells with Ms = 1, dJ/dm_y is positive where |x - x0| < sqrt(2) (y - y0)
    (the analytic line quoted with Fig. inverse_demo).  The gradient is the
    adjoint (transposed) convolution applied to a point source at the target."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    n = tuple(gold["inverse_design_grid"]["value"])
    d = tuple(gold["inverse_design_cell_m"]["value"])
    Ms = gold["inverse_design_Ms"]["value"]
    slope = gold["inverse_design_boundary_slope"]["value"]
    i0 = (n[0] // 2, 0, n[2] // 2)
    Nt = demag_tensor(n, d, p=20)
    src = np.zeros(n + (3,))
    src[i0 + (1,)] = 1.0
    grad = Ms * demag_fft(Nt, src)          # dJ/dm_j = -Ms N(j - i0) e_y
    # direct derivative of the definition at a few cells
    from oracle.newell import tensor_at
    for j in [(50, 10, 0), (10, 40, 0), (80, 3, 0)]:
        T = tensor_at(Nt, n, i0[0] - j[0], i0[1] - j[1], i0[2] - j[2])
        assert np.allclose(grad[j], -Ms * T[1], rtol=1e-12, atol=1e-15)
    X = np.arange(n[0])[:, None] - i0[0]
    Y = np.arange(n[1])[None, :] - i0[1]
    margin = np.abs(np.abs(X) - slope * Y) > 2.0          # away from the boundary line
    far = (X ** 2 + Y ** 2) > 16
    sel = margin & far
    expect_pos = np.abs(X) < slope * Y
    assert np.array_equal((grad[:, :, 0, 1] > 0)[sel], expect_pos[sel])
    assert sel.sum() > 0.8 * n[0] * n[1]
