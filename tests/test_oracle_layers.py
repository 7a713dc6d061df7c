"""Pins of the non-equidistant-layer oracle (Sec. 4.4) against the
equidistant tensor, exact identities of the cell-average integral and the
exchange energy."""
import numpy as np
import pytest

from oracle import layers as L
from oracle import newell as Nw
from oracle.constants import MU0
from oracle.demag import demag_fft, magnetization, tensor_spectrum
from oracle.fields import exchange_field, linear_energy
from oracle.llg import Problem

DX, DY, H = 2e-9, 3e-9, 1.5e-9


def _std(n, h=H):
    return Nw.demag_tensor(n, (DX, DY, h), p=None)


def test_equal_thickness_is_the_equidistant_tensor():
    n = (3, 2, 3)
    T = L.layered_tensor(n, DX, DY, [H] * 3, p=None)
    S = _std(n)
    for i in range(3):
        for j in range(3):
            np.testing.assert_allclose(T[:, i, j], S[:, :, :, i - j + 2], rtol=0, atol=1e-14)


def test_equal_thickness_dipole_switch_matches_equidistant_rule():
    n = (6, 2, 4)
    T = L.layered_tensor(n, DX, DY, [H] * 4, p=2)
    S = Nw.demag_tensor(n, (DX, DY, H), p=2)
    for i in range(4):
        for j in range(4):
            np.testing.assert_allclose(T[:, i, j], S[:, :, :, i - j + 3], rtol=0, atol=1e-14)


def test_source_layer_split_is_additive():
    # layers [h, 2h] cover cells {0} and {1, 2} of an equidistant 3-cell column:
    # the source integral is additive, the target average divides by its own volume
    n3 = (3, 2, 3)
    S = _std(n3)
    T = L.layered_tensor((3, 2, 2), DX, DY, [H, 2 * H], p=None)

    def s(k):   # standard entry, target-minus-source layer offset k
        return S[:, :, :, k + 2]

    np.testing.assert_allclose(T[:, 0, 1], s(-1) + s(-2), rtol=0, atol=1e-14)
    np.testing.assert_allclose(2 * T[:, 1, 0], s(1) + s(2), rtol=0, atol=1e-14)
    np.testing.assert_allclose(2 * T[:, 1, 1], 2 * s(0) + s(1) + s(-1), rtol=0, atol=1e-14)
    np.testing.assert_allclose(T[:, 0, 0], s(0), rtol=0, atol=1e-14)


def test_three_to_one_thickness_ratio_split():
    # thickness ratio 3: layer of 3h against single h cells of the same column
    S = Nw.demag_tensor((2, 2, 4), (DX, DY, H), p=None)
    T = L.layered_tensor((2, 2, 2), DX, DY, [3 * H, H], p=None)
    s = lambda k: S[:, :, :, k + 3]
    np.testing.assert_allclose(T[:, 1, 0], s(3) + s(2) + s(1), rtol=0, atol=1e-14)
    np.testing.assert_allclose(3 * T[:, 0, 1], s(-1) + s(-2) + s(-3), rtol=0, atol=1e-14)


@pytest.mark.parametrize("p", [None, 1])
def test_reciprocity(p):
    h = np.array([1.0e-9, 2.7e-9, 0.6e-9])
    n = (4, 3, 3)
    T = L.layered_tensor(n, DX, DY, h, p=p)
    for i in range(3):
        for j in range(3):
            a = h[i] * T[:, i, j]
            b = h[j] * T[:, j, i][:, ::-1, ::-1]        # offset -r
            # entries are differences of large terms: compare on the scale of the largest entry
            np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * h.max() * np.abs(T).max())


def test_trace_is_the_overlap_fraction():
    # trace of the cell-average tensor = overlap volume / target volume: 1 for
    # the self entry, 0 for every other pair of (touching or distant) cells
    h = np.array([1.0e-9, 2.7e-9, 0.6e-9])
    T = L.layered_tensor((3, 3, 3), DX, DY, h, p=None)
    tr = T[0] + T[3] + T[5]
    expect = np.zeros(tr.shape)
    for i in range(3):
        expect[i, i, 2, 2] = 1.0
    np.testing.assert_allclose(tr, expect, rtol=0, atol=1e-12)


def test_whole_stack_average_is_the_box_factor():
    # uniform M: the volume-weighted sum of all entries is the self factor of
    # the whole box (nx dx, ny dy, sum h), an independent Newell evaluation
    h = np.array([0.8e-9, 2.1e-9, 1.3e-9])
    n = (3, 2, 3)
    T = L.layered_tensor(n, DX, DY, h, p=None)
    tot = np.zeros(6)
    for i in range(3):
        for j in range(3):
            # target cells x source cells at each offset: (nx - |X|)(ny - |Y|) pairs
            I = np.arange(-n[0] + 1, n[0])[:, None]
            J = np.arange(-n[1] + 1, n[1])[None, :]
            mult = (n[0] - np.abs(I)) * (n[1] - np.abs(J))
            tot += h[i] * DX * DY * np.sum(T[:, i, j] * mult, axis=(1, 2))
    Vt = n[0] * DX * n[1] * DY * h.sum()
    box = [Nw.newell_component(c, 0.0, 0.0, 0.0, n[0] * DX, n[1] * DY, h.sum()) for c in Nw.COMP_NAMES]
    np.testing.assert_allclose(tot / Vt, box, rtol=1e-10, atol=1e-13)


def test_far_entries_approach_the_dipole():
    h = np.array([0.7e-9, 2.0e-9])
    z0 = L.layer_bottoms(h)
    X, Y = 30 * DX, 7 * DY
    for name in Nw.COMP_NAMES:
        for i, j in ((0, 1), (1, 0), (1, 1)):
            nw = L.layer_component(name, X, Y, z0[i] - z0[j], DX, DY, h[i], h[j])
            dp = L.layer_dipole(name, X, Y, z0[i] - z0[j], DX, DY, h[i], h[j])
            scale = DX * DY * h[j] / (4 * np.pi * (X * X + Y * Y) ** 1.5)
            assert abs(nw - dp) < 2e-3 * scale, (name, i, j, nw, dp)


def test_layered_fft_equals_direct_sum():
    rng = np.random.default_rng(5)
    n = (5, 3, 3)
    h = np.array([1.1e-9, 0.5e-9, 2.2e-9])
    T = L.layered_tensor(n, DX, DY, h, p=2)
    M = rng.standard_normal(n + (3,)) * 4e5
    np.testing.assert_allclose(L.layered_demag_fft(T, M), L.layered_demag_direct(T, M), rtol=1e-10, atol=1e-6)


def test_equal_layers_demag_is_the_equidistant_demag():
    rng = np.random.default_rng(6)
    n = (4, 3, 3)
    M = rng.standard_normal(n + (3,)) * 4e5
    T = L.layered_tensor(n, DX, DY, [H] * 3, p=None)
    Nt = _std(n)
    np.testing.assert_allclose(L.layered_demag_fft(T, M), demag_fft(Nt, M, tensor_spectrum(Nt, n)),
                               rtol=1e-10, atol=1e-6)


def test_thickness_harmonic_cases():
    assert L.thickness_harmonic(3.0, 3.0, 1.0, 5.0) == pytest.approx(3.0)
    assert L.thickness_harmonic(2.0, 6.0, 1.0, 1.0) == pytest.approx(3.0)      # 2 a b / (a + b)
    assert L.thickness_harmonic(0.0, 6.0, 1.0, 2.0) == 0.0
    assert L.thickness_harmonic(0.0, 0.0, 1.0, 2.0) == 0.0
    # series resistances: d / A_link = (hi/2) / Ai + (hj/2) / Aj
    hi, hj, Ai, Aj = 1.0, 3.0, 2.0, 5.0
    assert L.thickness_harmonic(Ai, Aj, hi, hj) == pytest.approx((hi + hj) / 2 / (hi / 2 / Ai + hj / 2 / Aj))


def test_layer_exchange_equal_thickness_reduces():
    rng = np.random.default_rng(7)
    n = (4, 3, 5)
    m = rng.standard_normal(n + (3,))
    m /= np.linalg.norm(m, axis=-1, keepdims=True)
    A = rng.uniform(0.5e-11, 2e-11, n)
    Ms = rng.uniform(4e5, 9e5, n)
    a = L.exchange_field_layers(m, Ms, A, DX, DY, [H] * 5)
    b = exchange_field(m, Ms, A, (DX, DY, H))
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-3)


def test_layer_exchange_is_the_energy_gradient():
    rng = np.random.default_rng(8)
    n = (3, 2, 4)
    h = np.array([0.9e-9, 2.4e-9, 1.2e-9, 0.5e-9])
    m = rng.standard_normal(n + (3,))
    m /= np.linalg.norm(m, axis=-1, keepdims=True)
    A = rng.uniform(0.5e-11, 2e-11, n)
    Ms = rng.uniform(4e5, 9e5, n)
    hex_ = L.exchange_field_layers(m, Ms, A, DX, DY, h)
    V = DX * DY * h
    # -1/2 mu0 sum V Ms m.h equals the link energy for unit m
    E = L.exchange_energy_links(m, A, DX, DY, h)
    assert linear_energy(m, hex_, Ms, V[None, None, :]) == pytest.approx(E, rel=1e-12)
    # h = -1/(mu0 Ms V) dE/dm by central differences on unnormalised m
    eps = 1e-6
    for (x, y, z, c) in ((0, 0, 0, 0), (1, 1, 1, 2), (2, 0, 2, 1), (1, 0, 3, 0)):
        mp, mm_ = m.copy(), m.copy()
        mp[x, y, z, c] += eps
        mm_[x, y, z, c] -= eps
        g = (L.exchange_energy_links(mp, A, DX, DY, h) - L.exchange_energy_links(mm_, A, DX, DY, h)) / (2 * eps)
        assert hex_[x, y, z, c] == pytest.approx(-g / (MU0 * Ms[x, y, z] * V[z]), rel=1e-6)


def test_problem_with_equal_layers_is_the_equidistant_problem():
    rng = np.random.default_rng(9)
    n = (4, 3, 3)
    m = rng.standard_normal(n + (3,))
    m /= np.linalg.norm(m, axis=-1, keepdims=True)
    kw = dict(Ms=8e5, A=1.3e-11, alpha=0.1, Ku1=2e4, ku_axis=(0, 0, 1), h_ext=(1e4, 0, 2e3), p=None)
    a = Problem(n, (DX, DY, H), layers=[H] * 3, **kw)
    b = Problem(n, (DX, DY, H), **kw)
    np.testing.assert_allclose(a.heff(m, 0.0), b.heff(m, 0.0), rtol=1e-10, atol=1e-4)
    np.testing.assert_allclose(a.energies(m, 0.0), b.energies(m, 0.0), rtol=1e-10, atol=1e-30)


def test_problem_layers_refuses_dmi_and_bad_thickness():
    with pytest.raises(ValueError):
        Problem((2, 2, 2), (DX, DY, H), 8e5, 1e-11, 0.1, layers=[H, H], D=1e-3)
    with pytest.raises(ValueError):
        Problem((2, 2, 2), (DX, DY, H), 8e5, 1e-11, 0.1, layers=[H])
    with pytest.raises(ValueError):
        Problem((2, 2, 2), (DX, DY, H), 8e5, 1e-11, 0.1, layers=[H, 0.0])


def test_uniform_stack_energy_matches_box_factor():
    # uniformly magnetised stack: E_demag = 1/2 mu0 Ms^2 V_total N_box (m along each axis)
    h = np.array([0.8e-9, 2.1e-9, 1.3e-9])
    n = (3, 2, 3)
    Ms = 7e5
    pb = Problem(n, (DX, DY, 1e-9), Ms, 1e-11, 0.1, layers=h, p=None)
    Vt = n[0] * DX * n[1] * DY * h.sum()
    for ax, comp in ((0, "xx"), (1, "yy"), (2, "zz")):
        m = np.zeros(n + (3,))
        m[..., ax] = 1.0
        Ed = pb.energies(m, 0.0)[0]
        Nb = float(Nw.newell_component(comp, 0.0, 0.0, 0.0, n[0] * DX, n[1] * DY, h.sum()))
        assert Ed == pytest.approx(0.5 * MU0 * Ms * Ms * Vt * Nb, rel=1e-10)
