"""Pins for the oracle's exchange (Sec. 4.2), anisotropy (Sec. 4.1), Zeeman
and energies (Eq. linear_energy_discrete)."""
import numpy as np
import pytest

from oracle.constants import MU0
from oracle.fields import (anisotropy_field, dmi_average, dmi_field, exchange_field, linear_energy,
                           zeeman_energy, zeeman_field)


def test_uniform_magnetisation_has_no_exchange_field():
    n = (7, 4, 3)
    rng = np.random.default_rng(0)
    A = rng.uniform(0.5e-11, 2e-11, size=n)
    Ms = rng.uniform(5e5, 1e6, size=n)
    m = np.broadcast_to(np.array([0.6, 0.0, 0.8]), n + (3,)).copy()
    h = exchange_field(m, Ms, A, (2e-9, 3e-9, 1e-9))
    assert np.all(h == 0.0)


def test_spin_spiral_closed_form():
    """m = (cos kx, sin kx, 0): every interior cell has
    h = 2A/(mu0 Ms) * 2 (cos k dx - 1)/dx^2 * m."""
    nx, dx, k = 40, 2e-9, 0.31 / 2e-9
    n = (nx, 3, 2)
    x = (np.arange(nx) * dx)[:, None, None] * np.ones(n)
    m = np.stack([np.cos(k * x), np.sin(k * x), np.zeros(n)], axis=-1)
    A, Ms = 1.3e-11, 8e5
    h = exchange_field(m, Ms, A, (dx, 1e-9, 1e-9))
    expect = (2 * A / (MU0 * Ms)) * 2 * (np.cos(k * dx) - 1) / dx ** 2 * m
    inner = slice(1, nx - 1)
    scale = np.max(np.abs(expect))
    assert np.max(np.abs(h[inner] - expect[inner])) < 1e-12 * scale
    # Neumann boundary: the first cell only sees its +x neighbour
    h0 = (2 * A / (MU0 * Ms)) * (m[1] - m[0]) / dx ** 2
    assert np.max(np.abs(h[0] - h0)) < 1e-12 * scale


def test_homogeneous_A_reduces_to_laplacian():
    """With constant A the harmonic-mean form equals the paper's simplified
    second-difference form (Sec. 4.2), with the missing neighbour of a
    boundary cell replaced by the cell itself (zero normal derivative)."""
    n = (6, 5, 4)
    d = (1e-9, 2e-9, 1.5e-9)
    rng = np.random.default_rng(1)
    m = rng.normal(size=n + (3,))
    A, Ms = 1.5e-11, 1e6
    h = exchange_field(m, Ms, A, d)
    pad = np.pad(m, ((1, 1), (1, 1), (1, 1), (0, 0)), mode="edge")
    lap = np.zeros_like(m)
    c = (slice(1, -1),) * 3
    for ax in range(3):
        up = list(c)
        dn = list(c)
        up[ax] = slice(2, None)
        dn[ax] = slice(0, -2)
        lap += (pad[tuple(up)] - 2 * m + pad[tuple(dn)]) / d[ax] ** 2
    ref = 2 * A / (MU0 * Ms) * lap
    assert np.max(np.abs(h - ref)) < 1e-12 * np.max(np.abs(ref))


def test_exchange_energy_is_sum_over_links():
    """E = -1/2 mu0 V sum Ms m.h_ex equals V sum_links c_ij |m_i - m_j|^2 with
    c_ij = (2/d^2) A_i A_j / (A_i + A_j), for any m and any A."""
    n = (5, 4, 3)
    d = (1e-9, 2e-9, 3e-9)
    V = d[0] * d[1] * d[2]
    rng = np.random.default_rng(2)
    m = rng.normal(size=n + (3,))
    A = rng.uniform(0.5e-11, 2e-11, size=n)
    Ms = rng.uniform(5e5, 1e6, size=n)
    E = linear_energy(m, exchange_field(m, Ms, A, d), Ms, V)
    ref = 0.0
    for idx in np.ndindex(*n):
        for ax in range(3):
            j = list(idx)
            j[ax] += 1
            if j[ax] >= n[ax]:
                continue
            j = tuple(j)
            c = (2 / d[ax] ** 2) * A[idx] * A[j] / (A[idx] + A[j])
            ref += V * c * np.sum((m[idx] - m[j]) ** 2)
    assert abs(E - ref) < 1e-12 * abs(ref)


def test_zero_Ms_cells_carry_no_local_field():
    n = (4, 3, 2)
    m = np.random.default_rng(3).normal(size=n + (3,))
    Ms = np.full(n, 8e5)
    Ms[1, 1, 0] = 0.0
    h = exchange_field(m, Ms, 1e-11, (1e-9,) * 3)
    ha = anisotropy_field(m, Ms, 5e3, (0.0, 0.0, 1.0))
    assert np.all(h[1, 1, 0] == 0) and np.all(ha[1, 1, 0] == 0)
    assert np.all(np.isfinite(h)) and np.all(np.isfinite(ha))


def test_anisotropy_closed_forms():
    n = (3, 2, 2)
    e = np.array([1.0, 2.0, 2.0]) / 3.0
    Ku, Ms, V = 4e5, 1e6, 8e-27
    m_par = np.broadcast_to(e, n + (3,)).copy()
    h = anisotropy_field(m_par, Ms, Ku, e)
    assert np.allclose(h, 2 * Ku / (MU0 * Ms) * m_par, rtol=1e-14, atol=0)
    perp = np.array([2.0, -1.0, 0.0]) / np.sqrt(5.0)
    m_perp = np.broadcast_to(perp, n + (3,)).copy()
    assert np.max(np.abs(anisotropy_field(m_perp, Ms, Ku, e))) < 1e-20 * Ku / (MU0 * Ms) + 1e-9
    # E_u = -Ku V sum (e.m)^2
    rng = np.random.default_rng(4)
    m = rng.normal(size=n + (3,))
    m /= np.linalg.norm(m, axis=-1, keepdims=True)
    E = linear_energy(m, anisotropy_field(m, Ms, Ku, e), Ms, V)
    assert abs(E + Ku * V * np.sum((m @ e) ** 2)) < 1e-12 * Ku * V * m[..., 0].size


def test_zeeman_field_and_energy():
    n = (2, 2, 1)
    B = 0.010                       # 10 mT
    h = zeeman_field((B / MU0, 0.0, 0.0), n)
    assert abs(h[0, 0, 0, 0] - 7957.747154594767) < 1e-9
    m = np.zeros(n + (3,))
    m[..., 0] = 1.0
    Ms, V = 8e5, 1e-27
    assert abs(zeeman_energy(m, h, Ms, V) + 4 * Ms * V * B) < 1e-12 * 4 * Ms * V * B
    w = np.array([[[1.0], [0.0]], [[0.5], [2.0]]])
    hw = zeeman_field((1.0, 2.0, 3.0), n, w)
    assert np.allclose(hw[1, 0, 0], [0.5, 1.0, 1.5]) and np.all(hw[0, 1, 0] == 0)


# ---------------------------------------------------------------- DMI ----

def test_dmi_average():
    assert dmi_average(3e-3, 3e-3) == pytest.approx(3e-3, rel=1e-15)
    assert dmi_average(2e-3, 1e-3) == pytest.approx(2 * 2e-3 * 1e-3 / 3e-3, rel=1e-15)
    assert dmi_average(-2e-3, -1e-3) == pytest.approx(-2 * 2e-3 * 1e-3 / 3e-3, rel=1e-15)
    assert dmi_average(2e-3, 0.0) == 0.0 and dmi_average(0.0, 0.0) == 0.0
    assert dmi_average(2e-3, -2e-3) == 0.0
    # opposite signs: sign of the sum times sqrt(sqrt(-Di Dj) |Di + Dj| / 2)
    v = dmi_average(4e-3, -1e-3)
    assert v == pytest.approx(np.sqrt(np.sqrt(4e-6) * 3e-3 / 2), rel=1e-14)
    assert dmi_average(-1e-3, 4e-3) == v and dmi_average(-4e-3, 1e-3) == -v


def test_dmi_average_opposite_signs_properties():
    """The opposite-sign branch of Eq. D_avg is garbled in print; its reading
    is pinned by properties any sensible link average has, each of which a
    dropped square root, a lost factor 1/2 or a flipped sign breaks:
    symmetry, oddness, degree-1 homogeneity, continuity with the equal-sign
    branch where one strength vanishes, sign of D_i + D_j, a magnitude between
    the geometric sqrt(|D_i D_j|) and arithmetic |D_i + D_j| / 2 means (hence
    at most max(|D_i|, |D_j|)), and zero for equal and opposite strengths."""
    rng = np.random.default_rng(7)
    Di = rng.uniform(1e-4, 5e-3, 400)
    Dj = -rng.uniform(1e-4, 5e-3, 400)
    v = dmi_average(Di, Dj)
    assert np.array_equal(v, dmi_average(Dj, Di))                          # symmetric
    assert np.array_equal(dmi_average(-Di, -Dj), -v)                       # odd
    for lam in (0.5, 4.0):                                                 # homogeneous of degree 1
        assert np.array_equal(dmi_average(lam * Di, lam * Dj), lam * v)     # (exact for powers of two)
    for lam in (3.0, 1e3):
        assert np.allclose(dmi_average(lam * Di, lam * Dj), lam * v, rtol=1e-9, atol=0)
    assert np.array_equal(np.sign(v), np.sign(Di + Dj))                    # sign of the sum
    gm = np.sqrt(-Di * Dj)
    am = np.abs(Di + Dj) / 2
    tiny = 1e-12 * np.maximum(gm, am)
    assert np.all(np.abs(v) >= np.minimum(gm, am) - tiny)                 # between the two means
    assert np.all(np.abs(v) <= np.maximum(gm, am) + tiny)
    assert np.all(np.abs(v) <= np.maximum(np.abs(Di), np.abs(Dj)))
    # continuity through D_j = 0 from both sides (the equal-sign branch gives 0 there)
    # (from the opposite side it vanishes like |D_j|^(1/4))
    for d in (3e-3, -2e-3):
        sg = np.sign(d)
        opposite = [abs(dmi_average(d, -sg * e)) for e in (1e-6, 1e-12, 1e-30)]
        same = [abs(dmi_average(d, sg * e)) for e in (1e-6, 1e-9, 1e-12)]
        assert opposite[0] > opposite[1] > opposite[2] and opposite[2] < 1e-6 * abs(d)
        assert same[0] > same[1] > same[2] and same[2] < 1e-8 * abs(d)
        assert dmi_average(d, 0.0) == 0.0
    # equal magnitudes of opposite sign cancel
    assert np.all(dmi_average(Di, -Di) == 0.0)


@pytest.mark.parametrize("kind", ["interface", "bulk", "d2d"])
def test_dmi_uniform_m_has_no_interior_field(kind):
    n = (6, 5, 4)
    m = np.broadcast_to(np.array([0.36, 0.48, 0.8]), n + (3,)).copy()
    h = dmi_field(m, 8e5, 3e-3, (2e-9, 2e-9, 2e-9), kind)
    assert np.max(np.abs(h[1:-1, 1:-1, 1:-1])) < 1e-9
    assert np.max(np.abs(h)) > 1e3      # the boundary cells miss a neighbour


@pytest.mark.parametrize("kind,axis,plane,sign", [
    ("interface", 0, (0, 2), 1.0),      # m = (cos qx, 0, sin qx)
    ("interface", 1, (1, 2), 1.0),      # m = (0, cos qy, sin qy)
    ("d2d", 0, (1, 2), 1.0),            # m = (0, cos qx, sin qx)
    ("d2d", 1, (0, 2), 1.0),            # m = (cos qy, 0, sin qy)
    ("bulk", 0, (1, 2), -1.0),          # m = (0, cos qx, sin qx)
    ("bulk", 2, (0, 1), -1.0),          # m = (cos qz, sin qz, 0)
])
def test_dmi_spirals_closed_form(kind, axis, plane, sign):
    """For a spiral along one axis the central difference is exact:
    (m_{i+1} - m_{i-1}) / (2 D) = sin(q D)/D dm/d(qx), and the DMI vector
    turns it back onto m, so h = +-(2 D / (mu0 Ms)) sin(q D)/D m inside."""
    N, d, q, Ms, Dm = 24, 2e-9, 2 * np.pi / 17e-9, 8e5, 3e-3
    n = [1, 1, 1]
    n[axis] = N
    x = (np.arange(N) * d).reshape(n)
    m = np.zeros(tuple(n) + (3,))
    m[..., plane[0]] = np.cos(q * x)
    m[..., plane[1]] = np.sin(q * x)
    h = dmi_field(m, Ms, Dm, (d, d, d), kind)
    expect = sign * 2 * Dm / (MU0 * Ms) * np.sin(q * d) / d * m
    inner = [slice(None)] * 3
    inner[axis] = slice(1, N - 1)
    inner = tuple(inner)
    assert np.max(np.abs(h[inner] - expect[inner])) < 1e-9 * np.max(np.abs(expect))


@pytest.mark.parametrize("kind", ["interface", "bulk", "d2d"])
def test_dmi_operator_is_self_adjoint(kind):
    """sum Ms u . h(v) = sum Ms v . h(u) for per-cell D and Ms: the DMI energy
    is a linear-field energy (Eq. linear_energy_discrete)."""
    rng = np.random.default_rng(5)
    n = (5, 4, 3)
    Ms = rng.uniform(4e5, 9e5, size=n)
    D = rng.uniform(-3e-3, 3e-3, size=n)
    u = rng.normal(size=n + (3,))
    v = rng.normal(size=n + (3,))
    dx = (2e-9, 3e-9, 2.5e-9)
    a = np.sum(Ms[..., None] * u * dmi_field(v, Ms, D, dx, kind))
    b = np.sum(Ms[..., None] * v * dmi_field(u, Ms, D, dx, kind))
    assert abs(a - b) < 1e-12 * (abs(a) + abs(b))

