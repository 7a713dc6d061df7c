"""Pins for the oracle's Newell tensor (Sec. 4.4) against closed forms,
symmetries, the dipole far field (Eq. dipole) and the exact coarse-graining
property of a cell-averaged tensor."""
import math

import numpy as np
import pytest

from oracle.newell import (COMP_NAMES, demag_tensor, dipole_component,
                           newell_component, tensor_at)


def _self(d):
    return {c: float(newell_component(c, 0.0, 0.0, 0.0, *d)) for c in COMP_NAMES}


def test_cube_self_term_is_one_third():
    s = _self((1.0, 1.0, 1.0))
    for c in ("xx", "yy", "zz"):
        assert abs(s[c] - 1.0 / 3.0) < 1e-15
    for c in ("xy", "xz", "yz"):
        assert abs(s[c]) < 1e-15


@pytest.mark.parametrize("d", [(2.5e-9, 2.5e-9, 3e-9), (1.0, 2.0, 3.0), (3.90625, 3.90625, 3.0),
                               (5.0, 1.0, 0.2), (0.3, 7.0, 1.0)])
def test_self_term_trace_is_one(d):
    s = _self(d)
    assert abs(s["xx"] + s["yy"] + s["zz"] - 1.0) < 1e-13
    # a flat cell (small z extent) has the largest N_zz
    if d[2] < min(d[0], d[1]):
        assert s["zz"] > s["xx"] and s["zz"] > s["yy"]


def test_parity_symmetry():
    rng = np.random.default_rng(0)
    d = (1.0, 1.3, 0.7)
    odd = {"xx": (), "yy": (), "zz": (), "xy": (0, 1), "xz": (0, 2), "yz": (1, 2)}
    for _ in range(20):
        X = rng.integers(-6, 7, 3) * np.array(d)
        for c in COMP_NAMES:
            v0 = float(newell_component(c, *X, *d))
            for ax in range(3):
                Xf = X.copy()
                Xf[ax] = -Xf[ax]
                v1 = float(newell_component(c, *Xf, *d))
                sgn = -1.0 if ax in odd[c] else 1.0
                # the 27-term sum cancels ~6 digits at these offsets, and the
                # mirrored offset sums its terms in another order
                assert abs(v1 - sgn * v0) <= 1e-12


def test_far_field_approaches_dipole():
    d = (1.0, 1.0, 1.0)
    direction = np.array([1.0, 0.7, 0.3])
    errs = []
    for r in (4.0, 8.0, 16.0):
        X = r * direction
        e = 0.0
        for c in COMP_NAMES:
            nw = float(newell_component(c, *X, *d))
            dp = float(dipole_component(c, *X, *d))
            e = max(e, abs(nw - dp))
        scale = 1.0 / (4 * math.pi * r ** 3)
        errs.append(e / scale)
    # leading correction to the point dipole is O((d/r)^2)
    assert errs[1] < errs[0] / 3.0
    assert errs[2] < errs[1] / 3.0
    assert errs[2] < 1e-2


@pytest.mark.parametrize("block", [(2, 2, 2), (2, 3, 1), (3, 1, 2)])
def test_coarse_graining_identity(block):
    """A cell-averaged tensor is exact: summing the fine tensor over all cell
    pairs of two coarse blocks equals (#fine cells per block) times the
    tensor of the coarse cells, for every component and coarse offset."""
    d = (1.0, 1.2, 0.8)
    bx, by, bz = block
    D = (bx * d[0], by * d[1], bz * d[2])
    nb = bx * by * bz
    for off in [(0, 0, 0), (1, 0, 0), (1, 2, -1), (-2, 1, 3), (0, -1, 1)]:
        fine = np.zeros((3, 3))
        for a in np.ndindex(bx, by, bz):
            for b in np.ndindex(bx, by, bz):
                o = [off[i] * block[i] + a[i] - b[i] for i in range(3)]
                for c, name in enumerate(COMP_NAMES):
                    v = float(newell_component(name, o[0] * d[0], o[1] * d[1], o[2] * d[2], *d))
                    p, q = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)][c]
                    fine[p, q] += v
                    if p != q:
                        fine[q, p] += v
        coarse = np.zeros((3, 3))
        for c, name in enumerate(COMP_NAMES):
            v = float(newell_component(name, off[0] * D[0], off[1] * D[1], off[2] * D[2], *D))
            p, q = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)][c]
            coarse[p, q] = coarse[q, p] = v
        assert np.max(np.abs(fine - nb * coarse)) < 1e-11 * max(1.0, np.max(np.abs(nb * coarse)))


def test_tensor_assembly_switch_rule():
    n = (30, 3, 2)
    d = (1.0, 1.0, 1.0)
    Nt = demag_tensor(n, d, p=20)
    Nn = demag_tensor(n, d, p=None)
    # inside the Chebyshev radius the Newell values are used as they are
    assert np.array_equal(Nt[:, 29 - 20:29 + 21], Nn[:, 29 - 20:29 + 21])
    # outside, the dipole
    T = tensor_at(Nt, n, 25, 1, 1)
    X = np.array([25.0, 1.0, 1.0])
    r = np.linalg.norm(X)
    D = -(1.0 / (4 * math.pi * r ** 3)) * (3 * np.outer(X, X) / r ** 2 - np.eye(3))
    assert np.allclose(T, D, rtol=1e-14, atol=0)
    # and the two agree closely at the switch distance
    assert np.max(np.abs(Nt[:, 29 + 21] - Nn[:, 29 + 21])) < 1e-3 * np.max(np.abs(Nn[:, 29 + 21]))
