"""Local field terms and energies.  TEST INFRASTRUCTURE ONLY.

exchange_field     : Sec. 4.2, discretised exchange field with the harmonic
                     mean of A on every link and the Neumann boundary (a link
                     to a cell outside the grid does not exist).
anisotropy_field   : Sec. 4.1, first-order uniaxial anisotropy (the Ku1 term
                     of the anisotropy equation; the code listing of Sec. 4.1
                     maps the 0/0 of an Ms = 0 cell to 0 with nan_to_num).
zeeman_field       : external field; Sec. 5.1 only shows ``ExternalField``.
                     It is given here as h(t) * w_i with an optional per-cell
                     weight w (1 where absent).
dmi_field          : Sec. 4.3, the central-difference DMI field
                     h_i = 2/(mu0 Ms_i) sum_{k=+-x,+-y,+-z} Dt_{i,k} e_k x m_{i+k} / (2 D_k)
                     with the DMI vectors of the paper's table (e_{-k} = -e_k);
                     a neighbour outside the grid is left out (the "ignore
                     the non-existing values" option of Sec. 4.3).
dmi_average        : Eq. D_avg, the effective coupling Dt of a link (see the
                     readings there).
linear_energy      : Eq. linear_energy_discrete, E = -1/2 mu0 V sum Ms m.h.
zeeman_energy      : E = -mu0 V sum Ms m.h_ext (no 1/2; the paper gives no
                     Zeeman energy, this is the standard one for a field that
                     does not depend on m).

Arrays: m is (nx, ny, nz, 3); Ms, A, Ku1 are scalars or (nx, ny, nz);
the easy axis is a (3,) vector or an (nx, ny, nz, 3) array of unit vectors.
"""
import numpy as np

from .constants import MU0


def _grid(v, shape):
    return np.broadcast_to(np.asarray(v, dtype=np.float64), shape)


def _inv_ms(Ms, shape):
    """1/Ms with 0 where Ms == 0 (the nan_to_num of Sec. 4.1)."""
    Ms = _grid(Ms, shape)
    out = np.zeros(shape)
    np.divide(1.0, Ms, out=out, where=Ms != 0)
    return out


def exchange_field(m, Ms, A, dx, axes=(0, 1, 2)):
    """h_i = 2/(mu0 Ms_i) sum_{k=+-x,+-y,+-z} 2/D_k^2 A_{i+k} A_i/(A_{i+k}+A_i) (m_{i+k} - m_i).

    A link whose harmonic-mean denominator A_i + A_{i+k} is 0 carries no
    weight (reading: both cells have A = 0).  ``axes`` limits the sum to
    the links along the given axes."""
    shape = m.shape[:3]
    A = _grid(A, shape)
    h = np.zeros_like(m)
    for ax in axes:
        d2 = float(dx[ax]) ** 2
        n = shape[ax]
        if n < 2:
            continue
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, n - 1)
        hi[ax] = slice(1, n)
        lo, hi = tuple(lo), tuple(hi)
        Alo, Ahi = A[lo], A[hi]
        den = Alo + Ahi
        w = np.zeros(den.shape)
        np.divide(Alo * Ahi, den, out=w, where=den != 0)
        coef = (2.0 / d2) * w
        diff = m[hi] - m[lo]
        h[lo] += coef[..., None] * diff     # cell i gets its +k neighbour
        h[hi] -= coef[..., None] * diff     # cell i+k gets its -k neighbour
    return h * (2.0 / MU0) * _inv_ms(Ms, shape)[..., None]


def anisotropy_field(m, Ms, Ku1, axis):
    """h = 2 Ku1 / (mu0 Ms) e (e . m)."""
    shape = m.shape[:3]
    e = np.broadcast_to(np.asarray(axis, dtype=np.float64), m.shape)
    Ku1 = _grid(Ku1, shape)
    em = np.sum(e * m, axis=-1)
    return (2.0 / MU0) * (Ku1 * _inv_ms(Ms, shape) * em)[..., None] * e


def zeeman_field(h_ext, shape, weight=None):
    """h_i = w_i h_ext (h_ext a (3,) vector in A/m)."""
    h = np.broadcast_to(np.asarray(h_ext, dtype=np.float64), tuple(shape) + (3,)).copy()
    if weight is not None:
        h *= np.asarray(weight, dtype=np.float64)[..., None]
    return h


def linear_energy(m, h, Ms, V):
    """Eq. linear_energy_discrete: E = -1/2 mu0 V sum_i Ms_i m_i . h_i
    (V a scalar, or per cell: an array broadcastable to the grid)."""
    Ms = _grid(Ms, m.shape[:3])
    if np.ndim(V) == 0:
        return -0.5 * MU0 * V * float(np.sum(Ms * np.sum(m * h, axis=-1)))
    return -0.5 * MU0 * float(np.sum(_grid(V, m.shape[:3]) * Ms * np.sum(m * h, axis=-1)))


def zeeman_energy(m, h, Ms, V):
    """E = -mu0 V sum_i Ms_i m_i . h_i (V as in linear_energy)."""
    Ms = _grid(Ms, m.shape[:3])
    if np.ndim(V) == 0:
        return -MU0 * V * float(np.sum(Ms * np.sum(m * h, axis=-1)))
    return -MU0 * float(np.sum(_grid(V, m.shape[:3]) * Ms * np.sum(m * h, axis=-1)))


# DMI vectors (e_x, e_y, e_z) of the paper's table of DMI types
DMI_VECTORS = {
    "interface": ((0.0, 1.0, 0.0), (-1.0, 0.0, 0.0), (0.0, 0.0, 0.0)),
    "bulk": ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0)),
    "d2d": ((-1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 0.0)),
}


def dmi_average(Di, Dj):
    """Eq. D_avg, element-wise.  Readings of the printed formula (garbled):
    equal signs (Di Dj >= 0) take the harmonic mean 2 Di Dj / (Di + Dj)
    (0 when both are 0), as the text says; opposite signs take the geometric
    mean of the geometric mean sqrt(-Di Dj) and the arithmetic mean
    |Di + Dj| / 2, with the sign of Di + Dj."""
    Di = np.asarray(Di, dtype=np.float64)
    Dj = np.asarray(Dj, dtype=np.float64)
    prod = Di * Dj
    s = Di + Dj
    harm = np.zeros(np.broadcast(Di, Dj).shape)
    np.divide(2.0 * prod, s, out=harm, where=(s != 0) & (prod >= 0))
    opp = np.sign(s) * np.sqrt(np.sqrt(np.maximum(-prod, 0.0)) * np.abs(s) / 2.0)
    return np.where(prod >= 0, harm, opp)


def dmi_field(m, Ms, D, dx, kind="interface"):
    """h_i = 2/(mu0 Ms_i) sum_k Dt_{i,k} e_k x m_{i+k} / (2 D_k), k = +-x, +-y, +-z."""
    shape = m.shape[:3]
    D = _grid(D, shape)
    vecs = DMI_VECTORS[kind]
    h = np.zeros_like(m)
    for ax in range(3):
        e = np.asarray(vecs[ax], dtype=np.float64)
        n = shape[ax]
        if n < 2 or not e.any():
            continue
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, n - 1)
        hi[ax] = slice(1, n)
        lo, hi = tuple(lo), tuple(hi)
        Dt = dmi_average(D[lo], D[hi]) / (2.0 * float(dx[ax]))
        eb = np.broadcast_to(e, m[hi].shape)
        h[lo] += Dt[..., None] * np.cross(eb, m[hi])      # cell i, neighbour +k, vector +e
        h[hi] -= Dt[..., None] * np.cross(eb, m[lo])      # cell i+k, neighbour -k, vector -e
    return h * (2.0 / MU0) * _inv_ms(Ms, shape)[..., None]
