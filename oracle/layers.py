"""Demag for a stack of layers of unequal thickness (Sec. 4.4, the
non-equidistant layers).  TEST INFRASTRUCTURE ONLY.

Sec. 4.4 notes that for several thin layers that are not equidistant the
convolution theorem can still be used in the two lateral dimensions, with a
dense coupling between the nz layers.  The tensor between a target cell of
layer i and a source cell of layer j is Newell's cell average (same f and g
as ``oracle.newell``) with the z part of the stencil written for two boxes of
different thickness: where equal cells combine 2 F(Z) - F(Z + h) - F(Z - h),
boxes of thickness h_i (target) and h_j (source) whose lower faces are Z0
apart combine

    F(Z0) - F(Z0 + h_i) - F(Z0 - h_j) + F(Z0 + h_i - h_j),

and the sum is divided by 4 pi dx dy h_i (the target volume).  For h_i = h_j
this is the equidistant tensor; it satisfies h_i N_ij(r) = h_j N_ji(-r)
(the double integral is symmetric), and it is additive when a source layer
is split in two.

Readings (the paper gives the idea and a citation only):
* the layers are stacked without gaps, layer k between z_k and z_k + h_k;
* Newell's formula is used where the Chebyshev distance
  max(|I|, |J|, |i - j|) of (lateral cell offset, layer offset) is <= p
  (p = 20 as for the equidistant grid), the point dipole of Eq. dipole
  beyond, with the source cell's moment dx dy h_j M and the centre offset
  (X, Y, Z0 + (h_i - h_j) / 2); this keeps h_i N_ij(r) = h_j N_ji(-r);
* exchange between neighbouring layers is the finite-volume difference
  (2 / (mu0 Ms)) A_link (m_{k+1} - m_k) / (h_k d_{k,k+1}) with the
  centre distance d_{k,k+1} = (h_k + h_{k+1}) / 2, which is the equidistant
  1 / dz^2 when the layers are equal (see ``oracle.fields``);
* energies use each cell's own volume dx dy h_k.

Arrays: m, M are (nx, ny, nz, 3); the tensor is (6, nz, nz, 2nx-1, 2ny-1)
with entry [c, i, j, X + nx - 1, Y + ny - 1] for target layer i, source
layer j and lateral offset (X dx, Y dy) of target minus source.
"""
import math

import numpy as np

from .demag import fft2, ifft2
from .fields import exchange_field
from .newell import COMP_NAMES, dipole_component, newell_f, newell_g


def _zterms(Z0, hi, hj):
    """The four z arguments and signs of the unequal-box stencil."""
    return ((Z0, 1.0), (Z0 + hi, -1.0), (Z0 - hj, -1.0), (Z0 + hi - hj, 1.0))


def layer_component(comp, X, Y, Z0, dx, dy, hi, hj):
    """Tensor component ``comp`` between a target cell of thickness hi and a
    source cell of thickness hj, lateral centre offset (X, Y) (target minus
    source) and lower-face offset Z0 (target minus source)."""
    acc = np.zeros(np.broadcast(X, Y, Z0).shape)
    for a in (-1, 0, 1):
        wa = 2.0 if a == 0 else -1.0
        for b in (-1, 0, 1):
            wb = 2.0 if b == 0 else -1.0
            x = X + a * dx
            y = Y + b * dy
            for z, wz in _zterms(Z0, hi, hj):
                if comp == "xx":
                    v = newell_f(x, y, z)
                elif comp == "yy":
                    v = newell_f(y, x, z)
                elif comp == "zz":
                    v = newell_f(z, y, x)
                elif comp == "xy":
                    v = newell_g(x, y, z)
                elif comp == "xz":
                    v = newell_g(x, z, y)
                elif comp == "yz":
                    v = newell_g(y, z, x)
                else:
                    raise ValueError(comp)
                acc = acc + wa * wb * wz * v
    return acc / (4.0 * math.pi * dx * dy * hi)


def layer_bottoms(h):
    """Lower faces of the stacked layers."""
    h = np.asarray(h, dtype=np.float64)
    return np.concatenate(([0.0], np.cumsum(h)[:-1]))


def layer_dipole(comp, X, Y, Z0, dx, dy, hi, hj):
    """Point-dipole value of the same entry: source moment dx dy hj, centre
    offset (X, Y, Z0 + (hi - hj) / 2)."""
    Zc = Z0 + 0.5 * (hi - hj)
    # dipole_component takes the source volume as dx dy dz
    return dipole_component(comp, X, Y, Zc, dx, dy, hj)


def layered_tensor(n, dx, dy, h, p=20):
    """Tensor for every lateral offset and layer pair of an (nx, ny, nz) grid
    with lateral cells dx, dy and layer thicknesses h (length nz); Newell
    where max(|I|, |J|, |i - j|) <= p (everywhere if p is None), the dipole
    beyond."""
    nx, ny, nz = (int(v) for v in n)
    h = np.asarray(h, dtype=np.float64)
    if h.shape != (nz,) or np.any(h <= 0):
        raise ValueError("one positive thickness per layer")
    z0 = layer_bottoms(h)
    I, J = np.meshgrid(np.arange(-nx + 1, nx), np.arange(-ny + 1, ny), indexing="ij")
    X, Y = I * float(dx), J * float(dy)
    lat = np.maximum(np.abs(I), np.abs(J))
    out = np.zeros((6, nz, nz) + I.shape)
    for c, name in enumerate(COMP_NAMES):
        for i in range(nz):
            for j in range(nz):
                near = np.ones(I.shape, dtype=bool) if p is None else (np.maximum(lat, abs(i - j)) <= p)
                Z0 = z0[i] - z0[j]
                vals = np.zeros(I.shape)
                if near.any():
                    vals[near] = layer_component(name, X[near], Y[near], Z0, float(dx), float(dy), h[i], h[j])
                if (~near).any():
                    vals[~near] = layer_dipole(name, X[~near], Y[~near], Z0, float(dx), float(dy), h[i], h[j])
                out[c, i, j] = vals
    return out


def layered_demag_direct(T, M):
    """h_i(r) = -sum_j sum_r' N_ij(r - r') M_j(r'): the definition, summed out."""
    nx, ny, nz, _ = M.shape
    h = np.zeros_like(M)
    for i in range(nz):
        for j in range(nz):
            for xs in range(nx):
                for ys in range(ny):
                    Xo = np.arange(nx)[:, None] - xs + nx - 1
                    Yo = np.arange(ny)[None, :] - ys + ny - 1
                    v = T[:, i, j][:, Xo, Yo]                     # (6, nx, ny)
                    m = M[xs, ys, j]
                    h[:, :, i, 0] -= v[0] * m[0] + v[1] * m[1] + v[2] * m[2]
                    h[:, :, i, 1] -= v[1] * m[0] + v[3] * m[1] + v[4] * m[2]
                    h[:, :, i, 2] -= v[2] * m[0] + v[4] * m[1] + v[5] * m[2]
    return h


def layered_demag_fft(T, M):
    """The lateral convolution by 2-D FFTs zero-padded to (2nx, 2ny), the
    layers coupled densely at every lateral wave number."""
    nx, ny, nz, _ = M.shape
    Px, Py = 2 * nx, 2 * ny
    # circulant embedding of the lateral offsets; the unused offset (nx, ny) stays 0
    K = np.zeros((6, nz, nz, Px, Py))
    for X in range(-nx + 1, nx):
        for Y in range(-ny + 1, ny):
            K[:, :, :, X % Px, Y % Py] = T[:, :, :, X + nx - 1, Y + ny - 1]
    Kh = fft2(K, axes=(3, 4))
    Mh = fft2(np.pad(M, ((0, Px - nx), (0, Py - ny), (0, 0), (0, 0))), axes=(0, 1))
    comp = ((0, 1, 2), (1, 3, 4), (2, 4, 5))
    hh = np.zeros((Px, Py, nz, 3), dtype=complex)
    for i in range(nz):
        for j in range(nz):
            for a in range(3):
                for b in range(3):
                    hh[:, :, i, a] -= Kh[comp[a][b], i, j] * Mh[:, :, j, b]
    return np.real(ifft2(hh, axes=(0, 1)))[:nx, :ny]


def thickness_harmonic(Ai, Aj, hi, hj):
    """A of the link between cells of thickness hi, hj (in series): the link
    of length (hi + hj) / 2 runs hi / 2 through A_i and hj / 2 through A_j,
    so A_link = (hi + hj) A_i A_j / (hi A_j + hj A_i); 0 where both A are 0.
    Equal thicknesses give the harmonic mean of the equidistant grid."""
    Ai = np.asarray(Ai, dtype=np.float64)
    Aj = np.asarray(Aj, dtype=np.float64)
    den = hi * Aj + hj * Ai
    out = np.zeros(np.broadcast(Ai, Aj, den).shape)
    np.divide((hi + hj) * Ai * Aj, den, out=out, where=den != 0)
    return out


def exchange_field_layers(m, Ms, A, dx, dy, h):
    """Exchange field with unequal layers: the lateral links of the
    equidistant rule, and between layers k and k+1
    h_k += 2 / (mu0 Ms_k) A_link (m_{k+1} - m_k) / (h_k d),
    h_{k+1} -= 2 / (mu0 Ms_{k+1}) A_link (m_{k+1} - m_k) / (h_{k+1} d),
    d = (h_k + h_{k+1}) / 2 (the layer-centre distance)."""
    from .constants import MU0
    shape = m.shape[:3]
    h = np.asarray(h, dtype=np.float64)
    out = exchange_field(m, Ms, A, (dx, dy, 1.0), axes=(0, 1))
    A = np.broadcast_to(np.asarray(A, dtype=np.float64), shape)
    Ms = np.broadcast_to(np.asarray(Ms, dtype=np.float64), shape)
    inv = np.zeros(shape)
    np.divide(1.0, Ms, out=inv, where=Ms != 0)
    for k in range(shape[2] - 1):
        d = 0.5 * (h[k] + h[k + 1])
        Al = thickness_harmonic(A[:, :, k], A[:, :, k + 1], h[k], h[k + 1])
        diff = m[:, :, k + 1] - m[:, :, k]
        out[:, :, k] += ((2.0 / MU0) * inv[:, :, k] * Al / (h[k] * d))[..., None] * diff
        out[:, :, k + 1] -= ((2.0 / MU0) * inv[:, :, k + 1] * Al / (h[k + 1] * d))[..., None] * diff
    return out


def exchange_energy_links(m, A, dx, dy, h):
    """The discrete exchange energy written per link, sum_links A_link S |m_a - m_b|^2 / d
    (S the face area, d the centre distance): the energy whose gradient
    the exchange field is, h = -1/(mu0 Ms V) dE/dm."""
    shape = m.shape[:3]
    h = np.asarray(h, dtype=np.float64)
    A = np.broadcast_to(np.asarray(A, dtype=np.float64), shape)
    E = 0.0
    for ax, (d, S) in enumerate(((dx, dy * h[None, None, :]), (dy, dx * h[None, None, :]))):
        n = shape[ax]
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, n - 1)
        hi[ax] = slice(1, n)
        lo, hi = tuple(lo), tuple(hi)
        Al = thickness_harmonic(A[lo], A[hi], 1.0, 1.0)
        S_l = np.broadcast_to(S, shape)[lo]
        E += float(np.sum(Al * S_l * np.sum((m[hi] - m[lo]) ** 2, axis=-1) / d))
    for k in range(shape[2] - 1):
        d = 0.5 * (h[k] + h[k + 1])
        Al = thickness_harmonic(A[:, :, k], A[:, :, k + 1], h[k], h[k + 1])
        E += float(np.sum(Al * dx * dy * np.sum((m[:, :, k + 1] - m[:, :, k]) ** 2, axis=-1) / d))
    return E


def layered_demag_at(n, dx, dy, h, M, cells, p=20):
    """Demag field at the listed target cells (x, y, layer) by the direct sum
    over every source cell, the entries evaluated on the fly with the same
    rule as layered_tensor: for spot checks of grids too large for the whole
    tensor."""
    nx, ny, nz = (int(v) for v in n)
    h = np.asarray(h, dtype=np.float64)
    z0 = layer_bottoms(h)
    out = np.zeros((len(cells), 3))
    for q, (x, y, i) in enumerate(cells):
        I = (x - np.arange(nx))[:, None] + np.zeros((1, ny), dtype=int)
        J = (y - np.arange(ny))[None, :] + np.zeros((nx, 1), dtype=int)
        X, Y = I * float(dx), J * float(dy)
        lat = np.maximum(np.abs(I), np.abs(J))
        for j in range(nz):
            near = np.ones(I.shape, dtype=bool) if p is None else (np.maximum(lat, abs(i - j)) <= p)
            Z0 = z0[i] - z0[j]
            N = np.zeros((6,) + I.shape)
            for c, name in enumerate(COMP_NAMES):
                if near.any():
                    N[c][near] = layer_component(name, X[near], Y[near], Z0, float(dx), float(dy), h[i], h[j])
                if (~near).any():
                    N[c][~near] = layer_dipole(name, X[~near], Y[~near], Z0, float(dx), float(dy), h[i], h[j])
            Mj = M[:, :, j]
            out[q, 0] -= np.sum(N[0] * Mj[..., 0] + N[1] * Mj[..., 1] + N[2] * Mj[..., 2])
            out[q, 1] -= np.sum(N[1] * Mj[..., 0] + N[3] * Mj[..., 1] + N[4] * Mj[..., 2])
            out[q, 2] -= np.sum(N[2] * Mj[..., 0] + N[4] * Mj[..., 1] + N[5] * Mj[..., 2])
    return out


def layered_rounding_sensitivity(n, dx, dy, h, p, M, scales=(1e9, 3.7e8)):
    """Floating-point noise of the oracle's own layered demag: the tensor is
    dimensionless, so building it with lengths in other units must give the
    same field; the largest relative max-norm change over the scales bounds
    what an FP64 evaluation can reproduce (the 36-term stencil cancels
    strongly at large offsets)."""
    h = np.asarray(h, dtype=np.float64)
    ref = layered_demag_fft(layered_tensor(n, dx, dy, h, p), M)
    sc = np.max(np.abs(ref))
    worst = 0.0
    for s in scales:
        hs = layered_demag_fft(layered_tensor(n, dx * s, dy * s, h * s, p), M)
        worst = max(worst, float(np.max(np.abs(hs - ref)) / sc))
    return worst
