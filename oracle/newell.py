"""Newell demag tensor and dipole far field (Sec. 4.4).  TEST INFRASTRUCTURE ONLY.

Sec. 4.4 computes the average interaction between two cells with Newell's
formula (Newell, Williams & Dunlop, J. Geophys. Res. 98 (1993) 9551, the
reference cited there) for the ``p`` nearest cells and with the point-dipole
field of Eq. dipole beyond, ``p = 20`` by default.

Sign convention.  ``N`` here is the positive-trace tensor, so that the field of
a uniformly magnetised source cell averaged over a target cell is
``h = -N M``; the self term of a cube is ``N_xx = N_yy = N_zz = 1/3``.  The
kernel written in the discrete convolution of Sec. 4.4 is therefore ``-N``.

Component order everywhere: ``COMPS = (xx, xy, xz, yy, yz, zz)``.

Reading of "the p next neighbors" (Sec. 4.4): Newell's formula is used where
the Chebyshev distance ``max(|i|, |j|, |k|)`` of the cell offset is ``<= p``,
the dipole elsewhere.  ``p=None`` means Newell everywhere.
"""
import math

import numpy as np

COMPS = ((0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2))
COMP_NAMES = ("xx", "xy", "xz", "yy", "yz", "zz")


def newell_f(x, y, z):
    """Newell's f(x, y, z) (diagonal component generator).

    f = y/2 (z^2 - x^2) asinh(y / sqrt(x^2 + z^2))
      + z/2 (y^2 - x^2) asinh(z / sqrt(x^2 + y^2))
      - x y z atan(y z / (x R))
      + (2 x^2 - y^2 - z^2) R / 6,          R = sqrt(x^2 + y^2 + z^2).

    f is even in each argument.  A term whose polynomial prefactor vanishes is
    taken as 0 (this removes the 0 * inf and 0/0 cases on the axes).
    """
    x = np.abs(np.asarray(x, dtype=np.float64))
    y = np.abs(np.asarray(y, dtype=np.float64))
    z = np.abs(np.asarray(z, dtype=np.float64))
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    out = (2.0 * x2 - y2 - z2) * R / 6.0
    with np.errstate(divide="ignore", invalid="ignore"):
        rxz = np.sqrt(x2 + z2)
        rxy = np.sqrt(x2 + y2)
        t1 = 0.5 * y * (z2 - x2) * np.arcsinh(y / rxz)
        t2 = 0.5 * z * (y2 - x2) * np.arcsinh(z / rxy)
        t3 = x * y * z * np.arctan(y * z / (x * R))
    out = out + np.where((y > 0) & (rxz > 0), t1, 0.0)
    out = out + np.where((z > 0) & (rxy > 0), t2, 0.0)
    out = out - np.where((x > 0) & (y > 0) & (z > 0), t3, 0.0)
    return out


def newell_g(x, y, z):
    """Newell's g(x, y, z) (off-diagonal xy component generator).

    g = x y z asinh(z / sqrt(x^2 + y^2))
      + y/6 (3 z^2 - y^2) asinh(x / sqrt(y^2 + z^2))
      + x/6 (3 z^2 - x^2) asinh(y / sqrt(x^2 + z^2))
      - z^3/6 atan(x y / (z R))
      - z y^2/2 atan(x z / (y R))
      - z x^2/2 atan(y z / (x R))
      - x y R / 3.

    g is odd in x, odd in y and even in z; it is evaluated at |x|, |y|, |z|
    and multiplied by sign(x) sign(y).  Vanishing-prefactor terms are 0.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    sgn = np.sign(x) * np.sign(y)
    x, y, z = np.abs(x), np.abs(y), np.abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    out = -x * y * R / 3.0
    with np.errstate(divide="ignore", invalid="ignore"):
        g1 = x * y * z * np.arcsinh(z / np.sqrt(x2 + y2))
        g2 = y / 6.0 * (3.0 * z2 - y2) * np.arcsinh(x / np.sqrt(y2 + z2))
        g3 = x / 6.0 * (3.0 * z2 - x2) * np.arcsinh(y / np.sqrt(x2 + z2))
        g4 = z * z2 / 6.0 * np.arctan(x * y / (z * R))
        g5 = z * y2 / 2.0 * np.arctan(x * z / (y * R))
        g6 = z * x2 / 2.0 * np.arctan(y * z / (x * R))
    out = out + np.where((x > 0) & (y > 0) & (z > 0), g1, 0.0)
    out = out + np.where((x > 0) & (y > 0), g2, 0.0)
    out = out + np.where((x > 0) & (y > 0), g3, 0.0)
    out = out - np.where((z > 0) & (x > 0) & (y > 0), g4, 0.0)
    out = out - np.where((z > 0) & (y > 0) & (x > 0), g5, 0.0)
    out = out - np.where((z > 0) & (x > 0) & (y > 0), g6, 0.0)
    return sgn * out


def _stencil(fun, X, Y, Z, dx, dy, dz):
    """Newell's 27-point combination sum_e w(e) fun(X + e1 dx, Y + e2 dy, Z + e3 dz),
    with w(e) = prod_i (2 if e_i == 0 else -1), divided by 4 pi dx dy dz."""
    acc = np.zeros(np.broadcast(X, Y, Z).shape)
    for a in (-1, 0, 1):
        wa = 2.0 if a == 0 else -1.0
        for b in (-1, 0, 1):
            wb = 2.0 if b == 0 else -1.0
            for c in (-1, 0, 1):
                wc = 2.0 if c == 0 else -1.0
                acc = acc + wa * wb * wc * fun(X + a * dx, Y + b * dy, Z + c * dz)
    return acc / (4.0 * math.pi * dx * dy * dz)


def newell_component(comp, X, Y, Z, dx, dy, dz):
    """Cell-averaged tensor component ``comp`` (one of COMP_NAMES) between two
    cells of size (dx, dy, dz) whose centres are offset by (X, Y, Z) metres.

    The other components follow from f and g by permuting the axes (and the
    cell sizes with them): N_yy(X,Y,Z) = N_xx(Y,X,Z), N_zz(X,Y,Z) = N_xx(Z,Y,X),
    N_xz(X,Y,Z) = N_xy(X,Z,Y), N_yz(X,Y,Z) = N_xy(Y,Z,X)."""
    if comp == "xx":
        return _stencil(newell_f, X, Y, Z, dx, dy, dz)
    if comp == "yy":
        return _stencil(newell_f, Y, X, Z, dy, dx, dz)
    if comp == "zz":
        return _stencil(newell_f, Z, Y, X, dz, dy, dx)
    if comp == "xy":
        return _stencil(newell_g, X, Y, Z, dx, dy, dz)
    if comp == "xz":
        return _stencil(newell_g, X, Z, Y, dx, dz, dy)
    if comp == "yz":
        return _stencil(newell_g, Y, Z, X, dy, dz, dx)
    raise ValueError(comp)


def dipole_component(comp, X, Y, Z, dx, dy, dz):
    """Point-dipole approximation of the same tensor (Eq. dipole).

    Eq. dipole gives the field of a moment V*M at offset r as
    (1/4pi) (3 r (M.r) - |r|^2 M) / |r|^5, i.e. h = -N M with
    N = -(V / (4 pi |r|^3)) (3 r r^T / |r|^2 - I)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    V = dx * dy * dz
    r2 = X * X + Y * Y + Z * Z
    r = np.sqrt(r2)
    pref = -V / (4.0 * math.pi * r2 * r)
    a, b = COMPS[COMP_NAMES.index(comp)]
    va = (X, Y, Z)[a]
    vb = (X, Y, Z)[b]
    delta = 1.0 if a == b else 0.0
    return pref * (3.0 * va * vb / r2 - delta)


def demag_tensor(n, dx, p=20):
    """Demag tensor for every cell offset of an n = (nx, ny, nz) grid of cells
    dx = (dx, dy, dz).

    Returns an array of shape (6, 2nx-1, 2ny-1, 2nz-1) whose entry
    [c, i + nx - 1, j + ny - 1, k + nz - 1] is component COMP_NAMES[c] at
    offset (i dx, j dy, k dz).  Newell where max(|i|,|j|,|k|) <= p (all
    offsets if p is None), the dipole elsewhere."""
    nx, ny, nz = (int(v) for v in n)
    ddx, ddy, ddz = (float(v) for v in dx)
    I, J, K = np.meshgrid(np.arange(-nx + 1, nx), np.arange(-ny + 1, ny),
                          np.arange(-nz + 1, nz), indexing="ij")
    cheb = np.maximum(np.maximum(np.abs(I), np.abs(J)), np.abs(K))
    near = np.ones(I.shape, dtype=bool) if p is None else (cheb <= p)
    X, Y, Z = I * ddx, J * ddy, K * ddz
    out = np.zeros((6,) + I.shape)
    for c, name in enumerate(COMP_NAMES):
        vals = np.zeros(I.shape)
        if near.any():
            vals[near] = newell_component(name, X[near], Y[near], Z[near], ddx, ddy, ddz)
        far = ~near
        if far.any():
            vals[far] = dipole_component(name, X[far], Y[far], Z[far], ddx, ddy, ddz)
        out[c] = vals
    return out


def tensor_at(Nt, n, i, j, k):
    """3x3 tensor at integer offset (i, j, k) taken from a demag_tensor array."""
    nx, ny, nz = n
    v = Nt[:, i + nx - 1, j + ny - 1, k + nz - 1]
    T = np.empty((3, 3))
    for c, (a, b) in enumerate(COMPS):
        T[a, b] = T[b, a] = v[c]
    return T
