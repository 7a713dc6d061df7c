"""Demag field as a discrete convolution (Sec. 4.4).  TEST INFRASTRUCTURE ONLY.

Sec. 4.4 discretises the demag field as h_i = sum_j N_{i-j} M_j with
M = Ms m.  With the positive-trace tensor of ``oracle.newell`` this reads

    h_i = - sum_j N(i - j) (Ms_j m_j).

Two independent routes are provided:

* ``demag_direct`` / ``demag_direct_c``: the definition, summed term by term
  (NumPy per target cell, or plain C with one OpenMP thread per target cell);
* ``demag_fft``: the zero-padded FFT convolution Sec. 4.4 describes ("zero
  padding of the magnetization ... point-wise multiplication in Fourier
  space"), over a padding P_a = 2 n_a (P_a = 1 where n_a = 1).

The discrete Fourier transforms are library calls: scipy.fft with one worker
thread per host core where SciPy is installed, numpy.fft otherwise (the same
pocketfft algorithm; ``FFT_BACKEND`` says which).

Padding reading: a linear convolution of length n needs P >= 2n - 1.  With
P = 2n the wrapped offset index n is never used by a valid output; it is set
to 0 (keeps the tensor's parity symmetry exact).
"""
import ctypes
import os
import subprocess

import numpy as np

from .newell import COMPS

try:
    import scipy.fft as _sfft

    FFT_WORKERS = os.cpu_count() or 1
    FFT_BACKEND = "scipy.fft, %d workers" % FFT_WORKERS

    def rfftn(a, s, axes):
        return _sfft.rfftn(a, s=s, axes=axes, workers=FFT_WORKERS)

    def irfftn(a, s, axes):
        return _sfft.irfftn(a, s=s, axes=axes, workers=FFT_WORKERS)

    def fft2(a, axes):
        return _sfft.fft2(a, axes=axes, workers=FFT_WORKERS)

    def ifft2(a, axes):
        return _sfft.ifft2(a, axes=axes, workers=FFT_WORKERS)
except ImportError:   # numpy.fft: one thread
    FFT_WORKERS = 1
    FFT_BACKEND = "numpy.fft, 1 thread"

    def rfftn(a, s, axes):
        return np.fft.rfftn(a, s=s, axes=axes)

    def irfftn(a, s, axes):
        return np.fft.irfftn(a, s=s, axes=axes)

    def fft2(a, axes):
        return np.fft.fft2(a, axes=axes)

    def ifft2(a, axes):
        return np.fft.ifft2(a, axes=axes)


def _full(Nt):
    """(6, ...) component array -> (3, 3, ...) symmetric view."""
    T = np.empty((3, 3) + Nt.shape[1:])
    for c, (a, b) in enumerate(COMPS):
        T[a, b] = Nt[c]
        T[b, a] = Nt[c]
    return T


def magnetization(m, Ms):
    """M = Ms m, with Ms a scalar or an (nx, ny, nz) array."""
    Ms = np.broadcast_to(np.asarray(Ms, dtype=np.float64), m.shape[:3])
    return m * Ms[..., None]


def demag_direct(Nt, M):
    """h_i = -sum_j N(i-j) M_j, summed target by target (small grids)."""
    nx, ny, nz = M.shape[:3]
    T = _full(Nt)
    h = np.zeros_like(M)
    si, sj, sk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    for i in range(nx):
        for j in range(ny):
            for k in range(nz):
                oi = i - si + nx - 1
                oj = j - sj + ny - 1
                ok = k - sk + nz - 1
                Nij = T[:, :, oi, oj, ok]  # (3, 3, nx, ny, nz)
                h[i, j, k] = -np.einsum("abxyz,xyzb->a", Nij, M)
    return h


_CLIB = None


def _clib():
    """Load (building if needed) the plain-C brute-force sum in direct_demag.c."""
    global _CLIB
    if _CLIB is None:
        here = os.path.dirname(os.path.abspath(__file__))
        so = os.path.join(here, "_direct_demag.so")
        src = os.path.join(here, "direct_demag.c")
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            build_c()
        lib = ctypes.CDLL(so)
        lib.direct_demag.argtypes = [ctypes.c_int] * 3 + [ctypes.c_void_p] * 3
        lib.direct_demag.restype = None
        _CLIB = lib
    return _CLIB


def build_c():
    """Compile oracle/direct_demag.c into oracle/_direct_demag.so with gcc."""
    here = os.path.dirname(os.path.abspath(__file__))
    so = os.path.join(here, "_direct_demag.so")
    src = os.path.join(here, "direct_demag.c")
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", so, src])
    return so


def demag_direct_c(Nt, M):
    """Same definition as demag_direct, summed in plain C (OpenMP over targets)."""
    nx, ny, nz = M.shape[:3]
    Nt = np.ascontiguousarray(Nt, dtype=np.float64)
    M = np.ascontiguousarray(M, dtype=np.float64)
    assert Nt.shape == (6, 2 * nx - 1, 2 * ny - 1, 2 * nz - 1)
    h = np.zeros_like(M)
    _clib().direct_demag(nx, ny, nz, Nt.ctypes.data, M.ctypes.data, h.ctypes.data)
    return h


def padded_shape(n):
    return tuple(1 if v == 1 else 2 * v for v in n)


def periodic_kernel(Nt, n):
    """Embed the offset tensor into the periodic P-grid: entry a holds N(a)
    for 0 <= a <= n-1, N(a - P) for P-n+1 <= a <= P-1, and 0 otherwise."""
    P = padded_shape(n)
    out = np.zeros((6,) + P)
    idx = []
    for v, p in zip(n, P):
        src = np.array([a if a <= v - 1 else a - p for a in range(p)])
        valid = np.array([(a <= v - 1) or (a >= p - v + 1) for a in range(p)])
        idx.append((src + v - 1, valid))
    (ix, vx), (iy, vy), (iz, vz) = idx
    sub = Nt[:, ix][:, :, iy][:, :, :, iz]
    mask = vx[:, None, None] & vy[None, :, None] & vz[None, None, :]
    out[:] = np.where(mask[None], sub, 0.0)
    return out


def tensor_spectrum(Nt, n):
    """rfftn of the six periodic tensor components over the padded grid."""
    P = padded_shape(n)
    K = periodic_kernel(Nt, n)
    return np.stack([rfftn(K[c], s=P, axes=(0, 1, 2)) for c in range(6)])


def demag_fft(Nt, M, Nhat=None):
    """h = -N * M by zero-padded FFT convolution over P = 2n (Sec. 4.4)."""
    n = M.shape[:3]
    P = padded_shape(n)
    if Nhat is None:
        Nhat = tensor_spectrum(Nt, n)
    Mhat = [rfftn(M[..., b], s=P, axes=(0, 1, 2)) for b in range(3)]
    h = np.empty_like(M)
    for a in range(3):
        acc = np.zeros_like(Mhat[0])
        for c, (p, q) in enumerate(COMPS):
            if p == a:
                acc = acc + Nhat[c] * Mhat[q]
            elif q == a:
                acc = acc + Nhat[c] * Mhat[p]
        h[..., a] = -irfftn(acc, s=P, axes=(0, 1, 2))[: n[0], : n[1], : n[2]]
    return h


def rounding_sensitivity(n, dx, p, M, scales=(1e9, 3.7e8)):
    """The oracle's own floating-point sensitivity of h = -N * M to the
    rounding of Newell's formula: the tensor is dimensionless, so evaluating
    it with the cell sizes expressed in other units (dx * s) must give the same
    tensor; the largest relative max-norm change of h over the scales is the
    noise floor of a double-precision evaluation (the 27-term sum of Sec. 4.4
    cancels about (r/dx)^6 at offset r).  Used to state the FP64 parity bound
    as max(1e-10, this)."""
    from .newell import demag_tensor
    h = demag_fft(demag_tensor(n, dx, p), M)
    sc = np.max(np.abs(h))
    worst = 0.0
    for s in scales:
        hs = demag_fft(demag_tensor(n, tuple(v * s for v in dx), p), M)
        worst = max(worst, float(np.max(np.abs(hs - h)) / sc))
    return worst
