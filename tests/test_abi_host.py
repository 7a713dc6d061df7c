"""CPU-side checks of the C-ABI library: it loads, exports every symbol that
include/mm.h declares, and its host-built demag tensor and tensor spectrum
(Sec. 4.4, built in double precision on the host) agree with the oracle."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mmlib():
    from paper_2302_08843_gb300 import binding
    if not os.path.exists(binding.LIB_PATH):
        from paper_2302_08843_gb300 import build
        build.build()
    return binding


def test_every_declared_symbol_is_exported(mmlib):
    hdr = open(os.path.join(ROOT, "include", "mm.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    declared = set(re.findall(r"\b(mm_[a-z0-9_]+)\s*\(", hdr))
    declared.discard("mm_field_fn")
    assert declared, "no declarations found"
    lib = mmlib.lib()
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(mmlib.EXPORTS)
    assert lib.mm_version().decode().startswith("libmm")


@pytest.mark.parametrize("n,d,p", [((7, 5, 3), (2.5e-9, 3e-9, 2e-9), 20), ((30, 4, 2), (1e-9, 1e-9, 1e-9), 20),
                                   ((25, 3, 3), (1.0, 1.3, 0.7), 4), ((1, 1, 1), (2e-9, 2e-9, 2e-9), 20)])
def test_host_tensor_matches_oracle(mmlib, n, d, p):
    from oracle.newell import demag_tensor
    ours = mmlib.demag_tensor_host(n, d, p)
    ref = demag_tensor(n, d, p)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(ours - ref)) < 1e-12 * scale


@pytest.mark.parametrize("n,d,p", [((8, 4, 2), (2.5e-9, 2.5e-9, 3e-9), 20), ((16, 8, 4), (1.0, 1.2, 0.8), 3),
                                   ((4, 1, 1), (1.0, 1.0, 1.0), 20), ((1, 4, 2), (1.0, 2.0, 1.0), 20),
                                   ((32, 32, 1), (2e-9, 2e-9, 2e-9), 20)])
def test_host_spectrum_matches_oracle_fft(mmlib, n, d, p):
    """Power-of-two grids pad to the same P = 2n as the oracle, so the octant of
    the library's real spectrum equals the oracle's numpy.fft spectrum there
    (times -1/P); the imaginary part of the exact spectrum is zero.  The two
    real-space tensors differ by the rounding noise of Newell's formula, and a
    DFT moves each coefficient by at most the L1 norm of that difference: the
    transform itself may add no more than FFT rounding."""
    from oracle.demag import tensor_spectrum
    from oracle.newell import demag_tensor
    P = mmlib.padded_extents(n)
    ours = mmlib.demag_spectrum_host(n, d, p)
    ref_t = demag_tensor(n, d, p)
    ref = tensor_spectrum(ref_t, n)       # (6, Px, Py, Pz//2+1)
    scale = -1.0 / (P[0] * P[1] * P[2])
    ref_oct = ref[:, : P[0] // 2 + 1, : P[1] // 2 + 1, : P[2] // 2 + 1]   # [c][kx][ky][kz]
    ref_oct = np.transpose(ref_oct, (0, 3, 2, 1)) * scale                # -> [c][kz][ky][kx]
    mag = np.max(np.abs(ref_oct))
    # the exact spectrum is real; numpy's rounding leaves ~1e-12 relative imaginary noise
    assert np.max(np.abs(ref_oct.imag)) < 1e-10 * mag
    l1 = np.sum(np.abs(mmlib.demag_tensor_host(n, d, p) - ref_t), axis=(1, 2, 3)) * abs(scale)
    for c in range(6):
        assert np.max(np.abs(ours[c] - ref_oct[c].real)) <= l1[c] + 1e-13 * mag, c


@pytest.mark.parametrize("n,h,p", [((8, 4, 3), (1.0e-9, 2.5e-9, 0.7e-9), 20),
                                   ((16, 8, 2), (3.0e-9, 1.0e-9), 3),
                                   ((4, 1, 4), (0.6e-9, 1.1e-9, 2.4e-9, 0.8e-9), 20),
                                   ((1, 4, 2), (2.0e-9, 0.5e-9), 20)])
def test_host_layers_spectrum_matches_oracle_fft(mmlib, n, h, p):
    """The library's layer-pair spectrum (pairs i <= j) against numpy.fft of
    the oracle's layer-pair tensor embedded in the library's padded lateral
    grid: real components equal the real part, xz and yz store t with
    spectrum -i t, and every other part vanishes.  The two real-space tensors
    are independent FP64 evaluations, so the bound is their rounding noise,
    far below the size of a wrong sign, pair or scale."""
    from oracle.layers import layered_tensor
    dx, dy = 2e-9, 2.5e-9
    nx, ny, nz = n
    P = mmlib.padded_extents((nx, ny, 1))
    ours = mmlib.layers_spectrum_host(n, dx, dy, h, p)
    T = layered_tensor(n, dx, dy, h, p)                    # (6, nz, nz, 2nx-1, 2ny-1)
    K = np.zeros((6, nz, nz, P[0], P[1]))
    for X in range(-nx + 1, nx):
        for Y in range(-ny + 1, ny):
            K[:, :, :, X % P[0], Y % P[1]] = T[:, :, :, X + nx - 1, Y + ny - 1]
    Kh = np.fft.fft2(K, axes=(3, 4)) * (-1.0 / (P[0] * P[1]))
    Kh = Kh[:, :, :, : P[0] // 2 + 1, : P[1] // 2 + 1]
    mag = np.max(np.abs(Kh))
    q = 0
    for i in range(nz):
        for j in range(i, nz):
            for c in range(6):
                ref = np.transpose(Kh[c, i, j])             # [ky][kx]
                if c in (2, 4):                             # spectrum -i t
                    assert np.max(np.abs(ref.real)) < 1e-10 * mag
                    assert np.max(np.abs(ours[c, q] + ref.imag)) < 1e-9 * mag, (c, i, j)
                else:
                    assert np.max(np.abs(ref.imag)) < 1e-10 * mag
                    assert np.max(np.abs(ours[c, q] - ref.real)) < 1e-9 * mag, (c, i, j)
            q += 1
