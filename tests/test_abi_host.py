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
