"""mm_demag_noalloc: the demag field for callers that cannot allocate device
memory at the moment they need a field (a framework whose allocator owns all
device memory, or a loop that must not stall on the CUDA allocator).  Its
spectrum scratch is a fixed array inside the library, so each case calls it
twice in a row -- the second call finds the first call's data in that array
-- and compares every result with the oracle's FFT convolution (FP64 bound
max(1e-10, the oracle's own rounding floor), FP32 1e-5) and with the demag
field that mm_heff computes with its own allocated buffers.  The shapes reach
the three layouts of the scratch: a 3-D grid, a 2-D grid (nz = 1, where the
tensor multiply runs along y and only the x-spectrum is used), a grid with
ny = 1 (the y-spectrum aliases the x-spectrum) and mixed-radix padded
extents.  Kept in a file that pytest collects last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [
    ((24, 20, 6), (2.5e-9, 2.5e-9, 3e-9)),
    ((50, 48, 1), (2e-9, 2e-9, 2e-9)),       # 2-D: padded 100 x 96 x 1
    ((40, 1, 4), (2e-9, 3e-9, 2e-9)),        # ny = 1
    ((48, 96, 6), (2e-9, 2e-9, 2.5e-9)),     # padded 96 x 192 x 16
]


def _np(t):
    return t.detach().double().cpu().numpy()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("per_cell_ms", [True, False])
@pytest.mark.parametrize("n,d", SHAPES)
def test_noalloc_matches_oracle_and_heff_on_two_calls(n, d, precision, per_cell_ms):
    import torch
    from oracle.demag import demag_fft, magnetization, rounding_sensitivity
    from oracle.newell import demag_tensor
    from paper_2302_08843_gb300 import binding as B
    from paper_2302_08843_gb300.workloads import from_soa, to_soa
    dtype = torch.float64 if precision == "fp64" else torch.float32
    prec = B.MM_FP64 if precision == "fp64" else B.MM_FP32_FIELDS
    rng = np.random.default_rng(21)
    Ms = rng.uniform(5e5, 1.1e6, size=n) if per_cell_ms else None
    Ms0 = 0.0 if per_cell_ms else 8e5
    spec = torch.from_numpy(B.demag_spectrum_host(n, d, 20)).to(dtype).cuda()
    Ms_dev = torch.from_numpy(to_soa(Ms)).to(dtype).cuda() if per_cell_ms else None
    # the existing entry point: a state with only the demag term
    s = B.State(n, d, precision)
    s.set_material(Ms=Ms0, A=0.0, alpha=0.1, Ms_cell=to_soa(Ms) if per_cell_ms else None)
    s.demag_setup(20)
    g = B.mm_grid(n[0], n[1], n[2], d[0], d[1], d[2])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    Nt = demag_tensor(n, d, 20)
    for seed in (1, 2):
        m = np.random.default_rng(seed).normal(size=n + (3,))
        m /= np.linalg.norm(m, axis=-1, keepdims=True)
        mt = torch.from_numpy(to_soa(m)).to(dtype).cuda()
        h = torch.full_like(mt, float("nan"))
        B.check(B.lib().mm_demag_noalloc(ctypes.byref(g), prec, mt.data_ptr(),
                                         None if Ms_dev is None else Ms_dev.data_ptr(), Ms0, spec.data_ptr(),
                                         h.data_ptr(), stream))
        ref_lib = s.heff(m=mt)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(h).all())
        M = magnetization(m, Ms if per_cell_ms else Ms0)
        ref = demag_fft(Nt, M)
        tol = max(1e-10, rounding_sensitivity(n, d, 20, M)) if precision == "fp64" else 1e-5
        hg = from_soa(_np(h))
        assert _rel(hg, ref) < tol, (seed, _rel(hg, ref), tol)
        assert _rel(_np(h), _np(ref_lib)) < tol
    s.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    from paper_2302_08843_gb300 import binding as B
    g = B.mm_grid(256, 256, 64, 2e-9, 2e-9, 2e-9)
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    st = B.lib().mm_demag_noalloc(ctypes.byref(g), B.MM_FP32_FIELDS, dummy.data_ptr(), None, 1e6,
                                  dummy.data_ptr(), dummy.data_ptr(), None)
    assert st == B.MM_EINVAL
    msg = B.lib().mm_last_error().decode()
    assert "maximum" in msg and "256 x 256 x 64" in msg
