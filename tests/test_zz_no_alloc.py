"""mm_demag_noalloc: the demag field for callers that cannot allocate device
memory when they need a field (for example while capturing a stream into a
CUDA graph, or inside a framework whose allocator owns all device memory).
Its spectra scratch is a fixed array inside the library, so these tests call
it twice in a row -- the second call finds the first call's data in that
array -- and compare each result with the demag field that mm_heff computes
with its own allocated buffers.  Kept in a file that pytest collects last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = a.detach().double().cpu().numpy()
    b = b.detach().double().cpu().numpy()
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("per_cell_ms", [True, False])
def test_noalloc_matches_heff_on_two_calls(precision, per_cell_ms):
    import torch
    from paper_2302_08843_gb300 import binding as B
    from paper_2302_08843_gb300.workloads import to_soa
    n = (24, 20, 6)
    d = (2.5e-9, 2.5e-9, 3e-9)
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
    tol = 1e-10 if precision == "fp64" else 1e-5
    for seed in (1, 2):
        m = np.random.default_rng(seed).normal(size=n + (3,))
        m /= np.linalg.norm(m, axis=-1, keepdims=True)
        mt = torch.from_numpy(to_soa(m)).to(dtype).cuda()
        h = torch.full_like(mt, float("nan"))
        B.check(B.lib().mm_demag_noalloc(ctypes.byref(g), prec, mt.data_ptr(),
                                         None if Ms_dev is None else Ms_dev.data_ptr(), Ms0, spec.data_ptr(),
                                         h.data_ptr(), stream))
        ref = s.heff(m=mt)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(h).all())
        assert _rel(h, ref) < tol
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
