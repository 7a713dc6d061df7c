"""Helpers shared by the GPU parity tests (marshalling and comparison only)."""
import numpy as np


def rel(a, b):
    """Relative max-norm ||a - b||_inf / ||b||_inf."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def to_host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def oracle_problem(w, p=20, demag=True, Nt=None):
    from oracle.llg import Problem
    ku_axis = w.ku_axis_cells() if w.grain_id is not None else w.ku_axis
    return Problem(w.n, w.dx, Ms=w.Ms, A=w.A, alpha=w.alpha, Ku1=w.Ku1, ku_axis=ku_axis, h_ext=w.h_ext,
                   h_ext_weight=w.h_ext_weight, p=p, demag=demag, Nt=Nt)


FP32_TOL = 1e-5
