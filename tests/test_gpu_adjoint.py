"""GPU parity of the hand-written adjoint (mm_llg_step_adjoint): one RK4 step
against the oracle's FP64 adjoint, and the gradient of a checkpointed rollout
with respect to the density w of the inverse-design problem (Sec. 5.2,
Ms = sigmoid(w) Ms0) against central finite differences of the GPU forward."""
import numpy as np
import pytest

from gpu_util import rel, to_host

pytestmark = pytest.mark.gpu


def test_adjoint_step_matches_oracle_fp64():
    import torch
    from oracle.adjoint import rk4_step_vjp
    from oracle.constants import MU0
    from oracle.llg import Problem, normalize
    from paper_2302_08843_gb300.binding import State
    from paper_2302_08843_gb300.workloads import from_soa, to_soa
    n, d = (8, 6, 3), (3e-9, 2.5e-9, 3e-9)
    rng = np.random.default_rng(12)
    Ms = rng.uniform(5e5, 1e6, size=n)
    m = normalize(rng.normal(size=n + (3,)))
    lam1 = rng.normal(size=n + (3,))
    hfun = lambda t: np.array([0.02 / MU0, 0.01 / MU0 * np.cos(2e10 * t), 0.0])
    prob = Problem(n, d, Ms=Ms, A=1.3e-11, alpha=0.3, Ku1=2e5, ku_axis=(0.0, 0.6, 0.8), h_ext=hfun)
    dt, t = 5e-14, 1e-12
    lam_ref, g_ref = rk4_step_vjp(prob, m, t, dt, lam1)
    s = State(n, d, "fp64")
    s.set_material(Ms=0.0, A=1.3e-11, alpha=0.3, Ku1=2e5, ku_axis=(0.0, 0.6, 0.8), Ms_cell=to_soa(Ms))
    s.set_zeeman(fn=hfun)
    s.demag_setup(20)
    gMs = torch.zeros((n[2], n[1], n[0]), dtype=torch.float64, device="cuda")
    lam = s.step_adjoint(to_soa(m), to_soa(lam1), dt, t, grad_Ms=gMs)
    assert rel(from_soa(to_host(lam)), lam_ref) < 1e-9
    assert rel(from_soa(to_host(gMs)), g_ref) < 1e-9
    s.close()


def _rollout_loss(s, w, Ms0, m0, weight, dt, steps, every, mat, grad=False):
    import torch
    from paper_2302_08843_gb300.autodiff import rk4_observable
    wt = torch.tensor(w, dtype=torch.float64, device="cuda", requires_grad=grad)
    Ms = torch.sigmoid(wt) * Ms0
    obs = rk4_observable(Ms, s, m0, weight, dt, steps, every, mat)
    loss = obs.mean()
    if grad:
        loss.backward()
        return float(loss.detach()), wt.grad.detach().cpu().numpy()
    return float(loss.detach())


def test_rollout_gradient_matches_central_differences_fp64():
    """16x16x1 version of the inverse-design workload, 60 RK4 steps with a
    checkpoint every 7 steps; dL/dw by the adjoint vs (L(w+e) - L(w-e)) / 2e."""
    import torch
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import State
    from paper_2302_08843_gb300.workloads import to_soa
    w0 = W.inverse_design(n=(16, 16, 1), strip=3, out_box=((11, 14), (6, 10)))
    s = State(w0.n, w0.dx, "fp64")
    s.set_zeeman(fn=w0.h_ext, weight=to_soa(w0.h_ext_weight))
    s.demag_setup(20)
    m0 = torch.from_numpy(to_soa(w0.m0)).cuda()
    weight = np.zeros(w0.n + (3,))
    (x0, x1), (y0, y1) = w0.extra["out_box"]
    weight[x0:x1, y0:y1, :, 1] = 1.0 / ((x1 - x0) * (y1 - y0))
    weight = torch.from_numpy(to_soa(weight)).cuda()
    mat = dict(A=1.3e-11, alpha=0.05)
    wz = to_soa(w0.extra["w"])
    L, g = _rollout_loss(s, wz, 8e5, m0, weight, 2e-13, 60, 7, mat, grad=True)
    eps = 1e-6
    for idx in [(0, 8, 2), (0, 8, 9), (0, 3, 12), (0, 12, 12)]:
        wp = wz.copy(); wp[idx] += eps
        wm = wz.copy(); wm[idx] -= eps
        fd = (_rollout_loss(s, wp, 8e5, m0, weight, 2e-13, 60, 7, mat)
              - _rollout_loss(s, wm, 8e5, m0, weight, 2e-13, 60, 7, mat)) / (2 * eps)
        assert abs(g[idx] - fd) <= 1e-6 * abs(fd) + 1e-12 * np.max(np.abs(g)), (idx, g[idx], fd)
    s.close()


def test_inverse_design_fp32_gradient_vs_fp64():
    """The inverse-design workload at full size: 128x128x1, 2000 RK4 steps of
    5e-14 s, loss = time average of the mean m_y over the 10x10 output region,
    checkpoints every 100 steps.  The FP32-fields gradient against the FP64
    gradient of the same GPU path (the FP64 adjoint is pinned above)."""
    import torch
    from paper_2302_08843_gb300 import workloads as W
    from paper_2302_08843_gb300.binding import State
    from paper_2302_08843_gb300.workloads import to_soa
    w0 = W.inverse_design()
    grads = {}
    for prec in ("fp64", "fp32"):
        s = State(w0.n, w0.dx, prec)
        s.set_zeeman(fn=w0.h_ext, weight=to_soa(w0.h_ext_weight))
        s.demag_setup(20)
        dtype = torch.float64 if prec == "fp64" else torch.float32
        m0 = torch.from_numpy(to_soa(w0.m0)).to(dtype).cuda()
        weight = np.zeros(w0.n + (3,))
        (x0, x1), (y0, y1) = w0.extra["out_box"]
        weight[x0:x1, y0:y1, :, 1] = 1.0 / ((x1 - x0) * (y1 - y0))
        weight = torch.from_numpy(to_soa(weight)).to(dtype).cuda()
        L, g = _rollout_loss(s, to_soa(w0.extra["w"]), 8e5, m0, weight, w0.dt, w0.steps, 100,
                             dict(A=1.3e-11, alpha=0.05), grad=True)
        grads[prec] = g
        s.close()
    g64, g32 = grads["fp64"].ravel(), grads["fp32"].ravel()
    cos = float(g64 @ g32 / (np.linalg.norm(g64) * np.linalg.norm(g32)))
    err = float(np.max(np.abs(g32 - g64)) / np.max(np.abs(g64)))
    print("inverse-design gradient FP32 vs FP64: cos %.8f rel max-norm %.3e" % (cos, err))
    assert np.all(np.isfinite(g32)) and np.max(np.abs(g64)) > 0
    # measured: cos 1 - 1e-8, rel 3.2e-6
    assert cos > 0.99999 and err < 1e-4
