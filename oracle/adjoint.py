"""Hand-derived discrete adjoint of one RK4 step.  TEST INFRASTRUCTURE ONLY.

Sec. 5.2 obtains gradients with PyTorch's autograd; this module writes the
same derivative out by hand for the LLG right-hand side (Eq. llg) and the
classic RK4 step with renormalisation, in float64.

For f(m) = -g' [p m x h + a m x (m x h)], h = H m + h_ext (H linear: demag,
exchange, anisotropy, DMI), g' = gamma / (1 + a^2), p = 1 with the
precession term and 0 without it (Sec. 3), and a cotangent u of f:

    v = p u + a (u x m),   w = v x m,   G = m x h
    (df/dm)^T u  = -g' [ h x v + a G x u + H^T w ]
    (df/dMs)^T u = -g' (dh/dMs)^T w

with, per cell j (positive-trace N, M = Ms m):
    demag      H^T w = Ms * (-N * w),   d<w,h_dem>/dMs_j = m_j . (-N * w)_j
    exchange   H^T w = Ms * h_ex(w / Ms) (the operator is D L with L symmetric),
               d<w,h_ex>/dMs_j = -w_j . h_ex_j / Ms_j
    DMI        the same form: h_dmi = diag(2/(mu0 Ms)) Q m with Q symmetric
               (a link i, i+k adds c (e_k x m_{i+k}) to cell i and c (e_{-k} x m_i)
               = -c (e_k x m_i) to cell i+k, and u.(e x m') - u'.(e x m) is
               symmetric under (u, u') <-> (m, m')), so H^T w = Ms * h_dmi(w / Ms),
               d<w,h_dmi>/dMs_j = -w_j . h_dmi_j / Ms_j
    anisotropy H^T w = h_u(w) (symmetric per cell), d<w,h_u>/dMs_j = -w_j . h_u_j / Ms_j
    Zeeman     no m or Ms dependence.

RK4 step m' = R(y), y = m + dt sum_s b_s k_s, k_s = f(m_s, t_s),
m_1 = m, m_s = m + dt c_s k_{s-1}; R(y) = y/|y| with (dR)^T l = (l - r (r.l))/|y|.
Reverse sweep: cot k_s = dt b_s l_y + dt c_{s+1} l_{m_{s+1}}, l_{m_s} = (df/dm)^T cot k_s,
l_m = l_y + sum_s l_{m_s}.
"""
import numpy as np

from .constants import GAMMA
from .demag import demag_fft
from .fields import anisotropy_field, dmi_field, exchange_field
from .llg import RK4_B, RK4_C, llg_rhs, normalize


def _gp(prob):
    alpha = np.broadcast_to(np.asarray(prob.alpha, dtype=np.float64), prob.n)
    return alpha, GAMMA / (1.0 + alpha * alpha)


def _ms(prob):
    return np.broadcast_to(np.asarray(prob.Ms, dtype=np.float64), prob.n)


def rhs_vjp(prob, m, t, u):
    """Returns ((df/dm)^T u, (df/dMs)^T u) at (m, t); the second is (nx, ny, nz).
    Covers the LLG with and without the precession term and DMI of any kind
    (equidistant grids; non-equidistant layers are not covered)."""
    if getattr(prob, "layers", None) is not None:
        raise ValueError("rhs_vjp covers equidistant grids")
    alpha, gp = _gp(prob)
    Ms = _ms(prob)
    pc = 1.0 if getattr(prob, "precession", True) else 0.0
    h = prob.heff(m, t)
    hex_ = exchange_field(m, prob.Ms, prob.A, prob.dx)
    hu = anisotropy_field(m, prob.Ms, prob.Ku1, prob.ku_axis)
    hd = dmi_field(m, prob.Ms, prob.D, prob.dx, prob.dmi)
    a = alpha[..., None]
    ok = Ms != 0
    # a cell with Ms = 0 has f = 0 identically: its cotangent reaches nothing
    v = pc * u + a * np.cross(u, m)
    w = np.cross(v, m) * ok[..., None]
    G = np.cross(m, h)
    inv = np.zeros(prob.n)
    np.divide(1.0, Ms, out=inv, where=Ms != 0)
    hw = demag_fft(prob.Nt, w, prob.Nhat) if prob.demag else np.zeros_like(m)   # -N * w
    q = w * inv[..., None]
    HTw = Ms[..., None] * hw + Ms[..., None] * exchange_field(q, prob.Ms, prob.A, prob.dx) \
        + Ms[..., None] * dmi_field(q, prob.Ms, prob.D, prob.dx, prob.dmi) \
        + anisotropy_field(w, prob.Ms, prob.Ku1, prob.ku_axis)
    lam = -gp[..., None] * (np.cross(h, v) + a * np.cross(G, u) + HTw)
    dMs = np.sum(m * hw, axis=-1) - np.sum(w * (hex_ + hu + hd), axis=-1) * inv
    gMs = -gp * dMs
    lam = lam * ok[..., None]
    gMs = gMs * ok
    return lam, gMs


def rk4_step_vjp(prob, m, t, dt, lam_next, renorm=True):
    """Cotangent of m (and of Ms) for one RK4 step from (m, t), given the
    cotangent lam_next of its result."""
    ms = [m]
    ks = []
    for s in range(4):
        ks.append(prob.rhs(ms[s], t + RK4_C[s] * dt))
        if s < 3:
            ms.append(m + dt * RK4_C[s + 1] * ks[s])
    y = m + dt * sum(RK4_B[s] * ks[s] for s in range(4))
    if renorm:
        ny = np.linalg.norm(y, axis=-1, keepdims=True)
        r = y / ny
        lam_y = (lam_next - r * np.sum(r * lam_next, axis=-1, keepdims=True)) / ny
    else:
        lam_y = lam_next
    lam_m = lam_y.copy()
    gMs = np.zeros(prob.n)
    lam_ms_next = None
    for s in (3, 2, 1, 0):
        cot = dt * RK4_B[s] * lam_y
        if lam_ms_next is not None:
            cot = cot + dt * RK4_C[s + 1] * lam_ms_next
        lam_ms, g = rhs_vjp(prob, ms[s], t + RK4_C[s] * dt, cot)
        lam_m = lam_m + lam_ms
        gMs = gMs + g
        lam_ms_next = lam_ms
    return lam_m, gMs


def rollout_loss_and_grad(prob_factory, Ms_cell, m0, dt, steps, weight, t0=0.0):
    """L = sum_n <weight, m_n> over n = 1..steps for an RK4 rollout with
    per-cell Ms (prob_factory(Ms_cell) builds the problem); returns
    (L, dL/dMs_cell) by the adjoint sweep (all states kept)."""
    prob = prob_factory(Ms_cell)
    ms = [m0]
    m = m0
    for n in range(steps):
        from .llg import rk4_step
        m = rk4_step(prob, m, t0 + n * dt, dt)
        ms.append(m)
    L = float(sum(np.sum(weight * ms[n]) for n in range(1, steps + 1)))
    lam = weight.copy()
    g = np.zeros(prob.n)
    for n in range(steps - 1, -1, -1):
        lam_n, gn = rk4_step_vjp(prob, ms[n], t0 + n * dt, dt, lam)
        g += gn
        lam = lam_n + (weight if n >= 1 else 0.0)
    return L, g
