"""LLG right-hand side, Runge-Kutta integrators and relaxation (Sec. 3).
TEST INFRASTRUCTURE ONLY.

llg_rhs  : Eq. llg, dm/dt = -gamma/(1+alpha^2) [m x h + alpha m x (m x h)].
Problem  : one micromagnetic problem (grid, material, field terms); evaluates
           the effective field as the sum of demag (Sec. 4.4), exchange
           (Sec. 4.2), uniaxial anisotropy (Sec. 4.1) and Zeeman terms, as
           the solver of Sec. 5.1 sums [demag, aniso, exchange, external].
rk4_step : classic fourth-order Runge-Kutta (Sec. 3: explicit RK methods).
dp45_*   : Dormand-Prince 5(4) with first-same-as-last and an embedded
           fourth-order error estimate (the adaptive explicit RK family of
           Sec. 3).
rkf45_*  : Runge-Kutta-Fehlberg 4(5), the paper's default solver (Sec. 3):
           the fourth-order solution is propagated, the fifth-order one only
           controls the error.
relax    : integrate with the material's damping until the maximum torque is
           small (Sec. 3, ground state by integrating the LLG).

Readings where the paper is silent:
* m is renormalised to |m| = 1 after every (accepted) step (flag ``renorm``).
* DP45 error norm: err = max over cells and components of
  |y5 - y4| / (atol + rtol * max(|y_n|, |y5|)), atol = rtol; the step is
  accepted if err <= 1; dt <- dt * min(5, max(0.2, 0.9 err^(-1/5))).
* First-same-as-last: the last stage derivative k7 = f(y5), evaluated before
  renormalisation, is the first stage of the next step.
* Relaxation stops when max_i |y5_i x h(y5)_i| / Ms_i < tol, read from the
  field of that last stage (no extra field evaluation).
* RKF45 uses the same error norm with the propagated (fourth-order) solution
  in place of y5, the same accept rule and the same step-size factor; it has
  no first-same-as-last stage, so the torque that stops a relaxation is read
  from the first stage of the next step (the field at the new m).
* "Without the precession term" (Sec. 3, ground states): the m x h term of
  Eq. llg is dropped and the damping term keeps its factor
  gamma alpha / (1 + alpha^2).
"""
import numpy as np

from .constants import GAMMA
from .demag import demag_fft, magnetization, tensor_spectrum
from .fields import (anisotropy_field, dmi_field, exchange_field, linear_energy,
                     zeeman_energy, zeeman_field)
from .layers import exchange_field_layers, layered_demag_fft, layered_tensor
from .newell import demag_tensor


def llg_rhs(m, h, alpha, precession=True):
    """Eq. llg with the reduced gyromagnetic ratio gamma = 2.21e5 m/(A s);
    without the precession term the m x h summand is left out."""
    alpha = np.broadcast_to(np.asarray(alpha, dtype=np.float64), m.shape[:3])[..., None]
    mxh = np.cross(m, h)
    damp = alpha * np.cross(m, mxh)
    return -GAMMA / (1.0 + alpha * alpha) * ((mxh + damp) if precession else damp)


class Problem:
    """A micromagnetic problem on an n = (nx, ny, nz) grid of cells dx.

    Ms, A, Ku1, alpha: scalar or (nx, ny, nz); ku_axis: (3,) or (nx, ny, nz, 3);
    h_ext: (3,) in A/m or a callable t -> (3,); h_ext_weight: optional
    (nx, ny, nz) multiplier of the external field; p: Newell radius;
    layers: optional nz layer thicknesses (Sec. 4.4, non-equidistant layers,
    see ``oracle.layers``), which replace dx[2]; DMI is not defined there."""

    def __init__(self, n, dx, Ms, A, alpha, Ku1=0.0, ku_axis=(1.0, 0.0, 0.0),
                 h_ext=(0.0, 0.0, 0.0), h_ext_weight=None, p=20, demag=True, Nt=None, precession=True,
                 D=0.0, dmi="interface", layers=None):
        self.n = tuple(int(v) for v in n)
        self.dx = tuple(float(v) for v in dx)
        self.layers = None if layers is None else np.asarray(layers, dtype=np.float64)
        if self.layers is not None:
            if self.layers.shape != (self.n[2],) or np.any(self.layers <= 0):
                raise ValueError("one positive thickness per layer")
            if np.any(np.asarray(D) != 0):
                raise ValueError("DMI with non-equidistant layers is not defined")
            self.V = self.dx[0] * self.dx[1] * self.layers[None, None, :]
        else:
            self.V = self.dx[0] * self.dx[1] * self.dx[2]
        self.Ms = Ms
        self.A = A
        self.alpha = alpha
        self.Ku1 = Ku1
        self.ku_axis = ku_axis
        self.h_ext = h_ext
        self.h_ext_weight = h_ext_weight
        self.demag = demag
        self.precession = precession
        self.D = D
        self.dmi = dmi
        if demag and self.layers is not None:
            self.Nt = layered_tensor(self.n, self.dx[0], self.dx[1], self.layers, p) if Nt is None else Nt
        elif demag:
            self.Nt = demag_tensor(self.n, self.dx, p) if Nt is None else Nt
            self.Nhat = tensor_spectrum(self.Nt, self.n)

    def h_ext_at(self, t):
        return np.asarray(self.h_ext(t) if callable(self.h_ext) else self.h_ext, dtype=np.float64)

    def field_terms(self, m, t):
        terms = {}
        if self.demag and self.layers is not None:
            terms["demag"] = layered_demag_fft(self.Nt, magnetization(m, self.Ms))
        elif self.demag:
            terms["demag"] = demag_fft(self.Nt, magnetization(m, self.Ms), self.Nhat)
        else:
            terms["demag"] = np.zeros_like(m)
        if self.layers is not None:
            terms["exchange"] = exchange_field_layers(m, self.Ms, self.A, self.dx[0], self.dx[1], self.layers)
        else:
            terms["exchange"] = exchange_field(m, self.Ms, self.A, self.dx)
        terms["anisotropy"] = anisotropy_field(m, self.Ms, self.Ku1, self.ku_axis)
        terms["zeeman"] = zeeman_field(self.h_ext_at(t), self.n, self.h_ext_weight)
        terms["dmi"] = dmi_field(m, self.Ms, self.D, self.dx, self.dmi)
        # reading: a cell with Ms = 0 carries no field at all (the nan_to_num
        # of Sec. 4.1 extended to every term)
        ms = np.broadcast_to(np.asarray(self.Ms, dtype=np.float64), self.n)
        if np.any(ms == 0):
            for key in ("demag", "zeeman"):
                terms[key] = terms[key] * (ms != 0)[..., None]
        return terms

    def heff(self, m, t):
        terms = self.field_terms(m, t)
        return terms["demag"] + terms["exchange"] + terms["anisotropy"] + terms["zeeman"] + terms["dmi"]

    def energies(self, m, t):
        """(E_demag, E_exchange, E_anisotropy, E_zeeman, E_dmi) in J."""
        terms = self.field_terms(m, t)
        return (linear_energy(m, terms["demag"], self.Ms, self.V),
                linear_energy(m, terms["exchange"], self.Ms, self.V),
                linear_energy(m, terms["anisotropy"], self.Ms, self.V),
                zeeman_energy(m, terms["zeeman"], self.Ms, self.V),
                linear_energy(m, terms["dmi"], self.Ms, self.V))

    def rhs(self, m, t):
        return llg_rhs(m, self.heff(m, t), self.alpha, self.precession)

    def max_torque(self, m, h):
        """max_i |m_i x h_i| / Ms_i over cells with Ms_i != 0."""
        ms = np.broadcast_to(np.asarray(self.Ms, dtype=np.float64), self.n)
        tq = np.linalg.norm(np.cross(m, h), axis=-1)
        ok = ms != 0
        return float(np.max(tq[ok] / ms[ok])) if ok.any() else 0.0


def normalize(m):
    return m / np.linalg.norm(m, axis=-1, keepdims=True)


# classic RK4: nodes, stage coefficients, weights
RK4_C = (0.0, 0.5, 0.5, 1.0)
RK4_B = (1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0)


def rk4_step(prob, m, t, dt, renorm=True):
    """One classic RK4 step; returns m_{n+1}."""
    k1 = prob.rhs(m, t)
    k2 = prob.rhs(m + 0.5 * dt * k1, t + 0.5 * dt)
    k3 = prob.rhs(m + 0.5 * dt * k2, t + 0.5 * dt)
    k4 = prob.rhs(m + dt * k3, t + dt)
    out = m + dt * (RK4_B[0] * k1 + RK4_B[1] * k2 + RK4_B[2] * k3 + RK4_B[3] * k4)
    return normalize(out) if renorm else out


# Dormand-Prince 5(4) tableau (Dormand & Prince, J. Comput. Appl. Math. 6 (1980) 19)
DP_C = (0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0)
DP_A = (
    (),
    (1.0 / 5.0,),
    (3.0 / 40.0, 9.0 / 40.0),
    (44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0),
    (19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0),
    (9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0),
    (35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0),
)
DP_B5 = (35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0.0)
DP_B4 = (5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0, -92097.0 / 339200.0,
         187.0 / 2100.0, 1.0 / 40.0)


def dp45_attempt(prob, m, t, dt, k1, rtol, atol=None):
    """One Dormand-Prince attempt from (m, t) with step dt and first stage k1.

    Returns (y5, k7, h7, err): the fifth-order solution (not renormalised),
    its derivative, the effective field it was computed from, and the error
    norm of the embedded fourth-order estimate."""
    atol = rtol if atol is None else atol
    ks = [k1]
    h7 = None
    for s in range(1, 7):
        y = m.copy()
        for j, a in enumerate(DP_A[s]):
            if a != 0.0:
                y = y + dt * a * ks[j]
        h = prob.heff(y, t + DP_C[s] * dt)
        ks.append(llg_rhs(y, h, prob.alpha, prob.precession))
        if s == 6:
            y5, h7 = y, h
    e = np.zeros_like(m)
    for j in range(7):
        e = e + dt * (DP_B5[j] - DP_B4[j]) * ks[j]
    sc = atol + rtol * np.maximum(np.abs(m), np.abs(y5))
    err = float(np.max(np.abs(e) / sc))
    return y5, ks[6], h7, err


def dp45_factor(err):
    if err == 0.0:
        return 5.0
    return min(5.0, max(0.2, 0.9 * err ** (-0.2)))


def dp45_integrate(prob, m, t0, t1, dt0=1e-13, rtol=1e-5, atol=None, renorm=True,
                   max_steps=10**7, callback=None):
    """Integrate from t0 to t1 (last step clipped to land on t1).

    Returns (m, t, dt, accepted, rejected)."""
    t = t0
    dt = dt0
    k1 = prob.rhs(m, t)
    acc = rej = 0
    while t < t1 and acc < max_steps:
        h_try = min(dt, t1 - t)
        y5, k7, _, err = dp45_attempt(prob, m, t, h_try, k1, rtol, atol)
        if err <= 1.0:
            t = t + h_try
            m = normalize(y5) if renorm else y5
            k1 = k7
            acc += 1
            if callback is not None:
                callback(m, t)
        else:
            rej += 1
        dt = h_try * dp45_factor(err)
    return m, t, dt, acc, rej


# Runge-Kutta-Fehlberg 4(5) tableau (E. Fehlberg, NASA TR R-315, 1969)
RKF_C = (0.0, 1.0 / 4.0, 3.0 / 8.0, 12.0 / 13.0, 1.0, 1.0 / 2.0)
RKF_A = (
    (),
    (1.0 / 4.0,),
    (3.0 / 32.0, 9.0 / 32.0),
    (1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0),
    (439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0),
    (-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0),
)
RKF_B4 = (25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0.0)
RKF_B5 = (16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0)


def rkf45_attempt(prob, m, t, dt, k1, rtol, atol=None):
    """One Fehlberg attempt from (m, t) with step dt and first stage k1 = f(m, t).

    Returns (y4, err): the fourth-order solution (not renormalised) and the
    error norm of its difference to the fifth-order one."""
    atol = rtol if atol is None else atol
    ks = [k1]
    for s in range(1, 6):
        y = m.copy()
        for j, a in enumerate(RKF_A[s]):
            if a != 0.0:
                y = y + dt * a * ks[j]
        ks.append(prob.rhs(y, t + RKF_C[s] * dt))
    y4 = m.copy()
    e = np.zeros_like(m)
    for j in range(6):
        y4 = y4 + dt * RKF_B4[j] * ks[j]
        e = e + dt * (RKF_B5[j] - RKF_B4[j]) * ks[j]
    sc = atol + rtol * np.maximum(np.abs(m), np.abs(y4))
    return y4, float(np.max(np.abs(e) / sc))


def rkf45_step(prob, m, t, dt, rtol=1e-5, atol=None, renorm=True, k1=None):
    """Attempts from (m, t) until one is accepted (step-size factor as for
    DP45).  Returns (m_new, t_new, dt_next)."""
    if k1 is None:
        k1 = prob.rhs(m, t)
    while True:
        y4, err = rkf45_attempt(prob, m, t, dt, k1, rtol, atol)
        f = dp45_factor(err)
        if err <= 1.0:
            return (normalize(y4) if renorm else y4), t + dt, dt * f
        dt = dt * f


def relax(prob, m, tol=1e-3, max_steps=20000, dt0=1e-13, rtol=1e-5, atol=None, renorm=True, t0=0.0,
          method="dp45"):
    """Integrate with DP45 (or RKF45) until max |m x h| / Ms < tol (or
    max_steps accepted steps).  Returns (m, steps, max_torque, t)."""
    if method == "rkf45":
        t, dt, steps = t0, dt0, 0
        while True:
            h = prob.heff(m, t)
            tq = prob.max_torque(m, h)
            if tq < tol or steps >= max_steps:
                return m, steps, tq, t
            k1 = llg_rhs(m, h, prob.alpha, prob.precession)
            m, t, dt = rkf45_step(prob, m, t, dt, rtol, atol, renorm, k1)
            steps += 1
    t = t0
    dt = dt0
    h = prob.heff(m, t)
    k1 = llg_rhs(m, h, prob.alpha, prob.precession)
    tq = prob.max_torque(m, h)
    steps = 0
    while tq >= tol and steps < max_steps:
        y5, k7, h7, err = dp45_attempt(prob, m, t, dt, k1, rtol, atol)
        if err <= 1.0:
            t = t + dt
            tq = prob.max_torque(y5, h7)
            m = normalize(y5) if renorm else y5
            k1 = k7
            steps += 1
        dt = dt * dp45_factor(err)
    return m, steps, tq, t
