"""Gradients of RK4 rollouts through the hand-written adjoint (mm_llg_step_adjoint).

``rk4_observable(Ms_cell, state, m0, weight, dt, steps, every, material)``
returns the series o_n = <weight, m_n>, n = 1..steps, of an RK4 rollout with
per-cell saturation magnetisation ``Ms_cell``; it is a torch.autograd.Function,
so any loss built from the series back-propagates to ``Ms_cell`` (and from
there, e.g., through Ms = sigmoid(w) Ms0 of the inverse-design example of
Sec. 5.2).  The forward pass keeps m only every ``every`` steps; the backward
pass recomputes each segment from its checkpoint and sweeps the adjoint of
every step backwards through it (memory ~ steps/every + every states).
"""
import torch


class RK4Observable(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Ms_cell, state, m0, weight, dt, steps, every, material, t0):
        state.set_material(Ms=0.0, Ms_cell=Ms_cell.detach().to(torch.float64).contiguous(), **material)
        state.set_m(m0)
        ckpt = {0: m0.detach().clone()}
        obs = torch.empty(steps, dtype=torch.float64, device=m0.device)
        t = t0
        for n in range(steps):
            t, _ = state.step(dt, t, "rk4")
            mn = state.get_m()
            obs[n] = (weight * mn).sum(dtype=torch.float64)
            if (n + 1) % every == 0 and n + 1 < steps:
                ckpt[n + 1] = mn
        ctx.state, ctx.weight, ctx.dt, ctx.steps, ctx.every, ctx.t0 = state, weight, dt, steps, every, t0
        ctx.ckpt = ckpt
        ctx.ms_shape = Ms_cell.shape
        ctx.ms_dtype = Ms_cell.dtype
        return obs

    @staticmethod
    def backward(ctx, gobs):
        s, w, dt, steps, every, t0 = ctx.state, ctx.weight, ctx.dt, ctx.steps, ctx.every, ctx.t0
        gMs = torch.zeros(ctx.ms_shape, dtype=s.dtype, device=w.device)
        lam = (gobs[steps - 1] * w).to(s.dtype)
        for c in reversed(range(0, steps, every)):
            end = min(c + every, steps)
            states = [ctx.ckpt[c]]
            s.set_m(ctx.ckpt[c])
            t = t0 + c * dt
            for n in range(c, end - 1):
                t, _ = s.step(dt, t, "rk4")
                states.append(s.get_m())
            for n in range(end - 1, c - 1, -1):
                lam = s.step_adjoint(states[n - c], lam, dt, t0 + n * dt, grad_Ms=gMs)
                if n >= 1:
                    lam = lam + (gobs[n - 1] * w).to(s.dtype)
        return gMs.to(ctx.ms_dtype), None, None, None, None, None, None, None, None


def rk4_observable(Ms_cell, state, m0, weight, dt, steps, every=100, material=None, t0=0.0):
    return RK4Observable.apply(Ms_cell, state, m0, weight, dt, steps, every, material or {}, t0)
