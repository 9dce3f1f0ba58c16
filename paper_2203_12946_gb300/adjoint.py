"""Gradients of a rollout through the hand-written adjoint kernels.

``KineticEnergyRollout`` is a ``torch.autograd.Function``: its forward runs
``nsteps`` steps of the library from f = f^eq(rho0, u0) and returns the kinetic
energy L = 1/2 sum rho |u|^2 of the final state; its backward returns dL/du0
(and dL/drho0) by running ``elbm_adjoint_step`` backwards through the steps.

Memory: the forward keeps a checkpoint of the state every ``every`` steps
(default ceil(sqrt(nsteps))); the backward recomputes one segment at a time from
its checkpoint, keeping that segment's states, and runs the adjoint through it.
So about 2 sqrt(nsteps) states are held instead of nsteps, at the cost of one
extra forward pass.  Every step, forward or backward, runs in libelbm.so; torch
only holds the buffers.

With ``force`` (D values, float64) the rollout runs under that uniform body force
(``elbm_set_force``; not from the paper) and the backward also returns dL/dF, the
sum over the reverse sweep of each step's derivative with respect to F.

The step is differentiable away from the near-equilibrium cutoff and the
positivity clamp (both branches): use ``cutoff=False`` for gradient studies.
"""
from __future__ import annotations

import math

import torch

from . import elbm as E


class KineticEnergyRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, rho0, force, sim: E.Simulation, nsteps: int, every: int = 0):
        if u0.device != sim.device or u0.dtype != torch.float64:
            raise ValueError("u0 must be a float64 tensor on the simulation's device")
        every = every or max(1, math.ceil(math.sqrt(nsteps)))
        u0c = u0.detach().contiguous()
        r0c = None if rho0 is None else rho0.detach().to(sim.device, torch.float64).contiguous()
        Fh = None if force is None else force.detach().to("cpu", torch.float64).numpy().copy()
        sim.set_force(Fh)
        sim.init_equilibrium(r0c, u0c)
        ckpts = {0: sim.state_copy()}
        for t in range(nsteps):
            sim.step(1)
            if (t + 1) % every == 0 and t + 1 < nsteps:
                ckpts[t + 1] = sim.state_copy()
        L = sim.kinetic_energy()
        ctx.sim, ctx.nsteps, ctx.every, ctx.ckpts = sim, nsteps, every, ckpts
        ctx.u0, ctx.rho0, ctx.Fh, ctx.force_like = u0c, r0c, Fh, force
        ctx.final = sim.state_copy()
        return torch.tensor(L, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gL):
        sim = ctx.sim
        sim.set_force(ctx.Fh)
        want_F = ctx.force_like is not None and ctx.needs_input_grad[2]
        dF = torch.zeros(sim.D, dtype=torch.float64, device=sim.device) if want_F else None
        _, g = sim.kinetic_energy(ctx.final, with_grad=True)
        g = g * float(gL)
        starts = sorted(ctx.ckpts)
        for s in reversed(starts):
            e = min(s + ctx.every, ctx.nsteps)
            sim.restore(ctx.ckpts[s])
            states = [ctx.ckpts[s]]
            for _ in range(s + 1, e):
                sim.step(1)
                states.append(sim.state_copy())
            for t in range(e - 1, s - 1, -1):
                g = sim.adjoint_step(states[t - s], g, dforce=dF)
        drho, du = sim.equilibrium_vjp(ctx.rho0, ctx.u0, g)
        sim.restore(ctx.final)
        gF = dF.to(ctx.force_like.device, ctx.force_like.dtype) if want_F else None
        return du, (drho if ctx.rho0 is not None else None), gF, None, None, None


def kinetic_energy_rollout(u0, sim: E.Simulation, nsteps: int, rho0=None, every: int = 0, force=None):
    """L(u0, F) = kinetic energy after nsteps steps from f^eq(rho0, u0) under the uniform
    body force F (None: no force); differentiable in u0 and in F."""
    return KineticEnergyRollout.apply(u0, rho0, force, sim, nsteps, every)
