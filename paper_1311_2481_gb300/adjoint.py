"""Differentiation form of the time step: gradient of the final perturbation kinetic energy
with respect to the initial state, by the hand-written adjoint of libtc (tc_adjoint_step,
tc_adjoint_start) behind a torch.autograd.Function, with checkpointing.

Forward: the cold state u0 gets its AB2BD2 history (tc_step with nsteps = 0) and is
advanced n steps; the state (u, u_prev, N_prev) is kept every `checkpoint` steps.
Backward: each segment between checkpoints is recomputed forward from its checkpoint, its
states kept, and the adjoint steps run backwards through it; the cold start is then
differentiated by tc_adjoint_start.  All arithmetic runs in libtc's kernels; torch supplies
device memory only.
"""
from __future__ import annotations

import torch

from . import tc


def _clone_state(plan, st):
    c = tc.State.__new__(tc.State)
    c.u, c.u_prev, c.N_prev, c.p = st.u.clone(), st.u_prev.clone(), st.N_prev.clone(), st.p.clone()
    c.started = st.started
    return c


def _energy(plan, u):
    return plan.diagnostics(u).energy


class FinalEnergy(torch.autograd.Function):
    """J(u0) = perturbation energy after nsteps steps from the cold state u0."""

    @staticmethod
    def forward(ctx, u0, plan, nsteps, checkpoint):
        st = tc.State(plan, u0.detach())
        plan.step(st, 0)                                   # history of the cold state
        ckpts = {0: _clone_state(plan, st)}
        for i in range(nsteps):
            plan.step(st, 1)
            if (i + 1) % checkpoint == 0 and i + 1 < nsteps:
                ckpts[i + 1] = _clone_state(plan, st)
        ctx.plan, ctx.nsteps, ctx.checkpoint, ctx.ckpts = plan, nsteps, checkpoint, ckpts
        ctx.save_for_backward(u0.detach(), st.u.clone())
        return torch.tensor(_energy(plan, st.u), dtype=torch.float64, device=u0.device)

    @staticmethod
    def backward(ctx, gJ):
        plan, n, C, ckpts = ctx.plan, ctx.nsteps, ctx.checkpoint, ctx.ckpts
        u0, uN = ctx.saved_tensors
        ub = plan.energy_gradient(uN) * gJ.to(torch.float64)
        bar = tc.StateBar(ub.contiguous(), torch.zeros_like(ub), torch.zeros_like(ub))
        starts = sorted(ckpts)
        for s0 in reversed(starts):
            s1 = min(s0 + C, n) if s0 + C <= n else n
            seg_end = min([s for s in starts if s > s0] + [n])
            st = _clone_state(plan, ckpts[s0])
            states = [_clone_state(plan, st)]
            for _ in range(s0, seg_end - 1):
                plan.step(st, 1)
                states.append(_clone_state(plan, st))
            for fwd in reversed(states):
                plan.adjoint_step(fwd, bar)
            del s1
        g = plan.adjoint_start(u0, bar)
        return g, None, None, None


def final_energy(u0, plan, nsteps, checkpoint=20):
    """Differentiable J(u0); u0 is a complex128 CUDA tensor of the plan's vector shape."""
    return FinalEnergy.apply(u0, plan, nsteps, checkpoint)
