"""Differentiation form of the time step: gradient of the final perturbation kinetic energy
with respect to the initial state, by the hand-written adjoint of libtc (tc_adjoint_step,
tc_adjoint_start) behind a torch.autograd.Function, with checkpointing.

Forward: the cold state u0 gets its AB2BD2 history (tc_step with nsteps = 0) and is
advanced n steps; the state (u, u_prev, N_prev) is kept every `checkpoint` steps.
Backward: each segment between checkpoints is recomputed forward from its checkpoint, the
velocity u of each of its steps kept (the only field an adjoint step reads), and the adjoint
steps run backwards through it; the cold start is then differentiated by tc_adjoint_start.

`state_gradient` differentiates a run from a started state with respect to that state, with
its checkpoints in pinned host memory and a bounded number of device copies of u, for
workloads whose states do not fit the device several times over.  All arithmetic runs in
libtc's kernels; torch supplies device and host memory only.
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


class _ForwardU:
    """The forward state an adjoint step reads: u^i only (tc_adjoint_step reads no other
    field of it)."""

    def __init__(self, u):
        self.u = u

    def c_struct(self):
        return tc.tc_state(self.u.data_ptr(), None, None, None, 1)


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
        ctx.plan, ctx.nsteps, ctx.ckpts = plan, nsteps, ckpts
        ctx.save_for_backward(u0.detach(), st.u.clone())
        return torch.tensor(_energy(plan, st.u), dtype=torch.float64, device=u0.device)

    @staticmethod
    def backward(ctx, gJ):
        plan, n, ckpts = ctx.plan, ctx.nsteps, ctx.ckpts
        u0, uN = ctx.saved_tensors
        ub = plan.energy_gradient(uN) * gJ.to(torch.float64)
        bar = tc.StateBar(ub.contiguous(), torch.zeros_like(ub), torch.zeros_like(ub))
        starts = sorted(ckpts)
        for s0 in reversed(starts):
            seg_end = min([s for s in starts if s > s0] + [n])
            st = _clone_state(plan, ckpts[s0])
            us = [st.u.clone()]
            for _ in range(s0, seg_end - 1):
                plan.step(st, 1)
                us.append(st.u.clone())
            for u in reversed(us):
                plan.adjoint_step(_ForwardU(u), bar)
        g = plan.adjoint_start(u0, bar)
        return g, None, None, None


def final_energy(u0, plan, nsteps, checkpoint=20):
    """Differentiable J(u0); u0 is a complex128 CUDA tensor of the plan's vector shape."""
    return FinalEnergy.apply(u0, plan, nsteps, checkpoint)


def _host_bytes_available():
    """MemAvailable of this machine in bytes (None where /proc/meminfo is absent)."""
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        return None
    return None


def state_gradient(plan, st, nsteps, checkpoint=10, slots=None, spill=True, host_fraction=0.6):
    """Gradient of the final perturbation energy J after `nsteps` steps from the started
    state st with respect to that state's (u, u_prev, N_prev), by the hand-written adjoint.

    Forward: st is advanced `nsteps` steps; its (u, u_prev, N_prev) is kept every
    `checkpoint` steps, in pinned host memory when `spill` (else on the device).  Backward:
    the segments between checkpoints are reversed last first.  A segment is recomputed from
    its checkpoint with st as the working state, the velocity of its last `slots` steps not
    yet reversed is copied into device buffers, and the adjoint steps run back through them;
    this repeats until the segment is reversed (`slots` = None: the whole segment at once).
    Only u is read by an adjoint step, so a slot holds one vector field.

    st is the working state: on return it holds its initial (u, u_prev, N_prev) again; p is
    left as the last recomputed step wrote it.  Refuses (ValueError) host checkpoints that
    would take more than `host_fraction` of the machine's available memory.
    Returns (J, bar), bar a tc.StateBar of the three gradients."""
    if not st.started:
        raise ValueError("state_gradient needs a started state (tc_step has built its history)")
    C = int(checkpoint)
    if C < 1 or nsteps < 1:
        raise ValueError("checkpoint and nsteps must be >= 1")
    starts = list(range(0, nsteps, C))
    k = C if slots is None else max(1, min(int(slots), C))
    field_bytes = st.u.numel() * st.u.element_size()
    if spill:
        need = len(starts) * 3 * field_bytes
        avail = _host_bytes_available()
        if avail is not None and need > host_fraction * avail:
            raise ValueError(f"host checkpoints need {need / 1e9:.1f} GB, more than "
                             f"{host_fraction:.0%} of the {avail / 1e9:.1f} GB available")

    def save():
        if spill:
            out = []
            for t in (st.u, st.u_prev, st.N_prev):
                h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
                h.copy_(t, non_blocking=True)
                out.append(h)
            return out
        return [st.u.clone(), st.u_prev.clone(), st.N_prev.clone()]

    def restore(c):
        for t, h in zip((st.u, st.u_prev, st.N_prev), c):
            t.copy_(h, non_blocking=True)
        st.started = True

    ckpts = {}
    for i in range(nsteps):
        if i % C == 0:
            ckpts[i] = save()
        plan.step(st, 1)
    J = _energy(plan, st.u)
    ub = plan.energy_gradient(st.u)
    bar = tc.StateBar(ub.contiguous(), torch.zeros_like(ub), torch.zeros_like(ub))
    buf = [torch.empty_like(st.u) for _ in range(k)]
    for s0 in reversed(starts):
        hi = min(s0 + C, nsteps)          # forward states s0 .. hi-1 still to reverse
        while hi > s0:
            lo = max(s0, hi - k)
            restore(ckpts[s0])
            for j in range(s0, hi):       # st holds the state of step j
                if j >= lo:
                    buf[j - lo].copy_(st.u)
                if j < hi - 1:
                    plan.step(st, 1)
            for j in reversed(range(lo, hi)):
                plan.adjoint_step(_ForwardU(buf[j - lo]), bar)
            hi = lo
        if s0 > 0:
            del ckpts[s0]
    restore(ckpts[0])
    if spill:
        torch.cuda.current_stream().synchronize()   # the pinned checkpoints are released after the copies
    del ckpts
    return J, bar


def energy_weights(plan, like):
    """W with J(u) = 1/2 sum W |u - U|^2 over the stored coefficients, so that dJ/du = W (u - U):
    taken from the library's gradient kernel as W = g(u + 1) - g(u)."""
    z = torch.zeros_like(like)
    return (plan.energy_gradient(z + 1) - plan.energy_gradient(z)).real.contiguous()


def _real_field_m0(d):
    """Project the m = 0 line onto the symmetry of a real field: d_+(0,k) = conj d_-(0,-k),
    d_z(0,k) = conj d_z(0,-k)."""
    line = d[:, :, 0, :]
    p, m, z = line[0], line[1], line[2]
    pm = 0.5 * (p + torch.conj(torch.flip(m, dims=[-1])))
    zz = 0.5 * (z + torch.conj(torch.flip(z, dims=[-1])))
    d = d.clone()
    d[0, :, 0, :] = pm
    d[1, :, 0, :] = torch.conj(torch.flip(pm, dims=[-1]))
    d[2, :, 0, :] = zz
    return d


def _grad_and_value(u, plan, nsteps, checkpoint):
    x = u.detach().clone().requires_grad_(True)
    J = final_energy(x, plan, nsteps, checkpoint)
    J.backward()
    return float(J.detach()), x.grad.detach()


def optimal_perturbation(plan, u_base, nsteps, delta0, energy=1e-6, iters=10, checkpoint=20):
    """Largest energy gain over nsteps steps of a perturbation of the state u_base, and the
    perturbation that attains it (the optimal initial perturbation from which transition
    studies start), by power iteration in the energy inner product of tc_diag:

        delta <- W^{-1} (dJ(u_base + delta) - dJ(u_base)),  rescaled to E(delta) = energy,

    with the gradients from the hand-written adjoint (final_energy), the wall rows held at
    zero and the m = 0 line kept that of a real field.  For small `energy` the iteration
    converges to the leading right singular vector of the step map's linearisation about
    u_base in the energy norm.  The gain of each iterate is the second-order part of J,
    (J(u_base + delta) - J(u_base) - <dJ(u_base), delta>) / E(delta), which is insensitive to
    a slow drift of the base state itself.  Returns (delta, gains)."""
    W = energy_weights(plan, u_base)

    def E(d):
        return 0.5 * float((W * d.abs() ** 2).sum())

    def admissible(d):
        d = _real_field_m0(d)
        d[:, 0] = 0
        d[:, -1] = 0
        return d

    J0, g0 = _grad_and_value(u_base, plan, nsteps, checkpoint)
    d = admissible(delta0.to(u_base.device, torch.complex128))
    gains = []
    for _ in range(iters):
        d = d * (energy / E(d)) ** 0.5
        J, g = _grad_and_value(u_base + d, plan, nsteps, checkpoint)
        lin = float(torch.sum(torch.view_as_real(g0) * torch.view_as_real(d)))
        gains.append((J - J0 - lin) / energy)
        d = admissible((g - g0) / W)
    return d * (energy / E(d)) ** 0.5, gains
