"""Gradients through amrfd steps: torch.autograd wrappers of the discrete adjoint.

AmrfdStep: forward = one SSPRK step (amrfd_step_batched on a copy of U),
backward = amrfd_adjoint (splitting speeds, GLM speed and psi damping held at
their forward values; the time step is a fixed input).
rollout: n steps with checkpoints every k steps; the backward pass recomputes
each segment's states from its checkpoint and runs the adjoints in reverse.
"""
import torch


class AmrfdStep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, dt, solver):
        ctx.solver = solver
        ctx.save_for_backward(U, dt)
        # step a buffer kept on the solver, so that repeated calls replay one captured graph
        buf = getattr(solver, "_step_buf", None)
        if buf is None or buf.shape != U.shape or buf.device != U.device:
            buf = solver._step_buf = torch.empty_like(U)
        buf.copy_(U.detach())
        solver.step_batched(buf, dt)
        return buf.clone()

    @staticmethod
    def backward(ctx, g):
        U, dt = ctx.saved_tensors
        gU = torch.empty_like(U)
        ctx.solver.adjoint(U.detach().contiguous(), dt, g.contiguous(), gU)
        return gU, None, None


def step(solver, U, dt):
    return AmrfdStep.apply(U, dt, solver)


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U0, dt, solver, nsteps, every):
        ctx.solver, ctx.nsteps, ctx.every = solver, nsteps, every
        U = U0.detach().clone()
        ckpts = []
        for n in range(nsteps):
            if n % every == 0:
                ckpts.append(U.clone())
            solver.step_batched(U, dt)
        ctx.ckpts = ckpts
        ctx.save_for_backward(dt)
        return U

    @staticmethod
    def backward(ctx, g):
        (dt,) = ctx.saved_tensors
        solver, nsteps, every = ctx.solver, ctx.nsteps, ctx.every
        g = g.contiguous().clone()
        gn = torch.empty_like(g)
        # the recomputation steps one work buffer (one captured graph, replayed) and keeps
        # a copy of every state of the segment for the reverse sweep
        states = [torch.empty_like(g) for _ in range(min(every, nsteps))]
        wb = getattr(solver, "_step_buf", None)
        if wb is None or wb.shape != g.shape or wb.device != g.device:
            wb = solver._step_buf = torch.empty_like(g)
        for seg in reversed(range(len(ctx.ckpts))):
            start = seg * every
            count = min(every, nsteps - start)
            wb.copy_(ctx.ckpts[seg])
            for j in range(count):
                states[j].copy_(wb)
                if j + 1 < count:
                    solver.step_batched(wb, dt)
            for j in reversed(range(count)):
                solver.adjoint(states[j], dt, g, gn)
                g, gn = gn, g
        return g, None, None, None, None


def rollout(solver, U0, dt, nsteps, every):
    """U after `nsteps` fixed-dt steps, differentiable w.r.t. U0 (checkpoint every `every` steps)."""
    return _Rollout.apply(U0, dt, solver, nsteps, every)


def checkpointed_rollout(solver, U0, dt, nsteps, k):
    """Alias of rollout: nsteps fixed-dt steps with checkpoints every k steps."""
    return rollout(solver, U0, dt, nsteps, k)
