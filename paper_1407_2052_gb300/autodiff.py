"""Gradients through amrfd steps: torch.autograd wrappers of the discrete adjoint.

AmrfdStep: forward = one SSPRK step (amrfd_step_batched on a copy of U),
backward = amrfd_adjoint (splitting speeds, GLM speed and psi damping held at
their forward values; the time step is a fixed input).
rollout: n steps with checkpoints every k steps; the backward pass recomputes
each segment's states from its checkpoint, recording every step (amrfd_step_record),
and runs the recorded adjoints in reverse (amrfd_adjoint_recorded).
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
    def forward(ctx, U0, dt, solver, nsteps, every, stats):
        ctx.solver, ctx.nsteps, ctx.every, ctx.stats = solver, nsteps, every, stats
        ev = _events(stats, 2)
        if ev:
            ev[0].record()
        U = U0.detach().clone()
        ckpts = []
        for n in range(nsteps):
            if n % every == 0:
                ckpts.append(U.clone())
            solver.step_batched(U, dt)
        if ev:
            ev[1].record()
            ctx.fwd_events = ev
        ctx.ckpts = ckpts
        ctx.save_for_backward(dt)
        return U

    @staticmethod
    def backward(ctx, g):
        (dt,) = ctx.saved_tensors
        solver, nsteps, every, stats = ctx.solver, ctx.nsteps, ctx.every, ctx.stats
        g = g.contiguous().clone()
        gn = torch.empty_like(g)
        # the recomputation steps one work buffer and keeps every state of the segment and
        # every step's record (stage states, limiter pieces, speeds), so that the reverse
        # sweep needs no second forward pass per step
        m = min(every, nsteps)
        states = [torch.empty_like(g) for _ in range(m)]
        records = [solver.new_record() for _ in range(m)]
        wb = getattr(solver, "_step_buf", None)
        if wb is None or wb.shape != g.shape or wb.device != g.device:
            wb = solver._step_buf = torch.empty_like(g)
        ev = _events(stats, 3 * len(ctx.ckpts))
        for i, seg in enumerate(reversed(range(len(ctx.ckpts)))):
            if ev:
                ev[3 * i].record()
            start = seg * every
            count = min(every, nsteps - start)
            wb.copy_(ctx.ckpts[seg])
            for j in range(count):
                states[j].copy_(wb)
                solver.step_record(wb, dt, records[j])
            if ev:
                ev[3 * i + 1].record()
            for j in reversed(range(count)):
                solver.adjoint_recorded(states[j], dt, records[j], g, gn)
                g, gn = gn, g
            if ev:
                ev[3 * i + 2].record()
        if ev:
            ev[-1].synchronize()
            f0, f1 = ctx.fwd_events
            stats["forward_ms"] = stats.get("forward_ms", 0.0) + f0.elapsed_time(f1)
            stats["recompute_ms"] = stats.get("recompute_ms", 0.0) + sum(
                ev[3 * i].elapsed_time(ev[3 * i + 1]) for i in range(len(ctx.ckpts)))
            stats["adjoint_ms"] = stats.get("adjoint_ms", 0.0) + sum(
                ev[3 * i + 1].elapsed_time(ev[3 * i + 2]) for i in range(len(ctx.ckpts)))
            stats["backward_ms"] = stats.get("backward_ms", 0.0) + ev[0].elapsed_time(ev[-1])
        return g, None, None, None, None, None


def _events(stats, n):
    if stats is None:
        return None
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def rollout(solver, U0, dt, nsteps, every, stats=None):
    """U after `nsteps` fixed-dt steps, differentiable w.r.t. U0 (checkpoint every `every` steps).
    With a dict `stats`, the device time of the forward run, of the backward pass's
    recomputation and of its adjoint steps is added to it (milliseconds, CUDA events on the
    current stream; the backward pass then waits for its last event)."""
    return _Rollout.apply(U0, dt, solver, nsteps, every, stats)


def checkpointed_rollout(solver, U0, dt, nsteps, k, stats=None):
    """Alias of rollout: nsteps fixed-dt steps with checkpoints every k steps."""
    return rollout(solver, U0, dt, nsteps, k, stats)
