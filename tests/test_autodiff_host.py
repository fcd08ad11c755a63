"""Host logic of the checkpointed rollout and the single-step autograd function (CPU): a
stand-in solver with the library's call pattern (step_batched, new_record, step_record,
adjoint_recorded, adjoint) whose step is U_i <- U_i + dt sin(U_{i-1}) (periodic) and whose
adjoint is g_k <- g_k + dt cos(U_k) g_{k+1}: the steps' Jacobians do not commute, so an
adjoint applied out of order changes the gradient. Its records hold the state the step
started from, and its recorded adjoint checks that the record and the state it is given
belong together, so a mis-paired checkpoint, state or record fails; the gradients are
compared with torch's autograd of the same map."""
import pytest

torch = pytest.importorskip("torch")

from paper_1407_2052_gb300 import autodiff  # noqa: E402


class _Rec:
    def __init__(self):
        self.u = None


class FakeSolver:
    def __init__(self):
        self.steps = 0
        self.adjoints = 0

    def step_batched(self, U, dt):
        U.add_(dt * torch.sin(torch.roll(U, 1)))
        self.steps += 1

    def new_record(self):
        return _Rec()

    def step_record(self, U, dt, rec):
        rec.u = U.clone()
        self.step_batched(U, dt)

    def adjoint_recorded(self, U_n, dt, rec, g, gn):
        assert rec.u is not None and torch.equal(rec.u, U_n), "record and state do not belong together"
        self.adjoint(U_n, dt, g, gn)

    def adjoint(self, U_n, dt, g, gn):
        gn.copy_(g + dt * torch.cos(U_n) * torch.roll(g, -1))
        self.adjoints += 1


def _reference(U0, dt, n, w):
    U = U0.clone().requires_grad_(True)
    V = U
    for _ in range(n):
        V = V + dt * torch.sin(torch.roll(V, 1))
    (V * w).sum().backward()
    return V.detach(), U.grad


@pytest.mark.parametrize("nsteps,every", [(1, 1), (7, 3), (8, 4), (5, 10), (12, 1), (9, 9)])
def test_rollout_matches_autograd_of_the_step(nsteps, every):
    gen = torch.Generator().manual_seed(nsteps * 31 + every)
    U0 = torch.randn(64, dtype=torch.float64, generator=gen)
    w = torch.randn(64, dtype=torch.float64, generator=gen)
    dt = torch.full((1,), 0.1, dtype=torch.float64)
    s = FakeSolver()
    U = U0.clone().requires_grad_(True)
    out = autodiff.rollout(s, U, dt, nsteps, every)
    (out * w).sum().backward()
    Vr, gr = _reference(U0, dt, nsteps, w)
    assert torch.equal(out.detach(), Vr)
    assert torch.allclose(U.grad, gr, rtol=1e-13, atol=1e-15)
    # forward run + one recomputation of every step; one recorded adjoint per step
    assert s.steps == 2 * nsteps and s.adjoints == nsteps


def test_single_step_function():
    gen = torch.Generator().manual_seed(5)
    U0 = torch.randn(32, dtype=torch.float64, generator=gen)
    w = torch.randn(32, dtype=torch.float64, generator=gen)
    dt = torch.full((1,), 0.05, dtype=torch.float64)
    s = FakeSolver()
    U = U0.clone().requires_grad_(True)
    out = autodiff.step(s, U, dt)
    out2 = autodiff.step(s, out, dt)
    (out2 * w).sum().backward()
    Vr, gr = _reference(U0, dt, 2, w)
    assert torch.equal(out2.detach(), Vr) and torch.equal(U0, U.detach())
    assert torch.allclose(U.grad, gr, rtol=1e-13, atol=1e-15)
