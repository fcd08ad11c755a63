"""Discrete adjoint (amrfd_adjoint) against independent derivatives.

The forward map being transposed is one SSPRK step with the splitting speeds of
every stage, the GLM speed and the psi damping factor held at their forward
values (and a fixed dt). References:
  * autograd of tests/torchref.py (plain FP64 PyTorch ops, CPU) with the speeds
    the oracle's step used, relative max error <= 1e-10;
  * central finite differences of the oracle's frozen-speed step along random
    directions (h = 1e-6), relative error <= 1e-6;
  * the checkpointed multi-step rollout equals the chain of single-step adjoints.
"""
import numpy as np
import pytest

import oracle as O
from paper_1407_2052_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()


def _A():
    from paper_1407_2052_gb300 import amrfd
    return amrfd


def _torchref():
    import os
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    import torchref
    return torchref


def _odom(d):
    return O.dom(d.n, d.dx, bc=[list(b) for b in d.bc], nb=d.nb, asym=d.asym)


def _gpu_adjoint(w, dt, g):
    A = _A()
    s = A.Solver.from_workload(w)
    U = torch.from_numpy(np.ascontiguousarray(w.U.ravel())).cuda()
    dtt = torch.full((s.ndom,), dt, dtype=torch.float64, device="cuda")
    gg = torch.from_numpy(np.ascontiguousarray(g.ravel())).cuda()
    out = torch.empty_like(U)
    s.adjoint(U, dtt, gg, out)
    assert s.error() == A.OK
    return out.cpu().numpy().reshape(w.U.shape), s


def _ref_grad(w, dt, g):
    T = _torchref()
    c = O.cfg(w.physics, w.ndim, w.integrator, w.gamma, w.glm_cr, recon=w.recon, limo3_r=w.limo3_r)
    _, fl, al, ch = O.step(c, _odom(w.domains[0]), w.U, dt)
    U = torch.from_numpy(w.U.copy()).requires_grad_(True)
    out = T.step(U, dt, w.domains[0].dx, w.domains[0].bc, w.physics, w.ndim, w.gamma, w.integrator, al, ch,
                 w.glm_cr, asym=w.domains[0].asym, recon=w.recon, limo3_r=w.limo3_r)
    (out * torch.from_numpy(g)).sum().backward()
    return U.grad.numpy(), al, ch


def _smooth(physics, ndim, n, bc, seed, integrator, asym=((0, 0),) * 3, nb=(1, 1, 1)):
    rng = np.random.default_rng(seed)
    g = 1.4 if physics == O.EULER else 5 / 3
    dx = [1.0 / n[0], 1.0 / max(n[1], 1), 1.0 / max(n[2], 1)]
    axes = [(np.arange(m) + 0.5) / m for m in n]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")

    def f(a):
        k = rng.integers(1, 3, 3) * np.array([1, ndim > 1, ndim > 2])
        return a * np.sin(2 * np.pi * (k[0] * X + k[1] * Y + k[2] * Z) + rng.uniform(0, 6.28))
    rho, p = 1.0 + f(0.2), 1.0 + f(0.2)
    vel = [f(0.3) + 0.1 for _ in range(3)]
    if physics == O.EULER:
        U = W.conserved_euler(rho, vel[:ndim], p, g)
    else:
        U = W.conserved_mhd(rho, vel, p, [0.5 + f(0.1), 0.2 + f(0.1), 0.1 + f(0.1)], g, psi=f(0.01))
    dom = W.Domain(tuple(n), tuple(dx), bc=bc, asym=asym, nb=nb)
    return W.Workload("smooth", physics, ndim, integrator, g, 0.4, [dom], U,
                      active=np.ones(nb[0] * nb[1] * nb[2], np.uint8))


CASES = [
    ("mhd2d_ssprk3", lambda: W.adjoint2d(32), 1e-3),
    ("mhd2d_ssprk54", lambda: W.Workload(**{**W.adjoint2d(32).__dict__, "integrator": O.SSPRK54}), 1e-3),
    ("euler1d_outflow", lambda: _smooth(O.EULER, 1, (40, 1, 1), ((1, 1), (0, 0), (0, 0)), 1, O.SSPRK3), 2e-3),
    ("euler2d_mixed", lambda: _smooth(O.EULER, 2, (24, 20, 1), ((1, 1), (0, 0), (0, 0)), 2, O.SSPRK54), 2e-3),
    ("mhd3d_mixed", lambda: _smooth(O.MHD_GLM, 3, (12, 10, 8), ((0, 0), (1, 1), (0, 0)), 3, O.SSPRK3), 1e-3),
    ("euler3d_ssprk43", lambda: _smooth(O.EULER, 3, (10, 8, 12), ((0, 0), (0, 0), (1, 1)), 4, O.SSPRK43), 2e-3),
    # mirror faces: a closed 1D tube, MHD walls normal to y, and mixed mirror / outflow
    # faces with a no-slip mask on 3 x 2 blocks
    ("euler1d_walls", lambda: _smooth(O.EULER, 1, (40, 1, 1), ((2, 2), (0, 0), (0, 0)), 5, O.SSPRK3,
                                      asym=((2, 2), (0, 0), (0, 0))), 2e-3),
    ("mhd2d_wall_y", lambda: _smooth(O.MHD_GLM, 2, (24, 20, 1), ((0, 0), (2, 2), (0, 0)), 6, O.SSPRK54,
                                     asym=((0, 0), (W.MHD_WALL_Y, W.MHD_WALL_Y), (0, 0))), 1e-3),
    ("euler2d_mirror_outflow_blocks", lambda: _smooth(O.EULER, 2, (36, 16, 1), ((2, 1), (2, 2), (0, 0)), 7,
                                                      O.SSPRK3, asym=((6, 0), (6, 6), (0, 0)), nb=(3, 2, 1)),
     2e-3),
]


@pytest.mark.parametrize("name,make,dt", CASES, ids=[c[0] for c in CASES])
def test_adjoint_matches_autograd_of_torch_reference(name, make, dt):
    w = make()
    g = np.random.default_rng(7).standard_normal(w.U.shape)
    got, _ = _gpu_adjoint(w, dt, g)
    want, _, _ = _ref_grad(w, dt, g)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err <= 1e-10, err


FD_CASES = [
    # well resolved (>= 32 cells per wavelength): the limiter stays on one linear piece
    # under the perturbation; at 32^2 the same data sits on MP5 kinks near extrema
    ("mhd2d_128", lambda: W.adjoint2d(128), 1e-3),
    CASES[4],
]


@pytest.mark.parametrize("name,make,dt", FD_CASES, ids=[c[0] for c in FD_CASES])
def test_adjoint_against_oracle_central_differences(name, make, dt):
    w = make()
    rng = np.random.default_rng(11)
    g = rng.standard_normal(w.U.shape)
    got, _ = _gpu_adjoint(w, dt, g)
    c = O.cfg(w.physics, w.ndim, w.integrator, w.gamma, w.glm_cr)
    d = _odom(w.domains[0])
    _, _, al, ch = O.step(c, d, w.U, dt)
    h = 1e-6
    for _ in range(5):
        v = rng.standard_normal(w.U.shape)
        v /= np.linalg.norm(v)
        up, _ = O.step_frozen(c, d, w.U + h * v, dt, al, ch)
        um, _ = O.step_frozen(c, d, w.U - h * v, dt, al, ch)
        fd = float(np.sum(g * (up - um)) / (2 * h))
        ad = float(np.sum(got * v))
        assert abs(fd - ad) <= 1e-6 * max(abs(fd), 1e-12), (fd, ad)


def test_checkpointed_rollout_equals_chained_adjoints():
    from paper_1407_2052_gb300 import autodiff
    A = _A()
    w = W.adjoint2d(48)
    s = A.Solver.from_workload(w)
    U0 = torch.from_numpy(w.U.ravel().copy()).cuda()
    dt = torch.full((1,), 1e-3, dtype=torch.float64, device="cuda")
    nsteps, every = 12, 5
    U0r = U0.clone().requires_grad_(True)
    Uf = autodiff.rollout(s, U0r, dt, nsteps, every)
    B = Uf.view(9, -1)[5:8]
    J = 0.5 * (B * B).sum() * w.domains[0].dx[0] * w.domains[0].dx[1]
    J.backward()
    grad = U0r.grad.clone()
    # chain of single-step adjoints over stored states
    states = [U0.clone()]
    for _ in range(nsteps):
        nxt = states[-1].clone()
        s.step_batched(nxt, dt)
        states.append(nxt)
    assert torch.equal(states[-1], Uf.detach())
    gB = torch.zeros_like(U0).view(9, -1)
    gB[5:8] = states[-1].view(9, -1)[5:8] * (w.domains[0].dx[0] * w.domains[0].dx[1])
    g = gB.view(-1).clone()
    out = torch.empty_like(g)
    for j in reversed(range(nsteps)):
        s.adjoint(states[j], dt, g, out)
        g, out = out, g
    assert torch.equal(g, grad)


def test_rollout_matches_torch_reference_over_steps():
    """Three steps at 24^2: GPU rollout gradient vs autograd through three torchref steps,
    each with the speeds of the oracle's trajectory."""
    from paper_1407_2052_gb300 import autodiff
    A = _A()
    T = _torchref()
    w = W.adjoint2d(24)
    dtv, nsteps = 1e-3, 3
    s = A.Solver.from_workload(w)
    U0 = torch.from_numpy(w.U.ravel().copy()).cuda().requires_grad_(True)
    dt = torch.full((1,), dtv, dtype=torch.float64, device="cuda")
    Uf = autodiff.rollout(s, U0, dt, nsteps, 2)
    g = torch.from_numpy(np.random.default_rng(3).standard_normal(w.U.size)).cuda()
    (Uf * g).sum().backward()
    c = O.cfg(w.physics, w.ndim, w.integrator, w.gamma, w.glm_cr)
    d = _odom(w.domains[0])
    Ut = torch.from_numpy(w.U.copy()).requires_grad_(True)
    Uc, Un = Ut, w.U.copy()
    for _ in range(nsteps):
        Un, _, al, ch = O.step(c, d, Un, dtv)
        Uc = T.step(Uc, dtv, w.domains[0].dx, w.domains[0].bc, w.physics, w.ndim, w.gamma, w.integrator, al, ch,
                    w.glm_cr)
    (Uc * g.cpu().view(w.U.shape)).sum().backward()
    want = Ut.grad.numpy().ravel()
    got = U0.grad.cpu().numpy()
    assert np.abs(got - want).max() / np.abs(want).max() <= 1e-10


def test_adjoint_passive_blocks_pass_through():
    A = _A()
    w = W.batched(nblocks=12, sizes=(8, 12))
    s = A.Solver.from_workload(w)
    U = torch.from_numpy(w.U.copy()).cuda()
    dt = torch.full((s.ndom,), 1e-4, dtype=torch.float64, device="cuda")
    g = torch.from_numpy(np.random.default_rng(5).standard_normal(w.U.size)).cuda()
    out = torch.empty_like(U)
    s.adjoint(U, dt, g, out)
    got, gg = out.cpu().numpy(), g.cpu().numpy()
    T = _torchref()
    c = O.cfg(w.physics, w.ndim, w.integrator, w.gamma, w.glm_cr)
    for i, dd in enumerate(w.domains):
        sl = slice(dd.offset, dd.offset + 9 * dd.ncell)
        if not w.active[i]:
            assert np.array_equal(got[sl], gg[sl])
            continue
        shape = (9,) + tuple(dd.n[::-1])
        _, _, al, ch = O.step(c, _odom(dd), w.U[sl].reshape(shape), 1e-4)
        Ut = torch.from_numpy(w.U[sl].reshape(shape).copy()).requires_grad_(True)
        o = T.step(Ut, 1e-4, dd.dx, dd.bc, w.physics, w.ndim, w.gamma, w.integrator, al, ch, w.glm_cr)
        (o * torch.from_numpy(gg[sl].reshape(shape))).sum().backward()
        want = Ut.grad.numpy().ravel()
        assert np.abs(got[sl] - want).max() / np.abs(want).max() <= 1e-10, i


def test_adjoint_matches_autograd_at_128():
    """The torch-reference comparison at 128^2 (MHD+GLM, SSPRK3, dt 1e-3)."""
    w = W.adjoint2d(128)
    g = np.random.default_rng(17).standard_normal(w.U.shape)
    got, _ = _gpu_adjoint(w, 1e-3, g)
    want, _, _ = _ref_grad(w, 1e-3, g)
    assert np.abs(got - want).max() / np.abs(want).max() <= 1e-10


def test_rollout_gradient_against_oracle_central_differences():
    """dJ/dU^0 of J = sum |B|^2/2 dx dy after 10 steps (checkpoints every 4) at 128^2,
    against central differences (h = 1e-6) of the oracle's frozen-speed steps along
    random unit directions, each step with the speeds of the oracle's own trajectory:
    agreement to 1e-6 of the gradient's norm, on 20 seeded directions."""
    from paper_1407_2052_gb300 import autodiff
    A = _A()
    w = W.adjoint2d(128)
    dtv, nsteps = 1e-3, 10
    area = w.domains[0].dx[0] * w.domains[0].dx[1]
    s = A.Solver.from_workload(w)
    U0 = torch.from_numpy(w.U.ravel().copy()).cuda().requires_grad_(True)
    dt = torch.full((1,), dtv, dtype=torch.float64, device="cuda")
    Uf = autodiff.rollout(s, U0, dt, nsteps, 4)
    B = Uf.view(9, -1)[5:8]
    (0.5 * (B * B).sum() * area).backward()
    grad = U0.grad.cpu().numpy().reshape(w.U.shape)
    c = O.cfg(w.physics, w.ndim, w.integrator, w.gamma, w.glm_cr)
    d = _odom(w.domains[0])
    frozen, U = [], w.U.copy()
    for _ in range(nsteps):
        U, fl, al, ch = O.step(c, d, U, dtv)
        assert fl == 0
        frozen.append((al, ch))

    def final(U):
        for al, ch in frozen:
            U, _ = O.step_frozen(c, d, U, dtv, al, ch)
        return U
    rng = np.random.default_rng(23)
    h = 1e-6
    gnorm = float(np.linalg.norm(grad))
    for _ in range(20):
        v = rng.standard_normal(w.U.shape)
        v /= np.linalg.norm(v)
        Bp, Bm = final(w.U + h * v)[5:8], final(w.U - h * v)[5:8]
        # J(+) - J(-) as sum (B+ - B-)(B+ + B-)/2: no cancellation between two large totals
        fd = 0.5 * float(np.sum((Bp - Bm) * (Bp + Bm))) * area / (2 * h)
        ad = float(np.sum(grad * v))
        # relative to the gradient's norm, the scale of a derivative along a unit direction
        assert abs(fd - ad) <= 1e-6 * gnorm, (fd, ad, gnorm)


def test_adjoint_independent_of_flux_tile():
    """The forward recomputation inside the adjoint records the same limiter pieces under
    every flux tile: bitwise equal gradients."""
    A = _A()
    w = W.adjoint2d(64)
    U = torch.from_numpy(w.U.ravel().copy()).cuda()
    dt = torch.full((1,), 1e-3, dtype=torch.float64, device="cuda")
    g = torch.from_numpy(np.random.default_rng(29).standard_normal(w.U.size)).cuda()
    outs = []
    for tile in [None, (16, 8, 128), (32, 16, 160)]:
        s = A.Solver.from_workload(w)
        if tile:
            s.set_tile(*tile)
        out = torch.empty_like(U)
        s.adjoint(U, dt, g, out)
        assert s.error() == A.OK
        outs.append(out.cpu())
    assert all(torch.equal(o, outs[0]) for o in outs[1:])


@pytest.mark.parametrize("name,make,dt", [CASES[1], CASES[8]], ids=[CASES[1][0], CASES[8][0]])
def test_recorded_step_and_adjoint_equal_plain_ones(name, make, dt):
    """amrfd_step_record advances U exactly as amrfd_step_batched does, and
    amrfd_adjoint_recorded from its record gives exactly amrfd_adjoint's gradient (bitwise),
    also for a partly active domain and for LIMO3."""
    A = _A()
    cases = [make(), _mixed_workload(MIXED[2][1]), _limo3(W.adjoint2d(32), 0.05)]
    for w in cases:
        s = A.Solver.from_workload(w)
        U = torch.from_numpy(np.ascontiguousarray(w.U.ravel())).cuda()
        dtt = torch.full((s.ndom,), dt, dtype=torch.float64, device="cuda")
        g = torch.from_numpy(np.random.default_rng(43).standard_normal(w.U.size)).cuda()
        rec = s.new_record()
        assert rec.numel() == s.record_bytes() > 0
        V1, V2 = U.clone(), U.clone()
        s.step_batched(V1, dtt)
        s.step_record(V2, dtt, rec)
        assert torch.equal(V1, V2)
        a1, a2 = torch.empty_like(U), torch.empty_like(U)
        s.adjoint(U, dtt, g, a1)
        s.adjoint_recorded(U, dtt, rec, g, a2)
        assert s.error() == A.OK
        assert torch.equal(a1, a2)


def test_adjoint_independent_of_adjoint_tile():
    """The transposed flux pass gathers every cell's gradient from the same faces in the same
    order under every tile of its own (amrfd_set_adjoint_tile): bitwise equal gradients, also
    across mirror and outflow faces with passive blocks; out-of-range tiles are rejected."""
    A = _A()
    w = _mixed_workload(MIXED[2][1])
    U = torch.from_numpy(np.ascontiguousarray(w.U.ravel())).cuda()
    dt = torch.full((1,), 2e-3, dtype=torch.float64, device="cuda")
    g = torch.from_numpy(np.random.default_rng(41).standard_normal(w.U.size)).cuda()
    s = A.Solver.from_workload(w)
    outs = []
    for tile in [None, (16, 16, 160), (32, 8, 128), (6, 1, 32), (64, 4, 64)]:
        if tile:
            s.set_adjoint_tile(*tile)
        out = torch.empty_like(U)
        s.adjoint(U, dt, g, out)
        assert s.error() == A.OK
        outs.append(out.cpu())
    assert all(torch.equal(o, outs[0]) for o in outs[1:])
    for bad in [(5, 8, 128), (16, 33, 128), (16, 8, 100), (16, 8, 512), (64, 32, 256)]:
        with pytest.raises(A.AmrfdError) as e:
            s.set_adjoint_tile(*bad)
        assert e.value.code == A.ERR_INVALID_ARG


def test_rollout_200_steps_checkpoint_20_at_512():
    """The adjoint workload's full length: 512^2, 200 fixed-dt steps, checkpoints every 20,
    J = sum |B|^2/2 dx dy; the rollout gradient equals (bitwise) the chain of single-step
    adjoints over the stored trajectory, and is finite."""
    from paper_1407_2052_gb300 import autodiff
    A = _A()
    w = W.adjoint2d(512)
    area = w.domains[0].dx[0] * w.domains[0].dx[1]
    s = A.Solver.from_workload(w)
    U0 = torch.from_numpy(w.U.ravel().copy()).cuda()
    dt = torch.full((1,), 1e-3, dtype=torch.float64, device="cuda")
    nsteps = 200
    U0r = U0.clone().requires_grad_(True)
    Uf = autodiff.rollout(s, U0r, dt, nsteps, 20)
    B = Uf.view(9, -1)[5:8]
    (0.5 * (B * B).sum() * area).backward()
    grad = U0r.grad.clone()
    assert bool(torch.isfinite(grad).all())
    states = [U0.clone()]
    for _ in range(nsteps):
        nxt = states[-1].clone()
        s.step_batched(nxt, dt)
        states.append(nxt)
    assert torch.equal(states[-1], Uf.detach())
    gB = torch.zeros_like(U0).view(9, -1)
    gB[5:8] = states[-1].view(9, -1)[5:8] * area
    g = gB.view(-1).clone()
    out = torch.empty_like(g)
    for j in reversed(range(nsteps)):
        s.adjoint(states[j], dt, g, out)
        g, out = out, g
    assert s.error() == A.OK
    assert torch.equal(g, grad)


# partly active domains (App. C): passive blocks keep U^n, and active blocks next to them
# read that U^n as halo, so the gradient reaches U^n there through the fluxes as well as
# through the identity (blocks of >= 3 cells along every dimension)
MIXED = [
    ("euler1d_periodic", (O.EULER, 1, (40, 1, 1), ((0, 0), (0, 0), (0, 0)), ((0, 0),) * 3, O.SSPRK3, (5, 1, 1),
                          [1, 0, 1, 0, 0]), 2e-3),
    ("mhd2d_periodic_4x4", (O.MHD_GLM, 2, (24, 20, 1), ((0, 0), (0, 0), (0, 0)), ((0, 0),) * 3, O.SSPRK54,
                            (4, 4, 1), [1, 1, 0, 1, 0, 1, 1, 0, 1, 0, 0, 1, 1, 1, 0, 1]), 1e-3),
    ("euler3d_outflow_mirror", (O.EULER, 3, (12, 12, 9), ((1, 1), (2, 2), (0, 0)), ((0, 0), (4, 4), (0, 0)),
                                O.SSPRK3, (3, 2, 3), [1, 0, 1, 1, 1, 0, 0, 1, 1, 0, 1, 1, 1, 1, 0, 0, 1, 0]), 2e-3),
    ("mhd3d_last_block_passive", (O.MHD_GLM, 3, (12, 10, 8), ((0, 0), (1, 1), (0, 0)), ((0, 0),) * 3, O.SSPRK3,
                                  (2, 2, 2), [1, 1, 1, 1, 1, 1, 1, 0]), 1e-3),
]


def _mixed_workload(spec):
    physics, ndim, n, bc, asym, integ, nb, act = spec
    w = _smooth(physics, ndim, n, bc, 50 + sum(n), integ, asym=asym, nb=nb)
    w.active = np.array(act, np.uint8)
    return w


def _ref_grad_mixed(w, dt, g):
    T = _torchref()
    d = w.domains[0]
    c = O.cfg(w.physics, w.ndim, w.integrator, w.gamma, w.glm_cr, recon=w.recon, limo3_r=w.limo3_r)
    _, fl, al, ch = O.step(c, _odom(d), w.U, dt, active=w.active)
    assert fl == 0
    U = torch.from_numpy(w.U.copy()).requires_grad_(True)
    out = T.step(U, dt, d.dx, d.bc, w.physics, w.ndim, w.gamma, w.integrator, al, ch, w.glm_cr, asym=d.asym,
                 mask=T.block_mask(d.n, d.nb, w.active), recon=w.recon, limo3_r=w.limo3_r)
    (out * torch.from_numpy(g)).sum().backward()
    return U.grad.numpy()


@pytest.mark.parametrize("name,spec,dt", MIXED, ids=[c[0] for c in MIXED])
def test_adjoint_partly_active_domain_matches_autograd(name, spec, dt):
    w = _mixed_workload(spec)
    g = np.random.default_rng(11).standard_normal(w.U.shape)
    got, _ = _gpu_adjoint(w, dt, g)
    want = _ref_grad_mixed(w, dt, g)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err <= 1e-10, err
    # the halo dependence is there: passive cells next to active ones get more than g
    T = _torchref()
    m = T.block_mask(w.domains[0].n, w.domains[0].nb, w.active).numpy()
    assert np.abs(want[:, ~m] - g[:, ~m]).max() > 1e-3 * np.abs(g).max()


def test_adjoint_partly_active_against_oracle_central_differences():
    """Central differences (h = 1e-6) of the oracle's frozen-speed step with passive blocks,
    along 8 seeded directions, against <v, adjoint(g)>."""
    name, spec, dt = MIXED[1]
    w = _mixed_workload(spec)
    d = _odom(w.domains[0])
    c = O.cfg(w.physics, w.ndim, w.integrator, w.gamma, w.glm_cr)
    _, _, al, ch = O.step(c, d, w.U, dt, active=w.active)
    rng = np.random.default_rng(23)
    g = rng.standard_normal(w.U.shape)
    got, _ = _gpu_adjoint(w, dt, g)
    h = 1e-6
    for _ in range(8):
        v = rng.standard_normal(w.U.shape)
        v /= np.linalg.norm(v)
        up, _ = O.step_frozen(c, d, w.U + h * v, dt, al, ch, active=w.active)
        um, _ = O.step_frozen(c, d, w.U - h * v, dt, al, ch, active=w.active)
        fd = float(((up - um) / (2 * h) * g).sum())
        ad = float((got * v).sum())
        assert abs(fd - ad) <= 1e-6 * np.linalg.norm(got), (fd, ad)


@pytest.mark.slow
def test_rollout_gradient_at_512_against_oracle_central_differences():
    """The adjoint workload at its stated size: 512^2 MHD+GLM, fixed dt 1e-3, a checkpointed
    rollout of 20 steps (checkpoints every 10) of J = sum |B|^2/2 dx dy, against central
    differences (h = 1e-6) of the oracle's frozen-speed trajectory along 20 seeded unit
    directions, to 1e-6 of the gradient's norm. The differences run on the host cores in a
    spawn process pool (the test process already holds a CUDA context)."""
    import multiprocessing as mp
    import os
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    import fd_oracle
    from paper_1407_2052_gb300 import autodiff
    A = _A()
    w = W.adjoint2d(512)
    dtv, nsteps, every = 1e-3, 20, 10
    area = w.domains[0].dx[0] * w.domains[0].dx[1]
    s = A.Solver.from_workload(w)
    U0 = torch.from_numpy(w.U.ravel().copy()).cuda().requires_grad_(True)
    dt = torch.full((1,), dtv, dtype=torch.float64, device="cuda")
    Uf = autodiff.rollout(s, U0, dt, nsteps, every)
    B = Uf.view(9, -1)[5:8]
    (0.5 * (B * B).sum() * area).backward()
    assert s.error() == A.OK
    grad = U0.grad.cpu().numpy().reshape(w.U.shape)
    c = O.cfg(w.physics, w.ndim, w.integrator, w.gamma, w.glm_cr)
    d0 = w.domains[0]
    d = _odom(d0)
    frozen, U = [], w.U.copy()
    for _ in range(nsteps):
        U, fl, al, ch = O.step(c, d, U, dtv)
        assert fl == 0
        frozen.append((al, ch))
    rng = np.random.default_rng(31)
    dirs = []
    for _ in range(20):
        v = rng.standard_normal(w.U.shape)
        dirs.append(v / np.linalg.norm(v))
    cfgt = (w.physics, w.ndim, w.integrator, w.gamma, w.glm_cr)
    domt = (d0.n, d0.dx, [list(b) for b in d0.bc])
    jobs = [(cfgt, domt, w.U, v, 1e-6, dtv, frozen, area) for v in dirs]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        fds = pool.map(fd_oracle.fd_along, jobs)
    gnorm = float(np.linalg.norm(grad))
    worst = 0.0
    for v, fd in zip(dirs, fds):
        ad = float(np.sum(grad * v))
        worst = max(worst, abs(fd - ad) / gnorm)
    assert worst <= 1e-6, worst


# LIMO3 reconstruction (Sec. 2.2): the forward recomputation records which piece the
# limiter took at every face, the adjoint applies that piece's coefficients
def _limo3(w, r):
    w.recon, w.limo3_r = O.LIMO3, r
    return w


LIMO_CASES = [
    ("mhd2d_ssprk3_r1", lambda: _limo3(W.adjoint2d(32), 1.0), 1e-3),
    ("mhd2d_ssprk3_limited", lambda: _limo3(W.adjoint2d(32), 0.05), 1e-3),
    ("euler1d_outflow_ssprk43", lambda: _limo3(_smooth(O.EULER, 1, (40, 1, 1), ((1, 1), (0, 0), (0, 0)), 8,
                                                       O.SSPRK43), 0.2), 2e-3),
    ("euler2d_mirror_outflow_blocks", lambda: _limo3(_smooth(O.EULER, 2, (36, 16, 1), ((2, 1), (2, 2), (0, 0)), 9,
                                                             O.SSPRK3, asym=((6, 0), (6, 6), (0, 0)),
                                                             nb=(3, 2, 1)), 0.1), 2e-3),
]


@pytest.mark.parametrize("name,make,dt", LIMO_CASES, ids=[c[0] for c in LIMO_CASES])
def test_limo3_adjoint_matches_autograd(name, make, dt):
    w = make()
    g = np.random.default_rng(13).standard_normal(w.U.shape)
    got, _ = _gpu_adjoint(w, dt, g)
    want, _, _ = _ref_grad(w, dt, g)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err <= 1e-10, err


def test_limo3_adjoint_partly_active_matches_autograd():
    name, spec, dt = MIXED[2]
    w = _limo3(_mixed_workload(spec), 0.2)
    g = np.random.default_rng(17).standard_normal(w.U.shape)
    got, _ = _gpu_adjoint(w, dt, g)
    want = _ref_grad_mixed(w, dt, g)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err <= 1e-10, err


def test_limo3_adjoint_against_oracle_central_differences():
    """Central differences (h = 1e-6) of the oracle's frozen-speed LIMO3 step along 8 seeded
    directions, on data resolved enough that the pieces hold under the perturbation."""
    w = _limo3(W.adjoint2d(128), 1.0)
    dt = 1e-3
    c = O.cfg(w.physics, w.ndim, w.integrator, w.gamma, w.glm_cr, recon=w.recon, limo3_r=w.limo3_r)
    d = _odom(w.domains[0])
    _, _, al, ch = O.step(c, d, w.U, dt)
    rng = np.random.default_rng(37)
    g = rng.standard_normal(w.U.shape)
    got, _ = _gpu_adjoint(w, dt, g)
    h = 1e-6
    for _ in range(8):
        v = rng.standard_normal(w.U.shape)
        v /= np.linalg.norm(v)
        up, _ = O.step_frozen(c, d, w.U + h * v, dt, al, ch)
        um, _ = O.step_frozen(c, d, w.U - h * v, dt, al, ch)
        fd = float(((up - um) / (2 * h) * g).sum())
        ad = float((got * v).sum())
        assert abs(fd - ad) <= 1e-6 * np.linalg.norm(got), (fd, ad)
