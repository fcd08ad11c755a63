"""Dynamic grid activation (App. C) on the GPU against the oracle's restatement.

Criterion (amrfd_flag_steady), safety belt and work-list rebuild (amrfd_activate) are
integer work: compared bitwise. A run that re-evaluates the criterion every step is
compared with the oracle doing the same, and with the all-active run (the belt keeps
ahead of the blast, so the passive blocks hold exactly what the full update gives)."""
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


def _odom(d):
    return O.dom(d.n, d.dx, bc=[list(b) for b in d.bc], nb=d.nb, asym=d.asym)


def _multi_domain_workload():
    """Five Euler 3D domains of different block grids and boundary kinds."""
    rng = np.random.default_rng(3)
    doms, parts, off = [], [], 0
    specs = [((4, 4, 4), 0), ((5, 3, 2), 1), ((1, 6, 3), 2), ((2, 2, 7), 0), ((3, 1, 1), 1)]
    for nb, bck in specs:
        n = tuple(4 * b for b in nb)
        bc = ((bck, bck), (0, 0), (bck, bck))
        d = W.Domain(n, (0.1, 0.1, 0.1), bc=bc, nb=nb, offset=off)
        shp = n[::-1]
        U = W.conserved_euler(1 + 0.1 * rng.random(shp), [0.1 * rng.random(shp) for _ in range(3)],
                              1 + 0.1 * rng.random(shp), 1.4)
        doms.append(d)
        parts.append(U.ravel())
        off += U.size
    nblk = sum(int(np.prod(d.nb)) for d in doms)
    return W.Workload("multi", O.EULER, 3, O.SSPRK3, 1.4, 0.4, doms, np.concatenate(parts),
                      active=np.ones(nblk, np.uint8))


@pytest.mark.parametrize("belt", [0, 1, 2, 3])
def test_activate_matches_oracle_bitwise(belt):
    w = _multi_domain_workload()
    s = _A().Solver.from_workload(w)
    rng = np.random.default_rng(belt)
    flag = (rng.random(s.nblocks) > 0.1).astype(np.uint8)
    s.activate(torch.from_numpy(flag).cuda(), belt)
    got = s.active().cpu().numpy()
    b0 = 0
    for d in w.domains:
        nbl = int(np.prod(d.nb))
        want = O.activate(_odom(d), flag[b0:b0 + nbl], belt)
        assert np.array_equal(got[b0:b0 + nbl], want), (belt, d.nb, d.bc)
        b0 += nbl


def test_flag_steady_matches_oracle_bitwise():
    w = W.blast3d(32, 8)
    s = _A().Solver.from_workload(w)
    c = O.cfg(w.physics, w.ndim, w.integrator, w.gamma, w.glm_cr)
    d = _odom(w.domains[0])
    R = w.U.copy()
    U = R.copy()
    rng = np.random.default_rng(9)
    for _ in range(12):
        z, y, x = rng.integers(0, 32, 3)
        U[rng.integers(0, 9), z, y, x] += rng.choice([1e-11, 1e-9, np.nan])
    for tol in (0.0, 1e-10, 1e-8):
        got = s.flag_steady(torch.from_numpy(U.ravel()).cuda(), torch.from_numpy(R.ravel()).cuda(), tol)
        assert np.array_equal(got.cpu().numpy(), O.flag_steady(c, d, U, R, tol)), tol


def _run_activation_gpu(w, nsteps, tol, belt, batched=True):
    s = _A().Solver.from_workload(w)
    R = torch.from_numpy(w.extra["background"].ravel().copy()).cuda()
    U = torch.from_numpy(w.U.ravel().copy()).cuda()
    acts, dts = [], []
    for _ in range(nsteps):
        s.activate(s.flag_steady(U, R, tol), belt)
        acts.append(s.active().cpu().numpy())
        dt = s.dt(U)
        dts.append(float(dt[0].item()))
        (s.step_batched if batched else s.step)(U, dt)
    assert s.error() == _A().OK
    return U.cpu().numpy().reshape(w.U.shape), acts, dts


@pytest.mark.parametrize("batched", [True, False])
def test_dynamic_activation_run_vs_oracle_and_full_update(batched):
    """Quiet 3D MHD blast (uniform background) at 64^3 in 8^3-cell blocks, 8 SSPRK3 steps,
    criterion |U - U_background| <= 1e-12 (blocks the blast has not reached are passive)
    and a two-block belt, re-evaluated before every step."""
    w = W.blast3d(64, 8, noise=0.0)
    nsteps, tol, belt = 8, 1e-12, 2
    got, acts, dts = _run_activation_gpu(w, nsteps, tol, belt, batched)
    c = O.cfg(w.physics, w.ndim, w.integrator, w.gamma, w.glm_cr)
    d = _odom(w.domains[0])
    U = w.U.copy()
    R = w.extra["background"]
    for k in range(nsteps):
        act = O.activate(d, O.flag_steady(c, d, U, R, tol), belt)
        assert np.array_equal(acts[k], act), k
        h, _ = O.dt(c, d, U, w.cfl, active=act)
        # dt of U^0 bitwise; later states differ by rounding, most at the strong blast
        # front where the largest speed sits
        assert dts[k] == h if k == 0 else abs(dts[k] - h) <= 1e-11 * h, (k, dts[k], h)
        U, fl, _, ch = O.step(c, d, U, h, active=act)
        assert fl == 0
    assert 0 < acts[0].sum() < acts[0].size          # the blast starts with a passive rim
    assert acts[-1].sum() > acts[0].sum()              # and activates blocks as it spreads
    err = np.abs(got - U).sum() / np.abs(U).sum()
    assert err <= 1e-10, err
    # all-active GPU run with the same time steps: the passive blocks held what the full
    # update gives (uniform states are steady up to the rounding of the stage combination)
    s = _A().Solver.from_workload(w)
    Uf = torch.from_numpy(w.U.ravel().copy()).cuda()
    for k in range(nsteps):
        dt = torch.full((1,), dts[k], dtype=torch.float64, device="cuda")
        s.step_batched(Uf, dt)
    full = Uf.cpu().numpy().reshape(w.U.shape)
    assert np.abs(full - got).max() <= 1e-12 * np.abs(full).max()


def test_activation_keeps_graph_valid_and_plain_path_in_step():
    """amrfd_activate between graph replays of amrfd_step_batched, then amrfd_step (which
    refreshes its host copy of the flags): both paths give the same bits."""
    w = W.blast3d(64, 8, noise=0.0)
    A = _A()
    outs = []
    for batched in (True, False):
        s = A.Solver.from_workload(w)
        R = torch.from_numpy(w.extra["background"].ravel().copy()).cuda()
        U = torch.from_numpy(w.U.ravel().copy()).cuda()
        dt = torch.full((1,), 2e-4, dtype=torch.float64, device="cuda")
        for k in range(6):
            s.activate(s.flag_steady(U, R, 1e-12), 1 + k % 2)
            (s.step_batched if batched else s.step)(U, dt)
        assert s.error() == A.OK
        outs.append(U.cpu())
    assert torch.equal(outs[0], outs[1])
