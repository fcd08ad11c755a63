"""The checked build (libamrfd_checked.so, -DAMRFD_CHECKS: every work descriptor and the
tile, halo and window indices checked in the kernels, a failure recorded as
AMRFD_ERR_CHECK instead of an access) runs the parity workloads without a failed check
and gives bitwise the results of the normal build; reruns are bitwise deterministic
(no floating-point atomics: the maxima are integer maxima of bit patterns)."""
import numpy as np
import pytest

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


def _cases():
    A = _A()
    w1 = W.blast3d(32, 8)
    w1.active = np.ones(64, np.uint8)
    w1.active[[3, 17, 42]] = 0
    w2 = W.wall_blast2d(64, 16)
    w3 = W.batched(nblocks=24, sizes=(8, 12, 16))
    w4 = W.brio_wu(128)
    w5 = W.vortex2d(64)
    w5.recon = A.LIMO3
    w6 = W.sod(200)
    w6.integrator = A.SSPRK43
    return [("blast_passive", w1), ("wall_mirror", w2), ("batched", w3), ("briowu_outflow", w4),
            ("vortex_limo3", w5), ("sod_ssprk43", w6)]


def _run(w, checked, nsteps=3, tile=None, plain=False):
    A = _A()
    s = A.Solver.from_workload(w, checked=checked)
    if tile:
        s.set_tile(*tile)
    U = torch.from_numpy(np.ascontiguousarray(w.U).ravel().copy()).cuda()
    dts = []
    for _ in range(nsteps):
        dt = s.dt(U)
        (s.step if plain else s.step_batched)(U, dt)
        dts.append(dt.cpu())
    return s.error(), U.cpu(), dts


@pytest.mark.parametrize("idx", range(6))
def test_checked_build_passes_and_matches(idx):
    A = _A()
    name, w = _cases()[idx]
    for tile in [None, (16, 8, 128), (8, 1, 32), (32, 16, 320)]:
        if tile and w.ndim == 1 and tile[1] != 1:
            continue
        e1, U1, d1 = _run(w, False, tile=tile)
        e2, U2, d2 = _run(w, True, tile=tile)
        e3, U3, _ = _run(w, True, tile=tile, plain=True)
        assert e1 == A.OK and e2 == A.OK and e3 == A.OK, (name, tile, e2, e3)
        assert torch.equal(U1, U2) and torch.equal(U1, U3), (name, tile)
        assert all(torch.equal(a, b) for a, b in zip(d1, d2))


def test_checked_adjoint_and_activation():
    A = _A()
    w = W.adjoint2d(32)
    U = torch.from_numpy(w.U.ravel().copy()).cuda()
    dt = torch.full((1,), 1e-3, dtype=torch.float64, device="cuda")
    g = torch.from_numpy(np.random.default_rng(1).standard_normal(w.U.size)).cuda()
    outs = []
    for checked in (False, True):
        s = A.Solver.from_workload(w, checked=checked)
        out = torch.empty_like(U)
        s.adjoint(U, dt, g, out)
        assert s.error() == A.OK
        outs.append(out.cpu())
    assert torch.equal(outs[0], outs[1])
    # a partly active domain next to mirror walls, with MP5 and with LIMO3: the adjoint's
    # items over passive neighbours and the LIMO3 pieces under the checks
    wb = W.wall_blast2d(64, 16)
    wb.active = (np.random.default_rng(3).random(len(wb.active)) > 0.35).astype(np.uint8)
    for recon in (0, 1):
        wb.recon = recon
        Ub = torch.from_numpy(np.ascontiguousarray(wb.U.ravel())).cuda()
        gb = torch.from_numpy(np.random.default_rng(2).standard_normal(Ub.numel())).cuda()
        dtb = torch.full((1,), 1e-4, dtype=torch.float64, device="cuda")
        outs = []
        for checked in (False, True):
            s = A.Solver.from_workload(wb, checked=checked)
            out = torch.empty_like(Ub)
            s.adjoint(Ub, dtb, gb, out)
            assert s.error() == A.OK, (recon, checked)
            outs.append(out.cpu())
        assert torch.equal(outs[0], outs[1]), recon
    w = W.blast3d(64, 8, noise=0.0)
    res = []
    for checked in (False, True):
        s = A.Solver.from_workload(w, checked=checked)
        R = torch.from_numpy(w.extra["background"].ravel().copy()).cuda()
        U = torch.from_numpy(w.U.ravel().copy()).cuda()
        for _ in range(3):
            s.activate(s.flag_steady(U, R, 1e-12), 2)
            s.step_cfl(U)
        assert s.error() == A.OK
        res.append((U.cpu(), s.active().cpu()))
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])


def test_reruns_are_bitwise_deterministic():
    A = _A()
    w = W.blast3d(32, 8)
    outs = []
    for _ in range(3):
        s = A.Solver.from_workload(w)
        U = torch.from_numpy(w.U.ravel().copy()).cuda()
        for _ in range(4):
            s.step_cfl(U)
        outs.append(U.cpu())
    assert all(torch.equal(o, outs[0]) for o in outs[1:])
