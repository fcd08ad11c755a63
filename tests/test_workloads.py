"""The seeded synthetic inputs hold the recipe they are documented with (CPU): shapes,
value ranges, the fields that must be uniform, block layout, and determinism."""
import numpy as np

from paper_1407_2052_gb300 import workloads as W


def _pressure_mhd(U, gamma):
    rho, m, E, B = U[0], U[1:4], U[4], U[5:8]
    return (gamma - 1.0) * (E - 0.5 * (m * m).sum(axis=0) / rho - 0.5 * (B * B).sum(axis=0))


def test_blast3d_recipe():
    w = W.blast3d(32, 8)
    assert w.U.shape == (9, 32, 32, 32) and w.ndim == 3 and w.cfl == 0.3 and w.nsteps == 200
    rho = w.U[0]
    assert np.all(np.abs(rho - 1.0) <= 1e-3) and rho.std() > 1e-4   # rho = 1 + 1e-3 (2u - 1)
    assert np.all(w.U[1:4] == 0.0) and np.all(w.U[8] == 0.0)        # at rest, psi = 0
    b = 1.0 / np.sqrt(2.0)
    assert np.all(w.U[5] == b) and np.all(w.U[6] == b) and np.all(w.U[7] == 0.0)
    p = _pressure_mhd(w.U, w.gamma)
    x = (np.arange(32) + 0.5) / 32 - 0.5
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    inside = np.sqrt(X * X + Y * Y + Z * Z) < 0.1
    assert inside.any() and np.allclose(p[inside], 10.0, rtol=1e-12) and np.allclose(p[~inside], 0.1, rtol=1e-12)
    d = w.domains[0]
    assert tuple(d.n) == (32, 32, 32) and tuple(d.nb) == (4, 4, 4)
    assert w.active.shape == (64,) and np.all(w.active == 1)
    assert np.array_equal(w.U, W.blast3d(32, 8).U)                  # seeded
    q = W.blast3d(32, 8, noise=0.0)
    assert np.all(q.U[0] == 1.0) and "background" in q.extra


def test_batched_recipe():
    w = W.batched(nblocks=40)
    assert len(w.domains) == 40 and w.active.shape == (40,)
    off = 0
    for d in w.domains:
        m = d.n[0]
        assert tuple(d.n) == (m, m, m) and m in (8, 12, 16, 24, 32)
        assert 1e-3 <= d.dx[0] <= 1e-1 and d.dx[0] == d.dx[1] == d.dx[2]
        assert d.offset == off
        blk = w.U[off:off + 9 * m ** 3].reshape(9, m ** 3)
        assert np.all(np.abs(blk[0] - 1.0) <= 0.05)                  # rho = 1 + delta, |delta| <= 0.05
        assert np.all(blk[5] == 0.5) and np.all(blk[6] == 0.0) and np.all(blk[7] == 0.0) and np.all(blk[8] == 0.0)
        off += 9 * m ** 3
    assert off == w.U.size
    assert np.array_equal(w.U, W.batched(nblocks=40).U) and np.array_equal(w.active, W.batched(nblocks=40).active)


def test_adjoint2d_recipe():
    w = W.adjoint2d(64)
    assert w.U.shape == (9, 1, 64, 64) and w.extra == {"dt": 1e-3, "checkpoint_every": 20}
    for v in range(8):                                               # every component but psi varies
        assert w.U[v].std() > 0.0, v
    assert np.all(w.U[8] == 0.0)
    assert np.array_equal(w.U, W.adjoint2d(64).U)
