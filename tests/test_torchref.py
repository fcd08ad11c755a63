"""The plain-PyTorch reference step (tests/torchref.py), whose autograd serves as the
reference gradient of the discrete adjoint, reproduces the oracle's frozen-speed step
(both FP64 restatements of Sec. 2.1-2.3 written independently of each other), on
periodic, outflow and mirror faces. CPU only."""
import os
import sys

import numpy as np
import pytest

import oracle as O
from paper_1407_2052_gb300 import workloads as W

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(__file__))
import torchref as T  # noqa: E402


def _smooth(physics, ndim, n, bc, asym, seed, integrator):
    rng = np.random.default_rng(seed)
    g = 1.4 if physics == O.EULER else 5 / 3
    shp = tuple(n[::-1])
    rho, p = 1.0 + 0.2 * rng.random(shp), 1.0 + 0.2 * rng.random(shp)
    vel = [0.3 * rng.standard_normal(shp) for _ in range(3)]
    if physics == O.EULER:
        U = W.conserved_euler(rho, vel[:ndim], p, g)
    else:
        U = W.conserved_mhd(rho, vel, p, [0.5 + 0.1 * rng.standard_normal(shp) for _ in range(3)], g,
                            psi=0.01 * rng.standard_normal(shp))
    return W.Domain(tuple(n), (0.1, 0.08, 0.12), bc=bc, asym=asym), U, g


CASES = [
    (O.EULER, 1, (30, 1, 1), ((1, 1), (0, 0), (0, 0)), ((0, 0),) * 3, O.SSPRK3),
    (O.EULER, 1, (30, 1, 1), ((2, 2), (0, 0), (0, 0)), ((2, 2), (0, 0), (0, 0)), O.SSPRK43),
    (O.EULER, 2, (14, 12, 1), ((2, 1), (0, 0), (0, 0)), ((6, 0), (0, 0), (0, 0)), O.SSPRK54),
    (O.MHD_GLM, 2, (12, 14, 1), ((0, 0), (2, 2), (0, 0)), ((0, 0), (W.MHD_WALL_Y,) * 2, (0, 0)), O.SSPRK3),
    (O.MHD_GLM, 3, (8, 6, 7), ((1, 2), (0, 0), (2, 1)), ((0, 0x1F), (0, 0), (0x104, 0)), O.SSPRK3),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_torchref_step_equals_oracle_frozen_step(case):
    physics, ndim, n, bc, asym, integ = CASES[case]
    dom, U, g = _smooth(physics, ndim, n, bc, asym, 20 + case, integ)
    c = O.cfg(physics, ndim, integ, g)
    d = O.dom(dom.n, dom.dx, bc=[list(b) for b in bc], asym=asym)
    h = 0.5 * O.dt(c, d, U, 0.4)[0]
    want, fl, al, ch = O.step(c, d, U, h)
    assert fl == 0
    got = T.step(torch.from_numpy(U.copy()), h, dom.dx, bc, physics, ndim, g, integ, al, ch, asym=asym)
    err = np.abs(got.numpy() - want).max() / np.abs(want).max()
    assert err <= 1e-13, err


# partly active domains (App. C): blocks of >= 3 cells, passive ones keep U^n and feed
# their active neighbours' halos with it
MIXED = [
    (O.EULER, 1, (40, 1, 1), ((0, 0), (0, 0), (0, 0)), ((0, 0),) * 3, O.SSPRK3, (5, 1, 1), [1, 0, 1, 0, 0]),
    (O.MHD_GLM, 2, (24, 20, 1), ((0, 0), (0, 0), (0, 0)), ((0, 0),) * 3, O.SSPRK54, (4, 4, 1),
     [1, 1, 0, 1, 0, 1, 1, 0, 1, 0, 0, 1, 1, 1, 0, 1]),
    (O.EULER, 3, (12, 12, 9), ((1, 1), (2, 2), (0, 0)), ((0, 0), (4, 4), (0, 0)), O.SSPRK3, (3, 2, 3),
     [1, 0, 1, 1, 1, 0, 0, 1, 1, 0, 1, 1, 1, 1, 0, 0, 1, 0]),
]


@pytest.mark.parametrize("case", range(len(MIXED)))
def test_torchref_step_with_passive_blocks_equals_oracle(case):
    physics, ndim, n, bc, asym, integ, nb, act = MIXED[case]
    dom, U, g = _smooth(physics, ndim, n, bc, asym, 40 + case, integ)
    c = O.cfg(physics, ndim, integ, g)
    d = O.dom(dom.n, dom.dx, bc=[list(b) for b in bc], nb=nb, asym=asym)
    act = np.array(act, np.uint8)
    h = 0.5 * O.dt(c, d, U, 0.4, active=act)[0]
    want, fl, al, ch = O.step(c, d, U, h, active=act)
    assert fl == 0
    got = T.step(torch.from_numpy(U.copy()), h, dom.dx, bc, physics, ndim, g, integ, al, ch, asym=asym,
                 mask=T.block_mask(n, nb, act))
    err = np.abs(got.numpy() - want).max() / np.abs(want).max()
    assert err <= 1e-13, err
    # the passive blocks did not move, and some active cell next to one did
    m = T.block_mask(n, nb, act).numpy()
    assert np.array_equal(got.numpy()[:, ~m], U[:, ~m])
    assert np.abs(got.numpy()[:, m] - U[:, m]).max() > 0


# LIMO3 reconstruction (Sec. 2.2 cites Cada & Torrilhon 2009), r = 1 and a larger radius
LIMO = [
    (O.EULER, 1, (30, 1, 1), ((1, 1), (0, 0), (0, 0)), ((0, 0),) * 3, O.SSPRK3, 1.0),
    (O.MHD_GLM, 2, (12, 14, 1), ((0, 0), (2, 2), (0, 0)), ((0, 0), (W.MHD_WALL_Y,) * 2, (0, 0)), O.SSPRK43, 1.0),
    (O.EULER, 3, (8, 6, 7), ((0, 0), (1, 1), (2, 2)), ((0, 0), (0, 0), (8, 8)), O.SSPRK3, 0.05),
]


@pytest.mark.parametrize("case", range(len(LIMO)))
def test_torchref_limo3_step_equals_oracle_frozen_step(case):
    physics, ndim, n, bc, asym, integ, r = LIMO[case]
    dom, U, g = _smooth(physics, ndim, n, bc, asym, 60 + case, integ)
    c = O.cfg(physics, ndim, integ, g, recon=O.LIMO3, limo3_r=r)
    d = O.dom(dom.n, dom.dx, bc=[list(b) for b in bc], asym=asym)
    h = 0.5 * O.dt(c, d, U, 0.4)[0]
    want, fl, al, ch = O.step(c, d, U, h)
    assert fl == 0
    got = T.step(torch.from_numpy(U.copy()), h, dom.dx, bc, physics, ndim, g, integ, al, ch, asym=asym,
                 recon=1, limo3_r=r)
    err = np.abs(got.numpy() - want).max() / np.abs(want).max()
    assert err <= 1e-13, err
