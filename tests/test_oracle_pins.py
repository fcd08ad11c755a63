"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks one part of the oracle (oracle/amrfd_oracle.c) against a closed
form, an invariant, a special case reducing to a textbook result, a value
worked by hand from the published algorithm (tests/golden/), or a measured
convergence order the paper states (Porth et al. 2014, Sec. 4.5.1: fifth
order with MP5 + SSPRK(5,4)). The choice is such that a dropped term, a wrong
sign or index, or a transposed operand anywhere in the oracle fails at least one.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import riemann
from paper_1407_2052_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def _odom(d):
    return O.dom(d.n, d.dx, bc=[list(b) for b in d.bc], nb=d.nb, asym=d.asym)


def _ocfg(w, integrator=None):
    return O.cfg(w.physics, w.ndim, w.integrator if integrator is None else integrator, w.gamma, w.glm_cr,
                 recon=w.recon, limo3_r=w.limo3_r)


# ------------------------------------------------------------ point-wise pieces
@pytest.mark.parametrize("physics,ndim", [(O.EULER, 1), (O.EULER, 3), (O.MHD_GLM, 3)])
def test_cons2prim_round_trip(physics, ndim):
    rng = np.random.default_rng(0)
    g = 1.4 if physics == O.EULER else 5.0 / 3.0
    c = O.cfg(physics, ndim, gamma=g)
    U = W.random_states(rng, 200, physics, ndim, g)
    for j in range(U.shape[1]):
        w, ok = O.cons2prim(c, U[:, j])
        assert ok
        if physics == O.EULER:
            back = W.conserved_euler(w[0], list(w[1:1 + ndim]), w[4], g)
        else:
            back = W.conserved_mhd(w[0], list(w[1:4]), w[4], list(w[5:8]), g, w[8])
        np.testing.assert_allclose(back, U[:, j], rtol=2e-14, atol=1e-14)


def test_cons2prim_flags_nonphysical():
    c = O.cfg(O.MHD_GLM, 3, gamma=5 / 3)
    u = W.conserved_mhd(np.array(1.0), [np.array(0.0)] * 3, np.array(1.0), [np.array(0.0)] * 3, 5 / 3)
    assert O.cons2prim(c, u)[1]
    bad = u.copy(); bad[0] = -1.0
    assert not O.cons2prim(c, bad)[1]
    bad = u.copy(); bad[4] = 0.1 * bad[4] - 10.0  # negative pressure
    assert not O.cons2prim(c, bad)[1]
    bad = u.copy(); bad[6] = np.nan
    assert not O.cons2prim(c, bad)[1]


def test_char_speed_closed_forms():
    """|v_d| + c_s for Euler; MHD fast speed: B = 0 -> a, B perp d -> sqrt(a^2+b^2),
    B parallel d -> max(a, |B|/sqrt(rho))."""
    g = 5.0 / 3.0
    rng = np.random.default_rng(1)
    ce = O.cfg(O.EULER, 3, gamma=g)
    cm = O.cfg(O.MHD_GLM, 3, gamma=g)
    for _ in range(50):
        rho, p = rng.uniform(0.1, 3), rng.uniform(0.1, 3)
        v = rng.uniform(-2, 2, 3)
        a = math.sqrt(g * p / rho)
        ue = W.conserved_euler(np.array(rho), [np.array(x) for x in v], np.array(p), g)
        we, _ = O.cons2prim(ce, ue)
        for d in range(3):
            assert O.char_speed(ce, we, d) == pytest.approx(abs(v[d]) + a, rel=1e-15)
        for d in range(3):
            bmag = rng.uniform(0.1, 2)
            for kind in ("zero", "perp", "par"):
                B = np.zeros(3)
                if kind == "perp":
                    B[(d + 1) % 3] = bmag * 0.6
                    B[(d + 2) % 3] = bmag * 0.8
                elif kind == "par":
                    B[d] = bmag
                um = W.conserved_mhd(np.array(rho), [np.array(x) for x in v], np.array(p),
                                     [np.array(x) for x in B], g)
                wm, _ = O.cons2prim(cm, um)
                b2 = float(B @ B) / rho
                want = {"zero": a, "perp": math.sqrt(a * a + b2), "par": max(a, math.sqrt(b2))}[kind]
                assert O.char_speed(cm, wm, d) == pytest.approx(abs(v[d]) + want, rel=1e-13)


def _jacobian(c, u, d, ch):
    nv = O.nvar(c)
    J = np.zeros((nv, nv))
    for k in range(nv):
        h = 1e-6 * max(1.0, abs(u[k]))
        up, um = u.copy(), u.copy()
        up[k] += h
        um[k] -= h
        J[:, k] = (O.flux(c, up, d, ch) - O.flux(c, um, d, ch)) / (2 * h)
    return J


@pytest.mark.parametrize("d", [0, 1, 2])
def test_flux_jacobian_spectrum_mhd(d):
    """Eigenvalues of dF_d/dU are v_d +- c_f, v_d +- c_A, v_d +- c_slow, v_d and the GLM pair +-c_h:
    pins every term of the MHD+GLM flux and the fast speed together."""
    g = 5.0 / 3.0
    c = O.cfg(O.MHD_GLM, 3, gamma=g)
    rng = np.random.default_rng(10 + d)
    for _ in range(8):
        u = W.random_states(rng, 1, O.MHD_GLM, 3, g)[:, 0]
        w, ok = O.cons2prim(c, u)
        assert ok
        ch = 0.37
        ev = np.sort(np.linalg.eigvals(_jacobian(c, u, d, ch)).real)
        rho, p, B, vd = w[0], w[4], w[5:8], w[1 + d]
        a2, b2, bd2 = g * p / rho, (B @ B) / rho, B[d] ** 2 / rho
        disc = math.sqrt((a2 + b2) ** 2 - 4 * a2 * bd2)
        cf, cs, ca = math.sqrt(0.5 * (a2 + b2 + disc)), math.sqrt(0.5 * (a2 + b2 - disc)), math.sqrt(bd2)
        want = np.sort([vd - cf, vd - ca, vd - cs, vd, vd + cs, vd + ca, vd + cf, -ch, ch])
        np.testing.assert_allclose(ev, want, atol=2e-6)
        assert O.char_speed(c, w, d) == pytest.approx(abs(vd) + cf, rel=1e-13)


@pytest.mark.parametrize("ndim,d", [(1, 0), (2, 1), (3, 2)])
def test_flux_jacobian_spectrum_euler(ndim, d):
    g = 1.4
    c = O.cfg(O.EULER, ndim, gamma=g)
    rng = np.random.default_rng(20 + ndim)
    for _ in range(8):
        u = W.random_states(rng, 1, O.EULER, ndim, g)[:, 0]
        w, _ = O.cons2prim(c, u)
        a = math.sqrt(g * w[4] / w[0])
        vd = w[1 + d]
        ev = np.sort(np.linalg.eigvals(_jacobian(c, u, d, 0.0)).real)
        want = np.sort([vd - a] + [vd] * ndim + [vd + a])
        np.testing.assert_allclose(ev, want, atol=2e-6)


def test_mhd_without_field_is_euler_bitwise():
    """MHD+GLM with B = psi = 0 reduces to the Euler equations (1D: same alpha, c_h = alpha):
    one full SSPRK(5,4) step agrees bitwise on rho, m_x, E; B and psi stay zero."""
    w = W.sod(64)
    ce = O.cfg(O.EULER, 1, O.SSPRK54, 5.0 / 3.0)
    cm = O.cfg(O.MHD_GLM, 1, O.SSPRK54, 5.0 / 3.0)
    d = _odom(w.domains[0])
    rho, mx = w.U[0, 0, 0], w.U[1, 0, 0]
    p = (w.U[2, 0, 0] - 0.5 * mx * mx / rho) * (1.4 - 1.0)
    Ue = W.conserved_euler(rho, [mx / rho], p, 5.0 / 3.0).reshape(3, 1, 1, -1)
    z = np.zeros_like(rho)
    Um = W.conserved_mhd(rho, [mx / rho, z, z], p, [z, z, z], 5.0 / 3.0).reshape(9, 1, 1, -1)
    for _ in range(3):
        he, _ = O.dt(ce, d, Ue, 0.4)
        hm, _ = O.dt(cm, d, Um, 0.4)
        assert he == hm
        Ue, _, ae, _ = O.step(ce, d, Ue, he)
        Um, _, am, _ = O.step(cm, d, Um, hm)
        assert np.array_equal(ae[:, 0], am[:, 0])
        assert np.array_equal(Ue[0], Um[0]) and np.array_equal(Ue[1], Um[1]) and np.array_equal(Ue[2], Um[4])
        assert not np.any(Um[[2, 3, 5, 6, 7, 8]])


@pytest.mark.parametrize("physics,ndim", [(O.EULER, 2), (O.MHD_GLM, 3), (O.MHD_GLM, 1)])
def test_uniform_state_has_zero_residual(physics, ndim):
    rng = np.random.default_rng(3)
    g = 1.4 if physics == O.EULER else 5.0 / 3.0
    c = O.cfg(physics, ndim, gamma=g)
    u = W.random_states(rng, 1, physics, ndim, g)[:, 0]
    n = [7, 5, 6][:ndim]
    d = O.dom(n, [0.1, 0.2, 0.3][:ndim])
    shape = (O.nvar(c),) + tuple(([1] * (3 - ndim) + n[::-1]))
    U = np.broadcast_to(u.reshape(-1, 1, 1, 1), shape).copy()
    L, fl = O.residual(c, d, U, rng.uniform(1, 5, 3), ch=0.7)
    assert fl == 0 and np.all(L == 0.0)


# ------------------------------------------------------------------------- MP5
def test_mp5_hand_cases():
    for row in _golden("mp5_hand_cases.txt"):
        f = [float(x) for x in row[:5]]
        assert O.mp5(*f) == float(row[5]), row
        # the mirrored (right-biased) call on mirrored data gives the same value
        assert O.mp5(*f[::-1][:5]) == O.mp5(f[4], f[3], f[2], f[1], f[0])


def test_mp5_exact_on_quartic_cell_averages():
    """The unlimited stencil reproduces the face value of any quartic from its cell
    averages (which fixes all five coefficients); a quintic is not reproduced."""
    h = 0.05
    rng = np.random.default_rng(4)
    for deg in range(5):
        for _ in range(10):
            coef = np.zeros(6)
            coef[:deg + 1] = rng.uniform(-0.2, 0.2, deg + 1)
            coef[1] = 1.0 + abs(coef[1])  # monotone on the stencil, limiter inactive
            P = np.polynomial.Polynomial(coef)
            Pi = P.integ()
            x0 = rng.uniform(-1, 1)
            avg = [(Pi(x0 + (j + 0.5) * h) - Pi(x0 + (j - 0.5) * h)) / h for j in range(-2, 3)]
            face = P(x0 + 0.5 * h)
            assert O.mp5(*avg) == pytest.approx(face, rel=1e-13, abs=1e-13)
    P = np.polynomial.Polynomial([0, 1.0, 0, 0, 0, 5.0])
    Pi = P.integ()
    avg = [(Pi((j + 0.5) * h) - Pi((j - 0.5) * h)) / h for j in range(-2, 3)]
    assert abs(O.mp5(*avg) - P(0.5 * h)) > 1e-10


def test_mp5_monotone_and_step_data():
    """Monotonicity preservation: on monotone data the value stays in [f_i, f_{i+1}];
    on a step anywhere in the stencil no new extremum appears."""
    rng = np.random.default_rng(5)
    for _ in range(3000):
        f = np.sort(rng.normal(size=5)) * (1 if rng.random() < 0.5 else -1)
        r = O.mp5(*f)
        tol = 4e-16 * np.abs(f).max()  # f_or of uniform data is exact only up to rounding
        assert min(f[2], f[3]) - tol <= r <= max(f[2], f[3]) + tol
        k = rng.integers(0, 6)
        lo, hi = rng.normal(size=2)
        s = [lo] * k + [hi] * (5 - k)
        r = O.mp5(*s)
        tol = 4e-16 * max(abs(lo), abs(hi))
        assert min(lo, hi) - tol <= r <= max(lo, hi) + tol


def test_mp5_odd_symmetry_and_minmod():
    rng = np.random.default_rng(6)
    for _ in range(500):
        f = rng.normal(size=5)
        assert O.mp5(*(-f)) == -O.mp5(*f)
    assert O.minmod(1.0, 2.0) == 1.0 and O.minmod(-3.0, -2.0) == -2.0 and O.minmod(1.0, -1.0) == 0.0
    assert O.minmod(0.0, 5.0) == 0.0
    assert O.minmod4(1, 2, 3, 0.5) == 0.5 and O.minmod4(-1, -2, -3, -4) == -1 and O.minmod4(1, 2, -3, 4) == 0


# ------------------------------------------------------------------------ SSPRK
def _stability_poly(a, b):
    """R(z) of u' = lambda u, z = lambda dt, through the Shu-Osher stages (polynomial algebra)."""
    s = a.shape[0]
    stages = [np.polynomial.Polynomial([1.0])]
    z = np.polynomial.Polynomial([0.0, 1.0])
    for i in range(s):
        acc = np.polynomial.Polynomial([0.0])
        for k in range(i + 1):
            acc = acc + a[i, k] * stages[k] + b[i, k] * z * stages[k]
        stages.append(acc)
    return stages[-1].coef


def test_ssprk_tables_order_and_ssp_coefficient():
    s, a, b = O.ssprk_table(O.SSPRK3)
    assert s == 3
    np.testing.assert_allclose(_stability_poly(a, b), [1, 1, 1 / 2, 1 / 6], rtol=0, atol=1e-15)
    s, a, b = O.ssprk_table(O.SSPRK54)
    assert s == 5
    coef = _stability_poly(a, b)
    np.testing.assert_allclose(coef[:5], [1, 1, 1 / 2, 1 / 6, 1 / 24], rtol=0, atol=1e-10)
    gold = dict((r[0], r[1]) for r in _golden("ssprk54_ssp.txt"))
    s, a4, b4 = O.ssprk_table(O.SSPRK43)
    assert s == 4
    # SSPRK(4,3): third order, R(z) = 1 + z + z^2/2 + z^3/6 + z^4/48, SSP coefficient 2 (printed)
    np.testing.assert_allclose(_stability_poly(a4, b4), [1, 1, 1 / 2, 1 / 6, 1 / 48], rtol=0, atol=1e-15)
    r4 = [a4[i, k] / b4[i, k] for i in range(4) for k in range(4) if b4[i, k] != 0]
    assert min(r4) == float(gold["ssp_cfl_43"])
    ratios = [a[i, k] / b[i, k] for i in range(5) for k in range(5) if b[i, k] != 0]
    want = float(gold["ssp_cfl_54"])
    # the printed table is rounded to 14 digits, which moves the ratio by ~5e-11
    assert min(ratios) == pytest.approx(want, rel=1e-10)


@pytest.mark.parametrize("integrator,order", [(O.SSPRK3, 3), (O.SSPRK54, 4), (O.SSPRK43, 3)])
def test_step_temporal_order(integrator, order):
    """orc_step itself (stage storage and combination) converges in dt at the scheme's order."""
    w = W.sine_advection(24)
    c = O.cfg(O.EULER, 1, integrator, 1.4)
    d = _odom(w.domains[0])
    T = 0.25

    def run(k):
        U = w.U.copy()
        for _ in range(k):
            U, _, _, _ = O.step(c, d, U, T / k)
        return U

    ref = run(640)
    e = [np.abs(run(k) - ref).max() for k in (20, 40)]
    assert math.log2(e[0] / e[1]) == pytest.approx(order, abs=0.35)


# ---------------------------------------------------------------- whole solver
def test_sod_star_state_matches_textbook():
    gold = dict((r[0], float(r[1])) for r in _golden("sod_star.txt"))
    p, u = riemann.star_state(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    assert p == pytest.approx(gold["p_star"], abs=5e-6)
    assert u == pytest.approx(gold["u_star"], abs=5e-6)


def test_sod_against_exact_riemann():
    """L1 density error against the exact solution at t = 0.2 falls with resolution;
    at 512 cells it stays under 1.5x the value measured when this pin was set (1.09e-3)."""
    errs = []
    for n in (128, 256, 512):
        w = W.sod(n)
        c = _ocfg(w)
        U, t, ns, fl = O.evolve(c, _odom(w.domains[0]), w.U, w.cfl, w.t_end)
        assert fl == 0 and t == pytest.approx(0.2, abs=1e-14)
        x = w.extra["x"]
        r, _, _ = riemann.sample(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4, (x - 0.5) / 0.2)
        errs.append(np.mean(np.abs(U[0, 0, 0] - r)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1.5 * 1.09e-3


def test_sine_advection_fifth_order():
    """Smooth periodic advection: the L1 error of rho after one period falls at 5th order
    (MP5 with SSPRK(5,4) at a small CFL, as observed for the Alfven wave in Sec. 4.5.1)."""
    errs = []
    for n in (16, 32, 64):
        w = W.sine_advection(n)
        c = _ocfg(w)
        U, t, _, fl = O.evolve(c, _odom(w.domains[0]), w.U, 0.2, 1.0)
        errs.append(np.mean(np.abs(U[0] - w.U[0])))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert orders[-1] > 4.5, (errs, orders)


@pytest.mark.slow
def test_alfven_wave_convergence():
    """Circularly polarised Alfven wave (exact nonlinear solution, Sec. 4.5.1) on the
    diagonal of a periodic 2D box, one period with SSPRK(5,4) + MP5 + GLM: L1 error of
    the state vector falls at about fifth order (the paper measures 5 in 3D)."""
    errs = []
    for n in (16, 32, 64):
        w = W.alfven2d(n)
        c = _ocfg(w)
        U, t, _, fl = O.evolve(c, _odom(w.domains[0]), w.U, 0.2, w.t_end)
        assert fl == 0
        errs.append(np.mean(np.abs(U[:8] - w.U[:8])))
    order = math.log2(errs[1] / errs[2])
    assert order > 4.3, (errs, order)


def test_conservation_periodic():
    """Telescoping flux differences: totals of rho, m, E, B change only by roundoff."""
    w = W.batched(nblocks=3, seed_index=3)
    c = _ocfg(w)
    for dd in w.domains:
        U = w.U[dd.offset:dd.offset + 9 * dd.ncell].reshape(9, *dd.n[::-1]).copy()
        od = _odom(dd)
        tot0 = [math.fsum(U[v].ravel()) for v in range(8)]
        scale = [math.fsum(np.abs(U[v]).ravel()) for v in range(8)]
        h, _ = O.dt(c, od, U, 0.4)
        for _ in range(2):
            U, fl, _, _ = O.step(c, od, U, h)
            assert fl == 0
        for v in range(8):
            sc = max(scale[v], math.fsum(np.abs(U[v]).ravel()))
            assert abs(math.fsum(U[v].ravel()) - tot0[v]) <= 2e-13 * sc


def test_mirror_symmetry():
    """Data even under x -> -x with m_x, B_x odd stays so (ideal MHD is invariant under the
    reflection combined with B -> -B): 20 SSPRK3 steps of the 2D vortex at 32^2."""
    n = 32
    w = W.vortex2d(n, integrator=O.SSPRK3)
    U = w.U.copy()
    # make the data mirror-symmetric about x = pi by symmetrising it
    sgn = np.array([1, -1, 1, 1, 1, -1, 1, 1, 1]).reshape(9, 1, 1, 1)
    U = 0.5 * (U + sgn * U[..., ::-1])
    c = _ocfg(w)
    d = _odom(w.domains[0])
    for _ in range(20):
        h, _ = O.dt(c, d, U, 0.4)
        U, fl, _, _ = O.step(c, d, U, h)
        assert fl == 0
    err = np.abs(U - sgn * U[..., ::-1]).max() / np.abs(U).max()
    assert err <= 1e-13


def test_passive_blocks_frozen_and_excluded():
    """Passive blocks keep their state bitwise and do not enter c_max or dt (App. C)."""
    w = W.blast3d(16, 8)
    c = _ocfg(w)
    d = _odom(w.domains[0])
    act = np.array([1, 0, 1, 1, 0, 1, 1, 1], np.uint8)
    h, _ = O.dt(c, d, w.U, 0.3, active=act)
    U, fl, al, ch = O.step(c, d, w.U, h, active=act)
    assert fl == 0
    blk = w.U.reshape(9, 2, 8, 2, 8, 2, 8)
    nblk = U.reshape(9, 2, 8, 2, 8, 2, 8)
    for b in range(8):
        bz, by, bx = b // 4, (b // 2) % 2, b % 2
        same = np.array_equal(blk[:, bz, :, by, :, bx], nblk[:, bz, :, by, :, bx])
        assert same == (act[b] == 0)
    # alpha over active cells only: making a passive block extreme changes nothing
    U2 = w.U.copy().reshape(9, 2, 8, 2, 8, 2, 8)
    U2[4, 0, :, 0, :, 1] *= 50.0  # block 1 (passive): huge energy
    a1, r1, _ = O.speeds(c, d, w.U, act)
    a2, r2, _ = O.speeds(c, d, U2.reshape(w.U.shape), act)
    assert np.array_equal(a1, a2) and r1 == r2


def test_dt_closed_form_uniform():
    """Uniform state: Euler dt = CFL / sum_d (|v_d| + a)/dx_d; GLM dt = CFL / (c_h sum_d 1/dx_d)."""
    g = 1.4
    c = O.cfg(O.EULER, 2, gamma=g)
    d = O.dom([6, 5], [0.1, 0.3])
    rho, p, v = 1.3, 0.7, (0.4, -0.9)
    u = W.conserved_euler(np.array(rho), [np.array(x) for x in v], np.array(p), g)
    U = np.broadcast_to(u.reshape(-1, 1, 1, 1), (4, 1, 5, 6)).copy()
    a = math.sqrt(g * p / rho)
    want = 0.4 / ((abs(v[0]) + a) / 0.1 + (abs(v[1]) + a) / 0.3)
    h, fl = O.dt(c, d, U, 0.4)
    assert h == pytest.approx(want, rel=1e-14)
    assert O.dt(c, d, U, 0.4, t=0.0, t_end=1e-5)[0] == 1e-5
    cm = O.cfg(O.MHD_GLM, 2, gamma=5 / 3)
    um = W.conserved_mhd(np.array(rho), [np.array(0.4), np.array(-0.9), np.array(0.0)], np.array(p),
                         [np.array(0.3), np.array(0.5), np.array(0.2)], 5 / 3)
    Um = np.broadcast_to(um.reshape(-1, 1, 1, 1), (9, 1, 5, 6)).copy()
    wm, _ = O.cons2prim(cm, um)
    chh = max(O.char_speed(cm, wm, 0), O.char_speed(cm, wm, 1))
    assert O.dt(cm, d, Um, 0.4)[0] == pytest.approx(0.4 / (chh / 0.1 + chh / 0.3), rel=1e-14)


# ------------------------------------------------------------- GLM psi damping
def _uniform_mhd(rho, v, p, B, psi, n, g):
    u = W.conserved_mhd(np.array(rho), [np.array(x) for x in v], np.array(p), [np.array(x) for x in B], g,
                        np.array(psi))
    shape = (9,) + tuple(n[::-1])
    return u, np.broadcast_to(u.reshape(-1, 1, 1, 1), shape).copy()


@pytest.mark.parametrize("integrator", [O.SSPRK3, O.SSPRK54])
def test_psi_damping_closed_form_on_uniform_state(integrator):
    """Sec. 4.2: the GLM source -(c_h^2/c_p^2) psi, integrated exactly after the step with
    c_p^2/c_h = c_r, multiplies psi by exp(-dt c_h/c_r) once per step. A uniform state has
    L(U) = 0, so only the damping moves it. With B along x and v along z, c_h has a closed
    form: the z fast speed is the perpendicular one, sqrt(a^2 + b^2), and it is the largest
    of the three: c_h = |v_z| + sqrt(gamma p/rho + B_x^2/rho)."""
    g = 5.0 / 3.0
    rho, vz, p, bx, psi0, dt, cr = 1.25, -0.375, 0.5, 0.75, 0.125, 0.01, 0.18
    c = O.cfg(O.MHD_GLM, 3, integrator=integrator, gamma=g, glm_cr=cr)
    n = [4, 5, 6]
    d = O.dom(n, [0.1, 0.2, 0.3])
    u, U = _uniform_mhd(rho, (0.0, 0.0, vz), p, (bx, 0.0, 0.0), psi0, n, g)
    ch = abs(vz) + math.sqrt(g * p / rho + bx * bx / rho)
    Un, fl, _, ch_or = O.step(c, d, U, dt)
    assert fl == 0
    assert ch_or == pytest.approx(ch, rel=1e-15)
    want = psi0 * math.exp(-dt * ch / cr)
    np.testing.assert_allclose(Un[8], want, rtol=1e-14, atol=0)
    # a damping with the wrong exponent, once per stage, or not at all lies far outside
    assert abs(want - psi0 * math.exp(-dt * ch * cr)) > 1e-4 * psi0
    assert abs(want - psi0 * math.exp(-3 * dt * ch / cr)) > 1e-4 * psi0
    for v in range(8):
        np.testing.assert_allclose(Un[v], u[v], rtol=1e-14, atol=1e-15)
    # c_r <= 0 switches the damping off: psi stays (up to the stage sums' rounding)
    c0 = O.cfg(O.MHD_GLM, 3, integrator=integrator, gamma=g, glm_cr=0.0)
    U0, fl0, _, _ = O.step(c0, d, U, dt)
    assert fl0 == 0
    np.testing.assert_allclose(U0[8], psi0, rtol=1e-14, atol=0)


def test_psi_damping_uses_speed_of_step_start_once():
    """On non-uniform data the damping is the only difference between c_r > 0 and c_r <= 0:
    every other variable is bitwise the same, and psi differs by one factor
    exp(-dt c_h/c_r) with c_h the largest splitting speed of U^n (not of a later stage),
    applied once after the last stage."""
    w = W.vortex2d(32)
    c = _ocfg(w)
    d = _odom(w.domains[0])
    U = w.U.reshape(9, 1, 32, 32).copy()
    U[8] = 0.05 * np.sin(np.linspace(0.0, 7.0, 32 * 32)).reshape(1, 32, 32)
    h = 0.5 * O.dt(c, d, U, w.cfl)[0]
    cd = O.cfg(w.physics, w.ndim, w.integrator, w.gamma, 0.18)
    cz = O.cfg(w.physics, w.ndim, w.integrator, w.gamma, 0.0)
    Ud, fl1, _, ch = O.step(cd, d, U, h)
    Uz, fl2, _, _ = O.step(cz, d, U, h)
    assert fl1 == 0 and fl2 == 0
    assert np.array_equal(Ud[:8], Uz[:8])
    araw0, _, _ = O.speeds(cd, d, U)
    assert ch == max(araw0[:2])
    fac = math.exp(-h * ch / 0.18)
    nz = np.abs(Uz[8]) > 1e-6
    np.testing.assert_allclose(Ud[8][nz] / Uz[8][nz], fac, rtol=2e-16 * 4, atol=0)
    # the speeds of the step's end state differ from U^n's by far more than the tolerance
    # resolves, so a damping taken with a later state's c_h would fail the ratio above
    araw1, _, _ = O.speeds(cd, d, Ud)
    fac1 = math.exp(-h * max(araw1[:2]) / 0.18)
    assert abs(fac1 - fac) > 1e3 * 2e-16 * fac


def _mirror_double(U, axis, sgn):
    """Periodic data of twice the length: U followed by its mirror image times sgn."""
    return np.concatenate([U, sgn * np.flip(U, axis=axis)], axis=axis)


# (physics, ndim, mirror dimension, odd variables): reflections under which the
# equations are invariant -- Euler: the normal momentum; MHD (B a pseudovector):
# the normal momentum, the tangential field and psi (whose flux is c_h^2 B_d)
MIRROR_CASES = [
    (O.EULER, 1, 0, [1]),
    (O.EULER, 3, 2, [3]),
    (O.MHD_GLM, 2, 1, [2, 5, 7, 8]),
    (O.MHD_GLM, 2, 0, [1, 6, 7, 8]),
]


@pytest.mark.parametrize("physics,ndim,md,odd", MIRROR_CASES)
def test_symmetric_walls_equal_mirror_doubled_periodic_domain(physics, ndim, md, odd):
    """A domain with mirror (symmetric/antisymmetric) ghosts on both faces of dimension md
    evolves exactly like the first half of the periodic domain of twice the length holding
    the data followed by its mirror image: both see the same values at every face, and the
    update commutes with the reflection. Five SSPRK3 steps, compared bitwise."""
    rng = np.random.default_rng(40 + md + 10 * physics)
    g = 1.4 if physics == O.EULER else 5 / 3
    n = [12 if k < ndim else 1 for k in range(3)]
    n[md] = 10
    shape = (n[2], n[1], n[0])
    rho = 1.0 + 0.3 * rng.random(shape)
    p = 1.0 + 0.3 * rng.random(shape)
    vel = [0.5 * rng.standard_normal(shape) for _ in range(3)]
    if physics == O.EULER:
        U = W.conserved_euler(rho, vel[:ndim], p, g)
    else:
        U = W.conserved_mhd(rho, vel, p, [0.6 + 0.2 * rng.standard_normal(shape) for _ in range(3)], g,
                            psi=0.05 * rng.standard_normal(shape))
    nv = U.shape[0]
    sgn = np.ones((nv, 1, 1, 1))
    sgn[odd] = -1.0
    mask = sum(1 << v for v in odd)
    axis = 3 - md
    bc = [[O.PERIODIC, O.PERIODIC] for _ in range(3)]
    bc[md] = [O.SYMMETRIC, O.SYMMETRIC]
    asym = [[0, 0] for _ in range(3)]
    asym[md] = [mask, mask]
    dx = [0.1, 0.07, 0.05]
    c = O.cfg(physics, ndim, O.SSPRK3, g)
    dw = O.dom(n, dx, bc=bc, asym=asym)
    n2 = list(n)
    n2[md] *= 2
    dp = O.dom(n2, dx)
    Uw, Up = U.copy(), _mirror_double(U, axis, sgn)
    for _ in range(5):
        hw, _ = O.dt(c, dw, Uw, 0.4)
        hp, _ = O.dt(c, dp, Up, 0.4)
        assert hw == hp
        Uw, fw, _, _ = O.step(c, dw, Uw, hw)
        Up, fp, _, _ = O.step(c, dp, Up, hp)
        assert fw == 0 and fp == 0
    half = np.split(Up, 2, axis=axis)[0]
    assert np.array_equal(Uw, half)
    # and the doubled run itself kept its mirror symmetry
    assert np.array_equal(Up, _mirror_double(half, axis, sgn))


def test_symmetric_ghost_kinds_differ_from_outflow():
    """Mirror ghosts are not the zero-gradient copy: with a flow into the wall the
    reflecting face builds up pressure, the outflow face lets the flow leave."""
    n = 32
    U = W.conserved_euler(np.ones(n), [np.full(n, 0.5)], np.ones(n), 1.4).reshape(3, 1, 1, n)
    c = O.cfg(O.EULER, 1)
    dw = O.dom([n], [1.0 / n], bc=[[O.OUTFLOW, O.SYMMETRIC], [0, 0], [0, 0]], asym=[[0, 2], [0, 0], [0, 0]])
    do = O.dom([n], [1.0 / n], bc=O.OUTFLOW)
    Uw, Uo = U.copy(), U.copy()
    for _ in range(10):
        Uw, _, _, _ = O.step(c, dw, Uw, 0.2 / n)
        Uo, _, _, _ = O.step(c, do, Uo, 0.2 / n)
    assert np.array_equal(Uo, U)                    # uniform outflow state is exactly steady
    assert Uw[0, 0, 0, -1] > 1.05 and abs(Uw[1, 0, 0, -1]) < 0.5 * 0.5  # compressed, slowed at the wall


def test_brio_wu_contact_overshoot_matches_paper_magnitude():
    """Sec. 4.5.2: SSPRK(5,4)-MP5-FD overshoots the density at the contact of the
    Brio-Wu tube by +2.7% (512 cells on [-1,1]). The plateau left of the contact is taken
    from the same scheme at 1024 cells (the mean over 0 < x < 0.09 at t = 0.2); the
    overshoot is the maximum of the 512-cell density near the contact relative to it.
    This reading gives +2.1-2.2% (the paper's reference was a 65536-cell TVD run and
    the time is not printed); the pin holds the sign and magnitude: 1% .. 4%."""
    def run(n):
        w = W.brio_wu(n)
        c = _ocfg(w)
        d = _odom(w.domains[0])
        U, _, _, fl = O.evolve(c, d, w.U, 0.4, w.t_end)
        assert fl == 0
        return w.extra["x"], U[0, 0, 0]
    x, r = run(512)
    xr, rr = run(1024)
    plateau = rr[(xr > 0.0) & (xr < 0.09)].mean()
    over = r[(x > 0.05) & (x < 0.14)].max() / plateau - 1.0
    assert 0.01 <= over <= 0.04, over


# ------------------------------------------------------- dynamic activation (App. C)
def _chebyshev_activate(d, flag, belt):
    """Independent statement of the belt: a block is active when some unflagged block lies
    within Chebyshev distance <= belt (block units; distances wrap across periodic faces)."""
    nb = [d.nb[k] for k in range(3)]
    idx = np.array([(b % nb[0], (b // nb[0]) % nb[1], b // (nb[0] * nb[1])) for b in range(np.prod(nb))])
    src = idx[np.asarray(flag) == 0]
    out = np.zeros(len(idx), np.uint8)
    for b, i in enumerate(idx):
        if len(src) == 0:
            break
        dist = np.abs(src - i)
        for k in range(3):
            if d.bc[k][0] == O.PERIODIC:
                dist[:, k] = np.minimum(dist[:, k], nb[k] - dist[:, k])
        out[b] = np.any(dist.max(axis=1) <= belt)
    return out


def test_activate_hand_cases():
    d = O.dom([40], [0.1], bc=O.OUTFLOW, nb=(10, 1, 1))
    flag = np.ones(10, np.uint8)
    flag[4] = 0
    assert O.activate(d, flag, 0).tolist() == [0, 0, 0, 0, 1, 0, 0, 0, 0, 0]
    assert O.activate(d, flag, 1).tolist() == [0, 0, 0, 1, 1, 1, 0, 0, 0, 0]
    assert O.activate(d, flag, 2).tolist() == [0, 0, 1, 1, 1, 1, 1, 0, 0, 0]
    flag = np.ones(10, np.uint8)
    flag[0] = 0
    assert O.activate(d, flag, 1).tolist() == [1, 1, 0, 0, 0, 0, 0, 0, 0, 0]  # no wrap at outflow
    dp = O.dom([40], [0.1], bc=O.PERIODIC, nb=(10, 1, 1))
    assert O.activate(dp, flag, 1).tolist() == [1, 1, 0, 0, 0, 0, 0, 0, 0, 1]  # wrap
    # a corner neighbour counts
    d3 = O.dom([12, 12, 12], [0.1] * 3, bc=O.OUTFLOW, nb=(3, 3, 3))
    f3 = np.ones(27, np.uint8)
    f3[0] = 0
    a3 = O.activate(d3, f3, 1).reshape(3, 3, 3)
    assert a3[1, 1, 1] == 1 and a3[2, 2, 2] == 0 and a3[:2, :2, :2].all() and a3.sum() == 8


@pytest.mark.parametrize("seed", range(4))
def test_activate_equals_chebyshev_distance_rule(seed):
    rng = np.random.default_rng(seed)
    nb = [int(x) for x in rng.integers(1, 7, 3)]
    bc = [[int(b)] * 2 for b in rng.integers(0, 3, 3)]
    d = O.dom([4 * x for x in nb], [0.1] * 3, bc=bc, nb=nb)
    flag = (rng.random(int(np.prod(nb))) > 0.08).astype(np.uint8)
    for belt in range(4):
        assert np.array_equal(O.activate(d, flag, belt), _chebyshev_activate(d, flag, belt)), (belt, nb, bc)


def test_flag_steady_blockwise():
    w = W.blast3d(16, 8)
    c = _ocfg(w)
    d = _odom(w.domains[0])
    R = w.U.copy()
    U = R.copy()
    assert O.flag_steady(c, d, U, R, 0.0).tolist() == [1] * 8
    U[4, 3, 9, 2] += 1e-9         # block (x 0, y 1, z 0) = 2
    U[8, 12, 12, 12] = np.nan     # block 7
    assert O.flag_steady(c, d, U, R, 1e-10).tolist() == [1, 1, 0, 1, 1, 1, 1, 0]
    assert O.flag_steady(c, d, U, R, 1e-8).tolist() == [1, 1, 1, 1, 1, 1, 1, 0]


# ---------------------------------------------------------------- LIMO3 (Sec. 2.2, 4.5)
def test_limo3_unlimited_is_exact_for_quadratic_cell_averages():
    """Inside the asymptotic region (eta < 1) LIMO3 is the unlimited third-order
    reconstruction: exact face values from cell averages of any quadratic."""
    rng = np.random.default_rng(5)
    h = 0.1
    for _ in range(50):
        a, b, c = rng.standard_normal(3)

        def avg(x0):  # average of a + b x + c x^2 over [x0, x0 + h]
            F = lambda x: a * x + b * x * x / 2 + c * x ** 3 / 3  # noqa: E731
            return (F(x0 + h) - F(x0)) / h
        x0 = rng.uniform(-1, 1)
        um, u0, up = avg(x0 - h), avg(x0), avg(x0 + h)
        face = a + b * (x0 + h) + c * (x0 + h) ** 2
        got = O.limo3(um, u0, up, 1e6)
        assert abs(got - face) <= 1e-12 * max(1.0, abs(face))
        # the right-biased value at the same face from the cells on its right
        face_l = a + b * x0 + c * x0 * x0
        assert abs(O.limo3(up, u0, um, 1e6) - face_l) <= 1e-12 * max(1.0, abs(face_l))


def test_limo3_limited_properties():
    """Outside the asymptotic region (eta > 1) the limited function: values of monotone
    data stay between u_i and u_{i+1}; smooth profiles (theta in [0.4, 2.8], and smooth
    extrema with theta in [-2, -0.8]) keep the third-order value; steps and sharp
    extrema (theta <= -2) give u_i; a flat right neighbour gives u_i; the slope is
    capped at 1.6 delta_+ / 2 for steep left data; odd and translation symmetric."""
    rng = np.random.default_rng(6)
    tiny = 1e-9  # r dx: eta >> 1
    for _ in range(200):
        u0 = rng.standard_normal()
        dp = rng.uniform(0.1, 2.0) * rng.choice([-1, 1])
        th = rng.uniform(-4, 6)
        um, up = u0 - th * dp, u0 + dp
        v = O.limo3(um, u0, up, tiny)
        full = O.limo3(um, u0, up, 1e9)
        if th >= 0:
            assert min(u0, up) - 1e-15 <= v <= max(u0, up) + 1e-15
        if 0.4 <= th <= 2.8 or -2 <= th <= -0.8:
            assert abs(v - full) <= 1e-13
        if th <= -2:
            assert v == u0
        if th >= 3.0:
            assert abs(v - (u0 + 0.8 * dp)) <= 1e-13
        assert abs(O.limo3(-um, -u0, -up, tiny) + v) <= 1e-15
        assert abs(O.limo3(um + 3.0, u0 + 3.0, up + 3.0, tiny) - (v + 3.0)) <= 1e-13
    assert O.limo3(0.0, 0.0, 1.0, tiny) == 0.0      # theta = 0: first-order at the step
    assert O.limo3(0.0, 1.0, 1.0, tiny) == 1.0      # delta_+ = 0


def test_limo3_rk3_third_order():
    """RK3 + LIMO3 on smooth periodic advection converges at third order (Sec. 4.5.1
    reports third order for this pairing on the Alfven wave)."""
    errs = []
    for n in (32, 64, 128):
        w = W.sine_advection(n)
        c = O.cfg(w.physics, w.ndim, O.SSPRK3, w.gamma, recon=O.LIMO3, limo3_r=1.0)
        U, t, _, fl = O.evolve(c, _odom(w.domains[0]), w.U, 0.4, 1.0)
        assert fl == 0
        errs.append(np.mean(np.abs(U[0] - w.U[0])))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(2.8 < o < 3.3 for o in orders), (errs, orders)


def test_brio_wu_limo3_contact_and_max_ssp_cfl():
    """Sec. 4.5.2: RK3-LIM03-FD barely moves the contact density (-0.001% in the paper;
    this reading: a small undershoot, within -1% .. +0.5% of the 1024-cell MP5 plateau),
    and SSPRK(4,3)-LIMO3 runs the tube at its SSP limit, CFL 2.0, staying physical."""
    def run(n, integ, recon, cfl):
        w = W.brio_wu(n)
        c = O.cfg(w.physics, w.ndim, integ, w.gamma, w.glm_cr, recon=recon, limo3_r=1.0)
        U, _, ns, fl = O.evolve(c, _odom(w.domains[0]), w.U, cfl, w.t_end)
        assert fl == 0
        return w.extra["x"], U, ns
    xr, Ur, _ = run(1024, O.SSPRK54, O.MP5, 0.4)
    plateau = Ur[0, 0, 0][(xr > 0.0) & (xr < 0.09)].mean()
    x, U, _ = run(512, O.SSPRK3, O.LIMO3, 0.4)
    over = U[0, 0, 0][(x > 0.05) & (x < 0.14)].max() / plateau - 1.0
    assert -0.01 <= over <= 0.005, over
    x, U, ns = run(512, O.SSPRK43, O.LIMO3, 2.0)
    assert ns < 110 and U[0].min() > 0.1 and U[0].max() < 1.01
