"""Seeded synthetic initial conditions for the FD-MP5 update (numpy only).

This module is the one thing the CUDA path and the CPU oracle share: it
builds input arrays and nothing else. It holds none of the update's
arithmetic; the only physics here is the definition of the conserved state,
E = p/(gamma-1) + rho v^2/2 + B^2/2 (Porth et al. 2014, Sec. 3 and 4.3),
used to turn primitive initial data into conserved variables.

Layout of a domain: U[v][z][y][x] (x fastest), interior cells only.
  Euler   (nv = 2 + ndim): rho, m_1..m_ndim, E
  MHD+GLM (nv = 9):        rho, m_x, m_y, m_z, E, B_x, B_y, B_z, psi
Seeds are numpy default_rng(14072052 + k), k = the workload's index in the
list below (sod 0, vortex 1, blast 2, batched 3, adjoint 4).
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SEED0 = 14072052
EULER, MHD_GLM = 0, 1
SSPRK3, SSPRK54, SSPRK43 = 0, 1, 2
PERIODIC, OUTFLOW, SYMMETRIC = 0, 1, 2


@dataclass
class Domain:
    n: tuple            # interior cells (nx, ny, nz)
    dx: tuple           # cell sizes
    bc: tuple = ((PERIODIC, PERIODIC),) * 3
    nb: tuple = (1, 1, 1)  # blocks per dimension
    offset: int = 0     # element offset of this domain in a batched state buffer
    asym: tuple = ((0, 0),) * 3  # SYMMETRIC faces: bit mask of the odd variables

    @property
    def ncell(self):
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])


@dataclass
class Workload:
    name: str
    physics: int
    ndim: int
    integrator: int
    gamma: float
    cfl: float
    domains: List[Domain]
    U: np.ndarray                     # state: one domain (nv, nz, ny, nx) or flat batched buffer
    active: Optional[np.ndarray] = None  # uint8 per block (all blocks of all domains, in order)
    glm_cr: float = 0.18
    t_end: float = 0.0
    recon: int = 0                    # 0 MP5, 1 LIMO3
    limo3_r: float = 1.0
    nsteps: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def nv(self):
        return 2 + self.ndim if self.physics == EULER else 9


def conserved_euler(rho, vel, p, gamma):
    """(rho, m_1..m_ndim, E) from primitives; vel is a list of ndim arrays."""
    ekin = 0.5 * rho * sum(v * v for v in vel)
    return np.stack([rho] + [rho * v for v in vel] + [p / (gamma - 1.0) + ekin])


def conserved_mhd(rho, vel, p, B, gamma, psi=None):
    """(rho, m, E, B, psi) from primitives; vel, B are 3-lists of arrays."""
    ekin = 0.5 * rho * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)
    emag = 0.5 * (B[0] ** 2 + B[1] ** 2 + B[2] ** 2)
    psi = np.zeros_like(rho) if psi is None else psi
    return np.stack([rho, rho * vel[0], rho * vel[1], rho * vel[2],
                     p / (gamma - 1.0) + ekin + emag, B[0], B[1], B[2], psi])


def centres(n, lo, hi):
    dx = (hi - lo) / n
    return lo + (np.arange(n) + 0.5) * dx, dx


# ---------------------------------------------------------------- workloads
def sod(n=512):
    """1D Euler Sod tube on [0,1], gamma 1.4, outflow, SSPRK3, CFL 0.4, t = 0.2."""
    x, dx = centres(n, 0.0, 1.0)
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    U = conserved_euler(rho, [np.zeros(n)], p, 1.4).reshape(3, 1, 1, n)
    dom = Domain((n, 1, 1), (dx, 1.0, 1.0), bc=((OUTFLOW, OUTFLOW),) * 3)
    return Workload("sod1d", EULER, 1, SSPRK3, 1.4, 0.4, [dom], U, t_end=0.2,
                    extra={"x": x})


def closed_sod(n=400):
    """Sod's data in a closed tube [0,1] with reflecting walls at both ends (mirror
    ghosts, m_x odd), SSPRK3, CFL 0.4, t = 0.4: the shock reflects off x = 1."""
    w = sod(n)
    d = w.domains[0]
    dom = Domain(d.n, d.dx, bc=((SYMMETRIC, SYMMETRIC),) + d.bc[1:], asym=((2, 2), (0, 0), (0, 0)))
    return Workload("closed_sod", EULER, 1, SSPRK3, 1.4, 0.4, [dom], w.U, t_end=0.4, extra=w.extra)


# reflecting wall normal to y for MHD+GLM: m_y, B_x, B_z and psi odd (B a pseudovector)
MHD_WALL_Y = (1 << 2) | (1 << 5) | (1 << 7) | (1 << 8)


def wall_blast2d(n=128, block=32, integrator=SSPRK3, seed_index=5):
    """2D MHD+GLM blast next to reflecting walls: [-0.5,0.5]^2, periodic in x, mirror
    walls at y = -0.5 and 0.5; p = 10 inside r < 0.1 around (0.1, -0.35), 0.1 outside;
    rho = 1 (1 + 1e-3 (2u - 1)), B = (1, 1, 0)/sqrt(2), gamma 5/3, CFL 0.3."""
    rng = np.random.default_rng(SEED0 + seed_index)
    x, dx = centres(n, -0.5, 0.5)
    X, Y = np.meshgrid(x, x, indexing="xy")
    r = np.hypot(X - 0.1, Y + 0.35)
    rho = 1.0 + 1e-3 * (2.0 * rng.random((n, n)) - 1.0)
    p = np.where(r < 0.1, 10.0, 0.1)
    zero = np.zeros_like(rho)
    b = 1.0 / np.sqrt(2.0)
    U = conserved_mhd(rho, [zero, zero, zero], p, [zero + b, zero + b, zero], 5.0 / 3.0).reshape(9, 1, n, n)
    nb = n // block
    dom = Domain((n, n, 1), (dx, dx, 1.0), bc=((PERIODIC, PERIODIC), (SYMMETRIC, SYMMETRIC), (PERIODIC, PERIODIC)),
                 nb=(nb, nb, 1), asym=((0, 0), (MHD_WALL_Y, MHD_WALL_Y), (0, 0)))
    return Workload("wall_blast2d", MHD_GLM, 2, integrator, 5.0 / 3.0, 0.3, [dom], U,
                    active=np.ones(nb * nb, np.uint8))


def vortex2d(n=1024, integrator=SSPRK54):
    """2D MHD+GLM smooth vortex on periodic [0,2pi]^2, gamma 5/3."""
    x, dx = centres(n, 0.0, 2 * np.pi)
    X, Y = np.meshgrid(x, x, indexing="xy")  # [y][x]
    rho = np.full_like(X, 25.0 / 9.0)
    p = np.full_like(X, 5.0 / 3.0)
    vel = [-np.sin(Y), np.sin(X), np.zeros_like(X)]
    B = [-np.sin(Y), np.sin(2 * X), np.zeros_like(X)]
    U = conserved_mhd(rho, vel, p, B, 5.0 / 3.0).reshape(9, 1, n, n)
    dom = Domain((n, n, 1), (dx, dx, 1.0))
    return Workload("vortex2d", MHD_GLM, 2, integrator, 5.0 / 3.0, 0.4, [dom], U, nsteps=500)


def blast3d(n=256, block=16, seed_index=2, noise=1e-3):
    """3D MHD+GLM blast on periodic [-0.5,0.5]^3, gamma 5/3, SSPRK3, CFL 0.3.
    noise = 0 gives a uniform background, exactly steady away from the blast (the
    dynamic-activation case of App. C)."""
    rng = np.random.default_rng(SEED0 + seed_index)
    x, dx = centres(n, -0.5, 0.5)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    rho = 1.0 * (1.0 + noise * (2.0 * rng.random((n, n, n)) - 1.0))
    p = np.where(r < 0.1, 10.0, 0.1)
    zero = np.zeros_like(rho)
    b = 1.0 / np.sqrt(2.0)
    U = conserved_mhd(rho, [zero, zero, zero], p, [zero + b, zero + b, zero], 5.0 / 3.0)
    nb = n // block
    dom = Domain((n, n, n), (dx, dx, dx), nb=(nb, nb, nb))
    extra = {}
    if noise == 0.0:  # the stationary background the blast runs into
        extra["background"] = conserved_mhd(zero + 1.0, [zero, zero, zero], zero + 0.1, [zero + b, zero + b, zero],
                                            5.0 / 3.0)
    return Workload("blast3d", MHD_GLM, 3, SSPRK3, 5.0 / 3.0, 0.3, [dom], U, nsteps=200,
                    active=np.ones(nb ** 3, np.uint8), extra=extra)


def _kset3():
    return np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)
                     if (a, b, c) != (0, 0, 0)])


def batched(nblocks=20000, sizes=(8, 12, 16, 24, 32), passive_frac=0.3, seed_index=3):
    """Independent periodic 3D MHD+GLM blocks of uneven sizes, each its own domain.

    Interior edge m drawn per block from `sizes`; dx log-uniform in [1e-3, 1e-1];
    background rho = 1, p = 1, v = 0, B = (0.5, 0, 0); rho and p get (1 + delta),
    each velocity component + delta, where every delta is a fresh draw of
        0.05 * sum_{j=1..8} c_j sin(2 pi k_j . x / L + phi_j),
    k_j uniform in {-1,0,1}^3 minus 0, c_j ~ U[-1,1]/8, phi_j ~ U[0, 2 pi), L = m dx
    (so the phase only depends on the cell index); B uniform; a seeded Bernoulli
    draw flags `passive_frac` of the blocks passive. Blocks are stored one after
    another (domain offsets), each as U[v][z][y][x]."""
    rng = np.random.default_rng(SEED0 + seed_index)
    ks = _kset3()
    edges = rng.choice(np.asarray(sizes), size=nblocks)
    dxs = np.exp(rng.uniform(np.log(1e-3), np.log(1e-1), size=nblocks))
    active = (rng.random(nblocks) >= passive_frac).astype(np.uint8)
    nf, nm = 5, 8  # perturbed fields (rho, p, vx, vy, vz), modes per field
    kidx = rng.integers(len(ks), size=(nblocks, nf, nm))
    cj = rng.uniform(-1.0, 1.0, size=(nblocks, nf, nm)) / nm
    ph = rng.uniform(0.0, 2 * np.pi, size=(nblocks, nf, nm))
    # sin(theta_k + phi) = sin(theta_k) cos(phi) + cos(theta_k) sin(phi): per block and field the
    # perturbation is a weighted sum of the 2 x 26 basis fields sin/cos(2 pi k . (i + 1/2) / m)
    wts = np.zeros((nblocks, nf, 2 * len(ks)))
    rows = np.arange(nblocks)[:, None, None]
    fld = np.arange(nf)[None, :, None]
    np.add.at(wts, (rows, fld, kidx), cj * np.cos(ph))
    np.add.at(wts, (rows, fld, kidx + len(ks)), cj * np.sin(ph))
    offs = np.zeros(nblocks, dtype=np.int64)
    ncell = edges.astype(np.int64) ** 3
    offs[1:] = np.cumsum(9 * ncell)[:-1]
    U = np.empty(int(9 * ncell.sum()))
    for m in sizes:
        sel = np.flatnonzero(edges == m)
        if sel.size == 0:
            continue
        t = 2 * np.pi * (np.arange(m) + 0.5) / m
        Z, Y, X = np.meshgrid(t, t, t, indexing="ij")
        arg = ks[:, 0, None] * X.ravel()[None] + ks[:, 1, None] * Y.ravel()[None] + ks[:, 2, None] * Z.ravel()[None]
        basis = np.concatenate([np.sin(arg), np.cos(arg)])  # (52, m^3)
        for c0 in range(0, sel.size, 512):
            part = sel[c0:c0 + 512]
            delta = 0.05 * (wts[part].reshape(-1, basis.shape[0]) @ basis).reshape(part.size, nf, m ** 3)
            rho = 1.0 + delta[:, 0]
            p = 1.0 + delta[:, 1]
            vel = [delta[:, 2], delta[:, 3], delta[:, 4]]
            zero = np.zeros_like(rho)
            blk = conserved_mhd(rho, vel, p, [zero + 0.5, zero, zero], 5.0 / 3.0)  # (9, nb, m^3)
            blk = np.ascontiguousarray(blk.transpose(1, 0, 2))
            for q, b in enumerate(part):
                U[offs[b]:offs[b] + 9 * m ** 3] = blk[q].ravel()
    doms = [Domain((int(m), int(m), int(m)), (float(dxs[i]),) * 3, offset=int(offs[i]))
            for i, m in enumerate(edges)]
    return Workload("batched3d", MHD_GLM, 3, SSPRK3, 5.0 / 3.0, 0.4, doms, U, active=active)


def adjoint2d(n=512, seed_index=4, nmodes=16, amp=0.02):
    """2D MHD+GLM on periodic [0,2pi]^2, smooth seeded Fourier modes about the
    batched background (rho, p, all three velocity components and B_z perturbed;
    B_x, B_y perturbed through A_z so that the in-plane field is divergence free).
    Every component varies, so no flux is identically zero: the update is
    differentiable at the initial state (MP5 has kinks at exactly uniform data)."""
    rng = np.random.default_rng(SEED0 + seed_index)
    x, dx = centres(n, 0.0, 2 * np.pi)
    X, Y = np.meshgrid(x, x, indexing="xy")
    ks = [(a, b) for a in range(-4, 5) for b in range(-4, 5) if (a, b) != (0, 0)]

    def modes():
        out = np.zeros_like(X)
        for _ in range(nmodes):
            k = ks[rng.integers(len(ks))]
            c = rng.uniform(-1, 1) / nmodes
            ph = rng.uniform(0, 2 * np.pi)
            out += c * np.sin(k[0] * X + k[1] * Y + ph)
        return amp * out

    rho = 1.0 + modes()
    p = 1.0 + modes()
    vel = [modes(), modes(), modes()]
    # A_z = sum c sin(k.x + phi): B_x = dA/dy, B_y = -dA/dx (analytic)
    bx = np.full_like(X, 0.5)
    by = np.zeros_like(X)
    for _ in range(nmodes):
        k = ks[rng.integers(len(ks))]
        c = amp * rng.uniform(-1, 1) / nmodes
        ph = rng.uniform(0, 2 * np.pi)
        arg = k[0] * X + k[1] * Y + ph
        bx += c * k[1] * np.cos(arg)
        by -= c * k[0] * np.cos(arg)
    bz = modes()
    U = conserved_mhd(rho, vel, p, [bx, by, bz], 5.0 / 3.0).reshape(9, 1, n, n)
    dom = Domain((n, n, 1), (dx, dx, 1.0))
    return Workload("adjoint2d", MHD_GLM, 2, SSPRK3, 5.0 / 3.0, 0.4, [dom], U, nsteps=200,
                    extra={"dt": 1e-3, "checkpoint_every": 20})


def sine_advection(n, ndim=1, amp=0.2, gamma=1.4):
    """Euler: rho = 1 + amp sin(2 pi (x + y + ...)), v = (1, ...), p = 1 on the periodic unit box."""
    x, dx = centres(n, 0.0, 1.0)
    if ndim == 1:
        rho = 1.0 + amp * np.sin(2 * np.pi * x)
        U = conserved_euler(rho, [np.ones(n)], np.ones(n), gamma).reshape(3, 1, 1, n)
        dom = Domain((n, 1, 1), (dx, 1.0, 1.0))
    else:
        X, Y = np.meshgrid(x, x, indexing="xy")
        rho = 1.0 + amp * np.sin(2 * np.pi * (X + Y))
        one = np.ones_like(X)
        U = conserved_euler(rho, [one, one], one, gamma).reshape(4, 1, n, n)
        dom = Domain((n, n, 1), (dx, dx, 1.0))
    return Workload("sine%dd" % ndim, EULER, ndim, SSPRK54, gamma, 0.4, [dom], U)


def alfven2d(n, t=0.0, A=0.1, rho0=1.0, p0=0.1, vA=1.0, gamma=5.0 / 3.0):
    """Circularly polarised Alfven wave (exact nonlinear MHD solution, Sec. 4.5.1)
    travelling along k = (1,1) on periodic [0, L]^2 with L = 2 pi; the 1D wave
    (v_par = 0, v_perp1 = A sin phi, v_perp2 = A cos phi, B_par = vA sqrt(rho),
    B_perp = -sqrt(rho) v_perp) rotated onto the diagonal. Returned at time t."""
    L = 2 * np.pi
    x, dx = centres(n, 0.0, L)
    X, Y = np.meshgrid(x, x, indexing="xy")
    kx = ky = 2 * np.pi / L
    kk = np.hypot(kx, ky)
    phi = kx * X + ky * Y - vA * kk * t
    e_par = np.array([kx, ky, 0.0]) / kk
    e_p1 = np.array([-ky, kx, 0.0]) / kk
    e_p2 = np.array([0.0, 0.0, 1.0])
    vp1, vp2 = A * np.sin(phi), A * np.cos(phi)
    sq = np.sqrt(rho0)
    vel = [vp1 * e_p1[i] + vp2 * e_p2[i] for i in range(3)]
    B = [vA * sq * e_par[i] - sq * (vp1 * e_p1[i] + vp2 * e_p2[i]) for i in range(3)]
    rho = np.full_like(X, rho0)
    p = np.full_like(X, p0)
    U = conserved_mhd(rho, vel, p, B, gamma).reshape(9, 1, n, n)
    dom = Domain((n, n, 1), (dx, dx, 1.0))
    period = L / kk / vA
    return Workload("alfven2d", MHD_GLM, 2, SSPRK54, gamma, 0.4, [dom], U, t_end=period)


def brio_wu(n=512):
    """1D MHD Brio-Wu shock tube (Sec. 4.5.2) on [-1,1], gamma 5/3, outflow."""
    x, dx = centres(n, -1.0, 1.0)
    left = x < 0.0
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    zero = np.zeros(n)
    U = conserved_mhd(rho, [zero, zero, zero], p, [zero + 0.75, np.where(left, 1.0, -1.0), zero],
                      5.0 / 3.0).reshape(9, 1, 1, n)
    dom = Domain((n, 1, 1), (dx, 1.0, 1.0), bc=((OUTFLOW, OUTFLOW),) * 3)
    return Workload("briowu", MHD_GLM, 1, SSPRK54, 5.0 / 3.0, 0.4, [dom], U, t_end=0.2,
                    extra={"x": x})


def brio_wu2d(n=128):
    """The Brio-Wu states (Sec. 4.5.2) in bands along the diagonal of the periodic box
    [-1,1]^2: left state where (x + y) mod 2 < 1, else right (two tubes per period, one of
    them mirrored), B_parallel = 0.75 along (1,1)/sqrt(2), B_perp = +-1 along
    (-1,1)/sqrt(2), gamma 5/3, SSPRK(5,4), CFL 0.4."""
    x, dx = centres(n, -1.0, 1.0)
    X, Y = np.meshgrid(x, x, indexing="xy")
    left = np.mod(X + Y + 2.0, 2.0) < 1.0
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    bt = np.where(left, 1.0, -1.0)
    r2 = 1.0 / np.sqrt(2.0)
    zero = np.zeros_like(X)
    B = [0.75 * r2 - bt * r2, 0.75 * r2 + bt * r2, zero]
    U = conserved_mhd(rho, [zero, zero, zero], p, B, 5.0 / 3.0).reshape(9, 1, n, n)
    dom = Domain((n, n, 1), (dx, dx, 1.0))
    return Workload("briowu2d", MHD_GLM, 2, SSPRK54, 5.0 / 3.0, 0.4, [dom], U)


def random_states(rng, n, physics, ndim, gamma, beta_min=0.05):
    """n random physical cell states (for point-wise tests), shape (nv, n)."""
    rho = rng.uniform(0.2, 3.0, n)
    p = rng.uniform(0.05, 3.0, n)
    v = [rng.uniform(-2, 2, n) for _ in range(3)]
    if physics == EULER:
        return conserved_euler(rho, v[:ndim], p, gamma)
    B = [rng.uniform(-2, 2, n) for _ in range(3)]
    psi = rng.uniform(-0.5, 0.5, n)
    return conserved_mhd(rho, v, p, B, gamma, psi)
