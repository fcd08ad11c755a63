"""CPU FP64 oracle of the conservative finite-difference update (test infrastructure).

TEST INFRASTRUCTURE ONLY. Only tests/, the bench's CPU-baseline leg and the
smoke check may import this package. It wraps the plain C solver in
amrfd_oracle.c (single-threaded, -O2 -ffp-contract=off) through ctypes and
adds the exact Riemann solver of the Euler equations (oracle.riemann).

The physics follows Porth et al. (ApJS 2014): Sec. 2.1 (conservative FD),
Sec. 2.2 (global Lax-Friedrichs splitting + MP5 of Suresh & Huynh 1997),
Sec. 2.3 (SSPRK in Shu-Osher form), Sec. 4.1-4.4 (ideal MHD, GLM, time step),
App. C (active/passive blocks).
"""
import ctypes
import os

import numpy as np

from . import build as _build

EULER, MHD_GLM = 0, 1
SSPRK3, SSPRK54, SSPRK43 = 0, 1, 2
PERIODIC, OUTFLOW, SYMMETRIC = 0, 1, 2
MP5, LIMO3 = 0, 1
FLAG_NONPHYSICAL = 1


class Cfg(ctypes.Structure):
    _fields_ = [("physics", ctypes.c_int), ("ndim", ctypes.c_int), ("integrator", ctypes.c_int),
                ("recon", ctypes.c_int), ("gamma", ctypes.c_double), ("glm_cr", ctypes.c_double),
                ("limo3_r", ctypes.c_double)]


class Dom(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("nb", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
                ("bc", (ctypes.c_int * 2) * 3), ("asym", (ctypes.c_uint * 2) * 3)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        cp, mp = ctypes.POINTER(Cfg), ctypes.POINTER(Dom)
        L.orc_nvar.argtypes = [cp]
        L.orc_cons2prim.argtypes = [cp, dp, dp]
        L.orc_char_speed.argtypes = [cp, dp, ctypes.c_int]
        L.orc_char_speed.restype = ctypes.c_double
        L.orc_flux.argtypes = [cp, dp, dp, ctypes.c_int, ctypes.c_double, dp]
        L.orc_flux.restype = None
        for fn in ("orc_mp5",):
            getattr(L, fn).argtypes = [ctypes.c_double] * 5
            getattr(L, fn).restype = ctypes.c_double
        L.orc_limo3.argtypes = [ctypes.c_double] * 4
        L.orc_limo3.restype = ctypes.c_double
        L.orc_minmod.argtypes = [ctypes.c_double] * 2
        L.orc_minmod.restype = ctypes.c_double
        L.orc_minmod4.argtypes = [ctypes.c_double] * 4
        L.orc_minmod4.restype = ctypes.c_double
        L.orc_ssprk_table.argtypes = [ctypes.c_int, dp, dp]
        L.orc_speeds.argtypes = [cp, mp, dp, u8p, dp, dp]
        L.orc_residual.argtypes = [cp, mp, dp, dp, ctypes.c_double, dp]
        L.orc_step.argtypes = [cp, mp, dp, ctypes.c_double, u8p, dp, dp]
        L.orc_dt.argtypes = [cp, mp, dp, u8p, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        L.orc_step_frozen.argtypes = [cp, mp, dp, ctypes.c_double, u8p, dp, ctypes.c_double]
        L.orc_flag_steady.argtypes = [cp, mp, dp, dp, ctypes.c_double, u8p]
        L.orc_flag_steady.restype = None
        L.orc_activate.argtypes = [mp, u8p, ctypes.c_int, u8p]
        L.orc_activate.restype = None
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def cfg(physics, ndim, integrator=SSPRK3, gamma=1.4, glm_cr=0.18, recon=MP5, limo3_r=1.0):
    return Cfg(physics, ndim, integrator, recon, gamma, glm_cr, limo3_r)


def dom(n, dx, bc=PERIODIC, nb=(1, 1, 1), asym=None):
    """n, dx: per-dimension sequences (padded with 1 / 1.0); bc: one kind for all
    faces, or a 3x2 nested sequence; asym: 3x2 bit masks of the variables that are
    odd across a SYMMETRIC face (None = all even)."""
    n = list(n) + [1] * (3 - len(n))
    dx = list(dx) + [1.0] * (3 - len(dx))
    if isinstance(bc, int):
        bc = [[bc, bc]] * 3
    d = Dom()
    for k in range(3):
        d.n[k], d.nb[k], d.dx[k] = n[k], nb[k], dx[k]
        d.bc[k][0], d.bc[k][1] = bc[k][0], bc[k][1]
        if asym is not None:
            d.asym[k][0], d.asym[k][1] = int(asym[k][0]), int(asym[k][1])
    return d


def nvar(c):
    return 2 + c.ndim if c.physics == EULER else 9


def _check(c, d, U):
    shape = (nvar(c), d.n[2], d.n[1], d.n[0])
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(shape)
    for k in range(c.ndim):
        if d.bc[k][0] == PERIODIC and d.n[k] < 3:
            raise ValueError("periodic direction needs at least 3 cells")
        if SYMMETRIC in (d.bc[k][0], d.bc[k][1]) and d.n[k] < 3:
            raise ValueError("a mirror face needs at least 3 cells")
    return U


def _active(d, active):
    if active is None:
        return None
    a = np.ascontiguousarray(active, dtype=np.uint8).ravel()
    if a.size != d.nb[0] * d.nb[1] * d.nb[2]:
        raise ValueError("one active flag per block")
    return a


def cons2prim(c, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    w = np.zeros(9)
    ok = lib().orc_cons2prim(ctypes.byref(c), _dp(u), _dp(w))
    return w, bool(ok)


def char_speed(c, w, d):
    w = np.ascontiguousarray(w, dtype=np.float64)
    return lib().orc_char_speed(ctypes.byref(c), _dp(w), d)


def flux(c, u, d, ch=0.0):
    u = np.ascontiguousarray(u, dtype=np.float64)
    w, _ = cons2prim(c, u)
    f = np.zeros(9)
    lib().orc_flux(ctypes.byref(c), _dp(u), _dp(w), d, ch, _dp(f))
    return f[:nvar(c)]


def mp5(a, b, cc, d, e):
    return lib().orc_mp5(a, b, cc, d, e)


def limo3(um, u0, up, rdx):
    return lib().orc_limo3(um, u0, up, rdx)


def minmod(a, b):
    return lib().orc_minmod(a, b)


def minmod4(w, x, y, z):
    return lib().orc_minmod4(w, x, y, z)


def ssprk_table(integrator):
    a = np.zeros((5, 5))
    b = np.zeros((5, 5))
    s = lib().orc_ssprk_table(integrator, _dp(a), _dp(b))
    return s, a[:s, :s].copy(), b[:s, :s].copy()


def speeds(c, d, U, active=None):
    U = _check(c, d, U)
    a = _active(d, active)
    al = np.zeros(3)
    r = np.zeros(1)
    fl = lib().orc_speeds(ctypes.byref(c), ctypes.byref(d), _dp(U), _u8(a), _dp(al), _dp(r))
    return al, float(r[0]), fl


def residual(c, d, U, alpha, ch=0.0):
    U = _check(c, d, U)
    L = np.zeros_like(U)
    al = np.ascontiguousarray(alpha, dtype=np.float64)
    fl = lib().orc_residual(ctypes.byref(c), ctypes.byref(d), _dp(U), _dp(al), ch, _dp(L))
    return L, fl


def step(c, d, U, dt, active=None):
    """One SSPRK step; returns (U_new, flags, alpha_per_stage[s,3], c_h)."""
    U = _check(c, d, U).copy()
    a = _active(d, active)
    s = {SSPRK3: 3, SSPRK54: 5, SSPRK43: 4}[c.integrator]
    al = np.zeros((s, 3))
    ch = np.zeros(1)
    fl = lib().orc_step(ctypes.byref(c), ctypes.byref(d), _dp(U), float(dt), _u8(a), _dp(al), _dp(ch))
    return U, fl, al, float(ch[0])


def step_frozen(c, d, U, dt, alpha_stage, ch, active=None):
    """One SSPRK step with the per-stage splitting speeds and c_h held fixed."""
    U = _check(c, d, U).copy()
    a = _active(d, active)
    al = np.ascontiguousarray(alpha_stage, dtype=np.float64)
    fl = lib().orc_step_frozen(ctypes.byref(c), ctypes.byref(d), _dp(U), float(dt), _u8(a), _dp(al), float(ch))
    return U, fl


def dt(c, d, U, cfl, t=0.0, t_end=np.inf, active=None):
    U = _check(c, d, U)
    a = _active(d, active)
    out = np.zeros(1)
    fl = lib().orc_dt(ctypes.byref(c), ctypes.byref(d), _dp(U), _u8(a), cfl, t, t_end, _dp(out))
    return float(out[0]), fl


def evolve(c, d, U, cfl, t_end, max_steps=100000, fixed_dt=None):
    """Step from t = 0 to t_end with CFL steps (or a fixed dt); returns (U, t, nsteps, flags)."""
    t, n, flags = 0.0, 0, 0
    U = _check(c, d, U).copy()
    while t < t_end * (1 - 1e-14) and n < max_steps:
        if fixed_dt is None:
            h, fl = dt(c, d, U, cfl, t, t_end)
        else:
            h, fl = min(fixed_dt, t_end - t), 0
        U, fl2, _, _ = step(c, d, U, h)
        flags |= fl | fl2
        t += h
        n += 1
    return U, t, n, flags


def flag_steady(c, d, U, Uref, tol):
    """App. C step 1 criterion: 1 per block whose cells all lie within tol of Uref."""
    U = _check(c, d, U)
    R = _check(c, d, Uref)
    f = np.zeros(d.nb[0] * d.nb[1] * d.nb[2], np.uint8)
    lib().orc_flag_steady(ctypes.byref(c), ctypes.byref(d), _dp(U), _dp(R), float(tol), _u8(f))
    return f


def activate(d, flag, belt):
    """App. C steps 2-3: active flags from the candidates `flag` and `belt` safety layers."""
    f = _active(d, flag)
    a = np.zeros_like(f)
    lib().orc_activate(ctypes.byref(d), _u8(f), int(belt), _u8(a))
    return a
