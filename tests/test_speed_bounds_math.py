"""The claim behind the FP32 bounds of the exact c_max search (speed_bounds in
csrc/amrfd_device.cuh), checked on the oracle's characteristic speeds (Sec. 4.4).

The bounds enter momentum and field components below 2^-100 in magnitude as zero and
widen by 2^-20 of the speed, provided T/S < 2^10 (T = E + rho v^2/2 + B^2/2,
S = p/(gamma-1)) and q = (1.5 + gamma)(1/rho + 1/sqrt(rho))/a <= 2^76, a the sound
speed; any other cell is evaluated exactly. The derivation bounds the change of every
speed |v_d| + c_f by 3 * 2^-100 (1.5 + gamma)(1/rho + 1/sqrt(rho)), below 2^-21 of
the speed when q <= 2^76. Here that is checked where it is tightest (q just below
2^76, components just below 2^-100, small rho), and the threshold is shown to be
needed: far above it leaving the components out changes the speeds by more than the
widening.
"""
import math

import numpy as np

import oracle as O
from paper_1407_2052_gb300 import workloads as W

EPS = 2.0 ** -100


def _speeds(gamma, u):
    """Per-direction characteristic speeds of one MHD state (a 3^3 periodic box of it)."""
    c = O.cfg(O.MHD_GLM, 3, O.SSPRK3, gamma)
    d = O.dom((3, 3, 3), (1.0, 1.0, 1.0))
    U = np.repeat(np.asarray(u, dtype=np.float64)[:, None], 27, axis=1).reshape(9, 3, 3, 3)
    al, _, fl = O.speeds(c, d, U)
    assert fl == 0
    return al


def _state(rho, m, S, B):
    """Conserved state from rho, momentum m, thermal energy S = p/(gamma-1) and field B."""
    m = np.asarray(m, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    E = S + 0.5 * float(m @ m) / rho + 0.5 * float(B @ B)
    return [rho, *m, E, *B, 0.0]


def _q(gamma, rho, S):
    a = math.sqrt(gamma * (gamma - 1.0) * S / rho)
    return (1.5 + gamma) * (1.0 / rho + 1.0 / math.sqrt(rho)) / a


def test_flushed_components_move_the_speeds_by_less_than_2_pow_minus_21():
    rng = np.random.default_rng(W.SEED0 + 201)
    worst = 0.0
    checked = 0
    for _ in range(3000):
        gamma = float(rng.choice([5.0 / 3.0, 1.4, 2.0]))
        rho = 2.0 ** rng.uniform(-99.0, -40.0)
        q_target = 2.0 ** rng.uniform(70.0, 76.0)
        a = (1.5 + gamma) * (1.0 / rho + 1.0 / math.sqrt(rho)) / q_target
        S = a * a * rho / (gamma * (gamma - 1.0))  # thermal energy p / (gamma - 1)
        if S < 2.0 ** -99:                          # E below 2^-100: evaluated exactly
            continue
        tiny = lambda: EPS * rng.uniform(0.5, 1.0) * rng.choice([-1.0, 1.0])
        m = [tiny() for _ in range(3)]
        B = []
        for _k in range(3):
            kind = rng.integers(3)
            B.append(0.0 if kind == 0 else tiny() if kind == 1 else math.sqrt(S) * rng.uniform(-4.0, 4.0))
        B_kept = [b if abs(b) >= EPS else 0.0 for b in B]
        u = _state(rho, m, S, B)
        u_flushed = _state(rho, [0.0, 0.0, 0.0], S, B_kept)
        u_flushed[4] = u[4]                          # the bounds see the same E
        T = u[4] + 0.5 * float(np.dot(B_kept, B_kept))
        S_f = u[4] - 0.5 * float(np.dot(B_kept, B_kept))
        if not (S_f > 2.0 ** -10 * T) or _q(gamma, rho, S_f) > 2.0 ** 76:
            continue                                 # the kernel evaluates such cells exactly
        c = _speeds(gamma, u)
        cf = _speeds(gamma, u_flushed)
        bound = 3.0 * EPS * (1.5 + gamma) * (1.0 / rho + 1.0 / math.sqrt(rho))
        for d in range(3):
            change = abs(c[d] - cf[d])
            assert change <= bound * (1.0 + 1e-12) + 4e-16 * cf[d], (d, change, bound)
            assert change <= 2.0 ** -21 * cf[d], (d, change / cf[d])
            worst = max(worst, change / cf[d])
        checked += 1
    assert checked > 1000
    assert worst > 2.0 ** -26  # the sample reaches close to the bound, not only far below it


def test_far_above_the_threshold_the_change_exceeds_the_widening():
    """rho = 2^-95 with sound speed 5 and momenta of a few 2^-101 (the GPU parity test's
    adversarial cell): q is far above 2^76, and the momenta add 2/64 .. 4/64 to the speeds."""
    gamma = 5.0 / 3.0
    rho = 2.0 ** -95
    S = 25.0 * rho / gamma / (gamma - 1.0)
    m = np.array([4.0, 3.0, -2.0]) * 2.0 ** -101
    c = _speeds(gamma, _state(rho, m, S, [0.0, 0.0, 0.0]))
    cf = _speeds(gamma, _state(rho, [0.0, 0.0, 0.0], S, [0.0, 0.0, 0.0]))
    assert _q(gamma, rho, S) > 2.0 ** 90
    assert list(c) == [5.0625, 5.046875, 5.03125] and list(cf) == [5.0, 5.0, 5.0]
    assert min((c - cf) / cf) > 2.0 ** -20 * 1000
