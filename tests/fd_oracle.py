"""Central differences of the oracle's frozen-speed trajectory (tests only).

A worker evaluates, for one direction v, J(U0 + h v) - J(U0 - h v) of
J = sum |B|^2/2 dx dy after the given steps, each step with the splitting speeds
and GLM speed of the base trajectory (the oracle's frozen-speed step), so that
the difference quotient approximates the derivative the discrete adjoint
transposes. Module-level so that a spawn process pool can import it.
"""
import numpy as np

import oracle as O


def fd_along(args):
    """args = (cfg tuple, dom tuple, U0, v, h, dt, frozen, area); returns (J+ - J-) / (2h)."""
    cfgt, domt, U0, v, h, dt, frozen, area = args
    c = O.cfg(*cfgt)
    d = O.dom(*domt)

    def final_B(U):
        for al, ch in frozen:
            U, _ = O.step_frozen(c, d, U, dt, al, ch)
        return U[5:8]
    Bp, Bm = final_B(U0 + h * v), final_B(U0 - h * v)
    # J(+) - J(-) as sum (B+ - B-)(B+ + B-)/2: no cancellation between two large totals
    return 0.5 * float(np.sum((Bp - Bm) * (Bp + Bm))) * area / (2 * h)
