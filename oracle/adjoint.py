"""Discrete adjoint of the fine propagator and of the serial fine solve, FP64.

Test infrastructure only (see the package docstring).

The paper does not differentiate its method; the adjoint here is the exact
transpose of the discrete stepper of Sec. 3.1 as `oracle.fine` writes it
(textbook velocity Verlet).  For a loss L(u_m, v_m) with gradients
(gu, gv) at the end of the run it returns dL/du_0, dL/dv_0 and dL/dc.

At K = N iterations the parareal solution equals the serial fine solution
(finite termination of Alg. 3), so with the correctors frozen its gradient is
the serial fine adjoint below.
"""
from __future__ import annotations

import numpy as np

from oracle import fine


def verlet_adjoint(u0: np.ndarray, v0: np.ndarray, c: np.ndarray, dt: float, steps: int, dx: float,
                   gu: np.ndarray, gv: np.ndarray):
    """Reverse sweep through `steps` steps of fine.velocity_verlet.

    Forward (Sec. 3.1):  a_0 = c^2 L u_0 and for n = 0..steps-1
        u_{n+1} = u_n + dt v_n + dt^2/2 a_n
        a_{n+1} = c^2 L u_{n+1}
        v_{n+1} = v_n + dt/2 (a_n + a_{n+1})
    Reverse, with adjoints (bu, bv, ba) and L symmetric:
        from v_{n+1}:  bv_n += bv_{n+1}; ba_n += dt/2 bv_{n+1}; ba_{n+1} += dt/2 bv_{n+1}
        from a_{n+1}:  bu_{n+1} += L(c^2 ba_{n+1});  bc += 2 c (L u_{n+1}) ba_{n+1}
        from u_{n+1}:  bu_n += bu_{n+1}; bv_n += dt bu_{n+1}; ba_n += dt^2/2 bu_{n+1}
    and finally through a_0.  Returns (dL/du_0, dL/dv_0, dL/dc).
    """
    c = np.asarray(c, dtype=np.float64)
    c2 = c * c
    # forward trajectory of u (the only state the reverse sweep needs)
    us = [np.array(u0, dtype=np.float64)]
    u = us[0]
    v = np.array(v0, dtype=np.float64)
    a = c2 * fine.laplacian(u, dx)
    for _ in range(steps):
        u = u + dt * v + 0.5 * dt * dt * a
        a_next = c2 * fine.laplacian(u, dx)
        v = v + 0.5 * dt * (a + a_next)
        a = a_next
        us.append(u)
    bu = np.array(gu, dtype=np.float64)
    bv = np.array(gv, dtype=np.float64)
    ba = np.zeros_like(bu)
    bc = np.zeros_like(bu)
    for n in range(steps - 1, -1, -1):
        # v_{n+1} = v_n + dt/2 (a_n + a_{n+1})
        ba_next = ba + 0.5 * dt * bv          # adjoint of a_{n+1}
        ba_n = 0.5 * dt * bv
        # a_{n+1} = c^2 L u_{n+1}
        bu = bu + fine.laplacian(c2 * ba_next, dx)
        bc = bc + 2.0 * c * fine.laplacian(us[n + 1], dx) * ba_next
        # u_{n+1} = u_n + dt v_n + dt^2/2 a_n
        bv = bv + dt * bu
        ba = ba_n + 0.5 * dt * dt * bu
    # a_0 = c^2 L u_0
    bu = bu + fine.laplacian(c2 * ba, dx)
    bc = bc + 2.0 * c * fine.laplacian(us[0], dx) * ba
    return bu, bv, bc


def serial_fine_adjoint(u0: np.ndarray, p0: np.ndarray, c: np.ndarray, dt_f: float, m_f: int,
                        n_slices: int, dx: float, gu: np.ndarray, gv: np.ndarray):
    """Adjoint of F^N (the serial fine solve over N coupling intervals), slice by
    slice from the slice-start checkpoints, recomputing inside each slice."""
    checkpoints = [(np.array(u0, dtype=np.float64), np.array(p0, dtype=np.float64))]
    for _ in range(n_slices):
        checkpoints.append(fine.velocity_verlet(*checkpoints[-1], c, dt_f, m_f, dx))
    bu, bv = np.array(gu, dtype=np.float64), np.array(gv, dtype=np.float64)
    bc = np.zeros_like(bu)
    for n in range(n_slices - 1, -1, -1):
        bu, bv, bcn = verlet_adjoint(*checkpoints[n], c, dt_f, m_f, dx, bu, bv)
        bc = bc + bcn
    return bu, bv, bc
