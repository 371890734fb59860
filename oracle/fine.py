"""Fine and coarse propagators of Sec. 3.1, in plain FP64 numpy.

Test infrastructure only (see the package docstring).

The paper fixes the scheme in Sec. 3.1: "the standard second order central
difference scheme for the spatial derivatives and velocity Verlet for time
marching", on a uniform periodic grid of [0,1)^d, for u_tt = c(x)^2 Lap u
(Sec. 1, eq. waveequation).  Arrays are laid out [z][y][x] (x fastest); every
axis has the same spacing dx.
"""
from __future__ import annotations

import numpy as np


def laplacian(u: np.ndarray, dx: float) -> np.ndarray:
    """2nd-order central-difference Laplacian with periodic wrap (Sec. 3.1).

    (L u)_j = sum over axes e of (u_{j+e} - 2 u_j + u_{j-e}) / dx^2.
    """
    out = np.zeros_like(u, dtype=np.float64)
    for ax in range(u.ndim):
        out += (np.roll(u, -1, axis=ax) - 2.0 * u + np.roll(u, 1, axis=ax)) / (dx * dx)
    return out


def velocity_verlet(u: np.ndarray, v: np.ndarray, c: np.ndarray, dt: float, steps: int,
                    dx: float) -> tuple[np.ndarray, np.ndarray]:
    """`steps` velocity-Verlet steps of u_tt = c^2 L u (Sec. 3.1).

    Textbook velocity Verlet, acceleration a = c^2 L u evaluated pointwise:
        u_{n+1} = u_n + dt v_n + dt^2/2 a_n
        a_{n+1} = c^2 L u_{n+1}
        v_{n+1} = v_n + dt/2 (a_n + a_{n+1})
    The acceleration of the first step is computed from the input state,
    since a propagator call receives only [u, u_t] (Sec. 3.1, the pair
    [u_n, u_t n] passed between propagators).
    """
    u = np.array(u, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    c2 = np.asarray(c, dtype=np.float64) ** 2
    a = c2 * laplacian(u, dx)
    for _ in range(steps):
        u = u + dt * v + 0.5 * dt * dt * a
        a_next = c2 * laplacian(u, dx)
        v = v + 0.5 * dt * (a + a_next)
        a = a_next
    return u, v


def fine_all_slices(u_in: np.ndarray, v_in: np.ndarray, c: np.ndarray, dt_f: float,
                    m_f: int, dx: float) -> tuple[np.ndarray, np.ndarray]:
    """F applied independently to every slice of one iteration (Alg. 3, parFor).

    u_in, v_in have shape [N][grid]; slice n of the output is
    F[u_in[n], v_in[n]]: m_f fine steps of size dt_f over one coupling
    interval dt_com = m_f * dt_f (Sec. 3.1).
    """
    u_out = np.empty(u_in.shape, dtype=np.float64)
    v_out = np.empty(v_in.shape, dtype=np.float64)
    for n in range(u_in.shape[0]):
        u_out[n], v_out[n] = velocity_verlet(u_in[n], v_in[n], c, dt_f, m_f, dx)
    return u_out, v_out
