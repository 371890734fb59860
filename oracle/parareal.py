"""The proposed theta-parareal method (Alg. 3), its Omega = 1 and plain
parareal variants, and the serial fine reference, in FP64 numpy.

Test infrastructure only (see the package docstring).

Notation follows Alg. 3: u^k_n = [u, u_t] on the fine grid at t_n = n dt_com,
F / C the fine and coarse propagators over one coupling interval (Sec. 3.1),
R injection, I Fourier interpolation, Lambda / Lambda^dagger the energy maps
(Sec. 3.4), X, Sigma, Y the truncated SVD of the correlation matrix M
(Alg. 1).  Slices are indexed n = 0..N with n = 0 the initial state.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

from oracle import energy, fine, procrustes, transfer


@dataclasses.dataclass
class Problem:
    """Discretisation of one parareal run on the periodic unit box."""
    c_fine: np.ndarray      # wave speed at the fine nodes
    ratio: int              # Dx / dx (coarse nodes = every ratio-th fine node)
    n_slices: int           # N
    dt_com: float           # coupling interval
    m_f: int                # fine steps per interval
    m_c: int                # coarse steps per interval
    grad_order: int = 4     # nabla_h
    tol: float = 1e-13      # rank tolerance of Alg. 1
    corrector: str = "procrustes"   # "procrustes" | "omega1" | "plain"

    @property
    def dim(self) -> int:
        return self.c_fine.ndim

    @property
    def dx_f(self) -> float:
        return 1.0 / self.c_fine.shape[0]

    @property
    def dx_c(self) -> float:
        return self.dx_f * self.ratio

    @property
    def c_coarse(self) -> np.ndarray:
        # the coarse propagator uses c at the coarse nodes (Sec. 3.1)
        return transfer.restrict(self.c_fine, self.ratio)


def F(P: Problem, u: np.ndarray, ut: np.ndarray):
    """Fine propagator over one coupling interval (Sec. 3.1)."""
    return fine.velocity_verlet(u, ut, P.c_fine, P.dt_com / P.m_f, P.m_f, P.dx_f)


def C(P: Problem, U: np.ndarray, Ut: np.ndarray):
    """Coarse propagator over one coupling interval (Sec. 3.1)."""
    return fine.velocity_verlet(U, Ut, P.c_coarse, P.dt_com / P.m_c, P.m_c, P.dx_c)


def R(P: Problem, u: np.ndarray, ut: np.ndarray):
    return transfer.restrict(u, P.ratio), transfer.restrict(ut, P.ratio)


def I(P: Problem, U: np.ndarray, Ut: np.ndarray):
    return transfer.interpolate(U, P.ratio), transfer.interpolate(Ut, P.ratio)


def Lam(P: Problem, W: np.ndarray, Wt: np.ndarray) -> np.ndarray:
    return transfer.energy_map(W, Wt, P.c_coarse, P.dx_c, P.grad_order)


def serial_fine(P: Problem, u0: np.ndarray, p0: np.ndarray):
    """Reference solution at t_0..t_N: F applied serially (Sec. 6)."""
    out = [(np.array(u0, dtype=np.float64), np.array(p0, dtype=np.float64))]
    for _ in range(P.n_slices):
        out.append(F(P, *out[-1]))
    return out


def initial_guess(P: Problem, u0: np.ndarray, p0: np.ndarray):
    """Alg. 3 initialisation: u^1_0 = [u0, p0], u^1_n = I C R u^1_{n-1}."""
    out = [(np.array(u0, dtype=np.float64), np.array(p0, dtype=np.float64))]
    for _ in range(P.n_slices):
        out.append(I(P, *C(P, *R(P, *out[-1]))))
    return out


@dataclasses.dataclass
class IterationRecord:
    k: int
    rank: int                     # retained singular values s
    residual: Optional[float]     # ||F - Omega G||_F / ||F||_F of this iteration's data
    states: list                  # u^{k+1}_n, n = 0..N
    X: Optional[np.ndarray] = None   # Omega^k = X Y^T used in this iteration's serial update
    Y: Optional[np.ndarray] = None


def serial_sweep(P: Problem, start, v, Uc, X, Y):
    """The serial corrected sweep of Alg. 3: from u^{k+1}_0 = start, for
    n = 1..N, w = C R u^{k+1}_{n-1} and u^{k+1}_n = v_n + I(theta w - theta U_n),
    with v_n = F u^k_{n-1}, U_n = C R u^k_{n-1} and theta of P.corrector
    (Procrustes: I Lambda^dagger X Y^T Lambda).  Returns u^{k+1}_0..N."""
    new = [start]
    for n in range(1, P.n_slices + 1):
        w, wt = C(P, *R(P, *new[n - 1]))
        Un, Unt = Uc[n - 1]
        if P.corrector == "plain":
            du, dut = w - Un, wt - Unt
        else:
            lw, lU = Lam(P, w, wt), Lam(P, Un, Unt)
            if P.corrector == "procrustes":
                qp = procrustes.apply_corrector(X, Y, lw)
                qpt = procrustes.apply_corrector(X, Y, lU)
            else:   # Omega = 1
                qp, qpt = lw, lU
            q1, p = transfer.reconstruct(qp, float(np.sum(w)), P.c_coarse)
            q1t, pt = transfer.reconstruct(qpt, float(np.sum(Un)), P.c_coarse)
            du, dut = q1 - q1t, p - pt
        cu, cut = I(P, du, dut)
        new.append((v[n - 1][0] + cu, v[n - 1][1] + cut))
    return new


def iterate(P: Problem, u0: np.ndarray, p0: np.ndarray, K: int):
    """K iterations of Alg. 3 from the initial guess; returns the records."""
    u = initial_guess(P, u0, p0)
    X = S = Y = None
    records = []
    for k in range(1, K + 1):
        # parallel phase: v_n = F u^k_{n-1}, [U_n, U_t n] = C R u^k_{n-1}
        v = [F(P, *u[n - 1]) for n in range(1, P.n_slices + 1)]
        Uc = [C(P, *R(P, *u[n - 1])) for n in range(1, P.n_slices + 1)]
        residual = None
        if P.corrector == "procrustes":
            # data matrices: F = [Lambda R v_n], G = [Lambda U_n]
            Fm = np.stack([Lam(P, *R(P, *vn)) for vn in v], axis=1)
            Gm = np.stack([Lam(P, *Un) for Un in Uc], axis=1)
            X, S, Y = procrustes.update_svd(X, S, Y, Fm, Gm, P.tol)
            residual = float(np.linalg.norm(Fm - X @ (Y.T @ Gm)) / np.linalg.norm(Fm))
        u = serial_sweep(P, u[0], v, Uc, X, Y)
        records.append(IterationRecord(k, 0 if S is None else int(S.size), residual, u, X, Y))
    return records


def relative_errors(P: Problem, state, ref) -> tuple[float, float]:
    """(energy, l2) relative errors of a fine state against the reference (Sec. 6)."""
    e = energy.relative_energy_error(state[0], state[1], ref[0], ref[1], P.c_fine, P.dx_f,
                                     P.grad_order)
    return e, energy.relative_l2_error(state[0], ref[0])
