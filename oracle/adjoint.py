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

from oracle import energy, fine, parareal, transfer


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


# ============================================================================
# Adjoint of the parareal solve (Alg. 3) with the phase correctors frozen.
#
# The paper does not differentiate its method.  With every iteration's
# Omega^k = X_k Y_k^T held at the value the forward run computed from its data
# (Alg. 1), the map (u0, p0, c) -> u^{K+1}_N is a composition of F, C (Sec.
# 3.1), R, I (Sec. 6), Lambda, Lambda^dagger (Sec. 3.4, Alg. 2) and the fixed
# matrices Omega^k, linear in (u0, p0).  Its adjoint is the transpose of each
# of those maps applied in reverse order; each transpose below is checked
# against its forward map by the dot-product identity in the tests.
# ============================================================================

def restrict_T(Uc: np.ndarray, ratio: int, fine_shape) -> np.ndarray:
    """R^T: the coarse values at the coarse nodes of a zero fine field."""
    out = np.zeros(fine_shape)
    sl = tuple(slice(None, None, ratio) for _ in fine_shape)
    out[sl] = Uc
    return out


def _interp_axis_T(y: np.ndarray, n_coarse: int, axis: int) -> np.ndarray:
    """Transpose of transfer._interp_axis: with I = s Re(ifft_f P fft_c),
    s = n_f / n_c and P the zero padding with the Nyquist split,
    I^T y = s Re(fft_c(P^T ifft_f(y)))."""
    n_f = y.shape[axis]
    Y = np.fft.ifft(y, axis=axis)
    shape = list(y.shape)
    shape[axis] = n_coarse
    Z = np.zeros(shape, dtype=complex)

    def put(dst, src):
        ds = [slice(None)] * y.ndim
        ss = [slice(None)] * y.ndim
        ds[axis], ss[axis] = dst, src
        return tuple(ds), tuple(ss)

    half = n_coarse // 2
    if n_coarse % 2 == 0:
        d, s = put(slice(0, half), slice(0, half))
        Z[d] = Y[s]
        d, s = put(slice(half + 1, n_coarse), slice(n_f - half + 1, n_f))
        Z[d] = Y[s]
        d, s = put(half, half)
        Z[d] += 0.5 * Y[s]
        d, s = put(half, n_f - half)
        Z[d] += 0.5 * Y[s]
    else:
        d, s = put(slice(0, half + 1), slice(0, half + 1))
        Z[d] = Y[s]
        d, s = put(slice(half + 1, n_coarse), slice(n_f - half, n_f))
        Z[d] = Y[s]
    return np.real(np.fft.fft(Z, axis=axis)) * (n_f / n_coarse)


def interpolate_T(y: np.ndarray, ratio: int) -> np.ndarray:
    """I^T: fine -> coarse, the axes in the reverse order of interpolate."""
    out = np.asarray(y, dtype=np.float64)
    for ax in reversed(range(y.ndim)):
        out = _interp_axis_T(out, y.shape[ax] // ratio, ax)
    return out


def gradient_T(comps: list, dx: float, order: int) -> np.ndarray:
    """Transpose of energy.gradient (components ordered x, y, z): the central
    and spectral derivatives are skew-symmetric, so nabla_h^T q = -sum_a D_a q_a."""
    out = np.zeros_like(comps[0])
    nd = comps[0].ndim
    for i, q in enumerate(comps):
        out -= energy.derivative(q, nd - 1 - i, dx, order)
    return out


def energy_map_T(bvec: np.ndarray, wt: np.ndarray, c: np.ndarray, dx: float, order: int):
    """Transpose of Lambda[w, w_t] = [nabla_h w; c^-1 w_t] (transfer.energy_map)
    at (w_t, c): returns (dL/dw, dL/dw_t, dL/dc)."""
    grads, p = transfer.split_components(bvec, c.shape)
    return gradient_T(grads, dx, order), p / c, -p * wt / (c * c)


def reconstruct_T(bq1: np.ndarray, bu_t: np.ndarray, pvec: np.ndarray, c: np.ndarray):
    """Transpose of transfer.reconstruct: (vec, zero_mode) -> (grad2func(q,
    zero_mode), c p) at (p, c).  grad2func is w = Re(ifftn(W)), W(xi) =
    sum_a D_a(xi) fftn(q_a)(xi) with D_a = -i xi_a / |xi|^2 (xi != 0) and
    W(0) = zero_mode, so its transpose is q_a = Re(fftn(D_a ifftn(bw))) and
    zero_mode = sum(bw) / npts.  Returns (dL/dvec, dL/dzero_mode, dL/dc)."""
    shape = bq1.shape
    dim = len(shape)
    npts = bq1.size
    xi = [energy.wavenumbers(shape[dim - 1 - i]) for i in range(dim)]
    ks = []
    mag2 = np.zeros(shape)
    for i in range(dim):
        bshape = [1] * dim
        bshape[dim - 1 - i] = shape[dim - 1 - i]
        k = xi[i].reshape(bshape) * np.ones(shape)
        ks.append(k)
        mag2 = mag2 + k * k
    nz = mag2 > 0
    B = np.fft.ifftn(bq1)
    comps = []
    for i in range(dim):
        D = np.zeros(shape, dtype=complex)
        D[nz] = -1j * ks[i][nz] / mag2[nz]
        comps.append(np.real(np.fft.fftn(D * B)))
    p = transfer.split_components(pvec, c.shape)[1]
    bvec = np.concatenate([g.ravel() for g in comps] + [(c * bu_t).ravel()])
    return bvec, float(np.sum(bq1)) / npts, bu_t * p


def parareal_frozen(P: parareal.Problem, u0: np.ndarray, p0: np.ndarray, K: int, omegas: list):
    """Alg. 3 for K iterations with Omega^k = X_k Y_k^T given (omegas[k-1] =
    (X_k, Y_k)) instead of computed from the data; otherwise the steps of
    parareal.iterate.  Returns the states u^k_n for k = 1..K+1 (list of lists)."""
    u = parareal.initial_guess(P, u0, p0)
    hist = [u]
    for k in range(1, K + 1):
        v = [parareal.F(P, *u[n - 1]) for n in range(1, P.n_slices + 1)]
        Uc = [parareal.C(P, *parareal.R(P, *u[n - 1])) for n in range(1, P.n_slices + 1)]
        X, Y = omegas[k - 1] if P.corrector == "procrustes" else (None, None)
        new = [u[0]]
        for n in range(1, P.n_slices + 1):
            w, wt = parareal.C(P, *parareal.R(P, *new[n - 1]))
            Un, Unt = Uc[n - 1]
            if P.corrector == "plain":
                du, dut = w - Un, wt - Unt
            else:
                lw, lU = parareal.Lam(P, w, wt), parareal.Lam(P, Un, Unt)
                if P.corrector == "procrustes":
                    lw, lU = X @ (Y.T @ lw), X @ (Y.T @ lU)
                q1, p = transfer.reconstruct(lw, float(np.sum(w)), P.c_coarse)
                q1t, pt = transfer.reconstruct(lU, float(np.sum(Un)), P.c_coarse)
                du, dut = q1 - q1t, p - pt
            cu, cut = parareal.I(P, du, dut)
            new.append((v[n - 1][0] + cu, v[n - 1][1] + cut))
        u = new
        hist.append(u)
    return hist


def _coarse_step_T(P: parareal.Problem, state, bW, bWt):
    """Adjoint of w = C R state at `state` (fine): (d/dstate_u, d/dstate_ut, d/dc)."""
    Ru, Rut = parareal.R(P, *state)
    bU, bUt, bcc = verlet_adjoint(Ru, Rut, P.c_coarse, P.dt_com / P.m_c, P.m_c, P.dx_c, bW, bWt)
    shape = state[0].shape
    return (restrict_T(bU, P.ratio, shape), restrict_T(bUt, P.ratio, shape),
            restrict_T(bcc, P.ratio, shape))


def parareal_adjoint(P: parareal.Problem, u0: np.ndarray, p0: np.ndarray, K: int, omegas: list,
                     gu: np.ndarray, gv: np.ndarray):
    """Reverse mode through parareal_frozen for L with dL/du^{K+1}_N = gu and
    dL/du_t^{K+1}_N = gv: returns (dL/du0, dL/dp0, dL/dc), c the fine wave
    speed (the coarse c is R c, so its gradient is scattered back by R^T)."""
    hist = parareal_frozen(P, u0, p0, K, omegas)
    N = P.n_slices
    shape = np.shape(u0)
    zero = lambda: [np.zeros(shape), np.zeros(shape)]
    cc = P.c_coarse
    bc = np.zeros(shape)
    # b[n] = adjoint of the current iteration's states u^{k+1}_n
    b = [zero() for _ in range(N + 1)]
    b[N] = [np.array(gu, dtype=np.float64), np.array(gv, dtype=np.float64)]
    b_init0 = zero()    # adjoint of u^1_0 = [u0, p0] collected from every u^{k+1}_0
    for k in range(K, 0, -1):
        uk, uk1 = hist[k - 1], hist[k]          # u^k_n (input states), u^{k+1}_n (outputs)
        bv = [zero() for _ in range(N + 1)]       # adjoint of v_n = F u^k_{n-1}
        cshape = np.shape(P.c_coarse)
        bU = [[np.zeros(cshape), np.zeros(cshape)] for _ in range(N + 1)]   # adjoint of U_n = C R u^k_{n-1}
        X, Y = omegas[k - 1] if P.corrector == "procrustes" else (None, None)
        Uc = [None] + [parareal.C(P, *parareal.R(P, *uk[n - 1])) for n in range(1, N + 1)]
        for n in range(N, 0, -1):
            bs = b[n]
            bv[n][0] += bs[0]
            bv[n][1] += bs[1]
            bdu, bdut = interpolate_T(bs[0], P.ratio), interpolate_T(bs[1], P.ratio)
            w, wt = parareal.C(P, *parareal.R(P, *uk1[n - 1]))
            Un, Unt = Uc[n]
            if P.corrector == "plain":
                bw, bwt = bdu, bdut
                bU[n][0] -= bdu
                bU[n][1] -= bdut
            else:
                lw, lU = parareal.Lam(P, w, wt), parareal.Lam(P, Un, Unt)
                if P.corrector == "procrustes":
                    qw, qU = X @ (Y.T @ lw), X @ (Y.T @ lU)
                else:
                    qw, qU = lw, lU
                # du = q1 - q1t, dut = p - pt
                bqw, bzw, bcw = reconstruct_T(bdu, bdut, qw, cc)
                bqU, bzU, bcU = reconstruct_T(-bdu, -bdut, qU, cc)
                bcoarse = bcw + bcU
                if P.corrector == "procrustes":
                    bqw, bqU = Y @ (X.T @ bqw), Y @ (X.T @ bqU)
                bw, bwt, bcl = energy_map_T(bqw, wt, cc, P.dx_c, P.grad_order)
                bw = bw + bzw
                bUn, bUnt, bcl2 = energy_map_T(bqU, Unt, cc, P.dx_c, P.grad_order)
                bU[n][0] += bUn + bzU
                bU[n][1] += bUnt
                bc += restrict_T(bcoarse + bcl + bcl2, P.ratio, shape)
            # w = C R u^{k+1}_{n-1}
            gu_, gut_, gc_ = _coarse_step_T(P, uk1[n - 1], bw, bwt)
            b[n - 1][0] += gu_
            b[n - 1][1] += gut_
            bc += gc_
        # u^{k+1}_0 = u^1_0
        b_init0[0] += b[0][0]
        b_init0[1] += b[0][1]
        # parallel phase of iteration k: v_n = F u^k_{n-1}, U_n = C R u^k_{n-1}
        nb = [zero() for _ in range(N + 1)]
        for n in range(1, N + 1):
            fu, fut, fc = verlet_adjoint(*uk[n - 1], P.c_fine, P.dt_com / P.m_f, P.m_f, P.dx_f,
                                         bv[n][0], bv[n][1])
            cu_, cut_, cc_ = _coarse_step_T(P, uk[n - 1], bU[n][0], bU[n][1])
            nb[n - 1][0] += fu + cu_
            nb[n - 1][1] += fut + cut_
            bc += fc + cc_
        b = nb
    # the initial guess: u^1_n = I C R u^1_{n-1}
    u1 = hist[0]
    for n in range(N, 0, -1):
        bW, bWt = interpolate_T(b[n][0], P.ratio), interpolate_T(b[n][1], P.ratio)
        gu_, gut_, gc_ = _coarse_step_T(P, u1[n - 1], bW, bWt)
        b[n - 1][0] += gu_
        b[n - 1][1] += gut_
        bc += gc_
    return b[0][0] + b_init0[0], b[0][1] + b_init0[1], bc
