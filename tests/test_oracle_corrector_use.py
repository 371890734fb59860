"""Pins of how the Procrustes corrector Omega = X Y^T is applied (Sec. 3.3 and
the serial update of Alg. 3), independent of how it is built.

* If the fine data are an exact orthogonal image of the coarse data, F = Q G
  with G of full row rank, the minimiser of ||F - Omega G|| over orthogonal
  Omega is Q itself (Sec. 3.2-3.3: M = F G^T = Q (G G^T), whose polar factor
  is Q), so `apply_corrector(X, Y, g)` must return Q g.
* In the serial update, Omega multiplies the energy components of the newest
  coarse state.  When the fine propagator acts on energy components as an
  orthogonal map composed with the coarse one (Lambda F = Q Lambda C on the
  states the iteration visits), the corrected sweep of Alg. 3 reproduces
  u_n = F u_{n-1} exactly after one iteration: the correction
  I Lambda^dagger Omega (Lambda w - Lambda U_n) then equals
  F u^{k+1}_{n-1} - v_n.  The exact propagator of u_tt = u_xx on band-limited
  data, with a spectral nabla_h (Lambda^dagger Lambda = 1, Sec. 3.4), is such
  a pair: each Fourier mode turns by an angle in its energy plane.

Each pin is shown to fail for the plausible mistakes: X and Y swapped,
Omega^T applied, the corrector dropped (Omega = 1).
"""
import numpy as np
import pytest

from oracle import energy, parareal, procrustes


def _omega_apply_swapped(X, Y, g):
    return Y @ (X.T @ g)


def _omega_apply_transposed_product(X, Y, g):
    return (Y @ X.T) @ g


def _orthogonal(rng, n):
    Q, R = np.linalg.qr(rng.standard_normal((n, n)))
    return Q * np.sign(np.diag(R))


@pytest.mark.parametrize("rows,cols", [(6, 9), (12, 12), (20, 31)])
def test_exact_orthogonal_relation_is_recovered(rows, cols):
    rng = np.random.default_rng(rows)
    Q = _orthogonal(rng, rows)
    G = rng.standard_normal((rows, cols))
    F = Q @ G
    X, S, Y = procrustes.update_svd(None, None, None, F, G, 1e-14)
    assert S.size == rows
    g = rng.standard_normal(rows)
    np.testing.assert_allclose(procrustes.apply_corrector(X, Y, g), Q @ g, atol=1e-12)
    # and the same after a second update with more data of the same relation
    G2 = rng.standard_normal((rows, 5))
    X, S, Y = procrustes.update_svd(X, S, Y, Q @ G2, G2, 1e-14)
    np.testing.assert_allclose(procrustes.apply_corrector(X, Y, g), Q @ g, atol=1e-12)
    for bad in (_omega_apply_swapped, _omega_apply_transposed_product):
        assert np.linalg.norm(bad(X, Y, g) - Q @ g) > 1e-3 * np.linalg.norm(g)


def test_exact_relation_on_a_subspace_is_recovered_there():
    # rank-deficient G: Omega = Q on the span of G (Alg. 3 applies the
    # partial isometry X Y^T, reading A7), zero on its complement
    rng = np.random.default_rng(11)
    rows, r = 14, 5
    Q = _orthogonal(rng, rows)
    G = rng.standard_normal((rows, r)) @ rng.standard_normal((r, 9))
    X, S, Y = procrustes.update_svd(None, None, None, Q @ G, G, 1e-12)
    assert S.size == r
    g_in = G @ rng.standard_normal(9)
    np.testing.assert_allclose(procrustes.apply_corrector(X, Y, g_in), Q @ g_in, atol=1e-11)
    B, _ = np.linalg.qr(G)
    g_out = rng.standard_normal(rows)
    g_out -= B[:, :r] @ (B[:, :r].T @ g_out)
    assert np.linalg.norm(procrustes.apply_corrector(X, Y, g_out)) < 1e-11


# ---- the serial update of Alg. 3 with an exactly rotating fine/coarse pair ----

N_GRID = 16


def _exact_wave(u, ut, t):
    """u_tt = u_xx on [0,1) periodic, solved mode by mode (band-limited data,
    Nyquist mode kept at zero)."""
    n = u.size
    xi = energy.wavenumbers(n)
    w = np.abs(xi)
    uh, vh = np.fft.fft(u), np.fft.fft(ut)
    ou, ov = np.zeros(n, complex), np.zeros(n, complex)
    nz = w > 0
    ou[nz] = uh[nz] * np.cos(w[nz] * t) + vh[nz] * np.sin(w[nz] * t) / w[nz]
    ov[nz] = -w[nz] * uh[nz] * np.sin(w[nz] * t) + vh[nz] * np.cos(w[nz] * t)
    ou[0], ov[0] = uh[0] + t * vh[0], vh[0]
    ou[n // 2] = ov[n // 2] = 0.0
    return np.real(np.fft.ifft(ou)), np.real(np.fft.ifft(ov))


def _band_limited(rng, n, zero_mean=False):
    h = np.zeros(n, complex)
    h[1:n // 2] = rng.standard_normal(n // 2 - 1) + 1j * rng.standard_normal(n // 2 - 1)
    h[n // 2 + 1:] = np.conj(h[1:n // 2][::-1])
    h[0] = 0.0 if zero_mean else rng.standard_normal()
    return np.real(np.fft.ifft(h)) * n


@pytest.fixture
def rotating_pair(monkeypatch):
    """F = exact propagation over dt_com, C = exact propagation over 0.41 dt_com
    (so Lambda F C^-1 Lambda^dagger is the exact propagator over 0.59 dt_com,
    orthogonal in the energy components); one grid, spectral nabla_h."""
    monkeypatch.setattr(parareal, "F", lambda P, u, ut: _exact_wave(u, ut, P.dt_com))
    monkeypatch.setattr(parareal, "C", lambda P, u, ut: _exact_wave(u, ut, 0.41 * P.dt_com))
    rng = np.random.default_rng(3)
    u0 = _band_limited(rng, N_GRID)
    p0 = _band_limited(rng, N_GRID, zero_mean=True)
    P = parareal.Problem(c_fine=np.ones(N_GRID), ratio=1, n_slices=16, dt_com=0.3, m_f=1, m_c=1,
                         grad_order=0, tol=1e-14, corrector="procrustes")
    return P, u0, p0


def _max_error_after_one_iteration(P, u0, p0):
    ref = parareal.serial_fine(P, u0, p0)
    rec = parareal.iterate(P, u0, p0, 1)[0]
    scale = max(np.abs(r[0]).max() for r in ref)
    err = max(max(np.abs(rec.states[n][0] - ref[n][0]).max(),
                  np.abs(rec.states[n][1] - ref[n][1]).max() * P.dt_com)
              for n in range(P.n_slices + 1))
    return err / scale, rec


def test_serial_update_with_exact_corrector_is_exact_after_one_iteration(rotating_pair):
    P, u0, p0 = rotating_pair
    err, rec = _max_error_after_one_iteration(P, u0, p0)
    # the states visit 7 Fourier modes, two energy directions each
    assert rec.rank == 14
    assert rec.residual < 1e-12
    assert err < 1e-11, err


@pytest.mark.parametrize("mutant", ["swapped", "transposed", "omega1"])
def test_serial_update_pin_catches_a_misapplied_corrector(rotating_pair, monkeypatch, mutant):
    P, u0, p0 = rotating_pair
    if mutant == "swapped":
        monkeypatch.setattr(procrustes, "apply_corrector", _omega_apply_swapped)
    elif mutant == "transposed":
        monkeypatch.setattr(procrustes, "apply_corrector", _omega_apply_transposed_product)
    else:
        P.corrector = "omega1"
    err, _ = _max_error_after_one_iteration(P, u0, p0)
    assert err > 1e-2, (mutant, err)


# ---- Sec. 6.2: the phase correction keeps long-time iterations stable ----

def _sec62_errors(corrector: str, K: int) -> list:
    """Relative energy error at T after k = 1..K iterations for the Sec. 6.2
    study at T = 50: c = 1, one grid, Dx = 0.01, Dt_com = 0.05, Dt/Dx = 0.5,
    Dt/dt = 20, 2nd-order nabla_h, tol 1e-14, u(x,0) = cos(10 pi x)
    exp(-100 x^2) on [-0.5, 0.5), u_t(x,0) = 0 (the Sec. 6 initial data)."""
    import math
    n = 100
    x = np.arange(n) / n - 0.5
    u0 = np.cos(10 * math.pi * x) * np.exp(-100 * x ** 2)
    P = parareal.Problem(c_fine=np.ones(n), ratio=1, n_slices=1000, dt_com=0.05, m_f=200, m_c=10,
                         grad_order=2, tol=1e-14, corrector=corrector)
    ref = parareal.serial_fine(P, u0, np.zeros(n))
    return [parareal.relative_errors(P, r.states[-1], ref[-1])[0]
            for r in parareal.iterate(P, u0, np.zeros(n), K)]


def _sec62_errors_swapped(K: int) -> list:
    """The same study with a planted mistake: Omega applied as Y X^T."""
    procrustes.apply_corrector = _omega_apply_swapped
    return _sec62_errors("procrustes", K)


@pytest.mark.slow
def test_phase_correction_stabilises_long_time_iterations():
    """Sec. 6.2: for long terminal times the Omega = 1 coupling (Lambda^dagger
    Lambda damping alone) goes unstable, while the Procrustes corrector
    Omega^k_* stays stable.  At T = 50 (N = 1000 slices) the oracle's Omega = 1
    error turns upward after ~10 iterations and passes 10x the initial error
    by k = 14, while the Procrustes error decreases at every iteration.  With
    X and Y swapped in the serial update (a planted mistake, in a separate
    process) the error grows instead."""
    import concurrent.futures as cf
    import multiprocessing as mp
    K = 14
    with cf.ProcessPoolExecutor(3, mp_context=mp.get_context("spawn")) as ex:
        fo = ex.submit(_sec62_errors, "omega1", K)
        fp = ex.submit(_sec62_errors, "procrustes", K)
        fs = ex.submit(_sec62_errors_swapped, K)
        e1, ep, es = fo.result(), fp.result(), fs.result()
    assert max(e1) > 10 * e1[0], e1
    assert e1[-1] > e1[9] * 5, e1
    assert all(b < a for a, b in zip(ep, ep[1:])), ep
    assert ep[-1] < 0.5 * ep[0], ep
    assert es[-1] > 2 * es[0], es
