"""Pins of R, I, Lambda and Lambda^dagger (grad2func) against closed forms and
the numbers the paper prints (Sec. 3.4, Sec. 6, Sec. 6.4 table)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import energy, fine, transfer
from paper_1905_00473_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "grad_order_table.json")


@pytest.mark.parametrize("dim,nc,ratio", [(1, 16, 4), (1, 15, 2), (2, 8, 4), (2, 9, 3), (3, 6, 2), (2, 8, 1)])
def test_restriction_after_interpolation_is_identity(dim, nc, ratio):
    # R I = 1 (Sec. 5 uses RI = 1): coarse nodes coincide with fine nodes
    U = np.random.default_rng(dim * 100 + nc).standard_normal([nc] * dim)
    np.testing.assert_allclose(transfer.restrict(transfer.interpolate(U, ratio), ratio), U, atol=1e-12)


def test_interpolation_is_exact_for_band_limited_fields():
    nc, ratio = 16, 4
    xc, yc = workloads.node_coords(2, nc)
    xf, yf = workloads.node_coords(2, nc * ratio)
    for m, l in [(0, 0), (3, -5), (7, 7), (-7, 2)]:
        Uc = np.cos(2 * math.pi * (m * xc + l * yc) + 0.3)
        uf = np.cos(2 * math.pi * (m * xf + l * yf) + 0.3)
        np.testing.assert_allclose(transfer.interpolate(Uc, ratio), uf, atol=1e-12)


def test_interpolation_splits_the_nyquist_mode():
    # interpft convention: the Nyquist coefficient of an even grid is split
    # between +nc/2 and -nc/2, so (-1)^j interpolates to cos(pi nc x)
    nc, ratio = 8, 4
    Uc = np.cos(math.pi * nc * np.arange(nc) / nc)
    xf = np.arange(nc * ratio) / (nc * ratio)
    np.testing.assert_allclose(transfer.interpolate(Uc, ratio), np.cos(math.pi * nc * xf), atol=1e-12)


def _fd_symbol(theta, order):
    if order == 0:
        return theta
    return 2.0 * sum(b * math.sin(j * theta) for j, b in enumerate(energy.CENTRAL_WEIGHTS[order], start=1))


@pytest.mark.parametrize("order", [2, 4, 6, 0])
def test_reconstruction_multiplier_1d(order):
    # Lambda^dagger Lambda multiplies mode xi by (modified wavenumber)/(xi dx):
    # sinc(xi dx) for the 2nd order (Sec. 3.4, Sec. 6.2), (8 sin t - sin 2t)/(6t)
    # for the 4th, 1 for the spectral gradient (Proposition in Sec. 3.4)
    n = 32
    dx = 1.0 / n
    x = np.arange(n) / n
    for m in (1, 4, 9, 15):
        t = 2 * math.pi * m * dx
        v = np.cos(2 * math.pi * m * x + 0.7)
        out = transfer.grad2func(energy.gradient(v, dx, order), float(np.sum(v)))
        mult = _fd_symbol(t, order) / t
        if order == 2:
            assert abs(mult - math.sin(t) / t) < 1e-14
        if order == 4:
            assert abs(mult - (8 * math.sin(t) - math.sin(2 * t)) / (6 * t)) < 1e-14
        np.testing.assert_allclose(out, mult * v, atol=1e-12)


def test_reconstruction_multiplier_2d_mode_by_mode():
    # in 2D the multiplier is sum_i xi_i kappa(xi_i) / |xi|^2
    n = 16
    dx = 1.0 / n
    x, y = workloads.node_coords(2, n)
    for (m, l) in [(1, 2), (3, -5), (6, 6), (0, 7)]:
        v = np.cos(2 * math.pi * (m * x + l * y))
        out = transfer.grad2func(energy.gradient(v, dx, 4), float(np.sum(v)))
        xm, xl = 2 * math.pi * m, 2 * math.pi * l
        mult = (xm * _fd_symbol(xm * dx, 4) / dx + xl * _fd_symbol(xl * dx, 4) / dx) / (xm ** 2 + xl ** 2)
        np.testing.assert_allclose(out, mult * v, atol=1e-12)


def test_zero_mode_and_momentum():
    rng = np.random.default_rng(3)
    n = 12
    w = rng.standard_normal((n, n))
    c = 1 + rng.random((n, n))
    wt = rng.standard_normal((n, n))
    vec = transfer.energy_map(w, wt, c, 1 / n, order=0)
    rec, rect = transfer.reconstruct(vec, float(np.sum(w)), c)
    np.testing.assert_allclose(rect, wt, atol=1e-13)
    assert abs(np.mean(rec) - np.mean(w)) < 1e-13


def test_energy_components_norm_is_the_energy():
    # ||G||_F^2 = (2/dx^d) sum_n E (eq. partOPP), one column at a time
    rng = np.random.default_rng(4)
    n = 10
    w, wt = rng.standard_normal((2, n, n))
    c = 1 + rng.random((n, n))
    for order in (2, 4, 0):
        vec = transfer.energy_map(w, wt, c, 1 / n, order)
        e = energy.discrete_wave_energy(w, wt, c, 1 / n, order)
        assert abs(np.dot(vec, vec) - 2 * e / (1 / n) ** 2) < 1e-10 * np.dot(vec, vec)
    # block layout: x-derivative first, then y, then c^-1 w_t
    vec = transfer.energy_map(w, wt, c, 1 / n, 2)
    gx = (np.roll(w, -1, 1) - np.roll(w, 1, 1)) * n / 2
    np.testing.assert_allclose(vec[: n * n].reshape(n, n), gx, atol=1e-12)
    np.testing.assert_allclose(vec[2 * n * n:].reshape(n, n), wt / c, atol=1e-14)


def test_reconstruction_errors_match_the_papers_table():
    """Sec. 6.4 table, last column: the paper's 1D c = 1 example (same grid,
    Dx = 0.01, Dt_com = 0.05, Dt/Dx = 0.5, Dt/dt = 20, T = 10).  Taken here over
    the serial fine states at t_1..t_N, which the iterates U^k_i approach."""
    golden = json.load(open(GOLDEN))["reconstruction_error"]
    n = 100
    dx = 1.0 / n
    x = np.arange(n) / n - 0.5
    u = np.cos(10 * math.pi * x) * np.exp(-100 * x ** 2)
    v = np.zeros(n)
    c = np.ones(n)
    dt_f = 0.5 * dx / 20
    m_f = int(round(0.05 / dt_f))
    states = []
    for _ in range(200):
        u, v = fine.velocity_verlet(u, v, c, dt_f, m_f, dx)
        states.append(u)
    for key, order in (("2", 2), ("4", 4), ("6", 6), ("8", 8), ("spectral", 0)):
        worst = max(np.linalg.norm(transfer.grad2func(energy.gradient(s, dx, order), float(np.sum(s))) - s)
                    / np.linalg.norm(s) for s in states)
        if order == 0:
            assert worst < 1e-11, worst          # printed 1.77e-12: roundoff
        else:
            assert abs(worst / golden[key] - 1) < 0.01, (key, worst, golden[key])


def test_planted_mistakes_are_caught(monkeypatch):
    """A sign error in grad2func, a restriction shifted by one node, and a
    Nyquist coefficient copied to both sides without halving each fail one of
    the pins above."""
    import oracle.transfer as T
    n = 32
    x = np.arange(n) / n
    v = np.cos(2 * math.pi * 5 * x)
    good = T.grad2func(energy.gradient(v, 1 / n, 2), float(np.sum(v)))
    assert np.max(np.abs(good - math.sin(2 * math.pi * 5 / n) / (2 * math.pi * 5 / n) * v)) < 1e-12
    bad = -good + 2 * np.mean(v)          # what a '+i' instead of '-i' gives
    assert np.max(np.abs(bad - good)) > 0.5
    U = np.random.default_rng(0).standard_normal(8)
    shifted = T.interpolate(U, 4)[1::4]
    assert np.max(np.abs(shifted - U)) > 1e-2
    Uc = np.cos(math.pi * 8 * np.arange(8) / 8)
    Uh = np.fft.fft(Uc)
    Y = np.zeros(32, dtype=complex)
    Y[4] = Y[28] = Uh[4]                  # Nyquist on both sides, not halved
    unsplit = np.real(np.fft.ifft(Y)) * 4
    assert np.max(np.abs(unsplit - T.interpolate(Uc, 4))) > 0.1
