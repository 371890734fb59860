"""Pins of the oracle's nabla_h, discrete wave energy and error measures.

Checks against closed forms: convergence order of each central difference on
a smooth periodic function, exactness of the spectral derivative on
band-limited data, the 1D Fourier symbol of the 4th-order stencil, and the
energy of plane waves (Sec. 3.1, eq. discrete-wave-energy).
"""
import math

import numpy as np
import pytest

from oracle import energy
from paper_1905_00473_gb300 import workloads


def _smooth(n):
    x = np.arange(n) / n
    f = np.exp(np.sin(2 * math.pi * x))
    df = 2 * math.pi * np.cos(2 * math.pi * x) * f
    return f, df


@pytest.mark.parametrize("order", [2, 4, 6, 8])
def test_central_difference_convergence_order(order):
    errs = []
    for n in (32, 64):
        f, df = _smooth(n)
        errs.append(np.max(np.abs(energy.derivative(f, 0, 1.0 / n, order) - df)))
    rate = math.log2(errs[0] / errs[1])
    assert abs(rate - order) < 0.35, (order, rate)


def test_spectral_derivative_exact_on_band_limited():
    n = 32
    x = np.arange(n) / n
    f = np.sin(2 * math.pi * 3 * x) + 0.5 * np.cos(2 * math.pi * 11 * x)
    df = 2 * math.pi * (3 * np.cos(2 * math.pi * 3 * x) - 5.5 * np.sin(2 * math.pi * 11 * x))
    err = np.max(np.abs(energy.derivative(f, 0, 1.0 / n, 0) - df))
    assert err < 1e-11 * np.max(np.abs(df))


def test_fourth_order_symbol_1d():
    # symbol of the 4th-order central difference on e^{i xi x}: i (8 sin t - sin 2t)/(6 dx)
    n = 40
    dx = 1.0 / n
    x = np.arange(n) / n
    for m in (1, 5, 13, 19):
        t = 2 * math.pi * m * dx
        sym = (8 * math.sin(t) - math.sin(2 * t)) / (6 * dx)
        d = energy.derivative(np.sin(2 * math.pi * m * x), 0, dx, 4)
        np.testing.assert_allclose(d, sym * np.cos(2 * math.pi * m * x), atol=1e-11 * sym + 1e-12)


def test_gradient_component_order_2d():
    n = 16
    x, y = workloads.node_coords(2, n)
    f = np.sin(2 * math.pi * x) + 0 * y  # varies in x only
    gx, gy = energy.gradient(f, 1.0 / n, 0)
    assert np.max(np.abs(gy)) < 1e-12
    np.testing.assert_allclose(gx, 2 * math.pi * np.cos(2 * math.pi * x) + 0 * y, atol=1e-10)


def test_energy_of_plane_waves():
    n = 64
    dx = 1.0 / n
    x = np.arange(n) / n
    m = 5
    u = np.cos(2 * math.pi * m * x)
    z = np.zeros(n)
    c = np.full(n, 2.0)
    # potential: 1/2 sum (2 pi m)^2 sin^2 dx = (2 pi m)^2 / 4 with the spectral gradient
    e = energy.discrete_wave_energy(u, z, c, dx, order=0)
    assert abs(e - (2 * math.pi * m) ** 2 / 4) < 1e-10 * e
    # kinetic: 1/2 sum c^-2 cos^2 dx = 1/(4 c^2)
    e = energy.discrete_wave_energy(z, u, c, dx, order=4)
    assert abs(e - 1.0 / 16.0) < 1e-14
    # 2D: potential of cos(2 pi (m x + l y)) = (2 pi)^2 (m^2 + l^2)/4
    x2, y2 = workloads.node_coords(2, 32)
    u2 = np.cos(2 * math.pi * (3 * x2 + 4 * y2))
    e2 = energy.discrete_wave_energy(u2, np.zeros_like(u2), np.ones_like(u2), 1 / 32, order=0)
    assert abs(e2 - (2 * math.pi) ** 2 * 25 / 4) < 1e-9 * e2


def test_relative_errors():
    rng = np.random.default_rng(0)
    u, v = rng.standard_normal((2, 16, 16))
    c = np.ones((16, 16))
    assert energy.relative_energy_error(u, v, u, v, c, 1 / 16) == 0.0
    assert abs(energy.relative_energy_error(1.5 * u, 1.5 * v, u, v, c, 1 / 16) - 0.5) < 1e-14
    assert abs(energy.relative_l2_error(0.9 * u, u) - 0.1) < 1e-14
