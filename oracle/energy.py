"""Gradient approximations, discrete wave energy and error measures (FP64).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

# Central first-derivative weights beta_k of order 2m:
#   (D f)_j = sum_k beta_k (f_{j+k} - f_{j-k}) / dx
# (the beta_j form of Sec. 3.4; order 2 has beta_1 = 1/2 as stated there).
CENTRAL_WEIGHTS = {
    2: (1.0 / 2.0,),
    4: (2.0 / 3.0, -1.0 / 12.0),
    6: (3.0 / 4.0, -3.0 / 20.0, 1.0 / 60.0),
    8: (4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0),
}


def wavenumbers(n: int) -> np.ndarray:
    """Angular wavenumbers xi = 2 pi m of an n-point grid on [0,1), FFT order."""
    return 2.0 * np.pi * np.fft.fftfreq(n, d=1.0 / n)


def derivative(f: np.ndarray, axis: int, dx: float, order: int) -> np.ndarray:
    """Periodic first derivative along `axis` (nabla_h of Sec. 3.1, Sec. 6.4).

    order in {2, 4, 6, 8}: central differences with CENTRAL_WEIGHTS;
    order 0: spectral, ifft(i xi fft(f)) (Proposition in Sec. 3.4), with the
    Nyquist wavenumber of an even grid set to zero so the result is real.
    """
    if order == 0:
        n = f.shape[axis]
        xi = wavenumbers(n)
        if n % 2 == 0:
            xi[n // 2] = 0.0
        shape = [1] * f.ndim
        shape[axis] = n
        fh = np.fft.fft(f, axis=axis)
        return np.real(np.fft.ifft(1j * xi.reshape(shape) * fh, axis=axis))
    out = np.zeros_like(f, dtype=np.float64)
    for k, beta in enumerate(CENTRAL_WEIGHTS[order], start=1):
        out += beta * (np.roll(f, -k, axis=axis) - np.roll(f, k, axis=axis))
    return out / dx


def gradient(f: np.ndarray, dx: float, order: int) -> list[np.ndarray]:
    """nabla_h f as a list of components, ordered x, y, z (x = last array axis)."""
    return [derivative(f, f.ndim - 1 - i, dx, order) for i in range(f.ndim)]


def discrete_wave_energy(u: np.ndarray, v: np.ndarray, c: np.ndarray, dx: float,
                         order: int = 4) -> float:
    """E([u, u_t]) of Sec. 3.1 (eq. discrete-wave-energy).

    E = 1/2 sum_j |nabla_h u(x_j)|^2 dx^d + 1/2 sum_j c_j^-2 |u_t(x_j)|^2 dx^d.
    """
    vol = dx ** u.ndim
    grad_sq = sum(np.sum(g * g) for g in gradient(u, dx, order))
    kin = np.sum(v * v / (c * c))
    return 0.5 * grad_sq * vol + 0.5 * kin * vol


def relative_energy_error(u: np.ndarray, v: np.ndarray, u_ref: np.ndarray, v_ref: np.ndarray,
                          c: np.ndarray, dx: float, order: int = 4) -> float:
    """sqrt(E([u-u_ref, v-v_ref]) / E([u_ref, v_ref])) (Sec. 6, error at T)."""
    num = discrete_wave_energy(u - u_ref, v - v_ref, c, dx, order)
    den = discrete_wave_energy(u_ref, v_ref, c, dx, order)
    return float(np.sqrt(num / den))


def relative_l2_error(u: np.ndarray, u_ref: np.ndarray) -> float:
    """||u - u_ref||_2 / ||u_ref||_2 of the displacement (Sec. 6)."""
    return float(np.linalg.norm((u - u_ref).ravel()) / np.linalg.norm(u_ref.ravel()))
