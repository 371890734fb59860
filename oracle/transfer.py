"""Grid transfer and energy-component maps of the method, FP64 numpy.

Test infrastructure only (see the package docstring).

* restrict      R : fine -> coarse, pointwise injection (Sec. 6: coarse nodes
                coincide with fine nodes, R is pointwise evaluation).
* interpolate   I : coarse -> fine, Fourier interpolation (the paper's default
                `interpft`, Sec. 6), separable over the axes.
* energy_map    Lambda [w, w_t] = [nabla_h w, c^-1 w_t] (Sec. 3.4).
* reconstruct   Lambda^dagger via grad2func (Sec. 3.4, eq. gradient2coordinate,
                Alg. 2): the function from its gradient through the FFT, with
                the zero mode supplied as sum(w); u_t = c p.

Vectors of energy components are flattened as [d/dx w, d/dy w, (d/dz w),
c^-1 w_t], each block in the grid's C order, i.e. (d+1) N_Dx entries
(eq. matrixF/matrixG column layout).
"""
from __future__ import annotations

import numpy as np

from oracle import energy


def restrict(u: np.ndarray, ratio: int) -> np.ndarray:
    """Injection onto the coarse nodes J*ratio along every axis (Sec. 6)."""
    sl = tuple(slice(None, None, ratio) for _ in range(u.ndim))
    return np.array(u[sl])


def _interp_axis(U: np.ndarray, n_fine: int, axis: int) -> np.ndarray:
    """1D Fourier interpolation along `axis`: zero-pad the spectrum.

    The coarse spectrum (n_c modes) is copied into an n_f-mode spectrum at the
    same wavenumbers; for even n_c the Nyquist coefficient is split equally
    between +n_c/2 and -n_c/2 (the `interpft` convention).  Scaled by
    n_f/n_c so that values, not sums, are interpolated.
    """
    n_c = U.shape[axis]
    Uh = np.fft.fft(U, axis=axis)
    shape = list(U.shape)
    shape[axis] = n_fine
    Y = np.zeros(shape, dtype=complex)

    def put(dst, src):
        ds = [slice(None)] * U.ndim
        ss = [slice(None)] * U.ndim
        ds[axis], ss[axis] = dst, src
        return tuple(ds), tuple(ss)

    half = n_c // 2
    if n_c % 2 == 0:
        d, s = put(slice(0, half), slice(0, half))                   # 0 .. n_c/2 - 1
        Y[d] = Uh[s]
        d, s = put(slice(n_fine - half + 1, n_fine), slice(half + 1, n_c))  # negatives
        Y[d] = Uh[s]
        d, s = put(half, half)                                       # Nyquist, split
        Y[d] += 0.5 * Uh[s]
        d, s = put(n_fine - half, half)
        Y[d] += 0.5 * Uh[s]
    else:
        d, s = put(slice(0, half + 1), slice(0, half + 1))
        Y[d] = Uh[s]
        d, s = put(slice(n_fine - half, n_fine), slice(half + 1, n_c))
        Y[d] = Uh[s]
    return np.real(np.fft.ifft(Y, axis=axis)) * (n_fine / n_c)


def interpolate(U: np.ndarray, ratio: int) -> np.ndarray:
    """I: coarse n_c^d -> fine (ratio n_c)^d, Fourier, one axis at a time."""
    out = np.asarray(U, dtype=np.float64)
    for ax in range(U.ndim):
        out = _interp_axis(out, U.shape[ax] * ratio, ax)
    return out


def energy_map(w: np.ndarray, wt: np.ndarray, c: np.ndarray, dx: float,
               order: int = 4) -> np.ndarray:
    """Lambda[w, w_t] = [nabla_h w ; c^-1 w_t] as one (d+1) N vector (Sec. 3.4)."""
    comps = energy.gradient(w, dx, order) + [wt / c]
    return np.concatenate([g.ravel() for g in comps])


def grad2func(grad: list[np.ndarray], zero_mode: float) -> np.ndarray:
    """Alg. 2: w from nabla_h w with fft(w)(xi) = -i xi . fft(q) / |xi|^2 for
    xi != 0 and fft(w)(0) = zero_mode (= sum of w over the grid); real part of
    the inverse FFT (Alg. 3 takes real(.)).  xi = 2 pi m are the angular
    wavenumbers of the unit box in FFT order (numpy's convention for the
    Nyquist index of an even grid: m = -n/2)."""
    shape = grad[0].shape
    dim = len(shape)
    xi = [energy.wavenumbers(shape[dim - 1 - i]) for i in range(dim)]   # x, y, z
    num = np.zeros(shape, dtype=complex)
    mag2 = np.zeros(shape)
    for i in range(dim):
        bshape = [1] * dim
        bshape[dim - 1 - i] = shape[dim - 1 - i]
        k = xi[i].reshape(bshape)
        num = num + k * np.fft.fftn(grad[i])
        mag2 = mag2 + k * k
    wh = np.zeros(shape, dtype=complex)
    nz = mag2 > 0
    wh[nz] = -1j * num[nz] / mag2[nz]
    wh[(0,) * dim] = zero_mode
    return np.real(np.fft.ifftn(wh))


def split_components(vec: np.ndarray, shape: tuple[int, ...]) -> tuple[list[np.ndarray], np.ndarray]:
    """Inverse of the flattening in energy_map: ([grad components], momentum)."""
    npts = int(np.prod(shape))
    dim = len(shape)
    grads = [vec[i * npts:(i + 1) * npts].reshape(shape) for i in range(dim)]
    return grads, vec[dim * npts:(dim + 1) * npts].reshape(shape)


def reconstruct(vec: np.ndarray, zero_mode: float, c: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Lambda^dagger: [q, p] -> [grad2func(q, zero_mode), c p] (Sec. 3.4)."""
    grads, p = split_components(vec, c.shape)
    return grad2func(grads, zero_mode), c * p
