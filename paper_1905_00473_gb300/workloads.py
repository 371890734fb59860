"""Seeded synthetic workloads shaped like the paper's experiments.

This module only builds inputs: grids, wave-speed fields c(x), initial data
and per-slice states.  It holds none of the method's arithmetic (no
Laplacian, no time stepping, no grid transfer), so both the CUDA path and the
FP64 oracle can be fed from it without sharing any computation.

The five workloads mirror the paper's setting (Sec. 3.1: periodic unit box,
fine/coarse grids with coarse nodes on fine nodes, Sec. 6 eq. for the errors)
and its examples (Sec. 7.1 smooth 1D medium, Sec. 7.2.1 smooth 2D waveguide,
Sec. 7.2.2 piecewise-constant inclusion).  The paper's Marmousi model is not
available, so the smooth/discontinuous media below stand in for it.

Time-step rule (the paper requires integer m_F, m_C, Sec. 3.1): the fine step
is the largest step not above 0.25*dx_f/max(c) that divides the coupling
interval into a multiple of 4 steps; the coarse step is 4x the fine step.
max(c) is taken over the sampled fine nodes.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64(state: int) -> int:
    """One output of the SplitMix64 generator (Steele, Lea, Flood 2014)."""
    z = (state + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def node_coords(dim: int, n: int) -> list[np.ndarray]:
    """Node coordinates x_j = j/n on [0,1)^dim, broadcastable, x fastest.

    Arrays are laid out [z][y][x] (C order), so the returned list is
    ordered (x, y, z) but each entry is shaped for the C-order array.
    """
    x = np.arange(n, dtype=np.float64) / n
    coords = []
    for ax in range(dim):
        shape = [1] * dim
        shape[dim - 1 - ax] = n
        coords.append(x.reshape(shape))
    return coords


def periodic_gaussian(dim: int, n: int, center, width: float) -> np.ndarray:
    """exp(-|x-x0|^2/width^2) with the periodic minimum-image distance."""
    coords = node_coords(dim, n)
    r2 = np.zeros([n] * dim)
    for ax in range(dim):
        d = coords[ax] - center[ax]
        d = d - np.round(d)
        r2 = r2 + d * d
    return np.exp(-r2 / (width * width))


def fourier_mode_field(dim: int, n: int, rng: np.random.Generator, modes: int = 8,
                       kmax: int = 4) -> np.ndarray:
    """Smooth random field: sum of `modes` cosines a_m cos(2 pi k_m.x + phi_m).

    k_m is drawn from {-kmax..kmax}^dim without the zero vector,
    a_m ~ U(0,1), phi_m ~ U(0, 2 pi).
    """
    coords = node_coords(dim, n)
    s = np.zeros([n] * dim)
    for _ in range(modes):
        while True:
            k = rng.integers(-kmax, kmax + 1, size=dim)
            if np.any(k != 0):
                break
        a = rng.uniform(0.0, 1.0)
        phi = rng.uniform(0.0, 2.0 * math.pi)
        arg = np.zeros([n] * dim)
        for ax in range(dim):
            arg = arg + 2.0 * math.pi * k[ax] * coords[ax]
        s = s + a * np.cos(arg + phi)
    return s


def smooth_random_speed(dim: int, n: int, rng: np.random.Generator) -> np.ndarray:
    """c = 1.5 + 0.5 s/max|s|, so c lies in [1, 2] (8 random Fourier modes)."""
    s = fourier_mode_field(dim, n, rng)
    return 1.5 + 0.5 * s / np.max(np.abs(s))


def step_counts(dt_com: float, dx_f: float, cmax: float, ratio_t: int = 4,
                cfl: float = 0.25) -> tuple[int, int]:
    """(m_F, m_C): smallest multiple of ratio_t with dt_com/m_F <= cfl*dx_f/cmax."""
    m = dt_com * cmax / (cfl * dx_f)
    m_f = int(math.ceil(m / ratio_t - 1e-9)) * ratio_t
    return m_f, m_f // ratio_t


@dataclasses.dataclass
class Workload:
    """One parareal problem instance on the periodic unit box."""
    name: str
    dim: int
    n_fine: int
    ratio: int                       # coarse spacing / fine spacing
    n_slices: int                    # N
    t_final: float                   # T
    dtype: str                       # "f32" or "f64": arithmetic of the fine path
    c: np.ndarray                    # fine-grid wave speed, FP64 values
    u0: np.ndarray
    p0: np.ndarray
    tol: float = 1e-13
    grad_order: int = 4
    seed: int = 19050473
    m_f_fixed: Optional[int] = None  # overrides the time-step rule (test cases)

    @property
    def n_coarse(self) -> int:
        return self.n_fine // self.ratio

    @property
    def dx_f(self) -> float:
        return 1.0 / self.n_fine

    @property
    def dt_com(self) -> float:
        return self.t_final / self.n_slices

    @property
    def points(self) -> int:
        return self.n_fine ** self.dim

    @property
    def shape(self) -> tuple[int, ...]:
        return (self.n_fine,) * self.dim

    @property
    def cmax(self) -> float:
        return float(np.max(self.c))

    @property
    def m_f(self) -> int:
        if self.m_f_fixed is not None:
            return self.m_f_fixed
        return step_counts(self.dt_com, self.dx_f, self.cmax)[0]

    @property
    def m_c(self) -> int:
        if self.m_f_fixed is not None:
            return max(1, -(-self.m_f_fixed // 4))
        return step_counts(self.dt_com, self.dx_f, self.cmax)[1]

    @property
    def dt_f(self) -> float:
        return self.dt_com / self.m_f

    @property
    def dt_c(self) -> float:
        return self.dt_com / self.m_c

    @property
    def np_dtype(self):
        return np.float32 if self.dtype == "f32" else np.float64

    def cast(self, a: np.ndarray) -> np.ndarray:
        """Round to the path's storage precision and return FP64 values."""
        return np.asarray(a, dtype=self.np_dtype).astype(np.float64)

    def point_steps_per_sweep(self) -> int:
        return self.n_slices * self.m_f * self.points


def config1() -> Workload:
    """1D, FP64: c = 1 + 0.5 sin(2 pi x), u0 = exp(-(x-0.5)^2/0.005)."""
    n = 128
    (x,) = node_coords(1, n)
    c = 1.0 + 0.5 * np.sin(2 * math.pi * x)
    u0 = np.exp(-((x - 0.5) ** 2) / 0.005)
    return Workload("1d-128-N8-f64", 1, n, 4, 8, 1.0, "f64", c, u0, np.zeros_like(u0),
                    tol=1e-13)


def config2() -> Workload:
    """2D smooth: c = 1 + 0.5 sin(2 pi x) cos(2 pi y), pulse width 0.03 at centre."""
    n = 512
    x, y = node_coords(2, n)
    c = 1.0 + 0.5 * np.sin(2 * math.pi * x) * np.cos(2 * math.pi * y)
    u0 = periodic_gaussian(2, n, (0.5, 0.5), 0.03)
    w = Workload("2d-512-N32-f32", 2, n, 4, 32, 2.0, "f32", c, u0, np.zeros_like(u0),
                 tol=5e-3)
    w.c = w.cast(w.c)
    w.u0 = w.cast(w.u0)
    return w


def config3() -> Workload:
    """2D inclusion: c = 3 on [0.3,0.7]^2, else 1; pulse width 0.02 at (0.2, 0.5)."""
    n = 1024
    x, y = node_coords(2, n)
    inside = (x >= 0.3) & (x <= 0.7) & (y >= 0.3) & (y <= 0.7)
    c = np.where(inside, 3.0, 1.0)
    u0 = periodic_gaussian(2, n, (0.2, 0.5), 0.02)
    w = Workload("2d-1024-N64-inclusion-f32", 2, n, 4, 64, 2.0, "f32", c, u0,
                 np.zeros_like(u0), tol=5e-3)
    w.u0 = w.cast(w.u0)
    return w


def config4_instance(i: int) -> Workload:
    """Instance i of the batched uneven workload (48 instances)."""
    seed = splitmix64(19050473 + i)
    rng = np.random.default_rng(seed)
    n = int(rng.choice([256, 512, 1024, 2048]))
    n_slices = int(rng.choice([16, 32, 64, 128]))
    c = smooth_random_speed(2, n, rng)
    center = rng.uniform(0.3, 0.7, size=2)
    width = rng.uniform(0.02, 0.05)
    u0 = periodic_gaussian(2, n, center, width)
    w = Workload(f"2d-batch-{i}-{n}-N{n_slices}", 2, n, 4, n_slices, 2.0, "f32", c, u0,
                 np.zeros_like(u0), tol=5e-3, seed=seed)
    w.c = w.cast(w.c)
    w.u0 = w.cast(w.u0)
    return w


def config5(n: int = 256) -> Workload:
    """3D smooth random medium in [1,2], Gaussian width 0.05 at the centre."""
    rng = np.random.default_rng(19050473)
    c = smooth_random_speed(3, n, rng)
    u0 = periodic_gaussian(3, n, (0.5, 0.5, 0.5), 0.05)
    w = Workload(f"3d-{n}-N32-f32", 3, n, 4, 32, 1.0, "f32", c, u0, np.zeros_like(u0),
                 tol=5e-3)
    w.c = w.cast(w.c)
    w.u0 = w.cast(w.u0)
    return w


CONFIGS: dict[str, Callable[[], Workload]] = {
    "1": config1,
    "2": config2,
    "3": config3,
    "5": config5,
}


def scaled_copy(w: Workload, n: int, n_slices: Optional[int] = None,
                m_f: Optional[int] = None) -> Workload:
    """The same medium recipe and pulse on an n^d grid (for small parity cases).

    The speed field is re-sampled by nearest node from the full-size field
    (so the c range and the inclusion survive); the pulse is re-evaluated.
    """
    idx = (np.arange(n) * w.n_fine) // n
    c = w.c
    for ax in range(w.dim):
        c = np.take(c, idx, axis=ax)
    out = dataclasses.replace(w, name=f"{w.name}@{n}", n_fine=n, c=np.ascontiguousarray(c))
    out.u0 = np.zeros([n] * w.dim)
    out.p0 = np.zeros([n] * w.dim)
    if n_slices is not None:
        out.n_slices = n_slices
    return out


def slice_states(w: Workload, n_slices: Optional[int] = None, seed: int = 0,
                 pulses: int = 3) -> tuple[np.ndarray, np.ndarray]:
    """Per-slice input states [N][grid] for one parallel sweep of F.

    In an iteration the slices start from the wavefield at the N coupling
    times.  The synthetic stand-in gives slice n a superposition of `pulses`
    periodic Gaussians (seeded centres, widths in [w0, 3 w0], amplitudes in
    [0.25, 1]) for u and an independent superposition for u_t scaled by the
    medium's speed and pulse frequency, so both components carry energy like a
    travelling wave.  Values are rounded to the workload's dtype.
    """
    n_slices = w.n_slices if n_slices is None else n_slices
    rng = np.random.default_rng(splitmix64(w.seed * 1000003 + seed))
    w0 = {1: 0.0707, 2: 0.03, 3: 0.05}[w.dim]
    u = np.zeros((n_slices,) + w.shape)
    v = np.zeros((n_slices,) + w.shape)
    for s in range(n_slices):
        for _ in range(pulses):
            cen = rng.uniform(0.0, 1.0, size=w.dim)
            wid = rng.uniform(w0, 3 * w0)
            amp = rng.uniform(0.25, 1.0) * rng.choice([-1.0, 1.0])
            u[s] += amp * periodic_gaussian(w.dim, w.n_fine, cen, wid)
            cen = rng.uniform(0.0, 1.0, size=w.dim)
            wid = rng.uniform(w0, 3 * w0)
            amp = rng.uniform(0.25, 1.0) * rng.choice([-1.0, 1.0])
            v[s] += amp * (w.cmax / wid) * periodic_gaussian(w.dim, w.n_fine, cen, wid)
    return w.cast(u), w.cast(v)


def custom_case(dim: int, n: int, n_slices: int, m_f: int, dtype: str = "f32",
                medium: str = "smooth", seed: int = 5) -> Workload:
    """A small problem with a prescribed step count m_f at CFL 0.25/max c.

    medium: "smooth" (8 random modes, c in [1, 2]) or "inclusion"
    (c = 3 on [0.3,0.7]^dim, else 1).
    """
    rng = np.random.default_rng(seed)
    if medium == "inclusion":
        coords = node_coords(dim, n)
        inside = np.ones([n] * dim, dtype=bool)
        for x in coords:
            inside = inside & (x >= 0.3) & (x <= 0.7)
        c = np.where(inside, 3.0, 1.0)
    else:
        c = smooth_random_speed(dim, n, rng)
    w = Workload(f"{dim}d-{n}-N{n_slices}-m{m_f}-{medium}-{dtype}", dim, n, 4, n_slices, 1.0,
                 dtype, c, np.zeros([n] * dim), np.zeros([n] * dim), seed=seed, m_f_fixed=m_f)
    w.c = w.cast(w.c)
    dt_f = 0.25 * w.dx_f / w.cmax
    w.t_final = n_slices * m_f * dt_f
    return w
