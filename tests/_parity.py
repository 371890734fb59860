"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs, and compare them."""
from __future__ import annotations

import numpy as np

from oracle import energy, fine
from paper_1905_00473_gb300 import workloads

# Required accuracy: relative energy-norm error per fine slice in FP32.
TOL_ENERGY_F32 = 1e-5
# FP64: ~m_F roundings of O(1) values, amplified by (dx k)^-1 <= n in the
# energy norm: 1e-11 leaves two orders of margin for n <= 1024, m_F <= 400.
TOL_ENERGY_F64 = 1e-11


def make_ctx(w: workloads.Workload, block_depth: int = 0):
    import torch
    from paper_1905_00473_gb300 import binding
    dt = torch.float32 if w.dtype == "f32" else torch.float64
    c = torch.tensor(w.c, dtype=dt, device="cuda").contiguous()
    return binding.pr_create(w.dim, w.n_fine, w.ratio, c, w.dt_f, w.dt_c, w.n_slices, w.t_final,
                             dtype=binding.PR_F32 if w.dtype == "f32" else binding.PR_F64,
                             block_depth=block_depth)


def run_gpu(ctx, u: np.ndarray, v: np.ndarray, dtype: str, n_begin=0, n_end=None,
            inplace=False):
    import torch
    from paper_1905_00473_gb300 import binding
    dt = torch.float32 if dtype == "f32" else torch.float64
    ud = torch.tensor(u, dtype=dt, device="cuda").contiguous()
    vd = torch.tensor(v, dtype=dt, device="cuda").contiguous()
    if inplace:
        uo, vo = ud, vd
    else:
        uo = torch.full_like(ud, float("nan"))
        vo = torch.full_like(vd, float("nan"))
    binding.pr_fine_all_slices(ctx, ud, vd, uo, vo, n_begin, n_end)
    binding.pr_check(ctx)
    return uo.double().cpu().numpy(), vo.double().cpu().numpy()


def oracle_slice(w: workloads.Workload, u: np.ndarray, v: np.ndarray):
    return fine.velocity_verlet(u, v, w.c, w.dt_f, w.m_f, w.dx_f)


def slice_errors(w, ug, vg, ur, vr):
    e = energy.relative_energy_error(ug, vg, ur, vr, w.c, w.dx_f, order=4)
    l2 = energy.relative_l2_error(ug, ur)
    return e, l2


def tol_for(w) -> float:
    return TOL_ENERGY_F32 if w.dtype == "f32" else TOL_ENERGY_F64


def modified_energy(u, v, c, dt, dx):
    """The exactly conserved discrete energy of velocity Verlet for
    c^-2 u'' = L u (L the 2nd-order Laplacian, -L = D+^T D+ in the plain inner
    product): 1/2 sum c^-2 v^2 + 1/2 sum |D+ u|^2 - dt^2/8 sum c^-2 a^2, a = c^2 L u,
    times dx^d.  A property of the scheme at any grid size."""
    fwd = [(np.roll(u, -1, axis=ax) - u) / dx for ax in range(u.ndim)]
    lap = sum((g - np.roll(g, 1, axis=ax)) / dx for ax, g in enumerate(fwd))
    a = c * c * lap
    return ((0.5 * np.sum(v * v / (c * c)) + 0.5 * sum(np.sum(g * g) for g in fwd)
             - dt * dt / 8.0 * np.sum(a * a / (c * c))) * dx ** u.ndim)
