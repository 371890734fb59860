"""torch.autograd.Functions over the C ABI, argument marshalling only.

* SerialFineSolve: the serial fine solve and its hand-written adjoint
  (pr_adjoint); the forward chains pr_fine_all_slices over the N coupling
  intervals, the backward checkpoints slice-start states and recomputes
  inside each slice.
* PararealSolve: K iterations of Alg. 3 (pr_iterate) and the reverse sweep
  through them with the phase correctors frozen (pr_iterate_adjoint).

Gradients flow to the wave speed c and the initial data (u0, p0)."""
from __future__ import annotations

import torch

from paper_1905_00473_gb300 import binding


class SerialFineSolve(torch.autograd.Function):
    """(u(T), u_t(T)) = F^N (u0, p0; c) on the periodic unit box."""

    @staticmethod
    def forward(ctx, c, u0, p0, dt_f: float, m_f: int, n_slices: int):
        dtype = binding.PR_F32 if c.dtype == torch.float32 else binding.PR_F64
        dim, n = c.dim(), int(c.shape[0])
        dt_com = dt_f * m_f
        cc = c.detach().contiguous()
        one = binding.pr_create(dim, n, 1, cc, dt_f, dt_f, 1, dt_com, dtype=dtype)
        u = u0.detach().contiguous().clone()
        v = p0.detach().contiguous().clone()
        for _ in range(n_slices):
            binding.pr_fine_all_slices(one, u, v, u, v)
        ctx.save_for_backward(cc, u0.detach().contiguous(), p0.detach().contiguous())
        ctx.meta = (dim, n, dtype, dt_f, m_f, n_slices)
        return u, v

    @staticmethod
    def backward(ctx, gu, gv):
        c, u0, p0 = ctx.saved_tensors
        dim, n, dtype, dt_f, m_f, n_slices = ctx.meta
        full = binding.pr_create(dim, n, 1, c, dt_f, dt_f, n_slices, dt_f * m_f * n_slices,
                                 dtype=dtype)
        gu = torch.zeros_like(u0) if gu is None else gu.contiguous()
        gv = torch.zeros_like(p0) if gv is None else gv.contiguous()
        gc, gu0, gp0 = torch.empty_like(c), torch.empty_like(u0), torch.empty_like(p0)
        binding.pr_adjoint(full, u0, p0, gu, gv, gc, gu0, gp0)
        torch.cuda.current_stream().synchronize()
        return gc, gu0, gp0, None, None, None


def serial_fine_solve(c, u0, p0, dt_f: float, m_f: int, n_slices: int):
    return SerialFineSolve.apply(c, u0, p0, dt_f, m_f, n_slices)


class PararealSolve(torch.autograd.Function):
    """(u, u_t) at T after K iterations of Alg. 3 (pr_iterate), with the
    gradient of the map in which every iteration's phase corrector Omega^k is
    held at its forward value (pr_iterate_adjoint).  For the Omega = 1 and
    plain correctors, and for any corrector at K = N (the iteration then
    reproduces the serial fine solve whatever Omega is), that is the gradient
    of the forward map itself."""

    @staticmethod
    def forward(ctx, c, u0, p0, ratio: int, dt_f: float, dt_c: float, n_slices: int, t_final: float, K: int,
                corrector: int, tol: float, grad_order: int):
        dtype = binding.PR_F32 if c.dtype == torch.float32 else binding.PR_F64
        dim, n = c.dim(), int(c.shape[0])
        cc = c.detach().contiguous()
        pc = binding.pr_create(dim, n, ratio, cc, dt_f, dt_c, n_slices, t_final, dtype=dtype, tol=tol,
                               grad_order=grad_order)
        a, b = u0.detach().contiguous(), p0.detach().contiguous()
        us = torch.zeros((n_slices + 1,) + tuple(c.shape), dtype=c.dtype, device=c.device)
        vs = torch.zeros_like(us)
        binding.pr_iterate(pc, a, b, K, corrector, us, vs)
        ctx.save_for_backward(cc, a, b)
        ctx.meta = (ratio, dt_f, dt_c, n_slices, t_final, K, corrector, tol, grad_order, dtype)
        return us[n_slices].clone(), vs[n_slices].clone()

    @staticmethod
    def backward(ctx, gu, gv):
        c, u0, p0 = ctx.saved_tensors
        ratio, dt_f, dt_c, n_slices, t_final, K, corrector, tol, grad_order, dtype = ctx.meta
        pc = binding.pr_create(c.dim(), int(c.shape[0]), ratio, c, dt_f, dt_c, n_slices, t_final, dtype=dtype,
                               tol=tol, grad_order=grad_order)
        gu = torch.zeros_like(u0) if gu is None else gu.contiguous()
        gv = torch.zeros_like(p0) if gv is None else gv.contiguous()
        gc, gu0, gp0 = torch.empty_like(c), torch.empty_like(u0), torch.empty_like(p0)
        binding.pr_iterate_adjoint(pc, u0, p0, K, corrector, gu, gv, gc, gu0, gp0)
        return gc, gu0, gp0, None, None, None, None, None, None, None, None, None


def parareal_solve(c, u0, p0, ratio: int, dt_f: float, dt_c: float, n_slices: int, t_final: float, K: int,
                   corrector: int = binding.PR_CORR_PROCRUSTES, tol: float = 1e-13, grad_order: int = 4):
    return PararealSolve.apply(c, u0, p0, ratio, dt_f, dt_c, n_slices, t_final, K, corrector, tol, grad_order)
