"""torch.autograd.Function over the C ABI: the serial fine solve and its
hand-written adjoint (pr_adjoint).  Argument marshalling only: the forward
chains pr_fine_all_slices over the N coupling intervals, the backward calls
pr_adjoint, which checkpoints slice-start states and recomputes inside each
slice.  Gradients flow to the wave speed c and the initial data (u0, p0)."""
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
