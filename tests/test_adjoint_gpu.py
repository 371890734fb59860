"""GPU adjoint (pr_adjoint) against the FP64 oracle adjoint, a central
finite-difference check of the 3D plane-misfit loss on a 32^3 copy of the
differentiation workload in FP64, and torch.autograd.gradcheck through the
autograd.Function wrapper."""
import math

import numpy as np
import pytest

from oracle import adjoint, fine
from paper_1905_00473_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ctx(w, dtype, N):
    import torch
    from paper_1905_00473_gb300 import binding
    dt = torch.float32 if dtype == "f32" else torch.float64
    c = torch.tensor(w.c, dtype=dt, device="cuda")
    return binding.pr_create(w.dim, w.n_fine, 1, c, w.dt_f, w.dt_f, N, w.dt_com * N,
                             dtype=binding.PR_F32 if dtype == "f32" else binding.PR_F64)


def _gpu_adjoint(w, dtype, N, u0, p0, gu, gv):
    import torch
    from paper_1905_00473_gb300 import binding
    ctx = _ctx(w, dtype, N)
    dt = torch.float32 if dtype == "f32" else torch.float64
    t = lambda a: torch.tensor(a, dtype=dt, device="cuda").contiguous()
    gc, gu0, gp0 = (torch.zeros(w.shape, dtype=dt, device="cuda") for _ in range(3))
    binding.pr_adjoint(ctx, t(u0), t(p0), t(gu), t(gv), gc, gu0, gp0)
    torch.cuda.synchronize()
    return [x.double().cpu().numpy() for x in (gu0, gp0, gc)]


@pytest.mark.parametrize("dim,n,N,m,dtype", [(2, 24, 3, 8, "f64"), (3, 12, 2, 6, "f64"),
                                             (1, 48, 4, 10, "f64"), (2, 64, 3, 12, "f32"),
                                             (3, 16, 2, 6, "f32"), (2, 18, 3, 8, "f32")])
def test_adjoint_matches_oracle(lib, dim, n, N, m, dtype):
    w = W.custom_case(dim, n, N, m, dtype)
    rng = np.random.default_rng(dim)
    u0, p0, gu, gv = (w.cast(rng.standard_normal(w.shape)) for _ in range(4))
    got = _gpu_adjoint(w, dtype, N, u0, p0, gu, gv)
    ref = adjoint.serial_fine_adjoint(u0, p0, w.c, w.dt_f, m, N, w.dx_f, gu, gv)
    tol = 1e-10 if dtype == "f64" else 2e-4
    for g, r in zip(got, ref):
        assert np.linalg.norm(g - r) <= tol * np.linalg.norm(r), (dtype, np.linalg.norm(g - r) / np.linalg.norm(r))


def test_plane_misfit_gradient_fd_3d_fp64(lib):
    """Differentiation workload on a 32^3 copy: loss = 1/2 sum over the plane
    z = 0.5 of (u(T) - u_target)^2 dx^2, target from c (1 + 0.05 exp(-|x - x0|^2/0.1^2));
    dL/dc from pr_adjoint against central differences of the GPU forward."""
    import torch
    from paper_1905_00473_gb300 import binding
    n, N = 32, 4
    w = W.config5(n=n)
    w.n_slices, w.t_final = N, w.dt_com * N   # shorter horizon for the check
    x, y, z = W.node_coords(3, n)
    bump = np.exp(-(((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2) / 0.1 ** 2))
    u0, p0 = w.u0, np.zeros(w.shape)
    dt = torch.float64
    T = lambda a: torch.tensor(a, dtype=dt, device="cuda").contiguous()

    def forward(c):
        ctx1 = binding.pr_create(3, n, 1, T(c), w.dt_f, w.dt_f, 1, w.dt_com, dtype=binding.PR_F64)
        u, v = T(u0), T(p0)
        for _ in range(N):
            binding.pr_fine_all_slices(ctx1, u, v, u, v)
        return u.cpu().numpy(), v.cpu().numpy()

    u_tgt, _ = forward(w.c * (1 + 0.05 * bump))
    k = n // 2

    def loss(c):
        u, _ = forward(c)
        return 0.5 * np.sum((u[k] - u_tgt[k]) ** 2) / n ** 2

    uT, _ = forward(w.c)
    gu = np.zeros(w.shape)
    gu[k] = (uT[k] - u_tgt[k]) / n ** 2
    _, _, gc = _gpu_adjoint(w, "f64", N, u0, p0, gu, np.zeros(w.shape))
    rng = np.random.default_rng(0)
    for _ in range(2):
        d = rng.standard_normal(w.shape) * bump
        eps = 1e-5
        fd = (loss(w.c + eps * d) - loss(w.c - eps * d)) / (2 * eps)
        assert abs(fd - np.sum(gc * d)) <= 1e-6 * abs(fd), (fd, np.sum(gc * d))


def test_autograd_gradcheck(lib):
    import torch
    from paper_1905_00473_gb300 import autograd
    w = W.custom_case(2, 8, 2, 5, "f64")
    rng = np.random.default_rng(3)
    c = torch.tensor(w.c, device="cuda", requires_grad=True)
    u0 = torch.tensor(rng.standard_normal(w.shape), device="cuda", requires_grad=True)
    p0 = torch.tensor(rng.standard_normal(w.shape), device="cuda", requires_grad=True)
    f = lambda c_, a, b: autograd.serial_fine_solve(c_, a, b, w.dt_f, w.m_f, w.n_slices)
    assert torch.autograd.gradcheck(f, (c, u0, p0), eps=1e-6, atol=1e-7, rtol=1e-5)


def test_adjoint_full_size_dot_product_3d(lib):
    """The differentiation workload at full size (256^3, 32 slices of 64 fine
    steps, FP32), where the FP64 oracle adjoint would take hours: the map
    (u0, p0) -> (u, u_t)(T) of the serial fine solve is linear, so the input
    gradients of pr_adjoint for the output gradient y = F x must satisfy
    <x, F^T y> = <F x, y> = ||F x||^2 (the dot-product identity), here with a
    smooth random x; the per-slice checkpoint and recompute path runs at the
    size it exists for."""
    import torch
    from paper_1905_00473_gb300 import binding
    w = W.config5()
    n, N = w.n_fine, w.n_slices
    c = torch.tensor(w.c, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(5)
    x, y_, z = W.node_coords(3, n)
    fields = []
    for _ in range(2):
        f = np.zeros(w.shape)
        for _ in range(4):
            k = rng.integers(-6, 7, size=3)
            f += rng.standard_normal() * np.cos(2 * math.pi * (k[0] * x + k[1] * y_ + k[2] * z) + rng.uniform(0, 6.3))
        fields.append(torch.tensor(f, dtype=torch.float32, device="cuda"))
    u0, p0 = fields[0], fields[1] * 4.0
    ctx1 = binding.pr_create(3, n, 1, c, w.dt_f, w.dt_f, 1, w.dt_com)
    u, v = u0.clone(), p0.clone()
    for _ in range(N):
        binding.pr_fine_all_slices(ctx1, u, v, u, v)
    ctx = binding.pr_create(3, n, 1, c, w.dt_f, w.dt_f, N, w.t_final)
    gc, gu0, gp0 = (torch.zeros_like(u0) for _ in range(3))
    binding.pr_adjoint(ctx, u0, p0, u, v, gc, gu0, gp0)
    torch.cuda.synchronize()
    lhs = float(torch.sum(u.double() ** 2) + torch.sum(v.double() ** 2))
    rhs = float(torch.sum(u0.double() * gu0.double()) + torch.sum(p0.double() * gp0.double()))
    assert math.isfinite(lhs) and lhs > 0
    assert abs(lhs - rhs) <= 1e-4 * lhs, (lhs, rhs)
