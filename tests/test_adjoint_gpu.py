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


# ---- the adjoint of the parareal solve with the correctors frozen ----------
from oracle import parareal  # noqa: E402

_CORR = {"procrustes": 0, "omega1": 1, "plain": 2}


def _pr_case(dim, n, N, m_f, dtype, ratio, seed=3):
    w = W.custom_case(dim, n, N, m_f, dtype, "smooth", seed=seed)
    w.ratio = ratio
    w.u0 = w.cast(W.periodic_gaussian(dim, n, [0.4] * dim, 0.15))
    w.p0 = w.cast(0.3 * W.periodic_gaussian(dim, n, [0.6] * dim, 0.2))
    return w


def _gpu_iterate_adjoint(w, corrector, K, gu, gv, tol):
    import torch
    from paper_1905_00473_gb300 import binding
    dt = torch.float32 if w.dtype == "f32" else torch.float64
    T = lambda a: torch.tensor(a, dtype=dt, device="cuda").contiguous()
    ctx = binding.pr_create(w.dim, w.n_fine, w.ratio, T(w.c), w.dt_f, w.dt_c, w.n_slices, w.t_final,
                            dtype=binding.PR_F32 if w.dtype == "f32" else binding.PR_F64, tol=tol)
    gc, gu0, gp0 = (torch.zeros(w.shape, dtype=dt, device="cuda") for _ in range(3))
    binding.pr_iterate_adjoint(ctx, T(w.u0), T(w.p0), K, _CORR[corrector], T(gu), T(gv), gc, gu0, gp0)
    torch.cuda.synchronize()
    return ctx, [x.double().cpu().numpy() for x in (gu0, gp0, gc)]


def _oracle_iterate_adjoint(w, corrector, K, gu, gv, tol):
    P = parareal.Problem(c_fine=w.c, ratio=w.ratio, n_slices=w.n_slices, dt_com=w.dt_com, m_f=w.m_f,
                         m_c=w.m_c, grad_order=4, tol=tol, corrector=corrector)
    om = [(r.X, r.Y) for r in parareal.iterate(P, w.u0, w.p0, K)]
    return adjoint.parareal_adjoint(P, w.u0, w.p0, K, om, gu, gv)


@pytest.mark.parametrize("corrector", ["procrustes", "omega1", "plain"])
@pytest.mark.parametrize("dim,n,N,m_f,ratio", [(1, 32, 4, 8, 2), (2, 16, 4, 8, 2), (1, 24, 3, 8, 1)])
def test_iterate_adjoint_matches_oracle_fp64(lib, corrector, dim, n, N, m_f, ratio):
    """K = 2 < N iterations: dL/du0, dL/dp0, dL/dc of the GPU reverse sweep
    against the FP64 oracle adjoint (itself pinned by dot products and
    central differences), each corrector."""
    w = _pr_case(dim, n, N, m_f, "f64", ratio)
    rng = np.random.default_rng(dim * 7 + n)
    gu, gv = rng.standard_normal(w.shape), rng.standard_normal(w.shape)
    _, got = _gpu_iterate_adjoint(w, corrector, 2, gu, gv, 1e-12)
    ref = _oracle_iterate_adjoint(w, corrector, 2, gu, gv, 1e-12)
    for name, g, r in zip(("u0", "p0", "c"), got, ref):
        err = np.linalg.norm(g - r) / np.linalg.norm(r)
        assert err <= 1e-8, (corrector, name, err)


def test_iterate_adjoint_at_k_equal_n_is_the_serial_adjoint(lib):
    """At K = N (finite termination) the frozen-corrector gradient equals the
    serial fine solve's, which pr_adjoint computes."""
    import torch
    from paper_1905_00473_gb300 import binding
    w = _pr_case(2, 32, 3, 8, "f64", 2)
    rng = np.random.default_rng(5)
    gu, gv = rng.standard_normal(w.shape), rng.standard_normal(w.shape)
    ctx, got = _gpu_iterate_adjoint(w, "procrustes", w.n_slices, gu, gv, 1e-12)
    T = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda").contiguous()
    gc, gu0, gp0 = (torch.zeros(w.shape, dtype=torch.float64, device="cuda") for _ in range(3))
    binding.pr_adjoint(ctx, T(w.u0), T(w.p0), T(gu), T(gv), gc, gu0, gp0)
    for g, r in zip(got, (gu0, gp0, gc)):
        r = r.cpu().numpy()
        assert np.linalg.norm(g - r) <= 1e-9 * np.linalg.norm(r)


def test_iterate_adjoint_fp32_context(lib):
    """FP32 context (FP32 propagators and their transposes, tensor-core
    UpdateSVD) against the FP64 oracle on the same FP32-rounded inputs."""
    w = _pr_case(2, 64, 4, 12, "f32", 4)
    rng = np.random.default_rng(11)
    gu, gv = w.cast(rng.standard_normal(w.shape)), w.cast(rng.standard_normal(w.shape))
    _, got = _gpu_iterate_adjoint(w, "procrustes", 2, gu, gv, 1e-6)
    ref = _oracle_iterate_adjoint(w, "procrustes", 2, gu, gv, 1e-6)
    for name, g, r in zip(("u0", "p0", "c"), got, ref):
        err = np.linalg.norm(g - r) / np.linalg.norm(r)
        assert err <= 2e-3, (name, err)


def test_iterate_adjoint_3d_32_copy_of_the_differentiation_workload(lib):
    """32^3 copy of the 3D differentiation workload (coarse 8^3, 4 slices,
    Procrustes, K = 2 < N): plane-misfit gradient dL/dc and dL/du0 of the GPU
    reverse sweep against the FP64 oracle adjoint, in FP64."""
    n, N = 32, 4
    w = W.config5(n=n)
    w.n_slices, w.t_final = N, w.dt_com * N
    x, y, z = W.node_coords(3, n)
    w.p0 = np.zeros(w.shape)
    rng = np.random.default_rng(2)
    # dL/du(T) of 1/2 sum_{z = 0.5 plane} (u - u_target)^2 dx^2 with a seeded target
    gu = np.zeros(w.shape)
    gu[n // 2] = rng.standard_normal((n, n)) * (1.0 / n) ** 2
    gv = np.zeros(w.shape)
    w.dtype = "f64"
    _, got = _gpu_iterate_adjoint(w, "procrustes", 2, gu, gv, 1e-12)
    ref = _oracle_iterate_adjoint(w, "procrustes", 2, gu, gv, 1e-12)
    for name, g, r in zip(("u0", "p0", "c"), got, ref):
        err = np.linalg.norm(g - r) / np.linalg.norm(r)
        assert err <= 1e-8, (name, err)


@pytest.mark.parametrize("corrector,K", [("plain", 2), ("omega1", 2), ("procrustes", 3)])
def test_parareal_autograd_gradcheck(lib, corrector, K):
    """torch.autograd.gradcheck of PararealSolve in FP64 on a tiny 2D case:
    with the plain and Omega = 1 correctors the forward map has no data-driven
    corrector, and with Procrustes K = N makes the result independent of the
    corrector, so central differences of the forward see the same map as the
    frozen-corrector adjoint."""
    import torch
    from paper_1905_00473_gb300 import autograd, binding
    w = _pr_case(2, 8, 3, 4, "f64", 2)
    rng = np.random.default_rng(4)
    c = torch.tensor(w.c, device="cuda", requires_grad=True)
    u0 = torch.tensor(rng.standard_normal(w.shape), device="cuda", requires_grad=True)
    p0 = torch.tensor(rng.standard_normal(w.shape), device="cuda", requires_grad=True)

    def f(c_, a, b):
        return autograd.parareal_solve(c_, a, b, w.ratio, w.dt_f, w.dt_c, w.n_slices, w.t_final, K,
                                       _CORR[corrector], 1e-12, 4)

    assert torch.autograd.gradcheck(f, (c, u0, p0), eps=1e-6, atol=1e-7, rtol=1e-5)
