"""GPU parity of the method around the fine sweep (Alg. 3) against the FP64
oracle: the coarse sweep C R, the initial guess I C R, K iterations with each
corrector, UpdateSVD (Alg. 1) and finite termination after N iterations.

FP64 contexts are compared to ~1e-9 (same arithmetic, different rounding
order and FFT library); FP32 contexts against the bound of 1e-4 relative
energy-norm error required of the FP32 parareal solution."""
import json
import math
import os

import numpy as np
import pytest

from oracle import energy, parareal, procrustes
from paper_1905_00473_gb300 import workloads as W
from tests import _parity as P

pytestmark = pytest.mark.gpu

CORR = {"procrustes": 0, "omega1": 1, "plain": 2}


def _problem(w, corrector, grad_order=4, tol=1e-13):
    return parareal.Problem(c_fine=w.c, ratio=w.ratio, n_slices=w.n_slices, dt_com=w.dt_com,
                            m_f=w.m_f, m_c=w.m_c, grad_order=grad_order, tol=tol,
                            corrector=corrector)


def _ctx(w, ratio, grad_order=4, tol=1e-13):
    import torch
    from paper_1905_00473_gb300 import binding
    dt = torch.float32 if w.dtype == "f32" else torch.float64
    c = torch.tensor(w.c, dtype=dt, device="cuda")
    return binding.pr_create(w.dim, w.n_fine, ratio, c, w.dt_f, w.dt_c, w.n_slices, w.t_final,
                             dtype=binding.PR_F32 if w.dtype == "f32" else binding.PR_F64,
                             grad_order=grad_order, tol=tol)


def _case(dim, n, N, m_f, dtype, ratio, medium="smooth"):
    w = W.custom_case(dim, n, N, m_f, dtype, medium)
    w.ratio = ratio
    w.u0 = w.cast(W.periodic_gaussian(dim, n, [0.35] * dim, 0.12))
    w.p0 = np.zeros_like(w.u0)
    return w


def _run(w, corrector, K, grad_order=4, tol=1e-13):
    import torch
    from paper_1905_00473_gb300 import binding
    ctx = _ctx(w, w.ratio, grad_order, tol)
    dt = torch.float32 if w.dtype == "f32" else torch.float64
    u0 = torch.tensor(w.u0, dtype=dt, device="cuda")
    p0 = torch.tensor(w.p0, dtype=dt, device="cuda")
    us = torch.zeros((w.n_slices + 1,) + w.shape, dtype=dt, device="cuda")
    vs = torch.zeros_like(us)
    out = binding.pr_iterate(ctx, u0, p0, K, CORR[corrector], us, vs)
    return us.double().cpu().numpy(), vs.double().cpu().numpy(), out["residual"], out["rank"]


def test_coarse_sweep_matches_oracle(lib):
    import torch
    from paper_1905_00473_gb300 import binding
    for dim, n, dtype in ((2, 64, "f64"), (2, 256, "f32"), (1, 128, "f64"), (3, 16, "f64")):
        w = _case(dim, n, 3, 16, dtype, 4)
        ctx = _ctx(w, 4)
        u, v = W.slice_states(w, seed=3)
        dt = torch.float32 if dtype == "f32" else torch.float64
        ud, vd = torch.tensor(u, dtype=dt, device="cuda"), torch.tensor(v, dtype=dt, device="cuda")
        nc = n // 4
        U = torch.zeros((3,) + (nc,) * dim, dtype=dt, device="cuda")
        V = torch.zeros_like(U)
        binding.pr_coarse_sweep(ctx, ud, vd, U, V)
        Pr = _problem(w, "plain")
        for s in range(3):
            Ur, Vr = parareal.C(Pr, *parareal.R(Pr, u[s], v[s]))
            e = energy.relative_energy_error(U[s].double().cpu().numpy(), V[s].double().cpu().numpy(),
                                             Ur, Vr, Pr.c_coarse, Pr.dx_c)
            assert e <= (1e-11 if dtype == "f64" else 1e-5), (dim, n, s, e)


@pytest.mark.parametrize("corrector", ["procrustes", "omega1", "plain"])
@pytest.mark.parametrize("dim,n,ratio", [(1, 64, 4), (2, 32, 2)])
def test_iterations_match_oracle_fp64(lib, corrector, dim, n, ratio):
    w = _case(dim, n, 5, 8, "f64", ratio)
    K = 3
    us, vs, res, rk = _run(w, corrector, K)
    recs = parareal.iterate(_problem(w, corrector), w.u0, w.p0, K)
    final = recs[-1].states
    scale = max(np.max(np.abs(s[0])) for s in final)
    for nn in range(w.n_slices + 1):
        assert np.max(np.abs(us[nn] - final[nn][0])) <= 1e-9 * scale, (corrector, nn)
        assert np.max(np.abs(vs[nn] - final[nn][1])) <= 1e-9 * scale / w.dt_com, (corrector, nn)
    if corrector == "procrustes":
        assert rk == [r.rank for r in recs]
        np.testing.assert_allclose(res, [r.residual for r in recs], rtol=1e-6, atol=1e-12)


def test_initial_guess_matches_oracle(lib):
    w = _case(2, 64, 4, 8, "f64", 4)
    us, vs, _, _ = _run(w, "plain", 0)
    ref = parareal.initial_guess(_problem(w, "plain"), w.u0, w.p0)
    for nn in range(5):
        np.testing.assert_allclose(us[nn], ref[nn][0], atol=1e-11)
        np.testing.assert_allclose(vs[nn], ref[nn][1], atol=1e-9)


@pytest.mark.parametrize("corrector", ["procrustes", "plain"])
def test_finite_termination_on_gpu(lib, corrector):
    """After K = N iterations every state equals the serial fine solution
    (Alg. 3; the theta terms cancel), here with the GPU's own fine sweep."""
    for dtype, tol in (("f64", 1e-10), ("f32", 1e-4)):
        w = _case(2, 256 if dtype == "f32" else 64, 4, 12, dtype, 4, "inclusion")
        us, vs, _, _ = _run(w, corrector, w.n_slices)
        Pr = _problem(w, corrector)
        ref = parareal.serial_fine(Pr, w.u0, w.p0)
        for nn in range(1, w.n_slices + 1):
            e = energy.relative_energy_error(us[nn], vs[nn], ref[nn][0], ref[nn][1], w.c, w.dx_f)
            assert e <= tol, (dtype, corrector, nn, e)


def test_fp32_iterations_within_1e4_energy_bound(lib):
    """FP32 context vs FP64 oracle after K iterations of the Procrustes method:
    relative energy-norm error of every state <= 1e-4."""
    w = _case(2, 256, 6, 16, "f32", 4, "inclusion")
    K = 3
    us, vs, res, rk = _run(w, "procrustes", K, tol=1e-6)
    recs = parareal.iterate(_problem(w, "procrustes", tol=1e-6), w.u0, w.p0, K)
    for nn in range(1, w.n_slices + 1):
        s = recs[-1].states[nn]
        e = energy.relative_energy_error(us[nn], vs[nn], s[0], s[1], w.c, w.dx_f)
        assert e <= 1e-4, (nn, e)


def test_update_svd_matches_oracle(lib):
    import torch
    from paper_1905_00473_gb300 import binding
    w = _case(2, 32, 6, 8, "f64", 4)
    ctx = _ctx(w, 4, tol=1e-13)
    rows = ctx.rows
    rng = np.random.default_rng(0)
    U = S = V = None
    for k in range(3):
        F = rng.standard_normal((rows, 6))
        G = rng.standard_normal((rows, 6))
        binding.pr_procrustes_correct(ctx, torch.tensor(F.T.copy(), device="cuda"),
                                      torch.tensor(G.T.copy(), device="cuda"))
        U, S, V = procrustes.update_svd(U, S, V, F, G, 1e-13)
        g = rng.standard_normal(rows)
        out = torch.zeros(rows, dtype=torch.float64, device="cuda")
        rk = binding.pr_procrustes_apply(ctx, torch.tensor(g, device="cuda"), out)
        assert rk == S.size
        np.testing.assert_allclose(out.cpu().numpy(), U @ (V.T @ g), atol=1e-10 * np.abs(g).max())
    binding.pr_procrustes_reset(ctx)
    assert binding.pr_procrustes_apply(ctx) == 0


def test_papers_residual_table_on_gpu(lib):
    """Sec. 6.4 table (middle column) reproduced by the GPU driver in FP64:
    1D c = 1, Dx = 0.01, Dt_com = 0.05, Dt/Dx = 0.5, Dt/dt = 20, T = 10, one grid."""
    import torch
    from paper_1905_00473_gb300 import binding
    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "grad_order_table.json")))
    n = 100
    x = np.arange(n) / n - 0.5
    u0 = np.cos(10 * math.pi * x) * np.exp(-100 * x ** 2)
    c = torch.ones(n, dtype=torch.float64, device="cuda")
    dt_f = 0.5 / n / 20
    for key, order in (("2", 2), ("4", 4)):
        ctx = binding.pr_create(1, n, 1, c, dt_f, 20 * dt_f, 200, 10.0, dtype=binding.PR_F64,
                                grad_order=order, tol=1e-14)
        us = torch.zeros((201, n), dtype=torch.float64, device="cuda")
        vs = torch.zeros_like(us)
        res = binding.pr_iterate(ctx, torch.tensor(u0, device="cuda"),
                                 torch.zeros(n, dtype=torch.float64, device="cuda"), 3,
                                 binding.PR_CORR_PROCRUSTES, us, vs)["residual"]
        assert abs(np.mean(res) / golden["mean_relative_residual"][key] - 1) < 0.005, (key, res)


def test_error_history_and_early_stop(lib):
    """err_hist against a reference and the early stop at tol_err: with the
    serial fine solution as reference the error at T reaches roundoff by
    K = N (finite termination), so a loose tolerance stops earlier."""
    import torch
    from paper_1905_00473_gb300 import binding
    w = _case(2, 64, 4, 12, "f64", 4)
    ctx = _ctx(w, 4)
    Pr = _problem(w, "procrustes")
    ref = parareal.serial_fine(Pr, w.u0, w.p0)
    dt = torch.float64
    args = (torch.tensor(w.u0, dtype=dt, device="cuda"), torch.tensor(w.p0, dtype=dt, device="cuda"))
    us = torch.zeros((5,) + w.shape, dtype=dt, device="cuda")
    vs = torch.zeros_like(us)
    ur = torch.tensor(ref[-1][0], dtype=dt, device="cuda")
    vr = torch.tensor(ref[-1][1], dtype=dt, device="cuda")
    out = binding.pr_iterate(ctx, *args, 4, binding.PR_CORR_PROCRUSTES, us, vs, ur, vr, 0.0)
    assert out["k_done"] == 4 and len(out["err"]) == 4
    recs = parareal.iterate(Pr, w.u0, w.p0, 4)
    for k, rec in enumerate(recs):
        e = energy.relative_energy_error(rec.states[-1][0], rec.states[-1][1], ref[-1][0], ref[-1][1],
                                         w.c, w.dx_f)
        assert abs(out["err"][k] - e) <= 1e-8 + 1e-6 * e, (k, out["err"][k], e)
    assert out["err"][-1] < 1e-10
    stop = binding.pr_iterate(ctx, *args, 4, binding.PR_CORR_PROCRUSTES, us, vs, ur, vr,
                              out["err"][1] * 1.0001)
    assert stop["k_done"] == 2


@pytest.mark.gpu
def test_phase_timers_cover_the_call(lib):
    """pr_iterate_phases: the four phase totals of the last call (Sec. 7.2.4
    table columns) are non-negative, the parallel, corrector and serial phases
    are non-zero once an iteration ran, and together they stay within the
    call's wall time."""
    import time

    import torch
    from paper_1905_00473_gb300 import binding
    w = _case(2, 64, 4, 12, "f64", 4)
    ctx = _ctx(w, 4)
    dt = torch.float64
    args = (torch.tensor(w.u0, dtype=dt, device="cuda"), torch.tensor(w.p0, dtype=dt, device="cuda"))
    us = torch.zeros((5,) + w.shape, dtype=dt, device="cuda")
    vs = torch.zeros_like(us)
    assert all(v == 0.0 for v in binding.pr_iterate_phases(ctx).values())
    binding.pr_iterate(ctx, *args, 1, binding.PR_CORR_PROCRUSTES, us, vs)   # library set-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    binding.pr_iterate(ctx, *args, 3, binding.PR_CORR_PROCRUSTES, us, vs)
    wall_ms = 1e3 * (time.perf_counter() - t0)
    ph = binding.pr_iterate_phases(ctx)
    assert all(v >= 0.0 for v in ph.values()), ph
    assert ph["parallel_ms"] > 0 and ph["corrector_ms"] > 0 and ph["serial_update_ms"] > 0, ph
    assert sum(ph.values()) <= wall_ms * 1.05 + 0.5, (ph, wall_ms)


def _run_workload(w, corrector, K, tol):
    """pr_iterate on a named workload (its own u0, p0, ratio, grad order)."""
    import torch
    from paper_1905_00473_gb300 import binding
    ctx = _ctx(w, w.ratio, w.grad_order, tol)
    dt = torch.float32 if w.dtype == "f32" else torch.float64
    u0 = torch.tensor(w.u0, dtype=dt, device="cuda")
    p0 = torch.tensor(w.p0, dtype=dt, device="cuda")
    us = torch.zeros((w.n_slices + 1,) + w.shape, dtype=dt, device="cuda")
    vs = torch.zeros_like(us)
    out = binding.pr_iterate(ctx, u0, p0, K, CORR[corrector], us, vs)
    return us.double().cpu().numpy(), vs.double().cpu().numpy(), out


@pytest.mark.parametrize("K", [1, 2, 4, 8])
def test_config1_iterations_match_oracle(lib, K):
    """The 1D FP64 workload in full (n = 128 / 32, N = 8, Procrustes, tol 1e-13,
    K up to N = 8): every state u^{K+1}_n of the GPU driver equals the oracle's
    to ~1e-9 relative in the energy norm, and the ranks agree."""
    w = W.config1()
    us, vs, out = _run_workload(w, "procrustes", K, 1e-13)
    recs = parareal.iterate(_problem(w, "procrustes", tol=1e-13), w.u0, w.p0, K)
    assert out["rank"] == [r.rank for r in recs]
    final = recs[-1].states
    for nn in range(1, w.n_slices + 1):
        e = energy.relative_energy_error(us[nn], vs[nn], final[nn][0], final[nn][1], w.c, w.dx_f)
        assert e <= 1e-9, (K, nn, e)


@pytest.mark.slow
def test_config2_iterations_match_oracle_fp32(lib):
    """The smooth 2D FP32 workload at full size (512^2 / 128^2, N = 32, m_F =
    192, Procrustes with the rank tolerance of its time-to-1e-4 run, 1e-7),
    K = 2 iterations against the FP64 oracle on the same FP32-rounded inputs:
    relative energy-norm error of every state <= 1e-4 (the FP32 parareal
    bound).  The oracle takes about a minute here."""
    w = W.config2()
    K, tol = 2, 1e-7
    us, vs, out = _run_workload(w, "procrustes", K, tol)
    recs = parareal.iterate(_problem(w, "procrustes", tol=tol), w.u0, w.p0, K)
    final = recs[-1].states
    worst = 0.0
    for nn in range(1, w.n_slices + 1):
        e = energy.relative_energy_error(us[nn], vs[nn], final[nn][0], final[nn][1], w.c, w.dx_f)
        worst = max(worst, e)
    assert worst <= 1e-4, worst
    assert out["rank"] == [r.rank for r in recs]


def test_update_svd_fp32_context_matches_oracle(lib):
    """UpdateSVD of an FP32 context (tensor-core split-TF32 projections and
    deflations, reorthogonalised) against the FP64 oracle: three updates of
    well-conditioned data, Omega g to 1e-6 relative."""
    import torch
    from paper_1905_00473_gb300 import binding
    w = _case(2, 64, 6, 8, "f32", 4)
    ctx = _ctx(w, 4, tol=1e-10)
    rows = ctx.rows
    rng = np.random.default_rng(1)
    U = S = V = None
    for k in range(3):
        F = rng.standard_normal((rows, 6))
        G = rng.standard_normal((rows, 6))
        binding.pr_procrustes_correct(ctx, torch.tensor(F.T.copy(), device="cuda"),
                                      torch.tensor(G.T.copy(), device="cuda"))
        U, S, V = procrustes.update_svd(U, S, V, F, G, 1e-10)
        g = rng.standard_normal(rows)
        out = torch.zeros(rows, dtype=torch.float64, device="cuda")
        rk = binding.pr_procrustes_apply(ctx, torch.tensor(g, device="cuda"), out)
        assert rk == S.size
        ref = U @ (V.T @ g)
        assert np.linalg.norm(out.cpu().numpy() - ref) <= 1e-6 * np.linalg.norm(ref), k
    binding.pr_check(ctx)


@pytest.mark.parametrize("case", ["dependent", "in_span"])
def test_fp32_update_svd_with_degenerate_blocks(lib, case):
    """UpdateSVD in an FP32 context (tensor-core products, Cholesky QR twice,
    eigenproblem SVD with the Newton-Schulz re-orthonormalisation, the FP32
    copies of the bases in the apply) on blocks the QR must handle: columns
    that repeat earlier ones ("dependent") and a second block that lies in the
    span of the first ("in_span", the deflated residual is rounding noise).
    Omega g matches the oracle's X Y^T g to FP32 accuracy and the rank agrees."""
    import torch
    from paper_1905_00473_gb300 import binding
    w = _case(2, 64, 8, 8, "f32", 4)
    ctx = _ctx(w, 4, tol=1e-5)
    rows = ctx.rows
    rng = np.random.default_rng(11)
    base_f = rng.standard_normal((rows, 8)) * np.logspace(0, -1.5, 8)
    base_g = rng.standard_normal((rows, 8)) * np.logspace(0, -1.5, 8)
    blocks = []
    if case == "dependent":
        F, G = base_f.copy(), base_g.copy()
        F[:, 5] = F[:, 1]
        F[:, 7] = 2.0 * F[:, 0] - F[:, 2]
        G[:, 6] = G[:, 3]
        blocks.append((F, G))
    else:
        blocks.append((base_f, base_g))
        mix = rng.standard_normal((8, 8))
        blocks.append((base_f @ mix, base_g @ mix))
    U = S = V = None
    for F, G in blocks:
        binding.pr_procrustes_correct(ctx, torch.tensor(F.T.copy(), device="cuda"),
                                      torch.tensor(G.T.copy(), device="cuda"))
        U, S, V = procrustes.update_svd(U, S, V, F, G, 1e-5)
        g = rng.standard_normal(rows)
        out = torch.zeros(rows, dtype=torch.float64, device="cuda")
        rk = binding.pr_procrustes_apply(ctx, torch.tensor(g, device="cuda"), out)
        binding.pr_check(ctx)
        assert rk == S.size, (rk, S.size)
        ref = U @ (V.T @ g)
        err = np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(g)
        assert err <= 1e-5, err
