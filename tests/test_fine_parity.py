"""GPU parity of pr_fine_all_slices (F over all slices, Alg. 3 parFor; Sec. 3.1
scheme) against the FP64 oracle on the same seeded inputs.

Bar: relative energy-norm error per slice <= 1e-5 in FP32 (the accuracy
required of an FP32 fine slice) and <= 1e-11 in FP64; the relative l2 error of u is checked too.
Small cases span several passes of the fused kernel, a ragged last pass and
the slice-crossing row ranges of its persistent work split; the full-size
configurations are checked on sampled slices against the oracle and on every
slice through the exactly conserved modified Verlet energy.
"""
import math

import numpy as np
import pytest

from oracle import energy
from paper_1905_00473_gb300 import workloads as W
from tests import _parity as P

pytestmark = pytest.mark.gpu


def _check_all(w, ctx, u, v, slices=None):
    ug, vg = P.run_gpu(ctx, u, v, w.dtype)
    slices = range(u.shape[0]) if slices is None else slices
    worst = 0.0
    for s in slices:
        ur, vr = P.oracle_slice(w, u[s], v[s])
        e, l2 = P.slice_errors(w, ug[s], vg[s], ur, vr)
        worst = max(worst, e)
        assert e <= P.tol_for(w), (w.name, s, e)
        assert l2 <= P.tol_for(w), (w.name, s, l2)
    return ug, vg, worst


@pytest.mark.parametrize("cols", [2, 4])   # both fused kernels (pr_set_fused_columns)
@pytest.mark.parametrize("n,m_f,N,medium", [
    (256, 20, 3, "inclusion"),   # passes of 8, 8, 5 levels; rows split across 3 slices
    (256, 7, 2, "smooth"),       # one full pass of 8 levels
    (256, 1, 2, "smooth"),       # two levels: single short pass
    (512, 16, 2, "smooth"),      # 17 levels: 8 + 9 (four columns) or 8, 8, 1 (two)
    (128, 20, 3, "smooth"),      # narrowest tile: one warp per CTA with four columns
    (128, 15, 1, "inclusion"),   # 16 levels, every CTA's rows inside one slice
    (1024, 12, 1, "inclusion"),  # widest tile, 13 levels
])
def test_fused_2d_matches_oracle(lib, n, m_f, N, medium, cols):
    w = W.custom_case(2, n, N, m_f, "f32", medium)
    ctx = P.make_ctx(w)
    from paper_1905_00473_gb300 import binding
    binding.pr_set_fused_columns(ctx, cols)
    binding.pr_set_resident(ctx, False)   # the per-pass kernels (test_resident_gpu.py: the other path)
    assert binding.pr_info(ctx)["block_depth"] == 8
    u, v = W.slice_states(w, seed=1)
    _check_all(w, ctx, u, v)


@pytest.mark.parametrize("m_f,N", [(9, 2), (4, 1)])
def test_fused_2d_strips_2048(lib, m_f, N):
    """n = 2048 at depth 4 runs in two x-strips of 1040 columns (8-column halo
    each side, 1024 final): passes of 4, 4, 2 levels (m_f = 9) or 4 + 1 levels
    (m_f = 4), with rows of two slices and two strips split across the CTAs."""
    w = W.custom_case(2, 2048, N, m_f, "f32", "inclusion")
    ctx = P.make_ctx(w, block_depth=4)
    from paper_1905_00473_gb300 import binding
    assert binding.pr_info(ctx)["block_depth"] == 4
    u, v = W.slice_states(w, seed=11)
    _check_all(w, ctx, u, v)


@pytest.mark.parametrize("m_f,N,passes", [
    (20, 3, (3, 0)),   # 21 levels: first pass, middle pass, general pass of 5
    (16, 2, (2, 1)),   # 17 levels: 8 + 8 fused, the final half kick alone
    (7, 1, (1, 0)),    # 8 levels in one general pass (half kicks at both ends)
])
def test_fused_2d_cluster_rows_2048(lib, m_f, N, passes):
    """n = 2048 at depth 8 with the cluster rows (pr_set_wide_rows 1): every
    row shared by the two CTAs of a thread-block cluster, which exchange the
    x-edges of their half-rows through distributed shared memory.  The
    periodic wrap in x crosses from one CTA to the other at both ends; rows
    of several slices are split across the clusters."""
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(2, 2048, N, m_f, "f32", "inclusion", seed=20 + m_f)
    ctx = P.make_ctx(w)
    binding.pr_set_wide_rows(ctx, 1)
    assert binding.pr_info(ctx)["block_depth"] == 8
    u, v = W.slice_states(w, seed=12)
    binding.pr_profile(ctx, True)
    _check_all(w, ctx, u, v)
    binding.pr_profile(ctx, False)
    assert (binding.pr_profile_read(ctx, 0)[0], binding.pr_profile_read(ctx, 1)[0]) == passes


@pytest.mark.parametrize("wide", [1, 2])
def test_fused_2d_cluster_rows_2048_whole_slices(lib, wide):
    """160 slices of 2048^2, in cluster rows (1) or x-strips (2): a row range
    holds whole slices, whose halo rows wrap around the periodic slice at
    both ends.  Four distinct slice states are tiled over the batch; the
    first, two middle and the last slices are checked against the oracle."""
    import torch
    from paper_1905_00473_gb300 import binding
    N = 160
    w = W.custom_case(2, 2048, N, 9, "f32", "inclusion")   # 10 levels: 8 + 2
    ctx = P.make_ctx(w)
    binding.pr_set_wide_rows(ctx, wide)
    w4 = W.custom_case(2, 2048, 4, 9, "f32", "inclusion")
    u4, v4 = W.slice_states(w4, seed=13)
    u4d = torch.tensor(u4, dtype=torch.float32, device="cuda")
    v4d = torch.tensor(v4, dtype=torch.float32, device="cuda")
    reps = N // 4
    ud = u4d.repeat(reps, 1, 1).contiguous()
    vd = v4d.repeat(reps, 1, 1).contiguous()
    uo = torch.full_like(ud, float("nan"))
    vo = torch.full_like(vd, float("nan"))
    binding.pr_fine_all_slices(ctx, ud, vd, uo, vo)
    binding.pr_check(ctx)
    for s in (0, 77, 82, N - 1):
        ur, vr = P.oracle_slice(w, u4[s % 4], v4[s % 4])
        ug = uo[s].double().cpu().numpy()
        vg = vo[s].double().cpu().numpy()
        e, l2 = P.slice_errors(w, ug, vg, ur, vr)
        assert e <= P.tol_for(w), (s, e)
        assert l2 <= P.tol_for(w), (s, l2)


@pytest.mark.parametrize("cols", [2, 4])
@pytest.mark.parametrize("n,N", [(256, 1300), (512, 330)])
def test_fused_2d_whole_slice_segments(lib, n, N, cols):
    """So many slices that a CTA's row range holds whole slices: segments of
    H = n rows whose halo rows wrap around the periodic slice on both sides
    (row indices up to 2n + L).  Four distinct slice states are tiled over
    the batch; the oracle checks the first, a middle and the last slices."""
    w = W.custom_case(2, n, N, 9, "f32", "inclusion")   # 10 levels: 8 + 2
    ctx = P.make_ctx(w)
    from paper_1905_00473_gb300 import binding
    binding.pr_set_fused_columns(ctx, cols)
    binding.pr_set_resident(ctx, False)
    w4 = W.custom_case(2, n, 4, 9, "f32", "inclusion")
    u4, v4 = W.slice_states(w4, seed=7)
    reps = (N + 3) // 4
    u = np.ascontiguousarray(np.tile(u4, (reps, 1, 1))[:N])
    v = np.ascontiguousarray(np.tile(v4, (reps, 1, 1))[:N])
    _check_all(w, ctx, u, v, slices=[0, 1, N // 2, N - 1])


@pytest.mark.parametrize("dim,n,m_f,N,dtype", [
    (2, 48, 9, 3, "f32"),      # grid the fused kernel does not take: one level per pass
    (1, 64, 13, 4, "f32"),
    (3, 16, 6, 3, "f32"),
    (2, 40, 9, 2, "f64"),
    (3, 12, 5, 2, "f64"),
])
def test_single_level_path_matches_oracle(lib, dim, n, m_f, N, dtype):
    w = W.custom_case(dim, n, N, m_f, dtype)
    ctx = P.make_ctx(w)
    u, v = W.slice_states(w, seed=2)
    _check_all(w, ctx, u, v)


@pytest.mark.parametrize("n,m_f", [(256, 8), (256, 16), (512, 24), (1024, 8)])
def test_first_pass_and_nine_level_last_pass(lib, n, m_f):
    """Sweeps of 8 k + 1 levels: the first pass runs the specialised kernel
    with the half kick at level 0, and the lone final level joins the last
    pass (9 levels), so 9, 17 and 25 levels take 1, 2 and 3 fused passes."""
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(2, n, 3, m_f, "f32", "inclusion", seed=n + m_f)
    ctx = P.make_ctx(w)
    binding.pr_set_resident(ctx, False)
    u, v = W.slice_states(w, seed=8)
    for one_launch in (False, True):
        binding.pr_set_one_launch(ctx, one_launch)
        binding.pr_profile(ctx, True)
        _check_all(w, ctx, u, v)
        binding.pr_profile(ctx, False)
        fused, _ = binding.pr_profile_read(ctx, 0)
        single, _ = binding.pr_profile_read(ctx, 1)
        sweeps, _ = binding.pr_profile_read(ctx, 2)
        passes = (m_f + 1) // 8
        if one_launch and passes >= 2:   # every pass inside one launch
            assert (fused, single, sweeps) == (0, 0, 1), (fused, single, sweeps)
        else:
            assert (fused, single, sweeps) == (passes, 0, 0), (fused, single, sweeps)


@pytest.mark.parametrize("dim,n,m_f,N", [(2, 18, 9, 3), (1, 30, 11, 2), (3, 10, 5, 2)])
def test_single_level_path_width_not_multiple_of_4(lib, dim, n, m_f, N):
    """Widths the four-point form of the one-level kernel does not take fall
    back to one point per thread (coarse ratio 2 keeps n/ratio integral)."""
    w = W.custom_case(dim, n, N, m_f, "f32")
    w.ratio = 2
    ctx = P.make_ctx(w)
    u, v = W.slice_states(w, seed=6)
    _check_all(w, ctx, u, v)


def test_forced_single_level_path_on_fused_geometry(lib):
    w = W.custom_case(2, 256, 2, 10, "f32", "inclusion")
    ctx = P.make_ctx(w, block_depth=1)
    from paper_1905_00473_gb300 import binding
    assert binding.pr_info(ctx)["block_depth"] == 1
    u, v = W.slice_states(w, seed=3)
    _check_all(w, ctx, u, v)


def test_config1_1d_fp64_full(lib):
    w = W.config1()
    ctx = P.make_ctx(w)
    u, v = W.slice_states(w, seed=4)
    _check_all(w, ctx, u, v)


def test_inplace_and_slice_subset(lib):
    import torch
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(2, 256, 4, 12, "f32", "smooth")
    ctx = P.make_ctx(w)
    u, v = W.slice_states(w, seed=5)
    ud = torch.tensor(u, dtype=torch.float32, device="cuda")
    vd = torch.tensor(v, dtype=torch.float32, device="cuda")
    u_keep, v_keep = ud.clone(), vd.clone()
    binding.pr_fine_all_slices(ctx, ud, vd, ud, vd, 1, 3)   # in place, slices 1 and 2
    binding.pr_check(ctx)
    ug, vg = ud.double().cpu().numpy(), vd.double().cpu().numpy()
    for s in (0, 3):   # untouched
        assert torch.equal(ud[s], u_keep[s]) and torch.equal(vd[s], v_keep[s])
    for s in (1, 2):
        ur, vr = P.oracle_slice(w, u[s], v[s])
        e, _ = P.slice_errors(w, ug[s], vg[s], ur, vr)
        assert e <= P.TOL_ENERGY_F32
    # one-pass sweep in place goes through scratch
    w1 = W.custom_case(2, 256, 2, 3, "f32", "smooth")
    ctx1 = P.make_ctx(w1)
    u1, v1 = W.slice_states(w1, seed=6)
    ug1, vg1 = P.run_gpu(ctx1, u1, v1, "f32", inplace=True)
    for s in range(2):
        ur, vr = P.oracle_slice(w1, u1[s], v1[s])
        assert P.slice_errors(w1, ug1[s], vg1[s], ur, vr)[0] <= P.TOL_ENERGY_F32


def test_empty_range_and_invalid_arguments(lib):
    import torch
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(2, 256, 3, 8, "f32")
    ctx = P.make_ctx(w)
    u = torch.zeros((3, 256, 256), device="cuda")
    v = torch.zeros_like(u)
    uo = torch.full_like(u, 7.0)
    vo = torch.full_like(u, 7.0)
    binding.pr_fine_all_slices(ctx, u, v, uo, vo, 2, 2)   # empty: no-op
    binding.pr_check(ctx)
    assert bool((uo == 7.0).all())
    with pytest.raises(binding.PrError) as ei:
        binding.pr_fine_all_slices(ctx, u, v, uo, vo, 2, 4)
    assert ei.value.status == 1
    with pytest.raises(binding.PrError):
        binding.pr_fine_all_slices(ctx, u, v, v, uo)       # output overlaps input
    for bad in (1, 3, 8, -2):
        with pytest.raises(binding.PrError) as ei:
            binding.pr_set_fused_columns(ctx, bad)
        assert ei.value.status == 1
    big = torch.zeros(4 * 256 * 256, device="cuda")
    with pytest.raises(binding.PrError):
        binding.pr_fine_all_slices(ctx, big[1:1 + 3 * 65536].view(3, 256, 256), v, uo, vo)  # unaligned
    # zero input stays exactly zero
    binding.pr_fine_all_slices(ctx, u, v, uo, vo)
    binding.pr_check(ctx)
    assert not bool(uo.any()) and not bool(vo.any())


def test_create_validates_steps_and_cfl(lib):
    import torch
    from paper_1905_00473_gb300 import binding
    c = torch.ones(64 * 64, device="cuda")
    dx = 1 / 64
    with pytest.raises(binding.PrError):   # (T/N)/dt_f not an integer
        binding.pr_create(2, 64, 4, c, 0.3 * dx, 1.2 * dx, 4, 4 * 10.5 * 0.3 * dx)
    with pytest.raises(binding.PrError):   # CFL violated on the fine grid
        binding.pr_create(2, 64, 4, c, 0.8 * dx, 0.8 * dx, 4, 4 * 0.8 * dx)
    with pytest.raises(binding.PrError):   # c <= 0
        binding.pr_create(2, 64, 4, c * 0, 0.2 * dx, 0.8 * dx, 4, 4 * 0.8 * dx)
    with pytest.raises(binding.PrError):   # ratio does not divide n
        binding.pr_create(2, 64, 5, c, 0.2 * dx, 0.8 * dx, 4, 4 * 0.8 * dx)
    ctx = binding.pr_create(2, 64, 4, c, 0.2 * dx, 0.8 * dx, 4, 4 * 0.8 * dx)
    assert binding.pr_info(ctx)["m_f"] == 4 and binding.pr_info(ctx)["m_c"] == 1


def test_energy_matches_oracle(lib):
    import torch
    from paper_1905_00473_gb300 import binding
    for w in (W.custom_case(2, 256, 3, 4, "f32", "inclusion"), W.custom_case(1, 64, 2, 4, "f64"),
              W.custom_case(3, 16, 2, 4, "f32")):
        ctx = P.make_ctx(w)
        u, v = W.slice_states(w, seed=7)
        dt = torch.float32 if w.dtype == "f32" else torch.float64
        e = binding.pr_energy(ctx, torch.tensor(u, dtype=dt, device="cuda"),
                              torch.tensor(v, dtype=dt, device="cuda"))
        for s in range(w.n_slices):
            ref = energy.discrete_wave_energy(u[s], v[s], w.c, w.dx_f, order=4)
            assert abs(e[s] - ref) <= 1e-12 * ref, (w.name, s, e[s], ref)


@pytest.mark.parametrize("cfg", ["2", "3"])
def test_full_size_configs(lib, cfg):
    """Full configuration, all slices in the bench's launch configuration:
    the oracle on two sampled slices, the conserved modified energy on all."""
    w = W.CONFIGS[cfg]()
    ctx = P.make_ctx(w)
    u, v = W.slice_states(w, seed=0)
    ug, vg = P.run_gpu(ctx, u, v, w.dtype)
    rng = np.random.default_rng(int(cfg))
    for s in sorted(rng.choice(w.n_slices, size=2, replace=False)):
        ur, vr = P.oracle_slice(w, u[s], v[s])
        e, l2 = P.slice_errors(w, ug[s], vg[s], ur, vr)
        assert e <= P.TOL_ENERGY_F32 and l2 <= P.TOL_ENERGY_F32, (cfg, s, e, l2)
    for s in range(w.n_slices):
        h0 = P.modified_energy(u[s], v[s], w.c, w.dt_f, w.dx_f)
        h1 = P.modified_energy(ug[s], vg[s], w.c, w.dt_f, w.dx_f)
        assert math.isfinite(h1) and abs(h1 - h0) <= 2e-5 * abs(h0), (cfg, s, h0, h1)


@pytest.mark.parametrize("n,N,m_f", [(1024, 5, 384), (256, 7, 20), (512, 3, 44), (128, 9, 16)])
def test_one_launch_sweep_equals_per_pass_launches(lib, n, N, m_f):
    """The whole sweep in one persistent launch (grid barrier between passes)
    computes the same level recurrence in the same order as one launch per
    pass: bit-identical outputs.  Level counts 8k + 1 (the last pass takes 9
    levels) and 8k + 5 (a short last pass) are both covered, and the result
    is checked against the oracle."""
    import torch
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(2, n, N, m_f, "f32", "inclusion")
    ctx = P.make_ctx(w)
    binding.pr_set_resident(ctx, False)
    u, v = W.slice_states(w, seed=4)
    binding.pr_set_one_launch(ctx, True)
    binding.pr_profile(ctx, True)
    ug1, vg1 = P.run_gpu(ctx, u, v, "f32")
    binding.pr_profile(ctx, False)
    assert binding.pr_profile_read(ctx, 2)[0] == 1 and binding.pr_profile_read(ctx, 0)[0] == 0
    binding.pr_set_one_launch(ctx, False)
    ug2, vg2 = P.run_gpu(ctx, u, v, "f32")
    assert np.array_equal(ug1, ug2) and np.array_equal(vg1, vg2)
    for s in (0, N - 1):
        ur, vr = P.oracle_slice(w, u[s], v[s])
        assert P.slice_errors(w, ug1[s], vg1[s], ur, vr)[0] <= P.TOL_ENERGY_F32


@pytest.mark.parametrize("n,N,m_f", [(64, 3, 7), (64, 2, 10), (128, 2, 12), (64, 4, 3)])
def test_fused_3d_passes_match_oracle(lib, n, N, m_f):
    """3D FP32 at depth 4 (2.5D blocking: xy tiles of 64 x 16 with a 4-point
    halo, z streamed): 8, 11, 13 and 4 levels give full passes, a short last
    pass and the final one-level pass, with the periodic wrap in x, y and z
    crossing tile boundaries; every slice against the oracle."""
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(3, n, N, m_f, "f32", "smooth", seed=30 + n + m_f)
    ctx = P.make_ctx(w)
    assert binding.pr_info(ctx)["block_depth"] == 4
    u, v = W.slice_states(w, seed=5)
    binding.pr_profile(ctx, True)
    _check_all(w, ctx, u, v)
    binding.pr_profile(ctx, False)
    levels = m_f + 1
    assert binding.pr_profile_read(ctx, 0)[0] == levels // 4 + (1 if levels % 4 > 1 else 0)
    assert binding.pr_profile_read(ctx, 1)[0] == (1 if levels % 4 == 1 else 0)


def test_fused_3d_inclusion_medium(lib):
    """The discontinuous medium in 3D (c = 3 inside [0.3, 0.7]^3) at depth 4."""
    w = W.custom_case(3, 64, 2, 9, "f32", "inclusion", seed=3)
    ctx = P.make_ctx(w)
    u, v = W.slice_states(w, seed=9)
    _check_all(w, ctx, u, v)


def test_fused_3d_full_size_sampled(lib):
    """The 3D differentiation workload's sweep at full size (256^3, 32 slices,
    m_F = 64, depth 4): two sampled slices against the oracle."""
    w = W.config5()
    ctx = P.make_ctx(w)
    u, v = W.slice_states(w, seed=0)
    ug, vg = P.run_gpu(ctx, u, v, w.dtype)
    for s in (3, 30):
        ur, vr = P.oracle_slice(w, u[s], v[s])
        e, l2 = P.slice_errors(w, ug[s], vg[s], ur, vr)
        assert e <= P.TOL_ENERGY_F32 and l2 <= P.TOL_ENERGY_F32, (s, e, l2)


@pytest.mark.parametrize("m_f,N", [(20, 3), (7, 1), (9, 2)])
def test_fused_2d_xstrips_2048_depth8(lib, m_f, N):
    """n = 2048 at depth 8 in three x-strips of 704 columns per row
    (pr_set_wide_rows 2: 688 final columns, an 8-column halo each side; the
    third strip overlaps the first, which alone writes the overlap): the same
    level recurrence as the cluster rows, so bit-identical outputs, and every
    slice against the oracle."""
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(2, 2048, N, m_f, "f32", "inclusion", seed=60 + m_f)
    ctx = P.make_ctx(w)
    u, v = W.slice_states(w, seed=13)
    binding.pr_set_wide_rows(ctx, 2)
    ug2, vg2 = P.run_gpu(ctx, u, v, "f32")
    binding.pr_set_wide_rows(ctx, 1)
    ug1, vg1 = P.run_gpu(ctx, u, v, "f32")
    assert np.array_equal(ug1, ug2) and np.array_equal(vg1, vg2)
    for s in range(N):
        ur, vr = P.oracle_slice(w, u[s], v[s])
        assert P.slice_errors(w, ug2[s], vg2[s], ur, vr)[0] <= P.TOL_ENERGY_F32
