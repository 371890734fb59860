"""Failure detection without a GPU fault: a bounded wait that runs out is
reported as PR_ETIMEOUT and leaves the context usable; a non-finite state is
reported as PR_EUNSTABLE by the iteration's host-side guard."""
import numpy as np
import pytest

from paper_1905_00473_gb300 import workloads as W
from tests import _parity as P

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,m_f,wide", [(256, 7, 2), (2048, 7, 1), (2048, 7, 2), (256, 23, 2)])
def test_bounded_wait_times_out_and_context_recovers(lib, n, m_f, wide):
    """m_f = 7: one fused pass of 8 levels (whole rows per CTA; at n = 2048
    rows shared by a 2-CTA cluster, wide = 1, or x-strips, wide = 2); m_f =
    23: three passes in one persistent launch, whose grid barrier every CTA
    still reaches after giving up."""
    import time
    import torch
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(2, n, 2, m_f, "f32", "smooth")
    ctx = P.make_ctx(w)
    assert binding.pr_info(ctx)["block_depth"] == 8
    binding.pr_set_wide_rows(ctx, wide)
    binding.pr_set_one_launch(ctx, m_f == 23)
    u, v = W.slice_states(w, seed=1)
    ud = torch.tensor(u, dtype=torch.float32, device="cuda")
    vd = torch.tensor(v, dtype=torch.float32, device="cuda")
    uo, vo = torch.zeros_like(ud), torch.zeros_like(vd)
    binding.pr_debug_stall_waits(ctx, True)
    t0 = time.time()
    binding.pr_fine_all_slices(ctx, ud, vd, uo, vo)
    with pytest.raises(binding.PrError) as ei:
        binding.pr_check(ctx)
    assert ei.value.status == 4 and "bounded wait" in str(ei.value)
    assert time.time() - t0 < 30
    binding.pr_check(ctx)                                 # flag cleared
    binding.pr_debug_stall_waits(ctx, False)
    ug, vg = P.run_gpu(ctx, u, v, "f32")
    for s in range(2):
        ur, vr = P.oracle_slice(w, u[s], v[s])
        assert P.slice_errors(w, ug[s], vg[s], ur, vr)[0] <= P.TOL_ENERGY_F32


def test_non_finite_state_is_reported_unstable(lib):
    import torch
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(2, 64, 3, 8, "f64", "smooth")
    c = torch.tensor(w.c, device="cuda")
    ctx = binding.pr_create(2, 64, 4, c, w.dt_f, w.dt_c, 3, w.t_final, dtype=binding.PR_F64)
    u0 = torch.tensor(W.periodic_gaussian(2, 64, (0.5, 0.5), 0.1), device="cuda")
    u0[3, 7] = float("nan")
    us = torch.zeros((4, 64, 64), dtype=torch.float64, device="cuda")
    vs = torch.zeros_like(us)
    with pytest.raises(binding.PrError) as ei:
        binding.pr_iterate(ctx, u0, torch.zeros_like(u0), 2, binding.PR_CORR_PLAIN, us, vs)
    assert ei.value.status == 5


def test_bounded_wait_inside_iterate_is_reported(lib):
    """pr_iterate reads the fine and coarse contexts' device flags after each
    iteration: a fused pass that gave up waiting makes it return PR_ETIMEOUT
    instead of states that were never propagated."""
    import torch
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(2, 256, 2, 8, "f32", "smooth")
    c = torch.tensor(w.c, dtype=torch.float32, device="cuda")
    ctx = binding.pr_create(2, 256, 4, c, w.dt_f, w.dt_c, 2, w.t_final)
    assert binding.pr_info(ctx)["block_depth"] == 8
    u0 = torch.tensor(W.periodic_gaussian(2, 256, (0.5, 0.5), 0.1), dtype=torch.float32,
                      device="cuda")
    us = torch.zeros((3, 256, 256), dtype=torch.float32, device="cuda")
    vs = torch.zeros_like(us)
    binding.pr_debug_stall_waits(ctx, True)
    with pytest.raises(binding.PrError) as ei:
        binding.pr_iterate(ctx, u0, torch.zeros_like(u0), 1, binding.PR_CORR_PLAIN, us, vs)
    assert ei.value.status == 4 and "bounded wait" in str(ei.value)
    binding.pr_debug_stall_waits(ctx, False)
    binding.pr_check(ctx)                                  # the flag was cleared by pr_iterate
    out = binding.pr_iterate(ctx, u0, torch.zeros_like(u0), 1, binding.PR_CORR_PLAIN, us, vs)
    assert out["k_done"] == 1 and torch.isfinite(us).all()
