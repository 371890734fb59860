"""The cluster-resident 2D path (pr_set_resident): every kick of a slice in
one launch, the slice held in the shared memory of one thread-block cluster.
It runs the fused kernels' pass plan with the same operations in the same
order, so its outputs must equal the per-pass launches bit for bit, and both
must match the FP64 oracle (Sec. 3.1 velocity Verlet)."""
import numpy as np
import pytest

from paper_1905_00473_gb300 import workloads as W
from tests import _parity as P

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,N,m_f", [
    (128, 3, 48),   # 49 levels: 8 + 4 x 8 + 9 (the coarse grid of the 512^2 workload)
    (128, 2, 20),   # 21 levels: 8, 8, 5
    (256, 3, 7),    # one pass of 8 levels, half kicks at both ends
    (256, 2, 16),   # 17 levels: 8 + 9
    (128, 1, 1),    # two levels
    (256, 4, 12),   # 13 levels: 8 + 5
])
def test_resident_equals_per_pass_and_oracle(lib, n, N, m_f):
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(2, n, N, m_f, "f32", "inclusion", seed=40 + n + m_f)
    ctx = P.make_ctx(w)
    u, v = W.slice_states(w, seed=9)
    binding.pr_set_resident(ctx, True)
    binding.pr_profile(ctx, True)
    ug1, vg1 = P.run_gpu(ctx, u, v, "f32")
    binding.pr_profile(ctx, False)
    assert binding.pr_profile_read(ctx, 3)[0] == 1
    assert binding.pr_profile_read(ctx, 0)[0] == 0 and binding.pr_profile_read(ctx, 1)[0] == 0
    binding.pr_set_resident(ctx, False)
    binding.pr_profile(ctx, True)
    ug2, vg2 = P.run_gpu(ctx, u, v, "f32")
    binding.pr_profile(ctx, False)
    assert binding.pr_profile_read(ctx, 3)[0] == 0 and binding.pr_profile_read(ctx, 0)[0] >= 1
    assert np.array_equal(ug1, ug2) and np.array_equal(vg1, vg2)
    for s in range(N):
        ur, vr = P.oracle_slice(w, u[s], v[s])
        assert P.slice_errors(w, ug1[s], vg1[s], ur, vr)[0] <= P.TOL_ENERGY_F32


def test_resident_default_follows_the_width(lib):
    """Without a call to the setter, 128^2 slices run resident and 256^2
    slices run the per-pass kernels."""
    from paper_1905_00473_gb300 import binding
    for n, kind in ((128, 3), (256, 0)):
        w = W.custom_case(2, n, 2, 12, "f32", "smooth", seed=n)
        ctx = P.make_ctx(w)
        u, v = W.slice_states(w, seed=3)
        binding.pr_profile(ctx, True)
        P.run_gpu(ctx, u, v, "f32")
        binding.pr_profile(ctx, False)
        assert binding.pr_profile_read(ctx, kind)[0] >= 1


def test_resident_in_place_subset(lib):
    """In place on slices 1..2 of 4: the others untouched, the result equal to
    the out-of-place per-pass one."""
    import torch
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(2, 128, 4, 48, "f32", "smooth", seed=5)
    ctx = P.make_ctx(w)
    u, v = W.slice_states(w, seed=10)
    ud = torch.tensor(u, dtype=torch.float32, device="cuda")
    vd = torch.tensor(v, dtype=torch.float32, device="cuda")
    keep_u, keep_v = ud.clone(), vd.clone()
    binding.pr_set_resident(ctx, True)
    binding.pr_fine_all_slices(ctx, ud, vd, ud, vd, 1, 3)
    binding.pr_check(ctx)
    binding.pr_set_resident(ctx, False)
    uo, vo = torch.empty_like(ud), torch.empty_like(vd)
    binding.pr_fine_all_slices(ctx, keep_u, keep_v, uo, vo, 1, 3)
    binding.pr_check(ctx)
    for s in (0, 3):
        assert torch.equal(ud[s], keep_u[s]) and torch.equal(vd[s], keep_v[s])
    for s in (1, 2):
        assert torch.equal(ud[s], uo[s]) and torch.equal(vd[s], vo[s])


def test_unsupported_widths_keep_the_per_pass_path(lib):
    """512^2 does not fit one cluster: the setter changes nothing there."""
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(2, 512, 1, 8, "f32", "smooth")
    ctx = P.make_ctx(w)
    u, v = W.slice_states(w, seed=2)
    binding.pr_set_resident(ctx, True)
    binding.pr_profile(ctx, True)
    P.run_gpu(ctx, u, v, "f32")
    binding.pr_profile(ctx, False)
    assert binding.pr_profile_read(ctx, 3)[0] == 0 and binding.pr_profile_read(ctx, 0)[0] >= 1
