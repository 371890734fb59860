"""The allocation-free entry point, for callers that cannot allocate device
memory (a framework owning the whole memory pool, plugins running inside
another library's stream-ordered work, real-time loops), must compute what the
context path computes.

It keeps its scratch in one fixed device array shared by all calls, so the
test makes two calls in a row (the second sees the first call's leftovers) and
compares each with pr_fine_all_slices within the parity tolerance of the
other GPU tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1905_00473_gb300 import workloads as W
from tests import _parity as P

pytestmark = pytest.mark.gpu


def _energy_err(w, ug, vg, ur, vr):
    return max(P.slice_errors(w, ug[s], vg[s], ur[s], vr[s])[0] for s in range(ug.shape[0]))


@pytest.mark.parametrize("dim,n,N,m_f", [(2, 256, 3, 12), (1, 64, 4, 9), (3, 16, 2, 6)])
def test_noalloc_matches_context_path_twice(lib, dim, n, N, m_f):
    import torch
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(dim, n, N, m_f, "f32", "smooth")
    ctx = P.make_ctx(w)
    c = torch.tensor(w.c, dtype=torch.float32, device="cuda")
    for call, seed in enumerate((21, 22)):
        u, v = W.slice_states(w, seed=seed)
        ud = torch.tensor(u, dtype=torch.float32, device="cuda")
        vd = torch.tensor(v, dtype=torch.float32, device="cuda")
        ur, vr = torch.empty_like(ud), torch.empty_like(vd)
        binding.pr_fine_all_slices(ctx, ud, vd, ur, vr)
        un = torch.full_like(ud, float("nan"))
        vn = torch.full_like(vd, float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        binding.pr_fine_all_slices_noalloc(c, w.dt_f, w.m_f, ud, vd, un, vn)
        torch.cuda.synchronize()
        if call == 1:
            # the first call may load the kernels' code; the second, with the
            # same kernels, must leave the device's free memory unchanged
            assert torch.cuda.mem_get_info()[0] == free0
        a = [x.double().cpu().numpy() for x in (un, vn, ur, vr)]
        assert np.all(np.isfinite(a[0])) and np.all(np.isfinite(a[1]))
        err = _energy_err(w, *a)
        assert err <= P.TOL_ENERGY_F32, (call, err)


def test_noalloc_rejects_oversized_batches(lib):
    import torch
    from paper_1905_00473_gb300 import binding
    n = 1024
    c = torch.ones((n, n), device="cuda")
    u = torch.zeros((8, n, n), device="cuda")   # 8 slices of 1024^2 need ~148 MB of scratch
    with pytest.raises(binding.PrError) as ei:
        binding.pr_fine_all_slices_noalloc(c, 0.2 / n, 4, u, u, u.clone(), u.clone())
    assert ei.value.status == 1
    assert "PR_NOALLOC_SCRATCH_BYTES" in str(ei.value)
