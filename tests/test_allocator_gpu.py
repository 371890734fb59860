"""The caller allocator of pr_set_allocator (the survey's ownership rule:
context memory may come from the caller's pool, e.g. PyTorch's caching
allocator).  Every device allocation a context makes must go through the
pair and come back through it, and the results must not depend on where the
memory came from."""
import gc

import numpy as np
import pytest

from paper_1905_00473_gb300 import workloads as W
from tests import _parity as P

pytestmark = pytest.mark.gpu


class _Counting:
    def __init__(self, fail_after=None):
        import torch
        self.torch = torch
        self.live = {}
        self.calls = 0
        self.fail_after = fail_after

    def alloc(self, nbytes, dev):
        self.calls += 1
        if self.fail_after is not None and self.calls > self.fail_after:
            return 0
        p = self.torch.cuda.caching_allocator_alloc(nbytes, device=dev)
        self.live[p] = nbytes
        return p

    def release(self, ptr):
        assert ptr in self.live, "released a pointer the allocator did not hand out"
        del self.live[ptr]
        self.torch.cuda.caching_allocator_delete(ptr)


def _run(w, u, v):
    import torch
    from paper_1905_00473_gb300 import binding
    ctx = P.make_ctx(w)
    ug, vg = P.run_gpu(ctx, u, v, "f32")
    u0 = torch.tensor(w.u0, dtype=torch.float32, device="cuda")
    us = torch.zeros((w.n_slices + 1,) + w.shape, dtype=torch.float32, device="cuda")
    vs = torch.zeros_like(us)
    binding.pr_iterate(ctx, u0, torch.zeros_like(u0), 2, binding.PR_CORR_PROCRUSTES, us, vs)
    binding.pr_check(ctx)
    return ctx, ug, vg, us.cpu().numpy(), vs.cpu().numpy()


def test_context_memory_from_the_callers_pool(lib):
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(2, 256, 3, 20, "f32", "inclusion", seed=4)
    u, v = W.slice_states(w, seed=4)
    ctx0, ug0, vg0, us0, vs0 = _run(w, u, v)          # cudaMalloc
    del ctx0
    a = _Counting()
    binding.pr_set_allocator(a.alloc, a.release)
    try:
        ctx1, ug1, vg1, us1, vs1 = _run(w, u, v)
    finally:
        binding.pr_set_allocator(None, None)
    assert a.calls > 10 and len(a.live) > 0          # kappa, scratch, driver and SVD buffers
    assert np.array_equal(ug0, ug1) and np.array_equal(vg0, vg1)
    assert np.array_equal(us0, us1) and np.array_equal(vs0, vs1)
    del ctx1
    gc.collect()
    assert not a.live, f"{len(a.live)} allocations not released"


def test_failing_allocator_reports_and_releases(lib):
    from paper_1905_00473_gb300 import binding
    w = W.custom_case(2, 256, 3, 20, "f32", "smooth", seed=5)
    a = _Counting(fail_after=3)
    binding.pr_set_allocator(a.alloc, a.release)
    try:
        with pytest.raises(binding.PrError):
            P.make_ctx(w)
    finally:
        binding.pr_set_allocator(None, None)
    gc.collect()
    assert not a.live
    with pytest.raises(ValueError):
        binding.pr_set_allocator(a.alloc, None)
