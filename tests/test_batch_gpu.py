"""Batches of independent instances of uneven sizes in one captured CUDA graph
(pr_batch_*): every instance's sweep, after autotuning and on two replays of
the graph, matches the FP64 oracle like a single pr_fine_all_slices call."""
import numpy as np
import pytest

from paper_1905_00473_gb300 import workloads as W
from tests import _parity as P

pytestmark = pytest.mark.gpu


def test_batch_matches_oracle_after_autotune(lib):
    import torch
    from paper_1905_00473_gb300 import binding
    cases = [W.custom_case(2, 256, 3, 20, "f32", "inclusion", seed=1),
             W.custom_case(2, 512, 2, 12, "f32", "smooth", seed=2),
             W.custom_case(2, 1024, 1, 9, "f32", "smooth", seed=3),
             W.custom_case(2, 96, 4, 10, "f32", "smooth", seed=4),
             W.custom_case(1, 64, 3, 7, "f32", "smooth", seed=5)]
    ctxs, ui, vi, uo, vo, host = [], [], [], [], [], []
    for k, w in enumerate(cases):
        ctxs.append(P.make_ctx(w))
        u, v = W.slice_states(w, seed=10 + k)
        host.append((u, v))
        ui.append(torch.tensor(u, dtype=torch.float32, device="cuda"))
        vi.append(torch.tensor(v, dtype=torch.float32, device="cuda"))
        uo.append(torch.full_like(ui[-1], float("nan")))
        vo.append(torch.full_like(vi[-1], float("nan")))
    batch = binding.Batch(ctxs, ui, vi, uo, vo, autotune=True)
    depths = [batch.info(i)[0] for i in range(len(cases))]
    cols = [batch.info(i)[1] for i in range(len(cases))]
    assert depths[3] == 1 and depths[4] == 1          # sizes without a fused kernel
    assert all(d in (4, 8) for d in depths[:3])
    assert all(c in (2, 4) for c in cols[:3]) and cols[3] == 0 and cols[4] == 0
    for rep in range(2):
        for t in uo + vo:
            t.fill_(float("nan"))
        batch.launch()
        torch.cuda.synchronize()
        for k, w in enumerate(cases):
            u, v = host[k]
            ug, vg = uo[k].double().cpu().numpy(), vo[k].double().cpu().numpy()
            for s in range(w.n_slices):
                ur, vr = P.oracle_slice(w, u[s], v[s])
                e, _ = P.slice_errors(w, ug[s], vg[s], ur, vr)
                assert e <= P.TOL_ENERGY_F32, (rep, k, s, e)


@pytest.mark.parametrize("cols", [2, 4])
def test_depth4_kernel_matches_oracle(lib, cols):
    w = W.custom_case(2, 512, 2, 21, "f32", "inclusion")
    ctx = P.make_ctx(w, block_depth=4)
    from paper_1905_00473_gb300 import binding
    binding.pr_set_fused_columns(ctx, cols)
    assert binding.pr_info(ctx)["block_depth"] == 4
    u, v = W.slice_states(w, seed=7)
    ug, vg = P.run_gpu(ctx, u, v, "f32")
    for s in range(2):
        ur, vr = P.oracle_slice(w, u[s], v[s])
        assert P.slice_errors(w, ug[s], vg[s], ur, vr)[0] <= P.TOL_ENERGY_F32
