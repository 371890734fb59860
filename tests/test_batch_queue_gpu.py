"""The uneven batch as ONE persistent work-queue kernel (pr_batch_set_mode 1):
every instance's sweep matches the FP64 oracle like a single
pr_fine_all_slices call, on two replays of the graph; agrees with the
per-instance launch chains (mode 0) to FP32 rounding; refuses instances it
does not take; the timed choice (-1) keeps a valid graph; and a wait that
gives up stops the queue and is reported on every instance, after which the
batch recovers."""
import time

import numpy as np
import pytest

from paper_1905_00473_gb300 import workloads as W
from tests import _parity as P

pytestmark = pytest.mark.gpu


def _bind(cases, seed0=10):
    import torch
    ctxs, ui, vi, uo, vo, host = [], [], [], [], [], []
    for k, w in enumerate(cases):
        ctxs.append(P.make_ctx(w))
        u, v = W.slice_states(w, seed=seed0 + k)
        host.append((u, v))
        ui.append(torch.tensor(u, dtype=torch.float32, device="cuda"))
        vi.append(torch.tensor(v, dtype=torch.float32, device="cuda"))
        uo.append(torch.full_like(ui[-1], float("nan")))
        vo.append(torch.full_like(vi[-1], float("nan")))
    return ctxs, ui, vi, uo, vo, host


def _run(batch, uo, vo):
    import torch
    for t in uo + vo:
        t.fill_(float("nan"))
    batch.launch()
    torch.cuda.synchronize()
    return [(u.double().cpu().numpy(), v.double().cpu().numpy()) for u, v in zip(uo, vo)]


def _check_oracle(cases, host, res):
    for k, w in enumerate(cases):
        u, v = host[k]
        ug, vg = res[k]
        for s in range(w.n_slices):
            ur, vr = P.oracle_slice(w, u[s], v[s])
            e, l2 = P.slice_errors(w, ug[s], vg[s], ur, vr)
            assert e <= P.TOL_ENERGY_F32 and l2 <= P.TOL_ENERGY_F32, (w.name, s, e, l2)


def test_queue_kernel_matches_oracle_and_launch_chains(lib):
    from paper_1905_00473_gb300 import binding
    # every width class; level splits 8+8+5, 8+5, 8+2, 8+5+4 (a lone final
    # level) and 5+4; several slices and strips per counter; ragged units
    # (3 of 4 groups at n = 256, 2 + 1 of 2 at n = 512)
    cases = [W.custom_case(2, 256, 3, 20, "f32", "inclusion", seed=1),
             W.custom_case(2, 512, 3, 12, "f32", "smooth", seed=2),
             W.custom_case(2, 1024, 1, 9, "f32", "smooth", seed=3),
             W.custom_case(2, 2048, 2, 16, "f32", "smooth", seed=4),
             W.custom_case(2, 2048, 1, 8, "f32", "inclusion", seed=5)]
    ctxs, ui, vi, uo, vo, host = _bind(cases)
    batch = binding.Batch(ctxs, ui, vi, uo, vo, autotune=False)
    assert batch.set_mode(1) == 1
    assert all(batch.info(i)[:2] == (8, 4) for i in range(len(cases)))
    for rep in range(2):
        res_q = _run(batch, uo, vo)
        for ctx in ctxs:
            binding.pr_check(ctx)
        _check_oracle(cases, host, res_q)
    assert batch.set_mode(0) == 0
    res_c = _run(batch, uo, vo)
    for k, w in enumerate(cases):
        for s in range(w.n_slices):
            e, l2 = P.slice_errors(w, res_q[k][0][s], res_q[k][1][s], res_c[k][0][s], res_c[k][1][s])
            assert e <= 1e-6 and l2 <= 1e-6, (w.name, s, e, l2)


def test_queue_refuses_instances_it_does_not_take(lib):
    from paper_1905_00473_gb300 import binding
    cases = [W.custom_case(2, 256, 2, 12, "f32", "smooth", seed=6),
             W.custom_case(2, 96, 2, 10, "f32", "smooth", seed=7)]
    ctxs, ui, vi, uo, vo, host = _bind(cases)
    batch = binding.Batch(ctxs, ui, vi, uo, vo, autotune=False)
    with pytest.raises(binding.PrError) as ei:
        batch.set_mode(1)
    assert ei.value.status == 1
    _check_oracle(cases, host, _run(batch, uo, vo))   # the chains still run


def test_timed_choice_keeps_a_valid_graph(lib):
    from paper_1905_00473_gb300 import binding
    cases = [W.custom_case(2, 512, 4, 16, "f32", "smooth", seed=8),
             W.custom_case(2, 256, 8, 24, "f32", "inclusion", seed=9)]
    ctxs, ui, vi, uo, vo, host = _bind(cases)
    batch = binding.Batch(ctxs, ui, vi, uo, vo, autotune=True)
    assert batch.set_mode(-1) in (0, 1)
    _check_oracle(cases, host, _run(batch, uo, vo))


def test_queue_time_out_is_reported_on_every_instance(lib):
    from paper_1905_00473_gb300 import binding
    cases = [W.custom_case(2, 256, 2, 16, "f32", "smooth", seed=11),
             W.custom_case(2, 512, 1, 9, "f32", "smooth", seed=12)]
    ctxs, ui, vi, uo, vo, host = _bind(cases)
    batch = binding.Batch(ctxs, ui, vi, uo, vo, autotune=False)
    binding.pr_debug_stall_waits(ctxs[0], True)
    assert batch.set_mode(1) == 1                     # tables carry the stall hook
    t0 = time.time()
    _run(batch, uo, vo)
    for ctx in ctxs:
        with pytest.raises(binding.PrError) as ei:
            binding.pr_check(ctx)
        assert ei.value.status == 4
    assert time.time() - t0 < 30
    for ctx in ctxs:
        binding.pr_check(ctx)                         # flags cleared
    binding.pr_debug_stall_waits(ctxs[0], False)
    assert batch.set_mode(1) == 1                     # tables rebuilt without it
    res = _run(batch, uo, vo)
    for ctx in ctxs:
        binding.pr_check(ctx)
    _check_oracle(cases, host, res)
