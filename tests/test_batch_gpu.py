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


@pytest.mark.parametrize("mode", [0, 1], ids=["chains", "queue"])
def test_full_uneven_batch_48_instances(lib, mode):
    """The uneven-batch workload at full size, in the launch configurations
    the bench times: all 48 seeded instances (256^2..2048^2, 16..128 slices)
    in one captured graph, as autotuned per-instance launch chains (mode 0)
    or as the one work-queue kernel (mode 1), slice states built like the
    bench's (the instance's Gaussian u0 rolled by a seeded shift per slice,
    u_t = 0).  The oracle cannot sweep every instance in seconds, so every
    instance is checked on a sampled slice by the exactly conserved modified
    energy of the scheme, and the smallest instance's first slice against
    the FP64 oracle."""
    import gc
    import math

    import torch
    from paper_1905_00473_gb300 import binding
    gc.collect()                  # the other mode's contexts and arrays
    torch.cuda.empty_cache()
    ws = [W.config4_instance(i) for i in range(48)]
    need = sum(w.n_fine ** 2 * w.n_slices for w in ws) * 4 * (4 + 4 + 1)
    free, _ = torch.cuda.mem_get_info()
    assert need < 0.8 * free, f"the full batch needs {need / 2**30:.0f} GiB"
    ctxs, ui, vi, uo, vo, shifts = [], [], [], [], [], []
    for w in ws:
        c = torch.tensor(w.c, dtype=torch.float32, device="cuda")
        ctxs.append(binding.pr_create(2, w.n_fine, w.ratio, c, w.dt_f, w.dt_c, w.n_slices, w.t_final))
        sh = np.random.default_rng(w.seed).integers(0, w.n_fine, size=(w.n_slices, 2))
        shifts.append(sh)
        base = torch.tensor(w.u0, dtype=torch.float32, device="cuda")
        u = torch.stack([torch.roll(base, (int(a), int(b)), (0, 1)) for a, b in sh]).contiguous()
        ui.append(u)
        vi.append(torch.zeros_like(u))
        uo.append(torch.full_like(u, float("nan")))
        vo.append(torch.full_like(u, float("nan")))
    batch = binding.Batch(ctxs, ui, vi, uo, vo, autotune=(mode == 0))
    assert batch.set_mode(mode) == mode
    batch.launch()
    torch.cuda.synchronize()
    for ctx in ctxs:
        binding.pr_check(ctx)
    rng = np.random.default_rng(48)
    for k, w in enumerate(ws):
        u0 = w.u0.astype(np.float64)
        for s in rng.choice(w.n_slices, size=1):
            a, b = (int(x) for x in shifts[k][s])
            u_in = np.roll(u0, (a, b), (0, 1))
            h0 = P.modified_energy(u_in, np.zeros_like(u_in), w.c, w.dt_f, w.dx_f)
            ug = uo[k][s].double().cpu().numpy()
            vg = vo[k][s].double().cpu().numpy()
            h1 = P.modified_energy(ug, vg, w.c, w.dt_f, w.dx_f)
            assert math.isfinite(h1) and abs(h1 - h0) <= 2e-5 * abs(h0), (w.name, s, h0, h1)
    k = min(range(48), key=lambda i: ws[i].point_steps_per_sweep())
    w = ws[k]
    a, b = (int(x) for x in shifts[k][0])
    u_in = np.roll(w.u0.astype(np.float64), (a, b), (0, 1))
    ur, vr = P.oracle_slice(w, u_in, np.zeros_like(u_in))
    e, l2 = P.slice_errors(w, uo[k][0].double().cpu().numpy(), vo[k][0].double().cpu().numpy(), ur, vr)
    assert e <= P.TOL_ENERGY_F32 and l2 <= P.TOL_ENERGY_F32, (w.name, e, l2)
