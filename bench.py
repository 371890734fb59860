#!/usr/bin/env python
"""Benchmark of the hot path: F over all N slices of one parareal iteration.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config 3]

One step = one pr_fine_all_slices call on the whole batch of slices of the
chosen synthetic workload (default: the 2D discontinuous-inclusion problem,
1024^2 fine grid, 64 slices, m_F = 384 fine steps per slice).  The metric is
fine grid-point updates per second, slices * m_F * n^2 / time, whole job.
Inputs are resident in HBM and larger than L2 (0.54 GB per rank), so no L2
flush is needed between steps.

Besides `value` the JSON line carries
  * roofline  -- the fused pass kernel's algorithmic bytes (20 B per point
                 per pass: read u, u_t, kappa, write u, u_t in FP32) over its
                 mean launch time, timed with CUDA events on its stream,
                 against the measured HBM copy bandwidth;
  * e2e       -- the same metric through the C ABI with the slices coming from
                 pinned host memory and going back to it every step;
  * cpu_baseline -- the FP64 oracle on a bounded sample of the same workload
                 on the host cores (parallel over slices, like the paper's
                 parFor);
  * clocks    -- nvidia-smi samples taken during the timed region.
With --impl reference the oracle itself is the timed arm (bounded sample per
step).  Multi-GPU (torchrun): every rank propagates its own copy of the
workload (slices are independent units; weak scaling, no collective on the
data path); time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1905_00473_gb300 import sharding  # noqa: E402
from paper_1905_00473_gb300 import workloads as W  # noqa: E402

ALGO_BYTES_PER_POINT_PASS = 20  # read u, u_t, kappa + write u, u_t (FP32)
FALLBACK_HBM_GBS = 6800.0


def hbm_passes(m_f: int, depth: int, merge_last: bool = True) -> int:
    """HBM passes of one sweep of m_f steps (m_f + 1 kick levels) at `depth`
    levels per pass.  At depth 8 a lone final level joins the last pass where
    the fused kernel takes 9 levels (merge_last: whole rows of n <= 1024 at
    four columns per thread); elsewhere it is a pass of its own, and the
    work-queue batch kernel splits the last 9 levels as 5 + 4."""
    levels = m_f + 1
    passes = -(-levels // depth)
    if merge_last and depth == 8 and passes >= 2 and levels % depth == 1:
        passes -= 1
    return passes


# ---------------------------------------------------------------- CPU oracle
def _oracle_task(args):
    u, v, c, dt, steps, dx = args
    from oracle import fine
    t0 = time.perf_counter()
    fine.velocity_verlet(u, v, c, dt, steps, dx)
    return time.perf_counter() - t0


def _warm(_):
    import oracle.fine  # noqa: F401
    return 0


class OracleSampler:
    """The FP64 oracle on `procs` host processes, one slice per process."""

    def __init__(self, w: W.Workload, procs: int, steps: int):
        self.w, self.procs, self.steps = w, procs, steps
        u, v = W.slice_states(w, n_slices=procs, seed=11)
        self.tasks = [(u[i], v[i], w.c, w.dt_f, steps, w.dx_f) for i in range(procs)]
        self.pool = mp.get_context("spawn").Pool(procs)
        self.pool.map(_warm, range(procs))

    def run(self) -> tuple[float, float]:
        """(point-updates, wall seconds) of one sample."""
        t0 = time.perf_counter()
        self.pool.map(_oracle_task, self.tasks, chunksize=1)
        wall = time.perf_counter() - t0
        return self.procs * self.steps * self.w.points, wall

    def run_single(self) -> float:
        """Point-updates/s of one slice on one process (one host core)."""
        t = self.pool.map(_oracle_task, self.tasks[:1], chunksize=1)[0]
        return self.steps * self.w.points / t

    def baseline(self) -> dict:
        """The cpu_baseline object: all host cores, plus the one-core figure."""
        p, t = self.run()
        return {"value": p / t, "unit": "point-updates/s", "cores": self.procs,
                "host_cores": os.cpu_count(), "kind": "oracle", "sample": self.describe(),
                "single_core_value": self.run_single()}

    def close(self):
        self.pool.close()
        self.pool.join()

    def describe(self) -> str:
        return (f"{self.procs} slices x {self.steps} of {self.w.m_f} fine steps of "
                f"{self.w.name}, one slice per process")


def oracle_steps(w: W.Workload) -> int:
    """Fine steps per sampled slice: about 10 s of numpy work per process
    (64 steps of a 1024^2 slice, 8 of a 256^3 slice), at most m_F."""
    return max(4, min(w.m_f, 64, int(1.5e8 // w.points)))


def oracle_procs() -> int:
    """Every host core, one oracle process each."""
    return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows: list[list[str]] = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        for r in self.rows:
            if len(r) < 8:
                continue
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, r[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- helpers
def measured_peak() -> tuple[float, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


KERNEL_SOURCES = ("paper_1905_00473_gb300/csrc/tb2d_kernels.cuh", "paper_1905_00473_gb300/csrc/tb2d_sweep.cuh",
                  "paper_1905_00473_gb300/csrc/tb_common.cuh", "paper_1905_00473_gb300/csrc/pr_internal.cuh")


def code_only(text: str) -> str:
    """C/C++ source without comments and with whitespace collapsed, so that an
    edit of comments alone keeps the hash of the code."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_source_hash(read=None) -> str:
    """Hash of the fused kernel's code (comments excluded); `read(rel)` returns
    a file's text (default: the working tree)."""
    if read is None:
        read = lambda rel: open(os.path.join(ROOT, rel)).read()  # noqa: E731
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        h.update(code_only(read(rel)).encode())
    return h.hexdigest()[:16]


def ncu_traffic(workload_key: str, kernel: str = "fine_tb2d_kernel"):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "fine_tb2d_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    if d.get("source_hash") != kernel_source_hash():
        return None
    if not str(d.get("kernel", "fine_tb2d_kernel")).startswith(kernel):
        return None
    return d.get("per_launch_bytes", {}).get(workload_key)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_for(cfg: str, slices: int = 0) -> W.Workload:
    """The configuration's workload; slices > 0 keeps the grid, medium and
    time step but propagates only that many slices (small profiling runs)."""
    if cfg.startswith("4:"):   # one instance of the uneven batch, alone
        w = W.config4_instance(int(cfg[2:]))
    elif cfg in ("2", "3", "5"):
        w = W.CONFIGS[cfg]()
    else:
        raise SystemExit("--config must be 2, 3, 5 or 4:<instance> for a sweep, 4 for the batch, snapshot or "
                         "parareal")
    if slices and slices != w.n_slices:
        m_f = w.m_f
        w.t_final = w.t_final * slices / w.n_slices
        w.n_slices = slices
        w.m_f_fixed = m_f
        w.name = f"{w.name}[{slices} slices]"
    return w


def workload_desc(w: W.Workload) -> dict:
    return {"workload": w.name, "dim": w.dim, "n_fine": w.n_fine, "slices": w.n_slices,
            "m_f": w.m_f, "point_updates_per_step": w.point_steps_per_sweep(),
            "inputs": "seeded Gaussian-pulse slice states, c field of the configuration"}


# ---------------------------------------------------------------- end to end
E2E_BUFFERS = 3


def e2e_pipelined(binding, ctx, u_pin, v_pin, u_in, v_in, u_out, v_out, steps, barrier, warmup=3):
    """Time `steps` batches through the C ABI, each copied in from pinned host
    memory, propagated, and copied back to pinned host memory.

    Three device buffer sets rotate between batches: while batch k is
    propagated on the compute stream, later batches are copied in on a
    host-to-device stream and earlier ones copied out on a device-to-host
    stream (separate copy engines).  Events order each buffer's reuse.  Every
    batch still moves its full inputs in and results out inside the timed
    region; only their overlap with the propagation differs from a
    single-stream loop.  The third set lets one host copy that stalls (the
    host link is shared with other work on the node; stalls of ~20 ms were
    seen) finish during the next propagation instead of holding it up.
    `warmup` untimed batches first run the same pipeline over every buffer
    (the first transfers into freshly allocated buffers pay one-time costs).
    Returns (ms, mode).
    """
    import torch
    nb = E2E_BUFFERS
    comp = torch.cuda.current_stream()
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()
    bufs = [(u_in, v_in, u_out, v_out)] + [
        (torch.empty_like(u_in), torch.empty_like(v_in), torch.empty_like(u_out), torch.empty_like(v_out))
        for _ in range(nb - 1)]
    backs = [(torch.empty_like(u_pin).pin_memory(), torch.empty_like(v_pin).pin_memory()) for _ in range(nb)]
    ev = lambda: torch.cuda.Event()  # noqa: E731
    loaded = [ev() for _ in range(nb)]      # inputs of buffer b copied in
    computed = [ev() for _ in range(nb)]    # buffer b propagated (its inputs free, outputs ready)
    drained = [ev() for _ in range(nb)]     # outputs of buffer b copied out
    def batches(count):
        for k in range(count):
            b = k % nb
            ui, vi, uo, vo = bufs[b]
            with torch.cuda.stream(h2d):
                h2d.wait_event(computed[b])
                ui.copy_(u_pin, non_blocking=True)
                vi.copy_(v_pin, non_blocking=True)
                loaded[b].record(h2d)
            comp.wait_event(loaded[b])
            comp.wait_event(drained[b])
            binding.pr_fine_all_slices(ctx, ui, vi, uo, vo, stream=comp)
            computed[b].record(comp)
            with torch.cuda.stream(d2h):
                d2h.wait_event(computed[b])
                backs[b][0].copy_(uo, non_blocking=True)
                backs[b][1].copy_(vo, non_blocking=True)
                drained[b].record(d2h)
        comp.wait_stream(h2d)
        comp.wait_stream(d2h)

    for b in range(nb):        # every event starts recorded, so the first waits pass
        computed[b].record(comp)
        drained[b].record(comp)
    batches(max(nb, warmup))
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(comp)
    h2d.wait_event(e0)
    d2h.wait_event(e0)
    batches(steps)
    e1.record(comp)
    barrier()
    return e0.elapsed_time(e1), (f"{nb} buffer sets: H2D of later batches and D2H of earlier ones "
                                 "on their own streams overlap the propagation of batch k")


# ---------------------------------------------------------------- parareal vs serial fine
def parareal_time_to_tol(dev, tol_err: float = 1e-4, k_max: int = 32, svd_tol: float = 1e-5) -> dict:
    """Wall time of Alg. 3 (Procrustes corrector, pr_iterate) to a relative
    energy-norm error <= tol_err at T against the serial fine solution, and
    the serial fine solve itself (the same fine kernels, one slice after the
    other), both on this GPU, for the smooth 2D workload (512^2, 32 slices)."""
    import torch
    from paper_1905_00473_gb300 import binding
    w = W.config2()
    c = torch.tensor(w.c, dtype=torch.float32, device=dev)
    u0 = torch.tensor(w.u0, dtype=torch.float32, device=dev)
    p0 = torch.zeros_like(u0)
    ctx1 = binding.pr_create(2, w.n_fine, w.ratio, c, w.dt_f, w.dt_c, 1, w.dt_com)
    ctx = binding.pr_create(2, w.n_fine, w.ratio, c, w.dt_f, w.dt_c, w.n_slices, w.t_final,
                            tol=svd_tol)
    N = w.n_slices
    ref = torch.zeros((N + 1,) + w.shape, dtype=torch.float32, device=dev)
    refv = torch.zeros_like(ref)

    def serial():
        ref[0].copy_(u0)
        refv[0].copy_(p0)
        for n in range(N):
            binding.pr_fine_all_slices(ctx1, ref[n], refv[n], ref[n + 1], refv[n + 1])

    serial()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    serial()
    e1.record()
    torch.cuda.synchronize()
    t_serial = e0.elapsed_time(e1)
    e_ref = binding.pr_energy(ctx1, ref[N].contiguous(), refv[N].contiguous())[0]
    us = torch.zeros_like(ref)
    vs = torch.zeros_like(ref)
    # warm-up: library initialisation (cuFFT plans, cuBLAS/cuSOLVER handles and
    # the solvers' first calls at every size the run reaches)
    binding.pr_iterate(ctx, u0, p0, k_max, binding.PR_CORR_PROCRUSTES, us, vs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = binding.pr_iterate(ctx, u0, p0, k_max, binding.PR_CORR_PROCRUSTES, us, vs,
                             ref[N].contiguous(), refv[N].contiguous(), tol_err)
    t_par = 1e3 * (time.perf_counter() - t0)
    phases = binding.pr_iterate_phases(ctx)
    corr = binding.pr_iterate_corrector_phases(ctx)
    reached = out["err"] and out["err"][-1] <= tol_err
    return {"workload": w.name, "corrector": "procrustes", "svd_tol": svd_tol, "tol_err": tol_err,
            "serial_fine_ms": t_serial, "parareal_ms": t_par, "iterations": out["k_done"],
            "reached": bool(reached),
            "speedup_vs_serial_fine": (t_serial / t_par) if reached else None,
            "phases_ms": phases, "corrector_breakdown": corr,
            "err_hist": out["err"], "rank_hist": out["rank"],
            "note": "pr_iterate wall time, host-synchronised, stopping at the first iteration "
                    "within tol_err of the serial fine solution computed by the same fine "
                    "kernels on this GPU; K = N reproduces it exactly (finite termination)"}


# ---------------------------------------------------------------- uneven batch (config 4)
def run_batch(a) -> int:
    """One fine sweep of each of the first --instances instances of the seeded
    uneven workload (2D, 256^2..2048^2, N in {16..128}, smooth c in [1, 2]),
    all in one captured CUDA graph with autotuned block depths; one step = one
    graph launch.  Slice states: the instance's Gaussian u0 rolled by a seeded
    shift per slice, u_t = 0 (cheap to build for the large instances)."""
    import numpy as np
    rank, world, local = dist_env()
    ws = [W.config4_instance(i) for i in range(a.instances)]
    # the oracle pool is spawned before any CUDA call; it samples the
    # smallest instance (its cost per point-update is that of every instance)
    smp = None
    if not a.no_cpu_baseline:
        wsmall = min(ws, key=lambda x: x.points)
        smp = OracleSampler(wsmall, oracle_procs(), oracle_steps(wsmall))
    import torch
    from paper_1905_00473_gb300 import binding
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctxs, ui, vi, uo, vo = [], [], [], [], []
    units = 0
    for w in ws:
        c = torch.tensor(w.c, dtype=torch.float32, device=dev)
        ctxs.append(binding.pr_create(2, w.n_fine, w.ratio, c, w.dt_f, w.dt_c, w.n_slices, w.t_final))
        rng = np.random.default_rng(w.seed)
        base = torch.tensor(w.u0, dtype=torch.float32, device=dev)
        shifts = rng.integers(0, w.n_fine, size=(w.n_slices, 2))
        u = torch.stack([torch.roll(base, (int(a_), int(b_)), (0, 1)) for a_, b_ in shifts]).contiguous()
        ui.append(u)
        vi.append(torch.zeros_like(u))
        uo.append(torch.empty_like(u))
        vo.append(torch.empty_like(u))
        units += w.point_steps_per_sweep()
    t0 = time.perf_counter()
    batch = binding.Batch(ctxs, ui, vi, uo, vo, autotune=True)
    mode = batch.set_mode({"chains": 0, "queue": 1, "auto": -1}[a.batch_mode])
    tune_s = time.perf_counter() - t0
    for _ in range(a.warmup):
        batch.launch()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        batch.launch()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    # roofline of the whole graph: every instance's algorithmic traffic (20 B
    # per point per HBM pass) over the graph's time per step
    depths = [batch.info(i)[0] for i in range(len(ws))]
    cols = [batch.info(i)[1] for i in range(len(ws))]
    if mode == 1:   # the queue kernel: passes of 8 levels (a lone last level splits as 5 + 4)
        passes = [hbm_passes(w.m_f, 8, merge_last=False) for w in ws]
    else:
        passes = [hbm_passes(w.m_f, d, merge_last=(w.n_fine <= 1024 and c in (0, 4)))
                  for w, d, c in zip(ws, depths, cols)]
    step_bytes = sum(ALGO_BYTES_PER_POINT_PASS * w.points * w.n_slices * pz for w, pz in zip(ws, passes))
    peak, peak_src = measured_peak()
    achieved = step_bytes / (ms / a.steps * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": ("batch_queue_kernel (every instance's passes)" if mode == 1 else
                                       "the batch graph (every instance's passes)"), "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_src, "traffic": None,
            "algorithmic_bytes_per_launch": step_bytes, "mean_launch_ms": ms / a.steps}
    cpu = None
    if smp is not None:
        try:
            cpu = smp.baseline()
        finally:
            smp.close()
    line = {"metric": "fine grid-point updates/s", "value": units * a.steps / (ms * 1e-3),
            "unit": "point-updates/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"uneven batch: first {a.instances} seeded instances",
                       "instances": [{"n": w.n_fine, "N": w.n_slices, "m_f": w.m_f,
                                      "depth": batch.info(i)[0], "columns": batch.info(i)[1]}
                                     for i, w in enumerate(ws)],
                       "point_updates_per_step": units, "autotune_s": tune_s,
                       "graph": ("one CUDA graph: one persistent work-queue kernel" if mode == 1 else
                                 "one CUDA graph: per-instance pass launches on 8 streams"),
                       "batch_mode": {0: "chains", 1: "queue"}[mode],
                       "batch_mode_requested": a.batch_mode},
            "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
            # one launch per pass in the chains graph; one in all in the queue graph
            "gpu_launches": a.steps * (1 if mode == 1 else sum(passes))}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- reference arm
def run_reference(a) -> int:
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = workload_for(a.config, a.slices)
    procs = oracle_procs()
    steps_per_sample = oracle_steps(w)
    smp = OracleSampler(w, procs, steps_per_sample)
    try:
        for _ in range(a.warmup):
            smp.run()
        tot_pts, tot_t = 0, 0.0
        for _ in range(a.steps):
            p, t = smp.run()
            tot_pts += p
            tot_t += t
    finally:
        smp.close()
    value = tot_pts / tot_t
    line = {
        "impl": "reference", "metric": "fine grid-point updates/s", "value": value,
        "unit": "point-updates/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * tot_t / a.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_desc(w), parallelism="host processes over slices"),
        "cpu_baseline": {"value": value, "unit": "point-updates/s", "cores": procs,
                         "host_cores": os.cpu_count(), "kind": "oracle",
                         "sample": smp.describe() + " per step"},
        "e2e": {"value": value, "unit": "point-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- our arm
def run_ours(a) -> int:
    rank, world, local = dist_env()
    w = workload_for(a.config, a.slices)
    # the oracle pool is spawned before any CUDA call
    smp = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        smp = OracleSampler(w, oracle_procs(), oracle_steps(w))

    import torch
    from paper_1905_00473_gb300 import binding
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    u_h, v_h = W.slice_states(w, seed=rank)
    u_pin = torch.from_numpy(u_h.astype("float32")).pin_memory()
    v_pin = torch.from_numpy(v_h.astype("float32")).pin_memory()
    c = torch.tensor(w.c, dtype=torch.float32, device=dev)
    ctx = binding.pr_create(w.dim, w.n_fine, w.ratio, c, w.dt_f, w.dt_c, w.n_slices, w.t_final,
                            block_depth=a.block_depth)
    if a.columns:
        binding.pr_set_fused_columns(ctx, a.columns)
    if a.wide_rows:
        binding.pr_set_wide_rows(ctx, a.wide_rows)
    binding.pr_set_one_launch(ctx, a.one_launch == "on")
    info = binding.pr_info(ctx)
    u_in = u_pin.to(dev)
    v_in = v_pin.to(dev)
    u_out = torch.empty_like(u_in)
    v_out = torch.empty_like(v_in)
    stream = torch.cuda.current_stream()

    for _ in range(a.warmup):
        binding.pr_fine_all_slices(ctx, u_in, v_in, u_out, v_out)
    binding.pr_check(ctx)

    # between timed steps: inputs larger than L2, or an explicit L2 flush
    l2_bytes = torch.cuda.get_device_properties(dev).L2_cache_size
    in_bytes = 2 * u_in.numel() * 4
    flush = a.l2_flush == "on" or (a.l2_flush == "auto" and in_bytes < 2 * l2_bytes)
    flush_buf = torch.empty(max(2 * l2_bytes, 1 << 28) // 4, dtype=torch.float32, device=dev) if flush else None

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    binding.pr_profile(ctx, True)
    if flush:
        evs = []
        for _ in range(a.steps):
            flush_buf.fill_(1.0)
            e_a, e_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e_a.record(stream)
            binding.pr_fine_all_slices(ctx, u_in, v_in, u_out, v_out)
            e_b.record(stream)
            evs.append((e_a, e_b))
        barrier()
        ms = sum(e_a.elapsed_time(e_b) for e_a, e_b in evs)
    else:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(a.steps):
            binding.pr_fine_all_slices(ctx, u_in, v_in, u_out, v_out)
        ev1.record(stream)
        barrier()
        ms = ev0.elapsed_time(ev1)
    binding.pr_profile(ctx, False)
    clk = clocks.stop()
    binding.pr_check(ctx)
    fused_n, fused_ms = binding.pr_profile_read(ctx, 0)
    single_n, single_ms = binding.pr_profile_read(ctx, 1)
    sweep_n, sweep_ms = binding.pr_profile_read(ctx, 2)
    ms = sharding.max_over_ranks(ms, device=dev)
    l2_note = (f"L2 flushed between timed steps ({flush_buf.numel() * 4 >> 20} MiB write), "
               f"steps timed one by one" if flush else
               f"inputs larger than L2 ({in_bytes >> 20} MiB vs {l2_bytes >> 20} MiB), no flush")
    units = w.point_steps_per_sweep()
    value = world * units * a.steps / (ms * 1e-3)

    # end to end through the C ABI: every step's slices come from pinned host
    # memory and its results go back to it
    e2e_steps = max(3, min(a.steps, 20))
    e2e_ms, e2e_mode = e2e_pipelined(binding, ctx, u_pin, v_pin, u_in, v_in, u_out, v_out,
                                     e2e_steps, barrier, warmup=a.warmup)
    e2e_ms = sharding.max_over_ranks(e2e_ms, device=dev)
    e2e_value = world * units * e2e_steps / (e2e_ms * 1e-3)
    io_bytes = 2 * u_pin.numel() * 4

    # roofline of the dominant kernel (fused pass when present)
    peak, peak_src = measured_peak()
    passes = hbm_passes(w.m_f, info["block_depth"])
    if sweep_n > 0:
        # every pass of the sweep in one persistent launch
        kname, launches, kms = "fine_tb2d_sweep_kernel", sweep_n, sweep_ms
        levels_per_launch, passes_per_launch = w.m_f + 1, passes
    elif fused_n > 0:
        kname = "fine_tb3d_kernel" if w.dim == 3 else "fine_tb2d_kernel"
        launches, kms = fused_n, fused_ms
        levels_per_launch, passes_per_launch = info["block_depth"], 1
    else:
        kname, launches, kms = "level_f32 (one level per launch)", single_n, single_ms
        levels_per_launch, passes_per_launch = 1, 1
    per_launch_bytes = ALGO_BYTES_PER_POINT_PASS * w.points * w.n_slices * passes_per_launch
    avg_ms = kms / max(1, launches)
    achieved = per_launch_bytes / (avg_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_source": peak_src,
            "traffic": ncu_traffic(w.name, kname) if (w.dim == 2 and (fused_n > 0 or sweep_n > 0)) else None,
            "algorithmic_bytes_per_launch": per_launch_bytes,
            "levels_per_launch": levels_per_launch, "hbm_passes_per_launch": passes_per_launch,
            "mean_launch_ms": avg_ms,
            "launch_share": kms / ms if ms > 0 else None}

    cpu = None
    if smp is not None:
        try:
            cpu = smp.baseline()
        finally:
            smp.close()

    par = None
    if rank == 0 and not a.no_parareal:
        try:
            par = parareal_time_to_tol(dev)
        except Exception as ex:   # report, do not lose the headline line
            par = {"error": f"{type(ex).__name__}: {ex}"}

    if rank == 0:
        line = {
            "metric": "fine grid-point updates/s", "value": value, "unit": "point-updates/s",
            "n_gpus": world, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": dict(workload_desc(w), l2=l2_note, block_depth=info["block_depth"],
                           columns_per_thread=a.columns or "library default",
                           launches_per_sweep="one" if sweep_n > 0 else "one per pass",
                           parallelism=f"replica per GPU x{world}"),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "point-updates/s", "h2d_bytes_per_step": io_bytes,
                    "d2h_bytes_per_step": io_bytes, "steps": e2e_steps, "warmup": max(E2E_BUFFERS, a.warmup),
                    "mode": e2e_mode},
            "gpu_launches": fused_n + single_n + sweep_n,
            "clocks": clk,
            "parareal": par,
        }
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()
    return 0


# ---------------------------------------------------------------- the parareal line alone
def run_parareal(a) -> int:
    """Alg. 3 with the Procrustes corrector on the 512^2 x 32 workload to a
    1e-4 relative energy-norm error, as in the sweep line's `parareal` object,
    printed on its own (one JSON line; a short command for profiling the
    correction path)."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    r = parareal_time_to_tol(dev)
    out = {"metric": "parareal_time_to_1e-4", "impl": "ours", "unit": "ms", "value": r["parareal_ms"],
           "higher_is_better": False, "data": "synthetic", "config": {"workload": r["workload"]}, "parareal": r}
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------- snapshot products (Alg. 1)
def run_snapshot(a) -> int:
    """The two tall products of UpdateSVD on the tensor cores (split-TF32,
    pr_snapshot_project and pr_snapshot_deflate) at the shape the 512^2
    parareal workload reaches: rows = 3 * 128^2 Lambda features, 1024 stored
    basis columns, 32 new columns.  Both are bound by the HBM read of the
    FP64 basis (402 MB, above L2); one JSON line with the roofline of each."""
    import torch
    from paper_1905_00473_gb300 import binding
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    K, M, N = 3 * 128 * 128, 1024, 32
    g = torch.Generator(device=dev).manual_seed(19050473)
    A = torch.randn((M, K), dtype=torch.float64, device=dev, generator=g)   # the basis: M columns of K rows
    B = torch.randn((N, K), dtype=torch.float64, device=dev, generator=g)
    C = torch.empty((N, M), dtype=torch.float64, device=dev)
    T = torch.randn((N, M), dtype=torch.float64, device=dev, generator=g)
    O = torch.empty((N, K), dtype=torch.float64, device=dev)
    c = torch.ones((64, 64), dtype=torch.float32, device=dev)
    ctx = binding.pr_create(2, 64, 4, c, 0.25 / 64, 1.0 / 64, 2, 8.0 / 64)
    peak, peak_src = measured_peak()
    out = {"metric": "snapshot_products_hbm", "impl": "ours", "unit": "GB/s", "data": "synthetic",
           "config": {"workload": "UpdateSVD products, rows 49152 x basis 1024 x new 32 (FP64 operands)"},
           "steps": a.steps, "warmup": a.warmup}
    calls = {
        "project": (lambda: binding.pr_snapshot_project(ctx, A, B, C), (M * K + N * K) * 8 + M * N * 8),
        # O = F - A T with the same basis A (1024 columns of 49152 rows), F = B
        "deflate": (lambda: binding.pr_snapshot_deflate(ctx, A, T, B, O), (M * K + 2 * N * K) * 8 + M * N * 8),
    }
    for name, (fn, nbytes) in calls.items():
        for _ in range(a.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.steps
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "algorithmic_bytes": nbytes,
                     "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                  "frac": gbs / peak, "peak_source": peak_src},
                     "tflops_split_tf32": 4 * 2 * M * N * K / (ms * 1e-3) / 1e12}
    binding.pr_check(ctx)
    print(json.dumps(out), flush=True)
    return 0


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", default="3",
                    help="2, 3, 5: the sweep workloads; 4: the uneven batch; 4:<i>: instance i of the batch "
                         "alone; snapshot: the tensor-core products of UpdateSVD; parareal: the parareal line")
    ap.add_argument("--block-depth", type=int, default=0, help="0 = library default")
    ap.add_argument("--columns", type=int, default=0, choices=[0, 2, 4],
                    help="fused-kernel columns per thread (0 = library default)")
    ap.add_argument("--slices", type=int, default=0,
                    help="propagate only this many slices (smaller profiling runs; 0 = all)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--instances", type=int, default=48, help="--config 4: instances in the batch (all 48)")
    ap.add_argument("--batch-mode", choices=["chains", "queue", "auto"], default="auto",
                    help="--config 4: per-instance launch chains, the one work-queue kernel, or time both "
                         "and keep the faster (default)")
    ap.add_argument("--no-parareal", action="store_true",
                    help="skip the parareal time-to-1e-4 measurement")
    ap.add_argument("--wide-rows", type=int, default=0, choices=[0, 1, 2],
                    help="2048-point rows at depth 8: 1 cluster rows, 2 x-strips (0 = library default)")
    ap.add_argument("--one-launch", choices=["on", "off"], default="off",
                    help="on: a whole sweep in one persistent launch where supported; off (library default): "
                         "one launch per pass")
    ap.add_argument("--l2-flush", choices=["auto", "on", "off"], default="auto",
                    help="auto: flush L2 between timed steps when the inputs are smaller than 2x L2")
    a = ap.parse_args(argv)
    if a.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if a.impl == "reference":
        return run_reference(a)
    if a.config == "4":
        return run_batch(a)
    if a.config == "snapshot":
        return run_snapshot(a)
    if a.config == "parareal":
        return run_parareal(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
