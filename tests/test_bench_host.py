"""Host-side logic of bench.py (no GPU): workload selection, the kernel-source
hash that decides whether the committed ncu traffic figure still applies, and
the lookup of that figure."""
import json
import os

import pytest

import bench


def test_workload_selection():
    w3 = bench.workload_for("3")
    assert (w3.n_fine, w3.n_slices, w3.m_f) == (1024, 64, 384)
    w2 = bench.workload_for("2", slices=4)
    assert (w2.n_fine, w2.n_slices, w2.m_f) == (512, 4, 192)   # fewer slices, same step
    wi = bench.workload_for("4:3", slices=8)
    assert (wi.n_fine, wi.n_slices) == (2048, 8)
    assert wi.m_f == bench.workload_for("4:3").m_f
    w5 = bench.workload_for("5")
    assert (w5.dim, w5.n_fine, w5.n_slices) == (3, 256, 32)
    for bad in ("1", "4:x", "7"):
        with pytest.raises((SystemExit, ValueError)):
            bench.workload_for(bad)


def test_pass_counts():
    # 385 levels at depth 8: the lone last level joins the 48th pass where
    # the fused kernel takes 9 levels, else it is a 49th
    assert bench.hbm_passes(384, 8) == 48
    assert bench.hbm_passes(384, 8, merge_last=False) == 49
    assert bench.hbm_passes(383, 8) == 48 and bench.hbm_passes(64, 4) == 17 and bench.hbm_passes(7, 1) == 8
    # the work-queue kernel's plan (queue_plan.h, through the host harness)
    # has as many passes as the unmerged count
    from tests import _shipped
    ms = [8, 9, 15, 16, 17, 255, 256, 512, 2036]
    _, passes, _, _ = _shipped.queue_plan([(256, 1, m) for m in ms])
    for i, m in enumerate(ms):
        assert sum(1 for p in passes if p[0] == i) == bench.hbm_passes(m, 8, merge_last=False), m


def test_kernel_hash_ignores_comments_but_not_code():
    src = {rel: open(os.path.join(bench.ROOT, rel)).read() for rel in bench.KERNEL_SOURCES}
    base = bench.kernel_source_hash(lambda rel: src[rel])
    assert base == bench.kernel_source_hash()
    first = bench.KERNEL_SOURCES[0]
    commented = dict(src)
    commented[first] = "// a comment\n/* a block\n comment */\n" + src[first].replace("\n", "  \n", 3)
    assert bench.kernel_source_hash(lambda rel: commented[rel]) == base
    edited = dict(src)
    edited[first] = src[first] + "\nstatic int an_edit = 1;\n"
    assert bench.kernel_source_hash(lambda rel: edited[rel]) != base


def test_traffic_figure_only_for_the_profiled_source(monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "fine_tb2d_traffic.json")) as f:
        d = json.load(f)
    key, val = next(iter(d["per_launch_bytes"].items()))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda read=None: d["source_hash"])
    assert bench.ncu_traffic(key) == val
    assert bench.ncu_traffic("no-such-workload") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda read=None: "0" * 16)
    assert bench.ncu_traffic(key) is None
