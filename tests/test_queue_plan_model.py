"""The batch work-queue plan (csrc/queue_plan.h), run through the host harness:
the level split of every sweep, the coverage of the work items, and that the
queue order lets any number of claiming CTAs finish (no item waits for an
item behind it), simulated with the kernel's counter semantics: an item of
pass k of a slice starts once the slice's counter holds k * strips."""
import collections

import numpy as np
import pytest

from paper_1905_00473_gb300 import workloads as W
from tests import _shipped


def _passes_of(passes, inst):
    return [p for p in passes if p[0] == inst]


def test_level_split_covers_every_level_in_fused_passes():
    ms = list(range(8, 140)) + [255, 256, 257, 383, 384, 385, 2047, 2048]
    ndep, passes, _, _ = _shipped.queue_plan([(256, 1, m) for m in ms])
    assert ndep == len(ms)
    for i, m in enumerate(ms):
        ps = _passes_of(passes, i)
        g = 0
        for j, (_, k, _, g0, levels, _) in enumerate(ps):
            assert k == j and g0 == g and 2 <= levels <= 8, (m, ps)
            g += levels
        assert g == m + 1
        assert all(p[4] == 8 for p in ps[:-2])
        if (m + 1) % 8 == 1:
            assert [p[4] for p in ps[-2:]] == [5, 4]


def test_classes_and_strips_cover_the_rows():
    ndep, passes, _, _ = _shipped.queue_plan([(256, 2, 9), (512, 2, 9), (1024, 2, 9), (2048, 2, 9)])
    assert ndep == 8
    cls = {p[0]: (p[2], p[5]) for p in passes}
    assert cls == {0: (0, 1), 1: (1, 1), 2: (2, 1), 3: (3, 3)}
    # 2048-point rows: three strips of 4 x 192 columns, 8 of halo each side
    fin = 4 * 192 - 2 * 8
    assert 3 * fin >= 2048 > 2 * fin


def test_refuses_unsupported_instances():
    assert _shipped.queue_plan([(96, 2, 20)])[0] == -1
    assert _shipped.queue_plan([(256, 2, 7)])[0] == -1


def _check_queue(instances, workers, seed):
    ndep, passes, items, units = _shipped.queue_plan(instances)
    assert ndep == sum(s for _, s, _ in instances)
    # units: consecutive items of one pass, as many as the class runs side by
    # side (four at n = 256, two at 512, one at 1024 and 2048)
    groups = {0: 4, 1: 2, 2: 1, 3: 1}
    assert units[0][0] == 0 and sum(c for _, c in units) == len(items)
    for (a, ca), (b, _) in zip(units, units[1:] + [(len(items), 0)]):
        assert a + ca == b and 1 <= ca <= groups[passes[items[a][0]][2]]
        assert len({items[j][0] for j in range(a, a + ca)}) == 1
    # coverage: every (pass, slice, strip) exactly once, counters per slice
    seen = collections.Counter((it[0], it[1]) for it in items)
    want = {(j, v) for j, p in enumerate(passes) for v in range(instances[p[0]][1] * p[5])}
    assert set(seen) == want and all(c == 1 for c in seen.values())
    base = np.cumsum([0] + [s for _, s, _ in instances])
    for pj, v, dep, need in items:
        inst, k, _, _, _, strips = passes[pj]
        assert dep == base[inst] + v // strips and need == k * strips
    # topological: an item's need is met by items queued before it
    before = collections.Counter()
    for pj, v, dep, need in items:
        assert before[dep] >= need
        before[dep] += 1
    # claims of whole units in queue order by `workers` CTAs with random
    # durations: a unit starts once every item's counter is met (the CTA's
    # leader waits for each), and every claimed unit eventually starts, so
    # the queue drains
    rng = np.random.default_rng(seed)
    cnt = collections.Counter()
    nxt = 0
    running = []           # (finish time, deps) of started units
    waiting = []           # [(dep, need)] of claimed units not yet startable
    t = 0.0
    free = workers
    while nxt < len(units) or running or waiting:
        while free > 0 and nxt < len(units):
            a, ca = units[nxt]
            nxt += 1
            free -= 1
            waiting.append([(items[j][2], items[j][3]) for j in range(a, a + ca)])
        ready = [w for w in waiting if all(cnt[d] >= nd for d, nd in w)]
        waiting = [w for w in waiting if not all(cnt[d] >= nd for d, nd in w)]
        for w in ready:
            running.append((t + rng.uniform(0.5, 2.0), [d for d, _ in w]))
        assert running, "every claimed unit waits for an item behind it"
        running.sort(key=lambda r: r[0])
        t, deps = running.pop(0)
        for d in deps:
            cnt[d] += 1
        free += 1
    return passes, items


@pytest.mark.parametrize("workers", [1, 3, 152])
def test_queue_drains_for_any_number_of_ctas(workers):
    inst = [(2048, 2, 17), (256, 4, 40), (1024, 1, 9), (512, 3, 23), (2048, 1, 64)]
    _check_queue(inst, workers, seed=workers)


def test_full_uneven_workload_queue():
    """The 48 seeded instances of the uneven batch: coverage, order and a
    152-CTA claim simulation; the widest class first, and within a class the
    interleaving by progress (the longest pass chain of the class starts in
    the first hundredth of the class's items and ends in the last)."""
    ws = [W.config4_instance(i) for i in range(48)]
    inst = [(w.n_fine, w.n_slices, w.m_f) for w in ws]
    passes, items = _check_queue(inst, 152, seed=48)
    cls = [passes[it[0]][2] for it in items]
    assert cls == sorted(cls, reverse=True)
    for c in set(cls):
        span = [q for q, k in enumerate(cls) if k == c]
        members = {passes[it[0]][0] for it in items[span[0]:span[-1] + 1]}
        longest = max(members, key=lambda i: len(_passes_of(passes, i)))
        pos = [q for q in span if passes[items[q][0]][0] == longest]
        a, b = span[0], span[-1] + 1
        assert pos[0] - a < (b - a) // 100 + 1 and pos[-1] - a >= (b - a) * 99 // 100, (c, pos[0], pos[-1], a, b)
