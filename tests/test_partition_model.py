"""Model check of the fused kernels' work split, on the CPU.

The persistent grid cuts the N*n rows of a sweep into one contiguous range
per CTA (or per cluster).  A range is processed slice by slice; each segment
costs its rows plus K = L + B pipeline steps of halo and drain.  With
phi(r) = r + K * (slice boundaries below r), CTA b starts where phi crosses
b * phi_total / G (inside a boundary's jump, on the boundary itself).  This
restates that formula and checks its properties for the launch shapes the
kernels use: the ranges tile the rows exactly, in order, and no CTA's cost
exceeds the even share by more than one segment's overhead (K + 1).
"""
import random


def balanced_row(rows_total, n, K, b, G):
    slices = rows_total // n
    phi = (rows_total + (slices - 1) * K) * b // G
    j = phi // (n + K)
    r = min(phi - j * K, (j + 1) * n)
    return min(r, rows_total)


def range_costs(rows_total, n, K, G):
    cuts = [balanced_row(rows_total, n, K, b, G) for b in range(G + 1)]
    costs = []
    for b in range(G):
        lo, hi = cuts[b], cuts[b + 1]
        segments, r = 0, lo
        while r < hi:
            r = min(hi, (r // n + 1) * n)
            segments += 1
        costs.append(hi - lo + K * segments)
    return cuts, costs


def test_ranges_tile_the_rows_in_order():
    rng = random.Random(7)
    for _ in range(2000):
        n = rng.choice([128, 256, 512, 1024, 2048])
        N = rng.randint(1, 400)
        K = rng.choice([2, 8, 16, 18])
        G = rng.choice([1, 2, 76, 152, 304])
        cuts, _ = range_costs(N * n, n, K, G)
        assert cuts[0] == 0 and cuts[-1] == N * n
        assert all(a <= b for a, b in zip(cuts, cuts[1:]))


def test_costs_are_balanced():
    rng = random.Random(8)
    for _ in range(2000):
        n = rng.choice([128, 256, 512, 1024, 2048])
        N = rng.randint(1, 400)
        K = rng.choice([8, 16, 18])
        G = rng.choice([76, 152, 304])
        _, costs = range_costs(N * n, n, K, G)
        share = (N * n + (N - 1) * K) / G
        assert max(costs) <= share + K + 1, (n, N, K, G, max(costs), share)


def test_bench_workload_split():
    """1024^2 x 64 slices over 152 CTAs at depth 8 (K = 16): ~431 rows and
    1-2 segments per CTA, every CTA within one segment's overhead."""
    _, costs = range_costs(64 * 1024, 1024, 16, 152)
    share = (64 * 1024 + 63 * 16) / 152
    assert max(costs) - min(costs) <= 17
    assert abs(sum(costs) / 152 - share) < 17
