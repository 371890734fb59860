"""Model check of the fused kernels' work split, on the CPU.

The persistent grid cuts the N*n rows of a sweep into one contiguous range
per CTA (or per cluster).  A range is processed slice by slice; each segment
costs its rows plus K = L + B pipeline steps of halo and drain.  With
phi(r) = r + K * (slice boundaries below r), CTA b starts where phi crosses
b * phi_total / G (inside a boundary's jump, on the boundary itself).

The cuts come from the shipped tb::balanced_row (tb_common.cuh), compiled
into a host harness; a plain restatement of the formula cross-checks it.
The tests check the properties for the launch shapes the kernels use: the
ranges tile the rows exactly, in order, and no CTA's cost exceeds the even
share by more than one segment's overhead (K + 1).
"""
import random

from tests._shipped import balanced_rows


def balanced_row_restated(rows_total, n, K, b, G):
    slices = rows_total // n
    phi = (rows_total + (slices - 1) * K) * b // G
    j = phi // (n + K)
    r = min(phi - j * K, (j + 1) * n)
    return min(r, rows_total)


def all_cuts(cases):
    """cases: list of (rows_total, n, K, G) -> list of cut lists (G + 1 each),
    from the shipped function."""
    queries = [(rows, n, K, b, G) for rows, n, K, G in cases for b in range(G + 1)]
    vals = balanced_rows(queries)
    out, i = [], 0
    for rows, n, K, G in cases:
        out.append(vals[i:i + G + 1])
        i += G + 1
    return out


def range_costs(cuts, n, K):
    costs = []
    for lo, hi in zip(cuts, cuts[1:]):
        segments, r = 0, lo
        while r < hi:
            r = min(hi, (r // n + 1) * n)
            segments += 1
        costs.append(hi - lo + K * segments)
    return costs


def _random_cases(seed, Ks, Gs, count=2000):
    rng = random.Random(seed)
    cases = []
    for _ in range(count):
        n = rng.choice([128, 256, 512, 1024, 2048])
        N = rng.randint(1, 400)
        cases.append((N * n, n, rng.choice(Ks), rng.choice(Gs)))
    return cases


def test_shipped_function_matches_the_formula():
    cases = _random_cases(6, [2, 8, 16, 18], [1, 2, 76, 152, 304], count=300)
    for (rows, n, K, G), cuts in zip(cases, all_cuts(cases)):
        assert cuts == [balanced_row_restated(rows, n, K, b, G) for b in range(G + 1)]


def test_ranges_tile_the_rows_in_order():
    cases = _random_cases(7, [2, 8, 16, 18], [1, 2, 76, 152, 304])
    for (rows, n, K, G), cuts in zip(cases, all_cuts(cases)):
        assert cuts[0] == 0 and cuts[-1] == rows
        assert all(a <= b for a, b in zip(cuts, cuts[1:]))


def test_costs_are_balanced():
    cases = _random_cases(8, [8, 16, 18], [76, 152, 304])
    for (rows, n, K, G), cuts in zip(cases, all_cuts(cases)):
        costs = range_costs(cuts, n, K)
        N = rows // n
        share = (rows + (N - 1) * K) / G
        assert max(costs) <= share + K + 1, (n, N, K, G, max(costs), share)


def test_bench_workload_split():
    """1024^2 x 64 slices over 152 CTAs at depth 8 (K = 16): ~431 rows and
    1-2 segments per CTA, every CTA within one segment's overhead."""
    costs = range_costs(all_cuts([(64 * 1024, 1024, 16, 152)])[0], 1024, 16)
    share = (64 * 1024 + 63 * 16) / 152
    assert max(costs) - min(costs) <= 17
    assert abs(sum(costs) / 152 - share) < 17
