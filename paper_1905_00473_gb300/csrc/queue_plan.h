// Host-side plan of the batch work queue (batch_queue.cu): the geometry class
// of each grid width, the level split of a sweep into passes, and the order of
// the work items.  Plain C++ (no CUDA), so the CPU tests run it through the
// host harness.
#pragma once
#include <stdint.h>

#include <algorithm>
#include <utility>
#include <vector>

namespace qplan {

constexpr int kDepth = 8;      // levels of a full queued pass
constexpr int kCols = 4;       // grid columns per thread
constexpr int kThreads = 256;  // threads of a queue CTA

// Width classes: the thread group that holds one item's rows, the x-halo of
// its strips (0: whole periodic rows), and the groups a CTA runs side by side
// (one item each).  n = 2048 runs x-strips of 4 * 192 = 768 columns, 752 of
// them final.
struct Cls {
    int n, nt, xh, groups;
};
constexpr Cls kClasses[4] = {{256, 64, 0, 4}, {512, 128, 0, 2}, {1024, 256, 0, 1}, {2048, 192, 8, 1}};

inline int class_of(int64_t n) {
    for (int c = 0; c < 4; ++c)
        if (kClasses[c].n == n) return c;
    return -1;
}

// x-strips per row (the pass body covers a row with ceil(n / final width))
inline int strips_of(int c) {
    const Cls k = kClasses[c];
    if (k.xh == 0) return 1;
    const int fin = kCols * k.nt - 2 * k.xh;
    return (k.n + fin - 1) / fin;
}

// (first level, levels) of the passes of a sweep of m steps (m + 1 levels):
// passes of kDepth levels; a lone final level makes the last two passes
// 5 + 4 (the fused body takes 2 .. kDepth levels).
inline std::vector<std::pair<int, int>> level_plan(int m) {
    std::vector<std::pair<int, int>> plan;
    const int total = m + 1;
    for (int g = 0; g < total; g += kDepth) plan.push_back({g, std::min(kDepth, total - g)});
    if (plan.size() >= 2 && plan.back().second == 1) {
        const int g = plan[plan.size() - 2].first;
        plan.pop_back();
        plan.back() = {g, 5};
        plan.push_back({g + 5, 4});
    }
    return plan;
}

struct Inst {
    int64_t n;
    int slices, m;
};
struct Pass {
    int inst, k, cls, g0, levels, strips;
    bool first, last;
};
struct Item {
    int pass;        // index into the pass list
    int vslice;      // (slice, strip): rows vslice n .. vslice n + n - 1 of the pass's row space
    int dep;         // completion counter of the item's (instance, slice)
    unsigned need;   // completions of that counter before the item may start
};
// What one CTA claims: items first .. first + count - 1 (one pass), one per
// thread group of the pass's class.
struct Unit {
    int first, count;
};

// Passes of every instance, and the items in queue order: the widest class
// first, and within a class pass k of an instance of P passes at the key
// (k + 1/2) / P (instances interleaved by progress; ties keep instance
// order); then the pass's slices and strips in order, cut into units of the
// class's group count.  Pass k of a slice needs
// k * strips completions of the slice's counter, one per item of each
// earlier pass.  Returns the number of counters, or -1 if an instance has no
// class or fewer than 8 steps.
inline int build(const std::vector<Inst>& inst, std::vector<Pass>* passes, std::vector<Item>* items,
                 std::vector<Unit>* units) {
    passes->clear();
    items->clear();
    units->clear();
    struct Key {
        double key;
        int pass;
    };
    std::vector<Key> order;
    std::vector<int> dep_base;
    int ndep = 0;
    for (int i = 0; i < (int)inst.size(); ++i) {
        const int c = class_of(inst[i].n);
        if (c < 0 || inst[i].m < kDepth || inst[i].slices < 1) return -1;
        const auto plan = level_plan(inst[i].m);
        const int P = (int)plan.size();
        for (int k = 0; k < P; ++k) {
            order.push_back({(3 - c) + (k + 0.5) / P, (int)passes->size()});
            passes->push_back({i, k, c, plan[k].first, plan[k].second, strips_of(c), k == 0, k == P - 1});
            dep_base.push_back(ndep);
        }
        ndep += inst[i].slices;
    }
    std::stable_sort(order.begin(), order.end(), [](const Key& a, const Key& b) { return a.key < b.key; });
    for (const Key& o : order) {
        const Pass& p = (*passes)[o.pass];
        const int first = (int)items->size();
        for (int s = 0; s < inst[p.inst].slices; ++s)
            for (int x = 0; x < p.strips; ++x)
                items->push_back({o.pass, s * p.strips + x, dep_base[o.pass] + s, (unsigned)(p.k * p.strips)});
        const int end = (int)items->size(), g = kClasses[p.cls].groups;
        for (int a = first; a < end; a += g) units->push_back({a, std::min(g, end - a)});
    }
    return ndep;
}

}  // namespace qplan
