// Host-side harness for the CPU tests: evaluates functions of the shipped
// kernel headers on the host, so that the model tests check the code the
// kernels compile, not a restatement of it.
//   (no argument)  balanced_row: reads "rows_total n K b G" lines on stdin,
//                  prints the row.
//   plan           the batch work-queue plan (queue_plan.h): reads
//                  "n slices m" lines (one instance each) on stdin, prints
//                  "P inst k cls g0 levels strips" per pass, then
//                  "I pass vslice dep need" per item in queue order, then
//                  "U first count" per unit (what one CTA claims).
#include <cstdio>
#include <cstring>

#include "queue_plan.h"
#include "tb_common.cuh"

int main(int argc, char** argv) {
    if (argc > 1 && std::strcmp(argv[1], "plan") == 0) {
        std::vector<qplan::Inst> inst;
        long long n;
        int slices, m;
        while (std::scanf("%lld %d %d", &n, &slices, &m) == 3) inst.push_back({n, slices, m});
        std::vector<qplan::Pass> passes;
        std::vector<qplan::Item> items;
        std::vector<qplan::Unit> units;
        const int ndep = qplan::build(inst, &passes, &items, &units);
        std::printf("D %d\n", ndep);
        for (const auto& p : passes)
            std::printf("P %d %d %d %d %d %d\n", p.inst, p.k, p.cls, p.g0, p.levels, p.strips);
        for (const auto& it : items) std::printf("I %d %d %d %u\n", it.pass, it.vslice, it.dep, it.need);
        for (const auto& u : units) std::printf("U %d %d\n", u.first, u.count);
        return 0;
    }
    long long rows, b, G;
    int n, K;
    while (std::scanf("%lld %d %d %lld %lld", &rows, &n, &K, &b, &G) == 5)
        std::printf("%lld\n", (long long)tb::balanced_row(rows, n, K, b, G));
    return 0;
}
