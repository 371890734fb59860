// Host-side harness for the CPU tests: evaluates functions of the shipped
// kernel headers on the host, so that the model tests check the code the
// kernels compile, not a restatement of it.
//   balanced_row: reads "rows_total n K b G" lines on stdin, prints the row.
#include <cstdio>

#include "tb_common.cuh"

int main() {
    long long rows, b, G;
    int n, K;
    while (std::scanf("%lld %d %d %lld %lld", &rows, &n, &K, &b, &G) == 5)
        std::printf("%lld\n", (long long)tb::balanced_row(rows, n, K, b, G));
    return 0;
}
