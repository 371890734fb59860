// Whole-sweep launches for n = 128 and 256 (tb2d_sweep.cuh).
#include "tb2d_sweep.cuh"

pr_status pr_tb2d_sweep_small(pr_ctx* ctx, const pr_sweep& sw, cudaStream_t st) {
    return ctx->n == 128 ? launch_sweep_n<32>(ctx, sw, st) : launch_sweep_n<64>(ctx, sw, st);
}
