// Whole-sweep launches for n = 512 and 1024 (tb2d_sweep.cuh), and the entry
// points of the one-launch sweep.
#include "tb2d_sweep.cuh"

pr_status pr_tb2d_sweep_small(pr_ctx* ctx, const pr_sweep& sw, cudaStream_t st);

// Whether a whole sweep of this context runs as one launch
// (pr_launch_fine_tb2d_sweep): whole rows at depth 8 with four columns per
// thread (n <= 1024), at least two passes.
bool pr_tb2d_sweep_supported(const pr_ctx* ctx, int passes) {
    return ctx->one_launch && passes >= 2 && pr_tb2d_extra_level(ctx);
}

pr_status pr_launch_fine_tb2d_sweep(pr_ctx* ctx, const pr_sweep& sw, cudaStream_t st) {
    if (sw.last_levels < 1 || sw.last_levels > 9) return pr_fail(ctx, PR_EINVAL, "tb2d sweep: bad level count");
    switch (ctx->n) {
        case 128:
        case 256: return pr_tb2d_sweep_small(ctx, sw, st);
        case 512: return launch_sweep_n<128>(ctx, sw, st);
        case 1024: return launch_sweep_n<256>(ctx, sw, st);
        default: return pr_fail(ctx, PR_EINVAL, "tb2d sweep: unsupported grid size");
    }
}
