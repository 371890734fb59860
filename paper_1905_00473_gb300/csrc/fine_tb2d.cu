// Fused 2D FP32 passes, one launch per pass: dispatch by depth and width.
// Whole-row widths (n = 128 .. 1024) at depth 8 and 9 are instantiated here;
// depth 4 and the 2048-point rows in fine_tb2d_wide.cu.  The kernels
// themselves are in tb2d_kernels.cuh.
#include "tb2d_kernels.cuh"

pr_status pr_tb2d_launch_d4(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st);
pr_status pr_tb2d_launch_2048_d8(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st);

namespace {

pr_status launch_d8(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st) {
    // depth 8 + 1: the sweep's last pass absorbs the final half-kick level
    // (general variant only; the 12-row kappa/D0 ring holds 9 + kPre + 1 rows)
    if (ps.levels == 9) {
        switch (ctx->n) {
            case 128: return launch_cfg<32, 9, 0, false, false>(ctx, ps, st);
            case 256: return launch_cfg<64, 9, 0, false, false>(ctx, ps, st);
            case 512: return launch_cfg<128, 9, 0, false, false>(ctx, ps, st);
            case 1024: return launch_cfg<256, 9, 0, false, false>(ctx, ps, st);
            default: return pr_fail(ctx, PR_EINVAL, "tb2d: no depth-9 pass at this width");
        }
    }
    switch (ctx->n) {
        case 128: return launch_depth<32, 8, 0>(ctx, ps, st);   // one warp per CTA
        case 256: return launch_depth<64, 8, 0>(ctx, ps, st);
        case 512: return launch_depth<128, 8, 0>(ctx, ps, st);
        case 1024: return launch_depth<256, 8, 0>(ctx, ps, st);
        case 2048: return pr_tb2d_launch_2048_d8(ctx, ps, st);
        default: return pr_fail(ctx, PR_EINVAL, "tb2d: unsupported grid size");
    }
}

}  // namespace

// depths with an instantiated kernel: 8 (default) and 4 (smaller register and
// shared-memory footprint; the batch autotuner chooses between them)
bool pr_tb2d_supported(const pr_ctx* ctx, int depth) {
    if (ctx->dim != 2 || ctx->dtype != PR_F32 || (depth != 8 && depth != 4)) return false;
    return ctx->n == 128 || ctx->n == 256 || ctx->n == 512 || ctx->n == 1024 || ctx->n == 2048;
}

// whether a pass of block_depth + 1 levels can run fused (four columns per
// thread, whole rows, depth 8): the sweep's final single level then joins the
// last pass instead of taking a one-level pass of its own
bool pr_tb2d_extra_level(const pr_ctx* ctx) {
    const int cols = ctx->tb_cols ? ctx->tb_cols : 4;
    return cols == 4 && ctx->block_depth == 8 && pr_tb2d_supported(ctx, 8) && ctx->n <= 1024;
}

pr_status pr_launch_fine_tb2d(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st) {
    if (ps.levels == 1) return pr_launch_fine_naive(ctx, ps, st);
    if (ctx->dim == 3) return pr_launch_fine_tb3d(ctx, ps, st);
    if ((ps.r_in || ps.r_out) && ps.rfmt != PR_RESID_BF16)
        return pr_fail(ctx, PR_EINVAL, "tb2d: the fused pass carries a bfloat16 residual");
    // Thread geometry (pr_set_fused_columns); by default four columns per
    // thread (this file) at every width: with static rings it is the faster
    // geometry on a GB300 at n = 512 and 1024 as well (8 warps per SM, the
    // x-neighbour exchange and per-row overhead shared by four columns), and
    // two columns per thread (fine_tb2d_c2.cu, twice the warps) stays
    // selectable.  n = 2048 runs four columns per thread whatever is set.
    const int cols = ctx->tb_cols ? ctx->tb_cols : 4;
    if (cols == 2 && ctx->n <= 1024) return pr_launch_fine_tb2d_c2(ctx, ps, st);
    const int B = ctx->block_depth;
    if (ps.levels < 1 || ps.levels > B + (pr_tb2d_extra_level(ctx) ? 1 : 0))
        return pr_fail(ctx, PR_EINVAL, "tb2d: bad level count");
    if (B == 8) return launch_d8(ctx, ps, st);
    if (B == 4) return pr_tb2d_launch_d4(ctx, ps, st);
    return pr_fail(ctx, PR_EINVAL, "tb2d: unsupported depth");
}

