// Fused 2D FP32 passes at depth 4 (every width), and the 2048-point rows at
// depth 8, whose rows are shared by a two-CTA cluster (tb2d_kernels.cuh).
#include "tb2d_kernels.cuh"

pr_status pr_tb2d_launch_d4(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st) {
    switch (ctx->n) {
        case 128: return launch_depth<32, 4, 0>(ctx, ps, st);
        case 256: return launch_depth<64, 4, 0>(ctx, ps, st);
        case 512: return launch_depth<128, 4, 0>(ctx, ps, st);
        case 1024: return launch_depth<256, 4, 0>(ctx, ps, st);
        // two x-strips of 1040 columns (1024 final + 8 each side) per row,
        // 260 threads (9 warps, 3 on one SM sub-partition, at most 168
        // registers a thread)
        case 2048: return launch_depth<260, 4, 8>(ctx, ps, st);
        default: return pr_fail(ctx, PR_EINVAL, "tb2d: unsupported grid size");
    }
}

// depth 8 at n = 2048: three x-strips of 704 columns per row (688 final + 8
// each side; the third overlaps the first by 16 final columns, which only the
// first writes), 176 threads a CTA and no exchange (pr_set_wide_rows 2, the
// default: 8.3e11 against 7.8e11 point-updates/s on 2048^2 x 64), or every
// row shared by a cluster of two CTAs of 256 threads, which exchange the
// x-edges of the half-rows through distributed shared memory (1).  Two CTAs
// of 128 threads per SM in five strips of 512 columns measured 8.0e11.
pr_status pr_tb2d_launch_2048_d8(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st) {
    if (ctx->wide_rows == 1) return launch_depth<256, 8, 0, 2>(ctx, ps, st);
    return launch_depth<176, 8, 8>(ctx, ps, st);
}
