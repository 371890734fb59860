// A whole 2D FP32 slice propagated inside one thread-block cluster (Sec. 3.1,
// the velocity Verlet stepper F or C over one coupling interval).
//
// For grids small enough that a slice's state fits in the distributed shared
// memory of one cluster (n <= 256 with 8 CTAs: the coarse grids of the 2D
// workloads), the m + 1 kicks of a slice run in ONE launch: each CTA holds
// n/8 rows of u_hi, D0, du (two buffers), u_t and kappa in shared memory,
// reads its neighbours' edge rows through distributed shared memory, and the
// cluster synchronises once per level.  Nothing goes to HBM between the load
// of the slice and the store of its end state.
//
// The arithmetic is the fused 2D kernel's, operation for operation, on the
// same pass plan (passes of block_depth levels, a lone last level merged into
// the last pass): within a pass u = u_hi + du with D(u) = D0 + D(du), D0 the
// 5-point Laplacian of u_hi; at a pass boundary (u_hi, r) = TwoSum(u_hi, du)
// and the next pass starts from du = bf16(r); the last pass rounds u_hi + du.
// Results are therefore bit-identical to the per-pass launches (tested), so
// the coarse values the parareal iteration differences (Alg. 3) cancel
// exactly whichever path computed them.
#include <cooperative_groups.h>

#include "pr_internal.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kRsCl = 8;     // CTAs per cluster (one slice per cluster)
constexpr int kRsT = 512;    // threads per CTA (one 4-point quad each at n = 128)
constexpr int kRsMaxPasses = 64;
constexpr int kRsQ = 4;      // 4-point quads per thread at most (n = 256: 32 rows x 64 quads / 512)

struct ResParams {
    const float* u_in;
    const float* v_in;
    const float* kap;
    float* u_out;
    float* v_out;
    int64_t pts;      // n * n
    int n;
    int m;            // steps per slice (m + 1 kicks)
    int depth;        // levels per pass
    int passes;
    int last_levels;  // levels of the last pass
    float dt;
};

// r rounded to bfloat16 (round to nearest even) and widened back, as the
// fused kernel stores and reloads its residual
__device__ __forceinline__ float rs_bf16_round(float r) {
    uint32_t w;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(w) : "f"(0.0f), "f"(r));
    return __uint_as_float(w << 16);
}

// Q: 4-point quads per thread (1 at n = 128, up to kRsQ at n = 256); with one
// quad the kernel fits 64 registers, so two CTAs share an SM
template <int Q>
__global__ void __cluster_dims__(kRsCl, 1, 1) __launch_bounds__(kRsT, Q == 1 ? 2 : 1)
    resident2d_kernel(ResParams p) {
    extern __shared__ float rs_sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int64_t slice = blockIdx.x / kRsCl;
    const int n = p.n, H = n / kRsCl, hn = H * n, nq = n / 4;
    float* uh = rs_sm;                        // [H][n] u_hi
    float* d0 = uh + hn;                      // [H][n] D0 of this pass
    float* dub[2] = {d0 + hn, d0 + 2 * hn};   // [H][n] du, level input / output
    float* vv = d0 + 3 * hn;                  // [H][n] u_t
    float* kp = d0 + 4 * hn;                  // [H][n] kappa
    const int row0 = rank * H;
    const int64_t base = slice * p.pts + (int64_t)row0 * n;
    for (int idx = threadIdx.x; idx < hn / 4; idx += kRsT) {
        ((float4*)uh)[idx] = __ldcs((const float4*)(p.u_in + base) + idx);
        ((float4*)vv)[idx] = __ldcs((const float4*)(p.v_in + base) + idx);
        ((float4*)kp)[idx] = __ldg((const float4*)(p.kap + (int64_t)row0 * n) + idx);
        ((float4*)dub[0])[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // the neighbours' shared arrays: south = the row above this CTA's first
    // row (rank - 1), north = the row below its last (rank + 1), periodic
    const unsigned rs = (unsigned)((rank + kRsCl - 1) % kRsCl), rn = (unsigned)((rank + 1) % kRsCl);
    const float* const uh_s = cl.map_shared_rank(uh, rs);
    const float* const uh_n = cl.map_shared_rank(uh, rn);
    const float* const du_s0 = cl.map_shared_rank(dub[0], rs);
    const float* const du_s1 = cl.map_shared_rank(dub[1], rs);
    const float* const du_n0 = cl.map_shared_rank(dub[0], rn);
    const float* const du_n1 = cl.map_shared_rank(dub[1], rn);
    // this thread's quads (the same at every level): row, first column and
    // the periodic left / right neighbour columns, computed once
    int qr[Q], qc[Q], ql[Q], qx[Q];
    const int nquads = hn / 4;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int q = threadIdx.x + k * kRsT;
        const int r = q / nq, c0 = 4 * (q - r * nq);
        qr[k] = r;
        qc[k] = c0;
        ql[k] = c0 == 0 ? n - 1 : c0 - 1;
        qx[k] = c0 + 4 == n ? 0 : c0 + 4;
    }
    cl.sync();
    const float dt = p.dt;
    int cur = 0;
    for (int ps = 0; ps < p.passes; ++ps) {
        const bool last = ps == p.passes - 1;
        const int g0 = ps * p.depth;
        const int levels = last ? p.last_levels : p.depth;
        // D0 = ((W - C) + (E - C)) + ((S - C) + (N - C)) of u_hi
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            if (threadIdx.x + j * kRsT >= nquads) break;
            const int r = qr[j], c0 = qc[j];
            const float* rowc = uh + r * n;
            const float* rows = r > 0 ? uh + (r - 1) * n : uh_s + (H - 1) * n;
            const float* rown = r < H - 1 ? uh + (r + 1) * n : uh_n;
            const float4 C = *(const float4*)(rowc + c0);
            const float4 S = *(const float4*)(rows + c0);
            const float4 N = *(const float4*)(rown + c0);
            const float xl = rowc[ql[j]], xr = rowc[qx[j]];
            const float cc[4] = {C.x, C.y, C.z, C.w}, ss[4] = {S.x, S.y, S.z, S.w}, nn[4] = {N.x, N.y, N.z, N.w};
            float o[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float lf = k == 0 ? xl : cc[k - 1], rt = k == 3 ? xr : cc[k + 1];
                o[k] = __fadd_rn(__fadd_rn(__fsub_rn(lf, cc[k]), __fsub_rn(rt, cc[k])),
                                 __fadd_rn(__fsub_rn(ss[k], cc[k]), __fsub_rn(nn[k], cc[k])));
            }
            *(float4*)(d0 + r * n + c0) = make_float4(o[0], o[1], o[2], o[3]);
        }
        for (int l = 0; l < levels; ++l) {
            const int g = g0 + l;
            const float half = (g == 0 || g == p.m) ? 0.5f : 1.0f;
            const bool drift = g < p.m;
            const float* du = cur ? dub[1] : dub[0];
            float* dn = cur ? dub[0] : dub[1];
            const float* du_s = cur ? du_s1 : du_s0;
            const float* du_n = cur ? du_n1 : du_n0;
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                if (threadIdx.x + j * kRsT >= nquads) break;
                const int r = qr[j], c0 = qc[j];
                const float* rowc = du + r * n;
                const float* rows = r > 0 ? du + (r - 1) * n : du_s + (H - 1) * n;
                const float* rown = r < H - 1 ? du + (r + 1) * n : du_n;
                const float4 C = *(const float4*)(rowc + c0);
                const float4 S = *(const float4*)(rows + c0);
                const float4 N = *(const float4*)(rown + c0);
                const float4 D = *(const float4*)(d0 + r * n + c0);
                const float4 K = *(const float4*)(kp + r * n + c0);
                const float4 V = *(const float4*)(vv + r * n + c0);
                const float xl = rowc[ql[j]], xr = rowc[qx[j]];
                const float cc[4] = {C.x, C.y, C.z, C.w}, ss[4] = {S.x, S.y, S.z, S.w};
                const float nn[4] = {N.x, N.y, N.z, N.w}, dd[4] = {D.x, D.y, D.z, D.w};
                const float kk[4] = {K.x, K.y, K.z, K.w}, vi[4] = {V.x, V.y, V.z, V.w};
                float vo[4], uo[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    // the fused kernel's order: ((W + E) + S), then D0 + (. - 4 C),
                    // then + N, then the kick and the drift
                    const float lf = k == 0 ? xl : cc[k - 1], rt = k == 3 ? xr : cc[k + 1];
                    const float hs = __fadd_rn(__fadd_rn(lf, rt), ss[k]);
                    const float part = __fadd_rn(dd[k], __fmaf_rn(-4.0f, cc[k], hs));
                    vo[k] = __fmaf_rn(__fmul_rn(kk[k], half), __fadd_rn(part, nn[k]), vi[k]);
                    uo[k] = drift ? __fmaf_rn(dt, vo[k], cc[k]) : cc[k];
                }
                *(float4*)(vv + r * n + c0) = make_float4(vo[0], vo[1], vo[2], vo[3]);
                *(float4*)(dn + r * n + c0) = make_float4(uo[0], uo[1], uo[2], uo[3]);
            }
            cl.sync();
            cur ^= 1;
        }
        float* du = cur ? dub[1] : dub[0];
        if (!last) {
            // (u_hi, r) = TwoSum(u_hi, du); the next pass starts from bf16(r)
            for (int idx = threadIdx.x; idx < hn; idx += kRsT) {
                float r;
                uh[idx] = pr_two_sum(uh[idx], du[idx], &r);
                du[idx] = rs_bf16_round(r);
            }
            cl.sync();
        } else {
            for (int idx = threadIdx.x; idx < hn / 4; idx += kRsT) {
                const float4 a = ((const float4*)uh)[idx], b = ((const float4*)du)[idx];
                ((float4*)(p.u_out + base))[idx] =
                    make_float4(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y), __fadd_rn(a.z, b.z), __fadd_rn(a.w, b.w));
                ((float4*)(p.v_out + base))[idx] = ((const float4*)vv)[idx];
            }
        }
    }
    // no CTA leaves while a neighbour may still read its shared memory
    cl.sync();
}

// the per-pass plan of pr_fine_all_slices for this context
void rs_plan(const pr_ctx* ctx, int& passes, int& last_levels) {
    const int levels_total = ctx->m_f + 1;
    const int depth = ctx->block_depth;
    passes = (levels_total + depth - 1) / depth;
    const bool merge_last = passes >= 2 && levels_total % depth == 1 && pr_tb2d_extra_level(ctx);
    if (merge_last) --passes;
    last_levels = levels_total - (passes - 1) * depth;
}

}  // namespace

bool pr_resident2d_supported(const pr_ctx* ctx) {
    // exactly where the per-pass path runs the four-column fused kernel at depth 8
    const int cols = ctx->tb_cols ? ctx->tb_cols : 4;
    if (ctx->dim != 2 || ctx->dtype != PR_F32 || ctx->block_depth != 8 || cols != 4 || !pr_tb2d_supported(ctx, 8))
        return false;
    const int64_t n = ctx->n;
    if (n % (4 * kRsCl) != 0) return false;
    const int64_t H = n / kRsCl;
    if (6 * H * n * 4 > 227 * 1024 || H * (n / 4) > (int64_t)kRsQ * kRsT) return false;
    int passes = 0, last_levels = 0;
    rs_plan(ctx, passes, last_levels);
    // the per-pass plan runs lone levels through the one-level kernel (another
    // residual format): only plans of fused passes are reproduced here
    return passes <= kRsMaxPasses && last_levels >= 2;
}

pr_status pr_launch_resident2d(pr_ctx* ctx, const void* u_in, const void* v_in, void* u_out, void* v_out,
                               int nslices, cudaStream_t st) {
    ResParams p;
    p.u_in = (const float*)u_in;
    p.v_in = (const float*)v_in;
    p.kap = (const float*)ctx->kappa;
    p.u_out = (float*)u_out;
    p.v_out = (float*)v_out;
    p.pts = ctx->pts;
    p.n = (int)ctx->n;
    p.m = ctx->m_f;
    p.depth = ctx->block_depth;
    rs_plan(ctx, p.passes, p.last_levels);
    p.dt = (float)ctx->dt_f;
    const size_t smem = (size_t)6 * (ctx->n / kRsCl) * ctx->n * 4;
    const int64_t quads = (ctx->n / kRsCl) * (ctx->n / 4);
    auto kern = quads <= kRsT ? resident2d_kernel<1> : resident2d_kernel<kRsQ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "resident2d: shared memory attribute");
    kern<<<nslices * kRsCl, kRsT, smem, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "resident2d launch");
    return PR_OK;
}
