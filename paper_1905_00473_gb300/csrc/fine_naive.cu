// One velocity-Verlet level (kick, then drift) per launch, for every slice of
// a batch, any dimension, FP32 or FP64.  This is the straightforward
// data-parallel form of F over all slices (Alg. 3, parFor; Sec. 3.1 scheme):
// every thread owns one grid column x of the rows it visits and reads the
// 2*dim neighbours of each point through the cache.  The 2D FP32 production path fuses several
// levels per HBM pass (fine_tb2d.cu); this kernel serves 1D, 3D, FP64, small
// grids and the final levels of a sweep whose step count is not a multiple of
// the fused depth.
//
// Level g of a slice with m steps (g = 0..m) applies
//     kick:  v += w_g kappa D(u),  w_g = 1/2 if g == 0 or g == m, else 1
//     drift: u += dt v             (only if g < m)
// where D is the undivided 2nd-order Laplacian and kappa = c^2 dt/dx^2, which
// is velocity Verlet (u_{n+1} = u_n + dt v_n + dt^2/2 a_n,
// v_{n+1} = v_n + dt/2 (a_n + a_{n+1}), a = c^2 L u) with the two half kicks
// of consecutive steps merged.
//
// Indexing is row-wise (grid_rows.cuh): x from the thread, the (slice, z, y)
// row from the block, so no point pays for an integer division.
//
// FP32 keeps u as (u_hi, rounding residual) between levels and evaluates
// D(u_hi + du) as D(u_hi) + D(du), with D(u_hi) formed from differences
// (u_nb - u_hi) so that the stencil of the O(1) field loses no bits to
// cancellation; du starts at the decoded residual.
#include "grid_rows.cuh"
#include "pr_internal.cuh"

namespace {

// RT: the residual's storage type (int8_t byte or uint16_t bfloat16).
// Thread (blockIdx.x, threadIdx.x) owns grid column x of every row it visits
// (grid_rows.cuh): rows blockIdx.y, blockIdx.y + gridDim.y, ...
template <int DIM, typename RT>
__global__ void __launch_bounds__(256) level_f32(
    const float* __restrict__ u, const RT* __restrict__ r, const float* __restrict__ v,
    const float* __restrict__ kap, float* __restrict__ uo, RT* __restrict__ ro,
    float* __restrict__ vo, int64_t n, int64_t pts, int64_t total_rows, float wk, float dt, int drift) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    for (int64_t row = blockIdx.y; row < total_rows; row += gridDim.y) {
        const rows::Row rw = rows::row_of<DIM>(row, n, pts);
        const int64_t p = rw.off + x;            // point inside the slice
        const int64_t idx = rw.slice_off + p;    // point of the batch
        const float* us = u + rw.slice_off;
        const RT* rs = r ? r + rw.slice_off : nullptr;
        int64_t nb[2 * DIM];
        rows::nbrs_of<DIM>(rw, x, n, nb);
        const float u0 = us[p];
        float du = rs ? pr_resid_get(rs[p], u0) : 0.0f;
        float d0 = 0.0f, dn = 0.0f;
#pragma unroll
        for (int k = 0; k < 2 * DIM; ++k) {
            const float ub = us[nb[k]];
            d0 += (ub - u0);
            if (rs) dn += pr_resid_get(rs[nb[k]], ub);
        }
        const float lap = d0 + fmaf(-2.0f * DIM, du, dn);
        const float vn = fmaf(wk * kap[p], lap, v[idx]);
        if (drift) du = fmaf(dt, vn, du);
        vo[idx] = vn;
        if (ro) {
            RT q;
            uo[idx] = pr_resid_put(u0, du, &q);
            ro[idx] = q;
        } else {
            uo[idx] = u0 + du;
        }
    }
}

// The same level with four consecutive points per thread (n % 4 == 0): every
// field is read as 128-bit quads, the x-neighbours of the quad's ends as two
// scalars.  Per point the arithmetic, and its order, is that of level_f32, so
// both give the same bits; this form needs a quarter of the load and store
// instructions, which bound the one-point kernel in 3D.
template <typename RT> struct ResidVec;
template <> struct ResidVec<int8_t> { typedef char4 type; };
template <> struct ResidVec<uint16_t> { typedef ushort4 type; };

// (at least 4 blocks per SM: 32 warps to keep enough loads in flight)
template <int DIM, typename RT>
__global__ void __launch_bounds__(256, 4) level_f32_x4(
    const float* __restrict__ u, const RT* __restrict__ r, const float* __restrict__ v,
    const float* __restrict__ kap, float* __restrict__ uo, RT* __restrict__ ro,
    float* __restrict__ vo, int64_t n, int64_t pts, int64_t total_rows, float wk, float dt, int drift) {
    typedef typename ResidVec<RT>::type RV;
    const int64_t x0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (x0 >= n) return;
    int64_t xl, xr;
    rows::quad_edges(x0, n, &xl, &xr);
    for (int64_t row = blockIdx.y; row < total_rows; row += gridDim.y) {
        const rows::Row rw = rows::row_of<DIM>(row, n, pts);
        const int64_t p = rw.off + x0;
        const int64_t idx = rw.slice_off + p;
        const auto uq = rows::load_quad<DIM, float, float4>(u + rw.slice_off, rw, x0, xl, xr);
        rows::Quad<DIM, RT, RV> rq;
        if (r) rq = rows::load_quad<DIM, RT, RV>(r + rw.slice_off, rw, x0, xl, xr);
        const float4 k4 = *(const float4*)(kap + p);
        const float4 v4 = *(const float4*)(v + idx);
        float uo_[4], vo_[4];
        RT ro_[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float u0 = rows::Quad<DIM, float, float4>::comp(uq.c, j);
            float du = r ? pr_resid_get(rows::Quad<DIM, RT, RV>::comp(rq.c, j), u0) : 0.0f;
            float d0 = 0.0f, dn = 0.0f;
#pragma unroll
            for (int k = 0; k < 2 * DIM; ++k) {
                const float ub = uq.nb(j, k);
                d0 += (ub - u0);
                if (r) dn += pr_resid_get(rq.nb(j, k), ub);
            }
            const float lap = d0 + fmaf(-2.0f * DIM, du, dn);
            const float vn = fmaf(wk * rows::Quad<DIM, float, float4>::comp(k4, j), lap,
                                  rows::Quad<DIM, float, float4>::comp(v4, j));
            if (drift) du = fmaf(dt, vn, du);
            vo_[j] = vn;
            if (ro) uo_[j] = pr_resid_put(u0, du, &ro_[j]);
            else uo_[j] = u0 + du;
        }
        *(float4*)(vo + idx) = make_float4(vo_[0], vo_[1], vo_[2], vo_[3]);
        *(float4*)(uo + idx) = make_float4(uo_[0], uo_[1], uo_[2], uo_[3]);
        if (ro) {
            RV q4;
            q4.x = ro_[0];
            q4.y = ro_[1];
            q4.z = ro_[2];
            q4.w = ro_[3];
            *(RV*)(ro + idx) = q4;
        }
    }
}

template <int DIM>
__global__ void __launch_bounds__(256) level_f64(
    const double* __restrict__ u, const double* __restrict__ v, const double* __restrict__ kap,
    double* __restrict__ uo, double* __restrict__ vo, int64_t n, int64_t pts, int64_t total_rows,
    double wk, double dt, int drift) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    for (int64_t row = blockIdx.y; row < total_rows; row += gridDim.y) {
        const rows::Row rw = rows::row_of<DIM>(row, n, pts);
        const int64_t p = rw.off + x;
        const int64_t idx = rw.slice_off + p;
        const double* us = u + rw.slice_off;
        int64_t nb[2 * DIM];
        rows::nbrs_of<DIM>(rw, x, n, nb);
        const double u0 = us[p];
        double lap = 0.0;
#pragma unroll
        for (int k = 0; k < 2 * DIM; ++k) lap += (us[nb[k]] - u0);
        const double vn = fma(wk * kap[p], lap, v[idx]);
        vo[idx] = vn;
        uo[idx] = drift ? fma(dt, vn, u0) : u0;
    }
}

// threads per row: n, or n / 4 for the four-point form
void launch_shape(const pr_ctx* ctx, int64_t nslices, int64_t per_row, dim3* grid, dim3* block) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    rows::shape_for(per_row, nslices * (ctx->pts / ctx->n), sms > 0 ? sms : 1, grid, block);
}

template <int DIM, typename RT>
void launch_f32(pr_ctx* ctx, const pr_pass& p, double wk, int drift, cudaStream_t st) {
    dim3 grid, block;
    const bool quads = ctx->n % 4 == 0;
    launch_shape(ctx, p.nslices, quads ? ctx->n / 4 : ctx->n, &grid, &block);
    auto kern = quads ? level_f32_x4<DIM, RT> : level_f32<DIM, RT>;
    kern<<<grid, block, 0, st>>>(
        (const float*)p.u_in, (const RT*)p.r_in, (const float*)p.v_in, (const float*)ctx->kappa,
        (float*)p.u_out, (RT*)p.r_out, (float*)p.v_out, ctx->n, ctx->pts,
        (int64_t)p.nslices * (ctx->pts / ctx->n), (float)wk, (float)ctx->dt_f, drift);
}

template <int DIM>
pr_status run_level(pr_ctx* ctx, const pr_pass& p, int g, const void* ui, const void* vi,
                    void* uo, void* vo, cudaStream_t st) {
    const int drift = g < p.m;
    const double wk = (g == 0 || g == p.m) ? 0.5 : 1.0;
    if (ctx->dtype == PR_F32) {
        if (p.rfmt == PR_RESID_BF16) launch_f32<DIM, uint16_t>(ctx, p, wk, drift, st);
        else launch_f32<DIM, int8_t>(ctx, p, wk, drift, st);
    } else {
        dim3 grid, block;
        launch_shape(ctx, p.nslices, ctx->n, &grid, &block);
        level_f64<DIM><<<grid, block, 0, st>>>(
            (const double*)ui, (const double*)vi, (const double*)ctx->kappa, (double*)uo,
            (double*)vo, ctx->n, ctx->pts, (int64_t)p.nslices * (ctx->pts / ctx->n), wk, ctx->dt_f, drift);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "fine level kernel launch");
    return PR_OK;
}

}  // namespace

// One pass of exactly one level (kick g0, drift if g0 < m).
pr_status pr_launch_fine_naive(pr_ctx* ctx, const pr_pass& p, cudaStream_t st) {
    if (p.levels != 1) return pr_fail(ctx, PR_EINVAL, "internal: naive pass must have one level");
    switch (ctx->dim) {
        case 1: return run_level<1>(ctx, p, p.g0, p.u_in, p.v_in, p.u_out, p.v_out, st);
        case 2: return run_level<2>(ctx, p, p.g0, p.u_in, p.v_in, p.u_out, p.v_out, st);
        default: return run_level<3>(ctx, p, p.g0, p.u_in, p.v_in, p.u_out, p.v_out, st);
    }
}
