// One velocity-Verlet level (kick, then drift) per launch, for every slice of
// a batch, any dimension, FP32 or FP64.  This is the straightforward
// data-parallel form of F over all slices (Alg. 3, parFor; Sec. 3.1 scheme):
// every thread owns one grid point of one slice and reads its 2*dim
// neighbours through the cache.  The 2D FP32 production path fuses several
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
// FP32 keeps u as (u_hi, rounding residual) between levels and evaluates
// D(u_hi + du) as D(u_hi) + D(du), with D(u_hi) formed from differences
// (u_nb - u_hi) so that the stencil of the O(1) field loses no bits to
// cancellation; du starts at the decoded residual.
#include "pr_internal.cuh"

namespace {

template <int DIM>
__device__ __forceinline__ void neighbours(int64_t p, int64_t n, int64_t* nb) {
    // nb[2*a] = +1 along axis a, nb[2*a+1] = -1 along axis a (periodic)
    int64_t stride = 1;
    int64_t rem = p;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        int64_t i = rem % n;
        rem /= n;
        int64_t ip = (i + 1 == n) ? 0 : i + 1;
        int64_t im = (i == 0) ? n - 1 : i - 1;
        nb[2 * a] = p + (ip - i) * stride;
        nb[2 * a + 1] = p + (im - i) * stride;
        stride *= n;
    }
}

// RT: the residual's storage type (int8_t byte or uint16_t bfloat16)
template <int DIM, typename RT>
__global__ void __launch_bounds__(256) level_f32(
    const float* __restrict__ u, const RT* __restrict__ r, const float* __restrict__ v,
    const float* __restrict__ kap, float* __restrict__ uo, RT* __restrict__ ro,
    float* __restrict__ vo, int64_t n, int64_t pts, int64_t total, float wk, float dt, int drift) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += stride) {
        const int64_t s = idx / pts;
        const int64_t p = idx - s * pts;
        const float* us = u + s * pts;
        const RT* rs = r ? r + s * pts : nullptr;
        int64_t nb[2 * DIM];
        neighbours<DIM>(p, n, nb);
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

template <int DIM>
__global__ void __launch_bounds__(256) level_f64(
    const double* __restrict__ u, const double* __restrict__ v, const double* __restrict__ kap,
    double* __restrict__ uo, double* __restrict__ vo, int64_t n, int64_t pts, int64_t total,
    double wk, double dt, int drift) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += stride) {
        const int64_t s = idx / pts;
        const int64_t p = idx - s * pts;
        const double* us = u + s * pts;
        int64_t nb[2 * DIM];
        neighbours<DIM>(p, n, nb);
        const double u0 = us[p];
        double lap = 0.0;
#pragma unroll
        for (int k = 0; k < 2 * DIM; ++k) lap += (us[nb[k]] - u0);
        const double vn = fma(wk * kap[p], lap, v[idx]);
        vo[idx] = vn;
        uo[idx] = drift ? fma(dt, vn, u0) : u0;
    }
}

template <typename K>
int grid_for(K kernel, int64_t total) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0);
    int64_t want = (total + 255) / 256;
    int64_t cap = (int64_t)sms * (per_sm > 0 ? per_sm : 1) * 4;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

template <int DIM, typename RT>
void launch_f32(pr_ctx* ctx, const pr_pass& p, int64_t total, double wk, int drift, cudaStream_t st) {
    auto k = level_f32<DIM, RT>;
    k<<<grid_for(k, total), 256, 0, st>>>(
        (const float*)p.u_in, (const RT*)p.r_in, (const float*)p.v_in, (const float*)ctx->kappa,
        (float*)p.u_out, (RT*)p.r_out, (float*)p.v_out, ctx->n, ctx->pts, total, (float)wk,
        (float)ctx->dt_f, drift);
}

template <int DIM>
pr_status run_level(pr_ctx* ctx, const pr_pass& p, int g, const void* ui, const void* vi,
                    void* uo, void* vo, cudaStream_t st) {
    const int64_t total = (int64_t)p.nslices * ctx->pts;
    const int drift = g < p.m;
    const double wk = (g == 0 || g == p.m) ? 0.5 : 1.0;
    if (ctx->dtype == PR_F32) {
        if (p.rfmt == PR_RESID_BF16) launch_f32<DIM, uint16_t>(ctx, p, total, wk, drift, st);
        else launch_f32<DIM, int8_t>(ctx, p, total, wk, drift, st);
    } else {
        auto k = level_f64<DIM>;
        k<<<grid_for(k, total), 256, 0, st>>>(
            (const double*)ui, (const double*)vi, (const double*)ctx->kappa, (double*)uo,
            (double*)vo, ctx->n, ctx->pts, total, wk, ctx->dt_f, drift);
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
