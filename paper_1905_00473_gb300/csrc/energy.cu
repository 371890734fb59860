// Discrete wave energy of every slice (Sec. 3.1, eq. discrete-wave-energy):
//   E = 1/2 sum_j |nabla_h u(x_j)|^2 dx^d + 1/2 sum_j c_j^-2 |u_t(x_j)|^2 dx^d
// with nabla_h the 4th-order central difference (Sec. 6.4), accumulated in
// FP64 with a fixed-order two-level reduction (deterministic).
#include "pr_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 512;

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) energy_partials(
    const T* __restrict__ u, const T* __restrict__ v, const double* __restrict__ cinv2,
    int64_t n, int64_t pts, double inv_dx, double* __restrict__ partials) {
    const int s = blockIdx.y;
    const T* us = u + (int64_t)s * pts;
    const T* vs = v + (int64_t)s * pts;
    double acc = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x; p < pts;
         p += (int64_t)gridDim.x * kThreads) {
        int64_t rem = p, stride = 1;
        double g2 = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const int64_t i = rem % n;
            rem /= n;
            const int64_t base = p - i * stride;
            auto at = [&](int64_t k) { return (double)us[base + ((i + k + n) % n) * stride]; };
            const double d = (2.0 / 3.0) * (at(1) - at(-1)) - (1.0 / 12.0) * (at(2) - at(-2));
            g2 += d * d;
            stride *= n;
        }
        const double vv = (double)vs[p];
        acc += g2 * inv_dx * inv_dx + cinv2[p] * vv * vv;
    }
    __shared__ double red[kThreads];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[(int64_t)s * gridDim.x + blockIdx.x] = red[0];
}

__global__ void energy_finish(const double* __restrict__ partials, int nblocks, double scale,
                              double* __restrict__ out) {
    const int s = blockIdx.x;
    if (threadIdx.x == 0) {
        double acc = 0.0;
        for (int b = 0; b < nblocks; ++b) acc += partials[(int64_t)s * nblocks + b];
        out[s] = 0.5 * acc * scale;
    }
}

template <typename T, int DIM>
void launch(const pr_ctx* ctx, const void* u, const void* v, int ns, int nb, double* part,
            cudaStream_t st) {
    energy_partials<T, DIM><<<dim3(nb, ns), kThreads, 0, st>>>(
        (const T*)u, (const T*)v, ctx->cinv2, ctx->n, ctx->pts, 1.0 / ctx->dx, part);
}

}  // namespace

pr_status pr_launch_energy(pr_ctx* ctx, const void* u, const void* v, int ns, double* e_host,
                           cudaStream_t st) {
    int64_t nb = (ctx->pts + kThreads * 8 - 1) / (kThreads * 8);
    if (nb > kMaxBlocks) nb = kMaxBlocks;
    if (nb < 1) nb = 1;
    const int64_t need = (int64_t)ns * nb + ns;
    if (need > ctx->partials_len) {
        pr_dev_free(ctx, ctx->partials);
        ctx->partials = nullptr;
        ctx->partials_len = 0;
        PR_CUDA_TRY(ctx, pr_dev_malloc(ctx, (void**)&ctx->partials, need * sizeof(double)));
        ctx->partials_len = need;
    }
    double* part = ctx->partials;
    double* out = ctx->partials + (int64_t)ns * nb;
    const bool f32 = ctx->dtype == PR_F32;
    switch (ctx->dim) {
        case 1: f32 ? launch<float, 1>(ctx, u, v, ns, (int)nb, part, st) : launch<double, 1>(ctx, u, v, ns, (int)nb, part, st); break;
        case 2: f32 ? launch<float, 2>(ctx, u, v, ns, (int)nb, part, st) : launch<double, 2>(ctx, u, v, ns, (int)nb, part, st); break;
        default: f32 ? launch<float, 3>(ctx, u, v, ns, (int)nb, part, st) : launch<double, 3>(ctx, u, v, ns, (int)nb, part, st); break;
    }
    double vol = 1.0;
    for (int a = 0; a < ctx->dim; ++a) vol *= ctx->dx;
    energy_finish<<<ns, 32, 0, st>>>(part, (int)nb, vol, out);
    PR_CUDA_TRY(ctx, cudaGetLastError());
    PR_CUDA_TRY(ctx, cudaMemcpyAsync(e_host, out, ns * sizeof(double), cudaMemcpyDeviceToHost, st));
    PR_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    return PR_OK;
}
