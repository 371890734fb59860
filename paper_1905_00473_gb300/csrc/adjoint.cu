// Reverse mode through the serial fine solve F^N (pr_adjoint).
//
// The forward map of one slice is the level recurrence of the fine kernels
// (Sec. 3.1 velocity Verlet with merged half kicks; g = 0..m):
//     v <- v + w_g kappa (D u_g);   u_{g+1} = u_g + dt v   (g < m)
// with D the undivided periodic Laplacian (symmetric) and kappa = c^2 dt/dx^2.
// Its transpose, level by level in reverse, for adjoints (lu, lv) of the
// level's outputs:
//     mu  = lv + dt lu            (lv at the last level, which does not drift)
//     gk += w_g (D u_g) mu        (dL/dkappa)
//     lu <- lu + w_g D(kappa mu)  (kappa inside the stencil: (K D)^T = D K)
//     lv <- mu
// and finally dL/dc = dL/dkappa * 2 c dt / dx^2.  Slice-start states are
// checkpointed in a forward pass; inside each slice the states u_g are
// recomputed from its checkpoint (memory: (N+1) + (m+1) fields).
// Arithmetic is plain in the context dtype; dL/dkappa accumulates in FP64.
#include <stdio.h>

#include "pr_internal.cuh"

namespace {

constexpr int kT = 256;

template <int DIM>
__device__ __forceinline__ void nbrs(int64_t p, int64_t n, int64_t* nb) {
    int64_t stride = 1, rem = p;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const int64_t i = rem % n;
        rem /= n;
        nb[2 * a] = p + (((i + 1 == n) ? 0 : i + 1) - i) * stride;
        nb[2 * a + 1] = p + (((i == 0) ? n - 1 : i - 1) - i) * stride;
        stride *= n;
    }
}

// forward level with trace: v += w kappa D(u_g) in place; u_{g+1} -> un
template <typename T, int DIM>
__global__ void fwd_level(const T* __restrict__ u, T* __restrict__ v, T* __restrict__ un,
                          const T* __restrict__ kap, int64_t n, int64_t pts, T w, T dt, int drift) {
    for (int64_t p = (int64_t)blockIdx.x * kT + threadIdx.x; p < pts; p += (int64_t)gridDim.x * kT) {
        int64_t nb[2 * DIM];
        nbrs<DIM>(p, n, nb);
        const T u0 = u[p];
        T lap = 0;
#pragma unroll
        for (int k = 0; k < 2 * DIM; ++k) lap += (u[nb[k]] - u0);
        const T vn = v[p] + w * kap[p] * lap;
        v[p] = vn;
        if (drift) un[p] = u0 + dt * vn;
    }
}

template <typename T, int DIM>
__global__ void adj_level(const T* __restrict__ lu, const T* __restrict__ lv, const T* __restrict__ ug,
                          const T* __restrict__ kap, T* __restrict__ lu_o, T* __restrict__ lv_o,
                          double* __restrict__ gk, int64_t n, int64_t pts, T w, T dt, int drift) {
    for (int64_t p = (int64_t)blockIdx.x * kT + threadIdx.x; p < pts; p += (int64_t)gridDim.x * kT) {
        int64_t nb[2 * DIM];
        nbrs<DIM>(p, n, nb);
        const T mu = drift ? lv[p] + dt * lu[p] : lv[p];
        const T kmu = kap[p] * mu;
        T dkm = 0, du = 0;
        const T u0 = ug[p];
#pragma unroll
        for (int k = 0; k < 2 * DIM; ++k) {
            const int64_t q = nb[k];
            const T muq = drift ? lv[q] + dt * lu[q] : lv[q];
            dkm += kap[q] * muq - kmu;
            du += ug[q] - u0;
        }
        gk[p] += (double)w * (double)du * (double)mu;
        lu_o[p] = lu[p] + w * dkm;
        lv_o[p] = mu;
    }
}

template <typename T>
__global__ void finish_grad(const double* __restrict__ gk, const double* __restrict__ c, T* __restrict__ gc,
                            int64_t pts, double scale) {
    for (int64_t p = (int64_t)blockIdx.x * kT + threadIdx.x; p < pts; p += (int64_t)gridDim.x * kT)
        gc[p] = (T)(gk[p] * 2.0 * c[p] * scale);
}

int nblocks(int64_t m) {
    int64_t b = (m + kT - 1) / kT;
    return (int)(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

template <typename T, int DIM>
pr_status run(pr_ctx* ctx, const T* u0, const T* p0, const T* guT, const T* gvT, T* gc, T* gu0, T* gp0,
              cudaStream_t st) {
    const int64_t pts = ctx->pts, n = ctx->n;
    const int N = ctx->N, m = ctx->m_f;
    const size_t fb = (size_t)pts * sizeof(T);
    // workspace: checkpoints (N+1) x (u, v), trace (m+1), v, 4 adjoint fields, FP64 gk
    const size_t need = (size_t)(2 * (N + 1) + (m + 1) + 1 + 4) * fb + (size_t)pts * 8;
    if (need > ctx->adj_bytes) {
        cudaFree(ctx->adj_ws);
        ctx->adj_ws = nullptr;
        ctx->adj_bytes = 0;
        cudaError_t e = cudaMalloc(&ctx->adj_ws, need);
        if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "pr_adjoint: workspace");
        ctx->adj_bytes = need;
    }
    T* base = (T*)ctx->adj_ws;
    T* cu = base;                           // [N+1][pts]
    T* cv = cu + (size_t)(N + 1) * pts;     // [N+1][pts]
    T* tr = cv + (size_t)(N + 1) * pts;     // [m+1][pts]
    T* vw = tr + (size_t)(m + 1) * pts;     // [pts]
    T* la[2] = {vw + pts, vw + 2 * pts};
    T* lb[2] = {vw + 3 * pts, vw + 4 * pts};
    double* gk = (double*)(vw + 5 * pts);
    const T* kap = (const T*)ctx->kappa;
    const T dt = (T)ctx->dt_f;
    auto w_of = [&](int g) { return (T)((g == 0 || g == m) ? 0.5 : 1.0); };
    const int nb = nblocks(pts);

    auto recompute = [&](int s) {   // trace of slice s from its checkpoint; leaves v in vw
        cudaMemcpyAsync(tr, cu + (size_t)s * pts, fb, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(vw, cv + (size_t)s * pts, fb, cudaMemcpyDeviceToDevice, st);
        for (int g = 0; g <= m; ++g)
            fwd_level<T, DIM><<<nb, kT, 0, st>>>(tr + (size_t)g * pts, vw, tr + (size_t)(g + 1 <= m ? g + 1 : g) * pts,
                                                 kap, n, pts, w_of(g), dt, g < m);
    };
    // forward: checkpoints
    cudaMemcpyAsync(cu, u0, fb, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(cv, p0, fb, cudaMemcpyDeviceToDevice, st);
    for (int s = 0; s < N; ++s) {
        recompute(s);
        cudaMemcpyAsync(cu + (size_t)(s + 1) * pts, tr + (size_t)m * pts, fb, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(cv + (size_t)(s + 1) * pts, vw, fb, cudaMemcpyDeviceToDevice, st);
    }
    // reverse
    cudaMemcpyAsync(la[0], guT, fb, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(lb[0], gvT, fb, cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(gk, 0, (size_t)pts * 8, st);
    int cur = 0;
    for (int s = N - 1; s >= 0; --s) {
        recompute(s);
        for (int g = m; g >= 0; --g) {
            adj_level<T, DIM><<<nb, kT, 0, st>>>(la[cur], lb[cur], tr + (size_t)g * pts, kap, la[cur ^ 1],
                                                 lb[cur ^ 1], gk, n, pts, w_of(g), dt, g < m);
            cur ^= 1;
        }
    }
    cudaMemcpyAsync(gu0, la[cur], fb, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(gp0, lb[cur], fb, cudaMemcpyDeviceToDevice, st);
    finish_grad<T><<<nb, kT, 0, st>>>(gk, ctx->c64, gc, pts, ctx->dt_f / (ctx->dx * ctx->dx));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "pr_adjoint: launch");
    return PR_OK;
}

}  // namespace

extern "C" pr_status pr_adjoint(pr_ctx* ctx, const void* u0, const void* p0, const void* gu_T,
                                const void* gv_T, void* gc, void* gu0, void* gp0, void* stream) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_adjoint: ctx is NULL");
    if (!u0 || !p0 || !gu_T || !gv_T || !gc || !gu0 || !gp0)
        return pr_fail(ctx, PR_EINVAL, "pr_adjoint: NULL array");
    cudaStream_t st = (cudaStream_t)stream;
    const bool f32 = ctx->dtype == PR_F32;
    switch (ctx->dim) {
        case 1: return f32 ? run<float, 1>(ctx, (const float*)u0, (const float*)p0, (const float*)gu_T, (const float*)gv_T, (float*)gc, (float*)gu0, (float*)gp0, st)
                           : run<double, 1>(ctx, (const double*)u0, (const double*)p0, (const double*)gu_T, (const double*)gv_T, (double*)gc, (double*)gu0, (double*)gp0, st);
        case 2: return f32 ? run<float, 2>(ctx, (const float*)u0, (const float*)p0, (const float*)gu_T, (const float*)gv_T, (float*)gc, (float*)gu0, (float*)gp0, st)
                           : run<double, 2>(ctx, (const double*)u0, (const double*)p0, (const double*)gu_T, (const double*)gv_T, (double*)gc, (double*)gu0, (double*)gp0, st);
        default: return f32 ? run<float, 3>(ctx, (const float*)u0, (const float*)p0, (const float*)gu_T, (const float*)gv_T, (float*)gc, (float*)gu0, (float*)gp0, st)
                            : run<double, 3>(ctx, (const double*)u0, (const double*)p0, (const double*)gu_T, (const double*)gv_T, (double*)gc, (double*)gu0, (double*)gp0, st);
    }
}
