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

#include "grid_rows.cuh"
#include "pr_internal.cuh"

namespace {

constexpr int kT = 256;

// The level kernels index one slice row-wise (grid_rows.cuh): x from the
// thread, the (z, y) row from a grid-stride loop over blockIdx.y.

// forward level with trace: v += w kappa D(u_g) in place; u_{g+1} -> un
template <typename T, int DIM>
__global__ void fwd_level(const T* __restrict__ u, T* __restrict__ v, T* __restrict__ un,
                          const T* __restrict__ kap, int64_t n, int64_t pts, T w, T dt, int drift) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    for (int64_t row = blockIdx.y; row < pts / n; row += gridDim.y) {
        const rows::Row rw = rows::row_of<DIM>(row, n, pts);
        const int64_t p = rw.off + x;
        int64_t nb[2 * DIM];
        rows::nbrs_of<DIM>(rw, x, n, nb);
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
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    for (int64_t row = blockIdx.y; row < pts / n; row += gridDim.y) {
        const rows::Row rw = rows::row_of<DIM>(row, n, pts);
        const int64_t p = rw.off + x;
        int64_t nb[2 * DIM];
        rows::nbrs_of<DIM>(rw, x, n, nb);
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

// FP32 forms of the two level kernels with four consecutive points per thread
// (n % 4 == 0): 128-bit quads of every field and of its y/z neighbours
// (grid_rows.cuh), the same arithmetic in the same order per point.
template <int DIM>
__global__ void __launch_bounds__(256, 4) fwd_level_x4(const float* __restrict__ u, float* __restrict__ v, float* __restrict__ un,
                             const float* __restrict__ kap, int64_t n, int64_t pts, float w, float dt, int drift) {
    typedef rows::Quad<DIM, float, float4> Q;
    const int64_t x0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (x0 >= n) return;
    int64_t xl, xr;
    rows::quad_edges(x0, n, &xl, &xr);
    for (int64_t row = blockIdx.y; row < pts / n; row += gridDim.y) {
        const rows::Row rw = rows::row_of<DIM>(row, n, pts);
        const int64_t p = rw.off + x0;
        const Q uq = rows::load_quad<DIM, float, float4>(u, rw, x0, xl, xr);
        const float4 k4 = *(const float4*)(kap + p);
        const float4 v4 = *(const float4*)(v + p);
        float vn[4], u1[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float u0 = Q::comp(uq.c, j);
            float lap = 0;
#pragma unroll
            for (int k = 0; k < 2 * DIM; ++k) lap += (uq.nb(j, k) - u0);
            vn[j] = Q::comp(v4, j) + w * Q::comp(k4, j) * lap;
            u1[j] = u0 + dt * vn[j];
        }
        *(float4*)(v + p) = make_float4(vn[0], vn[1], vn[2], vn[3]);
        if (drift) *(float4*)(un + p) = make_float4(u1[0], u1[1], u1[2], u1[3]);
    }
}

template <int DIM>
__global__ void __launch_bounds__(256) adj_level_x4(const float* __restrict__ lu, const float* __restrict__ lv,
                             const float* __restrict__ ug, const float* __restrict__ kap,
                             float* __restrict__ lu_o, float* __restrict__ lv_o, double* __restrict__ gk,
                             int64_t n, int64_t pts, float w, float dt, int drift) {
    typedef rows::Quad<DIM, float, float4> Q;
    const int64_t x0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (x0 >= n) return;
    int64_t xl, xr;
    rows::quad_edges(x0, n, &xl, &xr);
    for (int64_t row = blockIdx.y; row < pts / n; row += gridDim.y) {
        const rows::Row rw = rows::row_of<DIM>(row, n, pts);
        const int64_t p = rw.off + x0;
        const Q lvq = rows::load_quad<DIM, float, float4>(lv, rw, x0, xl, xr);
        const Q luq = rows::load_quad<DIM, float, float4>(lu, rw, x0, xl, xr);
        const Q kq = rows::load_quad<DIM, float, float4>(kap, rw, x0, xl, xr);
        const Q gq = rows::load_quad<DIM, float, float4>(ug, rw, x0, xl, xr);
        const double2 g01 = *(const double2*)(gk + p), g23 = *(const double2*)(gk + p + 2);
        double go[4] = {g01.x, g01.y, g23.x, g23.y};
        float luo[4], lvo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float lvj = Q::comp(lvq.c, j), luj = Q::comp(luq.c, j);
            const float mu = drift ? lvj + dt * luj : lvj;
            const float kmu = Q::comp(kq.c, j) * mu;
            float dkm = 0, du = 0;
            const float u0 = Q::comp(gq.c, j);
#pragma unroll
            for (int k = 0; k < 2 * DIM; ++k) {
                const float muq = drift ? lvq.nb(j, k) + dt * luq.nb(j, k) : lvq.nb(j, k);
                dkm += kq.nb(j, k) * muq - kmu;
                du += gq.nb(j, k) - u0;
            }
            go[j] += (double)w * (double)du * (double)mu;
            luo[j] = luj + w * dkm;
            lvo[j] = mu;
        }
        *(double2*)(gk + p) = make_double2(go[0], go[1]);
        *(double2*)(gk + p + 2) = make_double2(go[2], go[3]);
        *(float4*)(lu_o + p) = make_float4(luo[0], luo[1], luo[2], luo[3]);
        *(float4*)(lv_o + p) = make_float4(lvo[0], lvo[1], lvo[2], lvo[3]);
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
        pr_dev_free(ctx, ctx->adj_ws);
        ctx->adj_ws = nullptr;
        ctx->adj_bytes = 0;
        cudaError_t e = pr_dev_malloc(ctx, &ctx->adj_ws, need);
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
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    // level kernels: one slice, row-wise; FP32 grids with n % 4 == 0 take
    // four points per thread
    const bool quads = sizeof(T) == 4 && n % 4 == 0;
    dim3 lvl_grid, lvl_block;
    rows::shape_for(quads ? n / 4 : n, pts / n, sms > 0 ? sms : 1, &lvl_grid, &lvl_block);
    auto fwd = [&](const T* u, T* v, T* un, int g) {
        if constexpr (sizeof(T) == 4) {
            if (quads) {
                fwd_level_x4<DIM><<<lvl_grid, lvl_block, 0, st>>>(u, v, un, kap, n, pts, w_of(g), dt, g < m);
                return;
            }
        }
        fwd_level<T, DIM><<<lvl_grid, lvl_block, 0, st>>>(u, v, un, kap, n, pts, w_of(g), dt, g < m);
    };
    auto adj = [&](const T* lu, const T* lv, const T* ug, T* lu_o, T* lv_o, int g) {
        if constexpr (sizeof(T) == 4) {
            if (quads) {
                adj_level_x4<DIM><<<lvl_grid, lvl_block, 0, st>>>(lu, lv, ug, kap, lu_o, lv_o, gk, n, pts, w_of(g),
                                                                 dt, g < m);
                return;
            }
        }
        adj_level<T, DIM><<<lvl_grid, lvl_block, 0, st>>>(lu, lv, ug, kap, lu_o, lv_o, gk, n, pts, w_of(g), dt, g < m);
    };

    auto recompute = [&](int s) {   // trace of slice s from its checkpoint; leaves v in vw
        cudaMemcpyAsync(tr, cu + (size_t)s * pts, fb, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(vw, cv + (size_t)s * pts, fb, cudaMemcpyDeviceToDevice, st);
        for (int g = 0; g <= m; ++g)
            fwd(tr + (size_t)g * pts, vw, tr + (size_t)(g + 1 <= m ? g + 1 : g) * pts, g);
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
            adj(la[cur], lb[cur], tr + (size_t)g * pts, la[cur ^ 1], lb[cur ^ 1], g);
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

// Reverse of ONE slice of context c (fine or coarse) from its start state
// (u_in, v_in): recompute the slice's trace, then the m + 1 transposed
// levels, with (lu, lv) the adjoints of the slice's end state on entry and of
// its start state on return; dL/dkappa accumulates into gk (FP64, [pts]).
template <typename T, int DIM>
pr_status slice_adjoint_t(pr_ctx* c, const T* u_in, const T* v_in, T* lu, T* lv, double* gk, cudaStream_t st) {
    const int64_t pts = c->pts, n = c->n;
    const int m = c->m_f;
    const size_t fb = (size_t)pts * sizeof(T);
    // workspace: trace (m+1), v, two adjoint fields
    const size_t need = (size_t)((m + 1) + 1 + 2) * fb;
    if (need > c->sadj_bytes) {
        cudaError_t e = cudaStreamSynchronize(st);   // the old workspace may still be in use
        if (e != cudaSuccess) return pr_cuda_fail(c, e, "slice adjoint: synchronize");
        pr_dev_free(c, c->sadj_ws);
        c->sadj_ws = nullptr;
        c->sadj_bytes = 0;
        e = pr_dev_malloc(c, &c->sadj_ws, need);
        if (e != cudaSuccess) return pr_cuda_fail(c, e, "slice adjoint: workspace");
        c->sadj_bytes = need;
    }
    T* tr = (T*)c->sadj_ws;
    T* vw = tr + (size_t)(m + 1) * pts;
    T* la = vw + pts;
    T* lb = vw + 2 * pts;
    const T* kap = (const T*)c->kappa;
    const T dt = (T)c->dt_f;
    auto w_of = [&](int g) { return (T)((g == 0 || g == m) ? 0.5 : 1.0); };
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const bool quads = sizeof(T) == 4 && n % 4 == 0;
    dim3 grid, block;
    rows::shape_for(quads ? n / 4 : n, pts / n, sms > 0 ? sms : 1, &grid, &block);
    cudaMemcpyAsync(tr, u_in, fb, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(vw, v_in, fb, cudaMemcpyDeviceToDevice, st);
    for (int g = 0; g <= m; ++g) {
        const T* u = tr + (size_t)g * pts;
        T* un = tr + (size_t)(g + 1 <= m ? g + 1 : g) * pts;
        if constexpr (sizeof(T) == 4) {
            if (quads) {
                fwd_level_x4<DIM><<<grid, block, 0, st>>>(u, vw, un, kap, n, pts, w_of(g), dt, g < m);
                continue;
            }
        }
        fwd_level<T, DIM><<<grid, block, 0, st>>>(u, vw, un, kap, n, pts, w_of(g), dt, g < m);
    }
    // reverse: (lu, lv) -> la/lb ping-pong -> back into (lu, lv)
    T* src_u = lu;
    T* src_v = lv;
    for (int g = m; g >= 0; --g) {
        T* du = ((m - g) % 2 == 0) ? la : lu;
        T* dv = ((m - g) % 2 == 0) ? lb : lv;
        const T* ug = tr + (size_t)g * pts;
        if constexpr (sizeof(T) == 4) {
            if (quads) {
                adj_level_x4<DIM><<<grid, block, 0, st>>>(src_u, src_v, ug, kap, du, dv, gk, n, pts, w_of(g), dt, g < m);
                src_u = du;
                src_v = dv;
                continue;
            }
        }
        adj_level<T, DIM><<<grid, block, 0, st>>>(src_u, src_v, ug, kap, du, dv, gk, n, pts, w_of(g), dt, g < m);
        src_u = du;
        src_v = dv;
    }
    if (src_u != lu) {
        cudaMemcpyAsync(lu, src_u, fb, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(lv, src_v, fb, cudaMemcpyDeviceToDevice, st);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pr_cuda_fail(c, e, "slice adjoint: launch");
    return PR_OK;
}

}  // namespace

pr_status pr_slice_adjoint(pr_ctx* c, const void* u_in, const void* v_in, void* lu, void* lv, double* gk,
                           cudaStream_t st) {
    const bool f32 = c->dtype == PR_F32;
    switch (c->dim) {
        case 1: return f32 ? slice_adjoint_t<float, 1>(c, (const float*)u_in, (const float*)v_in, (float*)lu, (float*)lv, gk, st)
                           : slice_adjoint_t<double, 1>(c, (const double*)u_in, (const double*)v_in, (double*)lu, (double*)lv, gk, st);
        case 2: return f32 ? slice_adjoint_t<float, 2>(c, (const float*)u_in, (const float*)v_in, (float*)lu, (float*)lv, gk, st)
                           : slice_adjoint_t<double, 2>(c, (const double*)u_in, (const double*)v_in, (double*)lu, (double*)lv, gk, st);
        default: return f32 ? slice_adjoint_t<float, 3>(c, (const float*)u_in, (const float*)v_in, (float*)lu, (float*)lv, gk, st)
                            : slice_adjoint_t<double, 3>(c, (const double*)u_in, (const double*)v_in, (double*)lu, (double*)lv, gk, st);
    }
}

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
