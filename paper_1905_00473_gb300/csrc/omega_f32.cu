// The Procrustes corrector applied to one vector, g <- X (Y^T d) (Alg. 3's
// serial update; X = Xb WX, Y = Yb WY from Alg. 1), for FP32 contexts: the
// two tall products read single-precision copies of the stored bases Xb, Yb
// (half the bytes of the FP64 arrays; these matrix-vector products are bound
// by HBM), multiply in FP32 and add every eight products into a compensated
// (Kahan) FP32 sum, which reaches FP64 only per thread and in the block
// reductions (FP64 adds per product group held the FP64 pipe at 68 %).
// Each result is FP32-accurate, as the context's state is; a zero d still
// gives exactly zero, so the serial sweep's finite termination (Sec. 3.3)
// is unaffected.  The small products with WX, WY stay FP64.
//
//   t1 = Ys^T d     CTAs over column pairs x kOmR row parts, a block
//                   reduction each; the last CTA of a pair to finish adds
//                   the parts in order (deterministic)
//   out = Xs t2     CTAs over 1024-row blocks x kOmJ column chunks, partial
//                   sums per chunk, then a fixed-order sum (deterministic)
#include <algorithm>
#include <cstdint>

#include "pr_internal.cuh"

namespace {

constexpr int kOmT = 256;

// s + y in compensated FP32 (Kahan): c carries the low-order bits lost so far
__device__ __forceinline__ void kahan_add(float& s, float& c, float y) {
    const float yy = __fsub_rn(y, c);
    const float t = __fadd_rn(s, yy);
    c = __fsub_rn(__fsub_rn(t, s), yy);
    s = t;
}
__device__ __forceinline__ double kahan_value(float s, float c) { return (double)s - (double)c; }

__global__ void om_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t m) {
    for (int64_t i = (int64_t)blockIdx.x * kOmT + threadIdx.x; i < m; i += (int64_t)gridDim.x * kOmT)
        b[i] = (float)a[i];
}

// t1[j] = sum_i Ys[i + j rows] gs[i] for j in {2 b, 2 b + 1} (rows % 4 == 0),
// row part blockIdx.y of kOmR; part: [kOmR][hb] doubles, cnt: hb/2 + 1
// counters (zero on entry, left zero)
__global__ void __launch_bounds__(kOmT) om_gemv_t(const float* __restrict__ Ys, int64_t rows, int hb,
                                                   const float* __restrict__ gs, double* __restrict__ part,
                                                   unsigned* __restrict__ cnt, double* __restrict__ t1) {
    __shared__ double red[2][kOmT];
    __shared__ bool last;
    const int j0 = 2 * blockIdx.x;
    const bool two = j0 + 1 < hb;
    const float4* g4 = (const float4*)gs;
    const float4* a4 = (const float4*)(Ys + (int64_t)j0 * rows);
    const float4* b4 = (const float4*)(Ys + (int64_t)(two ? j0 + 1 : j0) * rows);
    const int64_t q4 = rows / 4;
    const int64_t per = (q4 + kOmR - 1) / kOmR;
    const int64_t qa = blockIdx.y * per, qb = min(q4, qa + per);
    float sa = 0.f, ca = 0.f, sb = 0.f, cb = 0.f;
    int64_t i = qa + threadIdx.x;
#pragma unroll 2
    for (; i + kOmT < qb; i += 2 * kOmT) {   // eight FP32 products, then one compensated add
        const float4 g0 = __ldg(g4 + i), g1 = __ldg(g4 + i + kOmT);
        const float4 x0 = __ldcs(a4 + i), x1 = __ldcs(a4 + i + kOmT);
        const float4 y0 = __ldcs(b4 + i), y1 = __ldcs(b4 + i + kOmT);
        float fa = x0.x * g0.x, fb = y0.x * g0.x;
        fa = fmaf(x0.y, g0.y, fa); fb = fmaf(y0.y, g0.y, fb);
        fa = fmaf(x0.z, g0.z, fa); fb = fmaf(y0.z, g0.z, fb);
        fa = fmaf(x0.w, g0.w, fa); fb = fmaf(y0.w, g0.w, fb);
        fa = fmaf(x1.x, g1.x, fa); fb = fmaf(y1.x, g1.x, fb);
        fa = fmaf(x1.y, g1.y, fa); fb = fmaf(y1.y, g1.y, fb);
        fa = fmaf(x1.z, g1.z, fa); fb = fmaf(y1.z, g1.z, fb);
        fa = fmaf(x1.w, g1.w, fa); fb = fmaf(y1.w, g1.w, fb);
        kahan_add(sa, ca, fa);
        kahan_add(sb, cb, fb);
    }
    for (; i < qb; i += kOmT) {
        const float4 g0 = __ldg(g4 + i), x0 = __ldcs(a4 + i), y0 = __ldcs(b4 + i);
        float fa = x0.x * g0.x, fb = y0.x * g0.x;
        fa = fmaf(x0.y, g0.y, fa); fb = fmaf(y0.y, g0.y, fb);
        fa = fmaf(x0.z, g0.z, fa); fb = fmaf(y0.z, g0.z, fb);
        fa = fmaf(x0.w, g0.w, fa); fb = fmaf(y0.w, g0.w, fb);
        kahan_add(sa, ca, fa);
        kahan_add(sb, cb, fb);
    }
    red[0][threadIdx.x] = kahan_value(sa, ca);
    red[1][threadIdx.x] = kahan_value(sb, cb);
    __syncthreads();
    for (int s = kOmT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[0][threadIdx.x] += red[0][threadIdx.x + s];
            red[1][threadIdx.x] += red[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[(int64_t)blockIdx.y * hb + j0] = red[0][0];
        if (two) part[(int64_t)blockIdx.y * hb + j0 + 1] = red[1][0];
        __threadfence();
        last = atomicAdd(cnt + blockIdx.x, 1u) == kOmR - 1;
    }
    __syncthreads();
    if (last && threadIdx.x < (two ? 2 : 1)) {
        __threadfence();
        double s = 0.0;
        for (int r = 0; r < kOmR; ++r) s += __ldcg(part + (int64_t)r * hb + j0 + threadIdx.x);
        t1[j0 + threadIdx.x] = s;
    }
    if (last && threadIdx.x == 0) cnt[blockIdx.x] = 0u;
}

// part[c][i] = sum_{j in chunk c} Xs[i + j rows] t2[j], four rows per thread
__global__ void __launch_bounds__(kOmT) om_gemv_n(const float* __restrict__ Xs, int64_t rows, int hb,
                                                   const double* __restrict__ t2, int jc, double* __restrict__ part) {
    __shared__ float ts[kOmMaxCols / kOmJ];
    const int c = blockIdx.y;
    const int per = (hb + jc - 1) / jc;
    const int ja = c * per, jb = min(hb, ja + per);
    for (int j = ja + threadIdx.x; j < jb; j += kOmT) ts[j - ja] = (float)t2[j];
    __syncthreads();
    const int64_t i4 = (int64_t)blockIdx.x * kOmT + threadIdx.x;
    if (4 * i4 >= rows) return;
    float s[4] = {0.f, 0.f, 0.f, 0.f}, cmp[4] = {0.f, 0.f, 0.f, 0.f};
    int j = ja;
    for (; j + 8 <= jb; j += 8) {   // eight FP32 products per row, then one compensated add
        float f0 = 0.f, f1 = 0.f, f2 = 0.f, f3 = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float4 x = __ldcs((const float4*)(Xs + (int64_t)(j + k) * rows) + i4);
            const float t = ts[j + k - ja];
            f0 = fmaf(x.x, t, f0);
            f1 = fmaf(x.y, t, f1);
            f2 = fmaf(x.z, t, f2);
            f3 = fmaf(x.w, t, f3);
        }
        kahan_add(s[0], cmp[0], f0);
        kahan_add(s[1], cmp[1], f1);
        kahan_add(s[2], cmp[2], f2);
        kahan_add(s[3], cmp[3], f3);
    }
    for (; j < jb; ++j) {
        const float4 x = __ldcs((const float4*)(Xs + (int64_t)j * rows) + i4);
        const float t = ts[j - ja];
        kahan_add(s[0], cmp[0], x.x * t);
        kahan_add(s[1], cmp[1], x.y * t);
        kahan_add(s[2], cmp[2], x.z * t);
        kahan_add(s[3], cmp[3], x.w * t);
    }
    double* o = part + (int64_t)c * rows + 4 * i4;
#pragma unroll
    for (int e = 0; e < 4; ++e) o[e] = kahan_value(s[e], cmp[e]);
}

// out[i] = sum_c part[c][i], chunks in order
__global__ void om_sum(const double* __restrict__ part, int jc, int64_t rows, double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * kOmT + threadIdx.x; i < rows; i += (int64_t)gridDim.x * kOmT) {
        double s = 0.0;
        for (int c = 0; c < jc; ++c) s += part[(int64_t)c * rows + i];
        out[i] = s;
    }
}

int om_blocks(int64_t m) { return (int)std::max<int64_t>(1, std::min<int64_t>((m + kOmT - 1) / kOmT, 152 * 16)); }

}  // namespace

pr_status omega_f32_supported(int64_t rows, int hb) { return (rows % 4 == 0 && hb <= kOmMaxCols) ? PR_OK : PR_EINVAL; }

void omega_to_f32(const double* a, float* b, int64_t m, cudaStream_t st) {
    om_to_f32<<<om_blocks(m), kOmT, 0, st>>>(a, b, m);
}

void omega_gemv_t_f32(const float* Ys, int64_t rows, int hb, const double* g, float* gs, double* part,
                      unsigned* cnt, double* t1, cudaStream_t st) {
    om_to_f32<<<om_blocks(rows), kOmT, 0, st>>>(g, gs, rows);
    om_gemv_t<<<dim3((unsigned)((hb + 1) / 2), kOmR), kOmT, 0, st>>>(Ys, rows, hb, gs, part, cnt, t1);
}

void omega_gemv_n_f32(const float* Xs, int64_t rows, int hb, const double* t2, double* part, double* out,
                      cudaStream_t st) {
    const dim3 grid((unsigned)((rows / 4 + kOmT - 1) / kOmT), kOmJ);
    om_gemv_n<<<grid, kOmT, 0, st>>>(Xs, rows, hb, t2, kOmJ, part);
    om_sum<<<om_blocks(rows), kOmT, 0, st>>>(part, kOmJ, rows, out);
}
