// The proposed method around the fine sweep (Alg. 3): coarse sweep C R over
// all slices, the energy maps Lambda / Lambda^dagger (Sec. 3.4, Alg. 2),
// Fourier interpolation I (interpft, Sec. 6), the Procrustes corrector and
// its incremental SVD (Sec. 3.3, Alg. 1), and the driver pr_iterate.
//
// Precision: propagators run in the context dtype; everything on the
// correction path (Lambda, Omega, Lambda^dagger, I and the data matrices) is
// FP64, as is the SVD.  Library calls: cuFFT (double complex transforms),
// cuBLAS (plain FP64 GEMM/GEMV) and cuSOLVER (FP64 QR and SVD of small or
// tall-skinny matrices); every other step is a kernel of this file.
#include <cublas_v2.h>
#include <cufft.h>
#include <cusolverDn.h>
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pr_internal.cuh"

namespace {

constexpr int kT = 256;

// ---------------------------------------------------------------- indexing
template <int DIM>
__device__ __forceinline__ void coords(int64_t j, int64_t n, int64_t* c) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        c[a] = j % n;
        j /= n;
    }
}
template <int DIM>
__device__ __forceinline__ int64_t lin(const int64_t* c, int64_t n) {
    int64_t j = 0;
#pragma unroll
    for (int a = DIM - 1; a >= 0; --a) j = j * n + c[a];
    return j;
}

// signed FFT frequency of index i on an n-point axis (numpy fftfreq: the
// Nyquist index of an even axis is -n/2)
__device__ __forceinline__ int64_t freq(int64_t i, int64_t n) { return (2 * i < n) ? i : i - n; }

// ---------------------------------------------------------------- R
// Injection onto the coarse nodes (Sec. 6): coarse J <- fine ratio*J.
template <typename T, int DIM>
__global__ void restrict_kernel(const T* __restrict__ u, const T* __restrict__ v, T* __restrict__ U,
                                T* __restrict__ V, int64_t n, int ratio, int64_t pts, int64_t cpts,
                                int64_t total) {
    const int64_t nc = n / ratio;
    for (int64_t idx = (int64_t)blockIdx.x * kT + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * kT) {
        const int64_t s = idx / cpts, J = idx - s * cpts;
        int64_t c[3];
        coords<DIM>(J, nc, c);
#pragma unroll
        for (int a = 0; a < DIM; ++a) c[a] *= ratio;
        const int64_t f = s * pts + lin<DIM>(c, n);
        U[idx] = u[f];
        V[idx] = v[f];
    }
}

// ---------------------------------------------------------------- Lambda
// out[a*cpts + J] (a < DIM) = nabla_h W along axis a at coarse node J, and
// out[DIM*cpts + J] = W_t / c; W is sampled at coarse nodes of an array with
// `stride`-spaced nodes (stride = ratio reads R u straight from a fine array,
// stride = 1 a coarse array).  sign = +1 writes, -1 subtracts (Lambda w - Lambda U).
__constant__ double c_beta[4];

template <typename T, int DIM>
__global__ void lambda_kernel(const T* __restrict__ w, const T* __restrict__ wt,
                              const double* __restrict__ cc, double* __restrict__ out,
                              int64_t nc, int stride, int64_t arr_n, int64_t arr_pts, int64_t cpts,
                              int order_half, double inv_dx, double sign, int nslices,
                              int64_t out_ld) {
    const int64_t total = (int64_t)nslices * cpts;
    for (int64_t idx = (int64_t)blockIdx.x * kT + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * kT) {
        const int64_t s = idx / cpts, J = idx - s * cpts;
        const T* ws = w + s * arr_pts;
        const T* wts = wt + s * arr_pts;
        double* o = out + s * out_ld;
        int64_t c[3];
        coords<DIM>(J, nc, c);
        int64_t f[3];
#pragma unroll
        for (int a = 0; a < DIM; ++a) f[a] = c[a] * stride;
        const int64_t base = lin<DIM>(f, arr_n);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            double acc = 0.0;
            int64_t astride = 1;
            for (int b = 0; b < a; ++b) astride *= arr_n;
            for (int k = 1; k <= order_half; ++k) {
                const int64_t cp = (c[a] + k) % nc, cm = (c[a] - k + nc) % nc;
                const double up = (double)ws[base + (cp * stride - f[a]) * astride];
                const double um = (double)ws[base + (cm * stride - f[a]) * astride];
                acc += c_beta[k - 1] * (up - um);
            }
            const double g = acc * inv_dx;
            if (sign > 0) o[a * cpts + J] = g;
            else o[a * cpts + J] -= g;
        }
        const double m = (double)wts[base] / cc[J];
        if (sign > 0) o[DIM * cpts + J] = m;
        else o[DIM * cpts + J] -= m;
    }
}

// zero mode of grad2func for the difference: sum_J (w_J - U_J) (one block, fixed order)
template <typename T>
__global__ void zero_mode_kernel(const T* __restrict__ w, const T* __restrict__ U, int64_t cpts,
                                 double* __restrict__ out) {
    __shared__ double red[1024];
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < cpts; j += blockDim.x) acc += (double)w[j] - (U ? (double)U[j] : 0.0);
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// ---------------------------------------------------------------- Lambda^dagger (grad2func)
__global__ void real_to_complex(const double* __restrict__ x, cufftDoubleComplex* __restrict__ z, int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x; j < m; j += (int64_t)gridDim.x * kT)
        z[j] = make_cuDoubleComplex(x[j], 0.0);
}

// w^(xi) = -i (xi . q^) / |xi|^2, w^(0) = zero mode (Alg. 2), in place into z[0..cpts)
template <int DIM>
__global__ void grad2func_combine(cufftDoubleComplex* __restrict__ z, int64_t nc, int64_t cpts,
                                  const double* __restrict__ zero_mode) {
    for (int64_t J = (int64_t)blockIdx.x * kT + threadIdx.x; J < cpts; J += (int64_t)gridDim.x * kT) {
        int64_t c[3];
        coords<DIM>(J, nc, c);
        double re = 0.0, im = 0.0, mag2 = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const double xi = 2.0 * M_PI * (double)freq(c[a], nc);
            const cufftDoubleComplex q = z[a * cpts + J];
            re += xi * q.x;
            im += xi * q.y;
            mag2 += xi * xi;
        }
        // -i (re + i im) = im - i re
        z[J] = mag2 > 0 ? make_cuDoubleComplex(im / mag2, -re / mag2) : make_cuDoubleComplex(*zero_mode, 0.0);
    }
}

// du = real(ifft(.)) (unnormalised inverse, so / cpts) and du_t = c p
__global__ void grad2func_finish(const cufftDoubleComplex* __restrict__ z, const double* __restrict__ p,
                                 const double* __restrict__ cc, double* __restrict__ du,
                                 double* __restrict__ dut, int64_t cpts) {
    const double inv = 1.0 / (double)cpts;
    for (int64_t J = (int64_t)blockIdx.x * kT + threadIdx.x; J < cpts; J += (int64_t)gridDim.x * kT) {
        du[J] = z[J].x * inv;
        dut[J] = cc[J] * p[J];
    }
}

// ---------------------------------------------------------------- I (interpft)
// fine spectrum from the coarse one: per axis, |m| < nc/2 copies, the coarse
// Nyquist coefficient goes half to +nc/2 and half to -nc/2 (both halves land
// on the same index when nf == nc); scaled by 1/cpts for the unnormalised
// inverse transform.  Two fields (u, u_t) one after the other.
template <int DIM>
__global__ void interp_pad(const cufftDoubleComplex* __restrict__ cs, cufftDoubleComplex* __restrict__ fs,
                           int64_t nc, int64_t nf, int64_t cpts, int64_t fpts) {
    const double scale = 1.0 / (double)cpts;
    for (int64_t idx = (int64_t)blockIdx.x * kT + threadIdx.x; idx < 2 * fpts; idx += (int64_t)gridDim.x * kT) {
        const int64_t fld = idx / fpts, jf = idx - fld * fpts;
        int64_t c[3];
        coords<DIM>(jf, nf, c);
        double wgt = scale;
        int64_t src[3];
        const int64_t half = nc / 2;
        bool zero = false;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const int64_t i = c[a];
            double wa = 0.0;
            int64_t sa = 0;
            if (nc % 2 == 0) {
                if (i < half) { wa = 1.0; sa = i; }
                else if (i > nf - half) { wa = 1.0; sa = i - nf + nc; }
                else {
                    if (i == half) { wa += 0.5; sa = half; }
                    if (i == nf - half) { wa += 0.5; sa = half; }
                }
            } else {
                if (i <= half) { wa = 1.0; sa = i; }
                else if (i >= nf - half) { wa = 1.0; sa = i - nf + nc; }
            }
            if (wa == 0.0) zero = true;
            wgt *= wa;
            src[a] = sa;
        }
        cufftDoubleComplex o = make_cuDoubleComplex(0.0, 0.0);
        if (!zero) {
            const cufftDoubleComplex x = cs[fld * cpts + lin<DIM>(src, nc)];
            o = make_cuDoubleComplex(x.x * wgt, x.y * wgt);
        }
        fs[idx] = o;
    }
}

// out = base + real(fine field) for both fields (base may alias out)
template <typename T>
__global__ void interp_add(const cufftDoubleComplex* __restrict__ fs, const T* bu, const T* bv, T* ou,
                           T* ov, int64_t fpts) {
    for (int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x; j < fpts; j += (int64_t)gridDim.x * kT) {
        const double a = fs[j].x, b = fs[fpts + j].x;
        ou[j] = (T)((bu ? (double)bu[j] : 0.0) + a);
        ov[j] = (T)((bv ? (double)bv[j] : 0.0) + b);
    }
}

template <typename T>
__global__ void to_double2(const T* __restrict__ a, const T* __restrict__ b, const T* __restrict__ sa,
                           const T* __restrict__ sb, cufftDoubleComplex* __restrict__ z, int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x; j < m; j += (int64_t)gridDim.x * kT) {
        z[j] = make_cuDoubleComplex((double)a[j] - (sa ? (double)sa[j] : 0.0), 0.0);
        z[m + j] = make_cuDoubleComplex((double)b[j] - (sb ? (double)sb[j] : 0.0), 0.0);
    }
}

__global__ void pair_to_complex(const double* __restrict__ a, const double* __restrict__ b,
                                cufftDoubleComplex* __restrict__ z, int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x; j < m; j += (int64_t)gridDim.x * kT) {
        z[j] = make_cuDoubleComplex(a[j], 0.0);
        z[m + j] = make_cuDoubleComplex(b[j], 0.0);
    }
}

template <typename T>
__global__ void diff_kernel(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ o, int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x; j < m; j += (int64_t)gridDim.x * kT)
        o[j] = (T)((double)a[j] - (double)b[j]);
}

// ---------------------------------------------------------------- small dense helpers
// R (n x n, upper) from a geqrf result (m x n, lda = m), zero below the diagonal
__global__ void extract_r(const double* __restrict__ A, double* __restrict__ R, int64_t m, int n) {
    for (int64_t idx = (int64_t)blockIdx.x * kT + threadIdx.x; idx < (int64_t)n * n; idx += (int64_t)gridDim.x * kT) {
        const int col = (int)(idx / n), row = (int)(idx - (int64_t)col * n);
        R[idx] = row <= col ? A[(int64_t)col * m + row] : 0.0;
    }
}
// copy rows [0, r) x cols [0, c) of A (lda) into B (ldb) at row offset ro
__global__ void copy_block(const double* __restrict__ A, int64_t lda, double* __restrict__ B, int64_t ldb,
                           int rows, int cols, int ro) {
    for (int64_t idx = (int64_t)blockIdx.x * kT + threadIdx.x; idx < (int64_t)rows * cols; idx += (int64_t)gridDim.x * kT) {
        const int col = (int)(idx / rows), row = (int)(idx - (int64_t)col * rows);
        B[(int64_t)col * ldb + ro + row] = A[(int64_t)col * lda + row];
    }
}
// B(ro + i, j) = A(j, i) for i < rows, j < cols (A with leading dimension lda)
__global__ void copy_block_t(const double* __restrict__ A, int64_t lda, double* __restrict__ B, int64_t ldb,
                             int rows, int cols, int ro) {
    for (int64_t idx = (int64_t)blockIdx.x * kT + threadIdx.x; idx < (int64_t)rows * cols; idx += (int64_t)gridDim.x * kT) {
        const int col = (int)(idx / rows), row = (int)(idx - (int64_t)col * rows);
        B[(int64_t)col * ldb + ro + row] = A[(int64_t)row * lda + col];
    }
}
__global__ void add_diag(double* __restrict__ H, int64_t ld, const double* __restrict__ S, int s) {
    for (int i = blockIdx.x * kT + threadIdx.x; i < s; i += gridDim.x * kT) H[(int64_t)i * ld + i] += S[i];
}

int blocks_for(int64_t m) {
    int64_t b = (m + kT - 1) / kT;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

}  // namespace

// ---------------------------------------------------------------- driver state
struct pr_driver {
    int dim = 0;
    int64_t n = 0, nc = 0, pts = 0, cpts = 0, rows = 0;   // rows = (d+1) cpts
    int N = 0;
    cufftHandle plan_c1 = 0, plan_cd = 0, plan_c2 = 0, plan_f2 = 0;
    bool have_plans = false;
    cublasHandle_t blas = nullptr;
    cusolverDnHandle_t sol = nullptr;
    // dtype buffers
    void* vF_u = nullptr; void* vF_v = nullptr;     // F u^k_{n-1}   [N][pts]
    void* Uc_u = nullptr; void* Uc_v = nullptr;     // C R u^k_{n-1} [N][cpts]
    void* w_u = nullptr; void* w_v = nullptr;       // serial-sweep coarse state [cpts]
    // FP64 buffers
    double* Fm = nullptr; double* Gm = nullptr;     // data matrices [rows][N], column-major
    double* dvec = nullptr; double* gvec = nullptr; // [rows]
    double* du = nullptr; double* dut = nullptr;    // coarse correction [cpts] each
    double* zero = nullptr;                         // device scalar
    cufftDoubleComplex* zc = nullptr;               // [max(d,2) * cpts]
    cufftDoubleComplex* zf = nullptr;               // [2 * pts]
    // SVD state of Alg. 1, kept factored: X = Xb WX, Y = Yb WY.  Xb, Yb
    // [rows][bcap] hold every orthonormalised block Q_F, Q_G appended so far
    // (hb columns); WX, WY [bcap][bcap] (hb x s in use) map them onto the s
    // kept singular directions, so an update rotates only WX, WY.
    double *Xb = nullptr, *Yb = nullptr, *WX = nullptr, *WY = nullptr, *WXn = nullptr, *WYn = nullptr;
    double *Tb = nullptr, *vb = nullptr;   // [bcap][N] and [2 bcap] scratch
    double* S = nullptr;                   // [bcap]
    int s = 0, hb = 0, bcap = 0;
    // UpdateSVD scratch
    double *QF = nullptr, *QG = nullptr, *RF = nullptr, *RG = nullptr, *tau = nullptr;
    double *UF = nullptr, *VG = nullptr, *A1 = nullptr, *A2 = nullptr, *H = nullptr;
    double *Xh = nullptr, *YhT = nullptr, *sig = nullptr, *work = nullptr, *rwork = nullptr;
    double *F2 = nullptr, *G2 = nullptr;            // copies of F, G for the residual
    int* info = nullptr;
    int64_t work_len = 0;
    int hcap = 0;   // allocated (s+N) capacity of the small matrices
    // phase timers of the last pr_iterate (Sec. 7.2.4 table columns): initial
    // coarse sweep, parallel computation, creating the corrector, serial update
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    double phase_ms[4] = {0.0, 0.0, 0.0, 0.0};
};

void pr_driver_free(pr_ctx* ctx) {
    pr_driver* d = ctx->drv;
    if (!d) return;
    if (d->have_plans) {
        cufftDestroy(d->plan_c1);
        cufftDestroy(d->plan_cd);
        cufftDestroy(d->plan_c2);
        cufftDestroy(d->plan_f2);
    }
    if (d->blas) cublasDestroy(d->blas);
    if (d->sol) cusolverDnDestroy(d->sol);
    for (cudaEvent_t e : d->ev)
        if (e) cudaEventDestroy(e);
    void* bufs[] = {d->vF_u, d->vF_v, d->Uc_u, d->Uc_v, d->w_u, d->w_v, d->Fm, d->Gm, d->dvec, d->gvec,
                    d->du, d->dut, d->zero, d->zc, d->zf, d->Xb, d->Yb, d->WX, d->WY, d->WXn, d->WYn,
                    d->Tb, d->vb, d->S, d->QF, d->QG, d->RF, d->RG, d->tau, d->UF, d->VG, d->A1, d->A2,
                    d->H, d->Xh, d->YhT, d->sig, d->work, d->rwork, d->F2, d->G2, d->info};
    for (void* b : bufs) cudaFree(b);
    delete d;
    ctx->drv = nullptr;
}

namespace {

pr_status cufft_fail(pr_ctx* ctx, cufftResult r, const char* what) {
    char buf[160];
    snprintf(buf, sizeof buf, "%s: cuFFT error %d", what, (int)r);
    return pr_fail(ctx, PR_ECUDA, buf);
}
pr_status blas_fail(pr_ctx* ctx, int r, const char* what) {
    char buf[160];
    snprintf(buf, sizeof buf, "%s: library status %d", what, r);
    return pr_fail(ctx, PR_ECUDA, buf);
}
#define PR_TRY_ST(x) do { pr_status s_ = (x); if (s_ != PR_OK) return s_; } while (0)
#define PR_FFT(ctx, x, what) do { cufftResult r_ = (x); if (r_ != CUFFT_SUCCESS) return cufft_fail(ctx, r_, what); } while (0)
#define PR_BLAS(ctx, x, what) do { int r_ = (int)(x); if (r_ != 0) return blas_fail(ctx, r_, what); } while (0)

pr_status alloc(pr_ctx* ctx, void** p, size_t bytes, const char* what) {
    cudaError_t e = cudaMalloc(p, bytes > 0 ? bytes : 16);
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, what);
    return PR_OK;
}

pr_status driver(pr_ctx* ctx, cudaStream_t st, pr_driver** out) {
    if (!ctx->coarse) return pr_fail(ctx, PR_EINVAL, "driver: context has no coarse grid");
    if (ctx->opts.grad_order != 2 && ctx->opts.grad_order != 4 && ctx->opts.grad_order != 6 &&
        ctx->opts.grad_order != 8)
        return pr_fail(ctx, PR_EINVAL, "driver: the GPU correction path supports grad_order 2, 4, 6, 8");
    if (!ctx->drv) {
        pr_driver* d = new pr_driver();
        ctx->drv = d;
        d->dim = ctx->dim;
        d->n = ctx->n;
        d->nc = ctx->coarse->n;
        d->pts = ctx->pts;
        d->cpts = ctx->coarse->pts;
        d->rows = (int64_t)(ctx->dim + 1) * d->cpts;
        d->N = ctx->N;
        const size_t esz = ctx->dtype == PR_F32 ? 4 : 8;
        PR_TRY_ST(alloc(ctx, &d->vF_u, (size_t)d->N * d->pts * esz, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, &d->vF_v, (size_t)d->N * d->pts * esz, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, &d->Uc_u, (size_t)d->N * d->cpts * esz, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, &d->Uc_v, (size_t)d->N * d->cpts * esz, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, &d->w_u, (size_t)d->cpts * esz, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, &d->w_v, (size_t)d->cpts * esz, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->Fm, (size_t)d->rows * d->N * 8, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->Gm, (size_t)d->rows * d->N * 8, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->dvec, (size_t)d->rows * 8, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->gvec, (size_t)d->rows * 8, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->du, (size_t)d->cpts * 8, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->dut, (size_t)d->cpts * 8, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->zero, 8, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->zc, (size_t)std::max(d->dim, 2) * d->cpts * 16, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->zf, (size_t)2 * d->pts * 16, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->info, sizeof(int), "driver: alloc"));
        int nn[3], nf[3];
        for (int a = 0; a < d->dim; ++a) {
            nn[a] = (int)d->nc;
            nf[a] = (int)d->n;
        }
        PR_FFT(ctx, cufftPlanMany(&d->plan_c1, d->dim, nn, nullptr, 1, (int)d->cpts, nullptr, 1, (int)d->cpts, CUFFT_Z2Z, 1), "plan");
        PR_FFT(ctx, cufftPlanMany(&d->plan_cd, d->dim, nn, nullptr, 1, (int)d->cpts, nullptr, 1, (int)d->cpts, CUFFT_Z2Z, d->dim), "plan");
        PR_FFT(ctx, cufftPlanMany(&d->plan_c2, d->dim, nn, nullptr, 1, (int)d->cpts, nullptr, 1, (int)d->cpts, CUFFT_Z2Z, 2), "plan");
        PR_FFT(ctx, cufftPlanMany(&d->plan_f2, d->dim, nf, nullptr, 1, (int)d->pts, nullptr, 1, (int)d->pts, CUFFT_Z2Z, 2), "plan");
        d->have_plans = true;
        PR_BLAS(ctx, cublasCreate(&d->blas), "cublasCreate");
        PR_BLAS(ctx, cusolverDnCreate(&d->sol), "cusolverDnCreate");
        // central first-derivative weights of order 2*h (Sec. 3.4 beta_j form)
        double beta[4] = {0, 0, 0, 0};
        switch (ctx->opts.grad_order) {
            case 2: beta[0] = 0.5; break;
            case 4: beta[0] = 2.0 / 3.0; beta[1] = -1.0 / 12.0; break;
            case 6: beta[0] = 0.75; beta[1] = -0.15; beta[2] = 1.0 / 60.0; break;
            default: beta[0] = 0.8; beta[1] = -0.2; beta[2] = 4.0 / 105.0; beta[3] = -1.0 / 280.0; break;
        }
        cudaError_t e = cudaMemcpyToSymbol(c_beta, beta, sizeof beta);
        if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "driver: upload beta");
    }
    pr_driver* d = ctx->drv;
    PR_FFT(ctx, cufftSetStream(d->plan_c1, st), "set stream");
    PR_FFT(ctx, cufftSetStream(d->plan_cd, st), "set stream");
    PR_FFT(ctx, cufftSetStream(d->plan_c2, st), "set stream");
    PR_FFT(ctx, cufftSetStream(d->plan_f2, st), "set stream");
    PR_BLAS(ctx, cublasSetStream(d->blas, st), "cublasSetStream");
    PR_BLAS(ctx, cusolverDnSetStream(d->sol, st), "cusolverDnSetStream");
    *out = d;
    return PR_OK;
}

// ---- typed launch helpers ----------------------------------------------------
template <typename T>
pr_status launch_restrict(pr_ctx* ctx, const void* u, const void* v, void* U, void* V, int ns, cudaStream_t st) {
    const int64_t cpts = ctx->coarse->pts, total = (int64_t)ns * cpts;
    switch (ctx->dim) {
        case 1: restrict_kernel<T, 1><<<blocks_for(total), kT, 0, st>>>((const T*)u, (const T*)v, (T*)U, (T*)V, ctx->n, ctx->ratio, ctx->pts, cpts, total); break;
        case 2: restrict_kernel<T, 2><<<blocks_for(total), kT, 0, st>>>((const T*)u, (const T*)v, (T*)U, (T*)V, ctx->n, ctx->ratio, ctx->pts, cpts, total); break;
        default: restrict_kernel<T, 3><<<blocks_for(total), kT, 0, st>>>((const T*)u, (const T*)v, (T*)U, (T*)V, ctx->n, ctx->ratio, ctx->pts, cpts, total); break;
    }
    return PR_OK;
}
pr_status restrict_(pr_ctx* ctx, const void* u, const void* v, void* U, void* V, int ns, cudaStream_t st) {
    return ctx->dtype == PR_F32 ? launch_restrict<float>(ctx, u, v, U, V, ns, st)
                                : launch_restrict<double>(ctx, u, v, U, V, ns, st);
}

// Lambda of `ns` slices into columns of `out` (leading dimension out_ld);
// stride 1: coarse arrays, stride ratio: fine arrays read at coarse nodes
template <typename T>
void launch_lambda_t(pr_ctx* ctx, const void* w, const void* wt, double* out, int stride, int64_t arr_n,
                     int64_t arr_pts, double sign, int ns, int64_t out_ld, cudaStream_t st) {
    const int64_t nc = ctx->coarse->n, cpts = ctx->coarse->pts, total = (int64_t)ns * cpts;
    const int h = ctx->opts.grad_order / 2;
    const double inv_dx = 1.0 / ctx->coarse->dx;
    switch (ctx->dim) {
        case 1: lambda_kernel<T, 1><<<blocks_for(total), kT, 0, st>>>((const T*)w, (const T*)wt, ctx->coarse->c64, out, nc, stride, arr_n, arr_pts, cpts, h, inv_dx, sign, ns, out_ld); break;
        case 2: lambda_kernel<T, 2><<<blocks_for(total), kT, 0, st>>>((const T*)w, (const T*)wt, ctx->coarse->c64, out, nc, stride, arr_n, arr_pts, cpts, h, inv_dx, sign, ns, out_ld); break;
        default: lambda_kernel<T, 3><<<blocks_for(total), kT, 0, st>>>((const T*)w, (const T*)wt, ctx->coarse->c64, out, nc, stride, arr_n, arr_pts, cpts, h, inv_dx, sign, ns, out_ld); break;
    }
}
void lambda_(pr_ctx* ctx, const void* w, const void* wt, double* out, int stride, int64_t arr_n,
             int64_t arr_pts, double sign, int ns, int64_t out_ld, cudaStream_t st) {
    if (ctx->dtype == PR_F32) launch_lambda_t<float>(ctx, w, wt, out, stride, arr_n, arr_pts, sign, ns, out_ld, st);
    else launch_lambda_t<double>(ctx, w, wt, out, stride, arr_n, arr_pts, sign, ns, out_ld, st);
}

// Lambda^dagger of gvec (rows) with zero mode *zero -> (du, dut) on the coarse grid
pr_status reconstruct_(pr_ctx* ctx, pr_driver* d, const double* g, cudaStream_t st) {
    const int64_t cpts = d->cpts;
    real_to_complex<<<blocks_for(d->dim * cpts), kT, 0, st>>>(g, d->zc, d->dim * cpts);
    PR_FFT(ctx, cufftExecZ2Z(d->plan_cd, d->zc, d->zc, CUFFT_FORWARD), "grad2func forward");
    switch (d->dim) {
        case 1: grad2func_combine<1><<<blocks_for(cpts), kT, 0, st>>>(d->zc, d->nc, cpts, d->zero); break;
        case 2: grad2func_combine<2><<<blocks_for(cpts), kT, 0, st>>>(d->zc, d->nc, cpts, d->zero); break;
        default: grad2func_combine<3><<<blocks_for(cpts), kT, 0, st>>>(d->zc, d->nc, cpts, d->zero); break;
    }
    PR_FFT(ctx, cufftExecZ2Z(d->plan_c1, d->zc, d->zc, CUFFT_INVERSE), "grad2func inverse");
    grad2func_finish<<<blocks_for(cpts), kT, 0, st>>>(d->zc, g + (int64_t)d->dim * cpts, ctx->coarse->c64,
                                                      d->du, d->dut, cpts);
    return PR_OK;
}

// fine (u, v) = base + I(coarse fields in zc[0..2*cpts)) ; zc must hold the
// two coarse fields as complex
template <typename T>
pr_status interp_t(pr_ctx* ctx, pr_driver* d, const void* bu, const void* bv, void* ou, void* ov, cudaStream_t st) {
    PR_FFT(ctx, cufftExecZ2Z(d->plan_c2, d->zc, d->zc, CUFFT_FORWARD), "interp forward");
    switch (d->dim) {
        case 1: interp_pad<1><<<blocks_for(2 * d->pts), kT, 0, st>>>(d->zc, d->zf, d->nc, d->n, d->cpts, d->pts); break;
        case 2: interp_pad<2><<<blocks_for(2 * d->pts), kT, 0, st>>>(d->zc, d->zf, d->nc, d->n, d->cpts, d->pts); break;
        default: interp_pad<3><<<blocks_for(2 * d->pts), kT, 0, st>>>(d->zc, d->zf, d->nc, d->n, d->cpts, d->pts); break;
    }
    PR_FFT(ctx, cufftExecZ2Z(d->plan_f2, d->zf, d->zf, CUFFT_INVERSE), "interp inverse");
    interp_add<T><<<blocks_for(d->pts), kT, 0, st>>>(d->zf, (const T*)bu, (const T*)bv, (T*)ou, (T*)ov, d->pts);
    return PR_OK;
}
pr_status interp_(pr_ctx* ctx, pr_driver* d, const void* bu, const void* bv, void* ou, void* ov, cudaStream_t st) {
    return ctx->dtype == PR_F32 ? interp_t<float>(ctx, d, bu, bv, ou, ov, st) : interp_t<double>(ctx, d, bu, bv, ou, ov, st);
}

// zc <- (a - sa, b - sb) for coarse dtype fields (sa/sb may be null)
void coarse_to_zc(pr_ctx* ctx, pr_driver* d, const void* a, const void* b, const void* sa, const void* sb, cudaStream_t st) {
    if (ctx->dtype == PR_F32)
        to_double2<float><<<blocks_for(d->cpts), kT, 0, st>>>((const float*)a, (const float*)b, (const float*)sa, (const float*)sb, d->zc, d->cpts);
    else
        to_double2<double><<<blocks_for(d->cpts), kT, 0, st>>>((const double*)a, (const double*)b, (const double*)sa, (const double*)sb, d->zc, d->cpts);
}

void zero_mode_(pr_ctx* ctx, pr_driver* d, const void* w, const void* U, cudaStream_t st) {
    if (ctx->dtype == PR_F32) zero_mode_kernel<float><<<1, 1024, 0, st>>>((const float*)w, (const float*)U, d->cpts, d->zero);
    else zero_mode_kernel<double><<<1, 1024, 0, st>>>((const double*)w, (const double*)U, d->cpts, d->zero);
}

// C R of ns fine slices into coarse arrays (in place on the outputs)
pr_status coarse_of(pr_ctx* ctx, const void* u, const void* v, void* U, void* V, int ns, cudaStream_t st) {
    PR_TRY_ST(restrict_(ctx, u, v, U, V, ns, st));
    pr_status s = pr_fine_all_slices(ctx->coarse, U, V, U, V, 0, ns, st);
    if (s != PR_OK) return pr_fail(ctx, s, std::string("coarse propagator: ") + pr_last_error(ctx->coarse));
    return PR_OK;
}

// ---------------------------------------------------------------- UpdateSVD (Alg. 1)
pr_status ensure_capacity(pr_ctx* ctx, pr_driver* d, int need_s, int ncols, cudaStream_t st) {
    const int64_t rows = d->rows;
    const int need_b = d->hb + ncols;   // stored columns after this update
    if (need_b > d->bcap || need_s > d->hcap) {
        cudaError_t e = cudaStreamSynchronize(st);   // buffers below are still in use by st
        if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "svd: synchronize");
    }
    if (need_b > d->bcap) {
        const int bc = std::max(need_b, d->bcap * 2);
        double *Xb = nullptr, *Yb = nullptr, *WX = nullptr, *WY = nullptr, *WXn = nullptr, *WYn = nullptr;
        double *Tb = nullptr, *vb = nullptr, *S = nullptr;
        PR_TRY_ST(alloc(ctx, (void**)&Xb, (size_t)rows * bc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&Yb, (size_t)rows * bc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&WX, (size_t)bc * bc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&WY, (size_t)bc * bc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&WXn, (size_t)bc * bc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&WYn, (size_t)bc * bc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&Tb, (size_t)bc * d->N * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&vb, (size_t)2 * bc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&S, (size_t)bc * 8, "svd: alloc"));
        if (d->s > 0) {
            cudaMemcpy(Xb, d->Xb, (size_t)rows * d->hb * 8, cudaMemcpyDeviceToDevice);
            cudaMemcpy(Yb, d->Yb, (size_t)rows * d->hb * 8, cudaMemcpyDeviceToDevice);
            // hb x s blocks, leading dimension bcap -> bc
            cudaMemcpy2D(WX, (size_t)bc * 8, d->WX, (size_t)d->bcap * 8, (size_t)d->hb * 8, d->s,
                         cudaMemcpyDeviceToDevice);
            cudaMemcpy2D(WY, (size_t)bc * 8, d->WY, (size_t)d->bcap * 8, (size_t)d->hb * 8, d->s,
                         cudaMemcpyDeviceToDevice);
            cudaMemcpy(S, d->S, (size_t)d->s * 8, cudaMemcpyDeviceToDevice);
        }
        double** olds[] = {&d->Xb, &d->Yb, &d->WX, &d->WY, &d->WXn, &d->WYn, &d->Tb, &d->vb, &d->S};
        for (double** o : olds) cudaFree(*o);
        d->Xb = Xb; d->Yb = Yb; d->WX = WX; d->WY = WY; d->WXn = WXn; d->WYn = WYn;
        d->Tb = Tb; d->vb = vb; d->S = S;
        d->bcap = bc;
    }
    const int h = need_s;   // (s + ncols)
    if (h > d->hcap || !d->QF) {
        const int hc = std::max(h, d->hcap * 2);
        double** smalls[] = {&d->RF, &d->RG, &d->UF, &d->VG, &d->A1, &d->A2, &d->H, &d->Xh, &d->YhT};
        for (double** p : smalls) {
            cudaFree(*p);
            *p = nullptr;
        }
        cudaFree(d->sig); cudaFree(d->tau); cudaFree(d->QF); cudaFree(d->QG); cudaFree(d->rwork);
        PR_TRY_ST(alloc(ctx, (void**)&d->RF, (size_t)ncols * ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->RG, (size_t)ncols * ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->UF, (size_t)hc * ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->VG, (size_t)hc * ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->A1, (size_t)hc * ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->A2, (size_t)hc * ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->H, (size_t)hc * hc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->Xh, (size_t)hc * hc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->YhT, (size_t)hc * hc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->sig, (size_t)hc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->rwork, (size_t)hc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->tau, (size_t)ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->QF, (size_t)rows * ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->QG, (size_t)rows * ncols * 8, "svd: alloc"));
        d->hcap = hc;
    }
    return PR_OK;
}

pr_status ensure_work(pr_ctx* ctx, pr_driver* d, int64_t need) {
    if (need > d->work_len) {
        cudaFree(d->work);
        d->work = nullptr;
        PR_TRY_ST(alloc(ctx, (void**)&d->work, (size_t)need * 8, "svd: alloc work"));
        d->work_len = need;
    }
    return PR_OK;
}

// reduced QR of A (rows x nc, overwritten): Q in A, R (nc x nc) in Rout
pr_status qr_(pr_ctx* ctx, pr_driver* d, double* A, double* Rout, int nc, cudaStream_t st) {
    const int m = (int)d->rows;
    int l1 = 0, l2 = 0;
    PR_BLAS(ctx, cusolverDnDgeqrf_bufferSize(d->sol, m, nc, A, m, &l1), "geqrf size");
    PR_BLAS(ctx, cusolverDnDorgqr_bufferSize(d->sol, m, nc, nc, A, m, d->tau, &l2), "orgqr size");
    PR_TRY_ST(ensure_work(ctx, d, std::max(l1, l2)));
    PR_BLAS(ctx, cusolverDnDgeqrf(d->sol, m, nc, A, m, d->tau, d->work, (int)d->work_len, d->info), "geqrf");
    extract_r<<<blocks_for((int64_t)nc * nc), kT, 0, st>>>(A, Rout, m, nc);
    PR_BLAS(ctx, cusolverDnDorgqr(d->sol, m, nc, nc, A, m, d->tau, d->work, (int)d->work_len, d->info), "orgqr");
    return PR_OK;
}

// SVD of the h x h matrix H: Xh, sig, YhT (full)
pr_status svd_(pr_ctx* ctx, pr_driver* d, int h, cudaStream_t st) {
    int lw = 0;
    PR_BLAS(ctx, cusolverDnDgesvd_bufferSize(d->sol, h, h, &lw), "gesvd size");
    PR_TRY_ST(ensure_work(ctx, d, lw));
    signed char all = 'A';
    PR_BLAS(ctx, cusolverDnDgesvd(d->sol, all, all, h, h, d->H, h, d->sig, d->Xh, h, d->YhT, h, d->work,
                                  (int)d->work_len, d->rwork, d->info), "gesvd");
    int info = 0;
    cudaMemcpyAsync(&info, d->info, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "gesvd");
    if (info != 0) return blas_fail(ctx, info, "gesvd did not converge");
    return PR_OK;
}

int rank_cut_host(const std::vector<double>& sig, double tol) {
    double mx = 0;
    for (double x : sig) mx = std::max(mx, x);
    if (!(mx > 0)) return 0;
    int r = 0;
    for (double x : sig) r += (x / mx > tol) ? 1 : 0;
    return r;
}

// C (rows x nc) = B^T A with B = Bb W (Bb rows x hb, W hb x s, ld bcap): C is
// s x nc, through T = Bb^T A (hb x nc)
pr_status project_(pr_ctx* ctx, pr_driver* d, const double* Bb, const double* W, const double* A, int nc,
                   double* C) {
    const double one = 1.0, zero = 0.0;
    const int64_t rows = d->rows;
    PR_BLAS(ctx, cublasDgemm(d->blas, CUBLAS_OP_T, CUBLAS_OP_N, d->hb, nc, (int)rows, &one, Bb, (int)rows, A, (int)rows, &zero, d->Tb, d->hb), "Bb^T A");
    PR_BLAS(ctx, cublasDgemm(d->blas, CUBLAS_OP_T, CUBLAS_OP_N, d->s, nc, d->hb, &one, W, d->bcap, d->Tb, d->hb, &zero, C, d->s), "W^T T");
    return PR_OK;
}
// A -= (Bb W) C for C (s x nc), through T = W C (hb x nc)
pr_status subtract_(pr_ctx* ctx, pr_driver* d, const double* Bb, const double* W, const double* C, int nc,
                    double* A) {
    const double one = 1.0, zero = 0.0, mone = -1.0;
    const int64_t rows = d->rows;
    PR_BLAS(ctx, cublasDgemm(d->blas, CUBLAS_OP_N, CUBLAS_OP_N, d->hb, nc, d->s, &one, W, d->bcap, C, d->s, &zero, d->Tb, d->hb), "W C");
    PR_BLAS(ctx, cublasDgemm(d->blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)rows, nc, d->hb, &mone, Bb, (int)rows, d->Tb, d->hb, &one, A, (int)rows), "A - Bb T");
    return PR_OK;
}

// Alg. 1 with F, G (rows x nc, column-major, consumed).  Updates the factored
// X, Y (X = Xb WX, Y = Yb WY), S and s: the new bases [X Q_F] X_h, [Y Q_G] Y_h
// are [Xb Q_F] [WX 0; 0 I] X_h and the same for Y, so Q_F, Q_G are appended
// to Xb, Yb and only the small WX, WY are rotated.
pr_status update_svd(pr_ctx* ctx, pr_driver* d, double* F, double* G, int nc, cudaStream_t st) {
    const int64_t rows = d->rows;
    const int s = d->s;
    const double one = 1.0, zero = 0.0;
    PR_TRY_ST(ensure_capacity(ctx, d, s + nc, nc, st));
    const int h = s + nc;
    if (s > 0) {
        // U_F = U^T F, V_G = V^T G, then F - U U_F, G - V V_G
        PR_TRY_ST(project_(ctx, d, d->Xb, d->WX, F, nc, d->UF));
        PR_TRY_ST(project_(ctx, d, d->Yb, d->WY, G, nc, d->VG));
        PR_TRY_ST(subtract_(ctx, d, d->Xb, d->WX, d->UF, nc, F));
        PR_TRY_ST(subtract_(ctx, d, d->Yb, d->WY, d->VG, nc, G));
    }
    cudaMemcpyAsync(d->QF, F, (size_t)rows * nc * 8, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(d->QG, G, (size_t)rows * nc * 8, cudaMemcpyDeviceToDevice, st);
    PR_TRY_ST(qr_(ctx, d, d->QF, d->RF, nc, st));
    PR_TRY_ST(qr_(ctx, d, d->QG, d->RG, nc, st));
    // A1 = [U_F; R_F], A2 = [V_G; R_G]  (h x nc), H = A1 A2^T + diag(S, 0)
    if (s > 0) {
        copy_block<<<blocks_for((int64_t)s * nc), kT, 0, st>>>(d->UF, s, d->A1, h, s, nc, 0);
        copy_block<<<blocks_for((int64_t)s * nc), kT, 0, st>>>(d->VG, s, d->A2, h, s, nc, 0);
    }
    copy_block<<<blocks_for((int64_t)nc * nc), kT, 0, st>>>(d->RF, nc, d->A1, h, nc, nc, s);
    copy_block<<<blocks_for((int64_t)nc * nc), kT, 0, st>>>(d->RG, nc, d->A2, h, nc, nc, s);
    PR_BLAS(ctx, cublasDgemm(d->blas, CUBLAS_OP_N, CUBLAS_OP_T, h, h, nc, &one, d->A1, h, d->A2, h, &zero, d->H, h), "H");
    if (s > 0) add_diag<<<1, kT, 0, st>>>(d->H, h, d->S, s);
    PR_TRY_ST(svd_(ctx, d, h, st));
    std::vector<double> sig(h);
    cudaMemcpy(sig.data(), d->sig, (size_t)h * 8, cudaMemcpyDeviceToHost);
    const int r = rank_cut_host(sig, ctx->opts.tol);
    if (r == 0) {
        d->s = 0;
        d->hb = 0;
        return PR_OK;
    }
    // U~ = [U Q_F] X_h(:, 1:r), V~ = [V Q_G] Y_h(:, 1:r)   (Y_h = YhT^T):
    // Xb <- [Xb Q_F], WX <- [WX X_h(1:s, 1:r); X_h(s+1:h, 1:r)], likewise Y
    const int hb = d->hb, ld = d->bcap;
    cudaMemcpyAsync(d->Xb + (int64_t)hb * rows, d->QF, (size_t)rows * nc * 8, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(d->Yb + (int64_t)hb * rows, d->QG, (size_t)rows * nc * 8, cudaMemcpyDeviceToDevice, st);
    if (s > 0) {
        PR_BLAS(ctx, cublasDgemm(d->blas, CUBLAS_OP_N, CUBLAS_OP_N, hb, r, s, &one, d->WX, ld, d->Xh, h, &zero, d->WXn, ld), "WX Xh");
        PR_BLAS(ctx, cublasDgemm(d->blas, CUBLAS_OP_N, CUBLAS_OP_T, hb, r, s, &one, d->WY, ld, d->YhT, h, &zero, d->WYn, ld), "WY Yh");
    }
    copy_block<<<blocks_for((int64_t)nc * r), kT, 0, st>>>(d->Xh + s, h, d->WXn, ld, nc, r, hb);
    copy_block_t<<<blocks_for((int64_t)nc * r), kT, 0, st>>>(d->YhT + (int64_t)s * h, h, d->WYn, ld, nc, r, hb);
    std::swap(d->WX, d->WXn);
    std::swap(d->WY, d->WYn);
    cudaMemcpyAsync(d->S, d->sig, (size_t)r * 8, cudaMemcpyDeviceToDevice, st);
    d->s = r;
    d->hb = hb + nc;
    return PR_OK;
}

// g <- X (Y^T g) using `tmp` (cap) as the s-vector
pr_status apply_omega(pr_ctx* ctx, pr_driver* d, const double* g, double* out, cudaStream_t st) {
    const double one = 1.0, zero = 0.0;
    if (d->s == 0) {
        cudaMemsetAsync(out, 0, (size_t)d->rows * 8, st);
        return PR_OK;
    }
    // X (Y^T g) = Xb (WX (WY^T (Yb^T g)))
    double* t1 = d->vb;
    double* t2 = d->vb + d->bcap;
    PR_BLAS(ctx, cublasDgemv(d->blas, CUBLAS_OP_T, (int)d->rows, d->hb, &one, d->Yb, (int)d->rows, g, 1, &zero, t1, 1), "Yb^T g");
    PR_BLAS(ctx, cublasDgemv(d->blas, CUBLAS_OP_T, d->hb, d->s, &one, d->WY, d->bcap, t1, 1, &zero, d->rwork, 1), "WY^T");
    PR_BLAS(ctx, cublasDgemv(d->blas, CUBLAS_OP_N, d->hb, d->s, &one, d->WX, d->bcap, d->rwork, 1, &zero, t2, 1), "WX");
    PR_BLAS(ctx, cublasDgemv(d->blas, CUBLAS_OP_N, (int)d->rows, d->hb, &one, d->Xb, (int)d->rows, t2, 1, &zero, out, 1), "Xb");
    return PR_OK;
}

// ||F - X Y^T G||_F / ||F||_F for the current data (F, G unmodified copies in Fm/Gm)
pr_status residual_(pr_ctx* ctx, pr_driver* d, const double* F, const double* G, int nc, double* res,
                    cudaStream_t st) {
    const int64_t rows = d->rows;
    double nf = 0, nr = 0;
    PR_BLAS(ctx, cublasDnrm2(d->blas, (int)(rows * nc), F, 1, &nf), "nrm2");
    // QF (rows x nc) <- F - X (Y^T G): reuse QF/UF scratch (UF has >= s*nc)
    cudaMemcpyAsync(d->QF, F, (size_t)rows * nc * 8, cudaMemcpyDeviceToDevice, st);
    if (d->s > 0) {
        PR_TRY_ST(project_(ctx, d, d->Yb, d->WY, G, nc, d->UF));
        PR_TRY_ST(subtract_(ctx, d, d->Xb, d->WX, d->UF, nc, d->QF));
    }
    PR_BLAS(ctx, cublasDnrm2(d->blas, (int)(rows * nc), d->QF, 1, &nr), "nrm2");
    *res = nf > 0 ? nr / nf : 0.0;
    return PR_OK;
}

}  // namespace

// ============================================================================ C ABI
extern "C" pr_status pr_coarse_sweep(pr_ctx* ctx, const void* u, const void* v, void* U_out, void* V_out,
                                     int n_begin, int n_end, void* stream) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_coarse_sweep: ctx is NULL");
    if (!u || !v || !U_out || !V_out) return pr_fail(ctx, PR_EINVAL, "pr_coarse_sweep: NULL array");
    if (n_begin < 0 || n_end < n_begin || n_end > ctx->N)
        return pr_fail(ctx, PR_EINVAL, "pr_coarse_sweep: slice range outside [0, N]");
    if (!ctx->coarse) return pr_fail(ctx, PR_EINVAL, "pr_coarse_sweep: no coarse grid");
    if (n_end == n_begin) return PR_OK;
    const size_t esz = ctx->dtype == PR_F32 ? 4 : 8;
    const size_t fo = (size_t)n_begin * ctx->pts * esz, co = (size_t)n_begin * ctx->coarse->pts * esz;
    cudaStream_t st = (cudaStream_t)stream;
    PR_TRY_ST(coarse_of(ctx, (const char*)u + fo, (const char*)v + fo, (char*)U_out + co, (char*)V_out + co,
                        n_end - n_begin, st));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "pr_coarse_sweep");
    return PR_OK;
}

extern "C" pr_status pr_procrustes_correct(pr_ctx* ctx, const double* Fcols, const double* Gcols, int ncols,
                                           void* stream) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_procrustes_correct: ctx is NULL");
    if (!Fcols || !Gcols || ncols < 1 || ncols > ctx->N)
        return pr_fail(ctx, PR_EINVAL, "pr_procrustes_correct: need 1 <= ncols <= N and non-NULL columns");
    cudaStream_t st = (cudaStream_t)stream;
    pr_driver* d = nullptr;
    PR_TRY_ST(driver(ctx, st, &d));
    cudaMemcpyAsync(d->Fm, Fcols, (size_t)d->rows * ncols * 8, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(d->Gm, Gcols, (size_t)d->rows * ncols * 8, cudaMemcpyDeviceToDevice, st);
    PR_TRY_ST(update_svd(ctx, d, d->Fm, d->Gm, ncols, st));
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "pr_procrustes_correct");
    return PR_OK;
}

extern "C" pr_status pr_procrustes_apply(pr_ctx* ctx, const double* g, double* out, int* rank, void* stream) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_procrustes_apply: ctx is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    pr_driver* d = nullptr;
    PR_TRY_ST(driver(ctx, st, &d));
    if (rank) *rank = d->s;
    if (!g || !out) return PR_OK;
    PR_TRY_ST(apply_omega(ctx, d, g, out, st));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "pr_procrustes_apply");
    return PR_OK;
}

extern "C" pr_status pr_procrustes_reset(pr_ctx* ctx) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_procrustes_reset: ctx is NULL");
    if (ctx->drv) {
        ctx->drv->s = 0;
        ctx->drv->hb = 0;
    }
    return PR_OK;
}

extern "C" pr_status pr_iterate(pr_ctx* ctx, const void* u0, const void* p0, int K, int corrector,
                                double tol_err, const void* u_ref, const void* v_ref, void* u_slices,
                                void* v_slices, double* err_hist, double* resid_hist, int* rank_hist,
                                int* k_done, void* stream) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_iterate: ctx is NULL");
    if (!u0 || !p0 || !u_slices || !v_slices) return pr_fail(ctx, PR_EINVAL, "pr_iterate: NULL array");
    if (K < 0) return pr_fail(ctx, PR_EINVAL, "pr_iterate: K must be >= 0");
    if (corrector < PR_CORR_PROCRUSTES || corrector > PR_CORR_PLAIN)
        return pr_fail(ctx, PR_EINVAL, "pr_iterate: unknown corrector");
    cudaStream_t st = (cudaStream_t)stream;
    pr_driver* d = nullptr;
    PR_TRY_ST(driver(ctx, st, &d));
    d->s = 0;   // a new run starts with an empty correlation matrix (Alg. 3)
    d->hb = 0;
    for (int i = 0; i < 4; ++i) {
        d->phase_ms[i] = 0.0;
        if (!d->ev[i]) PR_CUDA_TRY(ctx, cudaEventCreate(&d->ev[i]));
    }
    // elapsed time between two recorded events, added to a phase total
    auto add_phase = [&](int ph, int a, int b) -> pr_status {
        float ms = 0.0f;
        PR_CUDA_TRY(ctx, cudaEventSynchronize(d->ev[b]));
        PR_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, d->ev[a], d->ev[b]));
        d->phase_ms[ph] += ms;
        return PR_OK;
    };
    const size_t esz = ctx->dtype == PR_F32 ? 4 : 8;
    const int64_t pts = ctx->pts, cpts = d->cpts;
    const int N = ctx->N;
    if (k_done) *k_done = 0;
    // relative energy-norm error of u^{k+1}_N against the reference (Sec. 6)
    double e_ref = 0.0;
    if (u_ref && v_ref) PR_TRY_ST(pr_launch_energy(ctx, u_ref, v_ref, 1, &e_ref, st));
    char* us = (char*)u_slices;
    char* vs = (char*)v_slices;
    auto fu = [&](int n) { return us + (size_t)n * pts * esz; };
    auto fv = [&](int n) { return vs + (size_t)n * pts * esz; };
    auto cu = [&](void* base, int n) { return (char*)base + (size_t)n * cpts * esz; };

    // Alg. 3 initialisation: u^1_0 = [u0, p0], u^1_n = I C R u^1_{n-1}
    cudaEventRecord(d->ev[0], st);
    cudaMemcpyAsync(fu(0), u0, pts * esz, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(fv(0), p0, pts * esz, cudaMemcpyDeviceToDevice, st);
    for (int n = 1; n <= N; ++n) {
        PR_TRY_ST(coarse_of(ctx, fu(n - 1), fv(n - 1), d->w_u, d->w_v, 1, st));
        coarse_to_zc(ctx, d, d->w_u, d->w_v, nullptr, nullptr, st);
        PR_TRY_ST(interp_(ctx, d, nullptr, nullptr, fu(n), fv(n), st));
    }
    cudaEventRecord(d->ev[1], st);
    PR_TRY_ST(add_phase(0, 0, 1));
    for (int k = 1; k <= K; ++k) {
        // parallel phase: v_n = F u^k_{n-1}, U_n = C R u^k_{n-1}, n = 1..N
        cudaEventRecord(d->ev[0], st);
        pr_status s = pr_fine_all_slices(ctx, fu(0), fv(0), d->vF_u, d->vF_v, 0, N, st);
        if (s != PR_OK) return s;
        PR_TRY_ST(coarse_of(ctx, fu(0), fv(0), d->Uc_u, d->Uc_v, N, st));
        cudaEventRecord(d->ev[1], st);
        double res = 0.0;
        if (corrector == PR_CORR_PROCRUSTES) {
            // F = [Lambda R v_n], G = [Lambda U_n]; UpdateSVD (Alg. 1)
            lambda_(ctx, d->vF_u, d->vF_v, d->Fm, ctx->ratio, ctx->n, pts, 1.0, N, d->rows, st);
            lambda_(ctx, d->Uc_u, d->Uc_v, d->Gm, 1, d->nc, cpts, 1.0, N, d->rows, st);
            // the residual needs F, G after the update (update_svd consumes them)
            if (!d->F2) {
                PR_TRY_ST(alloc(ctx, (void**)&d->F2, (size_t)d->rows * N * 8, "pr_iterate: alloc"));
                PR_TRY_ST(alloc(ctx, (void**)&d->G2, (size_t)d->rows * N * 8, "pr_iterate: alloc"));
            }
            cudaMemcpyAsync(d->F2, d->Fm, (size_t)d->rows * N * 8, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(d->G2, d->Gm, (size_t)d->rows * N * 8, cudaMemcpyDeviceToDevice, st);
            PR_TRY_ST(update_svd(ctx, d, d->Fm, d->Gm, N, st));
            PR_TRY_ST(residual_(ctx, d, d->F2, d->G2, N, &res, st));
        }
        cudaEventRecord(d->ev[2], st);
        // serial corrected sweep; u^{k+1}_0 = u^k_0 stays
        for (int n = 1; n <= N; ++n) {
            PR_TRY_ST(coarse_of(ctx, fu(n - 1), fv(n - 1), d->w_u, d->w_v, 1, st));
            const void* Uu = cu(d->Uc_u, n - 1);
            const void* Uv = cu(d->Uc_v, n - 1);
            if (corrector == PR_CORR_PLAIN) {
                coarse_to_zc(ctx, d, d->w_u, d->w_v, Uu, Uv, st);
            } else {
                // d = Lambda w - Lambda U_n; zero mode sum w - sum U_n (A8, by linearity)
                lambda_(ctx, d->w_u, d->w_v, d->dvec, 1, d->nc, cpts, 1.0, 1, d->rows, st);
                lambda_(ctx, Uu, Uv, d->dvec, 1, d->nc, cpts, -1.0, 1, d->rows, st);
                zero_mode_(ctx, d, d->w_u, Uu, st);
                const double* g = d->dvec;
                if (corrector == PR_CORR_PROCRUSTES) {
                    PR_TRY_ST(apply_omega(ctx, d, d->dvec, d->gvec, st));
                    g = d->gvec;
                }
                PR_TRY_ST(reconstruct_(ctx, d, g, st));
                pair_to_complex<<<blocks_for(cpts), kT, 0, st>>>(d->du, d->dut, d->zc, cpts);
            }
            const size_t vo = (size_t)(n - 1) * pts * esz;
            PR_TRY_ST(interp_(ctx, d, (char*)d->vF_u + vo, (char*)d->vF_v + vo, fu(n), fv(n), st));
        }
        cudaEventRecord(d->ev[3], st);
        PR_TRY_ST(add_phase(1, 0, 1));
        PR_TRY_ST(add_phase(2, 1, 2));
        PR_TRY_ST(add_phase(3, 2, 3));
        if (resid_hist) resid_hist[k - 1] = res;
        if (rank_hist) rank_hist[k - 1] = d->s;
        if (k_done) *k_done = k;
        // stability guard: the energy of the state at T must stay finite
        double e_T = 0.0;
        PR_TRY_ST(pr_launch_energy(ctx, fu(N), fv(N), 1, &e_T, st));
        // a fused pass whose bounded wait gave up leaves its slices unpropagated
        // (later passes of that context skip their work): report it, do not
        // return this iteration's states as if they were valid
        PR_TRY_ST(pr_take_flag(ctx, ctx, st, "pr_iterate (fine sweep)"));
        if (ctx->coarse) PR_TRY_ST(pr_take_flag(ctx->coarse, ctx, st, "pr_iterate (coarse sweep)"));
        if (!isfinite(e_T)) {
            char buf[96];
            snprintf(buf, sizeof buf, "pr_iterate: energy at T is not finite after iteration %d", k);
            return pr_fail(ctx, PR_EUNSTABLE, buf);
        }
        if (u_ref && v_ref && e_ref > 0) {
            // difference into the (now free) fine-sweep buffer, slice 0
            if (ctx->dtype == PR_F32) {
                diff_kernel<float><<<blocks_for(pts), kT, 0, st>>>((const float*)fu(N), (const float*)u_ref, (float*)d->vF_u, pts);
                diff_kernel<float><<<blocks_for(pts), kT, 0, st>>>((const float*)fv(N), (const float*)v_ref, (float*)d->vF_v, pts);
            } else {
                diff_kernel<double><<<blocks_for(pts), kT, 0, st>>>((const double*)fu(N), (const double*)u_ref, (double*)d->vF_u, pts);
                diff_kernel<double><<<blocks_for(pts), kT, 0, st>>>((const double*)fv(N), (const double*)v_ref, (double*)d->vF_v, pts);
            }
            double e = 0.0;
            PR_TRY_ST(pr_launch_energy(ctx, d->vF_u, d->vF_v, 1, &e, st));
            const double rel = sqrt(e / e_ref);
            if (err_hist) err_hist[k - 1] = rel;
            if (rel <= tol_err) break;
        }
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "pr_iterate");
    return PR_OK;
}

extern "C" pr_status pr_iterate_phases(const pr_ctx* ctx, double* ms) {
    if (!ctx || !ms) return PR_EINVAL;
    for (int i = 0; i < 4; ++i) ms[i] = ctx->drv ? ctx->drv->phase_ms[i] : 0.0;
    return PR_OK;
}
