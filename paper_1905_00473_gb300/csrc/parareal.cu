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
    if (j <= 0x7fffffff && n <= 0x7fffffff) {
        // 32-bit division: several times fewer instructions than 64-bit
        uint32_t jj = (uint32_t)j;
        const uint32_t nn = (uint32_t)n;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            c[a] = (int64_t)(jj % nn);
            jj /= nn;
        }
        return;
    }
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
// central first-derivative weights beta_1..beta_h of nabla_h (Sec. 3.4),
// passed by value so that contexts of different orders never share them
struct Beta {
    double b[4];
};

template <typename T, int DIM>
__global__ void lambda_kernel(const T* __restrict__ w, const T* __restrict__ wt,
                              const double* __restrict__ cc, double* __restrict__ out,
                              int64_t nc, int stride, int64_t arr_n, int64_t arr_pts, int64_t cpts,
                              int order_half, Beta beta, double inv_dx, double sign, int nslices,
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
                int64_t cp = c[a] + k, cm = c[a] - k;   // periodic, k < nc
                if (cp >= nc) cp -= nc;
                if (cm < 0) cm += nc;
                const double up = (double)ws[base + (cp * stride - f[a]) * astride];
                const double um = (double)ws[base + (cm * stride - f[a]) * astride];
                acc += beta.b[k - 1] * (up - um);
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

// kZm blocks reduce the zero mode of grad2func for the difference,
// sum_J (w_J - U_J): each a fixed share in a fixed order into zbuf[1 + b];
// the block that finishes last adds the partials in block order into
// zbuf[0] and resets the arrival counter (after the partials), so the sum is
// the same on every run.
constexpr int kZm = 64;

// The serial sweep's d = Lambda w - Lambda U (coarse arrays, one slice;
// each term rounded as lambda_kernel rounds it, then subtracted) and the
// zero mode of w - U, in one launch of kZm blocks.
template <typename T, int DIM>
__global__ void __launch_bounds__(kT) lambda_diff_kernel(const T* __restrict__ w, const T* __restrict__ wt,
                                                         const T* __restrict__ U, const T* __restrict__ Ut,
                                                         const double* __restrict__ cc, double* __restrict__ out,
                                                         int64_t nc, int64_t cpts, int order_half, Beta beta,
                                                         double inv_dx, double* __restrict__ zbuf) {
    __shared__ double red[kT];
    __shared__ bool last;
    double zacc = 0.0;
    for (int64_t J = (int64_t)blockIdx.x * kT + threadIdx.x; J < cpts; J += (int64_t)gridDim.x * kT) {
        int64_t c[3];
        coords<DIM>(J, nc, c);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            int64_t astride = 1;
            for (int b = 0; b < a; ++b) astride *= nc;
            double aw = 0.0, au = 0.0;
            for (int k = 1; k <= order_half; ++k) {
                int64_t cp = c[a] + k, cm = c[a] - k;
                if (cp >= nc) cp -= nc;
                if (cm < 0) cm += nc;
                const int64_t jp = J + (cp - c[a]) * astride, jm = J + (cm - c[a]) * astride;
                aw += beta.b[k - 1] * ((double)w[jp] - (double)w[jm]);
                au += beta.b[k - 1] * ((double)U[jp] - (double)U[jm]);
            }
            out[a * cpts + J] = __dsub_rn(__dmul_rn(aw, inv_dx), __dmul_rn(au, inv_dx));
        }
        out[DIM * cpts + J] = (double)wt[J] / cc[J] - (double)Ut[J] / cc[J];
        zacc += (double)w[J] - (double)U[J];
    }
    red[threadIdx.x] = zacc;
    __syncthreads();
    for (int s = kT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    unsigned* count = (unsigned*)(zbuf + 1 + kZm);
    if (threadIdx.x == 0) {
        zbuf[1 + blockIdx.x] = red[0];
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double sum = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) sum += __ldcg(zbuf + 1 + b);
        zbuf[0] = sum;
        *count = 0u;
    }
}

// ---------------------------------------------------------------- Lambda^dagger (grad2func)
// CT: the transform's complex type, double2 (FP64 contexts, adjoints) or
// float2 (the forward path of FP32 contexts); real_of<CT> its real type
template <typename CT>
using real_of = decltype(CT::x);

template <typename CT>
__global__ void real_to_complex(const double* __restrict__ x, CT* __restrict__ z, int64_t m) {
    using RT = real_of<CT>;
    for (int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x; j < m; j += (int64_t)gridDim.x * kT)
        z[j] = CT{(RT)x[j], (RT)0};
}

// w^(xi) = -i (xi . q^) / |xi|^2, w^(0) = zero mode (Alg. 2), in place into z[0..cpts)
template <int DIM, typename CT>
__global__ void grad2func_combine(CT* __restrict__ z, int64_t nc, int64_t cpts, const double* __restrict__ zero_mode) {
    using RT = real_of<CT>;
    for (int64_t J = (int64_t)blockIdx.x * kT + threadIdx.x; J < cpts; J += (int64_t)gridDim.x * kT) {
        int64_t c[3];
        coords<DIM>(J, nc, c);
        RT re = 0, im = 0, mag2 = 0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const RT xi = (RT)(2.0 * M_PI * (double)freq(c[a], nc));
            const CT q = z[a * cpts + J];
            re += xi * q.x;
            im += xi * q.y;
            mag2 += xi * xi;
        }
        // -i (re + i im) = im - i re
        z[J] = mag2 > 0 ? CT{im / mag2, -re / mag2} : CT{(RT)*zero_mode, (RT)0};
    }
}

// du = real(ifft(.)) (unnormalised inverse, so / cpts) and du_t = c p, written
// back as the two complex coarse fields that I transforms next (a thread
// reads z[J] before it writes z[J] and z[cpts + J])
template <typename CT>
__global__ void grad2func_finish(CT* __restrict__ z, const double* __restrict__ p, const double* __restrict__ cc,
                                 int64_t cpts) {
    using RT = real_of<CT>;
    const double inv = 1.0 / (double)cpts;
    for (int64_t J = (int64_t)blockIdx.x * kT + threadIdx.x; J < cpts; J += (int64_t)gridDim.x * kT) {
        const double du = (double)z[J].x * inv;
        const double dut = cc[J] * p[J];
        z[J] = CT{(RT)du, (RT)0};
        z[cpts + J] = CT{(RT)dut, (RT)0};
    }
}

// ---------------------------------------------------------------- I (interpft)
// fine spectrum from the coarse one: per axis, |m| < nc/2 copies, the coarse
// Nyquist coefficient goes half to +nc/2 and half to -nc/2 (both halves land
// on the same index when nf == nc); scaled by 1/cpts for the unnormalised
// inverse transform.  Two fields (u, u_t) one after the other.
template <int DIM, typename CT>
__global__ void interp_pad(const CT* __restrict__ cs, CT* __restrict__ fs, int64_t nc, int64_t nf, int64_t cpts,
                           int64_t fpts) {
    using RT = real_of<CT>;
    const RT scale = (RT)(1.0 / (double)cpts);
    for (int64_t idx = (int64_t)blockIdx.x * kT + threadIdx.x; idx < 2 * fpts; idx += (int64_t)gridDim.x * kT) {
        const int64_t fld = idx < fpts ? 0 : 1, jf = idx - fld * fpts;
        int64_t c[3];
        coords<DIM>(jf, nf, c);
        RT wgt = scale;
        int64_t src[3];
        const int64_t half = nc / 2;
        bool zero = false;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const int64_t i = c[a];
            RT wa = 0;
            int64_t sa = 0;
            if (nc % 2 == 0) {
                if (i < half) { wa = 1; sa = i; }
                else if (i > nf - half) { wa = 1; sa = i - nf + nc; }
                else {
                    if (i == half) { wa += (RT)0.5; sa = half; }
                    if (i == nf - half) { wa += (RT)0.5; sa = half; }
                }
            } else {
                if (i <= half) { wa = 1; sa = i; }
                else if (i >= nf - half) { wa = 1; sa = i - nf + nc; }
            }
            if (wa == 0) zero = true;
            wgt *= wa;
            src[a] = sa;
        }
        CT o = CT{(RT)0, (RT)0};
        if (!zero) {
            const CT x = cs[fld * cpts + lin<DIM>(src, nc)];
            o = CT{x.x * wgt, x.y * wgt};
        }
        fs[idx] = o;
    }
}

// out = base + real(fine field) for both fields (base may alias out)
template <typename T, typename CT>
__global__ void interp_add(const CT* __restrict__ fs, const T* bu, const T* bv, T* ou,
                           T* ov, int64_t fpts) {
    for (int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x; j < fpts; j += (int64_t)gridDim.x * kT) {
        const double a = (double)fs[j].x, b = (double)fs[fpts + j].x;
        ou[j] = (T)((bu ? (double)bu[j] : 0.0) + a);
        ov[j] = (T)((bv ? (double)bv[j] : 0.0) + b);
    }
}

template <typename T, typename CT>
__global__ void to_complex2(const T* __restrict__ a, const T* __restrict__ b, const T* __restrict__ sa,
                            const T* __restrict__ sb, CT* __restrict__ z, int64_t m) {
    using RT = real_of<CT>;
    for (int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x; j < m; j += (int64_t)gridDim.x * kT) {
        z[j] = CT{(RT)((double)a[j] - (sa ? (double)sa[j] : 0.0)), (RT)0};
        z[m + j] = CT{(RT)((double)b[j] - (sb ? (double)sb[j] : 0.0)), (RT)0};
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

// V(:, i) = E(:, h-1-i) for i < r (eigenvectors of ascending eigenvalues,
// reordered by descending singular value)
__global__ void reverse_cols(const double* __restrict__ E, double* __restrict__ V, int h, int r) {
    for (int64_t idx = (int64_t)blockIdx.x * kT + threadIdx.x; idx < (int64_t)h * r; idx += (int64_t)gridDim.x * kT) {
        const int col = (int)(idx / h), row = (int)(idx - (int64_t)col * h);
        V[idx] = E[(int64_t)(h - 1 - col) * h + row];
    }
}
// E <- (3 I - E) / 2 (r x r): the Newton-Schulz factor
__global__ void ns_coef(double* __restrict__ E, int r) {
    for (int64_t idx = (int64_t)blockIdx.x * kT + threadIdx.x; idx < (int64_t)r * r; idx += (int64_t)gridDim.x * kT)
        E[idx] = ((idx % r) == (idx / r) ? 1.5 : 0.0) - 0.5 * E[idx];
}
// X(:, i) = Q(:, i) sg[i]
__global__ void scale_cols(const double* __restrict__ Q, const double* __restrict__ sg, double* __restrict__ X, int h,
                           int r) {
    for (int64_t idx = (int64_t)blockIdx.x * kT + threadIdx.x; idx < (int64_t)h * r; idx += (int64_t)gridDim.x * kT)
        X[idx] = Q[idx] * sg[idx / h];
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
    // FP32 contexts: single-precision transforms for the forward Lambda^dagger
    // and I (the FP64 plans above stay for the adjoint)
    bool fft32 = false;
    cufftHandle splan_c1 = 0, splan_cd = 0, splan_c2 = 0, splan_f2 = 0;
    float2* zc32 = nullptr;   // [max(d,2) * cpts]
    float2* zf32 = nullptr;   // [2 * pts]
    cublasHandle_t blas = nullptr;
    cusolverDnHandle_t sol = nullptr;
    // dtype buffers
    void* vF_u = nullptr; void* vF_v = nullptr;     // F u^k_{n-1}   [N][pts]
    void* Uc_u = nullptr; void* Uc_v = nullptr;     // C R u^k_{n-1} [N][cpts]
    void* w_u = nullptr; void* w_v = nullptr;       // serial-sweep coarse state [cpts]
    // FP64 buffers
    double* Fm = nullptr; double* Gm = nullptr;     // data matrices [rows][N], column-major
    double* dvec = nullptr; double* gvec = nullptr; // [rows]
    double* zero = nullptr;                         // device scalar (then the zero-mode partials)
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
    double *E = nullptr, *rsign = nullptr;   // SVD through the eigenproblem of H^T H
    double *cq = nullptr, *cq2 = nullptr;   // Cholesky QR workspace of each lane (zero-filled)
    double* rnorm = nullptr;                // ||F||, ||F - Omega G|| of the last residual
    // FP32 contexts: single-precision copies of Xb, Yb [rows][bcap] for the
    // corrector's matrix-vector products, and their scratch
    float *Xs = nullptr, *Ys = nullptr, *gs = nullptr;
    double* opart = nullptr;    // [kOmJ][rows]
    double* tpart = nullptr;    // [kOmR][kOmMaxCols]
    unsigned* tcnt = nullptr;   // [kOmMaxCols / 2], zero-filled
    // a second lane (stream, handles, scratch) on which G's projections,
    // deflations and QR run beside F's: those steps are latency-bound
    cudaStream_t st2 = nullptr;
    cublasHandle_t blas2 = nullptr;
    cusolverDnHandle_t sol2 = nullptr;
    double *Tb2 = nullptr, *work2 = nullptr, *tau2 = nullptr;
    int64_t work2_len = 0;
    int* info2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int* info = nullptr;
    int64_t work_len = 0;
    int hcap = 0;   // allocated (s+N) capacity of the small matrices
    // FP32 contexts: the tall-skinny products with the bases (projections
    // and deflations of Alg. 1) run on the tensor cores in split-TF32
    // (gram_tc.cu), with one reorthogonalisation pass; FP64 contexts use
    // FP64 DGEMM throughout
    bool tc = false;
    Beta beta = {{0.0, 0.0, 0.0, 0.0}};   // nabla_h weights of this context's order
    int eig_svds = 0, all_svds = 0;        // SVDs taken by svd_eig_, and all, since the last pr_iterate
    // per-call breakdown of creating the corrector (pr_iterate_corrector_phases):
    // projections and deflations, QR of the residual blocks, H and its SVD,
    // basis rotation, residual diagnostic
    cudaEvent_t cev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double corr_ms[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
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
        if (d->fft32) {
            cufftDestroy(d->splan_c1);
            cufftDestroy(d->splan_cd);
            cufftDestroy(d->splan_c2);
            cufftDestroy(d->splan_f2);
        }
    }
    if (d->blas) cublasDestroy(d->blas);
    if (d->sol) cusolverDnDestroy(d->sol);
    if (d->blas2) cublasDestroy(d->blas2);
    if (d->sol2) cusolverDnDestroy(d->sol2);
    if (d->st2) cudaStreamDestroy(d->st2);
    if (d->ev_fork) cudaEventDestroy(d->ev_fork);
    if (d->ev_join) cudaEventDestroy(d->ev_join);
    for (cudaEvent_t e : d->ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : d->cev)
        if (e) cudaEventDestroy(e);
    void* bufs[] = {d->vF_u, d->vF_v, d->Uc_u, d->Uc_v, d->w_u, d->w_v, d->Fm, d->Gm, d->dvec, d->gvec,
                    d->zero, d->zc, d->zf, d->Xb, d->Yb, d->WX, d->WY, d->WXn, d->WYn,
                    d->Tb, d->vb, d->S, d->QF, d->QG, d->RF, d->RG, d->tau, d->UF, d->VG, d->A1, d->A2,
                    d->H, d->Xh, d->YhT, d->sig, d->work, d->rwork, d->F2, d->G2, d->info, d->E,
                    d->rsign, d->Tb2, d->work2, d->tau2, d->info2, d->cq, d->cq2, d->rnorm, d->zc32, d->zf32, d->Xs, d->Ys, d->gs, d->opart, d->tpart, d->tcnt};
    for (void* b : bufs) pr_dev_free(ctx, b);
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
    cudaError_t e = pr_dev_malloc(ctx, p, bytes > 0 ? bytes : 16);
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
        // zero mode, kZm partials, the arrival counter
        PR_TRY_ST(alloc(ctx, (void**)&d->zero, (size_t)(2 + kZm) * 8, "driver: alloc"));
        PR_CUDA_TRY(ctx, cudaMemset(d->zero, 0, (size_t)(2 + kZm) * 8));
        PR_TRY_ST(alloc(ctx, (void**)&d->zc, (size_t)std::max(d->dim, 2) * d->cpts * 16, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->zf, (size_t)2 * d->pts * 16, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->info, sizeof(int), "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->info2, sizeof(int), "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->tau2, (size_t)d->N * 8, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->cq, (size_t)3 * kCqMaxCols * kCqMaxCols * 8, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->cq2, (size_t)3 * kCqMaxCols * kCqMaxCols * 8, "driver: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->rnorm, 2 * 8, "driver: alloc"));
        PR_CUDA_TRY(ctx, cudaMemset(d->cq, 0, (size_t)3 * kCqMaxCols * kCqMaxCols * 8));
        PR_CUDA_TRY(ctx, cudaMemset(d->cq2, 0, (size_t)3 * kCqMaxCols * kCqMaxCols * 8));
        if (ctx->dtype == PR_F32) {
            PR_TRY_ST(alloc(ctx, (void**)&d->gs, (size_t)d->rows * 4, "driver: alloc"));
            PR_TRY_ST(alloc(ctx, (void**)&d->opart, (size_t)kOmJ * d->rows * 8, "driver: alloc"));
            PR_TRY_ST(alloc(ctx, (void**)&d->tpart, (size_t)kOmR * kOmMaxCols * 8, "driver: alloc"));
            PR_TRY_ST(alloc(ctx, (void**)&d->tcnt, (size_t)kOmMaxCols / 2 * 4, "driver: alloc"));
            PR_CUDA_TRY(ctx, cudaMemset(d->tcnt, 0, (size_t)kOmMaxCols / 2 * 4));
        }
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
        if (ctx->dtype == PR_F32) {
            PR_TRY_ST(alloc(ctx, (void**)&d->zc32, (size_t)std::max(d->dim, 2) * d->cpts * 8, "driver: alloc"));
            PR_TRY_ST(alloc(ctx, (void**)&d->zf32, (size_t)2 * d->pts * 8, "driver: alloc"));
            PR_FFT(ctx, cufftPlanMany(&d->splan_c1, d->dim, nn, nullptr, 1, (int)d->cpts, nullptr, 1, (int)d->cpts, CUFFT_C2C, 1), "plan");
            PR_FFT(ctx, cufftPlanMany(&d->splan_cd, d->dim, nn, nullptr, 1, (int)d->cpts, nullptr, 1, (int)d->cpts, CUFFT_C2C, d->dim), "plan");
            PR_FFT(ctx, cufftPlanMany(&d->splan_c2, d->dim, nn, nullptr, 1, (int)d->cpts, nullptr, 1, (int)d->cpts, CUFFT_C2C, 2), "plan");
            PR_FFT(ctx, cufftPlanMany(&d->splan_f2, d->dim, nf, nullptr, 1, (int)d->pts, nullptr, 1, (int)d->pts, CUFFT_C2C, 2), "plan");
            d->fft32 = true;
        }
        d->tc = ctx->dtype == PR_F32;
        for (int i = 0; i < 6; ++i) PR_CUDA_TRY(ctx, cudaEventCreate(&d->cev[i]));
        PR_CUDA_TRY(ctx, cudaEventCreateWithFlags(&d->ev_fork, cudaEventDisableTiming));
        PR_CUDA_TRY(ctx, cudaEventCreateWithFlags(&d->ev_join, cudaEventDisableTiming));
        PR_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&d->st2, cudaStreamNonBlocking));
        PR_BLAS(ctx, cublasCreate(&d->blas2), "cublasCreate");
        PR_BLAS(ctx, cusolverDnCreate(&d->sol2), "cusolverDnCreate");
        PR_BLAS(ctx, cublasSetStream(d->blas2, d->st2), "cublasSetStream");
        PR_BLAS(ctx, cusolverDnSetStream(d->sol2, d->st2), "cusolverDnSetStream");
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
        for (int k = 0; k < 4; ++k) d->beta.b[k] = beta[k];
    }
    pr_driver* d = ctx->drv;
    PR_FFT(ctx, cufftSetStream(d->plan_c1, st), "set stream");
    PR_FFT(ctx, cufftSetStream(d->plan_cd, st), "set stream");
    PR_FFT(ctx, cufftSetStream(d->plan_c2, st), "set stream");
    PR_FFT(ctx, cufftSetStream(d->plan_f2, st), "set stream");
    if (d->fft32) {
        PR_FFT(ctx, cufftSetStream(d->splan_c1, st), "set stream");
        PR_FFT(ctx, cufftSetStream(d->splan_cd, st), "set stream");
        PR_FFT(ctx, cufftSetStream(d->splan_c2, st), "set stream");
        PR_FFT(ctx, cufftSetStream(d->splan_f2, st), "set stream");
    }
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
        case 1: lambda_kernel<T, 1><<<blocks_for(total), kT, 0, st>>>((const T*)w, (const T*)wt, ctx->coarse->c64, out, nc, stride, arr_n, arr_pts, cpts, h, ctx->drv->beta, inv_dx, sign, ns, out_ld); break;
        case 2: lambda_kernel<T, 2><<<blocks_for(total), kT, 0, st>>>((const T*)w, (const T*)wt, ctx->coarse->c64, out, nc, stride, arr_n, arr_pts, cpts, h, ctx->drv->beta, inv_dx, sign, ns, out_ld); break;
        default: lambda_kernel<T, 3><<<blocks_for(total), kT, 0, st>>>((const T*)w, (const T*)wt, ctx->coarse->c64, out, nc, stride, arr_n, arr_pts, cpts, h, ctx->drv->beta, inv_dx, sign, ns, out_ld); break;
    }
}
void lambda_(pr_ctx* ctx, const void* w, const void* wt, double* out, int stride, int64_t arr_n,
             int64_t arr_pts, double sign, int ns, int64_t out_ld, cudaStream_t st) {
    if (ctx->dtype == PR_F32) launch_lambda_t<float>(ctx, w, wt, out, stride, arr_n, arr_pts, sign, ns, out_ld, st);
    else launch_lambda_t<double>(ctx, w, wt, out, stride, arr_n, arr_pts, sign, ns, out_ld, st);
}

// the transforms of the forward path in the precision of the context
cufftResult fft_exec(cufftHandle p, cufftDoubleComplex* z, int dir) { return cufftExecZ2Z(p, z, z, dir); }
cufftResult fft_exec(cufftHandle p, cufftComplex* z, int dir) { return cufftExecC2C(p, z, z, dir); }
struct FftSet {
    cufftHandle c1, cd, c2, f2;
};
template <typename CT> CT* zc_of(pr_driver* d);
template <> double2* zc_of<double2>(pr_driver* d) { return d->zc; }
template <> float2* zc_of<float2>(pr_driver* d) { return d->zc32; }
template <typename CT> CT* zf_of(pr_driver* d);
template <> double2* zf_of<double2>(pr_driver* d) { return d->zf; }
template <> float2* zf_of<float2>(pr_driver* d) { return d->zf32; }
template <typename CT> FftSet plans_of(pr_driver* d);
template <> FftSet plans_of<double2>(pr_driver* d) { return {d->plan_c1, d->plan_cd, d->plan_c2, d->plan_f2}; }
template <> FftSet plans_of<float2>(pr_driver* d) { return {d->splan_c1, d->splan_cd, d->splan_c2, d->splan_f2}; }

// Lambda^dagger of gvec (rows) with zero mode *zero -> (du, dut) on the coarse
// grid, left in the complex coarse buffer as the two fields I interpolates
template <typename CT>
pr_status reconstruct_t(pr_ctx* ctx, pr_driver* d, const double* g, cudaStream_t st) {
    const int64_t cpts = d->cpts;
    CT* zc = zc_of<CT>(d);
    const FftSet P = plans_of<CT>(d);
    real_to_complex<CT><<<blocks_for(d->dim * cpts), kT, 0, st>>>(g, zc, d->dim * cpts);
    PR_FFT(ctx, fft_exec(P.cd, zc, CUFFT_FORWARD), "grad2func forward");
    switch (d->dim) {
        case 1: grad2func_combine<1, CT><<<blocks_for(cpts), kT, 0, st>>>(zc, d->nc, cpts, d->zero); break;
        case 2: grad2func_combine<2, CT><<<blocks_for(cpts), kT, 0, st>>>(zc, d->nc, cpts, d->zero); break;
        default: grad2func_combine<3, CT><<<blocks_for(cpts), kT, 0, st>>>(zc, d->nc, cpts, d->zero); break;
    }
    PR_FFT(ctx, fft_exec(P.c1, zc, CUFFT_INVERSE), "grad2func inverse");
    grad2func_finish<CT><<<blocks_for(cpts), kT, 0, st>>>(zc, g + (int64_t)d->dim * cpts, ctx->coarse->c64, cpts);
    return PR_OK;
}
pr_status reconstruct_(pr_ctx* ctx, pr_driver* d, const double* g, cudaStream_t st) {
    return d->fft32 ? reconstruct_t<float2>(ctx, d, g, st) : reconstruct_t<double2>(ctx, d, g, st);
}

// fine (u, v) = base + I(coarse fields in the complex coarse buffer); that
// buffer must hold the two coarse fields as complex
template <typename T, typename CT>
pr_status interp_t(pr_ctx* ctx, pr_driver* d, const void* bu, const void* bv, void* ou, void* ov, cudaStream_t st) {
    CT* zc = zc_of<CT>(d);
    CT* zf = zf_of<CT>(d);
    const FftSet P = plans_of<CT>(d);
    PR_FFT(ctx, fft_exec(P.c2, zc, CUFFT_FORWARD), "interp forward");
    switch (d->dim) {
        case 1: interp_pad<1, CT><<<blocks_for(2 * d->pts), kT, 0, st>>>(zc, zf, d->nc, d->n, d->cpts, d->pts); break;
        case 2: interp_pad<2, CT><<<blocks_for(2 * d->pts), kT, 0, st>>>(zc, zf, d->nc, d->n, d->cpts, d->pts); break;
        default: interp_pad<3, CT><<<blocks_for(2 * d->pts), kT, 0, st>>>(zc, zf, d->nc, d->n, d->cpts, d->pts); break;
    }
    PR_FFT(ctx, fft_exec(P.f2, zf, CUFFT_INVERSE), "interp inverse");
    interp_add<T, CT><<<blocks_for(d->pts), kT, 0, st>>>(zf, (const T*)bu, (const T*)bv, (T*)ou, (T*)ov, d->pts);
    return PR_OK;
}
pr_status interp_(pr_ctx* ctx, pr_driver* d, const void* bu, const void* bv, void* ou, void* ov, cudaStream_t st) {
    if (ctx->dtype == PR_F32)
        return d->fft32 ? interp_t<float, float2>(ctx, d, bu, bv, ou, ov, st)
                        : interp_t<float, double2>(ctx, d, bu, bv, ou, ov, st);
    return interp_t<double, double2>(ctx, d, bu, bv, ou, ov, st);
}

// complex coarse buffer <- (a - sa, b - sb) for coarse dtype fields (sa/sb may be null)
void coarse_to_zc(pr_ctx* ctx, pr_driver* d, const void* a, const void* b, const void* sa, const void* sb, cudaStream_t st) {
    if (ctx->dtype == PR_F32) {
        if (d->fft32)
            to_complex2<float, float2><<<blocks_for(d->cpts), kT, 0, st>>>((const float*)a, (const float*)b, (const float*)sa, (const float*)sb, d->zc32, d->cpts);
        else
            to_complex2<float, double2><<<blocks_for(d->cpts), kT, 0, st>>>((const float*)a, (const float*)b, (const float*)sa, (const float*)sb, d->zc, d->cpts);
    } else {
        to_complex2<double, double2><<<blocks_for(d->cpts), kT, 0, st>>>((const double*)a, (const double*)b, (const double*)sa, (const double*)sb, d->zc, d->cpts);
    }
}
// d = Lambda w - Lambda U and the zero mode of w - U (one slice, coarse arrays)
void lambda_diff_(pr_ctx* ctx, pr_driver* d, const void* w, const void* wt, const void* U, const void* Ut,
                  cudaStream_t st) {
    const int h = ctx->opts.grad_order / 2;
    const double inv_dx = 1.0 / ctx->coarse->dx;
    const int64_t nc = d->nc, cpts = d->cpts;
    const double* cc = ctx->coarse->c64;
#define PR_LDIFF(T, D)                                                                                  \
    lambda_diff_kernel<T, D><<<kZm, kT, 0, st>>>((const T*)w, (const T*)wt, (const T*)U, (const T*)Ut, cc, \
                                                 d->dvec, nc, cpts, h, d->beta, inv_dx, d->zero)
    if (ctx->dtype == PR_F32) {
        switch (ctx->dim) {
            case 1: PR_LDIFF(float, 1); break;
            case 2: PR_LDIFF(float, 2); break;
            default: PR_LDIFF(float, 3); break;
        }
    } else {
        switch (ctx->dim) {
            case 1: PR_LDIFF(double, 1); break;
            case 2: PR_LDIFF(double, 2); break;
            default: PR_LDIFF(double, 3); break;
        }
    }
#undef PR_LDIFF
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
        if (d->gs) {   // the FP32 copies of the bases follow the FP64 ones
            float *Xs = nullptr, *Ys = nullptr;
            PR_TRY_ST(alloc(ctx, (void**)&Xs, (size_t)rows * bc * 4, "svd: alloc"));
            PR_TRY_ST(alloc(ctx, (void**)&Ys, (size_t)rows * bc * 4, "svd: alloc"));
            if (d->s > 0) {
                cudaMemcpy(Xs, d->Xs, (size_t)rows * d->hb * 4, cudaMemcpyDeviceToDevice);
                cudaMemcpy(Ys, d->Ys, (size_t)rows * d->hb * 4, cudaMemcpyDeviceToDevice);
            }
            pr_dev_free(ctx, d->Xs);
            pr_dev_free(ctx, d->Ys);
            d->Xs = Xs;
            d->Ys = Ys;
        }
        double* Tb2 = nullptr;
        PR_TRY_ST(alloc(ctx, (void**)&Tb2, (size_t)bc * d->N * 8, "svd: alloc"));
        pr_dev_free(ctx, d->Tb2);
        d->Tb2 = Tb2;
        double** olds[] = {&d->Xb, &d->Yb, &d->WX, &d->WY, &d->WXn, &d->WYn, &d->Tb, &d->vb, &d->S};
        for (double** o : olds) pr_dev_free(ctx, *o);
        d->Xb = Xb; d->Yb = Yb; d->WX = WX; d->WY = WY; d->WXn = WXn; d->WYn = WYn;
        d->Tb = Tb; d->vb = vb; d->S = S;
        d->bcap = bc;
    }
    const int h = need_s;   // (s + ncols)
    if (h > d->hcap || !d->QF) {
        const int hc = std::max(h, d->hcap * 2);
        double** smalls[] = {&d->RF, &d->RG, &d->UF, &d->VG, &d->A1, &d->A2, &d->H, &d->Xh, &d->YhT,
                             &d->E, &d->rsign};
        for (double** p : smalls) {
            pr_dev_free(ctx, *p);
            *p = nullptr;
        }
        for (double* q : {d->sig, d->tau, d->QF, d->QG, d->rwork}) pr_dev_free(ctx, q);
        PR_TRY_ST(alloc(ctx, (void**)&d->RF, (size_t)ncols * ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->RG, (size_t)ncols * ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->UF, (size_t)hc * ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->VG, (size_t)hc * ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->A1, (size_t)hc * ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->A2, (size_t)hc * ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->H, (size_t)hc * hc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->Xh, (size_t)hc * hc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->YhT, (size_t)hc * hc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->E, (size_t)hc * hc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->rsign, (size_t)hc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->sig, (size_t)hc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->rwork, (size_t)hc * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->tau, (size_t)ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->QF, (size_t)rows * ncols * 8, "svd: alloc"));
        PR_TRY_ST(alloc(ctx, (void**)&d->QG, (size_t)rows * ncols * 8, "svd: alloc"));
        d->hcap = hc;
    }
    return PR_OK;
}

// One lane of the UpdateSVD products: its stream, library handles and scratch.
struct Lane {
    cudaStream_t st;
    cublasHandle_t blas;
    cusolverDnHandle_t sol;
    double* Tb;
    double** work;
    int64_t* work_len;
    double* tau;
    int* info;
    double* cq;
};
Lane lane_f(pr_driver* d, cudaStream_t st) {
    return {st, d->blas, d->sol, d->Tb, &d->work, &d->work_len, d->tau, d->info, d->cq};
}
Lane lane_g(pr_driver* d) {
    return {d->st2, d->blas2, d->sol2, d->Tb2, &d->work2, &d->work2_len, d->tau2, d->info2, d->cq2};
}

pr_status ensure_lane_work(pr_ctx* ctx, const Lane& L, int64_t need) {
    if (need > *L.work_len) {
        cudaError_t e = cudaStreamSynchronize(L.st);
        if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "svd: synchronize");
        pr_dev_free(ctx, *L.work);
        *L.work = nullptr;
        PR_TRY_ST(alloc(ctx, (void**)L.work, (size_t)need * 8, "svd: alloc work"));
        *L.work_len = need;
    }
    return PR_OK;
}

pr_status ensure_work(pr_ctx* ctx, pr_driver* d, int64_t need) {
    if (need > d->work_len) {
        pr_dev_free(ctx, d->work);
        d->work = nullptr;
        PR_TRY_ST(alloc(ctx, (void**)&d->work, (size_t)need * 8, "svd: alloc work"));
        d->work_len = need;
    }
    return PR_OK;
}

// reduced QR of A (rows x nc, overwritten): Q in A, R (nc x nc) in Rout
pr_status qr_(pr_ctx* ctx, pr_driver* d, const Lane& L, double* A, double* Rout, int nc) {
    const int m = (int)d->rows;
    if (d->tc && nc <= kCqMaxCols) {
        // FP32 contexts: Cholesky QR twice (a few FP64 passes over A instead
        // of cuSOLVER's latency-bound Householder panels)
        const pr_status s = cholqr2_launch(A, d->rows, nc, Rout, L.cq, L.st);
        if (s != PR_OK) return pr_fail(ctx, s, "qr: Cholesky QR launch failed");
        return PR_OK;
    }
    int l1 = 0, l2 = 0;
    PR_BLAS(ctx, cusolverDnDgeqrf_bufferSize(L.sol, m, nc, A, m, &l1), "geqrf size");
    PR_BLAS(ctx, cusolverDnDorgqr_bufferSize(L.sol, m, nc, nc, A, m, L.tau, &l2), "orgqr size");
    PR_TRY_ST(ensure_lane_work(ctx, L, std::max(l1, l2)));
    PR_BLAS(ctx, cusolverDnDgeqrf(L.sol, m, nc, A, m, L.tau, *L.work, (int)*L.work_len, L.info), "geqrf");
    extract_r<<<blocks_for((int64_t)nc * nc), kT, 0, L.st>>>(A, Rout, m, nc);
    PR_BLAS(ctx, cusolverDnDorgqr(L.sol, m, nc, nc, A, m, L.tau, *L.work, (int)*L.work_len, L.info), "orgqr");
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

// Singular values below this fraction of the largest are not resolved by the
// eigenproblem of H^T H in FP64 (their squares sit at 1e-12 of the largest,
// 1e4 ulps): svd_eig_ leaves such spectra to gesvd.
constexpr double kEigFloor = 1e-6;

// SVD of H (h x h) for FP32 contexts from the symmetric eigenproblem of
// H^T H (cuSOLVER syevd, several times faster than gesvd at h ~ 500):
// H^T H = V Lambda V^T gives Y_h = V (descending order) and sigma =
// sqrt(lambda); X_h is the orthonormal polar factor of H V Sigma^-1 (one or
// two Newton-Schulz steps), which restores the orthogonality that the squared
// spectrum loses for the small sigma.  Fills
// d->Xh, d->YhT (rows 0..r-1), d->sig and `sig`; *used = false (nothing
// written) when a kept sigma lies below kEigFloor sigma_max.
pr_status svd_eig_(pr_ctx* ctx, pr_driver* d, int h, double tol, std::vector<double>& sig, int& r, bool& used,
                   cudaStream_t st) {
    const double one = 1.0, zero = 0.0;
    used = false;
    // H^T H, lower triangle only (what syevd reads): half the FP64 flops of a GEMM
    PR_BLAS(ctx, cublasDsyrk(d->blas, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, h, h, &one, d->H, h, &zero, d->E, h), "H^T H");
    int lw = 0;
    PR_BLAS(ctx, cusolverDnDsyevd_bufferSize(d->sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, h, d->E, h,
                                             d->sig, &lw), "syevd size");
    PR_TRY_ST(ensure_work(ctx, d, lw));
    PR_BLAS(ctx, cusolverDnDsyevd(d->sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, h, d->E, h, d->sig,
                                  d->work, (int)d->work_len, d->info), "syevd");
    std::vector<double> lam(h);
    int info = 0;
    cudaMemcpyAsync(lam.data(), d->sig, (size_t)h * 8, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&info, d->info, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "syevd");
    if (info != 0) return PR_OK;   // not converged: gesvd instead
    sig.assign(h, 0.0);
    for (int i = 0; i < h; ++i) sig[i] = std::sqrt(std::max(lam[h - 1 - i], 0.0));
    r = rank_cut_host(sig, tol);
    if (r > 0 && sig[r - 1] < kEigFloor * sig[0]) return PR_OK;
    used = true;
    if (r == 0) return PR_OK;
    // V (descending, r columns) into Xh, then YhT = V^T
    reverse_cols<<<blocks_for((int64_t)h * r), kT, 0, st>>>(d->E, d->Xh, h, r);
    PR_BLAS(ctx, cublasDgeam(d->blas, CUBLAS_OP_T, CUBLAS_OP_N, r, h, &one, d->Xh, h, &zero, d->Xh, r, d->YhT, h),
            "V^T");
    // X_h = the orthonormal polar factor of U0 = H V Sigma^-1.  The
    // eigenproblem leaves U0 within delta ~ u (sigma_1 / sigma_r)^2 <= 1e-4 of
    // orthonormal (sigma_r >= kEigFloor sigma_1); each Newton-Schulz step
    // X <- X (3 I - X^T X) / 2 takes delta to ~1.5 delta^2 (in place of a
    // latency-bound Householder QR).  One step when delta <= 1e-5 (FP32
    // contexts: ~1e-10 after it; every kept ratio sigma_r / sigma_1 above
    // ~5e-6, so the default rank cut of 1e-5), else two.  The Gram matrix
    // is a symmetric rank-k product and the update a symmetric multiply.
    PR_BLAS(ctx, cublasDgemm(d->blas, CUBLAS_OP_N, CUBLAS_OP_N, h, r, h, &one, d->H, h, d->Xh, h, &zero, d->E, h), "H V");
    std::vector<double> inv(r);
    for (int i = 0; i < r; ++i) inv[i] = 1.0 / sig[i];
    cudaMemcpyAsync(d->rsign, inv.data(), (size_t)r * 8, cudaMemcpyHostToDevice, st);
    scale_cols<<<blocks_for((int64_t)h * r), kT, 0, st>>>(d->E, d->rsign, d->Xh, h, r);
    const double kappa = sig[0] / sig[r - 1];
    const int ns_steps = 2.2e-16 * kappa * kappa <= 1e-5 ? 1 : 2;
    double* nsb[2] = {d->Xh, d->H};   // H is not needed past this point
    for (int step = 0; step < ns_steps; ++step) {
        double* X = nsb[step & 1];
        double* Xn = nsb[(step + 1) & 1];
        PR_BLAS(ctx, cublasDsyrk(d->blas, CUBLAS_FILL_MODE_LOWER, CUBLAS_OP_T, r, h, &one, X, h, &zero, d->E, r),
                "X^T X");
        ns_coef<<<blocks_for((int64_t)r * r), kT, 0, st>>>(d->E, r);   // the upper triangle is not read
        PR_BLAS(ctx, cublasDsymm(d->blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_LOWER, h, r, &one, d->E, r, X, h, &zero,
                                 Xn, h),
                "X (3I - X^T X)/2");
    }
    if (ns_steps == 1)   // the result is in H's storage
        cudaMemcpyAsync(d->Xh, d->H, (size_t)h * r * 8, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(d->sig, sig.data(), (size_t)h * 8, cudaMemcpyHostToDevice, st);
    e = cudaStreamSynchronize(st);   // `sig` is a host vector the copy reads
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "svd_eig");
    return PR_OK;
}

// C (rows x nc) = B^T A with B = Bb W (Bb rows x hb, W hb x s, ld bcap): C is
// s x nc, through T = Bb^T A (hb x nc)
pr_status project_(pr_ctx* ctx, pr_driver* d, const Lane& L, const double* Bb, const double* W, const double* A,
                   int nc, double* C) {
    const double one = 1.0, zero = 0.0;
    const int64_t rows = d->rows;
    if (d->tc) {
        PR_TRY_ST(tc_gram_launch(Bb, rows, A, rows, rows, d->hb, nc, L.Tb, d->hb, ctx->dev_flag, L.st));
    } else {
        PR_BLAS(ctx, cublasDgemm(L.blas, CUBLAS_OP_T, CUBLAS_OP_N, d->hb, nc, (int)rows, &one, Bb, (int)rows, A, (int)rows, &zero, L.Tb, d->hb), "Bb^T A");
    }
    PR_BLAS(ctx, cublasDgemm(L.blas, CUBLAS_OP_T, CUBLAS_OP_N, d->s, nc, d->hb, &one, W, d->bcap, L.Tb, d->hb, &zero, C, d->s), "W^T T");
    return PR_OK;
}
// A -= (Bb W) C for C (s x nc), through T = W C (hb x nc)
pr_status subtract_(pr_ctx* ctx, pr_driver* d, const Lane& L, const double* Bb, const double* W, const double* C,
                    int nc, double* A) {
    const double one = 1.0, zero = 0.0, mone = -1.0;
    const int64_t rows = d->rows;
    PR_BLAS(ctx, cublasDgemm(L.blas, CUBLAS_OP_N, CUBLAS_OP_N, d->hb, nc, d->s, &one, W, d->bcap, C, d->s, &zero, L.Tb, d->hb), "W C");
    if (d->tc) {
        PR_TRY_ST(tc_update_launch(Bb, rows, L.Tb, d->hb, A, rows, rows, d->hb, nc, A, rows, ctx->dev_flag, L.st));
    } else {
        PR_BLAS(ctx, cublasDgemm(L.blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)rows, nc, d->hb, &mone, Bb, (int)rows, L.Tb, d->hb, &one, A, (int)rows), "A - Bb T");
    }
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
    cudaEventRecord(d->cev[0], st);
    // F's steps on lane f (the caller's stream), G's on lane g, joined below
    const Lane lf = lane_f(d, st), lg = lane_g(d);
    cudaEventRecord(d->ev_fork, st);
    cudaStreamWaitEvent(d->st2, d->ev_fork, 0);
    if (s > 0) {
        // U_F = U^T F, V_G = V^T G, then F - U U_F, G - V V_G
        PR_TRY_ST(project_(ctx, d, lf, d->Xb, d->WX, F, nc, d->UF));
        PR_TRY_ST(project_(ctx, d, lg, d->Yb, d->WY, G, nc, d->VG));
        PR_TRY_ST(subtract_(ctx, d, lf, d->Xb, d->WX, d->UF, nc, F));
        PR_TRY_ST(subtract_(ctx, d, lg, d->Yb, d->WY, d->VG, nc, G));
        if (d->tc) {
            // FP32-level products: project and deflate once more (classical
            // Gram-Schmidt twice), so that Q_F, Q_G stay orthogonal to the
            // bases to working accuracy when F, G lie nearly in their span
            PR_TRY_ST(project_(ctx, d, lf, d->Xb, d->WX, F, nc, d->A1));
            PR_TRY_ST(project_(ctx, d, lg, d->Yb, d->WY, G, nc, d->A2));
            PR_TRY_ST(subtract_(ctx, d, lf, d->Xb, d->WX, d->A1, nc, F));
            PR_TRY_ST(subtract_(ctx, d, lg, d->Yb, d->WY, d->A2, nc, G));
            PR_BLAS(ctx, cublasDaxpy(lf.blas, s * nc, &one, d->A1, 1, d->UF, 1), "UF += dUF");
            PR_BLAS(ctx, cublasDaxpy(lg.blas, s * nc, &one, d->A2, 1, d->VG, 1), "VG += dVG");
        }
    }
    cudaEventRecord(d->cev[1], st);
    cudaMemcpyAsync(d->QF, F, (size_t)rows * nc * 8, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(d->QG, G, (size_t)rows * nc * 8, cudaMemcpyDeviceToDevice, d->st2);
    PR_TRY_ST(qr_(ctx, d, lf, d->QF, d->RF, nc));
    PR_TRY_ST(qr_(ctx, d, lg, d->QG, d->RG, nc));
    cudaEventRecord(d->ev_join, d->st2);
    cudaStreamWaitEvent(st, d->ev_join, 0);
    cudaEventRecord(d->cev[2], st);
    // A1 = [U_F; R_F], A2 = [V_G; R_G]  (h x nc), H = A1 A2^T + diag(S, 0)
    if (s > 0) {
        copy_block<<<blocks_for((int64_t)s * nc), kT, 0, st>>>(d->UF, s, d->A1, h, s, nc, 0);
        copy_block<<<blocks_for((int64_t)s * nc), kT, 0, st>>>(d->VG, s, d->A2, h, s, nc, 0);
    }
    copy_block<<<blocks_for((int64_t)nc * nc), kT, 0, st>>>(d->RF, nc, d->A1, h, nc, nc, s);
    copy_block<<<blocks_for((int64_t)nc * nc), kT, 0, st>>>(d->RG, nc, d->A2, h, nc, nc, s);
    PR_BLAS(ctx, cublasDgemm(d->blas, CUBLAS_OP_N, CUBLAS_OP_T, h, h, nc, &one, d->A1, h, d->A2, h, &zero, d->H, h), "H");
    if (s > 0) add_diag<<<1, kT, 0, st>>>(d->H, h, d->S, s);
    std::vector<double> sig(h);
    int r = 0;
    bool eig_used = false;
    if (d->tc) PR_TRY_ST(svd_eig_(ctx, d, h, ctx->opts.tol, sig, r, eig_used, st));
    if (!eig_used) {
        PR_TRY_ST(svd_(ctx, d, h, st));
        cudaMemcpy(sig.data(), d->sig, (size_t)h * 8, cudaMemcpyDeviceToHost);
        r = rank_cut_host(sig, ctx->opts.tol);
    }
    d->eig_svds += eig_used ? 1 : 0;
    d->all_svds += 1;
    cudaEventRecord(d->cev[3], st);
    if (r == 0) {
        d->s = 0;
        d->hb = 0;
        cudaEventRecord(d->cev[4], st);
        return PR_OK;
    }
    // U~ = [U Q_F] X_h(:, 1:r), V~ = [V Q_G] Y_h(:, 1:r)   (Y_h = YhT^T):
    // Xb <- [Xb Q_F], WX <- [WX X_h(1:s, 1:r); X_h(s+1:h, 1:r)], likewise Y
    const int hb = d->hb, ld = d->bcap;
    cudaMemcpyAsync(d->Xb + (int64_t)hb * rows, d->QF, (size_t)rows * nc * 8, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(d->Yb + (int64_t)hb * rows, d->QG, (size_t)rows * nc * 8, cudaMemcpyDeviceToDevice, st);
    if (d->Xs) {
        omega_to_f32(d->QF, d->Xs + (int64_t)hb * rows, rows * nc, st);
        omega_to_f32(d->QG, d->Ys + (int64_t)hb * rows, rows * nc, st);
    }
    if (s > 0) {
        PR_BLAS(ctx, cublasDgemm(d->blas, CUBLAS_OP_N, CUBLAS_OP_N, hb, r, s, &one, d->WX, ld, d->Xh, h, &zero, d->WXn, ld), "WX Xh");
        PR_BLAS(ctx, cublasDgemm(d->blas, CUBLAS_OP_N, CUBLAS_OP_T, hb, r, s, &one, d->WY, ld, d->YhT, h, &zero, d->WYn, ld), "WY Yh");
    }
    copy_block<<<blocks_for((int64_t)nc * r), kT, 0, st>>>(d->Xh + s, h, d->WXn, ld, nc, r, hb);
    copy_block_t<<<blocks_for((int64_t)nc * r), kT, 0, st>>>(d->YhT + (int64_t)s * h, h, d->WYn, ld, nc, r, hb);
    std::swap(d->WX, d->WXn);
    std::swap(d->WY, d->WYn);
    cudaMemcpyAsync(d->S, d->sig, (size_t)r * 8, cudaMemcpyDeviceToDevice, st);
    cudaEventRecord(d->cev[4], st);
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
    const bool f32 = d->Xs && omega_f32_supported(d->rows, d->hb) == PR_OK;
    if (f32) omega_gemv_t_f32(d->Ys, d->rows, d->hb, g, d->gs, d->tpart, d->tcnt, t1, st);
    else PR_BLAS(ctx, cublasDgemv(d->blas, CUBLAS_OP_T, (int)d->rows, d->hb, &one, d->Yb, (int)d->rows, g, 1, &zero, t1, 1), "Yb^T g");
    PR_BLAS(ctx, cublasDgemv(d->blas, CUBLAS_OP_T, d->hb, d->s, &one, d->WY, d->bcap, t1, 1, &zero, d->rwork, 1), "WY^T");
    PR_BLAS(ctx, cublasDgemv(d->blas, CUBLAS_OP_N, d->hb, d->s, &one, d->WX, d->bcap, d->rwork, 1, &zero, t2, 1), "WX");
    if (f32) omega_gemv_n_f32(d->Xs, d->rows, d->hb, t2, d->opart, out, st);
    else PR_BLAS(ctx, cublasDgemv(d->blas, CUBLAS_OP_N, (int)d->rows, d->hb, &one, d->Xb, (int)d->rows, t2, 1, &zero, out, 1), "Xb");
    return PR_OK;
}

// ||F - X Y^T G||_F and ||F||_F for the current data (F, G unmodified copies)
// into d->rnorm[1], d->rnorm[0], on lane g: a diagnostic that runs beside the
// serial sweep (which touches none of QF, UF, the bases or lane g's scratch);
// the next UpdateSVD is ordered after it through ev_join.
pr_status residual_(pr_ctx* ctx, pr_driver* d, const double* F, const double* G, int nc) {
    const int64_t rows = d->rows;
    const Lane L = lane_g(d);
    PR_BLAS(ctx, cublasSetPointerMode(L.blas, CUBLAS_POINTER_MODE_DEVICE), "pointer mode");
    PR_BLAS(ctx, cublasDnrm2(L.blas, (int)(rows * nc), F, 1, d->rnorm), "nrm2");
    // QF (rows x nc) <- F - X (Y^T G): reuse QF/UF scratch (UF has >= s*nc)
    cudaMemcpyAsync(d->QF, F, (size_t)rows * nc * 8, cudaMemcpyDeviceToDevice, L.st);
    if (d->s > 0) {
        PR_BLAS(ctx, cublasSetPointerMode(L.blas, CUBLAS_POINTER_MODE_HOST), "pointer mode");
        PR_TRY_ST(project_(ctx, d, L, d->Yb, d->WY, G, nc, d->UF));
        PR_TRY_ST(subtract_(ctx, d, L, d->Xb, d->WX, d->UF, nc, d->QF));
        PR_BLAS(ctx, cublasSetPointerMode(L.blas, CUBLAS_POINTER_MODE_DEVICE), "pointer mode");
    }
    PR_BLAS(ctx, cublasDnrm2(L.blas, (int)(rows * nc), d->QF, 1, d->rnorm + 1), "nrm2");
    PR_BLAS(ctx, cublasSetPointerMode(L.blas, CUBLAS_POINTER_MODE_HOST), "pointer mode");
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

namespace {

// What the reverse sweep of pr_iterate_adjoint needs from the forward run:
// every iteration's states and its frozen corrector Omega^k = X_k Y_k^T, kept
// as (hb_k, s_k) and copies of W_X, W_Y (X_b, Y_b only grow, so their first
// hb_k columns are still those of iteration k).
struct IterRecord {
    char* hu = nullptr;            // [(K+1)][N+1][pts] dtype: u^k_n at hu + ((k-1)(N+1) + n) pts
    char* hv = nullptr;
    std::vector<int> hb, s;        // per iteration k = 1..K
    std::vector<double*> wx, wy;   // hb_k x s_k, column-major (ld hb_k)
};

pr_status serial_sweep_(pr_ctx* ctx, pr_driver* d, int corrector, const void* Fu, const void* Fv, const void* Uc_u,
                        const void* Uc_v, void* u, void* v, cudaStream_t st);
pr_status iterate_run(pr_ctx* ctx, const void* u0, const void* p0, int K, int corrector, double tol_err,
                      const void* u_ref, const void* v_ref, void* u_slices, void* v_slices, double* err_hist,
                      double* resid_hist, int* rank_hist, int* k_done, cudaStream_t st, IterRecord* rec);

}  // namespace

extern "C" pr_status pr_serial_sweep(pr_ctx* ctx, int corrector, const void* Fu, const void* Fv, const void* Uu,
                                     const void* Uv, void* u_slices, void* v_slices, void* stream) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_serial_sweep: ctx is NULL");
    if (!Fu || !Fv || !Uu || !Uv || !u_slices || !v_slices)
        return pr_fail(ctx, PR_EINVAL, "pr_serial_sweep: NULL array");
    if (corrector < PR_CORR_PROCRUSTES || corrector > PR_CORR_PLAIN)
        return pr_fail(ctx, PR_EINVAL, "pr_serial_sweep: unknown corrector");
    if (!ctx->coarse) return pr_fail(ctx, PR_EINVAL, "pr_serial_sweep: context has no coarse grid");
    {
        const size_t esz = ctx->dtype == PR_F32 ? 4 : 8;
        const size_t fb = (size_t)ctx->N * ctx->pts * esz, cb = (size_t)ctx->N * ctx->coarse->pts * esz;
        const char* lo[2] = {(const char*)u_slices + ctx->pts * esz, (const char*)v_slices + ctx->pts * esz};
        const char* in[4] = {(const char*)Fu, (const char*)Fv, (const char*)Uu, (const char*)Uv};
        const size_t ib[4] = {fb, fb, cb, cb};
        auto hit = [](const char* a, size_t na, const char* b, size_t nb) { return a < b + nb && b < a + na; };
        if (hit(lo[0], fb, lo[1], fb)) return pr_fail(ctx, PR_EINVAL, "pr_serial_sweep: u_slices and v_slices overlap");
        for (int i = 0; i < 4; ++i)
            for (int o = 0; o < 2; ++o)
                if (hit(in[i], ib[i], lo[o], fb))
                    return pr_fail(ctx, PR_EINVAL, "pr_serial_sweep: an input overlaps output slices 1..N");
    }
    cudaStream_t st = (cudaStream_t)stream;
    pr_driver* d = nullptr;
    PR_TRY_ST(driver(ctx, st, &d));
    PR_TRY_ST(serial_sweep_(ctx, d, corrector, Fu, Fv, Uu, Uv, u_slices, v_slices, st));
    PR_TRY_ST(pr_take_flag(ctx->coarse, ctx, st, "pr_serial_sweep (coarse propagation)"));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "pr_serial_sweep");
    return PR_OK;
}

extern "C" pr_status pr_iterate(pr_ctx* ctx, const void* u0, const void* p0, int K, int corrector,
                                double tol_err, const void* u_ref, const void* v_ref, void* u_slices,
                                void* v_slices, double* err_hist, double* resid_hist, int* rank_hist,
                                int* k_done, void* stream) {
    return iterate_run(ctx, u0, p0, K, corrector, tol_err, u_ref, v_ref, u_slices, v_slices, err_hist, resid_hist,
                       rank_hist, k_done, (cudaStream_t)stream, nullptr);
}

namespace {

// The serial corrected sweep of Alg. 3: for n = 1..N, w = C R u_{n-1} and
// u_n = F_n + I(correction), the correction w - U_n (plain), or Lambda^dagger
// of Lambda w - Lambda U_n (Omega = 1) or of Omega (Lambda w - Lambda U_n)
// (Procrustes), with the zero mode sum w - sum U_n (A8, by linearity).  F
// ([N][pts]) holds F u^k_{n-1}, U ([N][cpts]) C R u^k_{n-1}; u, v ([N+1][pts])
// hold u^{k+1}_0 in slice 0 and receive slices 1..N.
pr_status serial_sweep_(pr_ctx* ctx, pr_driver* d, int corrector, const void* Fu, const void* Fv, const void* Uc_u,
                        const void* Uc_v, void* u, void* v, cudaStream_t st) {
    const size_t esz = ctx->dtype == PR_F32 ? 4 : 8;
    const int64_t pts = ctx->pts, cpts = d->cpts;
    auto fu = [&](int n) { return (char*)u + (size_t)n * pts * esz; };
    auto fv = [&](int n) { return (char*)v + (size_t)n * pts * esz; };
    for (int n = 1; n <= ctx->N; ++n) {
        PR_TRY_ST(coarse_of(ctx, fu(n - 1), fv(n - 1), d->w_u, d->w_v, 1, st));
        const void* Uu = (const char*)Uc_u + (size_t)(n - 1) * cpts * esz;
        const void* Uv = (const char*)Uc_v + (size_t)(n - 1) * cpts * esz;
        if (corrector == PR_CORR_PLAIN) {
            coarse_to_zc(ctx, d, d->w_u, d->w_v, Uu, Uv, st);
        } else {
            lambda_diff_(ctx, d, d->w_u, d->w_v, Uu, Uv, st);
            const double* g = d->dvec;
            if (corrector == PR_CORR_PROCRUSTES) {
                PR_TRY_ST(apply_omega(ctx, d, d->dvec, d->gvec, st));
                g = d->gvec;
            }
            PR_TRY_ST(reconstruct_(ctx, d, g, st));
        }
        const size_t vo = (size_t)(n - 1) * pts * esz;
        PR_TRY_ST(interp_(ctx, d, (const char*)Fu + vo, (const char*)Fv + vo, fu(n), fv(n), st));
    }
    return PR_OK;
}

pr_status iterate_run(pr_ctx* ctx, const void* u0, const void* p0, int K, int corrector, double tol_err,
                      const void* u_ref, const void* v_ref, void* u_slices, void* v_slices, double* err_hist,
                      double* resid_hist, int* rank_hist, int* k_done, cudaStream_t st, IterRecord* rec) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_iterate: ctx is NULL");
    if (!u0 || !p0 || !u_slices || !v_slices) return pr_fail(ctx, PR_EINVAL, "pr_iterate: NULL array");
    if (K < 0) return pr_fail(ctx, PR_EINVAL, "pr_iterate: K must be >= 0");
    if (corrector < PR_CORR_PROCRUSTES || corrector > PR_CORR_PLAIN)
        return pr_fail(ctx, PR_EINVAL, "pr_iterate: unknown corrector");
    pr_driver* d = nullptr;
    PR_TRY_ST(driver(ctx, st, &d));
    d->s = 0;   // a new run starts with an empty correlation matrix (Alg. 3)
    d->hb = 0;
    for (int i = 0; i < 4; ++i) {
        d->phase_ms[i] = 0.0;
        if (!d->ev[i]) PR_CUDA_TRY(ctx, cudaEventCreate(&d->ev[i]));
    }
    for (int i = 0; i < 5; ++i) d->corr_ms[i] = 0.0;
    d->eig_svds = d->all_svds = 0;
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
    // the forward record: states of iteration k (k = 1: the initial guess)
    auto record_states = [&](int k) {
        if (!rec) return;
        const size_t b = (size_t)(N + 1) * pts * esz, o = (size_t)(k - 1) * b;
        cudaMemcpyAsync(rec->hu + o, us, b, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(rec->hv + o, vs, b, cudaMemcpyDeviceToDevice, st);
    };
    record_states(1);
    for (int k = 1; k <= K; ++k) {
        // parallel phase: v_n = F u^k_{n-1}, U_n = C R u^k_{n-1}, n = 1..N
        cudaEventRecord(d->ev[0], st);
        pr_status s = pr_fine_all_slices(ctx, fu(0), fv(0), d->vF_u, d->vF_v, 0, N, st);
        if (s != PR_OK) return s;
        PR_TRY_ST(coarse_of(ctx, fu(0), fv(0), d->Uc_u, d->Uc_v, N, st));
        cudaEventRecord(d->ev[1], st);
        double res = 0.0;
        bool resid_pending = false;
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
            // the residual diagnostic on lane g, beside the serial sweep
            cudaEventRecord(d->ev_fork, st);
            cudaStreamWaitEvent(d->st2, d->ev_fork, 0);
            PR_TRY_ST(residual_(ctx, d, d->F2, d->G2, N));
            cudaEventRecord(d->cev[5], d->st2);
            cudaEventRecord(d->ev_join, d->st2);
            resid_pending = true;
            if (rec) {
                // freeze Omega^k: the W blocks (hb x s, ld bcap) as they are now
                double* wx = nullptr;
                double* wy = nullptr;
                const size_t wb = (size_t)std::max(1, d->hb) * std::max(1, d->s) * 8;
                PR_TRY_ST(alloc(ctx, (void**)&wx, wb, "pr_iterate_adjoint: record"));
                rec->wx.push_back(wx);
                PR_TRY_ST(alloc(ctx, (void**)&wy, wb, "pr_iterate_adjoint: record"));
                rec->wy.push_back(wy);
                rec->hb.push_back(d->hb);
                rec->s.push_back(d->s);
                if (d->s > 0) {
                    cudaMemcpy2DAsync(wx, (size_t)d->hb * 8, d->WX, (size_t)d->bcap * 8, (size_t)d->hb * 8, d->s,
                                      cudaMemcpyDeviceToDevice, st);
                    cudaMemcpy2DAsync(wy, (size_t)d->hb * 8, d->WY, (size_t)d->bcap * 8, (size_t)d->hb * 8, d->s,
                                      cudaMemcpyDeviceToDevice, st);
                }
            }
        }
        cudaEventRecord(d->ev[2], st);
        // serial corrected sweep; u^{k+1}_0 = u^k_0 stays
        PR_TRY_ST(serial_sweep_(ctx, d, corrector, d->vF_u, d->vF_v, d->Uc_u, d->Uc_v, us, vs, st));
        cudaEventRecord(d->ev[3], st);
        if (resid_pending) {
            // the next iteration's UpdateSVD reuses the residual's scratch
            cudaStreamWaitEvent(st, d->ev_join, 0);
            double nrm[2] = {0.0, 0.0};
            PR_CUDA_TRY(ctx, cudaEventSynchronize(d->cev[5]));
            PR_CUDA_TRY(ctx, cudaMemcpy(nrm, d->rnorm, sizeof nrm, cudaMemcpyDeviceToHost));
            res = nrm[0] > 0 ? nrm[1] / nrm[0] : 0.0;
            for (int i = 0; i < 5; ++i) {
                float ms = 0.0f;
                PR_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, d->cev[i], d->cev[i + 1]));
                d->corr_ms[i] += ms;
            }
            resid_pending = false;
        }
        record_states(k + 1);
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

}  // namespace

extern "C" pr_status pr_iterate_corrector_phases(const pr_ctx* ctx, double* ms, int* eig_svds, int* svds) {
    if (!ctx || !ms) return PR_EINVAL;
    for (int i = 0; i < 5; ++i) ms[i] = ctx->drv ? ctx->drv->corr_ms[i] : 0.0;
    if (eig_svds) *eig_svds = ctx->drv ? ctx->drv->eig_svds : 0;
    if (svds) *svds = ctx->drv ? ctx->drv->all_svds : 0;
    return PR_OK;
}

extern "C" pr_status pr_iterate_phases(const pr_ctx* ctx, double* ms) {
    if (!ctx || !ms) return PR_EINVAL;
    for (int i = 0; i < 4; ++i) ms[i] = ctx->drv ? ctx->drv->phase_ms[i] : 0.0;
    return PR_OK;
}

// ============================================================================
// Adjoint of the parareal solve with the correctors frozen (pr_iterate_adjoint)
//
// The paper does not differentiate its method.  Every iteration's corrector
// Omega^k = X_k Y_k^T is held at the value the forward run computed (Alg. 1
// on its data), so the map (u0, p0, c) -> u^{K+1}_N is a composition of F, C
// (Sec. 3.1), R, I (Sec. 6), Lambda, Lambda^dagger (Sec. 3.4, Alg. 2) and
// fixed matrices.  The reverse sweep applies their transposes in reverse
// order:
//   R^T     scatter onto the coarse nodes of a zero fine field;
//   I^T     with I = Re(G_f^* P G_c) (G the unnormalised DFT, P the padding
//           with the Nyquist split and the 1/N_Dx scale): Re(G_c P^T G_f^* y);
//   Lambda^T [q; p] = [-sum_a D_a q_a ; p / c], D_a the central difference;
//   Lambda^dagger^T: q_a = Re(G D_a G^* w) / N_Dx with D_a = -i xi_a / |xi|^2,
//           zero mode sum(w) / N_Dx, p = c w_t;
//   Omega^T = Y X^T;  F^T, C^T the transposed level recurrence (adjoint.cu).
// dL/dc collects the fine kappa term, the coarse kappa term and the c
// dependence of Lambda (c^-1 w_t) and Lambda^dagger (c p), the coarse terms
// scattered back by R^T (the coarse c is R c).
// ============================================================================
namespace {

template <typename S, typename D, int DIM>
__global__ void restrict_T_add(const S* __restrict__ a, const S* __restrict__ b, D* __restrict__ fa,
                               D* __restrict__ fb, int64_t n, int ratio, int64_t cpts) {
    const int64_t nc = n / ratio;
    for (int64_t J = (int64_t)blockIdx.x * kT + threadIdx.x; J < cpts; J += (int64_t)gridDim.x * kT) {
        int64_t c[3];
        coords<DIM>(J, nc, c);
#pragma unroll
        for (int q = 0; q < DIM; ++q) c[q] *= ratio;
        const int64_t f = lin<DIM>(c, n);
        fa[f] = (D)((double)fa[f] + (double)a[J]);
        if (b) fb[f] = (D)((double)fb[f] + (double)b[J]);
    }
}

template <typename T>
__global__ void fine_pair_to_complex(const T* __restrict__ a, const T* __restrict__ b,
                                     cufftDoubleComplex* __restrict__ z, int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x; j < m; j += (int64_t)gridDim.x * kT) {
        z[j] = make_cuDoubleComplex((double)a[j], 0.0);
        z[m + j] = make_cuDoubleComplex((double)b[j], 0.0);
    }
}

// P^T of interp_pad: coarse coefficient (fld, J) = sum over the fine indices
// that interp_pad fills from it, with the same weights (1/cpts included)
template <int DIM>
__global__ void interp_pad_T(const cufftDoubleComplex* __restrict__ fs, cufftDoubleComplex* __restrict__ cs,
                             int64_t nc, int64_t nf, int64_t cpts, int64_t fpts) {
    const double scale = 1.0 / (double)cpts;
    const int64_t half = nc / 2;
    for (int64_t idx = (int64_t)blockIdx.x * kT + threadIdx.x; idx < 2 * cpts; idx += (int64_t)gridDim.x * kT) {
        const int64_t fld = idx / cpts, J = idx - fld * cpts;
        int64_t c[3];
        coords<DIM>(J, nc, c);
        // per axis: up to two fine indices with their weights
        int64_t fi[3][2];
        double fw[3][2];
        int cnt[3];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const int64_t j = c[a];
            cnt[a] = 1;
            fw[a][0] = 1.0;
            fw[a][1] = 0.0;
            fi[a][1] = 0;
            if (nc % 2 == 0) {
                if (j < half) fi[a][0] = j;
                else if (j > half) fi[a][0] = j - nc + nf;
                else {
                    fi[a][0] = half;
                    fw[a][0] = 0.5;
                    fi[a][1] = nf - half;
                    fw[a][1] = 0.5;
                    cnt[a] = 2;
                }
            } else {
                fi[a][0] = j <= half ? j : j - nc + nf;
            }
        }
        double re = 0.0, im = 0.0;
        const int combos = 1 << DIM;
        for (int m = 0; m < combos; ++m) {
            double w = scale;
            int64_t f[3];
            bool ok = true;
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const int bit = (m >> a) & 1;
                if (bit >= cnt[a]) ok = false;
                f[a] = fi[a][bit];
                w *= fw[a][bit];
            }
            if (!ok) continue;
            const cufftDoubleComplex x = fs[fld * fpts + lin<DIM>(f, nf)];
            re += w * x.x;
            im += w * x.y;
        }
        cs[idx] = make_cuDoubleComplex(re, im);
    }
}

__global__ void complex_real_pair(const cufftDoubleComplex* __restrict__ z, double* __restrict__ a,
                                  double* __restrict__ b, int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x; j < m; j += (int64_t)gridDim.x * kT) {
        a[j] = z[j].x;
        b[j] = z[m + j].x;
    }
}

// Z[a][J] = D_a(J) B[J], D_a = -i xi_a / |xi|^2 (0 at xi = 0), a < DIM
template <int DIM>
__global__ void grad2func_T_spread(const cufftDoubleComplex* __restrict__ B, cufftDoubleComplex* __restrict__ Z,
                                   int64_t nc, int64_t cpts) {
    for (int64_t J = (int64_t)blockIdx.x * kT + threadIdx.x; J < cpts; J += (int64_t)gridDim.x * kT) {
        int64_t c[3];
        coords<DIM>(J, nc, c);
        double xi[3], mag2 = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            xi[a] = 2.0 * M_PI * (double)freq(c[a], nc);
            mag2 += xi[a] * xi[a];
        }
        const cufftDoubleComplex b = B[J];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            // (-i xi / m)(x + i y) = xi y / m - i xi x / m
            Z[a * cpts + J] = mag2 > 0 ? make_cuDoubleComplex(xi[a] * b.y / mag2, -xi[a] * b.x / mag2)
                                       : make_cuDoubleComplex(0.0, 0.0);
        }
    }
}

// q[a*cpts + J] = Re(Z[a][J]) / cpts, the vector part of Lambda^dagger^T;
// q[DIM*cpts + J] = c_J bdut_J; bcc_J += bdut_J p_J (the c in u_t = c p)
template <int DIM>
__global__ void grad2func_T_finish(const cufftDoubleComplex* __restrict__ Z, const double* __restrict__ bdut,
                                   const double* __restrict__ cc, const double* __restrict__ pvec,
                                   double* __restrict__ q, double* __restrict__ bcc, int64_t cpts) {
    const double inv = 1.0 / (double)cpts;
    for (int64_t J = (int64_t)blockIdx.x * kT + threadIdx.x; J < cpts; J += (int64_t)gridDim.x * kT) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) q[a * cpts + J] = Z[a * cpts + J].x * inv;
        q[DIM * cpts + J] = cc[J] * bdut[J];
        bcc[J] += bdut[J] * pvec[J];
    }
}

// sum_J x_J / cpts into *out (one block, fixed order)
__global__ void mean_kernel(const double* __restrict__ x, int64_t cpts, double* __restrict__ out) {
    __shared__ double red[1024];
    double acc = 0.0;
    for (int64_t j = threadIdx.x; j < cpts; j += blockDim.x) acc += x[j];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] / (double)cpts;
}

// Lambda^T of q (rows = (DIM+1) cpts) for the difference Lambda w - Lambda U:
// bw = -sum_a D_a q_a + z, bwt = p / c, written to (bw, bwt) of w (dtype T)
// and subtracted from (bU, bUt) of U; bcc -= p (wt - Ut) / c^2.
template <typename T, int DIM>
__global__ void lambda_T_diff(const double* __restrict__ q, const double* __restrict__ cc, const T* __restrict__ wt,
                              const T* __restrict__ Ut, const double* __restrict__ zmode, T* __restrict__ bw,
                              T* __restrict__ bwt, T* __restrict__ bU, T* __restrict__ bUt, double* __restrict__ bcc,
                              int64_t nc, int64_t cpts, int order_half, Beta beta, double inv_dx) {
    for (int64_t J = (int64_t)blockIdx.x * kT + threadIdx.x; J < cpts; J += (int64_t)gridDim.x * kT) {
        int64_t c[3];
        coords<DIM>(J, nc, c);
        double g = 0.0;
        int64_t astride = 1;
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const double* qa = q + a * cpts;
            for (int k = 1; k <= order_half; ++k) {
                const int64_t cp = (c[a] + k) % nc, cm = (c[a] - k + nc) % nc;
                const double qp = qa[J + (cp - c[a]) * astride], qm = qa[J + (cm - c[a]) * astride];
                g += beta.b[k - 1] * (qm - qp);
            }
            astride *= nc;
        }
        const double vw = g * inv_dx + *zmode;
        const double p = q[DIM * cpts + J];
        const double vt = p / cc[J];
        bw[J] = (T)vw;
        bwt[J] = (T)vt;
        bU[J] = (T)((double)bU[J] - vw);
        bUt[J] = (T)((double)bUt[J] - vt);
        bcc[J] -= p * ((double)wt[J] - (double)Ut[J]) / (cc[J] * cc[J]);
    }
}

template <typename T>
__global__ void axpy_kernel(T* __restrict__ y, const T* __restrict__ x, double a, int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x; j < m; j += (int64_t)gridDim.x * kT)
        y[j] = (T)((double)y[j] + a * (double)x[j]);
}

template <typename T>
__global__ void from_double_kernel(T* __restrict__ y, const double* __restrict__ x, int64_t m) {
    for (int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x; j < m; j += (int64_t)gridDim.x * kT) y[j] = (T)x[j];
}

// gc_J (fine, FP64) = gk_J * 2 c_J scale
__global__ void kappa_to_c(const double* __restrict__ gk, const double* __restrict__ c, double* __restrict__ gc,
                           int64_t m, double scale, int accumulate) {
    for (int64_t j = (int64_t)blockIdx.x * kT + threadIdx.x; j < m; j += (int64_t)gridDim.x * kT)
        gc[j] = (accumulate ? gc[j] : 0.0) + gk[j] * 2.0 * c[j] * scale;
}

template <typename T>
struct AdjWork {
    T *bu = nullptr, *bv = nullptr;      // [N+1][pts] adjoints of u^{k+1}_n
    T *nu = nullptr, *nv = nullptr;      // [N+1][pts] adjoints of u^k_n (being formed)
    T *fvu = nullptr, *fvv = nullptr;    // [N][pts] adjoints of v_n = F u^k_{n-1}
    T *cU = nullptr, *cV = nullptr;      // [N][cpts] adjoints of U_n = C R u^k_{n-1}
    T *iu = nullptr, *iv = nullptr;      // [pts] adjoint of u^1_0 gathered from every u^{k+1}_0
    T *wu = nullptr, *wv = nullptr;      // [cpts] adjoint of w = C R u^{k+1}_{n-1}
    T *Ru = nullptr, *Rv = nullptr;      // [cpts] R of a fine state
    T *tu = nullptr, *tv = nullptr;      // [cpts] scratch
    double *gkf = nullptr, *gkc = nullptr, *bcc = nullptr;   // dL/dkappa fine, coarse; Lambda c terms
    double *bdu = nullptr, *bdut = nullptr, *q = nullptr, *zm = nullptr, *gcf = nullptr;
    std::vector<void*> all;
};

template <typename T>
pr_status adj_alloc(pr_ctx* ctx, AdjWork<T>& w, int64_t N, int64_t pts, int64_t cpts, int64_t rows) {
    auto get = [&](auto** p, size_t bytes) -> pr_status {
        void* q = nullptr;
        PR_TRY_ST(alloc(ctx, &q, bytes, "pr_iterate_adjoint: workspace"));
        cudaMemset(q, 0, bytes);
        w.all.push_back(q);
        *p = (std::remove_reference_t<decltype(*p)>)q;
        return PR_OK;
    };
    const size_t e = sizeof(T);
    PR_TRY_ST(get(&w.bu, (N + 1) * pts * e)); PR_TRY_ST(get(&w.bv, (N + 1) * pts * e));
    PR_TRY_ST(get(&w.nu, (N + 1) * pts * e)); PR_TRY_ST(get(&w.nv, (N + 1) * pts * e));
    PR_TRY_ST(get(&w.fvu, N * pts * e)); PR_TRY_ST(get(&w.fvv, N * pts * e));
    PR_TRY_ST(get(&w.cU, N * cpts * e)); PR_TRY_ST(get(&w.cV, N * cpts * e));
    PR_TRY_ST(get(&w.iu, pts * e)); PR_TRY_ST(get(&w.iv, pts * e));
    PR_TRY_ST(get(&w.wu, cpts * e)); PR_TRY_ST(get(&w.wv, cpts * e));
    PR_TRY_ST(get(&w.Ru, cpts * e)); PR_TRY_ST(get(&w.Rv, cpts * e));
    PR_TRY_ST(get(&w.tu, cpts * e)); PR_TRY_ST(get(&w.tv, cpts * e));
    PR_TRY_ST(get(&w.gkf, pts * 8)); PR_TRY_ST(get(&w.gkc, cpts * 8)); PR_TRY_ST(get(&w.bcc, cpts * 8));
    PR_TRY_ST(get(&w.bdu, cpts * 8)); PR_TRY_ST(get(&w.bdut, cpts * 8)); PR_TRY_ST(get(&w.q, rows * 8));
    PR_TRY_ST(get(&w.zm, 8)); PR_TRY_ST(get(&w.gcf, pts * 8));
    return PR_OK;
}

// Omega^k g or (Omega^k)^T g with the frozen W blocks of iteration k
pr_status apply_frozen(pr_ctx* ctx, pr_driver* d, const IterRecord& rec, int k, bool transpose, const double* g,
                       double* out, cudaStream_t st) {
    const int hb = rec.hb[k - 1], s = rec.s[k - 1];
    if (s == 0) {
        cudaMemsetAsync(out, 0, (size_t)d->rows * 8, st);
        return PR_OK;
    }
    const double one = 1.0, zero = 0.0;
    double* t1 = d->vb;
    double* t2 = d->vb + d->bcap;
    const double* Bin = transpose ? d->Xb : d->Yb;    // Omega = Xb WX WY^T Yb^T; Omega^T = Yb WY WX^T Xb^T
    const double* Bout = transpose ? d->Yb : d->Xb;
    const double* Win = transpose ? rec.wx[k - 1] : rec.wy[k - 1];
    const double* Wout = transpose ? rec.wy[k - 1] : rec.wx[k - 1];
    PR_BLAS(ctx, cublasDgemv(d->blas, CUBLAS_OP_T, (int)d->rows, hb, &one, Bin, (int)d->rows, g, 1, &zero, t1, 1), "frozen Omega: B^T g");
    PR_BLAS(ctx, cublasDgemv(d->blas, CUBLAS_OP_T, hb, s, &one, Win, hb, t1, 1, &zero, d->rwork, 1), "frozen Omega: W^T");
    PR_BLAS(ctx, cublasDgemv(d->blas, CUBLAS_OP_N, hb, s, &one, Wout, hb, d->rwork, 1, &zero, t2, 1), "frozen Omega: W");
    PR_BLAS(ctx, cublasDgemv(d->blas, CUBLAS_OP_N, (int)d->rows, hb, &one, Bout, (int)d->rows, t2, 1, &zero, out, 1), "frozen Omega: B");
    return PR_OK;
}

template <typename T, int DIM>
pr_status adjoint_run(pr_ctx* ctx, pr_driver* d, const IterRecord& rec, int K, int corrector, const T* guT,
                      const T* gvT, T* gc, T* gu0, T* gp0, cudaStream_t st) {
    const int64_t pts = ctx->pts, cpts = d->cpts, nc = d->nc, n = ctx->n;
    const int N = ctx->N;
    pr_ctx* cc = ctx->coarse;
    AdjWork<T> w;
    pr_status status = adj_alloc<T>(ctx, w, N, pts, cpts, d->rows);
    auto release = [&]() {
        cudaStreamSynchronize(st);
        for (void* p : w.all) pr_dev_free(ctx, p);
    };
    if (status != PR_OK) {
        release();
        return status;
    }
    auto fail = [&](pr_status s) {
        release();
        return s;
    };
#define PR_ADJ_TRY(x) do { pr_status s_ = (x); if (s_ != PR_OK) return fail(s_); } while (0)
    auto hu = [&](int k, int nn) { return (const T*)(rec.hu + ((size_t)(k - 1) * (N + 1) + nn) * pts * sizeof(T)); };
    auto hv = [&](int k, int nn) { return (const T*)(rec.hv + ((size_t)(k - 1) * (N + 1) + nn) * pts * sizeof(T)); };
    auto F_ = [&](T* base, int nn) { return base + (size_t)nn * pts; };
    auto C_ = [&](T* base, int nn) { return base + (size_t)nn * cpts; };
    const int h = ctx->opts.grad_order / 2;
    const double inv_dxc = 1.0 / cc->dx;
    // R u (coarse dtype) of a fine state into (Ru, Rv)
    auto R_of = [&](const T* u, const T* v) { return restrict_(ctx, u, v, w.Ru, w.Rv, 1, st); };
    // (fa, fb) += R^T (a, b)
    auto RT_add = [&](const T* a, const T* b, T* fa, T* fb) {
        restrict_T_add<T, T, DIM><<<blocks_for(cpts), kT, 0, st>>>(a, b, fa, fb, n, ctx->ratio, cpts);
    };
    // (bdu, bdut) (coarse FP64) = I^T (y_u, y_v) (fine dtype)
    auto IT = [&](const T* yu, const T* yv) -> pr_status {
        fine_pair_to_complex<T><<<blocks_for(pts), kT, 0, st>>>(yu, yv, d->zf, pts);
        PR_FFT(ctx, cufftExecZ2Z(d->plan_f2, d->zf, d->zf, CUFFT_INVERSE), "I^T fine inverse");
        interp_pad_T<DIM><<<blocks_for(2 * cpts), kT, 0, st>>>(d->zf, d->zc, nc, n, cpts, pts);
        PR_FFT(ctx, cufftExecZ2Z(d->plan_c2, d->zc, d->zc, CUFFT_FORWARD), "I^T coarse forward");
        complex_real_pair<<<blocks_for(cpts), kT, 0, st>>>(d->zc, w.bdu, w.bdut, cpts);
        return PR_OK;
    };
    // adjoint of w = C R (su, sv) with incoming (au, av) (coarse dtype, consumed):
    // (fu, fv) += R^T C^T (au, av), gkc += dL/dkappa_c
    auto CRT = [&](const T* su, const T* sv, T* au, T* av, T* fu, T* fv) -> pr_status {
        PR_TRY_ST(R_of(su, sv));
        PR_TRY_ST(pr_slice_adjoint(cc, w.Ru, w.Rv, au, av, w.gkc, st));
        RT_add(au, av, fu, fv);
        return PR_OK;
    };
    cudaMemcpyAsync(F_(w.bu, N), guT, pts * sizeof(T), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(F_(w.bv, N), gvT, pts * sizeof(T), cudaMemcpyDeviceToDevice, st);
    for (int k = K; k >= 1; --k) {
        cudaMemsetAsync(w.fvu, 0, (size_t)N * pts * sizeof(T), st);
        cudaMemsetAsync(w.fvv, 0, (size_t)N * pts * sizeof(T), st);
        cudaMemsetAsync(w.cU, 0, (size_t)N * cpts * sizeof(T), st);
        cudaMemsetAsync(w.cV, 0, (size_t)N * cpts * sizeof(T), st);
        // serial corrected sweep of iteration k, in reverse
        for (int nn = N; nn >= 1; --nn) {
            T* bsu = F_(w.bu, nn);
            T* bsv = F_(w.bv, nn);
            // u^{k+1}_n = v_n + I(du, dut)
            axpy_kernel<T><<<blocks_for(pts), kT, 0, st>>>(F_(w.fvu, nn - 1), bsu, 1.0, pts);
            axpy_kernel<T><<<blocks_for(pts), kT, 0, st>>>(F_(w.fvv, nn - 1), bsv, 1.0, pts);
            PR_ADJ_TRY(IT(bsu, bsv));
            // w = C R u^{k+1}_{n-1} and U_n = C R u^k_{n-1}, recomputed
            PR_ADJ_TRY(coarse_of(ctx, hu(k + 1, nn - 1), hv(k + 1, nn - 1), d->w_u, d->w_v, 1, st));
            PR_ADJ_TRY(coarse_of(ctx, hu(k, nn - 1), hv(k, nn - 1), w.tu, w.tv, 1, st));
            T* bUu = C_(w.cU, nn - 1);
            T* bUv = C_(w.cV, nn - 1);
            if (corrector == PR_CORR_PLAIN) {
                // du = w - U_n: the adjoint of w is (bdu, bdut), of U_n minus it
                from_double_kernel<T><<<blocks_for(cpts), kT, 0, st>>>(w.wu, w.bdu, cpts);
                from_double_kernel<T><<<blocks_for(cpts), kT, 0, st>>>(w.wv, w.bdut, cpts);
                axpy_kernel<T><<<blocks_for(cpts), kT, 0, st>>>(bUu, w.wu, -1.0, cpts);
                axpy_kernel<T><<<blocks_for(cpts), kT, 0, st>>>(bUv, w.wv, -1.0, cpts);
            } else {
                // forward quantities: d = Lambda w - Lambda U_n, g = Omega d (its p block feeds dL/dc)
                lambda_(ctx, d->w_u, d->w_v, d->dvec, 1, d->nc, cpts, 1.0, 1, d->rows, st);
                lambda_(ctx, w.tu, w.tv, d->dvec, 1, d->nc, cpts, -1.0, 1, d->rows, st);
                const double* g = d->dvec;
                if (corrector == PR_CORR_PROCRUSTES) {
                    PR_ADJ_TRY(apply_frozen(ctx, d, rec, k, false, d->dvec, d->gvec, st));
                    g = d->gvec;
                }
                // Lambda^dagger^T of (bdu, bdut) for the difference
                real_to_complex<<<blocks_for(cpts), kT, 0, st>>>(w.bdu, d->zc, cpts);
                PR_FFT(ctx, cufftExecZ2Z(d->plan_c1, d->zc, d->zc, CUFFT_INVERSE), "Lambda^dagger^T inverse");
                grad2func_T_spread<DIM><<<blocks_for(cpts), kT, 0, st>>>(d->zc, d->zc + cpts, nc, cpts);
                PR_FFT(ctx, cufftExecZ2Z(d->plan_cd, d->zc + cpts, d->zc + cpts, CUFFT_FORWARD), "Lambda^dagger^T forward");
                grad2func_T_finish<DIM><<<blocks_for(cpts), kT, 0, st>>>(d->zc + cpts, w.bdut, cc->c64,
                                                                          g + (int64_t)DIM * cpts, w.q, w.bcc, cpts);
                mean_kernel<<<1, 1024, 0, st>>>(w.bdu, cpts, w.zm);
                double* qv = w.q;
                if (corrector == PR_CORR_PROCRUSTES) {
                    PR_ADJ_TRY(apply_frozen(ctx, d, rec, k, true, w.q, d->gvec, st));
                    qv = d->gvec;
                }
                lambda_T_diff<T, DIM><<<blocks_for(cpts), kT, 0, st>>>(qv, cc->c64, (const T*)d->w_v, w.tv, w.zm,
                                                                      w.wu, w.wv, bUu, bUv, w.bcc, nc, cpts, h,
                                                                      d->beta, inv_dxc);
            }
            // w = C R u^{k+1}_{n-1}
            PR_ADJ_TRY(CRT(hu(k + 1, nn - 1), hv(k + 1, nn - 1), w.wu, w.wv, F_(w.bu, nn - 1), F_(w.bv, nn - 1)));
        }
        // u^{k+1}_0 = u^1_0
        axpy_kernel<T><<<blocks_for(pts), kT, 0, st>>>(w.iu, F_(w.bu, 0), 1.0, pts);
        axpy_kernel<T><<<blocks_for(pts), kT, 0, st>>>(w.iv, F_(w.bv, 0), 1.0, pts);
        // parallel phase of iteration k: v_n = F u^k_{n-1}, U_n = C R u^k_{n-1}
        cudaMemsetAsync(w.nu, 0, (size_t)(N + 1) * pts * sizeof(T), st);
        cudaMemsetAsync(w.nv, 0, (size_t)(N + 1) * pts * sizeof(T), st);
        for (int nn = 1; nn <= N; ++nn) {
            PR_ADJ_TRY(pr_slice_adjoint(ctx, hu(k, nn - 1), hv(k, nn - 1), F_(w.fvu, nn - 1), F_(w.fvv, nn - 1),
                                        w.gkf, st));
            axpy_kernel<T><<<blocks_for(pts), kT, 0, st>>>(F_(w.nu, nn - 1), F_(w.fvu, nn - 1), 1.0, pts);
            axpy_kernel<T><<<blocks_for(pts), kT, 0, st>>>(F_(w.nv, nn - 1), F_(w.fvv, nn - 1), 1.0, pts);
            PR_ADJ_TRY(CRT(hu(k, nn - 1), hv(k, nn - 1), C_(w.cU, nn - 1), C_(w.cV, nn - 1), F_(w.nu, nn - 1),
                           F_(w.nv, nn - 1)));
        }
        std::swap(w.bu, w.nu);
        std::swap(w.bv, w.nv);
    }
    // the initial guess u^1_n = I C R u^1_{n-1}, in reverse
    for (int nn = N; nn >= 1; --nn) {
        PR_ADJ_TRY(IT(F_(w.bu, nn), F_(w.bv, nn)));
        from_double_kernel<T><<<blocks_for(cpts), kT, 0, st>>>(w.wu, w.bdu, cpts);
        from_double_kernel<T><<<blocks_for(cpts), kT, 0, st>>>(w.wv, w.bdut, cpts);
        PR_ADJ_TRY(CRT(hu(1, nn - 1), hv(1, nn - 1), w.wu, w.wv, F_(w.bu, nn - 1), F_(w.bv, nn - 1)));
    }
    axpy_kernel<T><<<blocks_for(pts), kT, 0, st>>>(F_(w.bu, 0), w.iu, 1.0, pts);
    axpy_kernel<T><<<blocks_for(pts), kT, 0, st>>>(F_(w.bv, 0), w.iv, 1.0, pts);
    cudaMemcpyAsync(gu0, F_(w.bu, 0), pts * sizeof(T), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(gp0, F_(w.bv, 0), pts * sizeof(T), cudaMemcpyDeviceToDevice, st);
    // dL/dc: fine kappa term, then R^T of the coarse kappa and Lambda terms
    kappa_to_c<<<blocks_for(pts), kT, 0, st>>>(w.gkf, ctx->c64, w.gcf, pts, ctx->dt_f / (ctx->dx * ctx->dx), 0);
    kappa_to_c<<<blocks_for(cpts), kT, 0, st>>>(w.gkc, cc->c64, w.bcc, cpts, cc->dt_f / (cc->dx * cc->dx), 1);
    restrict_T_add<double, double, DIM><<<blocks_for(cpts), kT, 0, st>>>(w.bcc, nullptr, w.gcf, nullptr, n,
                                                                         ctx->ratio, cpts);
    from_double_kernel<T><<<blocks_for(pts), kT, 0, st>>>(gc, w.gcf, pts);
    cudaError_t e = cudaGetLastError();
    release();
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "pr_iterate_adjoint");
    return PR_OK;
#undef PR_ADJ_TRY
}

}  // namespace

extern "C" pr_status pr_iterate_adjoint(pr_ctx* ctx, const void* u0, const void* p0, int K, int corrector,
                                        const void* gu_T, const void* gv_T, void* gc, void* gu0, void* gp0,
                                        void* stream) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_iterate_adjoint: ctx is NULL");
    if (!u0 || !p0 || !gu_T || !gv_T || !gc || !gu0 || !gp0)
        return pr_fail(ctx, PR_EINVAL, "pr_iterate_adjoint: NULL array");
    if (K < 1) return pr_fail(ctx, PR_EINVAL, "pr_iterate_adjoint: K must be >= 1");
    if (corrector < PR_CORR_PROCRUSTES || corrector > PR_CORR_PLAIN)
        return pr_fail(ctx, PR_EINVAL, "pr_iterate_adjoint: unknown corrector");
    if (!ctx->coarse) return pr_fail(ctx, PR_EINVAL, "pr_iterate_adjoint: no coarse grid");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t esz = ctx->dtype == PR_F32 ? 4 : 8;
    const int N = ctx->N;
    const size_t slab = (size_t)(N + 1) * ctx->pts * esz;
    IterRecord rec;
    void* us = nullptr;
    void* vs = nullptr;
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);
        pr_dev_free(ctx, rec.hu);
        pr_dev_free(ctx, rec.hv);
        pr_dev_free(ctx, us);
        pr_dev_free(ctx, vs);
        for (double* p : rec.wx) pr_dev_free(ctx, p);
        for (double* p : rec.wy) pr_dev_free(ctx, p);
    };
    pr_status s = PR_OK;
    if (pr_dev_malloc(ctx, (void**)&rec.hu, slab * (K + 1)) != cudaSuccess ||
        pr_dev_malloc(ctx, (void**)&rec.hv, slab * (K + 1)) != cudaSuccess || pr_dev_malloc(ctx, &us, slab) != cudaSuccess ||
        pr_dev_malloc(ctx, &vs, slab) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return pr_fail(ctx, PR_ENOMEM, "pr_iterate_adjoint: state history");
    }
    int kd = 0;
    s = iterate_run(ctx, u0, p0, K, corrector, 0.0, nullptr, nullptr, us, vs, nullptr, nullptr, nullptr, &kd, st, &rec);
    if (s == PR_OK && kd != K) s = pr_fail(ctx, PR_ECUDA, "pr_iterate_adjoint: forward run stopped early");
    if (s == PR_OK) {
        pr_driver* d = ctx->drv;
        const bool f32 = ctx->dtype == PR_F32;
        switch (ctx->dim) {
            case 1: s = f32 ? adjoint_run<float, 1>(ctx, d, rec, K, corrector, (const float*)gu_T, (const float*)gv_T, (float*)gc, (float*)gu0, (float*)gp0, st)
                            : adjoint_run<double, 1>(ctx, d, rec, K, corrector, (const double*)gu_T, (const double*)gv_T, (double*)gc, (double*)gu0, (double*)gp0, st); break;
            case 2: s = f32 ? adjoint_run<float, 2>(ctx, d, rec, K, corrector, (const float*)gu_T, (const float*)gv_T, (float*)gc, (float*)gu0, (float*)gp0, st)
                            : adjoint_run<double, 2>(ctx, d, rec, K, corrector, (const double*)gu_T, (const double*)gv_T, (double*)gc, (double*)gu0, (double*)gp0, st); break;
            default: s = f32 ? adjoint_run<float, 3>(ctx, d, rec, K, corrector, (const float*)gu_T, (const float*)gv_T, (float*)gc, (float*)gu0, (float*)gp0, st)
                             : adjoint_run<double, 3>(ctx, d, rec, K, corrector, (const double*)gu_T, (const double*)gv_T, (double*)gc, (double*)gu0, (double*)gp0, st); break;
        }
    }
    if (s == PR_OK) s = pr_take_flag(ctx, ctx, st, "pr_iterate_adjoint (fine sweep)");
    if (s == PR_OK && ctx->coarse) s = pr_take_flag(ctx->coarse, ctx, st, "pr_iterate_adjoint (coarse sweep)");
    cleanup();
    return s;
}
