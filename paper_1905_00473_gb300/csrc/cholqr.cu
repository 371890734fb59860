// Tall-skinny QR of the deflated snapshot blocks by Cholesky QR, twice
// (CholeskyQR2), in FP64: the reduced QR that Alg. 1 (UpdateSVD, Sec. 3.3.1)
// takes of the part of the new columns outside the current basis.
//
// A (rows x nc, column-major, nc <= 64) is overwritten by Q and R (nc x nc,
// column-major, upper, zeros below the diagonal) is written, A = Q R.  One
// pass: G = A^T A, G = R^T R (Cholesky), A <- A R^-1; the second pass
// repeats it on the first pass's Q, which is orthonormal to O(u kappa(A)^2),
// and R = R2 R1.  Five launches in all, every product on the FP64 pipes.
//
// A column whose Cholesky pivot falls to tau * max_j G_jj or below lies in
// the span of the earlier ones to working accuracy: its row of R and its
// column of Q are set to zero.  Alg. 1 only needs A = Q R with the nonzero
// columns of Q orthonormal: a zero row of R is a zero row of the h x h core
// matrix, whose left singular vectors for nonzero singular values then have
// no component on it, so the zero column of Q never enters the bases.
// (Householder QR instead returns an arbitrary unit vector there, with a
// near-zero diagonal entry in R: the same after the rank cut.)
#include <algorithm>
#include <cstdint>

#include "pr_internal.cuh"

namespace {

constexpr int kCqT = 256;       // threads of the row-chunk kernels
constexpr int kCqRows = 32;     // rows per chunk
constexpr int kCqLd = kCqRows + 1;
constexpr int kCqPairs = (kCqMaxCols * (kCqMaxCols + 1) / 2 + kCqT - 1) / kCqT;   // pairs per thread

// Upper-triangle pair p (column-major packed: (0,0), (0,1), (1,1), (0,2), ...)
__device__ __forceinline__ void cq_pair(int p, int& i, int& j) {
    int c = (int)((sqrt(8.0 * p + 1.0) - 1.0) * 0.5);
    while (c * (c + 1) / 2 > p) --c;
    while ((c + 1) * (c + 2) / 2 <= p) ++c;
    j = c;
    i = p - c * (c + 1) / 2;
}

// One streaming pass over the rows of A in chunks of kCqRows:
//   Rinv != nullptr: the chunk becomes chunk * Rinv (upper, nc x nc) and is
//                    written to Out (may be A itself: a CTA reads a whole
//                    chunk before it writes it);
//   G != nullptr:    the Gram matrix of the (transformed) chunk is added to G
//                    (upper triangle, column-major nc x nc, FP64 atomics).
__global__ void __launch_bounds__(kCqT) cq_pass(const double* A, double* Out, int64_t rows, int nc,
                                                 const double* __restrict__ Rinv, double* __restrict__ G) {
    extern __shared__ double cq_sm[];
    double* T = cq_sm;               // [nc][kCqLd]
    double* T2 = T + nc * kCqLd;     // [nc][kCqLd]
    double* Ri = T2 + nc * kCqLd;    // [nc][nc]
    const int tid = threadIdx.x;
    if (Rinv)
        for (int idx = tid; idx < nc * nc; idx += kCqT) Ri[idx] = Rinv[idx];
    const int np = nc * (nc + 1) / 2;
    int pi[kCqPairs], pj[kCqPairs];
    double acc[kCqPairs];
#pragma unroll
    for (int q = 0; q < kCqPairs; ++q) {
        acc[q] = 0.0;
        pi[q] = pj[q] = 0;
        if (tid + q * kCqT < np) cq_pair(tid + q * kCqT, pi[q], pj[q]);
    }
    __syncthreads();
    const double* src = Rinv ? T2 : T;
    for (int64_t r0 = (int64_t)blockIdx.x * kCqRows; r0 < rows; r0 += (int64_t)gridDim.x * kCqRows) {
        for (int idx = tid; idx < nc * kCqRows; idx += kCqT) {
            const int c = idx / kCqRows, rr = idx - c * kCqRows;
            const int64_t row = r0 + rr;
            T[c * kCqLd + rr] = row < rows ? A[(int64_t)c * rows + row] : 0.0;
        }
        __syncthreads();
        if (Rinv) {
            // T2[c][rr] = sum_{k <= c} T[k][rr] Rinv[k][c]; a warp shares c
            const int rr = tid & 31;
            for (int c = tid >> 5; c < nc; c += kCqT / 32) {
                double s = 0.0;
                for (int k = 0; k <= c; ++k) s = fma(T[k * kCqLd + rr], Ri[k + c * nc], s);
                T2[c * kCqLd + rr] = s;
            }
            __syncthreads();
            for (int idx = tid; idx < nc * kCqRows; idx += kCqT) {
                const int c = idx / kCqRows, rr = idx - c * kCqRows;
                const int64_t row = r0 + rr;
                if (row < rows) Out[(int64_t)c * rows + row] = T2[c * kCqLd + rr];
            }
        }
        if (G) {
#pragma unroll
            for (int q = 0; q < kCqPairs; ++q) {
                if (tid + q * kCqT < np) {
                    const double* a = src + pi[q] * kCqLd;
                    const double* b = src + pj[q] * kCqLd;
                    double s = acc[q];
#pragma unroll 8
                    for (int rr = 0; rr < kCqRows; ++rr) s = fma(a[rr], b[rr], s);
                    acc[q] = s;
                }
            }
        }
        __syncthreads();
    }
    if (G) {
#pragma unroll
        for (int q = 0; q < kCqPairs; ++q)
            if (tid + q * kCqT < np) atomicAdd(&G[pi[q] + pj[q] * nc], acc[q]);
    }
}

// Cholesky G = R^T R of the upper triangle of G (nc x nc), with the pivot
// guard above; writes R^-1 (zero rows and columns at the dropped pivots) and
// Rout = R Rprev (or R when Rprev is null), then zeroes G for the next pass.
__global__ void __launch_bounds__(kCqT) cq_chol(double* __restrict__ G, int nc, double tau,
                                                 double* __restrict__ Rinv, const double* __restrict__ Rprev,
                                                 double* __restrict__ Rout) {
    extern __shared__ double cq_sm[];
    double* S = cq_sm;          // [nc][nc]
    double* R = S + nc * nc;    // [nc][nc]
    __shared__ double gmax;
    __shared__ int null_j;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < nc * nc; idx += kCqT) {
        const int j = idx / nc, i = idx - j * nc;
        S[idx] = i <= j ? G[idx] : 0.0;
        R[idx] = 0.0;
    }
    __syncthreads();
    for (int idx = tid; idx < nc * nc; idx += kCqT) G[idx] = 0.0;
    if (tid == 0) {
        double m = 0.0;
        for (int j = 0; j < nc; ++j) m = fmax(m, S[j + j * nc]);
        gmax = m;
    }
    __syncthreads();
    for (int j = 0; j < nc; ++j) {
        if (tid == 0) {
            const double piv = S[j + j * nc];
            null_j = !(piv > tau * gmax) || !(gmax > 0.0);
            R[j + j * nc] = null_j ? 0.0 : sqrt(piv);
        }
        __syncthreads();
        const bool nul = null_j != 0;
        const double d = R[j + j * nc];
        for (int k = j + 1 + tid; k < nc; k += kCqT) R[j + k * nc] = nul ? 0.0 : S[j + k * nc] / d;
        __syncthreads();
        if (!nul) {
            // trailing update of the upper triangle: S[k][l] -= R[j][k] R[j][l], j < k <= l
            const int m = nc - j - 1;
            for (int p = tid; p < m * (m + 1) / 2; p += kCqT) {
                int a, b;
                cq_pair(p, a, b);
                const int k = j + 1 + a, l = j + 1 + b;
                S[k + l * nc] -= R[j + k * nc] * R[j + l * nc];
            }
        }
        __syncthreads();
    }
    // column c of R^-1 by back substitution (thread c)
    if (tid < nc) {
        const int c = tid;
        double x[kCqMaxCols];
        for (int i = 0; i < nc; ++i) x[i] = 0.0;
        const double dc = R[c + c * nc];
        x[c] = dc != 0.0 ? 1.0 / dc : 0.0;
        for (int i = c - 1; i >= 0; --i) {
            const double di = R[i + i * nc];
            if (di == 0.0) continue;
            double s = 0.0;
            for (int k = i + 1; k <= c; ++k) s = fma(R[i + k * nc], x[k], s);
            x[i] = -s / di;
        }
        for (int i = 0; i < nc; ++i) Rinv[i + c * nc] = x[i];
    }
    // Rout = R Rprev (both upper)
    for (int idx = tid; idx < nc * nc; idx += kCqT) {
        const int j = idx / nc, i = idx - j * nc;
        double s = 0.0;
        if (i <= j) {
            if (Rprev) {
                for (int k = i; k <= j; ++k) s = fma(R[i + k * nc], Rprev[k + j * nc], s);
            } else {
                s = R[idx];
            }
        }
        Rout[idx] = s;
    }
}

}  // namespace

pr_status cholqr2_launch(double* A, int64_t rows, int nc, double* R, double* ws, cudaStream_t st) {
    if (nc < 1 || nc > kCqMaxCols || rows < 1) return PR_EINVAL;
    // workspace: G, Rinv, R1 (nc x nc each); G is zero on entry and on return
    double* G = ws;
    double* Rinv = ws + kCqMaxCols * kCqMaxCols;
    double* R1 = Rinv + kCqMaxCols * kCqMaxCols;
    const size_t smem = (size_t)(2 * nc * kCqLd + nc * nc) * 8;   // <= 66.5 KB
    const size_t smem_c = (size_t)2 * nc * nc * 8;                  // <= 64 KB
    if (cudaFuncSetAttribute(cq_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(cq_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_c) != cudaSuccess)
        return PR_ECUDA;
    const int64_t chunks = (rows + kCqRows - 1) / kCqRows;
    const int grid = (int)std::min<int64_t>(chunks, 2 * 152);
    // Pivots at or below tau * max G_jj (about a 1e-7 ratio of singular values)
    // are dropped: CholeskyQR2 is accurate for kappa up to ~u^-1/2.
    const double tau = 1e-14;
    cq_pass<<<grid, kCqT, smem, st>>>(A, A, rows, nc, nullptr, G);
    cq_chol<<<1, kCqT, smem_c, st>>>(G, nc, tau, Rinv, nullptr, R1);
    cq_pass<<<grid, kCqT, smem, st>>>(A, A, rows, nc, Rinv, G);
    cq_chol<<<1, kCqT, smem_c, st>>>(G, nc, tau, Rinv, R1, R);
    cq_pass<<<grid, kCqT, smem, st>>>(A, A, rows, nc, Rinv, nullptr);
    return cudaGetLastError() == cudaSuccess ? PR_OK : PR_ECUDA;
}
