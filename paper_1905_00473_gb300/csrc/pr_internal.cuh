// Internal declarations of the pr library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pr.h"

struct pr_ctx {
    int device = 0;
    int dim = 0;
    int64_t n = 0;            // fine points per axis
    int64_t pts = 0;          // n^dim
    int ratio = 1;
    int N = 0;                // slices
    int dtype = PR_F32;
    double T = 0, dt_com = 0, dt_f = 0, dt_c = 0, dx = 0;
    int m_f = 0, m_c = 0;
    int block_depth = 1;      // fine steps (kicks) per HBM pass
    int tb_cols = 0;          // fused 2D kernel: columns per thread (0 = default, 4)
    double cmax = 0;
    void* kappa = nullptr;    // dtype, c^2 dt_f / dx^2
    float* kappa_il = nullptr;  // 2D FP32: kappa per thread pair [y][x/2][k0 k1 0 0] (fine_tb2d_c2.cu)
    double* cinv2 = nullptr;  // FP64 c^-2 (energy weights)
    double* c64 = nullptr;    // FP64 c at the nodes of this grid
    pr_options opts = {PR_F32, 4, 0, 1e-13, 0, 0};
    pr_ctx* coarse = nullptr;         // the coarse propagator's context (C, Sec. 3.1)
    struct pr_driver* drv = nullptr;  // Alg. 3 driver state (parareal.cu), lazily created
    void* adj_ws = nullptr;           // pr_adjoint workspace (adjoint.cu), lazily created
    int debug_stall = 0;              // pr_debug_stall_waits (tests of the time-out path)
    size_t adj_bytes = 0;
    void* sadj_ws = nullptr;          // one-slice adjoint workspace (adjoint.cu), lazily created
    size_t sadj_bytes = 0;
    // ping-pong state between passes, [N][pts] each: u, v (dtype), r (the
    // residual: resid_bytes per point, 2 where a fused 2D sweep may run)
    void* su[2] = {nullptr, nullptr};
    void* sv[2] = {nullptr, nullptr};
    void* sr[2] = {nullptr, nullptr};
    int resid_bytes = 0;
    double* partials = nullptr;     // energy partial sums
    int64_t partials_len = 0;
    int* dev_flag = nullptr;        // device-side error flag (bounded waits)
    unsigned int* sweep_ctr = nullptr;   // grid-barrier counter of the one-launch sweep
    int one_launch = 0;             // run a supported sweep as one persistent launch (pr_set_one_launch)
    pr_alloc_fn ualloc = nullptr;     // the caller allocator at creation (pr_set_allocator), or cudaMalloc
    pr_release_fn urelease = nullptr;
    void* uarg = nullptr;
    int wide_rows = 2;              // n = 2048 at depth 8: 1 cluster rows, 2 x-strips (pr_set_wide_rows)
    int resident = -1;              // slices held in one cluster's shared memory: -1 auto (n <= 128), 0 off, 1 on
    std::string err;
    // pr_profile: event pairs around launches, by kernel kind
    bool prof_on = false;
    struct ProfRec { int kind; cudaEvent_t a, b; };
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
};

// ---- device memory owned by a context ------------------------------------------
// Through the caller allocator the context was created with, else cudaMalloc /
// cudaFree.  pr_dev_free synchronises the device before it hands memory to a
// caller allocator (cudaFree does so implicitly); NULL is a no-op.
cudaError_t pr_dev_malloc(const pr_ctx* ctx, void** p, size_t bytes);
void pr_dev_free(const pr_ctx* ctx, void* p);
// the process-wide pair that pr_create records into new contexts
void pr_current_allocator(pr_alloc_fn* a, pr_release_fn* r, void** user);

// ---- context construction / driver teardown ---------------------------------
pr_status pr_build_ctx(int dim, int64_t n, int ratio, int N, double T, double dt, int m,
                       double dt_c, int m_c, const pr_options& o, const std::vector<double>& c,
                       pr_ctx** out);
void pr_driver_free(pr_ctx* ctx);

// ---- adjoint of one slice (adjoint.cu) ---------------------------------------
// Reverse of the m_f + 1 levels of one slice of context c (fine or coarse)
// started from (u_in, v_in): (lu, lv) hold the adjoints of the slice's end
// state on entry and of its start state on return (dtype, [pts]); dL/dkappa
// is added to gk (FP64, [pts]).
pr_status pr_slice_adjoint(pr_ctx* c, const void* u_in, const void* v_in, void* lu, void* lv, double* gk,
                           cudaStream_t st);

// ---- snapshot products on the tensor cores (gram_tc.cu, split-TF32) -------------
// C (M x N, ldc) = A^T B, A (K x M, lda), B (K x N, ldb); C is overwritten.
pr_status tc_gram_launch(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t K, int64_t M, int N,
                         double* C, int64_t ldc, int* flag, cudaStream_t st);
// O (M x N, ldo) = F - A T, A (M x K, lda), T (K x N, ldt); O may equal F.
pr_status tc_update_launch(const double* A, int64_t lda, const double* T, int64_t ldt, const double* F, int64_t ldf,
                           int64_t M, int64_t K, int N, double* O, int64_t ldo, int* flag, cudaStream_t st);

// ---- tall-skinny QR (cholqr.cu) ----------------------------------------------
// A (rows x nc, column-major, nc <= kCqMaxCols) <- Q, R (nc x nc, column-major,
// upper) with A = Q R, by Cholesky QR twice in FP64; columns dependent on the
// earlier ones to working accuracy get a zero row of R and a zero column of Q.
// ws: 3 * kCqMaxCols^2 doubles, zero-filled before the first call (it is left
// zero-filled).
constexpr int kCqMaxCols = 64;
pr_status cholqr2_launch(double* A, int64_t rows, int nc, double* R, double* ws, cudaStream_t st);

// ---- the Procrustes corrector applied with FP32 copies of the bases (omega_f32.cu)
// Stored columns hb <= kOmMaxCols, rows % 4 == 0 (PR_EINVAL otherwise).
constexpr int kOmJ = 16;             // column chunks of the out = Xs t2 product
constexpr int kOmR = 4;              // row parts of the t1 = Ys^T g product
constexpr int kOmMaxCols = 8192;
pr_status omega_f32_supported(int64_t rows, int hb);
void omega_to_f32(const double* a, float* b, int64_t m, cudaStream_t st);
// t1 (hb, FP64) = Ys^T g, Ys rows x hb FP32 column-major; scratch: gs (rows
// floats), part (kOmR * kOmMaxCols doubles), cnt (kOmMaxCols / 2 counters,
// zero-filled before the first call; left zero-filled)
void omega_gemv_t_f32(const float* Ys, int64_t rows, int hb, const double* g, float* gs, double* part,
                      unsigned* cnt, double* t1, cudaStream_t st);
// out (rows, FP64) = Xs t2; part: kOmJ * rows doubles of scratch
void omega_gemv_n_f32(const float* Xs, int64_t rows, int hb, const double* t2, double* part, double* out,
                      cudaStream_t st);

// ---- status helpers --------------------------------------------------------
pr_status pr_fail(pr_ctx* ctx, pr_status st, const std::string& msg);
pr_status pr_cuda_fail(pr_ctx* ctx, cudaError_t e, const char* what);
// Read (after the work queued on st) and clear ctx's device-side error flag;
// PR_ETIMEOUT with the message recorded on `report` if a bounded wait gave up.
// Synchronises st.
pr_status pr_take_flag(pr_ctx* ctx, pr_ctx* report, cudaStream_t st, const char* where);

#define PR_CUDA_TRY(ctx, call)                                   \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return pr_cuda_fail(ctx, e_, #call); \
    } while (0)

// ---- the rounding-residual byte -------------------------------------------
// Between HBM passes the FP32 displacement is stored as u_hi (float) plus a
// signed byte q carrying the rounding residual r = (u0 + du) - u_hi in units
// of 2^(E-31), E the exponent of u_hi, i.e. ulp(u_hi)/256 (|r| <= ulp/2, so
// |q| <= 128; the convert saturates at [-128, 127]).  The scale is a power of
// two built from u_hi's exponent field (clamped below at 2^-95 so that it is
// always a normal number), so encode and decode are exact apart from the
// rounding of q itself: the stored displacement keeps ~33 significant bits.
__device__ __forceinline__ uint32_t pr_resid_efield(float uhi) {
    return max(__float_as_uint(uhi) & 0x7f800000u, 32u << 23);
}
__device__ __forceinline__ float pr_resid_decode(int8_t q, float uhi) {
    return (float)q * __uint_as_float(pr_resid_efield(uhi) - (31u << 23));
}
// s = fl(a + b) and the exact rounding error r = (a + b) - s (TwoSum, Knuth).
__device__ __forceinline__ float pr_two_sum(float a, float b, float* r) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    *r = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}
// Round u0 + du to float and encode the rounding error as the byte above.
__device__ __forceinline__ float pr_sum_encode(float u0, float du, int8_t* q) {
    float r;
    const float s = pr_two_sum(u0, du, &r);
    const float inv = __uint_as_float((285u << 23) - pr_resid_efield(s));  // 2^(31-E)
    int qi;
    asm("cvt.rni.sat.s8.f32 %0, %1;" : "=r"(qi) : "f"(__fmul_rn(r, inv)));
    *q = (int8_t)qi;
    return s;
}

// ---- the bfloat16 residual (sweeps with fused 2D passes) --------------------
// The temporally blocked 2D kernel keeps r itself, rounded to bfloat16: the
// float's exponent range with 8 significant bits, so |r - r_b| <= 2^-9 |r|
// <= ulp(u_hi)/1024 (half the byte format's worst case) and no scale is
// needed: decode is a shift, encode one convert per two values.  It costs a
// second byte per point per pass, which the fused kernel (bound by issue, not
// HBM) pays for with the instructions it saves; one-level sweeps, which are
// HBM-bound, keep the byte.
enum pr_resid_fmt { PR_RESID_I8 = 0, PR_RESID_BF16 = 1 };
__device__ __forceinline__ float pr_bf16_decode(uint32_t h) { return __uint_as_float(h << 16); }
// the two halves of a packed pair
__device__ __forceinline__ float pr_bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float pr_bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
// two residuals packed as bf16 pairs: lo in bits 0..15, hi in 16..31
__device__ __forceinline__ uint32_t pr_bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
// overloads for kernels templated on the residual type
__device__ __forceinline__ float pr_resid_get(int8_t q, float uhi) { return pr_resid_decode(q, uhi); }
__device__ __forceinline__ float pr_resid_get(uint16_t h, float) { return pr_bf16_decode(h); }
__device__ __forceinline__ float pr_resid_put(float u0, float du, int8_t* q) { return pr_sum_encode(u0, du, q); }
__device__ __forceinline__ float pr_resid_put(float u0, float du, uint16_t* h) {
    float r;
    const float s = pr_two_sum(u0, du, &r);
    *h = (uint16_t)pr_bf16x2(r, 0.0f);
    return s;
}

// ---- kernels launched by the API -------------------------------------------
struct pr_pass {
    // state in: u (dtype), v (dtype), r (FP32 only; null = zero residual)
    const void* u_in;
    const void* v_in;
    const void* r_in;
    // state out: r_out null on the last pass (residual folded into u)
    void* u_out;
    void* v_out;
    void* r_out;
    int rfmt;             // pr_resid_fmt of r_in / r_out
    int nslices;          // slices in this launch (pointers already offset)
    int g0;               // global kick index of the first level
    int levels;           // kicks in this pass
    int m;                // steps per slice (kick m is the final half kick)
};

// one kick(+drift) per launch, any dim/dtype (the reference path of the library)
pr_status pr_launch_fine_naive(pr_ctx* ctx, const pr_pass& p, cudaStream_t st);
// 2D FP32 temporally blocked streaming kernel; returns PR_EINVAL if the
// geometry is not supported (caller falls back to the naive path)
bool pr_tb2d_supported(const pr_ctx* ctx, int depth);
pr_status pr_launch_fine_tb2d(pr_ctx* ctx, const pr_pass& p, cudaStream_t st);
// whether the fused kernel takes a pass of block_depth + 1 levels (the last)
bool pr_tb2d_extra_level(const pr_ctx* ctx);
// the same passes with two columns per thread (16 warps per SM at n = 1024)
pr_status pr_launch_fine_tb2d_c2(pr_ctx* ctx, const pr_pass& p, cudaStream_t st);

// A whole sweep of fused passes in one persistent (cooperative) launch, a
// grid barrier between passes (fine_tb2d.cu): `passes` passes of 8 levels,
// the last one of last_levels (<= 9); pass scratch ping-pongs through su/sv/sr.
struct pr_sweep {
    const void* u_in;
    const void* v_in;
    void* u_out;
    void* v_out;
    void* su[2];
    void* sv[2];
    void* sr[2];
    int nslices, passes, last_levels;
};
bool pr_tb2d_sweep_supported(const pr_ctx* ctx, int passes);
// 3D FP32 temporally blocked kernel (fine_tb3d.cu): passes of 2..4 levels
bool pr_tb3d_supported(const pr_ctx* ctx, int depth);

// ---- the batch as one persistent work-queue kernel (batch_queue.cu) ----------
// Every fused pass of every slice (x-strip at n = 2048) of every instance is
// an item of a device queue claimed by one CTA per SM; pass k of a slice
// waits (bounded) for all items of pass k - 1 of that slice.  Instances: 2D
// FP32, n in {256, 512, 1024, 2048}, m_f >= 8, a bfloat16 residual scratch.
struct pr_queue;
bool pr_queue_supported(const pr_ctx* c);
pr_status pr_queue_create(int count, pr_ctx* const* ctx, const void* const* ui, const void* const* vi,
                          void* const* uo, void* const* vo, pr_queue** out);
pr_status pr_queue_launch(pr_queue* q, cudaStream_t st);   // counter reset + one launch; capturable
void pr_queue_destroy(pr_queue* q);

// ---- whole slices in one cluster's shared memory (resident2d.cu) ------------
// 2D FP32 grids up to 256^2 at block depth 8: all m + 1 kicks of each slice in
// one launch (a cluster of 8 CTAs per slice), bit-identical to the per-pass
// fused kernels.
bool pr_resident2d_supported(const pr_ctx* ctx);
pr_status pr_launch_resident2d(pr_ctx* ctx, const void* u_in, const void* v_in, void* u_out, void* v_out,
                               int nslices, cudaStream_t st);
pr_status pr_launch_fine_tb3d(pr_ctx* ctx, const pr_pass& p, cudaStream_t st);
pr_status pr_launch_fine_tb2d_sweep(pr_ctx* ctx, const pr_sweep& sw, cudaStream_t st);
pr_status pr_launch_energy(pr_ctx* ctx, const void* u, const void* v, int nslices,
                           double* e_host, cudaStream_t st);
