/*
 * pr.h -- C ABI of the GB300 parallel-in-time wave propagator.
 *
 * The library implements the data-parallel hot path of the stable
 * parareal-like method of Nguyen & Tsai, "A stable parareal-like method for
 * the second order wave equation" (arXiv 1905.00473): the fine propagator F
 * applied independently to every time slice of one parareal iteration
 * (Alg. 3, the parFor over n), for
 *
 *     u_tt = c(x)^2 Lap u  on the periodic unit box [0,1)^d   (Sec. 1, eq. waveequation)
 *
 * discretised, as in Sec. 3.1, by the 2nd-order central-difference Laplacian
 * on a uniform grid and velocity Verlet in time.
 *
 * Conventions shared by every entry point
 *  - All array arguments are DEVICE pointers on the context's device, in the
 *    context's dtype (float for PR_F32, double for PR_F64), unless stated.
 *  - A field on an n^d grid is stored row-major with x fastest:
 *    [z][y][x] (3D), [y][x] (2D), [x] (1D); "pts" = n^d.
 *    A batch of slices is [N][pts], slice-contiguous.
 *  - Pointers must be 16-byte aligned (torch allocations are).
 *  - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL is the
 *    legacy default stream) and is asynchronous w.r.t. the host.  Caller
 *    buffers are borrowed for the duration of the enqueued work.
 *  - No exception or abort crosses the ABI.  Every call returns a pr_status;
 *    on failure pr_last_error() holds a message.  Invalid arguments are
 *    rejected with PR_EINVAL before anything is launched.
 *  - A context is not thread-safe: serialise calls on one context.
 */
#ifndef PR_H
#define PR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pr_status {
    PR_OK = 0,
    PR_EINVAL = 1,      /* invalid argument; nothing was launched */
    PR_ENOMEM = 2,      /* device allocation failed */
    PR_ECUDA = 3,       /* a CUDA runtime call or a launch failed */
    PR_ETIMEOUT = 4,    /* a bounded device-side wait gave up (see pr_check) */
    PR_EUNSTABLE = 5,   /* pr_iterate: the energy of the state at T is not finite */
    PR_ENOTCONV = 6     /* reserved: iteration did not reach its tolerance */
} pr_status;

typedef enum pr_dtype { PR_F32 = 0, PR_F64 = 1 } pr_dtype;

/* Fine grid of the periodic unit box.  dim in {1,2,3}; nf[0..dim-1] are the
 * fine points per axis (x, y, z) and must be equal (dx = 1/nf on every axis,
 * Sec. 3.1 "uniform Cartesian grids"); ratio = coarse spacing / fine spacing
 * (coarse nodes coincide with fine nodes, Sec. 6), nf % ratio == 0. */
typedef struct pr_grid {
    int dim;
    int64_t nf[3];
    int ratio;
} pr_grid;

/* Options.  block_depth: fine steps fused per HBM pass of the 2D FP32 kernel
 * (0 = library default: 8; 8 or 4 use the fused kernel where it applies:
 * n = 128, 256, 512, 1024 and 2048, whose rows are shared by a two-CTA
 * cluster at depth 8 and split into x-strips at depth 4; 1 = one step per
 * pass).  Other fields are reserved for the coarse/correction stages and are
 * ignored by the fine path. */
typedef struct pr_options {
    int dtype;          /* pr_dtype */
    int grad_order;     /* 2, 4, 6, 8 or 0 = spectral (nabla_h, Sec. 6.4) */
    int interp;         /* 0 = Fourier (interpft, Sec. 6) */
    double tol;         /* rank tolerance of Alg. 1 */
    int block_depth;
    int max_iters;
} pr_options;

typedef struct pr_ctx pr_ctx;

/* pr_create -- set up one problem (Sec. 3.1: grids, steps, medium).
 *
 *  grid   fine grid (see pr_grid).
 *  c_dev  DEVICE pointer, dtype of opts->dtype, nf^dim wave-speed values
 *         c(x_j) > 0 at the fine nodes.  Read during the call only; the
 *         context keeps its own coefficient array kappa_j = c_j^2 dt_f/dx^2.
 *  dt_f   fine step delta t; dt_c coarse step Delta t.
 *  N      number of time slices (coupling intervals); T final time.
 *         Delta t_com = T/N.  m_F = Delta t_com/dt_f and m_C = Delta t_com/dt_c
 *         must be integers (Sec. 3.1, "m_F, m_C in N"), within 1e-9 relative.
 *  opts   may be NULL (defaults: F32, 4th-order nabla_h, Fourier I, tol 1e-13).
 *  out    receives the context.
 *
 * Checks the CFL condition of the Verlet/central-difference pair,
 * max c * dt * sqrt(dim) / dx <= 1, on both grids (PR_EINVAL if violated).
 * Reads c back on a private stream ordered after the work already queued on
 * the legacy default stream (write c there, or synchronise the stream that
 * wrote it, before the call); no other stream is waited for.
 */
pr_status pr_create(const pr_grid* grid, const void* c_dev, double dt_f, double dt_c, int N,
                    double T, const pr_options* opts, pr_ctx** out);

/* pr_destroy -- free the context and all device memory it owns (NULL is a no-op). */
void pr_destroy(pr_ctx* ctx);

/* Caller allocator (ownership: the context owns kappa, the pass scratch,
 * snapshot stores, SVD factors and workspaces; these can come from the
 * caller's pool, e.g. PyTorch's caching allocator, instead of cudaMalloc).
 *  alloc(bytes, device, user)  returns device memory of at least `bytes`
 *                              bytes on `device` (the current device), or
 *                              NULL on failure (reported as PR_ECUDA);
 *  release(ptr, user)          gives it back.
 * pr_set_allocator installs the pair process-wide for contexts created
 * afterwards; each context keeps the pair it was created with, so a context
 * and its frees always use the same allocator.  Both NULL restores
 * cudaMalloc / cudaFree; exactly one NULL is PR_EINVAL.  Not synchronised
 * with concurrent pr_create calls.  Before it hands memory back the library
 * synchronises the device (cudaFree does the same implicitly), so released
 * memory is idle.  Workspaces that cuFFT, cuBLAS and cuSOLVER allocate
 * inside their own handles and plans are not routed through the pair. */
typedef void* (*pr_alloc_fn)(size_t bytes, int device, void* user);
typedef void (*pr_release_fn)(void* ptr, void* user);
pr_status pr_set_allocator(pr_alloc_fn alloc, pr_release_fn release, void* user);

/* pr_last_error -- message of the last failing call on ctx (never NULL).
 * With ctx == NULL returns the last error of pr_create on this thread. */
const char* pr_last_error(const pr_ctx* ctx);

/* pr_fine_all_slices -- the fine propagator F on a batch of slices
 * (Alg. 3: [v_n, v_t n] = F[u^k_{n-1}, u_t^k_{n-1}] for all n, in parallel).
 *
 *  u_in, v_in    [N][pts] displacement u and velocity u_t at the start of
 *                each slice.
 *  u_out, v_out  [N][pts] results after m_F velocity-Verlet steps of dt_f
 *                (one coupling interval Delta t_com).
 *  n_begin,n_end slices [n_begin, n_end) are propagated, 0 <= n_begin <= n_end <= N;
 *                other slices of the outputs are not touched.
 *  stream        cudaStream_t.
 * out == in (u_out == u_in and v_out == v_in) is allowed; any other overlap
 * between inputs and outputs is rejected (PR_EINVAL).  Slices are
 * independent: out[n] depends on in[n] only.  Uses context-owned scratch
 * (allocated at pr_create).  Device-side wait time-outs are reported by
 * pr_check, not by this call.
 */
pr_status pr_fine_all_slices(pr_ctx* ctx, const void* u_in, const void* v_in, void* u_out,
                             void* v_out, int n_begin, int n_end, void* stream);

/* Phase correctors of pr_iterate (Alg. 3 and its variants, Sec. 6.2):
 * PR_CORR_PROCRUSTES  theta = I Lambda^dagger Omega Lambda with Omega = X Y^T from Alg. 1;
 * PR_CORR_OMEGA1      Omega = 1, theta = I Lambda^dagger Lambda (Sec. 6.2);
 * PR_CORR_PLAIN       theta = I, plain parareal on the two grids (Sec. 1). */
enum { PR_CORR_PROCRUSTES = 0, PR_CORR_OMEGA1 = 1, PR_CORR_PLAIN = 2 };

/* pr_coarse_sweep -- the coarse half of Alg. 3's parallel phase,
 * [U_n, U_t n] = C [R u_{n-1}, R u_t n-1], for slices [n_begin, n_end).
 *  u, v          fine states [N][n^d] (dtype), read.
 *  U_out, V_out  coarse states [N][(n/ratio)^d] (dtype), written for the range.
 * R is injection onto the coarse nodes (Sec. 6); C is m_C velocity-Verlet
 * steps of dt_c on the coarse grid with c taken at the coarse nodes (Sec. 3.1),
 * run by the same kernels as F. */
pr_status pr_coarse_sweep(pr_ctx* ctx, const void* u, const void* v, void* U_out, void* V_out,
                          int n_begin, int n_end, void* stream);

/* pr_serial_sweep -- the serial corrected sweep of Alg. 3 (the serial
 * update of one iteration; the coarse sweep in its corrected, serial form),
 * so that a caller can compose Alg. 3 from pr_fine_all_slices,
 * pr_coarse_sweep, pr_procrustes_correct and this call.  For n = 1..N:
 *   w = C R u_{n-1}  (this call's own, on the new states),
 *   u_n = F_n + I(theta(w) - theta(U_n))
 * with theta of the corrector (PR_CORR_*; PR_CORR_PROCRUSTES applies the
 * Omega = X Y^T that pr_procrustes_correct has built in this context, and an
 * empty one, rank 0, gives a zero correction).
 *  Fu, Fv    F u^k_{n-1} for n = 1..N: fine states [N][n^d] (dtype), read.
 *  Uu, Uv    C R u^k_{n-1} for n = 1..N: coarse states [N][(n/ratio)^d]
 *            (dtype), read (pr_coarse_sweep writes them).
 *  u_slices, v_slices  [N+1][n^d] (dtype): slice 0 holds u^{k+1}_0 on entry
 *            (read); slices 1..N receive u^{k+1}_n.  No input may overlap
 *            slices 1..N of the outputs.
 * Requires a context with a coarse grid (PR_EINVAL otherwise).  FP32
 * contexts apply Omega with single-precision copies of the stored bases
 * (FP32-accurate, as the state is).  Returns after queuing the work and
 * reading the coarse propagation's device error flag (synchronises). */
pr_status pr_serial_sweep(pr_ctx* ctx, int corrector, const void* Fu, const void* Fv, const void* Uu,
                          const void* Uv, void* u_slices, void* v_slices, void* stream);

/* pr_iterate -- the proposed method, Alg. 3, for up to K iterations.
 *  u0, p0      initial state [n^d] (dtype, device).
 *  K           maximum iterations (K = 0 returns the initial guess I C R u_{n-1}).
 *  corrector   PR_CORR_*.
 *  tol_err     with a reference: stop after the first iteration whose
 *              relative energy-norm error at T is <= tol_err (Sec. 6).
 *  u_ref, v_ref  reference state at T = N dt_com [n^d] (dtype, device), e.g.
 *              the serial fine solution, or NULL (no error, no early stop).
 *  u_slices, v_slices  [N+1][n^d] (dtype, device): on return the states
 *              u^{k+1}_n, n = 0..N, of the last iteration done (u^{k+1}_0 = [u0, p0]).
 *  err_hist    HOST double[K] or NULL: sqrt(E(u^{k+1}_N - ref)/E(ref)), E the
 *              discrete wave energy with the 4th-order nabla_h on the fine grid.
 *  resid_hist  HOST double[K] or NULL: ||F - Omega G||_F / ||F||_F of each
 *              iteration's data after the update (0 without Procrustes).
 *  rank_hist   HOST int[K] or NULL: retained singular values s.
 *  k_done      HOST int or NULL: iterations done.
 * Fine sweeps run in the context dtype; Lambda, Omega, Lambda^dagger, I, the
 * data matrices and the SVD in FP64 (cuFFT, cuBLAS, cuSOLVER for the FFTs and
 * the dense factorisations).  In FP32 contexts the tall products of UpdateSVD
 * with the kept bases run on the tensor cores in split-TF32 (see
 * pr_snapshot_project) with one reorthogonalisation pass, and the SVD of the
 * small matrix H is taken from the symmetric eigenproblem of H^T H when every
 * kept singular value is at least 1e-6 of the largest (else FP64 gesvd).  The correction of a slice is applied to the
 * difference Lambda w - Lambda U_n with zero mode sum w - sum U_n, which by
 * linearity equals Alg. 3's two applications.  Synchronises the stream.
 * Reads the device-side error flags of the fine and coarse sweeps after every
 * iteration: PR_ETIMEOUT (flags cleared) if a bounded wait gave up.
 * Requires grad_order 2, 4, 6 or 8.  Returns PR_EUNSTABLE if the energy of
 * the state at T stops being finite (the stability the method is built to
 * keep, Sec. 5). */
pr_status pr_iterate(pr_ctx* ctx, const void* u0, const void* p0, int K, int corrector,
                     double tol_err, const void* u_ref, const void* v_ref, void* u_slices,
                     void* v_slices, double* err_hist, double* resid_hist, int* rank_hist,
                     int* k_done, void* stream);

/* pr_iterate_phases -- device time of the phases of the last pr_iterate call
 * on this context, split like the per-phase columns of the paper's timing
 * table (Sec. 7.2.4): ms[0] the initial serial coarse sweep u^1_n = I C R
 * u^1_{n-1}; ms[1] the parallel computation (F and C R over all slices),
 * ms[2] creating the corrector (Lambda of the data, UpdateSVD, residual) and
 * ms[3] the serial corrected update, each summed over the iterations done.
 *  ms   HOST double[4], written (zeros before the first pr_iterate).
 * Timed with CUDA events on the call's stream.  PR_EINVAL for NULL pointers. */
pr_status pr_iterate_phases(const pr_ctx* ctx, double* ms);

/* pr_iterate_corrector_phases -- device time of "creating the corrector" in
 * the last pr_iterate call (Procrustes), split per step of Alg. 1 and summed
 * over the iterations: ms[0] projections and deflations of the new data
 * against the kept bases, ms[1] reduced QR of the residual blocks, ms[2] the
 * small matrix H and its SVD, ms[3] the basis rotation, ms[4] the residual
 * ||F - Omega G|| / ||F|| of the iteration's data.  *eig_svds (may be NULL)
 * receives how many of the *svds SVDs (may be NULL) were taken through the
 * symmetric eigenproblem of H^T H (FP32 contexts, when every kept singular
 * value is at least 1e-6 of the largest; otherwise FP64 gesvd).
 *  ms   HOST double[5], written.  PR_EINVAL for NULL ctx or ms. */
pr_status pr_iterate_corrector_phases(const pr_ctx* ctx, double* ms, int* eig_svds, int* svds);

/* pr_procrustes_correct -- UpdateSVD (Alg. 1): M <- M + F G^T with the
 * context's truncated SVD M = X Sigma Y^T (rank cut sigma_i/sigma_max > tol).
 *  Fcols, Gcols  DEVICE double [ncols][(d+1) n_c^d], one column per slice
 *                (eq. matrixF / matrixG: [nabla_h w ; c^-1 w_t], x-derivative
 *                block first), 1 <= ncols <= N.
 * X and Y are held factored (X = X_b W_X): every update appends its ncols
 * orthonormalised columns to X_b, Y_b in context memory (2 (d+1) n_c^d
 * doubles per column, plus single-precision copies in FP32 contexts) until
 * pr_procrustes_reset or the next pr_iterate.  FP32 contexts form the tall
 * products on the tensor cores (below), the QR of the deflated blocks by
 * Cholesky QR twice (columns dependent on earlier ones to working accuracy
 * get a zero column of Q) and the SVD from the eigenproblem of H^T H; FP64
 * contexts use FP64 BLAS, Householder QR and gesvd throughout.
 * Synchronises the stream. */
pr_status pr_procrustes_correct(pr_ctx* ctx, const double* Fcols, const double* Gcols, int ncols,
                                void* stream);

/* pr_procrustes_apply -- out = X Y^T g (the phase corrector Omega of Alg. 3)
 * for a DEVICE double vector g of (d+1) n_c^d entries; *rank (host, may be
 * NULL) receives s.  g == NULL only reports the rank.  FP32 contexts read
 * single-precision copies of the stored bases (FP32 products, compensated
 * sums; FP32-accurate, and exactly zero for g = 0); FP64 contexts are FP64. */
pr_status pr_procrustes_apply(pr_ctx* ctx, const double* g, double* out, int* rank, void* stream);

/* pr_procrustes_reset -- forget M (S empty, as at the start of Alg. 3). */
pr_status pr_procrustes_reset(pr_ctx* ctx);

/* pr_adjoint -- reverse mode through the serial fine solve F^N from (u0, p0)
 * (N coupling intervals of m_F fine steps, Sec. 3.1 scheme).  For a loss L of
 * the state at T with gradients (gu_T, gv_T) = (dL/du(T), dL/du_t(T)) it
 * returns gu0 = dL/du0, gp0 = dL/dp0 and gc = dL/dc at the fine nodes (all
 * [n^d], dtype, device).  Slice-start states are checkpointed and each slice
 * is recomputed during the reverse sweep ((N+1) + (m_F+1) fields of context
 * workspace); dL/dkappa accumulates in FP64.  The paper does not
 * differentiate its method: at K = N iterations the parareal solution equals
 * the serial fine solution (Alg. 3 terminates), so with the correctors frozen
 * this is also its gradient.  Asynchronous on `stream`. */
pr_status pr_adjoint(pr_ctx* ctx, const void* u0, const void* p0, const void* gu_T,
                     const void* gv_T, void* gc, void* gu0, void* gp0, void* stream);

/* ---- products of the snapshot store on the tensor cores ------------------
 * The tall-skinny products of UpdateSVD (Alg. 1): the projections of new
 * data onto the kept bases, U_F = U^T F, V_G = V^T G, and the deflations
 * F - U U_F, G - V V_G.  They run on the tcgen05 tensor cores: operands are
 * FP64 in device memory, split while staged into shared memory into two
 * TF32 values carrying the leading 11 + 11 significant bits (x = hi + lo),
 * and each product is formed as hi*hi + hi*lo + lo*hi + lo*lo with FP32
 * accumulation ("split-TF32": about 2^-21 relative error per product,
 * FP32-level accuracy).  pr_iterate uses them in FP32 contexts
 * (FP64 contexts keep FP64 DGEMM).  The context supplies the device error
 * flag of the bounded waits (reported by pr_check) and error messages; its
 * grid is not used.  Arrays are DEVICE double, column-major, 8-byte aligned;
 * asynchronous on `stream`.  PR_EINVAL for negative sizes, leading
 * dimensions below the matrix height or NULL arrays, before any launch. */

/* pr_snapshot_project -- C = A^T B.
 *  A  K x M (lda >= K), B  K x N (ldb >= K), C  M x N (ldc >= M), overwritten.
 * K is the long (snapshot-row) dimension; any M, N >= 0.  C must not overlap
 * A or B. */
pr_status pr_snapshot_project(pr_ctx* ctx, const double* A, int64_t lda, const double* B, int64_t ldb,
                              int64_t K, int64_t M, int N, double* C, int64_t ldc, void* stream);

/* pr_snapshot_deflate -- O = F - A T.
 *  A  M x K (lda >= M), T  K x N (ldt >= K), F and O  M x N (ldf, ldo >= M).
 * M is the long (snapshot-row) dimension.  O == F (same leading dimension)
 * is allowed; any other overlap of O with F, A or T is rejected. */
pr_status pr_snapshot_deflate(pr_ctx* ctx, const double* A, int64_t lda, const double* T, int64_t ldt,
                              const double* F, int64_t ldf, int64_t M, int64_t K, int N, double* O,
                              int64_t ldo, void* stream);

/* pr_iterate_adjoint -- reverse mode through K iterations of Alg. 3 (the
 * parareal solve itself, not only its K = N limit) with every iteration's
 * phase corrector Omega^k = X_k Y_k^T frozen at the value the forward run
 * computes from its data (Alg. 1).  The paper does not differentiate its
 * method; with the correctors frozen the map (u0, p0, c) -> u^{K+1}_N is a
 * composition of F, C (Sec. 3.1), R, I (Sec. 6), Lambda, Lambda^dagger
 * (Sec. 3.4, Alg. 2) and fixed matrices, and this call applies the
 * transposes of those maps in reverse order.
 *  u0, p0      initial state [n^d] (dtype, device); the forward run is
 *              pr_iterate(ctx, u0, p0, K, corrector, ...) without early stop.
 *  K           iterations, 1 <= K (K = N gives the serial fine gradient).
 *  corrector   PR_CORR_*.
 *  gu_T, gv_T  dL/du, dL/du_t of the loss at the state u^{K+1}_N [n^d].
 *  gc          dL/dc at the fine nodes [n^d] (the coarse c is R c, so its
 *              terms are scattered back onto the coarse nodes); includes the
 *              dependence of Lambda (c^-1 u_t) and Lambda^dagger (c p) on c.
 *  gu0, gp0    dL/du0, dL/dp0 [n^d].
 * Every iteration's states are kept ((K+1)(N+1) fine states, allocated and
 * freed by the call); each slice of F and C is recomputed from its start
 * state in the reverse sweep.  The propagators' transposes run in the
 * context dtype with dL/dkappa in FP64; the correction-path transposes in
 * FP64.  Synchronises the stream.  PR_ETIMEOUT if a bounded wait of the
 * forward run gave up. */
pr_status pr_iterate_adjoint(pr_ctx* ctx, const void* u0, const void* p0, int K, int corrector,
                             const void* gu_T, const void* gv_T, void* gc, void* gu0, void* gp0,
                             void* stream);

/* ---- batches of independent instances of uneven sizes ------------------- */
typedef struct pr_batch pr_batch;

/* pr_batch_create -- bind `count` instances (each its own context and its own
 * [N_i][pts_i] input/output arrays, all on the current device) for one fine
 * sweep each (Alg. 3 parallel phase, for every instance).
 *  autotune   non-zero: for every instance time one sweep at each instantiated
 *             fused configuration (block depth 8 or 4 with 2 or 4 columns
 *             per thread for the fused 2D kernels; depth 1 = one step per
 *             pass) on `stream` and keep the fastest (written into the
 *             instance's context); 0: keep each context's settings.
 * Then captures all sweeps into one CUDA graph: one branch per instance,
 * biggest first, spread over 8 library-owned streams between a fork and a
 * join (one launch per pass: pr_set_one_launch is switched off for the
 * bound contexts, whose sweeps run concurrently).  Runs (and synchronises)
 * the timing sweeps.  The bound arrays and the contexts (whose scratch, kappa
 * and error flags the graph uses) must stay valid while the batch is
 * launched; the contexts must not be used concurrently with a launch of the
 * batch.  PR_EINVAL if a context appears
 * twice or an output array overlaps an array of another instance (inputs may
 * be shared between instances; in == out within one instance is allowed). */
pr_status pr_batch_create(int count, pr_ctx* const* ctxs, const void* const* u_in,
                          const void* const* v_in, void* const* u_out, void* const* v_out,
                          int autotune, void* stream, pr_batch** out);

/* pr_batch_launch -- replay the captured graph on `stream` (asynchronous).
 * Device-side wait time-outs are reported by pr_check on each instance's
 * context, after the launch has completed. */
pr_status pr_batch_launch(pr_batch* b, void* stream);

/* pr_batch_info -- chosen block depth, fused-kernel columns per thread (0 =
 * the default; see pr_set_fused_columns) and the timed sweep (ms) of
 * instance i (in mode 1: depth 8 and 4 columns, the queue kernel's).  Any
 * output pointer may be NULL. */
pr_status pr_batch_info(const pr_batch* b, int i, int* block_depth, int* columns, double* tuned_ms);

/* pr_batch_set_mode -- the form of the batch's graph (Alg. 3 parallel phase
 * for every instance; both forms compute every instance's sweep):
 *   0   the per-instance chains of pass launches (pr_batch_create's form);
 *   1   ONE persistent kernel, one CTA per SM, that claims work items
 *       (instance, pass, slice, and x-strip of 752 final columns at
 *       n = 2048) from a device queue; pass k of a slice waits, bounded, until
 *       every item of pass k-1 of that slice has finished.  Passes of 8
 *       levels (a lone final level makes the last two 5 + 4), so results
 *       agree with mode 0 to FP32 rounding, not bit for bit.  Needs every
 *       instance 2D FP32 with n in {256, 512, 1024, 2048} and m_f >= 8
 *       (PR_EINVAL otherwise); each switch to it builds the queue tables
 *       from the contexts' current settings, in device memory (through the
 *       first context's allocator);
 *  -1   time both forms on `stream` (a warm-up and two replays each) and
 *       keep the faster.
 * The chosen mode is written to *chosen (may be NULL).  Synchronises the
 * device, then re-captures the graph; the bound arrays are written by the
 * timing replays.  In mode 1 a wait that gave up stops the queue, and
 * pr_check then reports PR_ETIMEOUT on every instance's context (items of
 * any instance may be left undone). */
pr_status pr_batch_set_mode(pr_batch* b, int mode, void* stream, int* chosen);

/* pr_batch_destroy -- free the graph and the streams (NULL is a no-op). */
void pr_batch_destroy(pr_batch* b);

/* pr_set_fused_columns -- thread geometry of the fused 2D FP32 passes of
 * this context: 2 or 4 grid columns per thread (n/2 or n/4 threads per row),
 * or 0 = the default (4, the faster geometry on a GB300 at n = 512 and 1024;
 * n = 2048 always runs four columns).  Both compute the same level
 * recurrence; results agree to rounding.  PR_EINVAL for any other value.
 * Takes effect at the next call. */
pr_status pr_set_fused_columns(pr_ctx* ctx, int columns);

/* pr_set_one_launch -- on != 0: where the fused 2D kernel runs whole rows at
 * depth 8 with four columns per thread (n = 128 .. 1024) and a sweep takes at
 * least two passes, pr_fine_all_slices runs every pass of the sweep (all
 * slices) in ONE persistent cooperative launch, one CTA per SM, with a
 * bounded grid-wide barrier between passes; on == 0 (the default): one launch
 * per pass, which measured faster on a GB300 (the pass loop costs the
 * middle-pass body its kappa register ring).  Both compute the same level
 * recurrence in the same order (bit-identical results).  Takes effect at the
 * next call. */
pr_status pr_set_one_launch(pr_ctx* ctx, int on);

/* pr_set_wide_rows -- how the fused 2D FP32 passes at depth 8 hold the
 * 2048-point rows, which no single CTA's registers hold: 1 = each row shared
 * by a two-CTA thread-block cluster that exchanges the half-rows' x-edges
 * through distributed shared memory; 2 = three overlapping x-strips of 704
 * columns per row (688 final columns, an 8-column halo each side recomputed
 * by the neighbouring strip), no exchange; the default, measured 6 % faster
 * on a GB300.  Both compute the same level recurrence in the same order
 * (bit-identical results).  PR_EINVAL for another mode.  Takes effect at the
 * next call. */
pr_status pr_set_wide_rows(pr_ctx* ctx, int mode);

/* pr_set_resident -- where a 2D FP32 slice fits in the shared memory of one
 * thread-block cluster (n = 128 or 256 at block depth 8 with four columns
 * per thread), on != 0 makes pr_fine_all_slices propagate every slice in ONE
 * launch, one cluster of 8 CTAs per slice holding its state on chip for all
 * m + 1 kicks (one cluster barrier per kick); on == 0 keeps the per-pass
 * fused launches.  Both run the same pass plan and the same operations in
 * the same order (bit-identical results).  Default (never called): on at
 * n = 128 (the coarse grid of the 512^2 workload, where it measured about
 * twice as fast for one slice), off at n = 256 (eight SMs per slice measured
 * slower than the per-pass kernels over all SMs).  Takes effect at the next
 * call. */
pr_status pr_set_resident(pr_ctx* ctx, int on);

/* pr_debug_stall_waits -- test hook for the time-out path.  While enabled,
 * fused-kernel launches of this context expect more bulk-copy bytes than
 * they issue, so each bounded shared-memory barrier wait runs out (after
 * 0.2 s instead of 2 s); the kernel records PR_ETIMEOUT, lets its copies
 * land and returns, and later fused launches skip their work until
 * pr_check reports and clears the error.  Nothing faults or hangs; results
 * of the affected calls are not valid. */
pr_status pr_debug_stall_waits(pr_ctx* ctx, int enable);

/* pr_check -- synchronise `stream`, then report and clear a device-side error
 * flag set by a kernel whose bounded wait gave up (PR_ETIMEOUT), or a pending
 * CUDA error (PR_ECUDA). */
pr_status pr_check(pr_ctx* ctx, void* stream);

/* pr_info -- derived constants of the context (any pointer may be NULL):
 * m_F, m_C, the number of fine points per slice, and the fine step count per
 * HBM pass the fine propagator uses. */
pr_status pr_info(const pr_ctx* ctx, int* m_f, int* m_c, int64_t* pts, int* block_depth);

/* pr_energy -- discrete wave energy of every slice (Sec. 3.1, eq.
 * discrete-wave-energy) on the fine grid, accumulated in FP64:
 *   E_n = 1/2 sum_j |nabla_h u_n(x_j)|^2 dx^d + 1/2 sum_j c_j^-2 |v_n(x_j)|^2 dx^d
 * with nabla_h the 4th-order central difference (Sec. 6.4, "4 order").
 *  u, v     [N][pts] device arrays (dtype), slices [n_begin, n_end) are read.
 *  e_host   HOST array of n_end - n_begin doubles receiving E_n.
 * Synchronises `stream` before returning. */
pr_status pr_energy(pr_ctx* ctx, const void* u, const void* v, int n_begin, int n_end,
                    double* e_host, void* stream);

/* pr_profile -- per-launch timing of the fine propagator with CUDA events
 * recorded on the launching stream (the per-phase timers of the paper's
 * Sec. 7.2.4 timing study, at kernel granularity).  on != 0 clears the record
 * and starts recording an event pair around every kernel that
 * pr_fine_all_slices launches; on == 0 stops recording. */
pr_status pr_profile(pr_ctx* ctx, int on);

/* pr_profile_read -- synchronise on the recorded events and report, for
 * kernel kind 0 (fused multi-level pass), 1 (single-level pass), 2 (a whole
 * sweep in one launch, pr_set_one_launch) or 3 (all slices resident in
 * cluster shared memory, pr_set_resident), the number of launches recorded
 * and their summed duration in milliseconds. */
pr_status pr_profile_read(pr_ctx* ctx, int kind, int* launches, double* total_ms);

/* Size in bytes of the fixed device scratch array behind
 * pr_fine_all_slices_noalloc (32 MiB). */
#define PR_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* pr_fine_all_slices_noalloc -- the fine propagator over a batch of slices
 * without any device allocation and without a context.  The paper has no
 * counterpart: this is an interface for callers that cannot allocate device
 * memory, so cannot use pr_create (which cudaMallocs the coefficient and
 * scratch arrays): code running inside a framework that owns the whole device
 * memory pool, plugins invoked from another library's stream-ordered work,
 * real-time loops where an allocation's latency or failure is unacceptable.
 *
 *  dim, n       grid: n points per axis on [0,1)^dim, dim in {1,2,3}, n in [4, 2^20].
 *  nslices      slices in the batch (0 = nothing to do).
 *  c            DEVICE float[n^dim], wave speed at the fine nodes.
 *  dt_f, m_f    fine step and steps per slice (m_f >= 1).  The CFL condition
 *               max c * dt_f * sqrt(dim) * n <= 1 is the caller's to meet
 *               (it is not checked: checking would need a device read-back).
 *  u_in, v_in   DEVICE float[nslices][n^dim] slice states; u_out, v_out the
 *               results, same layout; out == in allowed, other overlap is not.
 *  stream       cudaStream_t (void*).
 *  msg, msg_len optional caller buffer for an error message (may be NULL).
 * Computes what pr_fine_all_slices computes for FP32 (one launch per Verlet
 * level, the context path's single-level arithmetic).
 *
 * Scratch: one file-scope device array of PR_NOALLOC_SCRATCH_BYTES, held by
 * every GPU that loads the library until the process exits.  A call needs
 *   A(n^dim * 4) + 2 * (2 * A(nslices * n^dim * 4) + A(nslices * n^dim))
 * bytes, A() rounding up to 256; larger requests return PR_EINVAL with the
 * sizes in msg, before anything is launched.  No call allocates: no
 * cudaMalloc, cudaFree or allocating library routine.  All calls share the
 * array and it keeps the last call's contents (nothing in it needs to start at
 * zero); calls whose GPU work overlaps race on it, so serialise them on one
 * stream.  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it: make that
 * first call before any stream capture begins.
 * Returns PR_OK, PR_EINVAL (arguments or size) or PR_ECUDA. */
pr_status pr_fine_all_slices_noalloc(int dim, int64_t n, int nslices, const float* c, double dt_f,
                                     int m_f, const float* u_in, const float* v_in, float* u_out,
                                     float* v_out, void* stream, char* msg, size_t msg_len);

#ifdef __cplusplus
}
#endif

#endif /* PR_H */
