// Tall-skinny products of the snapshot store on the 5th-generation tensor
// cores (tcgen05, accumulators in tensor memory), for the UpdateSVD step of
// Alg. 1 in contexts that step the fine grid in FP32:
//
//   gram  (TN):  C  = A^T B            U_F = U^T F, V_G = V^T G (Alg. 1)
//   update (NN): O  = F - A T          F - U U_F, G - V V_G      (Alg. 1)
//
// A is a basis or data matrix of `rows` = (d+1) N_Dx rows (column-major,
// FP64), so K = rows is long for the gram and M = rows is long for the
// update; N (the number of new columns, at most 64 per launch) is small.
//
// Precision.  Operands stay FP64 in HBM.  Each element x is split while it
// is staged into shared memory as x = hi + lo (two tf32 values carrying the
// leading 11 + 11 significant bits, |x - hi - lo| <= 2^-21 |x|), and every
// product is formed as hi*hi + hi*lo + lo*hi + lo*lo by kind::tf32 MMAs into
// one FP32 accumulator: about 2^-21 relative per product, FP32-level, against
// TF32's 2^-11.  Partial sums leave tensor memory in FP32 and are combined in
// FP64.
//
// Kernel shape.  256 threads per CTA, two CTAs per SM (16 warps to hide the
// split's latency); the M = 128 accumulator rows map onto the 128
// tensor-memory lanes, and in the epilogue warps w and w + 4 read lanes
// 32w..32w+31, each half of the columns.  K advances in chunks of 32
// elements: the threads load the
// chunk's FP64 values, split them and store hi and lo into 128-byte-swizzled
// K-major tiles (two stages), then thread 0 issues 4 K-steps x 4 MMAs and
// commits them to the stage's mbarrier, which the threads wait on before
// they overwrite that stage.  Two chunks are held in registers: once chunk
// c is in shared memory the loads of chunk c + 2 are issued, so two chunks'
// HBM reads overlap the MMAs and the next split.  Every wait is bounded.
//
// The split-K gram sums its CTAs' partials with FP64 atomic adds into C,
// which the launcher clears first.
#include <stdio.h>

#include <algorithm>

#include "pr_internal.cuh"

namespace {

constexpr int kThreads = 256;   // two threads per tile row (kM rows)
constexpr int kM = 128;          // accumulator rows per CTA (tensor-memory lanes)
constexpr int kKc = 32;          // K elements per chunk: 32 tf32 = 128 bytes per row
constexpr int kStages = 2;       // smem stages (the loop below tracks exactly two)

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ bool bar_try(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// false after limit_ns without the phase completing
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity, uint64_t limit_ns) {
    if (bar_try(b, parity)) return true;
    const uint64_t t0 = now_ns();
    while (!bar_try(b, parity))
        if (now_ns() - t0 > limit_ns) return false;
    return true;
}

// tf32 split of one FP64 value by integer operations on its bits (no FP64
// arithmetic, which runs at a small fraction of the FP32 rate on this GPU):
// hi = x with its mantissa truncated to tf32's 10 bits, lo = the next 10
// significant bits of the remainder x - hi (same sign), so that
// |x - hi - lo| <= 2^-21 |x|.  Values below the float range (|x| < 2^-126)
// become 0; the operands here are O(1e-3..1e3).
__device__ __forceinline__ void split_tf32(double x, uint32_t& hi, uint32_t& lo) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t s = (uint32_t)(b >> 63) << 31;
    const int E = (int)((b >> 52) & 0x7ff);
    const uint64_t M = b & 0xFFFFFFFFFFFFFull;
    const int Ef = E - 1023 + 127;
    if (E == 0 || Ef <= 0) {
        hi = lo = 0u;
        return;
    }
    hi = s | ((uint32_t)Ef << 23) | ((uint32_t)(M >> 42) << 13);
    const uint64_t R = M & ((1ull << 42) - 1);   // remainder R * 2^(E - 1075)
    lo = 0u;
    if (R != 0) {
        const int lz = __clzll((long long)R);    // 22 .. 63
        const int Elo = (63 - lz) + E - 1075 + 127;
        if (Elo > 0) lo = s | ((uint32_t)Elo << 23) | ((uint32_t)((R << (lz + 1)) >> 54) << 13);
    }
}

// Byte offset of the 16-byte group c (K elements 4c..4c+3) of row m in a
// K-major tile with 128-byte rows, 128-byte swizzle: 8-row atoms of 1024
// bytes, group c of row m stored at group position c ^ (m mod 8).
__device__ __forceinline__ uint32_t sw128(int m, int c) {
    return (uint32_t)((m >> 3) * 1024 + (m & 7) * 128 + ((c ^ (m & 7)) << 4));
}

// Shared-memory matrix descriptor (tcgen05): K-major, 128-byte swizzle,
// 8-row groups 1024 bytes apart.  Start address, leading and stride byte
// offsets are encoded in 16-byte units; bits 46-47 hold the descriptor
// version (1); bits 61-63 the swizzle mode (2 = 128 bytes).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                 // version
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::tf32 with an FP32 accumulator, both
// operands K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4)                        // D format: F32
           | (2u << 7) | (2u << 10)         // A, B format: TF32
           | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// Shared memory of one CTA: kStages x (A hi, A lo: 128 rows; B hi, B lo: NB
// rows) of 128-byte rows, each tile 1024-byte aligned, then the mbarriers and
// the tensor-memory address.
template <int NB>
struct TcSmem {
    static constexpr uint32_t a_bytes = kM * 128, b_bytes = NB * 128;
    static constexpr uint32_t stage = 2 * a_bytes + 2 * b_bytes;
    static constexpr uint32_t total = kStages * stage + 64 + 1024;   // + barriers, + alignment slack
    static_assert(b_bytes % 1024 == 0, "B tiles must keep 1024-byte alignment");
};

struct GramArgs {
    const double* A;     // gram: element (m, k) at A[m * lda + k]; update: (r, j) at A[j * lda + r]
    int64_t lda;
    const double* B;     // gram: (n, k) at B[n * ldb + k]; update: T, (j, n) at B[n * ldb + j]
    int64_t ldb;
    const double* F;     // update only: (r, n) at F[n * ldf + r]
    int64_t ldf;
    double* C;           // gram: C[m + n * ldc] += ...; update: O[r + n * ldc] = F - ...
    int64_t ldc;
    int64_t M, K;        // rows of the result (gram: M = columns of A), contraction length
    int N;               // result columns, N <= NB
    int64_t chunks_per_cta;
    int* flag;           // device error flag (bounded waits)
    uint64_t wait_ns;
};

// One K chunk in registers: thread t's share of the A tile (4 groups of 4
// elements) and of the B tile (NB/32 groups).  MODE 0 (gram): A rows are
// contiguous in K, thread t takes group t % 8 of rows t/8 + 32 j.  MODE 1
// (update): A columns are contiguous in M, thread t takes row t % 128 and the
// groups 4 (t / 128) .. 4 (t / 128) + 3 of 4 columns, each element a load
// coalesced across the warp.  B (NB rows, contiguous in K) in both modes:
// item i = t + 256 j is group i % 8 of row i / 8.  Elements outside the
// matrices are zero.
template <int NB>
struct Chunk {
    double a[4][4];
    double b[NB / 32][4];
};

template <int MODE, int NB>
__device__ __forceinline__ void load_chunk(const GramArgs& g, int64_t m0, int64_t k0, Chunk<NB>& x) {
    const int t = threadIdx.x;
    if (MODE == 0) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t gm = m0 + t / 8 + 32 * j, gk = k0 + 4 * (t % 8);
            const double* src = g.A + gm * g.lda + gk;
            if (gm < g.M && gk + 3 < g.K && (((uintptr_t)src) & 15) == 0) {
                const double2 p0 = __ldcs((const double2*)src), p1 = __ldcs((const double2*)src + 1);
                x.a[j][0] = p0.x; x.a[j][1] = p0.y; x.a[j][2] = p1.x; x.a[j][3] = p1.y;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) x.a[j][e] = (gm < g.M && gk + e < g.K) ? __ldcs(src + e) : 0.0;
            }
        }
    } else {
        const int64_t gm = m0 + t % kM;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int64_t gk = k0 + 4 * (4 * (t / kM) + c) + e;
                x.a[c][e] = (gm < g.M && gk < g.K) ? __ldcs(g.A + gk * g.lda + gm) : 0.0;
            }
    }
#pragma unroll
    for (int j = 0; j < NB / 32; ++j) {
        const int i = t + kThreads * j;
        const int n = i / 8;
        const int64_t gk = k0 + 4 * (i % 8);
        const double* src = g.B + (int64_t)n * g.ldb + gk;
#pragma unroll
        for (int e = 0; e < 4; ++e) x.b[j][e] = (n < g.N && gk + e < g.K) ? src[e] : 0.0;
    }
}

// Split the chunk in registers into hi/lo tf32 tiles of one stage.
template <int MODE, int NB>
__device__ __forceinline__ void store_chunk(const Chunk<NB>& x, unsigned char* st) {
    using S = TcSmem<NB>;
    const int t = threadIdx.x;
    unsigned char* ahi = st;
    unsigned char* alo = st + S::a_bytes;
    unsigned char* bhi = st + 2 * S::a_bytes;
    unsigned char* blo = bhi + S::b_bytes;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int m = MODE == 0 ? t / 8 + 32 * j : t % kM;
        const int c = MODE == 0 ? t % 8 : 4 * (t / kM) + j;
        uint4 h, l;
        split_tf32(x.a[j][0], h.x, l.x); split_tf32(x.a[j][1], h.y, l.y);
        split_tf32(x.a[j][2], h.z, l.z); split_tf32(x.a[j][3], h.w, l.w);
        *(uint4*)(ahi + sw128(m, c)) = h;
        *(uint4*)(alo + sw128(m, c)) = l;
    }
#pragma unroll
    for (int j = 0; j < NB / 32; ++j) {
        const int i = t + kThreads * j;
        uint4 h, l;
        split_tf32(x.b[j][0], h.x, l.x); split_tf32(x.b[j][1], h.y, l.y);
        split_tf32(x.b[j][2], h.z, l.z); split_tf32(x.b[j][3], h.w, l.w);
        *(uint4*)(bhi + sw128(i / 8, i % 8)) = h;
        *(uint4*)(blo + sw128(i / 8, i % 8)) = l;
    }
    // generic-proxy shared stores become visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// MODE 0: gram, blockIdx.x = M tile, blockIdx.y = K split.
// MODE 1: update, blockIdx.x = M tile (rows), one CTA covers all of K.
template <int MODE, int NB>
__global__ void __launch_bounds__(kThreads, 2) gram_tc_kernel(const GramArgs g) {
    using S = TcSmem<NB>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(sm + kStages * S::stage);    // [kStages] MMA done
    uint32_t* tmem_slot = (uint32_t*)(bars + kStages);
    const int t = threadIdx.x, warp = t / 32;
    constexpr uint32_t kTmemCols = NB < 32 ? 32 : NB;

    if (t == 0) {
        for (int s = 0; s < kStages; ++s) bar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    const int64_t m0 = (int64_t)blockIdx.x * kM;
    const int64_t total_chunks = (g.K + kKc - 1) / kKc;
    const int64_t c_begin = MODE == 0 ? (int64_t)blockIdx.y * g.chunks_per_cta : 0;
    const int64_t c_end = MODE == 0 ? min(total_chunks, c_begin + g.chunks_per_cta) : total_chunks;
    constexpr uint32_t idesc = idesc_tf32(kM, NB);
    bool ok = true;
    // MMA batches committed per stage (stage s has been used issued_s times)
    uint32_t issued0 = 0, issued1 = 0;

    // Two chunks in registers: chunk c + 2 is requested as soon as chunk c is
    // in shared memory, so two chunks' loads are in flight while the MMAs and
    // the next chunk's split run (chunk c uses stage (c - c_begin) % 2).
    Chunk<NB> x0, x1;
    if (c_begin < c_end) load_chunk<MODE, NB>(g, m0, c_begin * kKc, x0);
    if (c_begin + 1 < c_end) load_chunk<MODE, NB>(g, m0, (c_begin + 1) * kKc, x1);
    auto step = [&](int64_t c, Chunk<NB>& x, int s, uint32_t& used) -> bool {
        unsigned char* st = sm + s * S::stage;
        // the stage's previous MMAs must be done before it is overwritten
        if (used > 0 && ok) {
            if (!bar_wait(&bars[s], (used - 1) & 1u, g.wait_ns)) ok = false;
        }
        if (!__syncthreads_and(ok)) {
            ok = false;
            return false;
        }
        store_chunk<MODE, NB>(x, st);
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_hi = smem_addr(st), a_lo = a_hi + S::a_bytes;
            const uint32_t b_hi = a_hi + 2 * S::a_bytes, b_lo = b_hi + S::b_bytes;
#pragma unroll
            for (int ks = 0; ks < kKc / 8; ++ks) {   // 8 tf32 = 32 bytes per MMA K-step
                const uint32_t off = 32u * ks;
                const uint32_t acc0 = (c > c_begin || ks > 0) ? 1u : 0u;
                mma_tf32(tmem, sdesc(a_hi + off), sdesc(b_hi + off), idesc, acc0);
                mma_tf32(tmem, sdesc(a_hi + off), sdesc(b_lo + off), idesc, 1u);
                mma_tf32(tmem, sdesc(a_lo + off), sdesc(b_hi + off), idesc, 1u);
                mma_tf32(tmem, sdesc(a_lo + off), sdesc(b_lo + off), idesc, 1u);
            }
            mma_commit(&bars[s]);
        }
        ++used;
        if (c + 2 < c_end) load_chunk<MODE, NB>(g, m0, (c + 2) * kKc, x);
        return true;
    };
    for (int64_t c = c_begin; c < c_end; c += 2) {
        if (!step(c, x0, 0, issued0)) break;
        if (c + 1 < c_end && !step(c + 1, x1, 1, issued1)) break;
    }
    // all MMAs done: wait for the last commit of every stage used
    bool done = true;
    if (issued0 > 0 && !bar_wait(&bars[0], (issued0 - 1) & 1u, g.wait_ns)) done = false;
    if (issued1 > 0 && !bar_wait(&bars[1], (issued1 - 1) & 1u, g.wait_ns)) done = false;
    if (!done) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool all_ok = __syncthreads_and(ok) != 0;
    if (!all_ok) {
        if (t == 0) atomicExch(g.flag, 1);
    } else if (c_end > c_begin) {
        // epilogue: accumulator row t % 128 (lane t % 128; warp w reads lanes
        // 32 (w % 4) ..), columns NB/2 (t / 128) .. NB/2 (t / 128) + NB/2 - 1
        constexpr int NH = NB / 2;
        const int half = t / kM;
        const uint32_t taddr = tmem + ((uint32_t)((warp % 4) * 32) << 16) + (uint32_t)(half * NH);
        float acc[NH];
#pragma unroll
        for (int j0 = 0; j0 < NH; j0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr + (uint32_t)j0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int e = 0; e < 16; ++e) acc[j0 + e] = __uint_as_float(r[e]);
        }
        const int64_t m = m0 + t % kM;
        if (m < g.M) {
#pragma unroll
            for (int j = 0; j < NH; ++j) {
                const int n = half * NH + j;
                if (n >= g.N) break;
                if (MODE == 0) {
                    atomicAdd(g.C + m + (int64_t)n * g.ldc, (double)acc[j]);
                } else {
                    g.C[m + (int64_t)n * g.ldc] = g.F[m + (int64_t)n * g.ldf] - (double)acc[j];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

template <int MODE, int NB>
pr_status launch_tc(GramArgs g, dim3 grid, cudaStream_t st) {
    using S = TcSmem<NB>;
    auto kern = gram_tc_kernel<MODE, NB>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::total);
        if (e != cudaSuccess) return pr_cuda_fail(nullptr, e, "gram_tc: smem attribute");
        configured = true;
    }
    kern<<<grid, kThreads, S::total, st>>>(g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pr_cuda_fail(nullptr, e, "gram_tc: launch");
    return PR_OK;
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

}  // namespace

// C (M x N, column-major, ldc) = A^T B with A (K x M, lda), B (K x N, ldb),
// all FP64, on the tensor cores in split-TF32 (see the file comment).
pr_status tc_gram_launch(const double* A, int64_t lda, const double* B, int64_t ldb, int64_t K, int64_t M, int N,
                         double* C, int64_t ldc, int* flag, cudaStream_t st) {
    if (M <= 0 || N <= 0) return PR_OK;
    if (N > 64) {
        for (int n0 = 0; n0 < N; n0 += 64) {
            const int nn = N - n0 < 64 ? N - n0 : 64;
            pr_status s = tc_gram_launch(A, lda, B + (int64_t)n0 * ldb, ldb, K, M, nn, C + (int64_t)n0 * ldc, ldc, flag, st);
            if (s != PR_OK) return s;
        }
        return PR_OK;
    }
    {
        // one clearing call for the N columns (the split-K CTAs add into C)
        cudaError_t e = ldc == M ? cudaMemsetAsync(C, 0, (size_t)M * N * sizeof(double), st)
                                 : cudaMemset2DAsync(C, (size_t)ldc * sizeof(double), 0, (size_t)M * sizeof(double),
                                                     (size_t)N, st);
        if (e != cudaSuccess) return pr_cuda_fail(nullptr, e, "gram_tc: clear");
    }
    if (K <= 0) return PR_OK;
    GramArgs g = {A, lda, B, ldb, nullptr, 0, C, ldc, M, K, N, 0, flag, 2000000000ull};
    const int64_t mt = (M + kM - 1) / kM;
    const int64_t chunks = (K + kKc - 1) / kKc;
    // split K so that about two CTAs per SM run, each with >= 8 chunks
    int64_t splits = (2 * (int64_t)sm_count() + mt - 1) / mt;
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, chunks / 8));
    g.chunks_per_cta = (chunks + splits - 1) / splits;
    splits = (chunks + g.chunks_per_cta - 1) / g.chunks_per_cta;
    const dim3 grid((unsigned)mt, (unsigned)splits);
    return N <= 32 ? launch_tc<0, 32>(g, grid, st) : launch_tc<0, 64>(g, grid, st);
}

// O (M x N, ldo) = F (M x N, ldf) - A T with A (M x K, lda) and T (K x N,
// ldt), all FP64, on the tensor cores in split-TF32.  O may equal F.
pr_status tc_update_launch(const double* A, int64_t lda, const double* T, int64_t ldt, const double* F, int64_t ldf,
                           int64_t M, int64_t K, int N, double* O, int64_t ldo, int* flag, cudaStream_t st) {
    if (M <= 0 || N <= 0) return PR_OK;
    if (N > 64) {
        for (int n0 = 0; n0 < N; n0 += 64) {
            const int nn = N - n0 < 64 ? N - n0 : 64;
            pr_status s = tc_update_launch(A, lda, T + (int64_t)n0 * ldt, ldt, F + (int64_t)n0 * ldf, ldf, M, K, nn,
                                       O + (int64_t)n0 * ldo, ldo, flag, st);
            if (s != PR_OK) return s;
        }
        return PR_OK;
    }
    if (K <= 0) {
        if (O != F)
            for (int n = 0; n < N; ++n) {
                cudaError_t e = cudaMemcpyAsync(O + (int64_t)n * ldo, F + (int64_t)n * ldf, (size_t)M * 8,
                                                cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) return pr_cuda_fail(nullptr, e, "gram_tc: copy");
            }
        return PR_OK;
    }
    GramArgs g = {A, lda, T, ldt, F, ldf, O, ldo, M, K, N, 0, flag, 2000000000ull};
    const dim3 grid((unsigned)((M + kM - 1) / kM), 1);
    return N <= 32 ? launch_tc<1, 32>(g, grid, st) : launch_tc<1, 64>(g, grid, st);
}

// [p, p + span) of a column-major matrix (rows x cols, ld) of doubles
inline bool spans_overlap(const double* a, int64_t arows, int64_t acols, int64_t lda, const double* b,
                          int64_t brows, int64_t bcols, int64_t ldb) {
    if (!a || !b || arows <= 0 || acols <= 0 || brows <= 0 || bcols <= 0) return false;
    const uintptr_t a0 = (uintptr_t)a, a1 = a0 + (uintptr_t)((acols - 1) * lda + arows) * 8;
    const uintptr_t b0 = (uintptr_t)b, b1 = b0 + (uintptr_t)((bcols - 1) * ldb + brows) * 8;
    return a0 < b1 && b0 < a1;
}

// ============================================================================ C ABI
extern "C" pr_status pr_snapshot_project(pr_ctx* ctx, const double* A, int64_t lda, const double* B, int64_t ldb,
                                         int64_t K, int64_t M, int N, double* C, int64_t ldc, void* stream) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_snapshot_project: ctx is NULL");
    if (K < 0 || M < 0 || N < 0) return pr_fail(ctx, PR_EINVAL, "pr_snapshot_project: negative size");
    if (M == 0 || N == 0) return PR_OK;
    if (!A || !B || !C) return pr_fail(ctx, PR_EINVAL, "pr_snapshot_project: NULL array");
    if (lda < K || ldb < K || ldc < M)
        return pr_fail(ctx, PR_EINVAL, "pr_snapshot_project: need lda, ldb >= K and ldc >= M");
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)C) & 7)
        return pr_fail(ctx, PR_EINVAL, "pr_snapshot_project: arrays must be 8-byte aligned");
    if (spans_overlap(C, M, N, ldc, A, K, M, lda) || spans_overlap(C, M, N, ldc, B, K, N, ldb))
        return pr_fail(ctx, PR_EINVAL, "pr_snapshot_project: C overlaps A or B");
    return tc_gram_launch(A, lda, B, ldb, K, M, N, C, ldc, ctx->dev_flag, (cudaStream_t)stream);
}

extern "C" pr_status pr_snapshot_deflate(pr_ctx* ctx, const double* A, int64_t lda, const double* T, int64_t ldt,
                                         const double* F, int64_t ldf, int64_t M, int64_t K, int N, double* O,
                                         int64_t ldo, void* stream) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_snapshot_deflate: ctx is NULL");
    if (K < 0 || M < 0 || N < 0) return pr_fail(ctx, PR_EINVAL, "pr_snapshot_deflate: negative size");
    if (M == 0 || N == 0) return PR_OK;
    if (!F || !O || (K > 0 && (!A || !T))) return pr_fail(ctx, PR_EINVAL, "pr_snapshot_deflate: NULL array");
    if ((K > 0 && (lda < M || ldt < K)) || ldf < M || ldo < M)
        return pr_fail(ctx, PR_EINVAL, "pr_snapshot_deflate: need lda, ldf, ldo >= M and ldt >= K");
    if (((uintptr_t)A | (uintptr_t)T | (uintptr_t)F | (uintptr_t)O) & 7)
        return pr_fail(ctx, PR_EINVAL, "pr_snapshot_deflate: arrays must be 8-byte aligned");
    // O and F may coincide, but must not partly overlap; O must not touch A or T
    if (!(O == F && ldo == ldf) && spans_overlap(O, M, N, ldo, F, M, N, ldf))
        return pr_fail(ctx, PR_EINVAL, "pr_snapshot_deflate: O overlaps F");
    if (K > 0 && (spans_overlap(O, M, N, ldo, A, M, K, lda) || spans_overlap(O, M, N, ldo, T, K, N, ldt)))
        return pr_fail(ctx, PR_EINVAL, "pr_snapshot_deflate: O overlaps A or T");
    return tc_update_launch(A, lda, T, ldt, F, ldf, M, K, N, O, ldo, ctx->dev_flag, (cudaStream_t)stream);
}
