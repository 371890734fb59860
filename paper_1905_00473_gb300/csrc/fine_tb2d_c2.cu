// 2D FP32 fine propagator with temporal blocking, two columns per thread.
//
// Same computation and pass structure as fine_tb2d.cu: B velocity-Verlet
// levels (kick v += w_g kappa D(u), drift u += dt v; Sec. 3.1 scheme) per HBM
// pass, every slice of a sweep in one persistent launch (Alg. 3, parFor), the
// residual carried between passes as bfloat16 and the stencil applied as
// D(u) = D0 + D(du) with D0 = D(u_hi) (pr_internal.cuh).  What differs is the
// thread geometry, chosen for latency hiding:
//
//   * thread t owns columns 2t, 2t+1 of full periodic rows, so a row of n
//     points takes n/2 threads: 16 warps per SM for n = 1024 against 8 with
//     four columns per thread.  The register state per thread halves (three
//     du rows and one u_t row per level, two columns each), which is what
//     lets twice as many warps fit the register file at depth 8.
//   * kappa is stored pre-interleaved per thread (kappa0 kappa1 . .), so the
//     TMA copy of a kappa row leaves room for D0 next to it and a level reads
//     both with one 128-bit shared load.
//   * static rings: the row loop is unrolled 12-fold, the depth of the
//     kappa/D0 ring, which the u_hi/u_t/residual ring (6), the x-edge buffers
//     (2) and the register rings (3) divide; every segment starts at a ring
//     position that is a multiple of 12, so each unrolled step addresses its
//     slots and mbarriers at compile-time offsets, and positions that get no
//     copy receive a plain mbarrier arrival (the wait parity is the lap
//     parity).
//   * the x-neighbour edges go through a double-buffered shared array: with
//     one barrier per row, a buffer written at row i is read at row i + 1 and
//     rewritten at row i + 2, after the barrier that ends row i + 1.
//
// Pipeline per row i (q the running row index of the CTA): row i + P is
// requested by TMA, row i arrives, D0 of row i - 1 is formed, level l advances
// row i - 1 - l, and row i - B leaves finished.
#include "pr_internal.cuh"
#include "tb_common.cuh"

namespace {
using namespace tb;

constexpr int kC = 2;     // columns per thread
constexpr int kPre = 2;   // rows requested ahead of the consumer
constexpr int kU = 12;    // loop unroll = rows of the kappa/D0 ring
constexpr int kRS = 6;    // u_hi / u_t / residual ring: rows q-2 .. q+kPre
static_assert(kU % 3 == 0 && kU % kRS == 0 && kU % 2 == 0, "every ring period must divide the unroll");
static_assert(kRS >= kPre + 3, "the shallow ring holds rows q-2 .. q+kPre");

template <int NT, int B>
struct C2Smem {
    static_assert(kU >= B + kPre + 1, "the kappa/D0 ring holds rows q-B .. q+kPre");
    static constexpr int W = NT * kC;                        // row width n
    static constexpr int RD = kU;                            // kappa/D0 ring: rows q-B .. q+kPre
    static constexpr uint32_t deep_row = NT * 16;            // [t][kappa0 kappa1 D0_0 D0_1]
    static constexpr uint32_t sh_row = W * 10;               // u_hi W | u_t W (float) | r W (bf16)
    static constexpr uint32_t xbuf_floats = B * 2 * NT;      // one buffer: [B][left|right][NT]
    static constexpr uint32_t deep_bytes = RD * deep_row;
    static constexpr uint32_t sh_bytes = kRS * sh_row;
    static constexpr uint32_t xbuf_bytes = 2 * xbuf_floats * 4;
    static constexpr uint32_t bar_bytes = RD * 8;
    static constexpr uint32_t total = deep_bytes + sh_bytes + xbuf_bytes + bar_bytes;
    static_assert((deep_row & (deep_row - 1)) == 0, "deep row must be a power of two");
    static_assert(sh_row % 16 == 0 && (W * 4) % 16 == 0, "TMA destinations must be 16-byte aligned");
};

template <int NT, int B>
struct C2Shared {
    unsigned char* deep;   // [RD][deep_row]
    unsigned char* shal;   // [kRS][sh_row]
    float* xbuf;           // [2][B][2][NT]
    uint64_t* bars;        // [RD], one per kappa/D0 slot, completes the row's copies
};

// Request local row rho of the segment (kappa, u_hi, u_t, residual) into the
// given slots; called by one thread.
template <int NT, int B>
__device__ __forceinline__ void c2_issue(const Tb2dParams& p, const Seg& sg, const C2Shared<NT, B>& sh,
                                         int rho, uint32_t doff, uint32_t soff) {
    using S = C2Smem<NT, B>;
    const int n = p.n;
    const int y = seg_row(sg.ylo, rho, n);
    const int64_t off = (int64_t)y * n;
    uint64_t* bar = &sh.bars[doff / S::deep_row];
    mbar_expect_tx(bar, S::deep_row + 8u * S::W + (sg.r_s ? 2u * S::W : 0u) + p.tx_extra);
    bulk_g2s(sh.deep + doff, p.kap + 2 * off, S::deep_row, bar, policy(1));
    bulk_g2s(sh.shal + soff, sg.u_s + off, 4u * S::W, bar, policy(2));
    bulk_g2s(sh.shal + soff + 4 * S::W, sg.v_s + off, 4u * S::W, bar, policy(0));
    if (sg.r_s) bulk_g2s(sh.shal + soff + 8 * S::W, sg.r_s + off, 2u * S::W, bar, policy(0));
}

// One row of the pipeline at ring position q = sg.base + i, K = q mod 12;
// K mod 3 names the register ring slots:
//   R[l][.]  du rows of level l's input: centre K%3, south (K+2)%3, north
//            (K+1)%3 (written this row by the level below)
//   VV[l][.] u_t of level l's input row: read (K+2)%3, written K%3
// `par` is the mbarrier phase parity of the current ring lap.  Returns true
// when some thread's bounded wait gave up.
template <int NT, int B, bool MID, int K>
__device__ __forceinline__ bool c2_iter(const Tb2dParams& p, const Seg& sg, const C2Shared<NT, B>& sh,
                                        int i, uint32_t par, float (&R)[B][3][kC], float (&VV)[B][3][kC],
                                        int& timed_out, uint32_t& consumed, uint32_t& issued_end) {
    using S = C2Smem<NT, B>;
    constexpr int W = S::W;
    constexpr int CUR = K % 3, PRV = (K + 2) % 3, NXT = (K + 1) % 3;
    constexpr uint32_t SQ = (K % kRS) * S::sh_row, S1 = ((K + kRS - 1) % kRS) * S::sh_row,
                       S2 = ((K + kRS - 2) % kRS) * S::sh_row;
    constexpr uint32_t DN = ((K + kPre) % kU) * S::deep_row, SN = ((K + kPre) % kRS) * S::sh_row;
    // deep slot of the row at offset c from position q
    auto dslot = [](int c) { return (uint32_t)(((K + c + 2 * kU) % kU) * S::deep_row); };
    const int t = threadIdx.x;
    const int n = p.n;
    const int L = MID ? B : sg.L;
    const uint32_t q = sg.base + (uint32_t)i;
    auto gy = [&](int rho) { return seg_row(sg.ylo, rho, n); };

    // ---- producer: row i + kPre ---------------------------------------------
    if (t == 0 && i + kPre < sg.nload) {
        c2_issue<NT, B>(p, sg, sh, i + kPre, DN, SN);
        issued_end = sg.base + (uint32_t)(i + kPre + 1);
    }

    // ---- the finished row's u_hi, fetched early from L2 ----------------------
    const int rho_out = i - B;
    const bool do_out = rho_out >= L && rho_out < L + sg.H;
    int64_t off_out = 0;
    float2 u0o = make_float2(0.f, 0.f);
    if (do_out) {
        off_out = sg.slice_off + (int64_t)gy(rho_out) * n + kC * t;
        u0o = __ldcs((const float2*)(p.u_in + off_out));
    }

    // ---- load stage: row i arrives; D0 of row i-1 -----------------------------
    float d0n[kC] = {0.f, 0.f};
    const bool have_row = i < sg.nload;
    if (have_row) {
        if (!timed_out && !mbar_wait_bounded(&sh.bars[K], par, p.wait_ns)) {
            atomicExch(p.flag, 1);
            timed_out = 1;
        }
        consumed = q + 1;
        const unsigned char* s0 = sh.shal + SQ;
        const float2 u2 = *(const float2*)(s0 + 8 * t);
        if (sg.r_s) {
            const uint32_t rw = *(const uint32_t*)(s0 + 8 * W + 4 * t);
            R[0][NXT][0] = pr_bf16_lo(rw);
            R[0][NXT][1] = pr_bf16_hi(rw);
        } else {
            R[0][NXT][0] = 0.0f;
            R[0][NXT][1] = 0.0f;
        }
        if (i >= 1) {
            // rows i-1 (centre) and i-2 (south; row i-1 again at i = 1, where
            // the south row does not exist and D0 only feeds halo rows)
            const float* s1 = (const float*)(sh.shal + S1);
            const float* s2 = (const float*)(sh.shal + (i >= 2 ? S2 : S1));
            const float2 a = *(const float2*)(s1 + kC * t);
            const float2 b = *(const float2*)(s2 + kC * t);
            const float xl = s1[(kC * t + W - 1) % W], xr = s1[(kC * t + kC) % W];
            d0n[0] = ((xl - a.x) + (a.y - a.x)) + ((b.x - a.x) + (u2.x - a.x));
            d0n[1] = ((a.x - a.y) + (xr - a.y)) + ((b.y - a.y) + (u2.y - a.y));
        }
    } else {
        R[0][NXT][0] = 0.0f;
        R[0][NXT][1] = 0.0f;
    }

    // ---- levels: level l advances row i-1-l -----------------------------------
    const float* xr = sh.xbuf + (size_t)((K & 1) ^ 1) * S::xbuf_floats;
    const int tl = (t + NT - 1) % NT, tr = (t + 1) % NT;
    const f2_t dt2 = f2_pack(p.dt, p.dt), m4 = f2_pack(-4.0f, -4.0f);
    float dout[kC], vout[kC];
#pragma unroll
    for (int l = 0; l < B; ++l) {
        const unsigned char* drow = sh.deep + dslot(-1 - l);
        float vin[kC];
        if (l == 0) {
            const float2 v2 = *(const float2*)(sh.shal + S1 + 4 * W + 8 * t);
            vin[0] = v2.x;
            vin[1] = v2.y;
        } else {
            vin[0] = VV[l][PRV][0];
            vin[1] = VV[l][PRV][1];
        }
        float dn[kC], vn[kC];
        if (MID || l < L) {
            float k0, k1, e0, e1;
            if (l == 0) {
                const float2 k2 = *(const float2*)(drow + 16 * t);
                k0 = k2.x;
                k1 = k2.y;
                e0 = d0n[0];
                e1 = d0n[1];
            } else {
                const float4 k4 = *(const float4*)(drow + 16 * t);
                k0 = k4.x;
                k1 = k4.y;
                e0 = k4.z;
                e1 = k4.w;
            }
            const float xl = xr[(2 * l + 1) * NT + tl];   // right edge of the left thread
            const float xrt = xr[(2 * l) * NT + tr];      // left edge of the right thread
            bool dr = true;
            if (!MID) {
                const int g = p.g0 + l;
                if (g == 0 || g == p.m) {
                    k0 *= 0.5f;
                    k1 *= 0.5f;
                }
                dr = g < p.m;
            }
            // D(u) = D0 + (du_S + du_N + du_W + du_E - 4 du_C); the fresh north
            // row enters last to keep the level-to-level chain short
            const float c0 = R[l][CUR][0], c1 = R[l][CUR][1];
            const f2_t cc = f2_pack(c0, c1);
            const f2_t hs = f2_add(f2_pack(xl + c1, c0 + xrt), f2_pack(R[l][PRV][0], R[l][PRV][1]));
            const f2_t part = f2_add(f2_pack(e0, e1), f2_fma(m4, cc, hs));
            const f2_t v2 = f2_fma(f2_pack(k0, k1), f2_add(part, f2_pack(R[l][NXT][0], R[l][NXT][1])),
                                   f2_pack(vin[0], vin[1]));
            const f2_t d2 = dr ? f2_fma(dt2, v2, cc) : cc;
            vn[0] = f2_lo(v2);
            vn[1] = f2_hi(v2);
            dn[0] = f2_lo(d2);
            dn[1] = f2_hi(d2);
        } else {
            vn[0] = vin[0];
            vn[1] = vin[1];
            dn[0] = R[l][CUR][0];
            dn[1] = R[l][CUR][1];
        }
        if (l + 1 < B) {
            R[l + 1][NXT][0] = dn[0];
            R[l + 1][NXT][1] = dn[1];
            VV[l + 1][CUR][0] = vn[0];
            VV[l + 1][CUR][1] = vn[1];
        } else {
            dout[0] = dn[0];
            dout[1] = dn[1];
            vout[0] = vn[0];
            vout[1] = vn[1];
        }
    }

    // ---- row i-B leaves the pipeline -------------------------------------------
    if (do_out) {
        float o0, o1;
        if (MID || p.r_out) {
            float r0, r1;
            o0 = pr_two_sum(u0o.x, dout[0], &r0);
            o1 = pr_two_sum(u0o.y, dout[1], &r1);
            *(uint32_t*)(p.r_out + off_out) = pr_bf16x2(r0, r1);
        } else {
            o0 = u0o.x + dout[0];
            o1 = u0o.y + dout[1];
        }
        *(float2*)(p.u_out + off_out) = make_float2(o0, o1);
        *(float2*)(p.v_out + off_out) = make_float2(vout[0], vout[1]);
    }

    // ---- shared stores, read only after the barrier ------------------------------
    float* xw = sh.xbuf + (size_t)(K & 1) * S::xbuf_floats;
#pragma unroll
    for (int l = 0; l < B; ++l) {
        if (MID || l < L) {   // level l's next input row: its edges, read by level l next row
            xw[(2 * l) * NT + t] = R[l][NXT][0];
            xw[(2 * l + 1) * NT + t] = R[l][NXT][1];
        }
    }
    if (have_row && i >= 1)
        *(float2*)(sh.deep + dslot(-1) + 16 * t + 8) = make_float2(d0n[0], d0n[1]);
    // one barrier per row; it also makes the abort decision uniform
    return __syncthreads_or(timed_out) != 0;
}

template <int NT, int B, bool MID>
__global__ void __launch_bounds__(NT, 512 / NT) fine_tb2d_c2_kernel(const Tb2dParams p) {
    using S = C2Smem<NT, B>;
    constexpr int kRD = S::RD;
    extern __shared__ __align__(128) unsigned char smem[];
    C2Shared<NT, B> sh;
    sh.deep = smem;
    sh.shal = smem + S::deep_bytes;
    sh.xbuf = (float*)(smem + S::deep_bytes + S::sh_bytes);
    sh.bars = (uint64_t*)(smem + S::deep_bytes + S::sh_bytes + S::xbuf_bytes);

    const int t = threadIdx.x;
    const int n = p.n;
    const int64_t pts = (int64_t)n * n;
    const int L = MID ? B : p.levels;
    // an earlier pass of this context gave up waiting: its results are not
    // valid, skip the work until pr_check reports and clears the flag
    if (*(volatile int*)p.flag) return;

    if (t == 0) {
        for (int s = 0; s < kRD; ++s) mbar_init(&sh.bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    // per-CTA row ranges of equal cost: rows + (L + B) steps per segment
    const int64_t r_begin = balanced_row(p.rows_total, n, L + B, blockIdx.x, gridDim.x);
    const int64_t r_end = balanced_row(p.rows_total, n, L + B, blockIdx.x + 1, gridDim.x);
    // ring positions: a segment occupies [base, base + niter) and the next one
    // starts at the following multiple of kU; positions that receive no copy
    // get a plain arrival, so slot s completes its phase j at position j kU + s
    uint32_t pos = 0, consumed = 0, issued_end = 0;
    int timed_out = 0;
    bool aborted = false;

    for (int64_t seg0 = r_begin; seg0 < r_end && !aborted;) {
        Seg sg;
        const int64_t slice = seg0 / n;
        const int ya = (int)(seg0 - slice * n);
        const int64_t seg1 = min(r_end, (slice + 1) * (int64_t)n);
        sg.H = (int)(seg1 - seg0);
        seg0 = seg1;
        sg.L = L;
        sg.nload = sg.H + 2 * L;
        sg.slice_off = slice * pts;
        sg.u_s = p.u_in + slice * pts;
        sg.v_s = p.v_in + slice * pts;
        sg.r_s = p.r_in ? p.r_in + slice * pts : nullptr;
        sg.base = pos;
        int ylo = (ya - L) % n;
        sg.ylo = ylo < 0 ? ylo + n : ylo;
        const int niter = sg.H + L + B;

        if (t == 0) {
            for (int rho = 0; rho < kPre && rho < sg.nload; ++rho) {
                c2_issue<NT, B>(p, sg, sh, rho, (uint32_t)rho * S::deep_row, (uint32_t)rho * S::sh_row);
                issued_end = pos + (uint32_t)rho + 1;
            }
        }

        float R[B][3][kC], VV[B][3][kC];
#pragma unroll
        for (int l = 0; l < B; ++l)
#pragma unroll
            for (int s = 0; s < 3; ++s)
#pragma unroll
                for (int k = 0; k < kC; ++k) R[l][s][k] = VV[l][s][k] = 0.0f;

        uint32_t par = (pos / kU) & 1u;
        int i = 0;
#define PR_C2_STEP(K)                                                                             \
    if (i >= niter) break;                                                                         \
    if (c2_iter<NT, B, MID, K>(p, sg, sh, i, par, R, VV, timed_out, consumed, issued_end)) {       \
        aborted = true;                                                                            \
        break;                                                                                     \
    }                                                                                              \
    ++i;
        for (;;) {
            PR_C2_STEP(0) PR_C2_STEP(1) PR_C2_STEP(2) PR_C2_STEP(3) PR_C2_STEP(4) PR_C2_STEP(5)
            PR_C2_STEP(6) PR_C2_STEP(7) PR_C2_STEP(8) PR_C2_STEP(9) PR_C2_STEP(10) PR_C2_STEP(11)
            par ^= 1u;
        }
#undef PR_C2_STEP
        if (aborted) break;
        // close the lap: complete the phases of the positions that got no copy
        const uint32_t next = (pos + (uint32_t)niter + kU - 1) / kU * kU;
        if (t == 0)
            for (uint32_t q = pos + (uint32_t)sg.nload; q < next; ++q) mbar_arrive(&sh.bars[q % kU]);
        pos = next;
    }
    if (aborted && t == 0) {
        // let copies still in flight land before the CTA's shared memory is
        // released (test hook: settle the tx_extra bytes no copy brings first)
        for (uint32_t q = consumed; q < issued_end; ++q) {
            if (p.tx_extra) mbar_complete_tx(&sh.bars[q % kU], p.tx_extra);
            (void)mbar_wait_bounded(&sh.bars[q % kU], (q / kU) & 1u, p.wait_ns / 10);
        }
    }
}

template <int NT, int B, bool MID>
pr_status c2_launch_cfg(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st) {
    using S = C2Smem<NT, B>;
    auto kern = fine_tb2d_c2_kernel<NT, B, MID>;
    static int configured_dev = -1;
    static int blocks_per_sm = 0;
    static int sms = 0;
    if (configured_dev != ctx->device) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::total);
        if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb2d-c2: set shared memory size");
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, NT, S::total);
        if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb2d-c2: occupancy");
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        if (blocks_per_sm < 1) return pr_fail(ctx, PR_ECUDA, "tb2d-c2: kernel does not fit on an SM");
        configured_dev = ctx->device;
    }
    Tb2dParams p;
    p.u_in = (const float*)ps.u_in;
    p.v_in = (const float*)ps.v_in;
    p.r_in = (const uint16_t*)ps.r_in;
    p.kap = (const float*)ctx->kappa_il;
    p.u_out = (float*)ps.u_out;
    p.v_out = (float*)ps.v_out;
    p.r_out = (uint16_t*)ps.r_out;
    p.flag = ctx->dev_flag;
    p.rows_total = (int64_t)ps.nslices * ctx->n;
    p.n = (int)ctx->n;
    p.g0 = ps.g0;
    p.levels = ps.levels;
    p.m = ps.m;
    p.dt = (float)ctx->dt_f;
    p.tx_extra = ctx->debug_stall ? 16u : 0u;
    p.wait_ns = ctx->debug_stall ? 200000000ull : 2000000000ull;
    int64_t grid = (int64_t)sms * blocks_per_sm;
    if (grid > p.rows_total) grid = p.rows_total;
    kern<<<(int)grid, NT, S::total, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb2d-c2: launch");
    return PR_OK;
}

template <int NT, int B>
pr_status c2_launch_depth(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st) {
    const bool mid = ps.levels == B && ps.g0 >= 1 && ps.g0 + B - 1 < ps.m && ps.r_in && ps.r_out;
    return mid ? c2_launch_cfg<NT, B, true>(ctx, ps, st) : c2_launch_cfg<NT, B, false>(ctx, ps, st);
}

template <int B>
pr_status c2_launch_n(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st) {
    switch (ctx->n) {
        case 128: return c2_launch_depth<64, B>(ctx, ps, st);
        case 256: return c2_launch_depth<128, B>(ctx, ps, st);
        case 512: return c2_launch_depth<256, B>(ctx, ps, st);
        case 1024: return c2_launch_depth<512, B>(ctx, ps, st);
        default: return pr_fail(ctx, PR_EINVAL, "tb2d-c2: unsupported grid size");
    }
}

}  // namespace

// A pass of 2..B levels with the two-column kernel (same contract as
// pr_launch_fine_tb2d; the caller has checked pr_tb2d_supported).
pr_status pr_launch_fine_tb2d_c2(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st) {
    if (!ctx->kappa_il) return pr_fail(ctx, PR_EINVAL, "tb2d-c2: interleaved kappa missing");
    const int B = ctx->block_depth;
    if (ps.levels < 2 || ps.levels > B) return pr_fail(ctx, PR_EINVAL, "tb2d-c2: bad level count");
    if (B == 8) return c2_launch_n<8>(ctx, ps, st);
    if (B == 4) return c2_launch_n<4>(ctx, ps, st);
    return pr_fail(ctx, PR_EINVAL, "tb2d-c2: unsupported depth");
}
