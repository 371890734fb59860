#pragma once
// 2D FP32 fine propagator with temporal blocking (device code shared by
// fine_tb2d.cu, fine_tb2d_wide.cu and fine_tb2d_sweep.cu): B velocity-Verlet levels
// per HBM pass, all slices of a sweep in one persistent launch.
//
// What is computed is exactly the level recurrence of fine_naive.cu (kick
// v += w_g kappa D(u), drift u += dt v, Sec. 3.1 scheme, Alg. 3 parFor over
// slices); this file only changes where the data lives while it is computed.
//
// Geometry.  A CTA owns full rows of one slice (periodic in x inside the
// CTA, so there is no x-halo): thread t holds columns 4t..4t+3 of every row
// in registers.  Rows stream through a B-deep software pipeline: at
// iteration i the row i arrives, level l (l = 0..B-1) advances row i-1-l by
// one kick+drift, and row i-B leaves the pipeline finished.  A level needs
// its own column's rows above/below (registers) and the x-neighbours of its
// edge columns, which come from the neighbouring threads through a small
// double-buffered shared array written one iteration earlier (in middle
// passes the edges of four levels travel as one 16-byte vector).  One barrier
// per row.
//
// Cluster rows (n = 2048 at depth 8).  A row is shared by the two CTAs of a
// thread-block cluster, each holding one half.  The threads at the ends of a
// half-row store their wrap-around x-edges into the partner's edge buffer
// with st.async, which completes transaction bytes on an mbarrier there;
// the partner's opposite end thread waits for them (bounded) and then reads
// its own buffer exactly as a whole-row CTA does.  No CTA reads the other's
// shared memory and there is no cluster barrier per row: a CTA can run at
// most one step ahead of its partner, which the double-buffered edges allow.
// D0 at the ends takes the u_hi columns beyond the half-row from a 16-byte
// bulk copy per side.  Cluster barriers at entry and exit (after the last
// pushes have landed) bracket the exchange.
//
// Register rings.  What a thread reads again for its own columns stays in
// registers: the du and u_t rows of every level, u_hi of the last three rows
// (for D0), and, in whole-row CTAs, kappa of the last 12 rows (read from
// shared memory once, when the row arrives) and, in middle passes of
// CTAs that hold whole rows alone, D0 of the last 12 rows.
//
// Loads.  One elected thread streams rows with cp.async.bulk (TMA bulk
// copies: rows are contiguous and 16-byte aligned) into shared-memory rings
// guarded by one mbarrier per row slot: kappa into a 12-row ring (whose other
// half holds D0 where D0 is not kept in registers), u_hi, u_t and the
// bfloat16 residual into a 6-row ring.  The finished row re-reads its u_hi
// from L2.
// Waits are bounded: after ~2 s the CTA records PR_ETIMEOUT in a device flag
// and all its threads leave the loop together.
//
// Static rings.  The row loop is unrolled 12-fold, the kappa/D0 ring depth,
// which the shallow ring (6), the x-edge buffers (2) and the register rings
// (3, 12) divide.  Every segment starts at a ring position that is a multiple of
// 12, so each unrolled step addresses its slots, mbarriers and buffers at
// compile-time offsets; positions that receive no copy (drain steps, the
// padding to the next multiple of 12) get a plain mbarrier arrival, so slot s
// completes its j-th phase at position 12 j + s and the wait parity is the
// parity of the ring lap.
//
// Precision.  Between passes u is (u_hi float, bfloat16 rounding residual:
// pr_internal.cuh); inside a pass
// the state is du = u - u_hi with the stencil applied as
// D(u) = D0 + D(du), D0 = D(u_hi) formed from differences once per pass.
//
// Work split.  The N*n rows of the batch are cut into one contiguous range
// per CTA (persistent grid of #SM * occupancy CTAs); a range that crosses a
// slice boundary is processed as separate segments, each with its own
// L-row halo above and below (periodic in y), and the cut points balance
// rows plus the halo and drain steps of every segment (balanced_row).
//
// Variants.  MID = a pass in which all B levels kick and drift and a residual
// goes out: the middle passes (no half kick) and, with HALF0, the first pass
// (half kick at level 0, no residual in).  The general variant handles the
// last pass (half kick at g = m, no drift, fewer than B levels: the missing
// levels pass rows through unchanged).  At depth 8 the last pass may hold 9
// levels, so that a sweep of 8 k + 1 levels needs no one-level pass.
#include "pr_internal.cuh"
#include "tb_common.cuh"

namespace {
using namespace tb;

constexpr int kCpt = 4;   // columns per thread
constexpr int kPre = 2;   // rows requested ahead of the consumer
constexpr int kU = 12;    // rows of the kappa/D0 ring, and the unroll of the row loop
constexpr int kRS = 6;    // rows of the u_hi / u_t / residual ring
static_assert(kU % 3 == 0 && kU % kRS == 0, "the small ring periods must divide the unroll");

// Deep-ring slot of the row at static offset c from ring position q, with
// kc = (q mod kU) + c a constant once the loops are unrolled.
__device__ __forceinline__ constexpr uint32_t dslot(int kc) { return (uint32_t)((kc + 2 * kU) % kU); }

// Shared memory of one CTA.  Every ring slot, mbarrier and x-edge buffer of
// the pipeline step that handles ring position q is (q mod its ring size), a
// compile-time constant inside the kU-fold unrolled loop, because every
// segment starts at a ring position that is a multiple of kU.
template <int NT, int B>
struct Smem {
    static_assert(kU >= B + kPre + 1, "the kappa/D0 ring holds rows q-B .. q+kPre");
    static constexpr int W = NT * kCpt;                          // columns held: n, or an x-strip
    static constexpr uint32_t deep_row = 2u * W * 4;             // kappa W | D0 W
    static constexpr uint32_t sh_row = 10u * W;                  // u_hi W | u_t W (float) | r W (bf16)
    static constexpr uint32_t deep_bytes = kU * deep_row;
    static constexpr uint32_t sh_bytes = kRS * sh_row;
    // x-edge exchange, double-buffered.  Middle passes: [2][left|right][NQ][NT]
    // float4, the edges of levels 4q..4q+3 of a thread in one 16-byte vector;
    // the general variant: [2][B][left|right][NT] float.
    // Depths 8 and 9 share one layout (the vector form is used only up to
    // depth 8, the scalar form is sized for 9 levels), so that the passes of
    // a whole sweep in one launch find the ring mbarriers at one address.
    static constexpr int NQ = (B + 3) / 4;
    static constexpr int BQ = B < 8 ? B : 8, BS = (B == 8 || B == 9) ? 9 : B;
    static constexpr uint32_t xq_bytes = 2u * 2 * ((BQ + 3) / 4) * NT * 16, xs_bytes = 2u * BS * 2 * NT * 4;
    static constexpr uint32_t xbuf_bytes = xq_bytes > xs_bytes ? xq_bytes : xs_bytes;
    // cluster rows: the u_hi columns just outside the half-row (4 each side)
    // per shallow slot, and the exchange mbarriers, one per (step parity b,
    // end s: 0 = thread 0, 1 = thread NT-1, part q = levels 4q..4q+3)
    static constexpr uint32_t halo_bytes = kRS * 2 * 16;
    static constexpr uint32_t bar_bytes = (kU + 2 * 2 * NQ) * 8;   // ring slots, then the exchange
    static constexpr uint32_t total = deep_bytes + sh_bytes + xbuf_bytes + halo_bytes + bar_bytes;
    static_assert(deep_row % 16 == 0 && sh_row % 16 == 0 && (W * 4) % 16 == 0,
                  "bulk-copy destinations must stay 16-byte aligned");
    __device__ static unsigned char* deep(unsigned char* sm, uint32_t slot) { return sm + slot * deep_row; }
    __device__ static unsigned char* shal(unsigned char* sm, uint32_t slot) {
        return sm + deep_bytes + slot * sh_row;
    }
    __device__ static float4* xbuf4(unsigned char* sm, uint32_t buf) {
        return (float4*)(sm + deep_bytes + sh_bytes) + buf * (2 * NQ * NT);
    }
    __device__ static float* xbuf1(unsigned char* sm, uint32_t buf) {
        return (float*)(sm + deep_bytes + sh_bytes) + buf * (B * 2 * NT);
    }
    __device__ static float4* halo(unsigned char* sm, uint32_t slot, uint32_t side) {
        return (float4*)(sm + deep_bytes + sh_bytes + xbuf_bytes) + slot * 2 + side;
    }
    __device__ static uint64_t* bar(unsigned char* sm, uint32_t slot) {
        return (uint64_t*)(sm + deep_bytes + sh_bytes + xbuf_bytes + halo_bytes) + slot;
    }
    __device__ static uint64_t* ebar(unsigned char* sm, uint32_t b, uint32_t s, uint32_t q) {
        return bar(sm, kU + (b * 2 + s) * NQ + q);
    }
    static constexpr uint32_t part_tx = 16;   // bytes pushed per part and step
};

struct Pols {
    uint64_t first, last, norm;   // L2 evict-first (streamed), evict-last (kappa), normal (u_hi)
};

// Rows shared by the two CTAs of a cluster (n = 8 NT): the count of steps
// this CTA has finished, the same in both CTAs because they walk the same
// segments.
struct Pair {
    uint32_t step;
};

// Cluster-row exchange.  The end threads of a half-row (t = 0 and NT-1)
// write their wrap-around x-edge entries (thread 0's left edges, thread
// NT-1's right edges) into the partner's x-edge buffer, at the same offset,
// instead of their own: each entry is then read by the partner's opposite
// end thread exactly as a whole-row CTA reads its own.  A push of part q
// (the edges of levels 4q..4q+3 of global step g) completes 16 bytes on the
// partner's mbarrier (g & 1, receiving end, q).  The receiving thread waits
// for phase ((g-1) >> 1) & 1 before reading part q at step g and re-arms
// the mbarrier (one arrival with 16 expected bytes) for step g+1.
template <int NT, int B>
__device__ __forceinline__ bool rx_wait(unsigned char* sm, uint32_t g, int q, uint64_t limit_ns) {
    using S = Smem<NT, B>;
    const uint32_t side = threadIdx.x == 0 ? 0u : 1u;
    return mbar_wait_bounded(S::ebar(sm, (g - 1) & 1u, side, q), ((g - 1) >> 1) & 1u, limit_ns);
}
template <int NT, int B>
__device__ __forceinline__ void rx_rearm(unsigned char* sm, uint32_t g, int q) {
    using S = Smem<NT, B>;
    const uint32_t side = threadIdx.x == 0 ? 0u : 1u;
    mbar_expect_tx(S::ebar(sm, (g - 1) & 1u, side, q), S::part_tx);
}
// the partner's mbarrier that a push of part q at step g completes
template <int NT, int B>
__device__ __forceinline__ uint32_t tx_bar(unsigned char* sm, uint32_t g, int q, uint32_t prank) {
    using S = Smem<NT, B>;
    const uint32_t side = threadIdx.x == 0 ? 1u : 0u;   // received by the partner's opposite end
    return mapa_rank(smem_u32(S::ebar(sm, g & 1u, side, q)), prank);
}

// Request local row rho of the segment (kappa, u_hi, u_t, residual) into the
// deep slot DS and the shallow slot SS; called by one thread.
template <int NT, int B, int XH, int CL>
__device__ __forceinline__ void issue_row(const Tb2dParams& p, const Seg& sg, unsigned char* sm, int rho,
                                          uint32_t DS, uint32_t SS, const Pols& pol) {
    using S = Smem<NT, B>;
    constexpr int W = S::W;
    const int n = p.n;
    // whole rows start at column 0; a cluster CTA's part of a row at x0
    const int64_t off = (int64_t)seg_row(sg.ylo, rho, n) * n + (CL > 1 ? sg.x0 : 0);
    uint64_t* bar = S::bar(sm, DS);
    unsigned char* drow = S::deep(sm, DS);
    unsigned char* srow = S::shal(sm, SS);
    constexpr uint32_t row_bytes = (uint32_t)W * 4;
    mbar_expect_tx(bar, 3 * row_bytes + (sg.r_s ? (uint32_t)W * 2 : 0u) + (CL > 1 ? 32u : 0u) + p.tx_extra);
    if (XH == 0) {
        bulk_g2s(drow, p.kap + off, row_bytes, bar, pol.last);
        bulk_g2s(srow, sg.u_s + off, row_bytes, bar, pol.norm);
        if (CL > 1) {
            // u_hi columns x0-4..x0-1 and x0+W..x0+W+3 (periodic), for D0 at
            // the ends of the half-row
            const int64_t row0 = off - sg.x0;
            const int xl = sg.x0 == 0 ? n - 4 : sg.x0 - 4, xr = sg.x0 + W == n ? 0 : sg.x0 + W;
            bulk_g2s(S::halo(sm, SS, 0), sg.u_s + row0 + xl, 16u, bar, pol.norm);
            bulk_g2s(S::halo(sm, SS, 1), sg.u_s + row0 + xr, 16u, bar, pol.norm);
        }
        bulk_g2s(srow + W * 4, sg.v_s + off, row_bytes, bar, pol.first);
        if (sg.r_s) bulk_g2s(srow + W * 8, sg.r_s + off, (uint32_t)W * 2, bar, pol.first);
    } else {
        bulk_row_g2s(drow, p.kap + off, sg.x0, W, n, 4, bar, pol.last);
        bulk_row_g2s(srow, sg.u_s + off, sg.x0, W, n, 4, bar, pol.norm);
        bulk_row_g2s(srow + W * 4, sg.v_s + off, sg.x0, W, n, 4, bar, pol.first);
        if (sg.r_s) bulk_row_g2s(srow + W * 8, sg.r_s + off, sg.x0, W, n, 2, bar, pol.first);
    }
}

// OR of v over the GB threads of a thread group (whole warps, all executing
// this barrier), at the named barrier `id` (1 + the group's index): the
// per-row barrier of a group that holds its rows alone inside a larger CTA.
template <int GB>
__device__ __forceinline__ bool group_or(int v, int id) {
    static_assert(GB % 32 == 0, "a named barrier counts whole warps");
    int r;
    if (id == 1) {   // the first group (the only one of single-group CTAs): an immediate barrier id
        asm volatile(
            "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
            : "=r"(r)
            : "r"(v), "n"(GB)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.or.pred q, %2, %3, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
            : "=r"(r)
            : "r"(v), "r"(id), "n"(GB)
            : "memory");
    }
    return r != 0;
}

// One pipeline step at ring position q = sg.base + i with K = q mod kU.
// Register rings per level l (period 3, K mod 3 selects the slots):
//   R[l][.]  du rows of level l's input: centre = K%3, south = (K+2)%3,
//            north = (K+1)%3 (written this step by the level below)
//   VV[l][.] u_t of level l's input row: read (K+2)%3, written K%3
// `par` is the mbarrier phase parity of the current ring lap.  Returns true
// when some thread's bounded wait gave up.
template <int NT, int B, int XH, bool MID, bool HALF0, int CL, int K, int SWEEP, int GB>
__device__ __forceinline__ bool tb2d_step(const Tb2dParams& p, const Seg& sg, unsigned char* sm, int i,
                                          uint32_t par, float (&R)[B][3][kCpt], float (&VV)[B][3][kCpt],
                                          float (&UH)[3][kCpt], float (&KR)[kU][kCpt], float (&DR)[kU][kCpt],
                                          int& timed_out, uint32_t& consumed, uint32_t& issued_end,
                                          const Pols& pol, Pair& pr, int grp) {
    using S = Smem<NT, B>;
    constexpr int W = S::W;
    constexpr int CUR = K % 3, PRV = (K + 2) % 3, NXT = (K + 1) % 3;
    constexpr uint32_t SQ = K % kRS, S1 = (K + kRS - 1) % kRS, S2 = (K + kRS - 2) % kRS;
    constexpr uint32_t SN = (K + kPre) % kRS;
    const int t = GB == 0 ? (int)threadIdx.x : (int)threadIdx.x - grp * GB;
    const int n = p.n;
    const int L = MID ? B : sg.L;

    // ---- producer: row i + kPre into the rings ---------------------------
    if (t == 0 && i + kPre < sg.nload) {
        issue_row<NT, B, XH, CL>(p, sg, sm, i + kPre, dslot(K + kPre), SN, pol);
        issued_end = sg.base + (uint32_t)(i + kPre + 1);
    }

    // ---- cluster rows: the partner's edges of the previous step have landed
    const bool xend = CL > 1 && (t == 0 || t == NT - 1);   // the ends of the half-row
    if constexpr (CL > 1) {
        if (xend && pr.step > 0 && !timed_out) {
#pragma unroll
            for (int q = 0; q < S::NQ; ++q) {
                if (!timed_out) {
                    if (rx_wait<NT, B>(sm, pr.step, q, p.wait_ns)) {
                        rx_rearm<NT, B>(sm, pr.step, q);
                    } else {
                        atomicExch(p.flag, 1);
                        timed_out = 1;
                    }
                }
            }
        }
    }

    // ---- the finished row's u_hi, fetched early from L2 ------------------
    const int rho_out = i - B;
    // in an x-strip only the columns at least XH from both strip edges are
    // final, and of the last strip of a row only those below n (strips of a
    // width that does not divide n overlap the first strip there)
    const bool do_out = rho_out >= L && rho_out < L + sg.H &&
                        (XH == 0 || (t >= XH / kCpt && t < NT - XH / kCpt && sg.x0 + kCpt * t < n));
    int64_t off_out = 0;
    float4 u0o = make_float4(0.f, 0.f, 0.f, 0.f);
    if (do_out) {
        off_out = sg.slice_off + (int64_t)seg_row(sg.ylo, rho_out, n) * n + sg.x0 + kCpt * t;
        if constexpr (SWEEP != 0) {
            // in a whole-sweep or work-queue launch the input was written by
            // other CTAs earlier in the launch: read it from L2, past this
            // SM's L1, marked evict-first there like the streamed rows
            const uint64_t ef = policy(0);
            asm volatile("ld.global.cg.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                         : "=f"(u0o.x), "=f"(u0o.y), "=f"(u0o.z), "=f"(u0o.w)
                         : "l"(p.u_in + off_out), "l"(ef));
        } else {
            u0o = __ldcs((const float4*)(p.u_in + off_out));
        }
    }

    // ---- load stage: row i arrives; D0 of row i-1 -------------------------
    float d0n[kCpt] = {0.f, 0.f, 0.f, 0.f};
    const bool have_row = i < sg.nload;
    if (have_row) {
        if (!timed_out && !mbar_wait_bounded(S::bar(sm, dslot(K)), par, p.wait_ns)) {
            atomicExch(p.flag, 1);
            timed_out = 1;
        }
        consumed = sg.base + (uint32_t)i + 1;
        const unsigned char* s0 = S::shal(sm, SQ);
        const float4 u4 = *(const float4*)(s0 + 16 * t);
        const float uu[4] = {u4.x, u4.y, u4.z, u4.w};
        // u_hi of rows i, i-1, i-2 in a register ring of period 3 (slot K % 3
        // holds row i), so D0 needs no shared loads for the thread's own columns
#pragma unroll
        for (int k = 0; k < kCpt; ++k) UH[CUR][k] = uu[k];
        // kappa of row i, read once: the B levels take it from a register ring
        // of kU rows (slot K) at the next B steps.  x-strip CTAs, whose 260
        // threads leave 168 registers a thread, and the whole-sweep kernel
        // (SWEEP 1, whose pass loop needs the registers) read it per level
        // instead.
        if constexpr (XH == 0 && SWEEP != 1) {
            const float4 kq = *(const float4*)((const float*)S::deep(sm, dslot(K)) + kCpt * t);
            KR[K][0] = kq.x;
            KR[K][1] = kq.y;
            KR[K][2] = kq.z;
            KR[K][3] = kq.w;
        }
        if (sg.r_s) {
            const uint2 r2 = *(const uint2*)(s0 + W * 8 + 2 * kCpt * t);
            R[0][NXT][0] = pr_bf16_lo(r2.x);
            R[0][NXT][1] = pr_bf16_hi(r2.x);
            R[0][NXT][2] = pr_bf16_lo(r2.y);
            R[0][NXT][3] = pr_bf16_hi(r2.y);
        } else {
#pragma unroll
            for (int k = 0; k < kCpt; ++k) R[0][NXT][k] = 0.0f;
        }
        if (i >= 1) {
            // rows i-1 (centre) and i-2 (south) from the register ring; at
            // i = 1 the south slot holds a stale row, and D0 of row 0 only
            // feeds halo rows
            const float* s1 = (const float*)S::shal(sm, S1);
            const float c[4] = {UH[PRV][0], UH[PRV][1], UH[PRV][2], UH[PRV][3]};
            const float s2v[4] = {UH[NXT][0], UH[NXT][1], UH[NXT][2], UH[NXT][3]};
            float xl, xrr;
            if (CL > 1 && t == 0) xl = S::halo(sm, S1, 0)->w;
            else xl = s1[(kCpt * t + W - 1) % W];
            if (CL > 1 && t == NT - 1) xrr = S::halo(sm, S1, 1)->x;
            else xrr = s1[(kCpt * t + kCpt) % W];
#if PR_TB2D_PACKED
            // columns (0,1) and (2,3) as f32x2 pairs, the same operations per lane
            const f2_t cp[2] = {f2_pack(c[0], c[1]), f2_pack(c[2], c[3])};
            const f2_t lp[2] = {f2_pack(xl, c[0]), f2_pack(c[1], c[2])};
            const f2_t rp[2] = {f2_pack(c[1], c[2]), f2_pack(c[3], xrr)};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const f2_t sp = f2_pack(s2v[2 * h], s2v[2 * h + 1]), up = f2_pack(uu[2 * h], uu[2 * h + 1]);
                const f2_t d = f2_add(f2_add(f2_sub(lp[h], cp[h]), f2_sub(rp[h], cp[h])),
                                      f2_add(f2_sub(sp, cp[h]), f2_sub(up, cp[h])));
                d0n[2 * h] = f2_lo(d);
                d0n[2 * h + 1] = f2_hi(d);
            }
#else
#pragma unroll
            for (int k = 0; k < kCpt; ++k) {
                const float left = k == 0 ? xl : c[k - 1];
                const float right = k == kCpt - 1 ? xrr : c[k + 1];
                d0n[k] = ((left - c[k]) + (right - c[k])) + ((s2v[k] - c[k]) + (uu[k] - c[k]));
            }
#endif
        }
    } else {
#pragma unroll
        for (int k = 0; k < kCpt; ++k) R[0][NXT][k] = 0.0f;
    }

    // ---- levels: level l advances row i-1-l ------------------------------
    // the neighbours' edges of the previous step: in the middle-pass kernel
    // one quad of levels per 128-bit load, else one level per scalar load
    const float4* xr4 = S::xbuf4(sm, (K & 1) ^ 1);
    const float* xr1 = S::xbuf1(sm, (K & 1) ^ 1);
    const int tl = (t + NT - 1) % NT, tr = (t + 1) % NT;
    float4 xlq, xrq;   // right edges of thread t-1, left edges of thread t+1
    const float dt = p.dt;
    float dout[kCpt], vout[kCpt];
#pragma unroll
    for (int l = 0; l < B; ++l) {
        const float* drow = (const float*)S::deep(sm, dslot(K - 1 - l));
        if (MID && l % 4 == 0) {
            xlq = xr4[(1 * S::NQ + l / 4) * NT + tl];
            xrq = xr4[(0 * S::NQ + l / 4) * NT + tr];
        }
        float vin[kCpt];
        if (l == 0) {
            const float4 v4 = *(const float4*)(S::shal(sm, S1) + W * 4 + 16 * t);
            vin[0] = v4.x; vin[1] = v4.y; vin[2] = v4.z; vin[3] = v4.w;
        } else {
#pragma unroll
            for (int k = 0; k < kCpt; ++k) vin[k] = VV[l][PRV][k];
        }
        float dn[kCpt], vn[kCpt];
        if (MID || l < L) {
            float kk[4];
            if constexpr (XH == 0 && SWEEP != 1) {
#pragma unroll
                for (int k = 0; k < kCpt; ++k) kk[k] = KR[(K + 2 * kU - 1 - l) % kU][k];
            } else {
                const float4 k4 = *(const float4*)(drow + kCpt * t);
                kk[0] = k4.x; kk[1] = k4.y; kk[2] = k4.z; kk[3] = k4.w;
            }
            float dd[4];
            if (l == 0) {
#pragma unroll
                for (int k = 0; k < kCpt; ++k) dd[k] = d0n[k];
            } else if constexpr (MID && XH == 0 && CL == 1) {
#pragma unroll
                for (int k = 0; k < kCpt; ++k) dd[k] = DR[(K + 2 * kU - 1 - l) % kU][k];
            } else {
                const float4 d4 = *(const float4*)(drow + W + kCpt * t);
                dd[0] = d4.x; dd[1] = d4.y; dd[2] = d4.z; dd[3] = d4.w;
            }
            float xl, xrt;
            if constexpr (MID) {
                xl = l % 4 == 0 ? xlq.x : l % 4 == 1 ? xlq.y : l % 4 == 2 ? xlq.z : xlq.w;
                xrt = l % 4 == 0 ? xrq.x : l % 4 == 1 ? xrq.y : l % 4 == 2 ? xrq.z : xrq.w;
            } else {
                xl = xr1[l * 2 * NT + NT + tl];
                xrt = xr1[l * 2 * NT + tr];
            }

            bool dr = true;
            if (MID && HALF0 && l == 0) {   // the first pass: level 0 is g = 0
#pragma unroll
                for (int k = 0; k < kCpt; ++k) kk[k] *= 0.5f;
            }
            if (!MID) {
                const int g = p.g0 + l;
                if (g == 0 || g == p.m) {
#pragma unroll
                    for (int k = 0; k < kCpt; ++k) kk[k] *= 0.5f;
                }
                dr = g < p.m;
            }
#if PR_TB2D_PACKED
            {
                // columns (0,1) and (2,3) as f32x2 pairs; the horizontal
                // neighbour sums cross the pairs and stay scalar
                const float* C = R[l][CUR];
                const float h0 = xl + C[1], h1 = C[0] + C[2], h2 = C[1] + C[3], h3 = C[2] + xrt;
                const f2_t m4 = f2_pack(-4.0f, -4.0f), dt2 = f2_pack(dt, dt);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = 2 * h;
                    const f2_t cc = f2_pack(C[k], C[k + 1]);
                    const f2_t hs = f2_add(h == 0 ? f2_pack(h0, h1) : f2_pack(h2, h3),
                                           f2_pack(R[l][PRV][k], R[l][PRV][k + 1]));
                    const f2_t part = f2_add(f2_pack(dd[k], dd[k + 1]), f2_fma(m4, cc, hs));
                    const f2_t v2 = f2_fma(f2_pack(kk[k], kk[k + 1]),
                                           f2_add(part, f2_pack(R[l][NXT][k], R[l][NXT][k + 1])),
                                           f2_pack(vin[k], vin[k + 1]));
                    const f2_t d2 = dr ? f2_fma(dt2, v2, cc) : cc;
                    vn[k] = f2_lo(v2);
                    vn[k + 1] = f2_hi(v2);
                    dn[k] = f2_lo(d2);
                    dn[k + 1] = f2_hi(d2);
                }
            }
#else
#pragma unroll
            for (int k = 0; k < kCpt; ++k) {
                const float left = k == 0 ? xl : R[l][CUR][k - 1];
                const float right = k == kCpt - 1 ? xrt : R[l][CUR][k + 1];
                // D(u) = D0 + (du_S + du_N + du_W + du_E - 4 du_C); the fresh
                // north row enters last to keep the level-to-level chain short
                const float part = dd[k] + fmaf(-4.0f, R[l][CUR][k], (left + right) + R[l][PRV][k]);
                vn[k] = fmaf(kk[k], part + R[l][NXT][k], vin[k]);
                dn[k] = dr ? fmaf(dt, vn[k], R[l][CUR][k]) : R[l][CUR][k];
            }
#endif
        } else {
#pragma unroll
            for (int k = 0; k < kCpt; ++k) {
                vn[k] = vin[k];
                dn[k] = R[l][CUR][k];
            }
        }
        if (l + 1 < B) {
#pragma unroll
            for (int k = 0; k < kCpt; ++k) {
                R[l + 1][NXT][k] = dn[k];
                VV[l + 1][CUR][k] = vn[k];
            }
        } else {
#pragma unroll
            for (int k = 0; k < kCpt; ++k) {
                dout[k] = dn[k];
                vout[k] = vn[k];
            }
        }
    }

    // ---- row i-B leaves the pipeline -------------------------------------
    if (do_out) {
        const float u0[4] = {u0o.x, u0o.y, u0o.z, u0o.w};
        float uo[4];
        if (MID || p.r_out) {
            float rr[4];
#if PR_TB2D_PACKED
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                f2_t r2;
                const f2_t s2 = f2_two_sum(f2_pack(u0[2 * h], u0[2 * h + 1]),
                                           f2_pack(dout[2 * h], dout[2 * h + 1]), &r2);
                uo[2 * h] = f2_lo(s2);
                uo[2 * h + 1] = f2_hi(s2);
                rr[2 * h] = f2_lo(r2);
                rr[2 * h + 1] = f2_hi(r2);
            }
#else
#pragma unroll
            for (int k = 0; k < kCpt; ++k) uo[k] = pr_two_sum(u0[k], dout[k], &rr[k]);
#endif
            *(uint2*)(p.r_out + off_out) = make_uint2(pr_bf16x2(rr[0], rr[1]), pr_bf16x2(rr[2], rr[3]));
        } else {
#pragma unroll
            for (int k = 0; k < kCpt; ++k) uo[k] = u0[k] + dout[k];
        }
        *(float4*)(p.u_out + off_out) = make_float4(uo[0], uo[1], uo[2], uo[3]);
        *(float4*)(p.v_out + off_out) = make_float4(vout[0], vout[1], vout[2], vout[3]);
    }

    // ---- shared stores, read only in later steps ----------------------------
    if constexpr (MID) {
        float4* xw = S::xbuf4(sm, K & 1);
#pragma unroll
        for (int q = 0; q < S::NQ; ++q) {   // level l's input rows: edges read by level l next step
            float e0[4], e1[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int l = 4 * q + j < B ? 4 * q + j : B - 1;
                e0[j] = R[l][NXT][0];
                e1[j] = R[l][NXT][kCpt - 1];
            }
            float4* d0 = xw + (0 * S::NQ + q) * NT + t;
            float4* d1 = xw + (1 * S::NQ + q) * NT + t;
            const float4 v0 = make_float4(e0[0], e0[1], e0[2], e0[3]), v1 = make_float4(e1[0], e1[1], e1[2], e1[3]);
            if (CL > 1 && t == 0) {
                // cluster rows: the wrap-around entry goes to the partner
                const uint32_t prank = cluster_rank() ^ 1u;
                st_async_f4(mapa_rank(smem_u32(d0), prank), v0, tx_bar<NT, B>(sm, pr.step, q, prank));
            } else {
                *d0 = v0;
            }
            if (CL > 1 && t == NT - 1) {
                const uint32_t prank = cluster_rank() ^ 1u;
                st_async_f4(mapa_rank(smem_u32(d1), prank), v1, tx_bar<NT, B>(sm, pr.step, q, prank));
            } else {
                *d1 = v1;
            }
        }
    } else {
        float* xw = S::xbuf1(sm, K & 1);
#pragma unroll
        for (int l = 0; l < B; ++l) {
            // cluster rows: the wrap-around entries go to the partner, every
            // level (16 bytes per part and step)
            if (CL > 1 && t == 0) {
                const uint32_t prank = cluster_rank() ^ 1u;
                st_async_f32(mapa_rank(smem_u32(xw + l * 2 * NT + t), prank), R[l][NXT][0],
                             tx_bar<NT, B>(sm, pr.step, l / 4, prank));
            } else if (l < L) {   // level l's input rows: edges read by level l next step
                xw[l * 2 * NT + t] = R[l][NXT][0];
            }
            if (CL > 1 && t == NT - 1) {
                const uint32_t prank = cluster_rank() ^ 1u;
                st_async_f32(mapa_rank(smem_u32(xw + l * 2 * NT + NT + t), prank), R[l][NXT][kCpt - 1],
                             tx_bar<NT, B>(sm, pr.step, l / 4, prank));
            } else if (l < L) {
                xw[l * 2 * NT + NT + t] = R[l][NXT][kCpt - 1];
            }
        }
    }
    if constexpr (CL > 1) ++pr.step;
    if (have_row && i >= 1) {
        // D0 of row i-1 for levels 1..B-1 at the next steps: a register ring
        // of kU rows in the middle-pass kernel (whole rows), else the deep ring
        if constexpr (MID && XH == 0 && CL == 1) {
#pragma unroll
            for (int k = 0; k < kCpt; ++k) DR[(K + kU - 1) % kU][k] = d0n[k];
        } else {
            float* dd = (float*)S::deep(sm, dslot(K - 1)) + W;
            *(float4*)(dd + kCpt * t) = make_float4(d0n[0], d0n[1], d0n[2], d0n[3]);
        }
    }
    // one barrier per row; it also makes the abort decision uniform
    if constexpr (GB == 0) return __syncthreads_or(timed_out) != 0;
    else return group_or<GB>(timed_out, 1 + grp);
}

// XH = 0: a CTA holds whole periodic rows (n = 4 NT).  XH > 0: it holds
// x-strips of 4 NT columns, of which the middle 4 NT - 2 XH are final (the
// stencil's reach grows one column per level, so XH >= B), and the rows of a
// slice are covered by ceil(n / (4 NT - 2 XH)) strips.
// The ring mbarriers (and, for cluster rows, the exchange mbarriers), armed
// once per launch by thread 0.
template <int NT, int B, int CL>
__device__ __forceinline__ void tb2d_init_bars(unsigned char* sm) {
    using S = Smem<NT, B>;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kU; ++s) mbar_init(S::bar(sm, s), 1);
        if (CL > 1) {
            // exchange barriers, armed for the partner's steps 0 and 1
            for (uint32_t b = 0; b < 2; ++b)
                for (uint32_t e = 0; e < 2; ++e)
                    for (int q = 0; q < S::NQ; ++q) {
                        mbar_init(S::ebar(sm, b, e, q), 1);
                        mbar_expect_tx(S::ebar(sm, b, e, q), S::part_tx);
                    }
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
}

// One pass of B levels (or p.levels in the general variant) over the rows
// [r_begin, r_end) of the pass's row space (rows_total = slices x strips x
// n), continuing the ring at position `pos` (a multiple of kU; advanced past
// the pass).  GB = 0: run by the whole CTA, which is NT threads.  GB = NT:
// run by thread group `grp` of a larger CTA (threads grp NT .. grp NT + NT-1,
// whole warps), whose shared memory `sm` is the group's own and whose
// per-row barrier is the named barrier 1 + grp.  Returns true if a bounded
// wait gave up.
template <int NT, int B, int XH, bool MID, bool HALF0, int CL, int SWEEP, int GB>
__device__ __forceinline__ bool tb2d_rows(const Tb2dParams& p, unsigned char* sm, uint32_t& pos_io, int64_t r_begin,
                                          int64_t r_end, int grp = 0) {
    static_assert(CL == 1 || (CL == 2 && XH == 0), "rows are shared by at most two CTAs, without x-strips");
    static_assert(GB == 0 || (GB == NT && CL == 1), "a thread group holds whole rows or x-strips alone");
    using S = Smem<NT, B>;
    const int t = GB == 0 ? (int)threadIdx.x : (int)threadIdx.x - grp * GB;
    const int n = p.n;
    const int64_t pts = (int64_t)n * n;
    const int L = MID ? B : p.levels;
    Pair pr = {0u};
    uint32_t rank = 0;
    if constexpr (CL > 1) {
        // both CTAs run and their mbarriers are initialised before either
        // touches the other's shared memory
        cluster_sync_all();
        rank = cluster_rank();
    }
    Pols pol = {0, 0, 0};
    if (t == 0) pol = {policy(0), policy(1), policy(2)};

    // ring positions: a segment occupies [base, base + niter) and the next one
    // starts at the following multiple of kU; positions that receive no
    // copy get a plain arrival, so slot s completes its phase j at position
    // j kU + s
    uint32_t pos = pos_io, consumed = pos_io, issued_end = pos_io;
    int timed_out = 0;
    bool aborted = false;

    // rows_total counts n rows per (slice, strip) pair
    constexpr int kStripW = S::W - 2 * XH;
    const int strips = XH ? (n + kStripW - 1) / kStripW : 1;
    for (int64_t seg0 = r_begin; seg0 < r_end && !aborted;) {
        Seg sg;
        const int64_t vslice = seg0 / n;
        const int64_t slice = vslice / strips;
        sg.x0 = XH ? (int)(vslice - slice * strips) * kStripW - XH : (int)rank * S::W;
        const int ya = (int)(seg0 - vslice * n);
        const int64_t seg1 = min(r_end, (vslice + 1) * (int64_t)n);
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
        // cluster rows: an even step count, so that consecutive steps of
        // consecutive segments alternate the x-edge buffers (ring positions
        // restart at a multiple of kU), as the partner's pushes need
        const int niter = sg.H + L + B + (CL > 1 ? ((sg.H + L + B) & 1) : 0);

        if (t == 0) {
            for (int rho = 0; rho < kPre && rho < sg.nload; ++rho) {
                issue_row<NT, B, XH, CL>(p, sg, sm, rho, (pos + (uint32_t)rho) % kU, (uint32_t)rho, pol);
                issued_end = pos + (uint32_t)rho + 1;
            }
        }

        float R[B][3][kCpt], VV[B][3][kCpt], UH[3][kCpt], KR[kU][kCpt], DR[kU][kCpt];
#pragma unroll
        for (int l = 0; l < B; ++l)
#pragma unroll
            for (int s = 0; s < 3; ++s)
#pragma unroll
                for (int k = 0; k < kCpt; ++k) R[l][s][k] = VV[l][s][k] = 0.0f;
#pragma unroll
        for (int s = 0; s < 3; ++s)
#pragma unroll
            for (int k = 0; k < kCpt; ++k) UH[s][k] = 0.0f;
#pragma unroll
        for (int s = 0; s < kU; ++s)
#pragma unroll
            for (int k = 0; k < kCpt; ++k) KR[s][k] = DR[s][k] = 0.0f;

        uint32_t par = (pos / kU) & 1u;   // phase parity of the current ring lap
        int i = 0;
#define PR_TB2D_STEP(K)                                                                                   \
    if (i >= niter) break;                                                                                 \
    if (tb2d_step<NT, B, XH, MID, HALF0, CL, K, SWEEP, GB>(p, sg, sm, i, par, R, VV, UH, KR, DR, timed_out, consumed, \
                                               issued_end, pol, pr, grp)) {                                \
        aborted = true;                                                                                    \
        break;                                                                                             \
    }                                                                                                      \
    ++i;
        for (;;) {
            PR_TB2D_STEP(0) PR_TB2D_STEP(1) PR_TB2D_STEP(2) PR_TB2D_STEP(3) PR_TB2D_STEP(4) PR_TB2D_STEP(5)
            PR_TB2D_STEP(6) PR_TB2D_STEP(7) PR_TB2D_STEP(8) PR_TB2D_STEP(9) PR_TB2D_STEP(10) PR_TB2D_STEP(11)
            par ^= 1u;
        }
#undef PR_TB2D_STEP
        if (aborted) break;
        // close the lap: complete the phases of the positions that got no copy
        const uint32_t next = (pos + (uint32_t)niter + kU - 1) / kU * kU;
        if (t == 0)
            for (uint32_t q = pos + (uint32_t)sg.nload; q < next; ++q) mbar_arrive(S::bar(sm, q % kU));
        pos = next;
    }
    if (aborted && t == 0) {
        // let copies still in flight land before the CTA's shared memory is
        // released.  Under the time-out test hook every issued slot expects
        // tx_extra bytes that no copy brings: settle them first, so that each
        // wait ends exactly when the slot's real copies have landed
        for (uint32_t q = consumed; q < issued_end; ++q) {
            if (p.tx_extra) mbar_complete_tx(S::bar(sm, q % kU), p.tx_extra);
            (void)mbar_wait_bounded(S::bar(sm, q % kU), (q / kU) & 1u, p.wait_ns / 10);
        }
    }
    if constexpr (CL > 1) {
        // The partner's pushes of its last step (and, after an abort, of the
        // step after this CTA's last one) land before this CTA's shared
        // memory is released: the end threads wait for them, bounded.
        if ((t == 0 || t == NT - 1) && pr.step > 0) {
            const int extra = aborted ? 2 : 1;
            for (int e = 0; e < extra; ++e)
                for (int q = 0; q < S::NQ; ++q)
                    (void)rx_wait<NT, B>(sm, pr.step + (uint32_t)e, q, p.wait_ns / 10);
        }
        cluster_sync_all();
    }
    pos_io = pos;
    return aborted;
}

// One pass over this CTA's (cluster's) share of the rows of the whole pass:
// contiguous ranges of equal cost, rows + (L + B) steps per segment.
template <int NT, int B, int XH, bool MID, bool HALF0, int CL, int SWEEP>
__device__ __forceinline__ bool tb2d_pass(const Tb2dParams& p, unsigned char* sm, uint32_t& pos_io, bool skip) {
    const int L = MID ? B : p.levels;
    const int64_t unit = blockIdx.x / CL, units = gridDim.x / CL;
    const int64_t r_begin = skip ? 0 : balanced_row(p.rows_total, p.n, L + B, unit, units);
    const int64_t r_end = skip ? 0 : balanced_row(p.rows_total, p.n, L + B, unit + 1, units);
    return tb2d_rows<NT, B, XH, MID, HALF0, CL, SWEEP, 0>(p, sm, pos_io, r_begin, r_end);
}

template <int NT, int B, int XH, bool MID, bool HALF0, int CL>
__global__ void __launch_bounds__(NT, 1) fine_tb2d_kernel(const Tb2dParams p) {
    extern __shared__ __align__(128) unsigned char sm[];
    // an earlier pass of this context gave up waiting: its results are not
    // valid, skip the work until pr_check reports and clears the flag (a
    // cluster CTA still meets its partner at the two cluster barriers)
    const bool skip = *(volatile int*)p.flag != 0;
    if (CL == 1 && skip) return;
    tb2d_init_bars<NT, B, CL>(sm);
    uint32_t pos = 0;
    (void)tb2d_pass<NT, B, XH, MID, HALF0, CL, false>(p, sm, pos, skip);
}

// Launch of one pass.  CL = 2: clusters of two CTAs, each holding one half
// of every row (n = 8 NT); the grid is as many clusters as fit at once.
template <int NT, int B, int XH, bool MID, bool HALF0, int CL = 1>
pr_status launch_cfg(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st) {
    using S = Smem<NT, B>;
    auto kern = fine_tb2d_kernel<NT, B, XH, MID, HALF0, CL>;
    static int configured_dev = -1;
    static int units = 0;   // CTAs (CL = 1) or clusters resident at once
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = S::total;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (configured_dev != ctx->device) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::total);
        if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb2d: set shared memory size");
        if (CL == 1) {
            int blocks_per_sm = 0, sms = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, NT, S::total);
            if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb2d: occupancy");
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
            units = blocks_per_sm * sms;
        } else {
            e = cudaOccupancyMaxActiveClusters(&units, kern, &cfg);
            if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb2d: cluster occupancy");
        }
        if (units < 1) return pr_fail(ctx, PR_ECUDA, "tb2d: kernel does not fit on an SM");
        configured_dev = ctx->device;
    }
    Tb2dParams p;
    p.u_in = (const float*)ps.u_in;
    p.v_in = (const float*)ps.v_in;
    p.r_in = (const uint16_t*)ps.r_in;
    p.kap = (const float*)ctx->kappa;
    p.u_out = (float*)ps.u_out;
    p.v_out = (float*)ps.v_out;
    p.r_out = (uint16_t*)ps.r_out;
    p.flag = ctx->dev_flag;
    const int strips = XH ? ((int)ctx->n + Smem<NT, B>::W - 2 * XH - 1) / (Smem<NT, B>::W - 2 * XH) : 1;
    p.rows_total = (int64_t)ps.nslices * strips * ctx->n;
    p.n = (int)ctx->n;
    p.g0 = ps.g0;
    p.levels = ps.levels;
    p.m = ps.m;
    p.dt = (float)ctx->dt_f;
    p.tx_extra = ctx->debug_stall ? 16u : 0u;
    p.wait_ns = ctx->debug_stall ? 200000000ull : 2000000000ull;
    int64_t grid = units;
    if (grid > p.rows_total) grid = p.rows_total;
    cudaError_t e;
    if (CL == 1) {
        kern<<<(int)grid, NT, S::total, st>>>(p);
        e = cudaGetLastError();
    } else {
        cfg.gridDim = dim3((unsigned)(grid * CL), 1, 1);
        e = cudaLaunchKernelEx(&cfg, kern, p);
    }
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb2d: launch");
    return PR_OK;
}

// Passes in which all B levels kick and drift and a residual goes out run the
// specialised kernel: the middle passes, and the first pass, which differs
// only by the half kick at level 0 and no residual in.  The general variant
// takes the rest (the last pass; passes of fewer levels).
template <int NT, int B, int XH, int CL = 1>
pr_status launch_depth(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st) {
    const bool full = ps.levels == B && ps.g0 + B - 1 < ps.m && ps.r_out;
    if (full && ps.g0 >= 1 && ps.r_in) return launch_cfg<NT, B, XH, true, false, CL>(ctx, ps, st);
    if (full && ps.g0 == 0 && !ps.r_in) return launch_cfg<NT, B, XH, true, true, CL>(ctx, ps, st);
    return launch_cfg<NT, B, XH, false, false, CL>(ctx, ps, st);
}

}  // namespace
