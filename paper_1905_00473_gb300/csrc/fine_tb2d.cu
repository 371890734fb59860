// 2D FP32 fine propagator with temporal blocking: B velocity-Verlet levels
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
// double-buffered shared array written by the level below one iteration
// earlier.  One barrier per row.
//
// Loads.  One elected thread streams rows with cp.async.bulk (TMA bulk
// copies: rows are contiguous and 16-byte aligned) into shared-memory rings
// guarded by one mbarrier per row slot: kappa into a 16-row ring that also
// holds D0 (below) for the rows in flight, u_hi, u_t and the bfloat16
// residual into a 5-row ring.  The finished row re-reads its u_hi from L2.  Waits are
// bounded: after ~2 s the CTA records PR_ETIMEOUT in a device flag and all
// its threads leave the loop together.
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
// Variants.  MID = a pass strictly inside the sweep (no half kick, every
// level drifts, all B levels active), which is nearly every pass; the
// general variant handles the first pass (half kick at g = 0), the last pass
// (half kick at g = m, no drift, fewer than B levels: the missing levels pass
// rows through unchanged).
#include "pr_internal.cuh"
#include "tb_common.cuh"

namespace {
using namespace tb;

#ifndef PR_TB2D_PREFETCH
#define PR_TB2D_PREFETCH 2
#endif
#ifndef PR_TB2D_RD
#define PR_TB2D_RD 16   // kappa/D0 ring rows; 0 = the minimum B + prefetch + 1
#endif
constexpr int kCpt = 4;                     // columns per thread
constexpr int kPrefetch = PR_TB2D_PREFETCH; // rows in flight ahead of the consumer
constexpr int kRS = kPrefetch + 3;          // u_hi, u_t, residual ring
// kappa/D0 ring for pipeline depth B: at least B + kPrefetch + 1 rows
constexpr int rd_for(int B) {
    return PR_TB2D_RD > B + kPrefetch + 1 ? PR_TB2D_RD : B + kPrefetch + 1;
}

template <int NT, int B>
struct Smem {
    // wider CTAs (x-strips of 1040 columns) keep the minimum ring to fit
    static constexpr int RD = NT > 256 ? B + kPrefetch + 1 : rd_for(B);
    static constexpr int W = NT * kCpt;                       // columns held = n, or a strip
    static constexpr size_t deep_row = (size_t)2 * W * 4;      // kappa, D0
    static constexpr size_t sh_row = (size_t)W * 4 * 2 + W * 2;  // u_hi, u_t, residual
    static constexpr size_t deep_bytes = RD * deep_row;
    static constexpr size_t sh_bytes = kRS * sh_row;
    static constexpr size_t xbuf_bytes = (size_t)3 * B * 2 * NT * 4;  // [3][B][2][NT]
    static constexpr size_t bar_bytes = (size_t)RD * 8;
    static constexpr size_t total = deep_bytes + sh_bytes + xbuf_bytes + bar_bytes;
};

template <int NT, int B>
struct Shared {
    unsigned char* deep;   // [RD][kappa W | D0 W]
    unsigned char* shal;   // [kRS][u W | v W | r 2W]
    float* xbuf;           // [3][B][2][NT]: edge columns of each level's output row
    uint64_t* bars;        // [RD]
};

template <int NT, int B>
using Pos = RingPos<B, Smem<NT, B>::RD, (uint32_t)Smem<NT, B>::deep_row, kRS, (uint32_t)Smem<NT, B>::sh_row,
                    kPrefetch>;

// Request local row rho of the segment (kappa, u_hi, u_t, residual) into the
// deep slot doff and the shallow slot soff; called by one thread.
template <int NT, int B, int XH>
__device__ __forceinline__ void issue_row(const Tb2dParams& p, const Seg& sg, const Shared<NT, B>& sh, int rho,
                                          uint32_t doff, uint32_t soff, uint64_t pol_first, uint64_t pol_last,
                                          uint64_t pol_norm) {
    using S = Smem<NT, B>;
    constexpr int W = S::W;
    const int n = p.n;
    const int64_t off = (int64_t)seg_row(sg.ylo, rho, n) * n;
    uint64_t* bar = &sh.bars[doff / S::deep_row];
    unsigned char* drow = sh.deep + doff;
    unsigned char* srow = sh.shal + soff;
    const uint32_t row_bytes = (uint32_t)W * 4;
    mbar_expect_tx(bar, 3 * row_bytes + (sg.r_s ? (uint32_t)W * 2 : 0u) + p.tx_extra);
    if (XH == 0) {
        bulk_g2s(drow, p.kap + off, row_bytes, bar, pol_last);
        bulk_g2s(srow, sg.u_s + off, row_bytes, bar, pol_norm);
        bulk_g2s(srow + W * 4, sg.v_s + off, row_bytes, bar, pol_first);
        if (sg.r_s) bulk_g2s(srow + W * 8, sg.r_s + off, (uint32_t)W * 2, bar, pol_first);
    } else {
        bulk_row_g2s(drow, p.kap + off, sg.x0, W, n, 4, bar, pol_last);
        bulk_row_g2s(srow, sg.u_s + off, sg.x0, W, n, 4, bar, pol_norm);
        bulk_row_g2s(srow + W * 4, sg.v_s + off, sg.x0, W, n, 4, bar, pol_first);
        if (sg.r_s) bulk_row_g2s(srow + W * 8, sg.r_s + off, sg.x0, W, n, 2, bar, pol_first);
    }
}

// One row iteration of the pipeline; PH = i mod 3 selects the register ring
// slots and the xbuf buffer at compile time.  Register rings per level l:
//   R[l][.]  du rows of level l's input: centre = slot PH, south = (PH+2)%3,
//            north = (PH+1)%3 (written this iteration by the level below)
//   VV[l][.] u_t of level l's input row: read (PH+2)%3, written PH
// Returns true when some thread's bounded wait gave up.
template <int NT, int B, int XH, bool MID, int PH>
__device__ __forceinline__ bool tb2d_iter(const Tb2dParams& p, const Seg& sg, const Shared<NT, B>& sh,
                                          int i, float (&R)[B][3][kCpt], float (&VV)[B][3][kCpt],
                                          Pos<NT, B>& ps, int& timed_out, uint32_t& consumed,
                                          uint64_t pol_first, uint64_t pol_last, uint64_t pol_norm) {
    using S = Smem<NT, B>;
    constexpr int W = S::W;
    constexpr int CUR = PH, PRV = (PH + 2) % 3, NXT = (PH + 1) % 3;
    const int t = threadIdx.x;
    const int n = p.n;
    const int L = MID ? B : sg.L;
    const uint32_t q = sg.base + (uint32_t)i;
    auto gy = [&](int rho) { return seg_row(sg.ylo, rho, n); };

    // ---- producer: row i + kPrefetch into the rings ---------------------
    if (t == 0 && i + kPrefetch < sg.nload)
        issue_row<NT, B, XH>(p, sg, sh, i + kPrefetch, ps.dn, ps.sn, pol_first, pol_last, pol_norm);

    // ---- the finished row's u_hi, fetched early from L2 ------------------
    const int rho_out = i - B;
    // in an x-strip only the columns at least XH from both strip edges are final
    const bool do_out = rho_out >= L && rho_out < L + sg.H &&
                        (XH == 0 || (t >= XH / kCpt && t < NT - XH / kCpt));
    int64_t off_out = 0;
    float4 u0o = make_float4(0.f, 0.f, 0.f, 0.f);
    if (do_out) {
        off_out = sg.slice_off + (int64_t)gy(rho_out) * n + sg.x0 + kCpt * t;
        u0o = __ldcs((const float4*)(p.u_in + off_out));
    }

    // ---- load stage: row i arrives; D0 of row i-1 -------------------------
    float d0n[kCpt] = {0.f, 0.f, 0.f, 0.f};
    const bool have_row = i < sg.nload;
    if (have_row) {
        if (!timed_out && !mbar_wait_bounded(&sh.bars[ps.bar_of(ps.dq)], ps.dpar, p.wait_ns)) {
            atomicExch(p.flag, 1);
            timed_out = 1;
        }
        consumed = q + 1;
        const unsigned char* s0 = sh.shal + ps.sq;
        const float4 u4 = *(const float4*)(s0 + 16 * t);
        const float uu[4] = {u4.x, u4.y, u4.z, u4.w};
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
            const float* s1 = (const float*)(sh.shal + ps.s1);
            const float* s2 = (const float*)(sh.shal + (i >= 2 ? ps.s2 : ps.s1));
            const float4 a = *(const float4*)(s1 + kCpt * t);
            const float4 b2 = *(const float4*)(s2 + kCpt * t);
            const float c[4] = {a.x, a.y, a.z, a.w};
            const float s2v[4] = {b2.x, b2.y, b2.z, b2.w};
            const float xl = s1[(kCpt * t + W - 1) % W], xrr = s1[(kCpt * t + kCpt) % W];
#pragma unroll
            for (int k = 0; k < kCpt; ++k) {
                const float left = k == 0 ? xl : c[k - 1];
                const float right = k == kCpt - 1 ? xrr : c[k + 1];
                d0n[k] = ((left - c[k]) + (right - c[k])) + ((s2v[k] - c[k]) + (uu[k] - c[k]));
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < kCpt; ++k) R[0][NXT][k] = 0.0f;
    }

    // ---- levels: level l advances row i-1-l ------------------------------
    const float* xr = sh.xbuf + (size_t)PRV * B * 2 * NT;
    const int tl = (t + NT - 1) % NT, tr = (t + 1) % NT;
    const float dt = p.dt;
    float dout[kCpt], vout[kCpt];
#pragma unroll
    for (int l = 0; l < B; ++l) {
        const float* drow = (const float*)(sh.deep + ps.lev[l]);
        float vin[kCpt];
        if (l == 0) {
            const float4 v4 = *(const float4*)(sh.shal + ps.s1 + W * 4 + 16 * t);
            vin[0] = v4.x; vin[1] = v4.y; vin[2] = v4.z; vin[3] = v4.w;
        } else {
#pragma unroll
            for (int k = 0; k < kCpt; ++k) vin[k] = VV[l][PRV][k];
        }
        float dn[kCpt], vn[kCpt];
        if (MID || l < L) {
            const float4 k4 = *(const float4*)(drow + kCpt * t);
            float kk[4] = {k4.x, k4.y, k4.z, k4.w};
            float dd[4];
            if (l == 0) {
#pragma unroll
                for (int k = 0; k < kCpt; ++k) dd[k] = d0n[k];
            } else {
                const float4 d4 = *(const float4*)(drow + W + kCpt * t);
                dd[0] = d4.x; dd[1] = d4.y; dd[2] = d4.z; dd[3] = d4.w;
            }
            const float xl = xr[l * 2 * NT + NT + tl];
            const float xrt = xr[l * 2 * NT + tr];
            bool dr = true;
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
#pragma unroll
            for (int k = 0; k < kCpt; ++k) uo[k] = pr_two_sum(u0[k], dout[k], &rr[k]);
            *(uint2*)(p.r_out + off_out) = make_uint2(pr_bf16x2(rr[0], rr[1]), pr_bf16x2(rr[2], rr[3]));
        } else {
#pragma unroll
            for (int k = 0; k < kCpt; ++k) uo[k] = u0[k] + dout[k];
        }
        *(float4*)(p.u_out + off_out) = make_float4(uo[0], uo[1], uo[2], uo[3]);
        *(float4*)(p.v_out + off_out) = make_float4(vout[0], vout[1], vout[2], vout[3]);
    }

    // ---- shared stores, read only in later iterations ----------------------
    float* xw = sh.xbuf + (size_t)CUR * B * 2 * NT;
#pragma unroll
    for (int l = 0; l < B; ++l) {
        if (MID || l < L) {   // level l's input rows: edges read by level l next iteration
            xw[l * 2 * NT + t] = R[l][NXT][0];
            xw[l * 2 * NT + NT + t] = R[l][NXT][kCpt - 1];
        }
    }
    if (have_row && i >= 1) {
        float* dd = (float*)(sh.deep + ps.lev[0]) + W;
        *(float4*)(dd + kCpt * t) = make_float4(d0n[0], d0n[1], d0n[2], d0n[3]);
    }
    ps.advance();
    // one barrier per row; it also makes the abort decision uniform
    return __syncthreads_or(timed_out) != 0;
}

// XH = 0: a CTA holds whole periodic rows (n = 4 NT).  XH > 0: it holds
// x-strips of 4 NT columns, of which the middle 4 NT - 2 XH are final (the
// stencil's reach grows one column per level, so XH >= B), and the rows of a
// slice are covered by n / (4 NT - 2 XH) strips.
template <int NT, int B, int XH, bool MID>
__global__ void __launch_bounds__(NT, 1) fine_tb2d_kernel(const Tb2dParams p) {
    using S = Smem<NT, B>;
    constexpr int kRD = S::RD;
    extern __shared__ __align__(128) unsigned char smem[];
    Shared<NT, B> sh;
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
    uint64_t pol_first = 0, pol_last = 0, pol_norm = 0;
    if (t == 0) {
        pol_first = policy(0);
        pol_last = policy(1);
        pol_norm = policy(2);
    }

    // per-CTA row ranges of equal cost: rows + (L + B) steps per segment
    const int64_t r_begin = balanced_row(p.rows_total, n, L + B, blockIdx.x, gridDim.x);
    const int64_t r_end = balanced_row(p.rows_total, n, L + B, blockIdx.x + 1, gridDim.x);
    uint32_t issued = 0, consumed = 0;
    int timed_out = 0;
    bool aborted = false;

    // rows_total counts n rows per (slice, strip) pair
    constexpr int kStripW = S::W - 2 * XH;
    const int strips = XH ? n / kStripW : 1;
    for (int64_t seg0 = r_begin; seg0 < r_end && !aborted;) {
        Seg sg;
        const int64_t vslice = seg0 / n;
        const int64_t slice = vslice / strips;
        sg.x0 = XH ? (int)(vslice - slice * strips) * kStripW - XH : 0;
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
        sg.base = issued;
        int ylo = (ya - L) % n;
        sg.ylo = ylo < 0 ? ylo + n : ylo;
        const int niter = sg.H + L + B;

        if (t == 0) {
            for (int rho = 0; rho < kPrefetch && rho < sg.nload; ++rho) {
                const uint32_t qq = sg.base + (uint32_t)rho;
                issue_row<NT, B, XH>(p, sg, sh, rho, (qq % kRD) * (uint32_t)S::deep_row,
                                     (qq % kRS) * (uint32_t)S::sh_row, pol_first, pol_last, pol_norm);
            }
        }
        issued += (uint32_t)sg.nload;
        Pos<NT, B> ps;
        ps.init(sg.base);

        float R[B][3][kCpt], VV[B][3][kCpt];
#pragma unroll
        for (int l = 0; l < B; ++l)
#pragma unroll
            for (int s = 0; s < 3; ++s)
#pragma unroll
                for (int k = 0; k < kCpt; ++k) R[l][s][k] = VV[l][s][k] = 0.0f;

        int i = 0;
        for (; i + 3 <= niter; i += 3) {
            if (tb2d_iter<NT, B, XH, MID, 0>(p, sg, sh, i, R, VV, ps, timed_out, consumed, pol_first, pol_last, pol_norm) ||
                tb2d_iter<NT, B, XH, MID, 1>(p, sg, sh, i + 1, R, VV, ps, timed_out, consumed, pol_first, pol_last, pol_norm) ||
                tb2d_iter<NT, B, XH, MID, 2>(p, sg, sh, i + 2, R, VV, ps, timed_out, consumed, pol_first, pol_last, pol_norm)) {
                aborted = true;
                break;
            }
        }
        if (!aborted && i < niter)
            aborted = tb2d_iter<NT, B, XH, MID, 0>(p, sg, sh, i, R, VV, ps, timed_out, consumed, pol_first, pol_last, pol_norm);
        if (!aborted && i + 1 < niter)
            aborted = tb2d_iter<NT, B, XH, MID, 1>(p, sg, sh, i + 1, R, VV, ps, timed_out, consumed, pol_first, pol_last, pol_norm);
    }
    if (aborted && t == 0) {
        // let copies still in flight land before the CTA's shared memory is released
        for (uint32_t q = consumed; q < issued; ++q)
            (void)mbar_wait_bounded(&sh.bars[q % kRD], (q / kRD) & 1u, p.wait_ns / 10);
    }
}

template <int NT, int B, int XH, bool MID>
pr_status launch_cfg(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st) {
    using S = Smem<NT, B>;
    auto kern = fine_tb2d_kernel<NT, B, XH, MID>;
    static int configured_dev = -1;
    static int blocks_per_sm = 0;
    static int sms = 0;
    if (configured_dev != ctx->device) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::total);
        if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb2d: set shared memory size");
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, NT, S::total);
        if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb2d: occupancy");
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        if (blocks_per_sm < 1) return pr_fail(ctx, PR_ECUDA, "tb2d: kernel does not fit on an SM");
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
    const int strips = XH ? (int)ctx->n / (Smem<NT, B>::W - 2 * XH) : 1;
    p.rows_total = (int64_t)ps.nslices * strips * ctx->n;
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
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb2d: launch");
    return PR_OK;
}

template <int NT, int B, int XH>
pr_status launch_depth(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st) {
    const bool mid = ps.levels == B && ps.g0 >= 1 && ps.g0 + B - 1 < ps.m && ps.r_in && ps.r_out;
    return mid ? launch_cfg<NT, B, XH, true>(ctx, ps, st) : launch_cfg<NT, B, XH, false>(ctx, ps, st);
}

template <int B>
pr_status launch_n(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st) {
    switch (ctx->n) {
        case 256: return launch_depth<64, B, 0>(ctx, ps, st);
        case 512: return launch_depth<128, B, 0>(ctx, ps, st);
        case 1024: return launch_depth<256, B, 0>(ctx, ps, st);
        // two x-strips of 1040 columns (1024 final + 8 each side) per row; 260
        // threads are 9 warps, 3 on one SM sub-partition, which caps a thread
        // at 168 registers: depth 4 fits, depth 8 would spill
        case 2048:
            if constexpr (B == 4) return launch_depth<260, B, 8>(ctx, ps, st);
            else return pr_fail(ctx, PR_EINVAL, "tb2d: n = 2048 runs at depth 4");
        default: return pr_fail(ctx, PR_EINVAL, "tb2d: unsupported grid size");
    }
}

}  // namespace

// depths with an instantiated kernel: 8 (default) and 4 (smaller register and
// shared-memory footprint; the batch autotuner chooses between them)
bool pr_tb2d_supported(const pr_ctx* ctx, int depth) {
    if (ctx->dim != 2 || ctx->dtype != PR_F32 || (depth != 8 && depth != 4)) return false;
    return ctx->n == 256 || ctx->n == 512 || ctx->n == 1024 || (ctx->n == 2048 && depth == 4);
}

pr_status pr_launch_fine_tb2d(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st) {
    if (ps.levels == 1) return pr_launch_fine_naive(ctx, ps, st);
    if ((ps.r_in || ps.r_out) && ps.rfmt != PR_RESID_BF16)
        return pr_fail(ctx, PR_EINVAL, "tb2d: the fused pass carries a bfloat16 residual");
    // Thread geometry (pr_set_fused_columns); by default two columns per thread
    // (fine_tb2d_c2.cu) for n <= 512, where four columns leave too few warps
    // per SM (n = 512: one CTA of 4 warps), and four (this file) for n = 1024,
    // where 8 warps fill the SM and the x-neighbour exchange and per-row
    // overhead are shared by twice the columns.
    // n = 2048 runs in x-strips with four columns per thread whatever is set.
    const int cols = ctx->tb_cols ? ctx->tb_cols : (ctx->n <= 512 ? 2 : 4);
    if (cols == 2 && ctx->n <= 1024) return pr_launch_fine_tb2d_c2(ctx, ps, st);
    const int B = ctx->block_depth;
    if (ps.levels < 1 || ps.levels > B) return pr_fail(ctx, PR_EINVAL, "tb2d: bad level count");
    if (B == 8) return launch_n<8>(ctx, ps, st);
    if (B == 4) return launch_n<4>(ctx, ps, st);
    return pr_fail(ctx, PR_EINVAL, "tb2d: unsupported depth");
}
