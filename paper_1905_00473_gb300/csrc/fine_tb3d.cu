// 3D FP32 fine propagator with temporal blocking: up to four velocity-Verlet
// levels per HBM pass, all slices in one persistent launch.
//
// What is computed is the level recurrence of fine_naive.cu (kick
// v += w_g kappa D(u), drift u += dt v; Sec. 3.1 scheme, Alg. 3 parFor over
// slices), with the FP32 displacement kept as (u_hi, bfloat16 rounding
// residual) between passes and stepped as du = u - u_hi inside a pass, the
// stencil applied as D(u) = D0 + D(du), D0 = D(u_hi) formed from differences.
//
// Geometry (2.5D blocking).  A work item is one xy tile of one slice, TX x TY
// = 64 x 16 points, streamed through the whole z column.  The CTA holds the
// tile extended by B = 4 points on every side in x and y (72 x 24 points):
// thread t owns the four consecutive x points of quad t % 18 on extended row
// t / 18.  Planes stream through a B-deep software pipeline: at step i plane
// i arrives, level l advances plane i-1-l, and plane i-B leaves finished.  A
// level reads its own points' z neighbours from register rings (the plane
// above was advanced this step by the level below), and the in-plane
// neighbours (x, y) of the plane it advances from a shared tile that the
// level below wrote one step earlier: one barrier per step.  Neighbours that
// fall outside the extended tile are replaced by the point itself; the
// error this makes moves inward one point per level, so after B levels it
// has not reached the interior tile, which is the only part written out
// (overlapped tiling: the halo is recomputed by the neighbouring tiles).
//
// Loads.  Every thread stages its own quads of plane i + 2 (u_hi, u_t,
// residual, kappa) into shared rings with cp.async (no other thread reads
// them, so its own wait_group orders them): three planes of u_hi, u_t and
// residual, twelve of kappa, which the levels read up to four steps later.
//
// Rings.  The plane loop is unrolled 12-fold; every ring period divides it:
// the du rings of the levels and the u_hi ring (3), the u_t and shared-tile
// parities (2), the D0 ring (4) and the staging rings (3, 12).  Plane
// indices advance by one per step, so their periodic wrap is a compare.
#include "pr_internal.cuh"

namespace {

constexpr int B3 = 4;                       // levels per pass
constexpr int TX = 64, TY = 16;             // interior tile
constexpr int EX = TX + 2 * B3, EY = TY + 2 * B3;   // extended tile (72 x 24)
constexpr int QX = EX / 4;                  // quads per extended row (18)
constexpr int NT3 = QX * EY;                // threads (432)
constexpr int kPF = 2;                      // planes staged ahead

struct Tb3dParams {
    const float* u_in;
    const float* v_in;
    const uint16_t* r_in;   // bfloat16 residual; null: zero (first pass)
    const float* kap;
    float* u_out;
    float* v_out;
    uint16_t* r_out;        // null: last pass, residual folded into u
    int n, nslices;
    int g0, levels, m;
    float dt;
};

struct __align__(16) Smem3 {
    float x[B3][2][EY][EX];      // input plane of level l, by step parity
    float uh[2][EY][EX];         // u_hi of the plane that arrived, by step parity
    float su[3][EY][EX];         // staged u_hi, u_t (by plane mod 3)
    float sv[3][EY][EX];
    uint16_t sr[3][EY][EX];      // staged residual
    float sk[12][EY][EX];        // staged kappa (by plane mod 12: read by the levels up to 4 steps later)
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

struct Item {
    int64_t base;    // slice offset + row offset of this thread's quad (without z)
    int64_t kbase;   // the same offset in kappa (no slice)
    int64_t n2;      // n * n
    int gx0, gy;     // global x of the quad's first point, global y of the row
    bool inner;      // the quad lies in the interior tile
};

// z - k wrapped into [0, n) for 0 <= z < n, -n < -k <= n
__device__ __forceinline__ int zwrap(int z, int k, int n) {
    int r = z + k;
    if (r >= n) r -= n;
    if (r < 0) r += n;
    return r;
}

// global plane z of local plane p of a column with L levels of halo
__device__ __forceinline__ int plane_z(int p, int L, int n) {
    int z = (p - L) % n;
    return z < 0 ? z + n : z;
}

// One step of the plane pipeline at ring position i (K = i mod 12).
// zi: global z of plane i (the arriving plane; planes wrap periodically)
template <int K>
__device__ __forceinline__ void tb3d_step(const Tb3dParams& p, Smem3& sm, const Item& it, int i, int zi, int nload,
                                          int L, float (&R)[B3][3][4], float (&VV)[B3][2][4], float (&UH)[3][4],
                                          float (&DR)[4][4]) {
    constexpr int CUR = K % 3, PRV = (K + 2) % 3, NXT = (K + 1) % 3;
    constexpr int PAR = K & 1, PPAR = PAR ^ 1;
    const int t = threadIdx.x, qx = t % QX, ey = t / QX, lx = 4 * qx;
    const int n = p.n;

    // ---- stage plane i + kPF (own quads only), then wait for plane i ------
    {
        const int q = i + kPF;
        if (q < nload) {
            constexpr int SS = (K + kPF) % 3, SK = (K + kPF) % 12;
            const int64_t zq = zwrap(zi, kPF, n);
            const int64_t off = it.base + zq * it.n2;
            cp_async16(&sm.su[SS][ey][lx], p.u_in + off);
            cp_async16(&sm.sv[SS][ey][lx], p.v_in + off);
            if (p.r_in) cp_async8(&sm.sr[SS][ey][lx], p.r_in + off);
            cp_async16(&sm.sk[SK][ey][lx], p.kap + it.kbase + zq * it.n2);
        }
        cp_commit();
        cp_wait<kPF>();
    }

    // ---- the finished plane's u_hi, fetched early from L2 ---------------
    const int p_out = i - B3;
    const bool do_out = it.inner && p_out >= L && p_out < L + n;
    int64_t off_out = 0;
    float4 u0o = make_float4(0.f, 0.f, 0.f, 0.f);
    if (do_out) {
        off_out = it.base + (int64_t)zwrap(zi, -B3, n) * it.n2;
        u0o = __ldcs((const float4*)(p.u_in + off_out));
    }

    // ---- load stage: plane i arrives; D0 of plane i-1 --------------------
    float d0n[4] = {0.f, 0.f, 0.f, 0.f};
    if (i < nload) {
        constexpr int SC = K % 3;
        const float4 u4 = *(const float4*)&sm.su[SC][ey][lx];
        const float4 v4 = *(const float4*)&sm.sv[SC][ey][lx];
        UH[CUR][0] = u4.x; UH[CUR][1] = u4.y; UH[CUR][2] = u4.z; UH[CUR][3] = u4.w;
        VV[0][PAR][0] = v4.x; VV[0][PAR][1] = v4.y; VV[0][PAR][2] = v4.z; VV[0][PAR][3] = v4.w;
        *(float4*)&sm.uh[PAR][ey][lx] = u4;
        if (p.r_in) {
            const uint2 r2 = *(const uint2*)&sm.sr[SC][ey][lx];
            R[0][NXT][0] = pr_bf16_lo(r2.x);
            R[0][NXT][1] = pr_bf16_hi(r2.x);
            R[0][NXT][2] = pr_bf16_lo(r2.y);
            R[0][NXT][3] = pr_bf16_hi(r2.y);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) R[0][NXT][k] = 0.0f;
        }
        if (i >= 1) {
            // D0 of plane i-1: centre UH[PRV], z neighbours UH[NXT] (i-2) and
            // UH[CUR] (i), in-plane neighbours from the tile written last step
            const float(*U)[EX] = sm.uh[PPAR];
            const float* c = UH[PRV];
            const float4 yl = *(const float4*)&U[ey > 0 ? ey - 1 : ey][lx];
            const float4 yr = *(const float4*)&U[ey < EY - 1 ? ey + 1 : ey][lx];
            const float xl = qx > 0 ? U[ey][lx - 1] : c[0];
            const float xr = qx < QX - 1 ? U[ey][lx + 4] : c[3];
            const float ylv[4] = {yl.x, yl.y, yl.z, yl.w}, yrv[4] = {yr.x, yr.y, yr.z, yr.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float left = k == 0 ? xl : c[k - 1];
                const float right = k == 3 ? xr : c[k + 1];
                const float ylk = ey > 0 ? ylv[k] : c[k];
                const float yrk = ey < EY - 1 ? yrv[k] : c[k];
                d0n[k] = ((left - c[k]) + (right - c[k])) + ((ylk - c[k]) + (yrk - c[k])) +
                         ((UH[NXT][k] - c[k]) + (UH[CUR][k] - c[k]));
            }
        }
        // the arriving plane's du is level 0's input tile next step
        *(float4*)&sm.x[0][PAR][ey][lx] = make_float4(R[0][NXT][0], R[0][NXT][1], R[0][NXT][2], R[0][NXT][3]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) R[0][NXT][k] = 0.0f;
    }
    constexpr int DW = (K + 3) % 4;   // D0 ring slot of plane i-1
#pragma unroll
    for (int k = 0; k < 4; ++k) DR[DW][k] = d0n[k];

    // ---- levels: level l advances plane i-1-l ----------------------------
    const float dt = p.dt;
    float dout[4], vout[4];
#pragma unroll
    for (int l = 0; l < B3; ++l) {
        const float* C = R[l][CUR];
        float vn[4], dn[4];
        if (l < L) {
            // kappa of plane r = i-1-l at the thread's points, staged with the plane
            const float4 kq = *(const float4*)&sm.sk[(K + 11 - l) % 12][ey][lx];
            float kk[4] = {kq.x, kq.y, kq.z, kq.w};
            const int g = p.g0 + l;
            const float wk = (g == 0 || g == p.m) ? 0.5f : 1.0f;
            const bool dr = g < p.m;
            const float(*X)[EX] = sm.x[l][PPAR];
            const float4 yl = *(const float4*)&X[ey > 0 ? ey - 1 : ey][lx];
            const float4 yr = *(const float4*)&X[ey < EY - 1 ? ey + 1 : ey][lx];
            const float xl = qx > 0 ? X[ey][lx - 1] : C[0];
            const float xr = qx < QX - 1 ? X[ey][lx + 4] : C[3];
            const float ylv[4] = {yl.x, yl.y, yl.z, yl.w}, yrv[4] = {yr.x, yr.y, yr.z, yr.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float left = k == 0 ? xl : C[k - 1];
                const float right = k == 3 ? xr : C[k + 1];
                const float ylk = ey > 0 ? ylv[k] : C[k];
                const float yrk = ey < EY - 1 ? yrv[k] : C[k];
                const float d0 = DR[(K + 11 - l) % 4][k];
                // D(u) = D0 + (neighbours of du - 6 du); the fresh plane above enters last
                const float part = d0 + fmaf(-6.0f, C[k], ((left + right) + (ylk + yrk)) + R[l][PRV][k]);
                vn[k] = fmaf(wk * kk[k], part + R[l][NXT][k], VV[l][PPAR][k]);
                dn[k] = dr ? fmaf(dt, vn[k], C[k]) : C[k];
            }
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                vn[k] = VV[l][PPAR][k];
                dn[k] = C[k];
            }
        }
        if (l + 1 < B3) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                R[l + 1][NXT][k] = dn[k];
                VV[l + 1][PAR][k] = vn[k];
            }
            *(float4*)&sm.x[l + 1][PAR][ey][lx] = make_float4(dn[0], dn[1], dn[2], dn[3]);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                dout[k] = dn[k];
                vout[k] = vn[k];
            }
        }
    }

    // ---- plane i-B leaves the pipeline ------------------------------------
    if (do_out) {
        const float u0[4] = {u0o.x, u0o.y, u0o.z, u0o.w};
        float uo[4];
        if (p.r_out) {
            float rr[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) uo[k] = pr_two_sum(u0[k], dout[k], &rr[k]);
            *(uint2*)(p.r_out + off_out) = make_uint2(pr_bf16x2(rr[0], rr[1]), pr_bf16x2(rr[2], rr[3]));
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) uo[k] = u0[k] + dout[k];
        }
        *(float4*)(p.u_out + off_out) = make_float4(uo[0], uo[1], uo[2], uo[3]);
        *(float4*)(p.v_out + off_out) = make_float4(vout[0], vout[1], vout[2], vout[3]);
    }
    // one barrier per step: the tiles of this step are read in the next
    __syncthreads();
}

__global__ void __launch_bounds__(NT3, 1) fine_tb3d_kernel(const Tb3dParams p) {
    extern __shared__ __align__(16) unsigned char smraw[];
    Smem3& sm = *(Smem3*)smraw;
    const int t = threadIdx.x, qx = t % QX, ey = t / QX;
    const int n = p.n;
    const int L = p.levels;
    const int tiles_x = n / TX, tiles_y = n / TY;
    const int64_t per_slice = (int64_t)tiles_x * tiles_y;
    const int64_t items = (int64_t)p.nslices * per_slice;
    const int nload = n + 2 * L;
    const int niter = L + n + B3;
    for (int64_t w = blockIdx.x; w < items; w += gridDim.x) {
        const int64_t slice = w / per_slice, rem = w - slice * per_slice;
        const int ty = (int)(rem / tiles_x), tx = (int)(rem - (int64_t)ty * tiles_x);
        Item it;
        it.n2 = (int64_t)n * n;
        it.gx0 = (tx * TX - B3 + 4 * qx + n) % n;
        it.gy = (ty * TY - B3 + ey + n) % n;
        it.inner = qx >= B3 / 4 && qx < B3 / 4 + TX / 4 && ey >= B3 && ey < B3 + TY;
        it.kbase = (int64_t)it.gy * n + it.gx0;
        it.base = slice * it.n2 * n + it.kbase;
        float R[B3][3][4], VV[B3][2][4], UH[3][4], DR[4][4];
#pragma unroll
        for (int l = 0; l < B3; ++l)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                R[l][0][k] = R[l][1][k] = R[l][2][k] = 0.0f;
                VV[l][0][k] = VV[l][1][k] = 0.0f;
            }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            UH[0][k] = UH[1][k] = UH[2][k] = 0.0f;
            DR[0][k] = DR[1][k] = DR[2][k] = DR[3][k] = 0.0f;
        }
        // stage planes 0 .. kPF-1
#pragma unroll
        for (int q = 0; q < kPF; ++q) {
            if (q < nload) {
                const int64_t zq = plane_z(q, L, n);
                const int64_t off = it.base + zq * it.n2;
                cp_async16(&sm.su[q % 3][ey][4 * qx], p.u_in + off);
                cp_async16(&sm.sv[q % 3][ey][4 * qx], p.v_in + off);
                if (p.r_in) cp_async8(&sm.sr[q % 3][ey][4 * qx], p.r_in + off);
                cp_async16(&sm.sk[q % 12][ey][4 * qx], p.kap + it.kbase + zq * it.n2);
            }
            cp_commit();
        }
        int i = 0, zi = plane_z(0, L, n);
#define PR_TB3D_STEP(K)                                                     \
    if (i >= niter) break;                                                   \
    tb3d_step<K>(p, sm, it, i, zi, nload, L, R, VV, UH, DR);                 \
    ++i;                                                                     \
    zi = zi + 1 == n ? 0 : zi + 1;
        for (;;) {
            PR_TB3D_STEP(0) PR_TB3D_STEP(1) PR_TB3D_STEP(2) PR_TB3D_STEP(3) PR_TB3D_STEP(4) PR_TB3D_STEP(5)
            PR_TB3D_STEP(6) PR_TB3D_STEP(7) PR_TB3D_STEP(8) PR_TB3D_STEP(9) PR_TB3D_STEP(10) PR_TB3D_STEP(11)
        }
#undef PR_TB3D_STEP
        cp_wait<0>();
        __syncthreads();
    }
}

}  // namespace

// 3D FP32 grids the fused kernel takes: n a multiple of the tile (64 x 16)
bool pr_tb3d_supported(const pr_ctx* ctx, int depth) {
    return ctx->dim == 3 && ctx->dtype == PR_F32 && depth == B3 && ctx->n % TX == 0 && ctx->n % TY == 0 &&
           ctx->n >= TX;
}

pr_status pr_launch_fine_tb3d(pr_ctx* ctx, const pr_pass& ps, cudaStream_t st) {
    if (ps.levels < 2 || ps.levels > B3) return pr_fail(ctx, PR_EINVAL, "tb3d: bad level count");
    if ((ps.r_in || ps.r_out) && ps.rfmt != PR_RESID_BF16)
        return pr_fail(ctx, PR_EINVAL, "tb3d: the fused pass carries a bfloat16 residual");
    static int configured_dev = -1;
    static int units = 0;
    if (configured_dev != ctx->device) {
        cudaError_t e = cudaFuncSetAttribute(fine_tb3d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(Smem3));
        if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb3d: set shared memory size");
        int bps = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fine_tb3d_kernel, NT3, sizeof(Smem3));
        if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb3d: occupancy");
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        units = bps * sms;
        if (units < 1) return pr_fail(ctx, PR_ECUDA, "tb3d: kernel does not fit on an SM");
        configured_dev = ctx->device;
    }
    Tb3dParams p;
    p.u_in = (const float*)ps.u_in;
    p.v_in = (const float*)ps.v_in;
    p.r_in = (const uint16_t*)ps.r_in;
    p.kap = (const float*)ctx->kappa;
    p.u_out = (float*)ps.u_out;
    p.v_out = (float*)ps.v_out;
    p.r_out = (uint16_t*)ps.r_out;
    p.n = (int)ctx->n;
    p.nslices = ps.nslices;
    p.g0 = ps.g0;
    p.levels = ps.levels;
    p.m = ps.m;
    p.dt = (float)ctx->dt_f;
    const int64_t items = (int64_t)ps.nslices * (ctx->n / TX) * (ctx->n / TY);
    const int64_t grid = items < units ? items : units;
    fine_tb3d_kernel<<<(unsigned)grid, NT3, sizeof(Smem3), st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb3d: launch");
    return PR_OK;
}
