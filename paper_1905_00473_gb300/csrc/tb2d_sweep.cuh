#pragma once
// A whole sweep of fused 2D FP32 passes in one persistent launch (the pass
// bodies are those of tb2d_kernels.cuh); instantiated by width in
// fine_tb2d_sweep.cu (n = 512, 1024) and fine_tb2d_sweep_s.cu (n = 128, 256).
#include "tb2d_kernels.cuh"

namespace {
using namespace tb;

// ---- a whole sweep in one launch --------------------------------------------
// Grid-wide barrier between passes (a cooperative launch keeps every CTA
// resident).  Each CTA's stores of the pass are released at GPU scope before
// its arrival and made visible to the async proxy (the TMA copies of the next
// pass); the wait is bounded and records PR_ETIMEOUT on expiry.
__device__ __forceinline__ bool grid_barrier(unsigned int* ctr, unsigned int target, int* flag, uint64_t limit_ns) {
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        const uint64_t t0 = global_ns();
        while (true) {
            unsigned int v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
            if (v >= target) break;
            if (global_ns() - t0 > limit_ns) {
                atomicExch(flag, 1);
                ok = 0;
                break;
            }
        }
        __threadfence();
        asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    return __syncthreads_and(ok) != 0;
}

// The last pass of the whole-sweep kernel (the general variant, once per
// sweep) as a separate function: inlined beside the middle-pass body it
// would push the kernel past the register file and make the hot loop spill.
template <int NT, int B>
__device__ __noinline__ bool sweep_last_pass(const Tb2dParams& p, unsigned char* sm, uint32_t& pos, bool skip) {
    return tb2d_pass<NT, B, 0, false, false, 1, true>(p, sm, pos, skip);
}

struct SweepParams {
    // pass parameters, all in the kernel's parameter space: the first pass,
    // the middle passes by parity of their index (the pass scratch
    // ping-pongs; a middle pass uses no level index) and the last pass
    Tb2dParams first, mid[2], last;
    unsigned int* ctr;        // grid-barrier counter, zero at launch
    int passes;
};

// All passes of a sweep (whole rows, depth 8, four columns per thread): the
// first pass (half kick at level 0), the middle passes and the last pass (the
// final half kick; 9 levels where the sweep has 8 k + 1) run back to back in
// one persistent launch, a grid barrier between passes.  The ring positions
// continue across passes, so the mbarriers are armed once.
template <int NT>
__global__ void __launch_bounds__(NT, 1) fine_tb2d_sweep_kernel(const SweepParams sp) {
    extern __shared__ __align__(128) unsigned char sm[];
    tb2d_init_bars<NT, 8, 1>(sm);
    uint32_t pos = 0;
    bool failed = false;
    for (int q = 0; q < sp.passes; ++q) {
        const bool first = q == 0, last = q == sp.passes - 1;
        const bool skip = failed || *(volatile int*)sp.first.flag != 0;
        bool ab;
        if (!last && first) ab = tb2d_pass<NT, 8, 0, true, true, 1, true>(sp.first, sm, pos, skip);
        else if (!last && (q & 1)) ab = tb2d_pass<NT, 8, 0, true, false, 1, true>(sp.mid[1], sm, pos, skip);
        else if (!last) ab = tb2d_pass<NT, 8, 0, true, false, 1, true>(sp.mid[0], sm, pos, skip);
        else if (sp.last.levels == 9) ab = sweep_last_pass<NT, 9>(sp.last, sm, pos, skip);
        else ab = sweep_last_pass<NT, 8>(sp.last, sm, pos, skip);
        failed = failed || ab;
        if (!last && !grid_barrier(sp.ctr, (unsigned int)(q + 1) * gridDim.x, sp.first.flag, sp.first.wait_ns))
            failed = true;
    }
}


template <int NT>
pr_status launch_sweep_n(pr_ctx* ctx, const pr_sweep& sw, cudaStream_t st) {
    using S = Smem<NT, 9>;   // the layout of depth 8 and 9 passes, sized for 9
    auto kern = fine_tb2d_sweep_kernel<NT>;
    static int configured_dev = -1;
    static int units = 0;
    if (configured_dev != ctx->device) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::total);
        if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb2d sweep: set shared memory size");
        int blocks_per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, NT, S::total);
        if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb2d sweep: occupancy");
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
        units = blocks_per_sm * sms;
        if (units < 1) return pr_fail(ctx, PR_ECUDA, "tb2d sweep: kernel does not fit on an SM");
        configured_dev = ctx->device;
    }
    SweepParams sp;
    Tb2dParams b = Tb2dParams{};
    b.kap = (const float*)ctx->kappa;
    b.flag = ctx->dev_flag;
    b.rows_total = (int64_t)sw.nslices * ctx->n;
    b.n = (int)ctx->n;
    b.m = ctx->m_f;
    b.dt = (float)ctx->dt_f;
    b.tx_extra = ctx->debug_stall ? 16u : 0u;
    b.wait_ns = ctx->debug_stall ? 200000000ull : 2000000000ull;
    // pass q reads scratch (q - 1) & 1 and writes scratch q & 1
    auto pass = [&](const void* ui, const void* vi, const void* ri, void* uo, void* vo, void* ro, int g0, int levels) {
        Tb2dParams p = b;
        p.u_in = (const float*)ui;
        p.v_in = (const float*)vi;
        p.r_in = (const uint16_t*)ri;
        p.u_out = (float*)uo;
        p.v_out = (float*)vo;
        p.r_out = (uint16_t*)ro;
        p.g0 = g0;
        p.levels = levels;
        return p;
    };
    sp.first = pass(sw.u_in, sw.v_in, nullptr, sw.su[0], sw.sv[0], sw.sr[0], 0, 8);
    for (int par = 0; par < 2; ++par)   // middle pass q with q & 1 == par
        sp.mid[par] = pass(sw.su[par ^ 1], sw.sv[par ^ 1], sw.sr[par ^ 1], sw.su[par], sw.sv[par], sw.sr[par], 0, 8);
    const int ql = sw.passes - 1;
    sp.last = pass(sw.su[(ql - 1) & 1], sw.sv[(ql - 1) & 1], sw.sr[(ql - 1) & 1], sw.u_out, sw.v_out, nullptr, ql * 8,
                   sw.last_levels);
    sp.ctr = ctx->sweep_ctr;
    sp.passes = sw.passes;
    int64_t grid = units;
    if (grid > b.rows_total) grid = b.rows_total;
    cudaError_t e = cudaMemsetAsync(ctx->sweep_ctr, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb2d sweep: clear counter");
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = S::total;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, sp);
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "tb2d sweep: launch");
    return PR_OK;
}

}  // namespace

