// One persistent kernel for a batch of independent 2D FP32 instances of uneven
// sizes (Alg. 3's parFor over slices, for many problems at once): every fused
// pass of every slice of every instance is a work item in a device queue, and
// a grid of one CTA per SM claims them in queue order until the queue is
// empty.
//
// Items.  An item is one pass (B = 8 levels, or fewer in the last passes) over
// one slice of one instance, or over one x-strip of a slice at n = 2048: the
// pass bodies are those of the per-pass kernels (tb2d_kernels.cuh), run by a
// thread group that holds the item's rows alone:
//   n = 256   64 threads, whole rows         n = 512   128 threads
//   n = 1024  256 threads                    n = 2048  192 threads, x-strips of
//                                                      768 columns (752 final)
// A CTA claims a unit: consecutive items of one pass, as many as its groups
// run side by side (four at n = 256, two at 512, one otherwise), each group
// on its own shared memory with its own named row barrier.  Warps without an
// item wait at the unit's closing barrier.
//
// Order.  Pass k of a slice reads what pass k-1 wrote for the whole slice
// (the y-halo, and at n = 2048 the x-halo of the neighbouring strips), so
// each (instance, slice) has a completion counter and a unit waits (bounded)
// until the counters show every item of its slices' previous pass.  Units
// are claimed in queue order, and the queue is a topological order (the
// passes of an instance in sequence), so a unit only ever waits for items
// that CTAs already hold: no co-residency of the grid is needed.  The widest
// class comes first; within a class, instances are interleaved by progress,
// the key of pass k of an instance of P passes being (k + 1/2) / P, so that
// the long pass chains (few slices, many steps each) run alongside the wide
// instances instead of after them (queue_plan.h).
//
// Visibility.  A finished unit's stores are fenced for the async proxy and
// released at GPU scope before its counters are incremented; the waiting CTA
// acquires the counters and fences the async proxy before its bulk copies of
// the rows, and reads the finished row's u_hi past L1 (the whole-sweep form
// of the pass body: L1 is not coherent within one launch).
//
// Shared memory is the largest of the classes' layouts (times their groups);
// the ring mbarriers of a class live at that class's offsets, so a CTA
// invalidates and re-arms them when consecutive units change class.
#include <algorithm>
#include <vector>

#include "queue_plan.h"
#include "tb2d_kernels.cuh"

namespace {

constexpr int kQT = qplan::kThreads;   // threads of a queue CTA
constexpr int kQB = qplan::kDepth;     // block depth of the queued passes
static_assert(qplan::kCols == kCpt, "the plan's strip widths are those of the pass body");

// A class's thread groups: NT threads each, G side by side, each with its own
// `stride` bytes of shared memory (the pass body's layout, 128-byte aligned).
template <int C>
struct QCls {
    static constexpr int NT = qplan::kClasses[C].nt, XH = qplan::kClasses[C].xh, n = qplan::kClasses[C].n;
    static constexpr int G = qplan::kClasses[C].groups;
    static constexpr uint32_t stride = (Smem<NT, kQB>::total + 127u) / 128u * 128u;
    static_assert(NT % 32 == 0 && G * NT <= kQT, "a class's thread groups are whole warps of the CTA");
};
constexpr uint32_t qmax(uint32_t a, uint32_t b) { return a > b ? a : b; }
constexpr uint32_t kQSmem = qmax(qmax(QCls<0>::G * QCls<0>::stride, QCls<1>::G * QCls<1>::stride),
                                 qmax(QCls<2>::G * QCls<2>::stride, QCls<3>::G * QCls<3>::stride));
static_assert(kQSmem <= 227u * 1024u, "a queue CTA's shared memory fits an SM");

struct QPass {
    Tb2dParams p;
    int cls;       // geometry class (QCls)
    int variant;   // 1: middle pass (all levels kick and drift, residual in and out), 2: any other
};

struct QItem {
    int pass;        // index into the pass table
    int vslice;      // (slice, strip) of the pass's row space: rows vslice n .. vslice n + n - 1
    int dep;         // completion counter of the item's (instance, slice)
    unsigned need;   // completions of that counter before the item may start
};

struct QUnit {
    int first, count;   // items first .. first + count - 1, one pass, one per thread group
};

struct QParams {
    const QItem* items;
    const QUnit* units;
    const QPass* passes;
    unsigned* head;   // next unclaimed unit (zero at launch)
    unsigned* done;   // per (instance, slice): items finished (zero at launch)
    int* stop;        // set when a wait gave up: nothing more is claimed (zero at launch)
    int* const* flags;   // every instance's error flag
    int nunits, ninst;
    uint64_t wait_ns;
};

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <int C>
__device__ __forceinline__ void q_bars(unsigned char* sm, bool arm) {
    using S = Smem<QCls<C>::NT, kQB>;
    for (int g = 0; g < QCls<C>::G; ++g)
        for (int s = 0; s < kU; ++s) {
            if (arm) mbar_init(S::bar(sm + g * QCls<C>::stride, s), 1);
            else mbar_inval(S::bar(sm + g * QCls<C>::stride, s));
        }
}
__device__ __forceinline__ void q_bars_of(unsigned char* sm, int c, bool arm) {
    switch (c) {
        case 0: q_bars<0>(sm, arm); break;
        case 1: q_bars<1>(sm, arm); break;
        case 2: q_bars<2>(sm, arm); break;
        case 3: q_bars<3>(sm, arm); break;
        default: break;
    }
}

// Retire the ring mbarriers of class `from` (none: -1) and arm those of
// class `to`.  Every copy on the old ones has landed and been consumed: the
// previous unit's items closed their ring laps before the unit's closing
// barrier.
__device__ __forceinline__ void q_switch(unsigned char* sm, int from, int to) {
    if (threadIdx.x == 0) {
        q_bars_of(sm, from, false);
        q_bars_of(sm, to, true);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
}

// Bounded wait of one thread until *ctr >= need (GPU-scope acquire).
__device__ __forceinline__ bool q_wait(const unsigned* ctr, unsigned need, uint64_t limit_ns) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
    if (v >= need) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        __nanosleep(128);
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
        if (v >= need) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// The middle-pass body (all levels kick and drift, a residual in and out) for
// the two widest classes, which carry nearly all of a mixed batch's work; the
// general body for every other pass (it takes the half kicks at g = 0 and
// g = m, and passes of fewer levels), which keeps the kernel to six bodies.
// The whole-sweep form of the body (SWEEP = 1: the finished row's u_hi read
// past L1, kappa read per level: with the pass parameters in registers the
// kappa register ring would spill).  Run by thread group `grp` on its own
// shared memory.
template <int C>
__device__ __forceinline__ bool q_run(const Tb2dParams& p, int variant, unsigned char* sm, uint32_t& pos, int vslice,
                                      int grp) {
    constexpr int NT = QCls<C>::NT, XH = QCls<C>::XH;
    const int64_t r0 = (int64_t)vslice * QCls<C>::n, r1 = r0 + QCls<C>::n;
    unsigned char* gsm = sm + grp * QCls<C>::stride;
    if constexpr (C >= 2) {
        if (variant == 1) return tb2d_rows<NT, kQB, XH, true, false, 1, 1, NT>(p, gsm, pos, r0, r1, grp);
    }
    return tb2d_rows<NT, kQB, XH, false, false, 1, 1, NT>(p, gsm, pos, r0, r1, grp);
}

template <int C>
__device__ __forceinline__ bool q_group(const QParams& qp, const QUnit& un, const Tb2dParams& p, int variant,
                                        unsigned char* sm, uint32_t& pos) {
    if constexpr (QCls<C>::G == 1) {
        if ((int)threadIdx.x >= QCls<C>::NT) return false;   // idle for the unit
        return q_run<C>(p, variant, sm, pos, qp.items[un.first].vslice, 0);
    } else {
        const int g = (int)threadIdx.x / QCls<C>::NT;   // this thread's group; g >= count: idle for the unit
        if (g >= un.count) return false;
        return q_run<C>(p, variant, sm, pos, qp.items[un.first + g].vslice, g);
    }
}

__global__ void __launch_bounds__(kQT, 1) batch_queue_kernel(const QParams qp) {
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ int s_unit;
    int cls = -1;
    // ring position of this thread's group: the same in every thread of a
    // group, which runs the same items
    uint32_t pos = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            int u = -1;
            if (*(volatile int*)qp.stop == 0) {
                const unsigned h = atomicAdd(qp.head, 1u);
                if (h < (unsigned)qp.nunits) u = (int)h;
            }
            s_unit = u;
        }
        __syncthreads();
        const int u = s_unit;
        if (u < 0) break;
        const QUnit un = qp.units[u];
        const QPass* qd = qp.passes + qp.items[un.first].pass;
        const int c = qd->cls;
        if (c != cls) {
            q_switch(sm, cls, c);
            cls = c;
            pos = 0;
        }
        int ok = 1;
        if (threadIdx.x == 0) {
            for (int j = 0; j < un.count && ok; ++j) {
                const QItem it = qp.items[un.first + j];
                ok = q_wait(qp.done + it.dep, it.need, qp.wait_ns);
            }
            if (!ok) {
                atomicExch(qd->p.flag, 1);
                atomicExch(qp.stop, 1);
            }
            __threadfence();
            asm volatile("fence.proxy.async.global;" ::: "memory");
        }
        if (!__syncthreads_and(ok)) break;
        // the pass parameters in registers (they spill ~100 bytes; read from
        // shared memory where used instead, the 2048 strips ran 9 % slower)
        const Tb2dParams p = qd->p;
        // an instance whose earlier work gave up (flag not yet read by
        // pr_check) skips its items, which still count as done
        const bool skip = *(volatile int*)p.flag != 0;
        bool ab = false;
        if (!skip) {
            switch (c) {
                case 0: ab = q_group<0>(qp, un, p, qd->variant, sm, pos); break;
                case 1: ab = q_group<1>(qp, un, p, qd->variant, sm, pos); break;
                case 2: ab = q_group<2>(qp, un, p, qd->variant, sm, pos); break;
                default: ab = q_group<3>(qp, un, p, qd->variant, sm, pos); break;
            }
        }
        asm volatile("fence.proxy.async.global;" ::: "memory");
        if (__syncthreads_or(ab)) {
            if (threadIdx.x == 0) atomicExch(qp.stop, 1);
            break;
        }
        if (threadIdx.x == 0) {
            __threadfence();
            for (int j = 0; j < un.count; ++j) atomicAdd(qp.done + qp.items[un.first + j].dep, 1u);
        }
    }
    // a queue that stopped early left items of any instance undone: every
    // instance reports the time-out
    if (threadIdx.x == 0 && *(volatile int*)qp.stop != 0)
        for (int i = 0; i < qp.ninst; ++i) atomicExch(qp.flags[i], 1);
}

}  // namespace

struct pr_queue {
    // the first instance's caller allocator (copied: the tables may outlive
    // that context), which holds the tables
    pr_ctx owner;
    int device = 0;
    QItem* items = nullptr;
    QUnit* units = nullptr;
    QPass* passes = nullptr;
    unsigned* ctr = nullptr;   // head, then one counter per (instance, slice)
    int* stop = nullptr;
    int** flags = nullptr;
    int ninst = 0;
    size_t ctr_bytes = 0;
    int nunits = 0;
    int grid = 0;
    uint64_t wait_ns = 0;
};

bool pr_queue_supported(const pr_ctx* c) {
    return c && c->dim == 2 && c->dtype == PR_F32 && qplan::class_of(c->n) >= 0 && c->resid_bytes >= 2 &&
           c->m_f >= qplan::kDepth;
}

void pr_queue_destroy(pr_queue* q) {
    if (!q) return;
    pr_dev_free(&q->owner, q->items);
    pr_dev_free(&q->owner, q->units);
    pr_dev_free(&q->owner, q->passes);
    pr_dev_free(&q->owner, q->ctr);
    pr_dev_free(&q->owner, q->stop);
    pr_dev_free(&q->owner, q->flags);
    delete q;
}

pr_status pr_queue_create(int count, pr_ctx* const* ctx, const void* const* ui, const void* const* vi,
                          void* const* uo, void* const* vo, pr_queue** out) {
    *out = nullptr;
    std::vector<qplan::Inst> inst;
    uint64_t wait_ns = 2000000000ull;
    for (int i = 0; i < count; ++i) {
        if (!pr_queue_supported(ctx[i]))
            return pr_fail(nullptr, PR_EINVAL,
                           "pr_batch (queue): every instance must be 2D FP32 with n in {256, 512, 1024, 2048}, "
                           "m_f >= 8 and a bfloat16 residual");
        inst.push_back({ctx[i]->n, ctx[i]->N, ctx[i]->m_f});
        if (ctx[i]->debug_stall) wait_ns = 200000000ull;
    }
    std::vector<qplan::Pass> plan;
    std::vector<qplan::Item> qitems;
    std::vector<qplan::Unit> qunits;
    const int ndep = qplan::build(inst, &plan, &qitems, &qunits);
    if (ndep < 0) return pr_fail(nullptr, PR_EINVAL, "pr_batch (queue): no plan");
    std::vector<QPass> passes;
    for (const qplan::Pass& pl : plan) {
        const pr_ctx* c = ctx[pl.inst];
        const int i = pl.inst, k = pl.k;
        QPass qp_;
        Tb2dParams& p = qp_.p;
        p = Tb2dParams{};
        // pass k reads scratch (k - 1) & 1 and writes scratch k & 1
        p.u_in = pl.first ? (const float*)ui[i] : (const float*)c->su[(k - 1) & 1];
        p.v_in = pl.first ? (const float*)vi[i] : (const float*)c->sv[(k - 1) & 1];
        p.r_in = pl.first ? nullptr : (const uint16_t*)c->sr[(k - 1) & 1];
        p.kap = (const float*)c->kappa;
        p.u_out = pl.last ? (float*)uo[i] : (float*)c->su[k & 1];
        p.v_out = pl.last ? (float*)vo[i] : (float*)c->sv[k & 1];
        p.r_out = pl.last ? nullptr : (uint16_t*)c->sr[k & 1];
        p.flag = c->dev_flag;
        p.rows_total = (int64_t)c->N * pl.strips * c->n;
        p.n = (int)c->n;
        p.g0 = pl.g0;
        p.levels = pl.levels;
        p.m = c->m_f;
        p.dt = (float)c->dt_f;
        p.tx_extra = c->debug_stall ? 16u : 0u;
        p.wait_ns = c->debug_stall ? 200000000ull : 2000000000ull;
        const bool full = p.levels == kQB && p.g0 + kQB - 1 < p.m && p.r_out;
        qp_.cls = pl.cls;
        qp_.variant = (full && p.r_in) ? 1 : 2;
        passes.push_back(qp_);
    }
    std::vector<QItem> items;
    items.reserve(qitems.size());
    for (const qplan::Item& it : qitems) items.push_back({it.pass, it.vslice, it.dep, it.need});
    std::vector<QUnit> units;
    units.reserve(qunits.size());
    for (const qplan::Unit& un : qunits) units.push_back({un.first, un.count});

    pr_queue* q = new pr_queue();
    q->owner.ualloc = ctx[0]->ualloc;
    q->owner.urelease = ctx[0]->urelease;
    q->owner.uarg = ctx[0]->uarg;
    cudaGetDevice(&q->device);
    q->nunits = (int)units.size();
    q->wait_ns = wait_ns;
    q->ctr_bytes = (1 + (size_t)ndep) * sizeof(unsigned);
    cudaError_t e = pr_dev_malloc(&q->owner, (void**)&q->items, items.size() * sizeof(QItem));
    if (e == cudaSuccess) e = pr_dev_malloc(&q->owner, (void**)&q->units, units.size() * sizeof(QUnit));
    if (e == cudaSuccess) e = pr_dev_malloc(&q->owner, (void**)&q->passes, passes.size() * sizeof(QPass));
    if (e == cudaSuccess) e = pr_dev_malloc(&q->owner, (void**)&q->ctr, q->ctr_bytes);
    if (e == cudaSuccess) e = pr_dev_malloc(&q->owner, (void**)&q->stop, sizeof(int));
    if (e == cudaSuccess) e = pr_dev_malloc(&q->owner, (void**)&q->flags, count * sizeof(int*));
    std::vector<int*> flags(count);
    for (int i = 0; i < count; ++i) flags[i] = ctx[i]->dev_flag;
    q->ninst = count;
    if (e == cudaSuccess) e = cudaMemcpy(q->flags, flags.data(), count * sizeof(int*), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(q->items, items.data(), items.size() * sizeof(QItem), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(q->units, units.data(), units.size() * sizeof(QUnit), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(q->passes, passes.data(), passes.size() * sizeof(QPass), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_queue_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kQSmem);
    int per_sm = 0, sms = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_queue_kernel, kQT, kQSmem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, q->device);
    if (e != cudaSuccess) {
        pr_queue_destroy(q);
        return pr_cuda_fail(nullptr, e, "pr_batch (queue): setup");
    }
    if (per_sm < 1 || sms < 1) {
        pr_queue_destroy(q);
        return pr_fail(nullptr, PR_ECUDA, "pr_batch (queue): the kernel does not fit on an SM");
    }
    q->grid = per_sm * sms;
    *out = q;
    return PR_OK;
}

// The counters, then the kernel (both capturable into a graph).
pr_status pr_queue_launch(pr_queue* q, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(q->ctr, 0, q->ctr_bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(q->stop, 0, sizeof(int), st);
    if (e != cudaSuccess) return pr_cuda_fail(nullptr, e, "pr_batch (queue): clear counters");
    QParams qp;
    qp.items = q->items;
    qp.units = q->units;
    qp.passes = q->passes;
    qp.head = q->ctr;
    qp.done = q->ctr + 1;
    qp.stop = q->stop;
    qp.flags = q->flags;
    qp.nunits = q->nunits;
    qp.ninst = q->ninst;
    qp.wait_ns = q->wait_ns;
    batch_queue_kernel<<<q->grid, kQT, kQSmem, st>>>(qp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return pr_cuda_fail(nullptr, e, "pr_batch (queue): launch");
    return PR_OK;
}
