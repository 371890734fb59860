// Batches of independent problem instances of uneven sizes (one parareal
// iteration's fine sweep per instance, Alg. 3 parFor, for many instances),
// replayed as one CUDA graph in one of two forms:
//   mode 0  per-instance block depth and fused-kernel geometry chosen by
//           timing, every instance's chain of pass launches a branch of the
//           graph, the branches spread over several streams;
//   mode 1  one persistent kernel that claims every (instance, pass, slice,
//           x-strip) item from a device queue (batch_queue.cu).
// pr_batch_set_mode switches between them, or times both and keeps the faster.
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "pr_internal.cuh"

struct pr_batch {
    std::vector<pr_ctx*> ctx;
    std::vector<const void*> ui, vi;
    std::vector<void*> uo, vo;
    std::vector<int> depth;
    std::vector<int> cols;
    std::vector<double> ms;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> ev;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int mode = 0;                 // 0 per-instance launch chains, 1 the work-queue kernel
    pr_queue* queue = nullptr;    // built on the first switch to mode 1
    std::string err;
};

namespace {

constexpr int kStreams = 8;

void destroy(pr_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    pr_queue_destroy(b->queue);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    delete b;
}

// time one sweep of instance i at depth d with cols columns per thread
// (after one warm-up sweep)
pr_status time_config(pr_batch* b, int i, int d, int cols, cudaStream_t st, double* ms) {
    pr_ctx* c = b->ctx[i];
    c->block_depth = d;
    c->tb_cols = cols;
    pr_status s = pr_fine_all_slices(c, b->ui[i], b->vi[i], b->uo[i], b->vo[i], 0, c->N, st);
    if (s != PR_OK) return s;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    s = pr_fine_all_slices(c, b->ui[i], b->vi[i], b->uo[i], b->vo[i], 0, c->N, st);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != PR_OK) return s;
    if (e != cudaSuccess) return pr_cuda_fail(nullptr, e, "pr_batch: timing");
    *ms = t;
    return PR_OK;
}

// (Re)capture the batch's graph in its current mode.
pr_status capture(pr_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    const int count = (int)b->ctx.size();
    cudaStream_t cap = b->streams[kStreams];
    cudaEvent_t fork = b->ev[kStreams];
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return pr_cuda_fail(nullptr, e, "pr_batch: begin capture");
    pr_status ps = PR_OK;
    if (b->mode == 1) {
        ps = pr_queue_launch(b->queue, cap);
    } else {
        // fork on kStreams streams, one branch per instance, join; biggest
        // instances first, spread over the streams
        cudaEventRecord(fork, cap);
        std::vector<int> order(count);
        for (int i = 0; i < count; ++i) order[i] = i;
        std::sort(order.begin(), order.end(), [&](int a, int c) {
            return (double)b->ctx[a]->pts * b->ctx[a]->N * b->ctx[a]->m_f >
                   (double)b->ctx[c]->pts * b->ctx[c]->N * b->ctx[c]->m_f;
        });
        for (int k = 0; k < kStreams; ++k) cudaStreamWaitEvent(b->streams[k], fork, 0);
        for (int j = 0; j < count && ps == PR_OK; ++j) {
            const int i = order[j];
            ps = pr_fine_all_slices(b->ctx[i], b->ui[i], b->vi[i], b->uo[i], b->vo[i], 0, b->ctx[i]->N,
                                    b->streams[j % kStreams]);
        }
        for (int k = 0; k < kStreams; ++k) {
            cudaEventRecord(b->ev[k], b->streams[k]);
            cudaStreamWaitEvent(cap, b->ev[k], 0);
        }
    }
    e = cudaStreamEndCapture(cap, &b->graph);
    if (ps != PR_OK) return ps;
    if (e != cudaSuccess) return pr_cuda_fail(nullptr, e, "pr_batch: end capture");
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) return pr_cuda_fail(nullptr, e, "pr_batch: instantiate");
    return PR_OK;
}

// time `reps` replays of the batch's graph on st, after one warm-up replay
pr_status time_graph(pr_batch* b, cudaStream_t st, int reps, double* ms) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t e = cudaGraphLaunch(b->exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(b->exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return pr_cuda_fail(nullptr, e, "pr_batch: timing");
    *ms = t / reps;
    return PR_OK;
}

}  // namespace

extern "C" pr_status pr_batch_create(int count, pr_ctx* const* ctxs, const void* const* u_in,
                                     const void* const* v_in, void* const* u_out, void* const* v_out,
                                     int autotune, void* stream, pr_batch** out) {
    if (!out) return pr_fail(nullptr, PR_EINVAL, "pr_batch_create: out is NULL");
    *out = nullptr;
    if (count < 1 || !ctxs || !u_in || !v_in || !u_out || !v_out)
        return pr_fail(nullptr, PR_EINVAL, "pr_batch_create: need count >= 1 and non-NULL arrays");
    pr_batch* b = new pr_batch();
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < count; ++i) {
        if (!ctxs[i] || !u_in[i] || !v_in[i] || !u_out[i] || !v_out[i]) {
            destroy(b);
            return pr_fail(nullptr, PR_EINVAL, "pr_batch_create: NULL instance entry");
        }
        b->ctx.push_back(ctxs[i]);
        b->ui.push_back(u_in[i]);
        b->vi.push_back(v_in[i]);
        b->uo.push_back(u_out[i]);
        b->vo.push_back(v_out[i]);
        b->depth.push_back(ctxs[i]->block_depth);
        b->cols.push_back(ctxs[i]->tb_cols);
        b->ms.push_back(0.0);
    }
    // instances run concurrently on different streams and the autotuner
    // writes every output while timing: a context used twice would race on its
    // scratch, and an output overlapping another instance's arrays would
    // clobber that instance's data
    {
        struct Span { uintptr_t lo, hi; int inst; bool out; };
        std::vector<Span> spans;
        for (int i = 0; i < count; ++i) {
            for (int j = 0; j < i; ++j)
                if (b->ctx[j] == b->ctx[i]) {
                    destroy(b);
                    return pr_fail(nullptr, PR_EINVAL, "pr_batch_create: a context appears twice");
                }
            const uintptr_t len = (uintptr_t)b->ctx[i]->N * (uintptr_t)b->ctx[i]->pts *
                                  (b->ctx[i]->dtype == PR_F32 ? 4u : 8u);
            spans.push_back({(uintptr_t)b->ui[i], (uintptr_t)b->ui[i] + len, i, false});
            spans.push_back({(uintptr_t)b->vi[i], (uintptr_t)b->vi[i] + len, i, false});
            spans.push_back({(uintptr_t)b->uo[i], (uintptr_t)b->uo[i] + len, i, true});
            spans.push_back({(uintptr_t)b->vo[i], (uintptr_t)b->vo[i] + len, i, true});
        }
        for (size_t a = 0; a < spans.size(); ++a)
            for (size_t c = 0; c < a; ++c) {
                const Span& x = spans[a];
                const Span& y = spans[c];
                if (x.inst == y.inst || !(x.out || y.out)) continue;
                if (x.lo < y.hi && y.lo < x.hi) {
                    destroy(b);
                    return pr_fail(nullptr, PR_EINVAL,
                                   "pr_batch_create: an output array overlaps another instance's array");
                }
            }
    }
    // the instances' sweeps run concurrently on several streams: each takes one
    // launch per pass (a whole-sweep cooperative launch holds every SM and
    // waits at grid barriers, which concurrent launches must not share)
    for (int i = 0; i < count; ++i) b->ctx[i]->one_launch = 0;
    // autotuner: the fastest instantiated (depth, columns) per instance, timed once
    if (autotune) {
        const int cands[5][2] = {{8, 4}, {8, 2}, {4, 4}, {4, 2}, {1, 0}};
        for (int i = 0; i < count; ++i) {
            double best = 1e300;
            int best_d = 1, best_c = 0;
            for (const auto& cd : cands) {
                const int d = cd[0], cols = cd[1];
                if (d > 1 && !pr_tb2d_supported(b->ctx[i], d)) continue;
                // 2048-point rows run four columns per thread whatever is set:
                // the two-column candidates would time the same kernels again
                if (cols == 2 && b->ctx[i]->n == 2048) continue;
                double t = 0;
                pr_status s = time_config(b, i, d, cols, st, &t);
                if (s != PR_OK) {
                    destroy(b);
                    return s;
                }
                if (t < best) {
                    best = t;
                    best_d = d;
                    best_c = cols;
                }
            }
            b->ctx[i]->block_depth = best_d;
            b->ctx[i]->tb_cols = best_c;
            b->depth[i] = best_d;
            b->cols[i] = best_c;
            b->ms[i] = best;
        }
    }
    // streams of the graph's branches, the fork event and the capture stream
    for (int k = 0; k < kStreams; ++k) {
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            destroy(b);
            return pr_fail(nullptr, PR_ECUDA, "pr_batch_create: stream/event creation");
        }
        b->streams.push_back(s);
        b->ev.push_back(e);
    }
    cudaEvent_t fork;
    cudaStream_t cap;
    if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) {
        destroy(b);
        return pr_fail(nullptr, PR_ECUDA, "pr_batch_create: stream/event creation");
    }
    b->ev.push_back(fork);
    b->streams.push_back(cap);
    const pr_status ps = capture(b);
    if (ps != PR_OK) {
        destroy(b);
        return ps;
    }
    *out = b;
    return PR_OK;
}

extern "C" pr_status pr_batch_launch(pr_batch* b, void* stream) {
    if (!b || !b->exec) return pr_fail(nullptr, PR_EINVAL, "pr_batch_launch: no batch");
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return pr_cuda_fail(nullptr, e, "pr_batch_launch");
    return PR_OK;
}

extern "C" pr_status pr_batch_info(const pr_batch* b, int i, int* block_depth, int* columns,
                                   double* tuned_ms) {
    if (!b || i < 0 || i >= (int)b->ctx.size()) return pr_fail(nullptr, PR_EINVAL, "pr_batch_info: bad index");
    // the work-queue kernel runs every instance at depth 8, four columns a thread
    if (block_depth) *block_depth = b->mode == 1 ? 8 : b->depth[i];
    if (columns) *columns = b->mode == 1 ? 4 : b->cols[i];
    if (tuned_ms) *tuned_ms = b->ms[i];
    return PR_OK;
}

extern "C" pr_status pr_batch_set_mode(pr_batch* b, int mode, void* stream, int* chosen) {
    if (!b || !b->exec) return pr_fail(nullptr, PR_EINVAL, "pr_batch_set_mode: no batch");
    if (mode < -1 || mode > 1) return pr_fail(nullptr, PR_EINVAL, "pr_batch_set_mode: mode must be -1, 0 or 1");
    cudaStream_t st = (cudaStream_t)stream;
    // replays of the graph that is about to be replaced may still be in flight
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return pr_cuda_fail(nullptr, e, "pr_batch_set_mode: synchronize");
    if (mode != 0) {
        // the queue tables, rebuilt from the contexts' current settings
        const int count = (int)b->ctx.size();
        pr_queue* q = nullptr;
        pr_status s = pr_queue_create(count, b->ctx.data(), b->ui.data(), b->vi.data(), b->uo.data(), b->vo.data(),
                                      &q);
        if (s != PR_OK) return s;
        if (b->mode == 1) {
            // the current graph launches the old tables: replace it first
            b->mode = 0;
            s = capture(b);
            if (s != PR_OK) {
                pr_queue_destroy(q);
                return s;
            }
        }
        pr_queue_destroy(b->queue);
        b->queue = q;
    }
    int pick = mode;
    if (mode == -1) {
        // time both forms (two replays each, after a warm-up) and keep the faster
        double t[2] = {0.0, 0.0};
        for (int m = 0; m < 2; ++m) {
            b->mode = m;
            pr_status s = capture(b);
            if (s == PR_OK) s = time_graph(b, st, 2, &t[m]);
            if (s != PR_OK) return s;
        }
        pick = t[1] < t[0] ? 1 : 0;
    }
    b->mode = pick;
    pr_status s = capture(b);
    if (s != PR_OK) return s;
    if (chosen) *chosen = pick;
    return PR_OK;
}

extern "C" void pr_batch_destroy(pr_batch* b) { destroy(b); }
