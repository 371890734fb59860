// C ABI entry points: context set-up (Sec. 3.1 grids, steps and medium) and
// the pass schedule of the fine propagator over all slices (Alg. 3, parFor).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pr_internal.cuh"

static thread_local std::string g_create_err;

pr_status pr_fail(pr_ctx* ctx, pr_status st, const std::string& msg) {
    if (ctx) ctx->err = msg;
    else g_create_err = msg;
    return st;
}

pr_status pr_cuda_fail(pr_ctx* ctx, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return pr_fail(ctx, e == cudaErrorMemoryAllocation ? PR_ENOMEM : PR_ECUDA, m);
}

extern "C" const char* pr_last_error(const pr_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

static pr_alloc_fn g_alloc = nullptr;
static pr_release_fn g_release = nullptr;
static void* g_alloc_user = nullptr;

void pr_current_allocator(pr_alloc_fn* a, pr_release_fn* r, void** user) {
    *a = g_alloc;
    *r = g_release;
    *user = g_alloc_user;
}

cudaError_t pr_dev_malloc(const pr_ctx* ctx, void** p, size_t bytes) {
    if (ctx && ctx->ualloc) {
        int dev = 0;
        cudaGetDevice(&dev);
        *p = ctx->ualloc(bytes, dev, ctx->uarg);
        return *p ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

void pr_dev_free(const pr_ctx* ctx, void* p) {
    if (!p) return;
    if (ctx && ctx->urelease) {
        cudaDeviceSynchronize();
        ctx->urelease(p, ctx->uarg);
        return;
    }
    cudaFree(p);
}

extern "C" pr_status pr_set_allocator(pr_alloc_fn alloc, pr_release_fn release, void* user) {
    if ((alloc == nullptr) != (release == nullptr))
        return pr_fail(nullptr, PR_EINVAL, "pr_set_allocator: give both functions or neither");
    g_alloc = alloc;
    g_release = release;
    g_alloc_user = alloc ? user : nullptr;
    return PR_OK;
}

static void free_all(pr_ctx* c) {
    pr_driver_free(c);
    if (c->coarse) {
        free_all(c->coarse);
        delete c->coarse;
        c->coarse = nullptr;
    }
    pr_dev_free(c, c->c64);
    pr_dev_free(c, c->adj_ws);
    c->adj_ws = nullptr;
    pr_dev_free(c, c->sadj_ws);
    c->sadj_ws = nullptr;
    pr_dev_free(c, c->kappa);
    pr_dev_free(c, c->kappa_il);
    pr_dev_free(c, c->cinv2);
    for (int h = 0; h < 2; ++h) {
        pr_dev_free(c, c->su[h]);
        pr_dev_free(c, c->sv[h]);
        pr_dev_free(c, c->sr[h]);
    }
    pr_dev_free(c, c->partials);
    pr_dev_free(c, c->dev_flag);
    pr_dev_free(c, c->sweep_ctr);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    c->ev_pool.clear();
}

static cudaEvent_t prof_event(pr_ctx* c) {
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

extern "C" pr_status pr_profile(pr_ctx* ctx, int on) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_profile: ctx is NULL");
    if (on) {
        ctx->prof.clear();
        ctx->ev_used = 0;
    }
    ctx->prof_on = on != 0;
    return PR_OK;
}

extern "C" pr_status pr_profile_read(pr_ctx* ctx, int kind, int* launches, double* total_ms) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_profile_read: ctx is NULL");
    int cnt = 0;
    double tot = 0.0;
    for (const auto& r : ctx->prof) {
        if (r.kind != kind) continue;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "pr_profile_read: event synchronize");
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "pr_profile_read: elapsed time");
        tot += ms;
        ++cnt;
    }
    if (launches) *launches = cnt;
    if (total_ms) *total_ms = tot;
    return PR_OK;
}

extern "C" void pr_destroy(pr_ctx* ctx) {
    if (!ctx) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(ctx->device);
    free_all(ctx);
    cudaSetDevice(cur);
    delete ctx;
}

// integer step count of a coupling interval, or -1
static int step_count(double dt_com, double dt) {
    if (!(dt > 0) || !(dt_com > 0)) return -1;
    double m = dt_com / dt;
    long long mi = llround(m);
    if (mi < 1 || mi > (1LL << 30)) return -1;
    if (fabs((double)mi * dt - dt_com) > 1e-9 * dt_com) return -1;
    return (int)mi;
}

extern "C" pr_status pr_create(const pr_grid* grid, const void* c_dev, double dt_f, double dt_c,
                               int N, double T, const pr_options* opts, pr_ctx** out) {
    if (!out) return pr_fail(nullptr, PR_EINVAL, "pr_create: out is NULL");
    *out = nullptr;
    if (!grid || !c_dev) return pr_fail(nullptr, PR_EINVAL, "pr_create: grid or c is NULL");
    if (grid->dim < 1 || grid->dim > 3)
        return pr_fail(nullptr, PR_EINVAL, "pr_create: dim must be 1, 2 or 3");
    const int64_t n = grid->nf[0];
    for (int a = 1; a < grid->dim; ++a)
        if (grid->nf[a] != n)
            return pr_fail(nullptr, PR_EINVAL, "pr_create: nf must be equal on every axis");
    if (n < 4 || n > (1 << 20)) return pr_fail(nullptr, PR_EINVAL, "pr_create: nf out of range [4, 2^20]");
    if (grid->ratio < 1 || n % grid->ratio != 0)
        return pr_fail(nullptr, PR_EINVAL, "pr_create: ratio must be >= 1 and divide nf");
    if (N < 1) return pr_fail(nullptr, PR_EINVAL, "pr_create: N must be >= 1");
    if (!(T > 0)) return pr_fail(nullptr, PR_EINVAL, "pr_create: T must be > 0");
    pr_options o = {PR_F32, 4, 0, 1e-13, 0, 0};
    if (opts) o = *opts;
    if (o.dtype != PR_F32 && o.dtype != PR_F64)
        return pr_fail(nullptr, PR_EINVAL, "pr_create: dtype must be PR_F32 or PR_F64");
    if (o.block_depth < 0 || o.block_depth > 64)
        return pr_fail(nullptr, PR_EINVAL, "pr_create: block_depth must be in [0, 64]");
    const double dt_com = T / N;
    const int m_f = step_count(dt_com, dt_f);
    const int m_c = step_count(dt_com, dt_c);
    if (m_f < 0) return pr_fail(nullptr, PR_EINVAL, "pr_create: (T/N)/dt_f is not a positive integer");
    if (m_c < 0) return pr_fail(nullptr, PR_EINVAL, "pr_create: (T/N)/dt_c is not a positive integer");

    int64_t pts = 1;
    for (int a = 0; a < grid->dim; ++a) pts *= n;
    const size_t esz = o.dtype == PR_F32 ? 4 : 8;

    // read c back to check it and to form kappa in FP64 on the host
    std::vector<double> c(pts);
    {
        cudaPointerAttributes attr;
        if (cudaPointerGetAttributes(&attr, c_dev) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            return pr_fail(nullptr, PR_EINVAL, "pr_create: c must be a device pointer");
        }
        // on a private non-blocking stream ordered after the work already
        // queued on the legacy default stream, so that no other stream of
        // the device is waited for
        std::vector<char> raw(pts * esz);
        cudaStream_t cs = nullptr;
        cudaEvent_t ce = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ce, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(ce, (cudaStream_t)0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ce, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(raw.data(), c_dev, pts * esz, cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (ce) cudaEventDestroy(ce);
        if (cs) cudaStreamDestroy(cs);
        if (e != cudaSuccess) return pr_cuda_fail(nullptr, e, "pr_create: copy c");
        for (int64_t i = 0; i < pts; ++i)
            c[i] = o.dtype == PR_F32 ? (double)((const float*)raw.data())[i] : ((const double*)raw.data())[i];
    }
    double cmax = 0, cmax_coarse = 0;
    for (int64_t i = 0; i < pts; ++i) {
        if (!(c[i] > 0) || !isfinite(c[i])) return pr_fail(nullptr, PR_EINVAL, "pr_create: c must be finite and > 0");
        cmax = std::max(cmax, c[i]);
    }
    {   // coarse nodes coincide with every ratio-th fine node (Sec. 6)
        const int64_t nc = n / grid->ratio;
        int64_t cpts = 1;
        for (int a = 0; a < grid->dim; ++a) cpts *= nc;
        for (int64_t J = 0; J < cpts; ++J) {
            int64_t rem = J, idx = 0, stride = 1;
            for (int a = 0; a < grid->dim; ++a) {
                idx += (rem % nc) * grid->ratio * stride;
                rem /= nc;
                stride *= n;
            }
            cmax_coarse = std::max(cmax_coarse, c[idx]);
        }
    }
    const double dx = 1.0 / (double)n;
    const double sd = sqrt((double)grid->dim);
    if (cmax * dt_f * sd / dx > 1.0) return pr_fail(nullptr, PR_EINVAL, "pr_create: fine step violates CFL");
    if (cmax_coarse * dt_c * sd / (dx * grid->ratio) > 1.0)
        return pr_fail(nullptr, PR_EINVAL, "pr_create: coarse step violates CFL");

    pr_ctx* ctx = nullptr;
    pr_status st = pr_build_ctx(grid->dim, n, grid->ratio, N, T, dt_f, m_f, dt_c, m_c, o, c, &ctx);
    if (st != PR_OK) return st;
    if (grid->ratio >= 1) {
        // the coarse propagator's own context: coarse grid, c at the coarse nodes,
        // step dt_c, m_C steps per interval (Sec. 3.1)
        const int64_t nc = n / grid->ratio;
        int64_t cpts = 1;
        for (int a = 0; a < grid->dim; ++a) cpts *= nc;
        std::vector<double> cc(cpts);
        for (int64_t J = 0; J < cpts; ++J) {
            int64_t rem = J, idx = 0, stride = 1;
            for (int a = 0; a < grid->dim; ++a) {
                idx += (rem % nc) * grid->ratio * stride;
                rem /= nc;
                stride *= n;
            }
            cc[J] = c[idx];
        }
        pr_status sc = pr_build_ctx(grid->dim, nc, 1, N, T, dt_c, m_c, dt_c, m_c, o, cc, &ctx->coarse);
        if (sc != PR_OK) {
            pr_destroy(ctx);
            return sc;
        }
    }
    *out = ctx;
    return PR_OK;
}

// Context of one grid: coefficient arrays and pass scratch for propagating
// N slices with step dt (m steps per coupling interval).
pr_status pr_build_ctx(int dim, int64_t n, int ratio, int N, double T, double dt, int m,
                       double dt_c, int m_c, const pr_options& o, const std::vector<double>& c,
                       pr_ctx** out) {
    int64_t pts = 1;
    for (int a = 0; a < dim; ++a) pts *= n;
    const size_t esz = o.dtype == PR_F32 ? 4 : 8;
    const double dx = 1.0 / (double)n;
    double cmax = 0;
    for (int64_t i = 0; i < pts; ++i) cmax = std::max(cmax, c[i]);
    pr_ctx* ctx = new pr_ctx();
    pr_current_allocator(&ctx->ualloc, &ctx->urelease, &ctx->uarg);
    cudaGetDevice(&ctx->device);
    ctx->dim = dim;
    ctx->n = n;
    ctx->pts = pts;
    ctx->ratio = ratio;
    ctx->N = N;
    ctx->dtype = o.dtype;
    ctx->T = T;
    ctx->dt_com = T / N;
    ctx->dt_f = dt;
    ctx->dt_c = dt_c;
    ctx->dx = dx;
    ctx->m_f = m;
    ctx->m_c = m_c;
    ctx->cmax = cmax;
    ctx->opts = o;
    // 0 = the deepest fused depth the geometry has (8, else 4), else one step per pass
    int depth = o.block_depth;
    if (depth == 0) depth = pr_tb2d_supported(ctx, 8) ? 8 : 4;
    ctx->block_depth = (pr_tb2d_supported(ctx, depth) || pr_tb3d_supported(ctx, depth)) ? depth : 1;

    std::vector<char> kap(pts * esz);
    std::vector<double> cinv2(pts);
    for (int64_t i = 0; i < pts; ++i) {
        const double k = c[i] * c[i] * dt / (dx * dx);
        if (o.dtype == PR_F32) ((float*)kap.data())[i] = (float)k;
        else ((double*)kap.data())[i] = k;
        cinv2[i] = 1.0 / (c[i] * c[i]);
    }
    auto fail = [&](cudaError_t e, const char* what) {
        pr_status s = pr_cuda_fail(nullptr, e, what);
        free_all(ctx);
        delete ctx;
        return s;
    };
    cudaError_t e;
    if ((e = pr_dev_malloc(ctx, &ctx->kappa, pts * esz)) != cudaSuccess) return fail(e, "pr_create: alloc kappa");
    if ((e = pr_dev_malloc(ctx, (void**)&ctx->cinv2, pts * 8)) != cudaSuccess) return fail(e, "pr_create: alloc cinv2");
    if ((e = pr_dev_malloc(ctx, (void**)&ctx->c64, pts * 8)) != cudaSuccess) return fail(e, "pr_create: alloc c");
    if ((e = cudaMemcpy(ctx->kappa, kap.data(), pts * esz, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "pr_create: upload kappa");
    if ((e = cudaMemcpy(ctx->cinv2, cinv2.data(), pts * 8, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "pr_create: upload cinv2");
    if ((pr_tb2d_supported(ctx, 8) || pr_tb2d_supported(ctx, 4)) && n <= 1024) {   // widths of the two-column kernel
        // kappa for the two-column fused kernel: per thread (k(2t), k(2t+1), -, -),
        // the free half filled with D0 in shared memory
        std::vector<float> il((size_t)pts * 2, 0.0f);
        const float* kf = (const float*)kap.data();
        for (int64_t j = 0; j < pts / 2; ++j) {
            il[4 * j] = kf[2 * j];
            il[4 * j + 1] = kf[2 * j + 1];
        }
        if ((e = pr_dev_malloc(ctx, (void**)&ctx->kappa_il, pts * 8)) != cudaSuccess) return fail(e, "pr_create: alloc kappa pairs");
        if ((e = cudaMemcpy(ctx->kappa_il, il.data(), pts * 8, cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(e, "pr_create: upload kappa pairs");
    }
    if ((e = cudaMemcpy(ctx->c64, c.data(), pts * 8, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e, "pr_create: upload c");
    const size_t state = (size_t)N * pts;
    // the fused 2D sweeps carry a bfloat16 residual, one-level sweeps a byte
    ctx->resid_bytes = o.dtype != PR_F32 ? 0
                       : (pr_tb2d_supported(ctx, 8) || pr_tb2d_supported(ctx, 4) || pr_tb3d_supported(ctx, 4)) ? 2 : 1;
    for (int h = 0; h < 2; ++h) {
        if ((e = pr_dev_malloc(ctx, &ctx->su[h], state * esz)) != cudaSuccess) return fail(e, "pr_create: alloc scratch u");
        if ((e = pr_dev_malloc(ctx, &ctx->sv[h], state * esz)) != cudaSuccess) return fail(e, "pr_create: alloc scratch v");
        if (ctx->resid_bytes && (e = pr_dev_malloc(ctx, &ctx->sr[h], state * ctx->resid_bytes)) != cudaSuccess)
            return fail(e, "pr_create: alloc scratch residual");
    }
    if ((e = pr_dev_malloc(ctx, (void**)&ctx->dev_flag, sizeof(int))) != cudaSuccess) return fail(e, "pr_create: alloc flag");
    if ((e = cudaMemset(ctx->dev_flag, 0, sizeof(int))) != cudaSuccess) return fail(e, "pr_create: clear flag");
    if ((e = pr_dev_malloc(ctx, (void**)&ctx->sweep_ctr, sizeof(unsigned int))) != cudaSuccess)
        return fail(e, "pr_create: alloc sweep counter");
    *out = ctx;
    return PR_OK;
}

extern "C" pr_status pr_info(const pr_ctx* ctx, int* m_f, int* m_c, int64_t* pts, int* block_depth) {
    if (!ctx) return PR_EINVAL;
    if (m_f) *m_f = ctx->m_f;
    if (m_c) *m_c = ctx->m_c;
    if (pts) *pts = ctx->pts;
    if (block_depth) *block_depth = ctx->block_depth;
    return PR_OK;
}

static bool overlaps(const void* a, const void* b, size_t bytes) {
    const char* x = (const char*)a;
    const char* y = (const char*)b;
    return x < y + bytes && y < x + bytes;
}

extern "C" pr_status pr_fine_all_slices(pr_ctx* ctx, const void* u_in, const void* v_in,
                                        void* u_out, void* v_out, int n_begin, int n_end,
                                        void* stream) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_fine_all_slices: ctx is NULL");
    if (!u_in || !v_in || !u_out || !v_out)
        return pr_fail(ctx, PR_EINVAL, "pr_fine_all_slices: NULL array");
    if (n_begin < 0 || n_end < n_begin || n_end > ctx->N)
        return pr_fail(ctx, PR_EINVAL, "pr_fine_all_slices: slice range outside [0, N]");
    const size_t esz = ctx->dtype == PR_F32 ? 4 : 8;
    const uintptr_t al = (uintptr_t)u_in | (uintptr_t)v_in | (uintptr_t)u_out | (uintptr_t)v_out;
    if (al & 15) return pr_fail(ctx, PR_EINVAL, "pr_fine_all_slices: arrays must be 16-byte aligned");
    if (n_end == n_begin) return PR_OK;
    const int ns = n_end - n_begin;
    const size_t off = (size_t)n_begin * ctx->pts * esz;
    const size_t bytes = (size_t)ns * ctx->pts * esz;
    const char* ui = (const char*)u_in + off;
    const char* vi = (const char*)v_in + off;
    char* uo = (char*)u_out + off;
    char* vo = (char*)v_out + off;
    const bool inplace = (ui == uo) && (vi == vo);
    if (!inplace) {
        if (overlaps(ui, uo, bytes) || overlaps(ui, vo, bytes) || overlaps(vi, uo, bytes) ||
            overlaps(vi, vo, bytes))
            return pr_fail(ctx, PR_EINVAL, "pr_fine_all_slices: inputs and outputs overlap");
    }
    if (overlaps(uo, vo, bytes)) return pr_fail(ctx, PR_EINVAL, "pr_fine_all_slices: u_out and v_out overlap");
    const int depth = ctx->block_depth;
    const int rfmt = depth > 1 ? PR_RESID_BF16 : PR_RESID_I8;
    const size_t rsz = rfmt == PR_RESID_BF16 ? 2 : 1;
    if (ctx->dtype == PR_F32 && (size_t)ctx->resid_bytes < rsz)
        return pr_fail(ctx, PR_EINVAL, "pr_fine_all_slices: residual scratch too small for the fused depth");
    cudaStream_t st = (cudaStream_t)stream;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != ctx->device) cudaSetDevice(ctx->device);

    const int m = ctx->m_f;
    const int levels_total = m + 1;            // m full steps = m + 1 kicks
    int passes = (levels_total + depth - 1) / depth;
    // a lone final level joins the previous pass where the fused kernel
    // takes depth + 1 levels
    const bool merge_last = depth > 1 && passes >= 2 && levels_total % depth == 1 &&
                            ctx->dtype == PR_F32 && pr_tb2d_extra_level(ctx);
    if (merge_last) --passes;
    auto scr_u = [&](int h) { return (char*)ctx->su[h] + off; };
    auto scr_v = [&](int h) { return (char*)ctx->sv[h] + off; };
    auto scr_r = [&](int h) -> void* {
        return ctx->dtype == PR_F32 ? (char*)ctx->sr[h] + (size_t)n_begin * ctx->pts * rsz : nullptr;
    };
    pr_status s = PR_OK;
    const bool resident = ctx->resident > 0 || (ctx->resident < 0 && ctx->n <= 128);
    if (resident && pr_resident2d_supported(ctx)) {
        // every kick of every slice in one launch, each slice inside one cluster
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (ctx->prof_on) {
            ea = prof_event(ctx);
            eb = prof_event(ctx);
            if (ea && eb) cudaEventRecord(ea, st);
        }
        s = pr_launch_resident2d(ctx, ui, vi, uo, vo, ns, st);
        if (ctx->prof_on && ea && eb) {
            cudaEventRecord(eb, st);
            ctx->prof.push_back({3, ea, eb});
        }
        if (cur != ctx->device && cur >= 0) cudaSetDevice(cur);
        return s;
    }
    if (ctx->dtype == PR_F32 && depth == 8 && pr_tb2d_sweep_supported(ctx, passes)) {
        // every pass of the sweep in one persistent launch
        pr_sweep sw;
        sw.u_in = ui;
        sw.v_in = vi;
        sw.u_out = uo;
        sw.v_out = vo;
        for (int h = 0; h < 2; ++h) {
            sw.su[h] = scr_u(h);
            sw.sv[h] = scr_v(h);
            sw.sr[h] = scr_r(h);
        }
        sw.nslices = ns;
        sw.passes = passes;
        sw.last_levels = levels_total - (passes - 1) * depth;
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (ctx->prof_on) {
            ea = prof_event(ctx);
            eb = prof_event(ctx);
            if (ea && eb) cudaEventRecord(ea, st);
        }
        s = pr_launch_fine_tb2d_sweep(ctx, sw, st);
        if (ctx->prof_on && ea && eb) {
            cudaEventRecord(eb, st);
            ctx->prof.push_back({2, ea, eb});
        }
        if (cur != ctx->device && cur >= 0) cudaSetDevice(cur);
        return s;
    }
    for (int p = 0; p < passes && s == PR_OK; ++p) {
        pr_pass ps;
        ps.nslices = ns;
        ps.g0 = p * depth;
        ps.levels = (merge_last && p == passes - 1) ? depth + 1 : std::min(depth, levels_total - ps.g0);
        ps.m = m;
        ps.rfmt = rfmt;
        const bool first = (p == 0), last = (p == passes - 1);
        ps.u_in = first ? (const void*)ui : scr_u((p - 1) & 1);
        ps.v_in = first ? (const void*)vi : scr_v((p - 1) & 1);
        ps.r_in = first ? nullptr : scr_r((p - 1) & 1);
        const bool single_inplace = first && last && inplace;
        ps.u_out = (last && !single_inplace) ? (void*)uo : scr_u(p & 1);
        ps.v_out = (last && !single_inplace) ? (void*)vo : scr_v(p & 1);
        ps.r_out = last ? nullptr : scr_r(p & 1);
        const int kind = ps.levels > 1 ? 0 : 1;
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (ctx->prof_on) {
            ea = prof_event(ctx);
            eb = prof_event(ctx);
            if (ea && eb) cudaEventRecord(ea, st);
        }
        if (ps.levels > 1)
            s = pr_launch_fine_tb2d(ctx, ps, st);
        else
            s = pr_launch_fine_naive(ctx, ps, st);
        if (ctx->prof_on && ea && eb) {
            cudaEventRecord(eb, st);
            ctx->prof.push_back({kind, ea, eb});
        }
        if (s == PR_OK && single_inplace) {
            cudaError_t e = cudaMemcpyAsync(uo, ps.u_out, bytes, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(vo, ps.v_out, bytes, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) s = pr_cuda_fail(ctx, e, "pr_fine_all_slices: in-place copy");
        }
    }
    if (cur != ctx->device && cur >= 0) cudaSetDevice(cur);
    return s;
}

extern "C" pr_status pr_set_fused_columns(pr_ctx* ctx, int columns) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_set_fused_columns: ctx is NULL");
    if (columns != 0 && columns != 2 && columns != 4)
        return pr_fail(ctx, PR_EINVAL, "pr_set_fused_columns: columns must be 0, 2 or 4");
    ctx->tb_cols = columns;
    return PR_OK;
}

extern "C" pr_status pr_set_wide_rows(pr_ctx* ctx, int mode) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_set_wide_rows: ctx is NULL");
    if (mode != 1 && mode != 2) return pr_fail(ctx, PR_EINVAL, "pr_set_wide_rows: mode must be 1 or 2");
    ctx->wide_rows = mode;
    return PR_OK;
}

extern "C" pr_status pr_set_resident(pr_ctx* ctx, int on) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_set_resident: ctx is NULL");
    ctx->resident = on != 0;
    return PR_OK;
}

extern "C" pr_status pr_set_one_launch(pr_ctx* ctx, int on) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_set_one_launch: ctx is NULL");
    ctx->one_launch = on != 0;
    return PR_OK;
}

extern "C" pr_status pr_debug_stall_waits(pr_ctx* ctx, int enable) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_debug_stall_waits: ctx is NULL");
    ctx->debug_stall = enable != 0;
    return PR_OK;
}

pr_status pr_take_flag(pr_ctx* ctx, pr_ctx* report, cudaStream_t st, const char* where) {
    int flag = 0;
    cudaError_t e = cudaMemcpyAsync(&flag, ctx->dev_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return pr_cuda_fail(report, e, where);
    if (flag) {
        e = cudaMemsetAsync(ctx->dev_flag, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return pr_cuda_fail(report, e, where);
        char buf[160];
        snprintf(buf, sizeof buf, "%s: a device-side bounded wait gave up (code %d)", where, flag);
        return pr_fail(report, PR_ETIMEOUT, buf);
    }
    return PR_OK;
}

extern "C" pr_status pr_check(pr_ctx* ctx, void* stream) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_check: ctx is NULL");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return pr_cuda_fail(ctx, e, "pr_check: stream synchronize");
    return pr_take_flag(ctx, ctx, (cudaStream_t)stream, "pr_check");
}

extern "C" pr_status pr_energy(pr_ctx* ctx, const void* u, const void* v, int n_begin, int n_end,
                               double* e_host, void* stream) {
    if (!ctx) return pr_fail(nullptr, PR_EINVAL, "pr_energy: ctx is NULL");
    if (!u || !v || !e_host) return pr_fail(ctx, PR_EINVAL, "pr_energy: NULL argument");
    if (n_begin < 0 || n_end < n_begin || n_end > ctx->N)
        return pr_fail(ctx, PR_EINVAL, "pr_energy: slice range outside [0, N]");
    if (n_end == n_begin) return PR_OK;
    const size_t off = (size_t)n_begin * ctx->pts * (ctx->dtype == PR_F32 ? 4 : 8);
    return pr_launch_energy(ctx, (const char*)u + off, (const char*)v + off, n_end - n_begin,
                            e_host, (cudaStream_t)stream);
}
