// pr_fine_all_slices_noalloc: the fine propagator over a batch of slices for
// callers that cannot allocate device memory.
//
// Who needs it.  pr_create allocates the coefficient array and the
// between-level state on the device with cudaMalloc.  Some callers cannot do
// that: code that runs inside a framework owning the whole device memory pool
// (a cudaMalloc would fail or fragment that pool), plugins invoked from
// another library's stream-ordered work, and real-time loops where the
// latency or the possible failure of an allocation is not acceptable.  This
// entry point takes every input and output from the caller and keeps its
// scratch (kappa and the ping-pong state between Verlet levels) in one
// file-scope device array of fixed size, PR_NOALLOC_SCRATCH_BYTES.
//
// Lifetime and sharing.  The array belongs to the loaded library module: each
// GPU on which the library is loaded holds it until the process exits.  Every
// call uses the same array and leaves its contents behind; nothing in it has
// to start at zero, because each call writes kappa and every level's state
// before reading them.  Calls whose GPU work overlaps (different streams, or
// host threads) race on the array: serialise them on one stream.
//
// Set-up.  Host code cannot use the array's name as a device address, so the
// first call on each device (with that device current) asks the runtime for
// the address with cudaGetSymbolAddress and caches it.  Make that first call
// before any stream capture begins.
//
// What it computes is the same level recurrence as the single-level kernel of
// the context path (kick v += w_g kappa D(u), drift u += dt v, FP32 with the
// rounding residual of u carried between levels), one launch per level.
#include <atomic>
#include <stdio.h>

#include "pr_internal.cuh"

static __device__ __align__(256) unsigned char g_noalloc_scratch[PR_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices];
std::atomic<int> g_scratch_ready[kMaxDevices];

cudaError_t scratch_for_current_device(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_scratch_ready[dev].load(std::memory_order_acquire)) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
        g_scratch_ready[dev].store(1, std::memory_order_release);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

__global__ void kappa_from_c(const float* __restrict__ c, float* __restrict__ kap, int64_t pts,
                             double scale) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < pts;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double cj = (double)c[j];
        kap[j] = (float)(cj * cj * scale);
    }
}

template <int DIM>
__device__ __forceinline__ void nb_index(int64_t p, int64_t n, int64_t* nb) {
    int64_t stride = 1, rem = p;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        const int64_t i = rem % n;
        rem /= n;
        nb[2 * a] = p + (((i + 1 == n) ? 0 : i + 1) - i) * stride;
        nb[2 * a + 1] = p + (((i == 0) ? n - 1 : i - 1) - i) * stride;
        stride *= n;
    }
}

template <int DIM>
__global__ void __launch_bounds__(256) noalloc_level(
    const float* __restrict__ u, const int8_t* __restrict__ r, const float* __restrict__ v,
    const float* __restrict__ kap, float* __restrict__ uo, int8_t* __restrict__ ro,
    float* __restrict__ vo, int64_t n, int64_t pts, int64_t total, float wk, float dt, int drift) {
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = idx / pts;
        const int64_t p = idx - s * pts;
        const float* us = u + s * pts;
        const int8_t* rs = r ? r + s * pts : nullptr;
        int64_t nb[2 * DIM];
        nb_index<DIM>(p, n, nb);
        const float u0 = us[p];
        float du = rs ? pr_resid_decode(rs[p], u0) : 0.0f;
        float d0 = 0.0f, dn = 0.0f;
#pragma unroll
        for (int k = 0; k < 2 * DIM; ++k) {
            const float ub = us[nb[k]];
            d0 += (ub - u0);
            if (rs) dn += pr_resid_decode(rs[nb[k]], ub);
        }
        const float vn = fmaf(wk * kap[p], d0 + fmaf(-2.0f * DIM, du, dn), v[idx]);
        if (drift) du = fmaf(dt, vn, du);
        vo[idx] = vn;
        if (ro) {
            int8_t q;
            uo[idx] = pr_sum_encode(u0, du, &q);
            ro[idx] = q;
        } else {
            uo[idx] = u0 + du;
        }
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

pr_status reject(char* msg, size_t msg_len, const char* text) {
    if (msg && msg_len) snprintf(msg, msg_len, "pr_fine_all_slices_noalloc: %s", text);
    return PR_EINVAL;
}

bool overlap(const void* a, const void* b, size_t bytes) {
    const char* x = (const char*)a;
    const char* y = (const char*)b;
    return x < y + bytes && y < x + bytes;
}

}  // namespace

extern "C" pr_status pr_fine_all_slices_noalloc(int dim, int64_t n, int nslices, const float* c,
                                                double dt_f, int m_f, const float* u_in,
                                                const float* v_in, float* u_out, float* v_out,
                                                void* stream, char* msg, size_t msg_len) {
    if (msg && msg_len) msg[0] = '\0';
    if (dim < 1 || dim > 3) return reject(msg, msg_len, "dim must be 1, 2 or 3");
    if (n < 4 || n > (1 << 20)) return reject(msg, msg_len, "n out of range [4, 2^20]");
    if (nslices < 0) return reject(msg, msg_len, "nslices must be >= 0");
    if (m_f < 1) return reject(msg, msg_len, "m_f must be >= 1");
    if (!(dt_f > 0)) return reject(msg, msg_len, "dt_f must be > 0");
    if (!c || !u_in || !v_in || !u_out || !v_out) return reject(msg, msg_len, "NULL array");
    if (((uintptr_t)c | (uintptr_t)u_in | (uintptr_t)v_in | (uintptr_t)u_out | (uintptr_t)v_out) & 15)
        return reject(msg, msg_len, "arrays must be 16-byte aligned");
    int64_t pts = 1;
    for (int a = 0; a < dim; ++a) pts *= n;
    if (nslices == 0) return PR_OK;
    const size_t state = (size_t)nslices * (size_t)pts;
    const size_t bytes = state * 4;
    const bool inplace = (u_in == u_out) && (v_in == v_out);
    if (!inplace && (overlap(u_in, u_out, bytes) || overlap(u_in, v_out, bytes) ||
                     overlap(v_in, u_out, bytes) || overlap(v_in, v_out, bytes)))
        return reject(msg, msg_len, "inputs and outputs overlap");
    if (overlap(u_out, v_out, bytes)) return reject(msg, msg_len, "u_out and v_out overlap");

    // scratch layout: kappa [pts] | set0: u, v [state] f32, r [state] i8 | set1: same
    const size_t kap_b = align256((size_t)pts * 4);
    const size_t f_b = align256(state * 4);
    const size_t r_b = align256(state);
    const size_t need = kap_b + 2 * (2 * f_b + r_b);
    if (need > (size_t)PR_NOALLOC_SCRATCH_BYTES) {
        if (msg && msg_len)
            snprintf(msg, msg_len,
                     "pr_fine_all_slices_noalloc: needs %zu bytes of scratch for %d slices of %lld "
                     "points, more than the fixed %zu (PR_NOALLOC_SCRATCH_BYTES)",
                     need, nslices, (long long)pts, (size_t)PR_NOALLOC_SCRATCH_BYTES);
        return PR_EINVAL;
    }

    void* base = nullptr;
    cudaError_t e = scratch_for_current_device(&base);
    if (e != cudaSuccess) {
        if (msg && msg_len) snprintf(msg, msg_len, "pr_fine_all_slices_noalloc: scratch address: %s", cudaGetErrorString(e));
        return PR_ECUDA;
    }
    unsigned char* sb = (unsigned char*)base;
    float* kap = (float*)sb;
    float* su[2];
    float* sv[2];
    int8_t* sr[2];
    for (int h = 0; h < 2; ++h) {
        unsigned char* set = sb + kap_b + (size_t)h * (2 * f_b + r_b);
        su[h] = (float*)set;
        sv[h] = (float*)(set + f_b);
        sr[h] = (int8_t*)(set + 2 * f_b);
    }

    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    cudaStream_t st = (cudaStream_t)stream;
    const double dx = 1.0 / (double)n;
    kappa_from_c<<<sms * 4, 256, 0, st>>>(c, kap, pts, dt_f / (dx * dx));

    const int64_t total = (int64_t)state;
    int64_t blocks = (total + 255) / 256;
    if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
    for (int g = 0; g <= m_f; ++g) {
        const float* ui = g == 0 ? u_in : su[(g - 1) & 1];
        const float* vi = g == 0 ? v_in : sv[(g - 1) & 1];
        const int8_t* ri = g == 0 ? nullptr : sr[(g - 1) & 1];
        float* uo = g == m_f ? u_out : su[g & 1];
        float* vo = g == m_f ? v_out : sv[g & 1];
        int8_t* ro = g == m_f ? nullptr : sr[g & 1];
        const float wk = (g == 0 || g == m_f) ? 0.5f : 1.0f;
        const int drift = g < m_f;
        switch (dim) {
            case 1: noalloc_level<1><<<(int)blocks, 256, 0, st>>>(ui, ri, vi, kap, uo, ro, vo, n, pts, total, wk, (float)dt_f, drift); break;
            case 2: noalloc_level<2><<<(int)blocks, 256, 0, st>>>(ui, ri, vi, kap, uo, ro, vo, n, pts, total, wk, (float)dt_f, drift); break;
            default: noalloc_level<3><<<(int)blocks, 256, 0, st>>>(ui, ri, vi, kap, uo, ro, vo, n, pts, total, wk, (float)dt_f, drift); break;
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        if (msg && msg_len) snprintf(msg, msg_len, "pr_fine_all_slices_noalloc: launch: %s", cudaGetErrorString(e));
        return PR_ECUDA;
    }
    return PR_OK;
}
