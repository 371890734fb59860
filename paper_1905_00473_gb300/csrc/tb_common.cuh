// Device helpers shared by the fused 2D fine-propagator kernels: mbarrier and
// TMA bulk-copy wrappers with bounded waits, L2 cache policies, packed FP32
// pairs, and the launch parameters.
#pragma once

#include <stdint.h>

namespace tb {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// complete `bytes` transaction bytes of the current phase without a copy
// (no arrival): settles bytes that an expect_tx announced but no copy brings
__device__ __forceinline__ void mbar_complete_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// a plain arrival (no transaction bytes): completes the phase of a slot that
// receives no copy, so every slot completes one phase per ring lap
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Thread-block clusters (distributed shared memory).  A CTA's shared::cta
// address is also a valid shared::cluster address of its own memory; mapa
// gives the same offset in another CTA of the cluster.
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t mapa_rank(uint32_t cta_addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(cta_addr), "r"(rank));
    return r;
}
// every thread of every CTA of the cluster: release what this thread wrote,
// acquire what the others wrote before their arrival
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait: false after `limit_ns` without completion
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}
// Stores into another CTA's shared memory that complete transaction bytes on
// an mbarrier there (no fence: the receiver's wait on that mbarrier makes the
// data visible to it).  Both addresses are shared::cluster addresses.
__device__ __forceinline__ void st_async_f4(uint32_t addr, float4 v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(addr),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void st_async_f32(uint32_t addr, float v, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];" ::"r"(addr), "f"(v),
                 "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t policy(int kind) {
    uint64_t p;
    if (kind == 0) asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    else if (kind == 1) asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    else asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// Packed FP32 pairs (Blackwell f32x2 arithmetic): two lanes of one 64-bit
// register, each lane rounded exactly like the scalar instruction.
#ifndef PR_TB2D_PACKED
#define PR_TB2D_PACKED 1
#endif
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2_pack(float a, float b) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float f2_lo(f2_t x) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
    return a;
}
__device__ __forceinline__ float f2_hi(f2_t x) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
    return b;
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b) {
    f2_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b) {
    f2_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// s = a + b and its exact rounding error r = (a + b) - s per lane (TwoSum,
// Knuth), the same operations as pr_two_sum
__device__ __forceinline__ f2_t f2_two_sum(f2_t a, f2_t b, f2_t* r) {
    const f2_t s = f2_add(a, b);
    const f2_t bb = f2_sub(s, a);
    *r = f2_add(f2_sub(a, f2_sub(s, bb)), f2_sub(b, bb));
    return s;
}
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c) {
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

struct Tb2dParams {
    const float* u_in;
    const float* v_in;
    const uint16_t* r_in; // bfloat16 residual; null: zero residual (first pass)
    const float* kap;
    float* u_out;
    float* v_out;
    uint16_t* r_out;      // null: last pass, residual folded into u
    int* flag;
    int64_t rows_total;   // nslices * n
    int n;
    int g0, levels, m;
    float dt;
    uint32_t tx_extra;    // test hook: bytes expected on top of those copied (0 normally)
    uint64_t wait_ns;     // limit of each bounded mbarrier wait
};

// First row of CTA b's share when the N*n rows of a batch of N slices are cut
// into G contiguous ranges of equal cost.  A range is processed slice by
// slice, and every segment costs its rows plus K pipeline steps of halo and
// drain, so a range that crosses slice boundaries gets fewer rows: with
// phi(r) = r + K * (slice boundaries below r) the cut points are where phi
// crosses multiples of phi_total / G (inside a boundary's jump the cut falls
// on the boundary itself).
// (host and device: the CPU tests compile it into a host harness)
__host__ __device__ __forceinline__ int64_t balanced_row(int64_t rows_total, int n, int K, int64_t b, int64_t G) {
    const int64_t slices = rows_total / n;
    const int64_t phi = (rows_total + (slices - 1) * K) * b / G;
    const int64_t j = phi / (n + K);
    const int64_t a = phi - j * K, c = (j + 1) * (int64_t)n;
    const int64_t r = a < c ? a : c;
    return r < rows_total ? r : rows_total;
}

// Global row of local row rho of a segment whose first local row is ylo
// (periodic in y).  A segment of H <= n rows loads H + 2L rows, so
// ylo + rho < n + (n + 2L) <= 3n for L <= n/2: at most two wraps.
__device__ __forceinline__ int seg_row(int ylo, int rho, int n) {
    int y = ylo + rho;
    if (y >= n) y -= n;
    if (y >= n) y -= n;
    return y;
}

// Per-segment constants of one CTA's current row range.
struct Seg {
    const float* u_s;
    const float* v_s;
    const uint16_t* r_s;
    int64_t slice_off;   // slice * n^2
    uint32_t base;       // ring index of local row 0
    int ylo;             // global row of local row 0
    int H, L, nload;
    int x0;              // first global column of the CTA's rows (x-strips; 0 = whole rows)
};

// Copy W elements of a periodic row starting at column x0 (-n < x0 < n) into
// shared memory: one bulk copy, or two where the range wraps past column n.
// Every piece must start on 16 bytes and span a multiple of 16 bytes.
__device__ __forceinline__ void bulk_row_g2s(void* dst, const void* row, int x0, int W, int n, uint32_t esz,
                                             uint64_t* bar, uint64_t pol) {
    const int a = x0 < 0 ? x0 + n : x0;
    const int first = min(W, n - a);
    bulk_g2s(dst, (const char*)row + (size_t)a * esz, (uint32_t)first * esz, bar, pol);
    if (first < W) bulk_g2s((char*)dst + (size_t)first * esz, row, (uint32_t)(W - first) * esz, bar, pol);
}


}  // namespace tb
