// ts_tc.cuh -- tcgen05 (5th-generation tensor core) helpers for sm_103a: TMEM allocation, shared
// memory matrix descriptors, the BF16 MMA with FP32 accumulation in TMEM, commit to an mbarrier,
// bounded mbarrier waits and TMEM loads.  Inline PTX only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ts {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ---- TMEM allocation (one full warp executes these) ----
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() { asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// ---- ordering between thread-level synchronisation and tcgen05 operations ----
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes become visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---- shared memory matrix descriptor, K-major, no swizzle ----
// Core matrices of 8 rows x 16 bytes are stored as 128 contiguous bytes; `lbo` is the byte distance
// between core matrices adjacent along K, `sbo` between core matrices adjacent along M / N.
// Fields: start address >> 4 [0,14), LBO >> 4 [16,30), SBO >> 4 [32,46), version 1 [46,48),
// base offset 0 [49,52), LBO mode 0 [52], layout (swizzle) 0 = none [61,64).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// MN-major, no swizzle: a core matrix is 8 columns k of 16 bytes (8 consecutive rows m each), 128
// contiguous bytes.  The leading byte offset is the distance between groups of 8 columns k, the
// stride byte offset the distance between core matrices adjacent along M / N (the reverse of the
// K-major roles; checked on the GPU against an FP64 DFT with both assignments).
__device__ __forceinline__ uint64_t smem_desc_mn(uint32_t addr, uint32_t k_group_stride, uint32_t mn_stride)
{
    return smem_desc(addr, k_group_stride, mn_stride);
}

// ---- instruction descriptor for kind::f16: BF16 x BF16 -> FP32, A and B K-major ----
// c_format F32 = 1 at [4,6), a_format BF16 = 1 at [7,10), b_format BF16 = 1 at [10,13),
// N >> 3 at [17,23), M >> 4 at [24,29).
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// bit 15 of the instruction descriptor: A is MN-major (transposed) instead of K-major
constexpr uint32_t kIdescTransposeA = 1u << 15;

// D[tmem] (+)= A[smem] x B[smem]; one thread issues
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// arrive on the mbarrier when all previously issued MMAs of this thread have completed
__device__ __forceinline__ void mma_commit(uint64_t* mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                 : "memory");
}

// ---- mbarrier ----
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* mbar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: true when the phase completed, false after `budget` clock64 cycles
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t parity, long long budget)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(mbar, parity)) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}

// ---- TMEM -> registers: 32 lanes x 32-bit, 16 consecutive columns per thread ----
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16])
{
    uint32_t u[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
          "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) r[i] = __uint_as_float(u[i]);
}
// 32 consecutive columns of this thread's TMEM lane into v[0..31].x (part 0) or .y (part 1); the
// wait for the load is part of the same statement, so no register is read before it has arrived
__device__ __forceinline__ void tmem_ld32_wait(uint32_t taddr, float2 (&v)[32], int part)
{
    if (part == 0) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=f"(v[0].x), "=f"(v[1].x), "=f"(v[2].x), "=f"(v[3].x), "=f"(v[4].x), "=f"(v[5].x), "=f"(v[6].x), "=f"(v[7].x), "=f"(v[8].x), "=f"(v[9].x), "=f"(v[10].x), "=f"(v[11].x), "=f"(v[12].x), "=f"(v[13].x), "=f"(v[14].x), "=f"(v[15].x), "=f"(v[16].x), "=f"(v[17].x), "=f"(v[18].x), "=f"(v[19].x), "=f"(v[20].x), "=f"(v[21].x), "=f"(v[22].x), "=f"(v[23].x), "=f"(v[24].x), "=f"(v[25].x), "=f"(v[26].x), "=f"(v[27].x), "=f"(v[28].x), "=f"(v[29].x), "=f"(v[30].x), "=f"(v[31].x)
            : "r"(taddr)
            : "memory");
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=f"(v[0].y), "=f"(v[1].y), "=f"(v[2].y), "=f"(v[3].y), "=f"(v[4].y), "=f"(v[5].y), "=f"(v[6].y), "=f"(v[7].y), "=f"(v[8].y), "=f"(v[9].y), "=f"(v[10].y), "=f"(v[11].y), "=f"(v[12].y), "=f"(v[13].y), "=f"(v[14].y), "=f"(v[15].y), "=f"(v[16].y), "=f"(v[17].y), "=f"(v[18].y), "=f"(v[19].y), "=f"(v[20].y), "=f"(v[21].y), "=f"(v[22].y), "=f"(v[23].y), "=f"(v[24].y), "=f"(v[25].y), "=f"(v[26].y), "=f"(v[27].y), "=f"(v[28].y), "=f"(v[29].y), "=f"(v[30].y), "=f"(v[31].y)
            : "r"(taddr)
            : "memory");
    }
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---- split of an FP32 pair into BF16 hi and lo pairs: x = hi + lo + O(2^-16 |x|) ----
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t& hi, uint32_t& lo)
{
    uint32_t h;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(b), "f"(a));  // low half = a, high half = b
    const float ha = __uint_as_float(h << 16), hb = __uint_as_float(h & 0xFFFF0000u);
    uint32_t l;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(b - hb), "f"(a - ha));
    hi = h;
    lo = l;
}

}  // namespace tc
}  // namespace ts
