// ts_async.cuh -- asynchronous-copy building blocks of the persistent N = 1024 passes (sm_103a):
// mbarriers with bounded waits, TMA tensor and bulk copies global -> shared, TMA tensor stores
// shared -> global with bulk-group waits, proxy fences, acquire loads, and the transfer-function multiply of a column tile (Eq. 1, angular-spectrum H).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ts_device.cuh"
#include "ts_prop_decl.h"

namespace ts {
namespace async {

__device__ __forceinline__ uint32_t s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* m, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(s32(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* m, uint32_t parity, long long budget)
{
    if (mbar_try(m, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(m, parity)) {
        if (clock64() - t0 > budget) return false;
    }
    return true;
}
// generic-proxy accesses of this thread (and those ordered before it by a barrier) before later
// asynchronous-proxy accesses of shared memory
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// generic-proxy global writes made visible to this thread (by an acquire) before its later
// asynchronous-proxy reads of global memory (TMA / bulk copies)
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// 2-D tiled tensor copy global -> shared, completion counted in bytes on the mbarrier
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* m)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            s32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(s32(m))
        : "memory");
}
// 2-D tiled tensor copy shared -> global, completion tracked by this thread's bulk groups
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(s32(src)), "r"(x), "r"(y)
                 : "memory");
}
// closes this thread's bulk stores issued since the last commit into one bulk group
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// waits until at most PENDING of this thread's most recent bulk groups still read shared memory
template <int PENDING = 0>
__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(PENDING) : "memory");
}
// waits until every bulk group of this thread has completed (its global writes performed)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// contiguous bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* m)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(s32(dst)),
                 "l"(src), "r"(bytes), "r"(s32(m))
                 : "memory");
}

// v[i] (frequency m = t + T i of column col) *= H or conj(H), with tab(m) = (P(m), ky(m)^2, -) read
// from the caller's shared-memory table (whatever its layout).  HMODE 0: exact angular-spectrum phase
// beyond its paraxial part; 1: separable P' with the cross term exp(-i e) as a short series;
// 2: separable with e <= 0.01 rad, exp(-i e) = 1 - e^2/2 - i e; 3: separable with e <= 4.4e-4 rad,
// exp(-i e) = 1 - i e (error e^2 / 2 <= 1e-7 rad, below the FP32 rounding of the product).
template <bool CONJ, int HMODE, class Tab, int T = 32>
__device__ __forceinline__ void transfer_tile_tab(float2 (&v)[32], Tab tab, int col, int t, float ccross,
                                                  float dcoef, float inv_k2)
{
    const float4 hx = tab(col);
    const float2 px = make_float2(hx.x, hx.y);
    const float kx2 = hx.z;
    const float cx = ccross * kx2;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const float4 hy = tab(t + T * i);
        const float2 q = cmul(px, make_float2(hy.x, hy.y));
        float2 h;
        if constexpr (HMODE == 0) {
            const float k2 = kx2 + hy.z;
            const float qq = k2 * inv_k2;
            if (qq >= 1.0f) {
                h = make_float2(0.0f, 0.0f);
            } else {
                const float d = 1.0f + sqrtf(1.0f - qq);
                const float del = __fdividef(dcoef * k2 * k2, d * d);
                const float d2 = del * del;
                const float cd = 1.0f - d2 * (0.5f - d2 * (1.0f / 24.0f - d2 * (1.0f / 720.0f)));
                const float sd = del * (1.0f - d2 * (1.0f / 6.0f - d2 * (1.0f / 120.0f - d2 * (1.0f / 5040.0f))));
                h = cmul(q, make_float2(cd, -sd));
            }
        } else if constexpr (HMODE == 1) {
            const float e = cx * hy.z;
            const float e2 = e * e;
            h = cmul(q, make_float2(1.0f - e2 * (0.5f - e2 * (1.0f / 24.0f)), -e * (1.0f - e2 * (1.0f / 6.0f))));
        } else if constexpr (HMODE == 2) {
            const float e = cx * hy.z;
            const float ce = fmaf(-0.5f * e, e, 1.0f);
            h = make_float2(fmaf(q.x, ce, q.y * e), fmaf(q.y, ce, -q.x * e));
        } else {
            const float e = cx * hy.z;
            h = make_float2(fmaf(e, q.y, q.x), fmaf(-e, q.x, q.y));
        }
        v[i] = CONJ ? cmulc(v[i], h) : cmul(v[i], h);
    }
}

template <bool CONJ, int HMODE>
__device__ __forceinline__ void transfer_tile(float2 (&v)[32], const float4* ht, int col, int t, float ccross,
                                              float dcoef, float inv_k2)
{
    transfer_tile_tab<CONJ, HMODE>(v, [ht](int m) { return ht[m]; }, col, t, ccross, dcoef, inv_k2);
}

// ---- host: the TMA tensor map of a batch of N x N complex64 fields, viewed as (2N floats) x (B N
// rows), with boxes of box_rows rows x box_floats floats (the driver's encoder, reached through the
// runtime's entry-point query, so no link against the driver library is needed) ----
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_tiled_fn()
{
    static EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(ptr);
    }();
    return fn;
}

// cudaErrorNotSupported when the encoder is unavailable, cudaErrorInvalidValue when it rejects the map
inline cudaError_t field_tensor_map(CUtensorMap* map, void* field, int N, int B, int box_floats, int box_rows)
{
    EncodeTiledFn enc = encode_tiled_fn();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)2 * N, (cuuint64_t)B * N};
    const cuuint64_t strides[1] = {(cuuint64_t)2 * N * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)box_floats, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, field, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    return cudaSuccess;
}

}  // namespace async
}  // namespace ts
