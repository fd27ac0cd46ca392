// ts_tc.cu -- split-BF16 tensor-core DFT building block (tcgen05, sm_103a).
//
// A batch of 32-point complex DFTs X = F x is one real GEMM D = A G with A = [Re x | Im x] (M x 64)
// and G the 64 x 64 real form of F.  Each factor is split into BF16 hi and lo parts and the product is
// formed as hi.hi + hi.lo + lo.hi in FP32 (TMEM accumulators), i.e. one K = 192 GEMM with
// A' = [A_hi | A_hi | A_lo] and G' = [G_hi ; G_lo ; G_hi]: about 2^-16 relative error instead of
// BF16's 2^-8.  One CTA of 128 threads owns 128 vectors (thread m <-> GEMM row m <-> TMEM lane m).
#include <cmath>

#include "ts_internal.h"
#include "ts_tc.cuh"

namespace ts {

namespace {

constexpr int kTcRows = 128;                 // M
constexpr int kTcK = 192;                    // 3 x 64
constexpr int kTcN = 64;                     // Re and Im of 32 outputs
constexpr int kChunk = 128;                  // one core matrix: 8 rows x 16 bytes
constexpr int kSbo = (kTcK / 8) * kChunk;    // 3072 bytes between 8-row groups
constexpr int kABytes = (kTcRows / 8) * kSbo;   // 49152
constexpr int kBBytes = (kTcN / 8) * kSbo;      // 24576
// MN-major A (layouts 1, 2): hi and lo parts of 128 x 64 BF16, 8 consecutive rows of one column k in
// 16 bytes; a core matrix is 8 columns k of those (128 bytes), 16 core matrices along M are
// adjacent, the next 8 columns follow after kMnK bytes.
constexpr int kMnK = (kTcRows / 8) * kChunk;    // 2048
constexpr int kMnPart = 8 * kMnK;               // 16384
// The A window covers every address a descriptor can reach under either reading of the MN-major
// strides (lo part, last K chunk, 15 core-matrix steps of 2048 bytes): 16384 + 12288 + 30976.
constexpr int kAWindow = 65536;
static_assert(kMnPart + 3 * 2 * kMnK + 15 * kMnK + 2 * kChunk <= kAWindow, "MN-major reach inside the A window");
static_assert(kABytes <= kAWindow, "K-major A inside its window");
// The B window is sized so that every address a descriptor can reach stays inside it even under a
// misread of the layout (offsets swapped, or B read with up to 256 rows).
constexpr int kWindowB = ((kTcK / 8) * kSbo + kChunk) > 32 * kSbo ? ((kTcK / 8) * kSbo + kChunk) : 32 * kSbo;
constexpr int kWindow = kAWindow + kWindowB;
static_assert(kBBytes <= kWindowB, "B operand inside its window");
constexpr int kSmem = kWindow + 64;          // + mbarrier and TMEM address slot

__device__ __forceinline__ uint32_t core_off(int row, int k)
{
    return (uint32_t)((row >> 3) * kSbo + (k >> 3) * kChunk + (row & 7) * 16 + (k & 7) * 2);
}
__device__ __forceinline__ uint32_t mn_off(int row, int k)
{
    return (uint32_t)((k >> 3) * kMnK + (row >> 3) * kChunk + (k & 7) * 16 + (row & 7) * 2);
}

// G (64 x 64, real form of the 32-point DFT with exponent sign `sign`), entry (kk, n):
// kk < 32: Re x_kk, else Im x_(kk-32); n < 32: Re X_n, else Im X_(n-32).
__device__ __forceinline__ double g_entry(int kk, int n, int sign)
{
    const int j = kk & 31, q = n & 31;
    double s, c;
    sincospi(2.0 * (double)((j * q) & 31) / 32.0, &s, &c);
    const bool im_in = kk >= 32, im_out = n >= 32;
    if (!im_in && !im_out) return c;
    if (im_in && im_out) return c;
    if (!im_in && im_out) return sign * s;
    return -sign * s;
}

__global__ void __launch_bounds__(kTcRows) tc_dft32_kernel(const float2* __restrict__ x, float2* __restrict__ X,
                                                           int nvec, int sign, int layout, long long budget, int* err)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* A = sm;
    unsigned char* Bm = sm + kAWindow;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kWindow);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kWindow + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        tc::tmem_alloc(tslot, 64);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the whole operand window starts zeroed, so a descriptor that reads outside the staged data (the
    // exchanged-stride check, layout 2) sees zeros rather than stale shared memory
    for (int i = tid; i < kWindow / 16; i += blockDim.x) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    // G' = [G_hi ; G_lo ; G_hi] stored K-major (row n, column k)
    for (int idx = tid; idx < kTcN * (kTcK / 2); idx += blockDim.x) {
        const int n = idx / (kTcK / 2), k = 2 * (idx % (kTcK / 2));
        const int slice = k / 64, kk = k % 64;
        uint32_t hi, lo;
        tc::split_bf16x2((float)g_entry(kk, n, sign), (float)g_entry(kk + 1, n, sign), hi, lo);
        *reinterpret_cast<uint32_t*>(Bm + core_off(n, k)) = (slice == 1) ? lo : hi;
    }
    // A' row of this thread: [hi | hi | lo] of [Re x_0..31, Im x_0..31]
    const int m = tid;
    const size_t v = (size_t)blockIdx.x * kTcRows + m;
    uint32_t hw[32], lw[32];
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
        if (v < (size_t)nvec) {
            a = x[v * 32 + 2 * p];
            b = x[v * 32 + 2 * p + 1];
        }
        tc::split_bf16x2(a.x, b.x, hw[p], lw[p]);        // Re pair
        tc::split_bf16x2(a.y, b.y, hw[16 + p], lw[16 + p]);  // Im pair
    }
    if (layout == 0) {
#pragma unroll
        for (int c = 0; c < 24; ++c) {
            const uint32_t* src = (c < 16) ? hw + 4 * (c & 7) : lw + 4 * (c - 16);
            *reinterpret_cast<uint4*>(A + core_off(m, 8 * c)) = make_uint4(src[0], src[1], src[2], src[3]);
        }
    } else {
        // one column k at a time (two BF16 of each packed word)
        for (int w = 0; w < 32; ++w) {
            const int k = 2 * (w & 15) + (w >= 16 ? 32 : 0);
            *reinterpret_cast<uint16_t*>(A + mn_off(m, k)) = (uint16_t)(hw[w] & 0xFFFFu);
            *reinterpret_cast<uint16_t*>(A + mn_off(m, k + 1)) = (uint16_t)(hw[w] >> 16);
            *reinterpret_cast<uint16_t*>(A + kMnPart + mn_off(m, k)) = (uint16_t)(lw[w] & 0xFFFFu);
            *reinterpret_cast<uint16_t*>(A + kMnPart + mn_off(m, k + 1)) = (uint16_t)(lw[w] >> 16);
        }
    }
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    if (tid == 0) {
        const uint32_t idesc = tc::idesc_bf16_f32(kTcRows, kTcN) | (layout != 0 ? tc::kIdescTransposeA : 0u);
        const uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(Bm);
#pragma unroll
        for (int kk = 0; kk < kTcK / 16; ++kk) {
            uint64_t ad;
            if (layout == 0) {
                ad = tc::smem_desc(a0 + kk * 2 * kChunk, kChunk, kSbo);
            } else {
                // slices: hi.hi, hi.lo, lo.hi; chunk c of 16 columns within a slice
                const uint32_t part = (kk >= 8) ? (uint32_t)kMnPart : 0u;
                const uint32_t start = a0 + part + (uint32_t)((kk & 3) * 2 * kMnK);
                ad = layout == 1 ? tc::smem_desc_mn(start, kMnK, kChunk) : tc::smem_desc_mn(start, kChunk, kMnK);
            }
            const uint64_t bd = tc::smem_desc(b0 + kk * 2 * kChunk, kChunk, kSbo);
            tc::mma_bf16(tbase, ad, bd, idesc, kk > 0 ? 1u : 0u);
        }
        tc::mma_commit(mbar);
    }
    bool ok = tc::mbar_wait_bounded(mbar, 0, budget);
    if (!ok) {
        atomicExch(err, 1);
        ok = tc::mbar_wait_bounded(mbar, 0, budget);  // give the MMA one more budget before freeing TMEM
    }
    tc::fence_after_sync();
    if (ok) {
        float d[64];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float r[16];
            tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + 16 * c, r);
#pragma unroll
            for (int i = 0; i < 16; ++i) d[16 * c + i] = r[i];
        }
        tc::tmem_wait_ld();
        if (v < (size_t)nvec) {
#pragma unroll
            for (int q = 0; q < 32; ++q) X[v * 32 + q] = make_float2(d[q], d[32 + q]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tbase, 64);
    (void)lane;
}

}  // namespace

cudaError_t launch_tc_dft32(const float2* x, float2* X, int nvec, int sign, int layout, long long budget, int* err,
                            cudaStream_t st)
{
    static_assert(kSmem <= 227 * 1024, "shared memory");
    cudaError_t e = cudaFuncSetAttribute(tc_dft32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    const int blocks = (nvec + kTcRows - 1) / kTcRows;
    tc_dft32_kernel<<<blocks, kTcRows, kSmem, st>>>(x, X, nvec, sign, layout, budget, err);
    return cudaGetLastError();
}

}  // namespace ts

extern "C" ts_status ts_tc_dft32(const void* x, void* X, int nvec, int sign, int layout, double timeout_s, int* err,
                                 void* stream)
{
    if (!x || !X || !err || nvec < 1 || (sign != 1 && sign != -1) || layout < 0 || layout > 2 || !(timeout_s > 0.0)) {
        ts::set_error("ts_tc_dft32: need x, X, err, nvec >= 1, sign +-1, layout 0..2 and a positive timeout");
        return TS_ERR_INVALID_ARG;
    }
    int dev = 0, khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    const long long budget = (long long)(timeout_s * (double)(khz > 0 ? khz : 2000000) * 1e3);
    return ts::cuda_check(ts::launch_tc_dft32(reinterpret_cast<const float2*>(x), reinterpret_cast<float2*>(X), nvec,
                                              sign, layout, budget, err, reinterpret_cast<cudaStream_t>(stream)),
                          "ts_tc_dft32");
}
