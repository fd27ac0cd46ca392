// ts_tc_prop.cu -- split-BF16 tensor-core variant of the propagation passes (N = 1024).
//
// The passes compute the same split step as the FP32 passes (Eq. 1: column pass
// C = IFFT_cols(H . FFT_cols(R)), row pass R' = FFT_rows(IFFT_rows(C) . exp(i phi))), with every line
// DFT on the 5th-generation tensor cores.  A 1024-point line DFT is factored 32 x 32 (four-step):
// with input index p = 32 h + l and output index q = l' + 32 h',
//   stage a: for every l, the 32-point DFT over h (-> l'), then the twiddle exp(sign 2 pi i l l' / 1024);
//   stage b: for every l', the 32-point DFT over l (-> h').
// Each stage is one real GEMM per 128 vectors, D[128 x 64] = A[128 x 64] G[64 x 64] (Re / Im parts
// of 32 complex values), formed from BF16 hi / lo splits of both factors as hi.hi + hi.lo + lo.hi with
// FP32 accumulation in tensor memory: 12 tcgen05.mma of K = 16 issued by one thread.
//
// Thread (line, l) owns TMEM lane (line, l) in stage a and writes its vector as a K-major row of A.
// After stage a the same thread holds column l of the line's 32 x 32 matrix; it writes it as an
// MN-major operand, so the transpose between the stages costs nothing.  After stage b thread
// (line, l') holds elements l' + 32 h' for all h': the same thread <-> element map as the input, so
// transforms chain without any exchange.  All waits on the MMAs are bounded: on a timeout the kernel
// sets the plan's error word, stops taking tiles, frees its tensor memory and returns.
#include <type_traits>

#include "ts_device.cuh"
#include "ts_internal.h"
#include "ts_prop_decl.h"
#include "ts_tc.cuh"

namespace ts {

namespace {

constexpr int kTN = 1024;
constexpr int kPart = 16384;          // one 128 x 64 BF16 operand part (hi or lo)
constexpr int kGroupA = 2 * kPart;    // hi + lo of one 128-vector group
constexpr int kBPart = 8192;          // one 64 x 64 BF16 DFT-matrix part
constexpr int kBBytes = 2 * kBPart;   // hi, lo of the forward 32-point DFT
constexpr int kTwBytes = 31 * 32 * 8; // exp(-2 pi i q l / 1024), [q - 1][l], q = 1..31
constexpr int kKRow = 1024;           // K-major: bytes between core matrices adjacent along M / N
constexpr int kMnK = 2048;            // MN-major: bytes between groups of 8 columns k
constexpr int kRowPerSm = 4;          // resident row-pass CTAs per SM (4 warps each)
constexpr int kColPerSm = 2;          // resident column-pass CTAs per SM, two groups (8 warps each)
constexpr int kColPerSm1 = 4;         // resident column-pass CTAs per SM, one group (4 warps each)

// Shared memory layout (bytes): A operands of G groups, the split DFT matrix, twiddles, mbarrier
// and TMEM address slot.  Only the forward DFT matrix is kept: an inverse transform is
// conj(F conj(x)).  The cos / sin values the tables are built from live in the A area until the
// first operand is written.
template <int G>
struct TcLayout {
    static constexpr int A = 0;
    static constexpr int B = G * kGroupA;
    static constexpr int TW = B + kBBytes;
    static constexpr int BAR = TW + kTwBytes;
    static constexpr int SIZE = BAR + 16;
};

struct TcRun {
    int B;             // fields in this launch
    int tiles;         // B * tiles per field
    long long budget;  // clock64 cycles a wait may take
    int* err;          // plan error word (nonzero after a timeout)
};

struct TcCtx {
    unsigned char* sm;
    uint64_t* bar;
    uint32_t tbase;
    uint32_t phase;
    long long budget;
    int* err;
};

// ---- tables staged per CTA: the split forward 32-point DFT matrix and the 1024-point twiddles ----
template <int NT, int BOFF, int TWOFF>
__device__ __forceinline__ void tc_build_tables(unsigned char* sm)
{
    float2* cs = reinterpret_cast<float2*>(sm);  // scratch in the A area
    if (threadIdx.x < 32) {
        float s, c;
        sincospif((float)threadIdx.x / 16.0f, &s, &c);  // exact arguments e / 16, e = 0..31
        cs[threadIdx.x] = make_float2(c, s);
    }
    float2* tw = reinterpret_cast<float2*>(sm + TWOFF);
    for (int i = threadIdx.x; i < 31 * 32; i += NT) {
        const int q = (i >> 5) + 1, l = i & 31;
        float s, c;
        sincospif((float)(q * l) / 512.0f, &s, &c);
        tw[i] = make_float2(c, -s);
    }
    __syncthreads();
    // real form of the 32-point DFT with exponent sign -1, entry (input kk, output n):
    // kk, n < 32 are real parts, >= 32 imaginary parts; stored K-major (row n, column kk)
    for (int task = threadIdx.x; task < 64 * 8; task += NT) {
        const int n = task >> 3, kc = task & 7;
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float g2[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int kk = 8 * kc + 2 * i + u;
                const float2 e = cs[((kk & 31) * (n & 31)) & 31];
                const bool im_in = kk >= 32, im_out = n >= 32;
                g2[u] = (im_in == im_out) ? e.x : (im_out ? -e.y : e.y);
            }
            tc::split_bf16x2(g2[0], g2[1], hi[i], lo[i]);
        }
        const uint32_t off = (uint32_t)((n >> 3) * kKRow + kc * 128 + (n & 7) * 16);
        *reinterpret_cast<uint4*>(sm + BOFF + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(sm + BOFF + kBPart + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
}

__device__ __forceinline__ void conj32(float2 (&v)[32])
{
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i].y = -v[i].y;
}

// ---- operand staging ----
// K-major row m of group g: columns 0..31 = Re v[0..31], 32..63 = Im v[0..31]
__device__ __forceinline__ void write_kmajor(unsigned char* A, int g, int m, const float2 (&v)[32])
{
    unsigned char* hi = A + g * kGroupA + (m >> 3) * kKRow + (m & 7) * 16;
    unsigned char* lo = hi + kPart;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 a = v[8 * (c & 3) + 2 * i], b = v[8 * (c & 3) + 2 * i + 1];
            if (c < 4) tc::split_bf16x2(a.x, b.x, h[i], l[i]);
            else tc::split_bf16x2(a.y, b.y, h[i], l[i]);
        }
        *reinterpret_cast<uint4*>(hi + c * 128) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(lo + c * 128) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// MN-major: v[q] becomes row 32 L + q, column k (Re) and 32 + k (Im) of group g
__device__ __forceinline__ void write_mnmajor(unsigned char* A, int g, int L, int k, const float2 (&v)[32])
{
#pragma unroll
    for (int part = 0; part < 2; ++part) {
        const int kk = k + 32 * part;
        unsigned char* hi = A + g * kGroupA + (kk >> 3) * kMnK + (kk & 7) * 16 + 4 * L * 128;
        unsigned char* lo = hi + kPart;
#pragma unroll
        for (int q8 = 0; q8 < 4; ++q8) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 a = v[8 * q8 + 2 * i], b = v[8 * q8 + 2 * i + 1];
                if (part == 0) tc::split_bf16x2(a.x, b.x, h[i], l[i]);
                else tc::split_bf16x2(a.y, b.y, h[i], l[i]);
            }
            *reinterpret_cast<uint4*>(hi + q8 * 128) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4*>(lo + q8 * 128) = make_uint4(l[0], l[1], l[2], l[3]);
        }
    }
}

// ---- one stage: all G groups, 12 MMAs each (forward 32-point DFTs), then a bounded wait ----
template <int G, int BOFF>
__device__ __forceinline__ bool tc_stage(TcCtx& cx, bool mn)
{
    tc::fence_proxy_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (threadIdx.x == 0) {
        const uint32_t a0 = tc::smem_u32(cx.sm), b0 = tc::smem_u32(cx.sm + BOFF);
        const uint32_t idesc = tc::idesc_bf16_f32(128, 64) | (mn ? tc::kIdescTransposeA : 0u);
#pragma unroll
        for (int g = 0; g < G; ++g) {
#pragma unroll
            for (int kk = 0; kk < 12; ++kk) {
                const int s = kk >> 2, c = kk & 3;  // slices hi.hi, hi.lo, lo.hi; 16 columns c
                const uint32_t ap = a0 + (uint32_t)(g * kGroupA + (s == 2 ? kPart : 0));
                const uint32_t bp = b0 + (s == 1 ? (uint32_t)kBPart : 0u);
                const uint64_t ad = mn ? tc::smem_desc_mn(ap + c * 2 * kMnK, kMnK, 128)
                                       : tc::smem_desc(ap + c * 256, 128, kKRow);
                const uint64_t bd = tc::smem_desc(bp + c * 256, 128, kKRow);
                tc::mma_bf16(cx.tbase + 64 * g, ad, bd, idesc, kk > 0 ? 1u : 0u);
            }
        }
        tc::mma_commit(cx.bar);
    }
    bool ok = tc::mbar_wait_bounded(cx.bar, cx.phase, cx.budget);
    ok = __syncthreads_and(ok) != 0;
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(cx.err, 1);
        tc::mbar_wait_bounded(cx.bar, cx.phase, cx.budget);  // one more budget before TMEM is freed
    }
    cx.phase ^= 1u;
    tc::fence_after_sync();
    return ok;
}

// TMEM lane of this thread, columns 64 g .. 64 g + 63 -> v (Re in 0..31, Im in 32..63)
__device__ __forceinline__ void tc_read(const TcCtx& cx, int g, float2 (&v)[32])
{
    const uint32_t addr = cx.tbase + ((uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16) + 64u * g;
    tc::tmem_ld32_wait(addr, v, 0);
    tc::tmem_ld32_wait(addr + 32, v, 1);
}

// twiddle of stage a (forward transform): v[q] *= exp(-2 pi i l q / 1024)
__device__ __forceinline__ void tc_twiddle(const float2* tw, int l, float2 (&v)[32])
{
#pragma unroll
    for (int q = 1; q < 32; ++q) v[q] = cmul(v[q], tw[(q - 1) * 32 + l]);
}

// ---- row pass: 4 rows per tile (one warp per row, lane l holds elements l + 32 i) ----
template <int FLAGS>
__global__ void __launch_bounds__(128, kRowPerSm) tc_row_kernel(const RowParams a, const TcRun run)
{
    using Lay = TcLayout<1>;
    extern __shared__ __align__(1024) unsigned char sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    TcCtx cx{sm, reinterpret_cast<uint64_t*>(sm + Lay::BAR), 0u, 0u, run.budget, run.err};
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + Lay::BAR + 8);
    constexpr bool kTransforms = (FLAGS & (RP_IN_FREQ | RP_OUT_FREQ)) != 0;
    if (kTransforms) {
        if (warp == 0) {
            tc::tmem_alloc(tslot, 64);
            tc::tmem_relinquish();
        }
        if (threadIdx.x == 0) {
            tc::mbar_init(cx.bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        tc_build_tables<128, Lay::B, Lay::TW>(sm);
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        cx.tbase = *tslot;
    }
    const float2* tw = reinterpret_cast<const float2*>(sm + Lay::TW);
    bool ok = true;
    for (int tile = blockIdx.x; tile < run.tiles && ok; tile += gridDim.x) {
        const int b = tile >> 8, j = ((tile & 255) << 2) + warp;
        float2* row = a.field + ((size_t)b * kTN + j) * kTN;
        float2 v[32];
        if constexpr (FLAGS & RP_IN_SOURCE) {
            const float coef = a.src_coef[(b + a.src_off) % a.n_src];
            const float y = (float)(j - kTN / 2);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float x = (float)(lane + 32 * i - kTN / 2);
                v[i] = coef < 0.0f ? make_float2(1.0f, 0.0f) : make_float2(expf(-(x * x + y * y) * coef), 0.0f);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = row[lane + 32 * i];
        }
        if constexpr (FLAGS & RP_IN_FREQ) {  // inverse transform: conj(F conj(v))
            conj32(v);
            write_kmajor(sm, 0, threadIdx.x, v);
            if (!(ok = tc_stage<1, Lay::B>(cx, false))) break;
            tc_read(cx, 0, v);
            tc_twiddle(tw, lane, v);
            write_mnmajor(sm, 0, warp, lane, v);
            if (!(ok = tc_stage<1, Lay::B>(cx, true))) break;
            tc_read(cx, 0, v);
            conj32(v);
        }
        if constexpr (FLAGS & RP_PHASOR) {
            const float2* ph = a.phasor + (long long)((b + a.phi_off) / a.phi_group) * a.phi_set_stride + (size_t)j * kTN;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float2 e = __ldg(ph + lane + 32 * i);
                v[i] = a.phase_sign > 0.0f ? cmul(v[i], e) : cmulc(v[i], e);
            }
        } else if constexpr (FLAGS & RP_PHASE) {
            if (a.phi != nullptr) {
                const float* ph = a.phi + (long long)((b + a.phi_off) / a.phi_group) * a.phi_set_stride + (size_t)j * kTN;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float2 e = expi_phase(__ldg(ph + lane + 32 * i));
                    v[i] = cmul(v[i], make_float2(e.x, a.phase_sign * e.y));
                }
            }
        }
        if constexpr (FLAGS & RP_INTENSITY) {
            float s0 = 0.0f, s1 = 0.0f;
            const float y = (float)(j - kTN / 2);
            float* irow = a.intensity + ((size_t)b * kTN + j) * kTN;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float I = v[i].x * v[i].x + v[i].y * v[i].y;
                const float x = (float)(lane + 32 * i - kTN / 2);
                irow[lane + 32 * i] = I;
                s0 += I;
                s1 = fmaf(x * x + y * y, I, s1);
            }
            if (a.rows != nullptr) {
                double d0 = s0, d1 = s1;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    d0 += __shfl_down_sync(0xffffffffu, d0, off);
                    d1 += __shfl_down_sync(0xffffffffu, d1, off);
                }
                if (lane == 0) {
                    double* dst = a.rows + ((size_t)b * kTN + j) * 2;
                    dst[0] = d0;
                    dst[1] = d1;
                }
            }
        }
        if constexpr (FLAGS & RP_OUT_FREQ) {
            write_kmajor(sm, 0, threadIdx.x, v);
            if (!(ok = tc_stage<1, Lay::B>(cx, false))) break;
            tc_read(cx, 0, v);
            tc_twiddle(tw, lane, v);
            write_mnmajor(sm, 0, warp, lane, v);
            if (!(ok = tc_stage<1, Lay::B>(cx, true))) break;
            tc_read(cx, 0, v);
        }
        if constexpr (FLAGS & RP_STORE) {
#pragma unroll
            for (int i = 0; i < 32; ++i) row[lane + 32 * i] = v[i];
        }
    }
    if (kTransforms) {
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) tc::tmem_dealloc(cx.tbase, 64);
    }
}

// ---- column pass: W = 4 G columns per tile, G 128-vector groups ----
// Load map (coalesced, 8 W bytes per row): thread t holds rows 32 h + t / W of column t % W.
// After the forward transform thread t holds column t >> 5, frequencies (t & 31) + 32 k2; after
// the inverse transform column t >> 5, rows (t & 31) + 32 j1, stored through a swizzled staging
// tile in shared memory so that the global stores are coalesced again (both staging patterns run
// at the 2-wavefront minimum).
template <int W>
__device__ __forceinline__ uint32_t stage_off(int r, int c)
{
    if constexpr (W == 8) return (uint32_t)(r * 64 + ((c ^ ((r ^ (r >> 3)) & 7)) * 8));
    else return (uint32_t)(r * 32 + ((c ^ ((r >> 2) & 3)) * 8));
}

template <int G>
constexpr int tc_col_per_sm() { return G == 1 ? kColPerSm1 : kColPerSm; }

template <int G, bool CONJ, bool SEP>
__global__ void __launch_bounds__(128 * G, tc_col_per_sm<G>()) tc_col_kernel(const ColParams a, const TcRun run)
{
    using Lay = TcLayout<G>;
    constexpr int W = 4 * G, NT = 128 * G;
    extern __shared__ __align__(1024) unsigned char sm[];
    const int t = threadIdx.x, warp = t >> 5;
    TcCtx cx{sm, reinterpret_cast<uint64_t*>(sm + Lay::BAR), 0u, 0u, run.budget, run.err};
    uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + Lay::BAR + 8);
    if (warp == 0) {
        tc::tmem_alloc(tslot, 64 * G);
        tc::tmem_relinquish();
    }
    if (t == 0) {
        tc::mbar_init(cx.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_build_tables<NT, Lay::B, Lay::TW>(sm);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    cx.tbase = *tslot;
    const float2* tw = reinterpret_cast<const float2*>(sm + Lay::TW);
    const int g = t >> 7, m = t & 127;
    bool ok = true;
    for (int tile = blockIdx.x; tile < run.tiles && ok; tile += gridDim.x) {
        const int b = tile / (kTN / W), col0 = (tile % (kTN / W)) * W;
        float2* base = a.field + (size_t)b * kTN * kTN + col0;
        float2 v[32];
        {
            const int l = t / W, c = t % W;
#pragma unroll
            for (int h = 0; h < 32; ++h) v[h] = base[(size_t)(32 * h + l) * kTN + c];
            // forward transform along the column
            write_kmajor(sm, g, m, v);
            if (!(ok = tc_stage<G, Lay::B>(cx, false))) break;
            tc_read(cx, g, v);
            tc_twiddle(tw, l, v);
            write_mnmajor(sm, c >> 2, c & 3, l, v);
            if (!(ok = tc_stage<G, Lay::B>(cx, true))) break;
            tc_read(cx, g, v);
        }
        // thread t: column col0 + (t >> 5), frequency (t & 31) + 32 i
        const int col = col0 + warp, k1 = t & 31;
        const float kx = a.dk * (float)kidx(col, kTN);
        const float2 px = __ldg(a.P + col);
        if constexpr (SEP) {
            const float cxx = a.ccross * kx * kx;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int mm = k1 + 32 * i;
                const float ky = a.dk * (float)kidx(mm, kTN);
                float2 h = cmul(px, __ldg(a.P + mm));
                const float e = cxx * ky * ky, e2 = e * e;
                h = cmul(h, make_float2(1.0f - e2 * (0.5f - e2 * (1.0f / 24.0f)), -e * (1.0f - e2 * (1.0f / 6.0f))));
                v[i] = CONJ ? cmulc(v[i], h) : cmul(v[i], h);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int mm = k1 + 32 * i;
                const float ky = a.dk * (float)kidx(mm, kTN);
                const float k2 = fmaf(kx, kx, ky * ky);
                const float q = k2 * a.inv_k2;
                float2 h = make_float2(0.0f, 0.0f);
                if (q < 1.0f) {
                    const float d = 1.0f + sqrtf(1.0f - q);
                    const float del = __fdividef(a.dcoef * k2 * k2, d * d);
                    const float d2 = del * del;
                    const float cd = 1.0f - d2 * (0.5f - d2 * (1.0f / 24.0f - d2 * (1.0f / 720.0f)));
                    const float sd = del * (1.0f - d2 * (1.0f / 6.0f - d2 * (1.0f / 120.0f - d2 * (1.0f / 5040.0f))));
                    h = cmul(cmul(px, __ldg(a.P + mm)), make_float2(cd, -sd));
                }
                v[i] = CONJ ? cmulc(v[i], h) : cmul(v[i], h);
            }
        }
        // inverse transform conj(F conj(v)): thread t's vector is (column t >> 5, k1 = t & 31) in
        // group g, lane m
        conj32(v);
        write_kmajor(sm, g, m, v);
        if (!(ok = tc_stage<G, Lay::B>(cx, false))) break;
        tc_read(cx, g, v);
        tc_twiddle(tw, k1, v);
        write_mnmajor(sm, warp >> 2, warp & 3, k1, v);
        if (!(ok = tc_stage<G, Lay::B>(cx, true))) break;
        tc_read(cx, g, v);
        conj32(v);
        // v[j1] = row k1 + 32 j1 of column col: stage through the (now free) operand area
#pragma unroll
        for (int j1 = 0; j1 < 32; ++j1)
            *reinterpret_cast<float2*>(sm + stage_off<W>(k1 + 32 * j1, warp)) = v[j1];
        __syncthreads();
#pragma unroll 4
        for (int idx = t; idx < kTN * W; idx += NT) {
            const int r = idx / W, c = idx % W;
            base[(size_t)r * kTN + c] = *reinterpret_cast<const float2*>(sm + stage_off<W>(r, c));
        }
        // the next tile's operand writes reuse the staging area
        __syncthreads();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(cx.tbase, 64 * G);
}

static_assert(kColPerSm * (TcLayout<2>::SIZE + 1024) <= 228 * 1024, "column-pass CTAs per SM (two groups)");
static_assert(kColPerSm1 * (TcLayout<1>::SIZE + 1024) <= 228 * 1024, "column-pass CTAs per SM (one group)");
static_assert(kRowPerSm * (TcLayout<1>::SIZE + 1024) <= 228 * 1024, "row-pass CTAs per SM");
static_assert(kColPerSm * 128 + kRowPerSm * 64 <= 512, "TMEM columns of co-resident CTAs");
static_assert(kTN * 8 * 8 <= 2 * kGroupA && kTN * 4 * 8 <= kGroupA, "staging tile inside the operand area");

// persistent grid: the CTAs that are resident at once (per SM: the launch bounds' minimum, which the
// register allocation and the shared-memory static_asserts above guarantee), at most one per tile
int tc_grid(int per_sm, int tiles)
{
    static int sms = 0;
    if (sms == 0) {
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        sms = n > 0 ? n : 1;
    }
    const int g = per_sm * sms;
    return tiles < g ? tiles : g;
}

template <int FLAGS>
cudaError_t tc_row_launch(const RowParams& rp, const TcRun& run, cudaStream_t st)
{
    constexpr int smem = TcLayout<1>::SIZE;
    const int grid = tc_grid(kRowPerSm, run.tiles);
    tc_row_kernel<FLAGS><<<grid, 128, smem, st>>>(rp, run);
    return cudaGetLastError();
}

template <int G, bool CONJ, bool SEP>
cudaError_t tc_col_launch(const ColParams& cp, int B, const TcRun& base, cudaStream_t st)
{
    constexpr int smem = TcLayout<G>::SIZE;
    TcRun run = base;
    run.tiles = B * (kTN / (4 * G));
    const int grid = tc_grid(tc_col_per_sm<G>(), run.tiles);
    tc_col_kernel<G, CONJ, SEP><<<grid, 128 * G, smem, st>>>(cp, run);
    return cudaGetLastError();
}

template <int FLAGS>
cudaError_t tc_row_attr()
{
    cudaError_t e = cudaFuncSetAttribute(tc_row_kernel<FLAGS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TcLayout<1>::SIZE);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_row_kernel<FLAGS>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

template <int G, bool CONJ, bool SEP>
cudaError_t tc_col_attr()
{
    cudaError_t e = cudaFuncSetAttribute(tc_col_kernel<G, CONJ, SEP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TcLayout<G>::SIZE);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_col_kernel<G, CONJ, SEP>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

#define TS_TC_ROW_FLAGS(X)                                        \
    X(RP_IN_SOURCE | RP_STORE)                                    \
    X(RP_IN_SOURCE | RP_OUT_FREQ | RP_STORE)                      \
    X(RP_OUT_FREQ | RP_STORE)                                     \
    X(RP_PHASE | RP_OUT_FREQ | RP_STORE)                          \
    X(RP_IN_FREQ | RP_PHASE | RP_OUT_FREQ | RP_STORE)             \
    X(RP_IN_FREQ | RP_PHASE | RP_STORE)                           \
    X(RP_IN_FREQ | RP_PHASE | RP_INTENSITY | RP_STORE)            \
    X(RP_IN_FREQ | RP_PHASE | RP_INTENSITY)                       \
    X(RP_IN_FREQ | RP_STORE)                                      \
    X(RP_PHASOR | RP_OUT_FREQ | RP_STORE)                         \
    X(RP_IN_FREQ | RP_PHASOR | RP_OUT_FREQ | RP_STORE)            \
    X(RP_IN_FREQ | RP_PHASOR | RP_STORE)                          \
    X(RP_IN_FREQ | RP_PHASOR | RP_INTENSITY | RP_STORE)           \
    X(RP_IN_FREQ | RP_PHASOR | RP_INTENSITY)

}  // namespace

cudaError_t tc_row_pass(int flags, const RowParams& rp, int B, long long budget, int* err, cudaStream_t st)
{
    const TcRun run{B, B * (kTN / 4), budget, err};
    switch (flags) {
#define TS_TC_CASE(F) \
    case F: return tc_row_launch<F>(rp, run, st);
        TS_TC_ROW_FLAGS(TS_TC_CASE)
#undef TS_TC_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t tc_col_pass(int groups, bool conj, bool sep, const ColParams& cp, int B, long long budget, int* err,
                        cudaStream_t st)
{
    const TcRun run{B, 0, budget, err};
#define TS_TC_COLG(G)                                                                                              \
    if (sep) return conj ? tc_col_launch<G, true, true>(cp, B, run, st) : tc_col_launch<G, false, true>(cp, B, run, st); \
    return conj ? tc_col_launch<G, true, false>(cp, B, run, st) : tc_col_launch<G, false, false>(cp, B, run, st);
    if (groups == 2) {
        TS_TC_COLG(2)
    }
    TS_TC_COLG(1)
#undef TS_TC_COLG
}

cudaError_t prepare_tc_prop()
{
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
#define TS_TC_ATTR(F) chk(tc_row_attr<F>());
    TS_TC_ROW_FLAGS(TS_TC_ATTR)
#undef TS_TC_ATTR
    chk(tc_col_attr<1, false, false>());
    chk(tc_col_attr<1, true, false>());
    chk(tc_col_attr<1, false, true>());
    chk(tc_col_attr<1, true, true>());
    chk(tc_col_attr<2, false, false>());
    chk(tc_col_attr<2, true, false>());
    chk(tc_col_attr<2, false, true>());
    chk(tc_col_attr<2, true, true>());
    return e;
}

}  // namespace ts
