// ts_prop_tma.cu -- persistent propagation passes for N = 512 and 1024 that prefetch their next input
// with the Tensor Memory Accelerator while the current one is transformed (Eq. 1: column pass
// FFT -> H -> IFFT, row pass IFFT -> exp(i phi) -> FFT).  32 points per thread, T = N / 32 threads per
// line.
//
// Column pass: a CTA of T W threads owns W-column tiles of 64 KiB (N = 1024: W = 8, or W = 4 with
// 32 KiB tiles; N = 512: W = 16).  The tile comes in by 2-D tensor copies (boxes of 256 rows x 2W
// floats) into the CTA's exchange buffer and goes out the same way: after the last FFT stage the
// threads write tile k into the buffer in its global layout, one thread issues the tensor stores of
// its boxes, and box q of tile k+1 is loaded into the buffer as soon as the store of box q has read
// it.  The stores leave the threads at once (no per-thread global stores to drain); the load of the
// next tile is covered by the other CTA on the SM.  Thread (t, c) = (tid / W, tid % W) holds points
// t + T i of column c.
//
// Row pass: every warp owns 32 / T consecutive rows at a time (one at N = 1024, two at 512) and its
// own 8 KiB of line buffers, with its own mbarrier: the phasor rows of the step are bulk-copied into
// the lines while the second stage of the inverse FFT runs, and the warp's next field rows while the
// second stage of the forward FFT runs.  Warps never wait for one another after the twiddles are
// staged.
//
// Every wait on an mbarrier is bounded by the plan's clock64 budget; a wait that runs out sets the
// plan's error word (read by ts_plan_device_status) and the CTA (column pass) or warp (row pass)
// returns after a second bounded wait for its copy in flight.
#include <cuda.h>

#include <algorithm>

#include "ts_async.cuh"
#include "ts_device.cuh"
#include "ts_prop_decl.h"

namespace ts {
namespace {

using namespace async;
constexpr int kErrTmaWait = 4;  // error word value: a prefetch wait ran out of its budget

// Stage 0 of a 1024-point line FFT (32 x 32, thread t holds points t + 32 i) with its exchange in
// 16-byte stores: thread t's 32 stage outputs land at line[34 t + r] (two float2 of padding per 32
// points, so pairs r, r + 1 are 16-byte aligned) and come back as line[t + 34 i].  With the line
// strides the passes choose, stores and loads run at their wavefront minimum (4 and 2 per warp).
template <int SIGN, class Bar>
__device__ __forceinline__ void stage0_exchange_x4(float2 (&v)[32], float2* line, int t, Bar bar)
{
    Dft<32, SIGN>::run(v);
    float4* w = reinterpret_cast<float4*>(line + 34 * t);
#pragma unroll
    for (int r = 0; r < 32; r += 2) w[r / 2] = make_float4(v[r].x, v[r].y, v[r + 1].x, v[r + 1].y);
    bar();
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = line[t + 34 * i];
    bar();
}

// ---------------------------------------------------------------------------------------------
// column pass
// ---------------------------------------------------------------------------------------------
// W columns per CTA (T W threads): N = 1024, W = 8, two CTAs per SM, the (P, ky^2) table as float4;
// or W = 4, four CTAs per SM (block barriers span 4 warps instead of 8), the table split into P
// (float2) and ky^2 (float) so that four CTAs fit the SM's shared memory; N = 512, W = 16, two per SM,
// or W = 8, four per SM (split table).  At N = 512 the line stride is the padded line (528 float2)
// plus 16 / W (529 for W = 16, 530 for W = 8), which keeps the exchanges and the tile accesses of a
// warp at the 2-wavefront minimum for 8-byte accesses.
template <int N_, int W_>
struct ColTma {
    static constexpr int N = N_, W = W_;
    using C = FftCfg<N, 32, true, true>;  // T = N / 32 threads per column, 32 points each
    static constexpr int T = C::T, THREADS = T * W, PER_SM = 512 / THREADS, BOX_ROWS = 256;
    static constexpr bool SPLIT = PER_SM > 2;
    static constexpr int TPF = N / W;                        // tiles per field
    // column stride of the exchange buffer (float2).  N = 1024 uses the 16-byte exchange: LS >= 1086,
    // and LS / 2 odd (8 columns) or = 2 mod 8 (4 columns) keeps both its 16-byte stores and its 8-byte
    // loads at the minimum number of shared-memory wavefronts
    static constexpr int LS = N == 1024 ? (W == 4 ? 1092 : 1086) : C::padded + (16 / W > 1 ? 16 / W : 1);
    static constexpr int TILE_BYTES = W * N * 8;
    static constexpr size_t off_ht = sizeof(float2) * C::tw_smem;
    static constexpr size_t ht_bytes = SPLIT ? (sizeof(float2) + sizeof(float)) * N : sizeof(float4) * N;
    static constexpr size_t off_buf = off_ht + ht_bytes;
    static constexpr size_t off_bar = off_buf + sizeof(float2) * W * LS;
    static constexpr size_t smem = off_bar + 16;
    static_assert(W * LS >= W * N, "the dense tile fits the exchange buffer");
    static_assert(off_buf % 128 == 0, "TMA destination alignment");
    static_assert(N % BOX_ROWS == 0 && (2 * W * 4) % 16 == 0, "whole boxes, 16-byte box rows");
    static_assert(PER_SM * (smem + 1024) <= 228 * 1024, "resident CTAs fit the SM's shared memory");
};

template <bool CONJ, int HMODE, class CT, bool SRC = false>
__global__ void __launch_bounds__(CT::THREADS, CT::PER_SM)
    col_pass_tma_kernel(const ColParams a, const __grid_constant__ CUtensorMap tmap, int B)
{
    using C = typename CT::C;
    constexpr int N = CT::N, W = CT::W, T = CT::T, TPF = CT::TPF;
    extern __shared__ __align__(128) unsigned char sm[];
    float2* tw = reinterpret_cast<float2*>(sm);
    float4* ht = reinterpret_cast<float4*>(sm + CT::off_ht);  // float4 table
    float2* hp = reinterpret_cast<float2*>(sm + CT::off_ht);  // split table: P, then ky^2
    float* hk = reinterpret_cast<float*>(sm + CT::off_ht + sizeof(float2) * N);
    float2* buf = reinterpret_cast<float2*>(sm + CT::off_buf);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + CT::off_bar);
    const int tid = threadIdx.x, c = tid % W, t = tid / W;
    const int tiles = B * TPF;
    int tile = blockIdx.x;
    if (tile >= tiles) return;  // uniform over the CTA
    auto issue = [&](int tl) {  // one thread: the boxes of tile tl
        const int b = tl / TPF, x = 2 * (tl % TPF) * W;
        mbar_expect_tx(bar, CT::TILE_BYTES);
#pragma unroll
        for (int q = 0; q < N / CT::BOX_ROWS; ++q)
            tma_load_2d(buf + q * CT::BOX_ROWS * W, &tmap, x, b * N + q * CT::BOX_ROWS, bar);
    };
    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
        if (!SRC && !a.stall) issue(tile);
    }
    stage_twiddles_c<C>(tw, a.tw);
    for (int i = tid; i < N; i += CT::THREADS) {
        const float2 p = __ldg(a.P + i);
        const float k = a.dk * (float)kidx(i, N);
        if constexpr (CT::SPLIT) {
            hp[i] = p;
            hk[i] = k * k;
        } else {
            ht[i] = make_float4(p.x, p.y, k * k, 0.0f);
        }
    }
    __syncthreads();
    uint32_t parity = 0;
    for (; tile < tiles; tile += gridDim.x, parity ^= 1u) {
        const int b = tile / TPF, col = (tile % TPF) * W + c;
        float2 v[32];
        if constexpr (SRC) {
            // the previous tile's bulk store has read the buffer (thread 0 waited) before it is reused
            __syncthreads();
            // the source's row transform: a rank-one product, no input to load
            const int s = (b + a.src_off) % a.n_src;
            const float2 fx = __ldg(a.src_fx + (size_t)s * N + col);
            const float* gy = a.src_gy + (size_t)s * N;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const float g = __ldg(gy + t + T * i);
                v[i] = make_float2(fx.x * g, fx.y * g);
            }
        } else {
            const bool ok = mbar_wait(bar, parity, a.budget);
            if (ok) {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = buf[(t + T * i) * W + c];
            }
            if (__syncthreads_or(!ok)) {  // every thread has read the tile before the exchange reuses it
                if (tid == 0) {
                    bulk_wait_all();
                    atomicExch(a.err, kErrTmaWait);
                    mbar_wait(bar, parity, a.budget);  // the copy in flight, bounded again
                }
                return;
            }
        }
        float2* line = buf + c * CT::LS;
        if constexpr (N == 1024)
            stage0_exchange_x4<-1>(v, line, t, BlockBar());
        else
            fft_stage_c<C, 0, -1>(v, line, t, tw, BlockBar());
        fft_stage_c<C, 1, -1>(v, line, t, tw, BlockBar());
        if constexpr (CT::SPLIT) {
            auto tab = [hp, hk](int m) {
                const float2 q = hp[m];
                return make_float4(q.x, q.y, hk[m], 0.0f);
            };
            transfer_tile_tab<CONJ, HMODE, decltype(tab), T>(v, tab, col, t, a.ccross, a.dcoef, a.inv_k2);
        } else {
            auto tab = [ht](int m) { return ht[m]; };
            transfer_tile_tab<CONJ, HMODE, decltype(tab), T>(v, tab, col, t, a.ccross, a.dcoef, a.inv_k2);
        }
        // stage 0 of the inverse: ends with a barrier after the last read
        if constexpr (N == 1024)
            stage0_exchange_x4<+1>(v, line, t, BlockBar());
        else
            fft_stage_c<C, 0, +1>(v, line, t, tw, BlockBar());
        fft_stage_c<C, 1, +1>(v, line, t, tw, BlockBar());
        // the tile goes out through the buffer by tensor stores; the next tile comes in once they
        // have read it
#pragma unroll
        for (int i = 0; i < 32; ++i) buf[(t + T * i) * W + c] = v[i];
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            constexpr int Q = N / CT::BOX_ROWS;
            static_assert(Q == 4 || Q == 2, "quarter or half boxes");
            const int x = 2 * (tile % TPF) * W;
#pragma unroll
            for (int q = 0; q < Q; ++q) {  // one bulk group per box
                tma_store_2d(&tmap, buf + q * CT::BOX_ROWS * W, x, b * N + q * CT::BOX_ROWS);
                bulk_commit();
            }
            if (!SRC && tile + (int)gridDim.x < tiles) {
                // box q of the next tile comes in as soon as the store of box q has read it
                const int tn = tile + gridDim.x, bn = tn / TPF, xn = 2 * (tn % TPF) * W;
                mbar_expect_tx(bar, CT::TILE_BYTES);
                auto load_box = [&](int q) { tma_load_2d(buf + q * CT::BOX_ROWS * W, &tmap, xn, bn * N + q * CT::BOX_ROWS, bar); };
                if constexpr (Q == 4) {
                    bulk_wait_read<3>();
                    load_box(0);
                    bulk_wait_read<2>();
                    load_box(1);
                    bulk_wait_read<1>();
                    load_box(2);
                    bulk_wait_read<0>();
                    load_box(3);
                } else {
                    bulk_wait_read<1>();
                    load_box(0);
                    bulk_wait_read<0>();
                    load_box(1);
                }
            } else {
                bulk_wait_read<0>();
            }
        }
    }
    if (tid == 0) bulk_wait_all();
}

// ---------------------------------------------------------------------------------------------
// row pass
// ---------------------------------------------------------------------------------------------
template <int N_>
struct RowTma {
    static constexpr int N = N_;
    using C = FftCfg<N, 32, true, true>;  // T = N / 32 threads per row, 32 / T rows per warp
    static constexpr int T = C::T, RPW = 32 / T;
    static constexpr int WARPS = 8, THREADS = 32 * WARPS;
    // line stride (float2); a line holds the dense row or the exchange (N = 1024: the 16-byte exchange)
    static constexpr int LS = N == 1024 ? 1086 : C::padded;
    static constexpr int ROW_BYTES = N * 8;
    static constexpr size_t off_line = sizeof(float2) * C::tw_smem;
    static constexpr size_t off_bar = off_line + sizeof(float2) * WARPS * RPW * LS;
    static constexpr size_t smem = off_bar + 8 * WARPS;
    static_assert(T <= 32 && 32 % T == 0, "whole rows per warp");
    static_assert(off_line % 128 == 0 && (sizeof(float2) * LS) % 16 == 0, "bulk-copy destination alignment");
};

template <class RT, int FLAGS>
__global__ void __launch_bounds__(RT::THREADS, 2) row_pass_tma_kernel(const RowParams a, int B)
{
    using C = typename RT::C;
    constexpr int N = RT::N, T = RT::T, RPW = RT::RPW;
    static_assert((FLAGS & RP_IN_FREQ) && (FLAGS & RP_PHASOR) && (FLAGS & RP_STORE) && !(FLAGS & RP_INTENSITY) &&
                      !(FLAGS & RP_IN_SOURCE),
                  "row pass of a step in the row-frequency domain");
    extern __shared__ __align__(128) unsigned char sm[];
    float2* tw = reinterpret_cast<float2*>(sm);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int h = lane / T, t = lane % T;  // this lane's row of the warp's RPW rows, and its thread index in it
    float2* lines = reinterpret_cast<float2*>(sm + RT::off_line) + warp * RPW * RT::LS;
    float2* line = lines + h * RT::LS;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + RT::off_bar) + warp;
    const int units = B * N / RPW;  // groups of RPW consecutive rows (never across fields)
    // units gw, gw + stride, ... of the launch (strided over every warp of the grid)
    const int gw = blockIdx.x * RT::WARPS + warp, stride = gridDim.x * RT::WARPS;
    auto load_rows = [&](int u) {  // lane 0: the RPW field rows of unit u
        mbar_expect_tx(bar, RPW * RT::ROW_BYTES);
#pragma unroll
        for (int k = 0; k < RPW; ++k)
            bulk_load(lines + k * RT::LS, a.field + ((size_t)u * RPW + k) * N, RT::ROW_BYTES, bar);
    };
    if (lane == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
        if (gw < units && !a.stall) load_rows(gw);
    }
    stage_twiddles_c<C>(tw, a.tw);
    __syncthreads();
    uint32_t parity = 0;
    for (int u = gw; u < units; u += stride) {
        const int r0 = u * RPW, b = r0 / N, j0 = r0 % N;
        float2 v[32];
        if (!__all_sync(0xffffffffu, mbar_wait(bar, parity, a.budget))) {
            if (lane == 0) {
                atomicExch(a.err, kErrTmaWait);
                mbar_wait(bar, parity, a.budget);  // the copy in flight, bounded again
            }
            return;
        }
        parity ^= 1u;
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = line[t + T * i];
        __syncwarp();  // every lane has its points before the exchange overwrites the rows
        if constexpr (N == 1024)
            stage0_exchange_x4<+1>(v, line, t, WarpBar());
        else
            fft_stage_c<C, 0, +1>(v, line, t, tw, WarpBar());
        if (lane == 0) {  // the lines are free: the step's screen phasor rows come in under the next stage
            const int set = (b + a.phi_off) / a.phi_group;
            const float2* src = a.phasor + (long long)set * a.phi_set_stride + (size_t)j0 * N;
            fence_proxy_async();
            mbar_expect_tx(bar, RPW * RT::ROW_BYTES);
#pragma unroll
            for (int k = 0; k < RPW; ++k) bulk_load(lines + k * RT::LS, src + (size_t)k * N, RT::ROW_BYTES, bar);
        }
        fft_stage_c<C, 1, +1>(v, line, t, tw, WarpBar());
        if (!__all_sync(0xffffffffu, mbar_wait(bar, parity, a.budget))) {
            if (lane == 0) {
                atomicExch(a.err, kErrTmaWait);
                mbar_wait(bar, parity, a.budget);
            }
            return;
        }
        parity ^= 1u;
        if (a.phase_sign > 0.0f) {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = cmul(v[i], line[t + T * i]);
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = cmulc(v[i], line[t + T * i]);
        }
        __syncwarp();
        if constexpr (FLAGS & RP_OUT_FREQ) {
            if constexpr (N == 1024)
                stage0_exchange_x4<-1>(v, line, t, WarpBar());
            else
                fft_stage_c<C, 0, -1>(v, line, t, tw, WarpBar());
            if (lane == 0 && u + stride < units) {
                fence_proxy_async();
                load_rows(u + stride);
            }
            fft_stage_c<C, 1, -1>(v, line, t, tw, WarpBar());
        } else {
            if (lane == 0 && u + stride < units) {
                fence_proxy_async();
                load_rows(u + stride);
            }
        }
        float2* row = a.field + ((size_t)r0 + h) * N;
#pragma unroll
        for (int i = 0; i < 32; ++i) row[t + T * i] = v[i];
    }
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------

// CTAs of a kernel resident on the current device at once (SMs x CTAs per SM), cached per device in
// `cache` (one slot per device ordinal below kMaxDevices; larger ordinals are queried every time)
constexpr int kMaxDevices = 64;
template <class K>
int max_ctas(K kernel, int threads, size_t smem, int (&cache)[kMaxDevices])
{
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev >= 0 && dev < kMaxDevices && cache[dev] > 0) return cache[dev];
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess) return 0;
    if (dev >= 0 && dev < kMaxDevices) cache[dev] = sms * per;
    return sms * per;
}


template <bool CONJ, int HMODE, class CT, bool SRC = false>
cudaError_t col_launch_tma(const ColParams& cp, int B, cudaStream_t st)
{
    CUtensorMap map;
    cudaError_t e = field_tensor_map(&map, cp.field, CT::N, B, 2 * CT::W, CT::BOX_ROWS);
    if (e != cudaSuccess) return e;
    static int cache[kMaxDevices] = {};
    const int resident = max_ctas(col_pass_tma_kernel<CONJ, HMODE, CT, SRC>, CT::THREADS, CT::smem, cache);
    if (resident <= 0) return cudaErrorInvalidConfiguration;
    // full residency, tiles strided over the CTAs: the CTAs an SM holds share its issue slots, so
    // filling every slot keeps each SM's tile count within one of the mean
    const int grid = std::min(B * CT::TPF, resident);
    col_pass_tma_kernel<CONJ, HMODE, CT, SRC><<<grid, CT::THREADS, CT::smem, st>>>(cp, map, B);
    return cudaGetLastError();
}

template <class CT>
cudaError_t col_dispatch_tma(bool conj, int hmode, const ColParams& cp, int B, cudaStream_t st, bool source)
{
    if (source) {  // forward only: the first column pass of a call that starts from the sources
        if (conj || cp.src_fx == nullptr || cp.src_gy == nullptr || cp.n_src < 1) return cudaErrorNotSupported;
        switch (hmode) {
        case 0: return col_launch_tma<false, 0, CT, true>(cp, B, st);
        case 1: return col_launch_tma<false, 1, CT, true>(cp, B, st);
        case 2: return col_launch_tma<false, 2, CT, true>(cp, B, st);
        case 3: return col_launch_tma<false, 3, CT, true>(cp, B, st);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (hmode * 2 + (conj ? 1 : 0)) {
    case 0: return col_launch_tma<false, 0, CT>(cp, B, st);
    case 1: return col_launch_tma<true, 0, CT>(cp, B, st);
    case 2: return col_launch_tma<false, 1, CT>(cp, B, st);
    case 3: return col_launch_tma<true, 1, CT>(cp, B, st);
    case 4: return col_launch_tma<false, 2, CT>(cp, B, st);
    case 5: return col_launch_tma<true, 2, CT>(cp, B, st);
    case 6: return col_launch_tma<false, 3, CT>(cp, B, st);
    case 7: return col_launch_tma<true, 3, CT>(cp, B, st);
    default: return cudaErrorInvalidValue;
    }
}

template <class RT, int FLAGS>
cudaError_t row_launch_tma(const RowParams& rp, int B, cudaStream_t st)
{
    static int cache[kMaxDevices] = {};
    const int resident = max_ctas(row_pass_tma_kernel<RT, FLAGS>, RT::THREADS, RT::smem, cache);
    if (resident <= 0) return cudaErrorInvalidConfiguration;
    const int units = B * RT::N / RT::RPW;
    const int grid = std::min((units + RT::WARPS - 1) / RT::WARPS, resident);  // full residency
    row_pass_tma_kernel<RT, FLAGS><<<grid, RT::THREADS, RT::smem, st>>>(rp, B);
    return cudaGetLastError();
}

template <class RT>
cudaError_t row_dispatch_tma(int flags, const RowParams& rp, int B, cudaStream_t st)
{
    switch (flags) {
    case RP_IN_FREQ | RP_PHASOR | RP_OUT_FREQ | RP_STORE:
        return row_launch_tma<RT, RP_IN_FREQ | RP_PHASOR | RP_OUT_FREQ | RP_STORE>(rp, B, st);
    case RP_IN_FREQ | RP_PHASOR | RP_STORE: return row_launch_tma<RT, RP_IN_FREQ | RP_PHASOR | RP_STORE>(rp, B, st);
    default: return cudaErrorNotSupported;
    }
}

template <class K>
cudaError_t tma_attr(K kernel, size_t bytes)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

}  // namespace

cudaError_t col_pass_tma(int N, int w, bool conj, int hmode, const ColParams& cp, int B, cudaStream_t st,
                         bool source)
{
    if ((reinterpret_cast<uintptr_t>(cp.field) & 15) != 0 || cp.err == nullptr) return cudaErrorNotSupported;
    if (N == 1024 && w == 8) return col_dispatch_tma<ColTma<1024, 8>>(conj, hmode, cp, B, st, source);
    if (N == 1024 && w == 4) return col_dispatch_tma<ColTma<1024, 4>>(conj, hmode, cp, B, st, source);
    if (N == 512 && w == 16) return col_dispatch_tma<ColTma<512, 16>>(conj, hmode, cp, B, st, source);
    if (N == 512 && w == 8) return col_dispatch_tma<ColTma<512, 8>>(conj, hmode, cp, B, st, source);
    return cudaErrorNotSupported;
}

cudaError_t row_pass_tma(int N, int flags, const RowParams& rp, int B, cudaStream_t st)
{
    if ((reinterpret_cast<uintptr_t>(rp.field) & 15) != 0 || (reinterpret_cast<uintptr_t>(rp.phasor) & 15) != 0 ||
        (rp.phi_set_stride & 1) != 0 || rp.err == nullptr || rp.phasor == nullptr)
        return cudaErrorNotSupported;
    if (N == 1024) return row_dispatch_tma<RowTma<1024>>(flags, rp, B, st);
    if (N == 512) return row_dispatch_tma<RowTma<512>>(flags, rp, B, st);
    return cudaErrorNotSupported;
}

namespace {
template <class CT>
void col_attrs(cudaError_t& e)
{
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    chk(tma_attr(col_pass_tma_kernel<false, 0, CT>, CT::smem));
    chk(tma_attr(col_pass_tma_kernel<true, 0, CT>, CT::smem));
    chk(tma_attr(col_pass_tma_kernel<false, 1, CT>, CT::smem));
    chk(tma_attr(col_pass_tma_kernel<true, 1, CT>, CT::smem));
    chk(tma_attr(col_pass_tma_kernel<false, 2, CT>, CT::smem));
    chk(tma_attr(col_pass_tma_kernel<true, 2, CT>, CT::smem));
    chk(tma_attr(col_pass_tma_kernel<false, 3, CT>, CT::smem));
    chk(tma_attr(col_pass_tma_kernel<true, 3, CT>, CT::smem));
    chk(tma_attr(col_pass_tma_kernel<false, 0, CT, true>, CT::smem));
    chk(tma_attr(col_pass_tma_kernel<false, 1, CT, true>, CT::smem));
    chk(tma_attr(col_pass_tma_kernel<false, 2, CT, true>, CT::smem));
    chk(tma_attr(col_pass_tma_kernel<false, 3, CT, true>, CT::smem));
}
template <class RT>
void row_attrs(cudaError_t& e)
{
    if (e == cudaSuccess) e = tma_attr(row_pass_tma_kernel<RT, RP_IN_FREQ | RP_PHASOR | RP_OUT_FREQ | RP_STORE>, RT::smem);
    if (e == cudaSuccess) e = tma_attr(row_pass_tma_kernel<RT, RP_IN_FREQ | RP_PHASOR | RP_STORE>, RT::smem);
}
}  // namespace

cudaError_t prepare_prop_tma(int N)
{
    cudaError_t e = cudaSuccess;
    if (N == 1024) {
        col_attrs<ColTma<1024, 8>>(e);
        col_attrs<ColTma<1024, 4>>(e);
        row_attrs<RowTma<1024>>(e);
    } else if (N == 512) {
        col_attrs<ColTma<512, 16>>(e);
        col_attrs<ColTma<512, 8>>(e);
        row_attrs<RowTma<512>>(e);
    }
    return e;
}

}  // namespace ts
