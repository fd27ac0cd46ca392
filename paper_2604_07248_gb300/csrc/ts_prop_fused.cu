// ts_prop_fused.cu -- the whole Eq. 1 propagation of a batch of N = 1024 fields (first row pass, then
// S x (column pass, row pass)) as ONE persistent launch.
//
// Work items are (phase, field, tile) in phase-major order: phase 0 = first row pass (source or
// field -> row FFT), phase 2s+1 = column pass of step s (column FFT, x H_s, column IFFT), phase 2s+2 =
// row pass of step s (row IFFT, x exp(i phi_s), row FFT unless s = S-1).  A tile is 8 columns (column
// phases) or 8 rows (row phases) of one field: 128 tiles per field and phase.  CTAs take items from a
// global counter; an item of phase p > 0 needs all 128 tiles of phase p-1 of its own field, and
// since items are handed out in order, every tile it waits for was taken earlier by a running CTA:
// the launch cannot deadlock for any grid size.  While one field's column pass drains, other
// fields' row passes already run, so no per-pass launch tail idles the GPU.
//
// Each CTA knows its next item while it runs the current one and issues the next item's input copies
// (a 64 KiB column tile by four 2-D TMA boxes plus the step's 16 KiB (P, ky^2) table, or one 8 KiB field
// row per warp by bulk copies) as soon as the buffer is free and the next item's dependency is already
// met; otherwise it waits for the dependency (bounded) when it gets there.  Row tiles run their eight
// warps independently: each warp has its own line and mbarrier, fetches its screen phasor row under
// the second stage of the inverse FFT and, when the next item is also a row tile, its next field row
// under the second stage of the forward FFT.  Column tiles synchronise the block at their exchanges.
//
// Completion: a tile's stores, a block barrier, then (during the CTA's next item, once the stores have
// had a stage to drain, or at once before any blocking wait) thread 0 fences and adds 1 to the
// (phase, field) counter; consumers acquire-load the counter and fence the async proxy before their
// copies read the data.  Each CTA also fetches its item indices one item ahead, so no global atomic
// sits between two of its items.  Every wait (dependency, copy) is bounded by the plan's clock64 budget; one that runs out
// sets the error word (read by ts_plan_device_status), after which every CTA stops at its next item.
#include <cuda.h>

#include <algorithm>

#include "ts_async.cuh"
#include "ts_device.cuh"
#include "ts_prop_decl.h"

namespace ts {
namespace {

using namespace async;
constexpr int kN = 1024;
constexpr int kErrDepWait = 5;  // error word: a dependency or copy wait of the fused launch ran out

struct Fused {
    using C = FftCfg<kN, 32>;
    static constexpr int THREADS = 256, WARPS = 8, W = 8, TPF = kN / W;
    static constexpr int LSC = C::padded + 2;  // column stride of the column-tile exchange
    static constexpr int LSR = C::padded;      // line stride of the row-tile lines
    static constexpr int TILE_BYTES = W * kN * 8;
    static constexpr int HT_BYTES = kN * 16;
    static constexpr size_t off_ht = sizeof(float2) * C::tw_smem;
    static constexpr size_t off_buf = off_ht + HT_BYTES;
    static constexpr size_t off_bar = off_buf + sizeof(float2) * W * LSC;
    static constexpr size_t off_int = off_bar + 8 * (1 + WARPS);
    static constexpr size_t smem = off_int + 4 * (2 + WARPS);
    static_assert(W * LSC >= W * kN && W * LSC >= WARPS * LSR, "tile, lines and exchanges fit the buffer");
    static_assert(off_buf % 128 == 0 && off_ht % 128 == 0 && (LSR * 8) % 16 == 0, "copy alignment");
};

// Work-item order: pass-major, then field, then tile, so every item's dependency (the previous pass
// of its field) has a smaller index.  (Interleaving the passes of two field groups, so that column and
// row tiles run side by side, measured 11 % slower at config 3.)
__device__ __forceinline__ void item_decode(int it, int B, int& p, int& b, int& tile)
{
    const int per_phase = B * Fused::TPF;
    p = it / per_phase;
    const int rem = it - p * per_phase;
    b = rem / Fused::TPF;
    tile = rem - b * Fused::TPF;
}

// the input copies of a column tile (thread 0): four 2-D TMA boxes + the step's transfer table
__device__ __forceinline__ void issue_col(const FusedParams& a, const CUtensorMap* map, int p, int b, int tile,
                                          float2* buf, float4* ht, uint64_t* bin)
{
    const int s = (p - 1) >> 1;
    mbar_expect_tx(bin, Fused::TILE_BYTES + Fused::HT_BYTES);
#pragma unroll
    for (int q = 0; q < 4; ++q) tma_load_2d(buf + q * 256 * Fused::W, map, 16 * tile, b * kN + q * 256, bin);
    bulk_load(ht, a.ht + (size_t)s * kN, Fused::HT_BYTES, bin);
}

// the input copy of row `w` of a row tile into warp w's line, on warp w's barrier
__device__ __forceinline__ void issue_row(const FusedParams& a, int b, int tile, int w, float2* buf, uint64_t* bw)
{
    mbar_expect_tx(bw + w, kN * 8);
    bulk_load(buf + w * Fused::LSR, a.field + ((size_t)b * kN + (size_t)tile * Fused::WARPS + w) * kN, kN * 8, bw + w);
}

template <int HMODE>
__global__ void __launch_bounds__(Fused::THREADS, 2) prop_fused_kernel(const FusedParams a,
                                                                       const __grid_constant__ CUtensorMap tmap)
{
    using C = Fused::C;
    extern __shared__ __align__(128) unsigned char sm[];
    float2* tw = reinterpret_cast<float2*>(sm);
    float4* ht = reinterpret_cast<float4*>(sm + Fused::off_ht);
    float2* buf = reinterpret_cast<float2*>(sm + Fused::off_buf);
    uint64_t* bin = reinterpret_cast<uint64_t*>(sm + Fused::off_bar);  // column-tile input
    uint64_t* bw = bin + 1;  // per warp: row input, then the phasor row
    int* s_int = reinterpret_cast<int*>(sm + Fused::off_int);  // [0] first item, [1] next item
    int* row_issued = s_int + 2;  // per warp: the row item whose input row was issued into its line
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int total = (2 * a.S + 1) * a.B * Fused::TPF;
    // thread-0 state: the column item whose tile copy is in flight or has landed; the item after the
    // next one (its fetch is in flight during the current item); the (pass, field) counter of the last
    // finished tile, signalled once its stores have drained (or before any blocking wait)
    int col_issued = -1, fetched = 0, pending = -1;

    if (tid == 0) {
        mbar_init(bin, 1);
        for (int w = 0; w < Fused::WARPS; ++w) mbar_init(bw + w, 1);
        mbar_init_fence();
        s_int[0] = atomicAdd(a.head, 1);
        fetched = atomicAdd(a.head, 1);
    }
    if (tid < Fused::WARPS) row_issued[tid] = -1;
    stage_twiddles_c<C>(tw, a.tw);
    __syncthreads();
    int cur = s_int[0];
    uint32_t pin = 0, pw = 0;  // parities of the column-tile barrier and of this warp's barrier

    auto signal = [&]() {  // thread 0
        if (pending >= 0) {
            __threadfence();
            atomicAdd(a.done + pending, 1);
            pending = -1;
        }
    };
    // whether item `it` needs input copies and its dependency is met now (acquire, no wait)
    auto ready = [&](int it, int& p, int& b, int& tile) {
        if (it >= total || a.stall) return false;
        item_decode(it, a.B, p, b, tile);
        if (p == 0 && a.source) return false;
        return p == 0 || ld_acquire(a.done + (p - 1) * a.B + b) >= Fused::TPF;
    };

    while (cur < total) {
        int p, b, tile;
        item_decode(cur, a.B, p, b, tile);
        const bool needs_input = p > 0 || !a.source;
        const bool col = (p & 1) != 0;
        int abort_local = 0, err_seen = 0;
        if (tid == 0) {
            s_int[1] = fetched;              // the next item, fetched during the previous one
            fetched = atomicAdd(a.head, 1);  // the one after: its latency hides under this item
            err_seen = ld_relaxed(a.err);    // read at the end of the item
            bool missing = false;
            if (needs_input) {
                if (col) {
                    missing = col_issued != cur;
                } else {
                    for (int w = 0; w < Fused::WARPS; ++w) missing |= row_issued[w] != cur;
                }
            }
            if (missing) {
                bool ok = true;
                if (p > 0) {
                    signal();  // never wait while holding an unsignalled tile
                    const int* ctr = a.done + (p - 1) * a.B + b;
                    const long long t0 = clock64();
                    while (ld_acquire(ctr) < Fused::TPF) {
                        if (ld_relaxed(a.err) != 0 || clock64() - t0 > a.budget) {
                            ok = false;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
                if (ok && !a.stall) {
                    fence_proxy_async_global();
                    if (col) {
                        issue_col(a, &tmap, p, b, tile, buf, ht, bin);
                        col_issued = cur;
                    } else {
                        for (int w = 0; w < Fused::WARPS; ++w) {
                            if (row_issued[w] != cur) {
                                issue_row(a, b, tile, w, buf, bw);
                                row_issued[w] = cur;
                            }
                        }
                    }
                }
                if (!ok) {
                    atomicExch(a.err, kErrDepWait);
                    abort_local = 1;
                }
            }
        }
        if (__syncthreads_or(abort_local)) {  // copies of this item in flight: wait for them (bounded)
            if (tid == 0 && col_issued == cur) mbar_wait(bin, pin, a.budget);
            if (lane == 0 && !col && row_issued[warp] == cur) mbar_wait(bw + warp, pw, a.budget);
            return;
        }
        const int nxt = s_int[1];
        bool bad = false;  // a wait of this thread's warp ran out (the launch then stops)
        float2 v[32];
        if (col) {
            // ---------------- column tile: FFT -> H_s -> IFFT over 8 columns ----------------
            const int c = tid % Fused::W, t = tid / Fused::W, s = (p - 1) >> 1;
            const bool ok = mbar_wait(bin, pin, a.budget);
            pin ^= 1u;
            if (ok) {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = buf[(t + 32 * i) * Fused::W + c];
            }
            if (__syncthreads_or(!ok)) {  // also: every thread has read the tile before the exchange
                if (tid == 0) {
                    atomicExch(a.err, kErrDepWait);
                    mbar_wait(bin, pin ^ 1u, a.budget);  // the copy in flight, bounded again
                }
                return;
            }
            float2* line = buf + c * Fused::LSC;
            const int colx = tile * Fused::W + c;
            fft_stage_c<C, 0, -1>(v, line, t, tw, BlockBar());
            if (tid == 0) signal();  // the previous tile's stores have had a stage to drain
            fft_stage_c<C, 1, -1>(v, line, t, tw, BlockBar());
            transfer_tile<false, HMODE>(v, ht, colx, t, a.ccross[s], a.dcoef[s], a.inv_k2);
            fft_stage_c<C, 0, +1>(v, line, t, tw, BlockBar());  // ends with a barrier after the last read
            if (tid == 0) {  // the whole buffer is free: the next item's input, if it is ready
                int pn, bn, tn;
                if (ready(nxt, pn, bn, tn)) {
                    fence_proxy_async_global();
                    fence_proxy_async();
                    if (pn & 1) {
                        issue_col(a, &tmap, pn, bn, tn, buf, ht, bin);
                        col_issued = nxt;
                    } else {
                        for (int w = 0; w < Fused::WARPS; ++w) {
                            issue_row(a, bn, tn, w, buf, bw);
                            row_issued[w] = nxt;
                        }
                    }
                }
            }
            fft_stage_c<C, 1, +1>(v, line, t, tw, BlockBar());
            float2* base = a.field + (size_t)b * kN * kN + colx;
#pragma unroll
            for (int i = 0; i < 32; ++i) base[(size_t)(t + 32 * i) * kN] = v[i];
        } else {
            // ---------------- row tile: one row per warp, warps independent ----------------
            float2* line = buf + warp * Fused::LSR;
            const int j = tile * Fused::WARPS + warp;
            float2* row = a.field + ((size_t)b * kN + j) * kN;
            if (p == 0 && a.source) {
                const float coef = a.src_coef[(b + a.src_off) % a.n_src];
                const float y = (float)(j - kN / 2);
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float x = (float)(lane + 32 * i - kN / 2);
                    v[i] = coef < 0.0f ? make_float2(1.0f, 0.0f) : make_float2(expf(-(x * x + y * y) * coef), 0.0f);
                }
            } else {
                const bool ok = __all_sync(0xffffffffu, mbar_wait(bw + warp, pw, a.budget));
                pw ^= 1u;
                if (!ok) {
                    bad = true;
                    if (lane == 0) mbar_wait(bw + warp, pw ^ 1u, a.budget);
                }
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = line[lane + 32 * i];
                __syncwarp();
            }
            if (tid == 0) signal();
            if (p > 0) {
                const int s = (p >> 1) - 1;
                fft_stage_c<C, 0, +1>(v, line, lane, tw, WarpBar());
                if (lane == 0) {  // the line is free: the screen phasor row comes in under the next stage
                    const int set = (b + a.phi_off) / a.phi_group;
                    fence_proxy_async();
                    mbar_expect_tx(bw + warp, kN * 8);
                    bulk_load(line, a.phasor + (long long)s * kN * kN + (long long)set * a.set_stride + (size_t)j * kN,
                              kN * 8, bw + warp);
                }
                fft_stage_c<C, 1, +1>(v, line, lane, tw, WarpBar());
                const bool okp = __all_sync(0xffffffffu, mbar_wait(bw + warp, pw, a.budget));
                pw ^= 1u;
                if (!okp) {
                    bad = true;
                    if (lane == 0) mbar_wait(bw + warp, pw ^ 1u, a.budget);
                }
                if (a.phase_sign > 0.0f) {
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] = cmul(v[i], line[lane + 32 * i]);
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i) v[i] = cmulc(v[i], line[lane + 32 * i]);
                }
                __syncwarp();
            }
            const bool out_freq = p < 2 * a.S;
            if (out_freq) fft_stage_c<C, 0, -1>(v, line, lane, tw, WarpBar());
            if (lane == 0) {  // this warp's line is free: its row of the next item, if that is a ready row tile
                int pn, bn, tn;
                if (ready(nxt, pn, bn, tn) && !(pn & 1)) {
                    fence_proxy_async_global();
                    fence_proxy_async();
                    issue_row(a, bn, tn, warp, buf, bw);
                    row_issued[warp] = nxt;
                }
            }
            if (out_freq) fft_stage_c<C, 1, -1>(v, line, lane, tw, WarpBar());
#pragma unroll
            for (int i = 0; i < 32; ++i) row[lane + 32 * i] = v[i];
        }
        // end of the tile: its completion is signalled by thread 0 during the next item
        const int ab = __syncthreads_or(bad || err_seen != 0);
        if (ab) {
            if (tid == 0) {
                if (bad) atomicExch(a.err, kErrDepWait);
                if (col_issued == nxt) mbar_wait(bin, pin, a.budget);  // prefetched copies in flight
            }
            if (lane == 0 && row_issued[warp] == nxt) mbar_wait(bw + warp, pw, a.budget);
            return;
        }
        if (tid == 0) pending = p * a.B + b;
        cur = nxt;
    }
    if (tid == 0) signal();
}

__global__ void ht_table_kernel(float4* ht, const float2* P, int S, float dk)
{
    const int n = S * kN;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int m = i % kN;
        const float k = dk * (float)kidx(m, kN);
        const float2 q = P[i];
        ht[i] = make_float4(q.x, q.y, k * k, 0.0f);
    }
}


template <int HMODE>
cudaError_t fused_launch(const FusedParams& fp, const CUtensorMap& map, cudaStream_t st)
{
    // CTAs resident on the current device at once, cached per device ordinal (below 64)
    static int cache[64] = {};
    int dev = 0, resident = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) resident = cache[dev];
    if (resident == 0) {
        int sms = 0, per = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, prop_fused_kernel<HMODE>, Fused::THREADS, Fused::smem);
        if (e != cudaSuccess) return e;
        resident = sms * per;
        if (dev >= 0 && dev < 64) cache[dev] = resident;
    }
    if (resident <= 0) return cudaErrorInvalidConfiguration;
    const int items = (2 * fp.S + 1) * fp.B * Fused::TPF;
    const int grid = std::min(items, resident);
    prop_fused_kernel<HMODE><<<grid, Fused::THREADS, Fused::smem, st>>>(fp, map);
    return cudaGetLastError();
}

}  // namespace

cudaError_t build_ht_table(float4* ht, const float2* P, int S, double dk, cudaStream_t st)
{
    ht_table_kernel<<<64, 256, 0, st>>>(ht, P, S, (float)dk);
    return cudaGetLastError();
}

cudaError_t prop_fused_1024(int hmode, const FusedParams& fp, cudaStream_t st)
{
    if ((reinterpret_cast<uintptr_t>(fp.field) & 15) != 0 || (reinterpret_cast<uintptr_t>(fp.phasor) & 15) != 0 ||
        (fp.set_stride & 1) != 0 || fp.err == nullptr || fp.done == nullptr || fp.B < 1 ||
        fp.S < 1 || fp.S > kMaxScreens || fp.n_src < 1)
        return cudaErrorNotSupported;
    CUtensorMap map;
    cudaError_t em = field_tensor_map(&map, fp.field, kN, fp.B, 2 * Fused::W, 256);
    if (em != cudaSuccess) return em;
    FusedParams f = fp;
    f.head = fp.done + (2 * fp.S + 1) * fp.B;  // the work counter follows the completion counters
    cudaError_t e = cudaMemsetAsync(f.done, 0, sizeof(int) * ((2 * f.S + 1) * f.B + 1), st);
    if (e != cudaSuccess) return e;
    switch (hmode) {
    case 0: return fused_launch<0>(f, map, st);
    case 1: return fused_launch<1>(f, map, st);
    case 2: return fused_launch<2>(f, map, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_prop_fused_1024()
{
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    auto attr = [&](auto kernel) {
        chk(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Fused::smem));
        chk(cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    };
    attr(prop_fused_kernel<0>);
    attr(prop_fused_kernel<1>);
    attr(prop_fused_kernel<2>);
    return e;
}

}  // namespace ts
