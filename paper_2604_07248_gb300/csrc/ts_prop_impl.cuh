// ts_prop_impl.cuh -- propagation pass kernels (templates) shared by the per-N translation units.
//
// The field is kept between steps in the "row-frequency" domain R = FFT_rows(U).  One step is
//   column pass:  C = IFFT_cols( H . FFT_cols(R) )          (H includes the 1/N^2 of IFFT2)
//   row pass:     U = IFFT_rows(C) . exp(i phi_s);  R = FFT_rows(U)   (next step)
// so each step reads and writes the field twice and reads the screen once.
// Row passes give each line of N points to T = N / E threads (E points per thread, registers);
// column passes load W adjacent columns per CTA so that every warp load touches W*8 contiguous
// bytes of each of 32 / W rows.
#pragma once
#include <type_traits>

#include "ts_device.cuh"
#include "ts_internal.h"
#include "ts_prop_decl.h"

namespace ts {
namespace {


constexpr int kRowThreads = 256;



template <int N, int E>
struct RowCfg {
    using C = FftCfg<N, E>;
    static constexpr int LPC = kRowThreads / C::T;  // lines per CTA
    static constexpr int LS = C::padded;            // line stride in shared memory (float2)
    static constexpr int WPL = C::T > 32 ? C::T / 32 : 1;  // warps per line
    static constexpr size_t smem = sizeof(float2) * (C::tw_smem + LPC * LS);
};

// One row tile: rows jblock * LPC .. + LPC - 1 of field b.  Shared by the per-pass kernel and the
// persistent uneven-batch kernel; `smem` holds the twiddles (staged here when stage_tw) and the
// per-line exchange buffers.
template <int N, int EE, int FLAGS>
__device__ __forceinline__ void row_tile(const RowParams& a, int jblock, int b, float2* smem, bool stage_tw)
{
    using C = FftCfg<N, EE>;
    using RC = RowCfg<N, EE>;
    constexpr int E = C::E, T = C::T;
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int j = jblock * RC::LPC + line;
    float2* tw = smem;
    float2* buf = smem + C::tw_smem + line * RC::LS;
    float2* row = a.field + ((size_t)b * N + j) * N;
    // a line of more than one warp synchronises only its own warps, on its own named barrier
    static_assert(T <= 32 || (T % 32 == 0 && kRowThreads / T <= 15), "lines of whole warps, at most 15 per CTA");
    using Bar = typename std::conditional<(T > 32), LineBar<(T > 32 ? T : 32)>, WarpBar>::type;
    Bar bar{};
    if constexpr (T > 32) bar.id = 1 + line;
    if (stage_tw) stage_twiddles_c<C>(tw, a.tw);
    __syncthreads();

    float2 v[E];
    if constexpr (FLAGS & RP_IN_SOURCE) {
        const float coef = a.src_coef[(b + a.src_off) % a.n_src];
        const float y = (float)(j - N / 2);
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const float x = (float)(t + i * T - N / 2);
            v[i] = coef < 0.0f ? make_float2(1.0f, 0.0f) : make_float2(expf(-(x * x + y * y) * coef), 0.0f);
        }
    } else {
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = row[t + i * T];
    }
    if constexpr (FLAGS & RP_IN_FREQ) line_fft_c<C, +1>(v, buf, t, tw, bar);
    if constexpr (FLAGS & RP_PHASOR) {
        // exp(i phi) precomputed once per screen: multiply (forward) or multiply by the conjugate (adjoint)
        const float2* ph = a.phasor + (long long)((b + a.phi_off) / a.phi_group) * a.phi_set_stride + (size_t)j * N;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const float2 e = __ldg(ph + t + i * T);
            v[i] = a.phase_sign > 0.0f ? cmul(v[i], e) : cmulc(v[i], e);
        }
    } else if constexpr (FLAGS & RP_PHASE) {
        if (a.phi != nullptr) {
            const float* ph = a.phi + (long long)((b + a.phi_off) / a.phi_group) * a.phi_set_stride + (size_t)j * N;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const float2 e = expi_phase(__ldg(ph + t + i * T));
                v[i] = cmul(v[i], make_float2(e.x, a.phase_sign * e.y));
            }
        }
    }
    if constexpr (FLAGS & RP_INTENSITY) {
        float s0 = 0.0f, s1 = 0.0f;
        const float y = (float)(j - N / 2);
        float* irow = a.intensity + ((size_t)b * N + j) * N;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const float I = v[i].x * v[i].x + v[i].y * v[i].y;
            const float x = (float)(t + i * T - N / 2);
            irow[t + i * T] = I;
            s0 += I;
            s1 = fmaf(x * x + y * y, I, s1);
        }
        if (a.rows != nullptr) {
            double d0 = s0, d1 = s1;
            constexpr int width = T < 32 ? T : 32;
#pragma unroll
            for (int off = width / 2; off > 0; off >>= 1) {
                d0 += __shfl_down_sync(0xffffffffu, d0, off, width);
                d1 += __shfl_down_sync(0xffffffffu, d1, off, width);
            }
            if ((t % width) == 0) {
                double* dst = a.rows + (((size_t)b * N + j) * RC::WPL + t / 32) * 2;
                dst[0] = d0;
                dst[1] = d1;
            }
        }
    }
    if constexpr (FLAGS & RP_OUT_FREQ) line_fft_c<C, -1>(v, buf, t, tw, bar);
    if constexpr (FLAGS & RP_STORE) {
#pragma unroll
        for (int i = 0; i < E; ++i) row[t + i * T] = v[i];
    }
}

// at least two CTAs per SM (E = 32: <= 128 registers); E = 16 kernels fit four
template <int N, int EE, int FLAGS>
__global__ void __launch_bounds__(kRowThreads, (FftCfg<N, EE>::E >= 32 ? 2 : 4)) row_pass_kernel(const RowParams a)
{
    extern __shared__ float2 smem[];
    row_tile<N, EE, FLAGS>(a, blockIdx.x, blockIdx.y, smem, true);
}



// Row pass with the screen phasor shared through shared memory (E = 32, one warp per row): the CTA's
// 8 warps are 8 / FPC rows x FPC fields that use the same screen set, so each phasor row is read from
// memory once per CTA, at kernel start (its latency overlaps the field loads and the inverse FFT),
// instead of once per field after the inverse FFT.  Requires the FPC fields of a CTA to share one set.
template <int N>
struct RowShCfg {
    using C = FftCfg<N, 32>;
    static_assert(C::T == 32, "one warp per row");
    static constexpr int LS = C::padded;
    static constexpr size_t smem(int fpc) { return sizeof(float2) * (C::tw_smem + (8 / fpc) * N + 8 * LS); }
};

template <int N, int FLAGS, int FPC>
__global__ void __launch_bounds__(kRowThreads, 2) row_pass_shared_kernel(const RowParams a)
{
    static_assert(FLAGS & RP_PHASOR, "shared phasor rows");
    using C = typename RowShCfg<N>::C;
    constexpr int E = C::E, T = C::T, RPC = 8 / FPC;
    extern __shared__ float2 smem[];
    float2* tw = smem;
    float2* phs = smem + C::tw_smem;
    const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
    const int rsub = warp / FPC, f = warp % FPC;
    const int j0 = blockIdx.x * RPC, j = j0 + rsub;
    const int b = blockIdx.y * FPC + f;
    float2* buf = phs + RPC * N + warp * RowShCfg<N>::LS;
    float2* row = a.field + ((size_t)b * N + j) * N;
    // the field row first (its loads are in flight while the twiddles and phasor rows are staged)
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = row[t + i * T];
    stage_twiddles_c<C>(tw, a.tw);
    {
        const int set = (blockIdx.y * FPC + a.phi_off) / a.phi_group;
        const float4* src = reinterpret_cast<const float4*>(a.phasor + (long long)set * a.phi_set_stride + (size_t)j0 * N);
        float4* dst = reinterpret_cast<float4*>(phs);
        for (int i = threadIdx.x; i < RPC * N / 2; i += kRowThreads) dst[i] = __ldg(src + i);
    }
    __syncthreads();
    if constexpr (FLAGS & RP_IN_FREQ) line_fft_c<C, +1>(v, buf, t, tw, WarpBar());
    const float2* ph = phs + rsub * N;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const float2 e = ph[t + i * T];
        v[i] = a.phase_sign > 0.0f ? cmul(v[i], e) : cmulc(v[i], e);
    }
    if constexpr (FLAGS & RP_INTENSITY) {
        float s0 = 0.0f, s1 = 0.0f;
        const float y = (float)(j - N / 2);
        float* irow = a.intensity + ((size_t)b * N + j) * N;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const float I = v[i].x * v[i].x + v[i].y * v[i].y;
            const float x = (float)(t + i * T - N / 2);
            irow[t + i * T] = I;
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
            if (t == 0) {
                double* dst = a.rows + ((size_t)b * N + j) * 2;
                dst[0] = d0;
                dst[1] = d1;
            }
        }
    }
    if constexpr (FLAGS & RP_OUT_FREQ) line_fft_c<C, -1>(v, buf, t, tw, WarpBar());
    if constexpr (FLAGS & RP_STORE) {
#pragma unroll
        for (int i = 0; i < E; ++i) row[t + i * T] = v[i];
    }
}

template <int N, int E>
struct ColCfg {
    using C = FftCfg<N, E>;
    // 512 threads when a line needs 64+ threads at N <= 1024, so a CTA still covers 8 columns (64-byte rows)
    static constexpr int THREADS = (C::T >= 64 && N <= 1024) ? 512 : 256;
    static constexpr int W = THREADS / C::T;                        // columns per CTA
    static constexpr int LS = C::padded + (16 / W > 1 ? 16 / W : 1);  // conflict-free column stride
    static constexpr size_t smem = sizeof(float2) * (C::tw_smem + N + W * LS);
};

// Exact form: H(ky, kx) = P(kx) P(ky) exp(-i delta), P = exp(-i dz kappa^2 / 2k) / N,
// delta = dz kappa^4 / (2k (k + sqrt(k^2 - kappa^2))^2) (the angular-spectrum phase beyond its paraxial
// part); 0 in the evanescent region.
__device__ __forceinline__ float2 transfer_exact(float2 px, float2 py, float k2, float inv_k2, float dcoef)
{
    const float q = k2 * inv_k2;
    if (q >= 1.0f) return make_float2(0.0f, 0.0f);
    const float d = 1.0f + sqrtf(1.0f - q);
    const float del = __fdividef(dcoef * k2 * k2, d * d);
    const float d2 = del * del;
    const float cd = 1.0f - d2 * (0.5f - d2 * (1.0f / 24.0f - d2 * (1.0f / 720.0f)));
    const float sd = del * (1.0f - d2 * (1.0f / 6.0f - d2 * (1.0f / 120.0f - d2 * (1.0f / 5040.0f))));
    return cmul(cmul(px, py), make_float2(cd, -sd));
}

// Separable form (used when the plan shows the dropped terms are below 1e-7 rad):
//   dz (k - sqrt(k^2 - kappa^2)) = dz kappa^2 / 2k + dz kappa^4 / 8k^3 + O(dz kappa^6 / 16 k^5),
// kappa^4 = kx^4 + ky^4 + 2 kx^2 ky^2, so H = P'(kx) P'(ky) exp(-i e) with
// P' = exp(-i dz (kappa^2 / 2k + kappa^4 / 8k^3)) / N (FP64-built) and e = dz kx^2 ky^2 / (4 k^3).
__device__ __forceinline__ float2 small_phase(float e)
{
    const float e2 = e * e;
    return make_float2(1.0f - e2 * (0.5f - e2 * (1.0f / 24.0f)), -e * (1.0f - e2 * (1.0f / 6.0f)));
}

// v[i] (frequency t + i T of column col) *= H, or conj(H) for the adjoint; Ps = the step's P table
template <int N, int E, bool CONJ, bool SEP>
__device__ __forceinline__ void apply_transfer(float2 (&v)[E], const ColParams& a, const float2* Ps, int col, int t, int T)
{
    const float kx = a.dk * (float)kidx(col, N);
    const float2 px = Ps[col];
    if constexpr (SEP) {
        const float cx = a.ccross * kx * kx;
        if (a.first_order_cross) {  // e <= 4.4e-4 rad on the whole grid: exp(-i e) = 1 - i e
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int m = t + i * T;
                const float ky = a.dk * (float)kidx(m, N);
                const float2 q = cmul(px, Ps[m]);
                const float e = cx * ky * ky;
                const float2 h = make_float2(fmaf(e, q.y, q.x), fmaf(-e, q.x, q.y));
                v[i] = CONJ ? cmulc(v[i], h) : cmul(v[i], h);
            }
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) {
                const int m = t + i * T;
                const float ky = a.dk * (float)kidx(m, N);
                const float2 h = cmul(cmul(px, Ps[m]), small_phase(cx * ky * ky));
                v[i] = CONJ ? cmulc(v[i], h) : cmul(v[i], h);
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int m = t + i * T;
            const float ky = a.dk * (float)kidx(m, N);
            const float2 h = transfer_exact(px, Ps[m], fmaf(kx, kx, ky * ky), a.inv_k2, a.dcoef);
            v[i] = CONJ ? cmulc(v[i], h) : cmul(v[i], h);
        }
    }
}

// One column tile: columns cblock * W .. + W - 1 of field b (see row_tile for smem).
template <int N, int EE, bool CONJ, bool SEP>
__device__ __forceinline__ void col_tile(const ColParams& a, int cblock, int b, float2* smem, bool stage_tw)
{
    using C = FftCfg<N, EE>;
    using CC = ColCfg<N, EE>;
    constexpr int E = C::E, T = C::T, W = CC::W;
    const int c = threadIdx.x % W, t = threadIdx.x / W;
    const int col = cblock * W + c;
    float2* tw = smem;
    float2* Ps = smem + C::tw_smem;
    float2* buf = Ps + N + c * CC::LS;
    float2* base = a.field + (size_t)b * N * N + col;

    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = base[(size_t)(t + i * T) * N];
    if (stage_tw) stage_twiddles_c<C>(tw, a.tw);
    for (int i = threadIdx.x; i < N; i += blockDim.x) Ps[i] = __ldg(a.P + i);
    __syncthreads();
    line_fft_c<C, -1>(v, buf, t, tw, BlockBar());
    apply_transfer<N, E, CONJ, SEP>(v, a, Ps, col, t, T);
    line_fft_c<C, +1>(v, buf, t, tw, BlockBar());
#pragma unroll
    for (int i = 0; i < E; ++i) base[(size_t)(t + i * T) * N] = v[i];
}

// Warp-owned columns (N = 1024 with 32 points per thread, so one warp holds one column): the CTA
// stages its 8-column tile through shared memory with coalesced loads, every warp then transforms
// its own column using that column's part of the tile as its exchange storage (warp-level
// synchronisation only, so warps progress independently), and the tile goes back with coalesced
// stores.  Element x of column c sits in the 128-byte line pair y = x / 2 at 8-byte slot
// ((x % 2) 8 + c) xor ((y xor y / 16) mod 16): the staging accesses, the Stockham stage-0 writes and
// the strided reads all run at the 2-wavefront minimum.
constexpr int kColWarpW = 8;

__device__ __forceinline__ int tile_slot(int x, int c)
{
    const int y = x >> 1;
    return y * 16 + ((((x & 1) << 3) + c) ^ ((y ^ (y >> 4)) & 15));
}

template <int N>
struct ColWarpCfg {
    using C = FftCfg<N, 32>;
    static_assert(C::T == 32, "one warp per column");
    static constexpr size_t smem = sizeof(float2) * (C::tw_smem + N + kColWarpW * N);
};

struct TileMap {
    float2* tile;
    int c;
    __device__ __forceinline__ float2* operator()(int x) const { return tile + tile_slot(x, c); }
};

template <int N, bool CONJ, bool SEP>
__global__ void __launch_bounds__(32 * kColWarpW, 2) col_pass_warp_kernel(const ColParams a)
{
    using C = typename ColWarpCfg<N>::C;
    constexpr int E = C::E;
    extern __shared__ float2 smem[];
    float2* tw = smem;
    float2* Ps = smem + C::tw_smem;
    float2* tile = Ps + N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col0 = blockIdx.x * kColWarpW;
    float2* base = a.field + (size_t)blockIdx.y * N * N + col0;
    stage_twiddles_c<C>(tw, a.tw);
    for (int i = threadIdx.x; i < N; i += blockDim.x) Ps[i] = __ldg(a.P + i);
#pragma unroll 8
    for (int idx = threadIdx.x; idx < kColWarpW * N; idx += blockDim.x) {
        const int r = idx >> 3, c = idx & 7;
        tile[tile_slot(r, c)] = base[(size_t)r * N + c];
    }
    __syncthreads();
    const TileMap map{tile, warp};
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = *map(lane + 32 * i);
    __syncwarp();  // every lane has its points before the exchange overwrites the column
    line_fft_m<C, -1>(v, map, lane, tw, WarpBar());
    apply_transfer<N, E, CONJ, SEP>(v, a, Ps, col0 + warp, lane, 32);
    line_fft_m<C, +1>(v, map, lane, tw, WarpBar());
#pragma unroll
    for (int i = 0; i < E; ++i) *map(lane + 32 * i) = v[i];
    __syncthreads();
#pragma unroll 8
    for (int idx = threadIdx.x; idx < kColWarpW * N; idx += blockDim.x) {
        const int r = idx >> 3, c = idx & 7;
        base[(size_t)r * N + c] = tile[tile_slot(r, c)];
    }
}

template <int N, int EE, bool CONJ, bool SEP>
__global__ void __launch_bounds__(ColCfg<N, EE>::THREADS, 2) col_pass_kernel(const ColParams a)
{
    extern __shared__ float2 smem[];
    col_tile<N, EE, CONJ, SEP>(a, blockIdx.x, blockIdx.y, smem, true);
}


template <int N, int E, int FLAGS>
cudaError_t row_launch(const RowParams& rp, int B, cudaStream_t st)
{
    using RC = RowCfg<N, E>;
    dim3 grid(N / RC::LPC, B);
    row_pass_kernel<N, E, FLAGS><<<grid, kRowThreads, RC::smem, st>>>(rp);
    return cudaGetLastError();
}

template <int N, int E>
cudaError_t row_dispatch(int flags, const RowParams& rp, int B, cudaStream_t st)
{
    switch (flags) {
    case RP_IN_SOURCE | RP_STORE: return row_launch<N, E, RP_IN_SOURCE | RP_STORE>(rp, B, st);
    case RP_IN_SOURCE | RP_OUT_FREQ | RP_STORE: return row_launch<N, E, RP_IN_SOURCE | RP_OUT_FREQ | RP_STORE>(rp, B, st);
    case RP_OUT_FREQ | RP_STORE: return row_launch<N, E, RP_OUT_FREQ | RP_STORE>(rp, B, st);
    case RP_PHASE | RP_OUT_FREQ | RP_STORE: return row_launch<N, E, RP_PHASE | RP_OUT_FREQ | RP_STORE>(rp, B, st);
    case RP_IN_FREQ | RP_PHASE | RP_OUT_FREQ | RP_STORE:
        return row_launch<N, E, RP_IN_FREQ | RP_PHASE | RP_OUT_FREQ | RP_STORE>(rp, B, st);
    case RP_IN_FREQ | RP_PHASE | RP_STORE: return row_launch<N, E, RP_IN_FREQ | RP_PHASE | RP_STORE>(rp, B, st);
    case RP_IN_FREQ | RP_PHASE | RP_INTENSITY | RP_STORE:
        return row_launch<N, E, RP_IN_FREQ | RP_PHASE | RP_INTENSITY | RP_STORE>(rp, B, st);
    case RP_IN_FREQ | RP_PHASE | RP_INTENSITY: return row_launch<N, E, RP_IN_FREQ | RP_PHASE | RP_INTENSITY>(rp, B, st);
    case RP_IN_FREQ | RP_STORE: return row_launch<N, E, RP_IN_FREQ | RP_STORE>(rp, B, st);
    case RP_PHASOR | RP_OUT_FREQ | RP_STORE: return row_launch<N, E, RP_PHASOR | RP_OUT_FREQ | RP_STORE>(rp, B, st);
    case RP_IN_FREQ | RP_PHASOR | RP_OUT_FREQ | RP_STORE:
        return row_launch<N, E, RP_IN_FREQ | RP_PHASOR | RP_OUT_FREQ | RP_STORE>(rp, B, st);
    case RP_IN_FREQ | RP_PHASOR | RP_STORE: return row_launch<N, E, RP_IN_FREQ | RP_PHASOR | RP_STORE>(rp, B, st);
    case RP_IN_FREQ | RP_PHASOR | RP_INTENSITY | RP_STORE:
        return row_launch<N, E, RP_IN_FREQ | RP_PHASOR | RP_INTENSITY | RP_STORE>(rp, B, st);
    case RP_IN_FREQ | RP_PHASOR | RP_INTENSITY: return row_launch<N, E, RP_IN_FREQ | RP_PHASOR | RP_INTENSITY>(rp, B, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int N, int FLAGS, int FPC>
cudaError_t row_launch_shared(const RowParams& rp, int B, cudaStream_t st)
{
    dim3 grid(N / (8 / FPC), B / FPC);
    row_pass_shared_kernel<N, FLAGS, FPC><<<grid, kRowThreads, RowShCfg<N>::smem(FPC), st>>>(rp);
    return cudaGetLastError();
}

// the shared-phasor row pass for the flag sets that modulate by a phasor; returns
// cudaErrorNotSupported when the combination has no shared variant
template <int N, int FPC>
cudaError_t row_dispatch_shared(int flags, const RowParams& rp, int B, cudaStream_t st)
{
    switch (flags) {
    case RP_IN_FREQ | RP_PHASOR | RP_OUT_FREQ | RP_STORE:
        return row_launch_shared<N, RP_IN_FREQ | RP_PHASOR | RP_OUT_FREQ | RP_STORE, FPC>(rp, B, st);
    case RP_IN_FREQ | RP_PHASOR | RP_STORE: return row_launch_shared<N, RP_IN_FREQ | RP_PHASOR | RP_STORE, FPC>(rp, B, st);
    case RP_IN_FREQ | RP_PHASOR | RP_INTENSITY | RP_STORE:
        return row_launch_shared<N, RP_IN_FREQ | RP_PHASOR | RP_INTENSITY | RP_STORE, FPC>(rp, B, st);
    case RP_IN_FREQ | RP_PHASOR | RP_INTENSITY:
        return row_launch_shared<N, RP_IN_FREQ | RP_PHASOR | RP_INTENSITY, FPC>(rp, B, st);
    case RP_PHASOR | RP_OUT_FREQ | RP_STORE: return row_launch_shared<N, RP_PHASOR | RP_OUT_FREQ | RP_STORE, FPC>(rp, B, st);
    default: return cudaErrorNotSupported;
    }
}

template <int N, int E, bool CONJ, bool SEP>
cudaError_t col_launch(const ColParams& cp, int B, cudaStream_t st)
{
    using CC = ColCfg<N, E>;
    dim3 grid(N / CC::W, B);
    col_pass_kernel<N, E, CONJ, SEP><<<grid, CC::THREADS, CC::smem, st>>>(cp);
    return cudaGetLastError();
}

template <int N, bool CONJ, bool SEP>
cudaError_t col_launch_warp(const ColParams& cp, int B, cudaStream_t st)
{
    dim3 grid(N / kColWarpW, B);
    col_pass_warp_kernel<N, CONJ, SEP><<<grid, 32 * kColWarpW, ColWarpCfg<N>::smem, st>>>(cp);
    return cudaGetLastError();
}

// dynamic shared memory limit plus the largest shared-memory carveout, so the occupancy the launch
// bounds ask for is not cut by the L1 / shared split
template <class K>
cudaError_t smem_attr(K kernel, int bytes)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

template <int N, int E, int FLAGS>
cudaError_t row_attr()
{
    return smem_attr(row_pass_kernel<N, E, FLAGS>, (int)RowCfg<N, E>::smem);
}

template <int N, int FPC>
cudaError_t row_attr_shared()
{
    cudaError_t e = cudaSuccess;
    const int sz = (int)RowShCfg<N>::smem(FPC);
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    chk(smem_attr(row_pass_shared_kernel<N, RP_IN_FREQ | RP_PHASOR | RP_OUT_FREQ | RP_STORE, FPC>, sz));
    chk(smem_attr(row_pass_shared_kernel<N, RP_IN_FREQ | RP_PHASOR | RP_STORE, FPC>, sz));
    chk(smem_attr(row_pass_shared_kernel<N, RP_IN_FREQ | RP_PHASOR | RP_INTENSITY | RP_STORE, FPC>, sz));
    chk(smem_attr(row_pass_shared_kernel<N, RP_IN_FREQ | RP_PHASOR | RP_INTENSITY, FPC>, sz));
    chk(smem_attr(row_pass_shared_kernel<N, RP_PHASOR | RP_OUT_FREQ | RP_STORE, FPC>, sz));
    return e;
}

template <int N, int E>
cudaError_t prepare_prop_for()
{
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    chk(row_attr<N, E, RP_IN_SOURCE | RP_STORE>());
    chk(row_attr<N, E, RP_IN_SOURCE | RP_OUT_FREQ | RP_STORE>());
    chk(row_attr<N, E, RP_OUT_FREQ | RP_STORE>());
    chk(row_attr<N, E, RP_PHASE | RP_OUT_FREQ | RP_STORE>());
    chk(row_attr<N, E, RP_IN_FREQ | RP_PHASE | RP_OUT_FREQ | RP_STORE>());
    chk(row_attr<N, E, RP_IN_FREQ | RP_PHASE | RP_STORE>());
    chk(row_attr<N, E, RP_IN_FREQ | RP_PHASE | RP_INTENSITY | RP_STORE>());
    chk(row_attr<N, E, RP_IN_FREQ | RP_PHASE | RP_INTENSITY>());
    chk(row_attr<N, E, RP_IN_FREQ | RP_STORE>());
    chk(row_attr<N, E, RP_PHASOR | RP_OUT_FREQ | RP_STORE>());
    chk(row_attr<N, E, RP_IN_FREQ | RP_PHASOR | RP_OUT_FREQ | RP_STORE>());
    chk(row_attr<N, E, RP_IN_FREQ | RP_PHASOR | RP_STORE>());
    chk(row_attr<N, E, RP_IN_FREQ | RP_PHASOR | RP_INTENSITY | RP_STORE>());
    chk(row_attr<N, E, RP_IN_FREQ | RP_PHASOR | RP_INTENSITY>());
    const int cs = (int)ColCfg<N, E>::smem;
    chk(smem_attr(col_pass_kernel<N, E, false, false>, cs));
    chk(smem_attr(col_pass_kernel<N, E, true, false>, cs));
    chk(smem_attr(col_pass_kernel<N, E, false, true>, cs));
    chk(smem_attr(col_pass_kernel<N, E, true, true>, cs));
    return e;
}



}  // namespace

template <int N>
cudaError_t row_pass_n(int E, int variant, int flags, const RowParams& rp, int B, cudaStream_t st)
{
    if constexpr (N == 512 || N == 1024) {
        // persistent warps with bulk-copy prefetch (middle and last row passes of a phasor path)
        if (variant == 2 && E == 32) {
            cudaError_t e = row_pass_tma(N, flags, rp, B, st);
            if (e != cudaErrorNotSupported) return e;
        }
    }
    if constexpr (N == 1024) {
        // shared phasor rows: FPC consecutive fields of one screen set per CTA
        // (the phasor rows are staged with 16-byte loads: only for 16-byte aligned phasor arrays)
        if (variant == 1 && E == 32 && (flags & RP_PHASOR) && (reinterpret_cast<uintptr_t>(rp.phasor) & 15) == 0 &&
            (rp.phi_set_stride & 1) == 0) {
            for (int fpc = 8; fpc >= 2; fpc >>= 1) {
                if (B % fpc || rp.phi_group % fpc || rp.phi_off % fpc) continue;
                cudaError_t e = fpc == 8 ? row_dispatch_shared<N, 8>(flags, rp, B, st)
                                : fpc == 4 ? row_dispatch_shared<N, 4>(flags, rp, B, st)
                                           : row_dispatch_shared<N, 2>(flags, rp, B, st);
                if (e != cudaErrorNotSupported) return e;
                break;
            }
        }
    }
    if constexpr (N <= 256) {
        return row_dispatch<N, 16>(flags, rp, B, st);
    } else {
        return E == 16 ? row_dispatch<N, 16>(flags, rp, B, st) : row_dispatch<N, 32>(flags, rp, B, st);
    }
}

template <int N>
cudaError_t col_pass_n(int E, int variant, bool conj, bool sep, const ColParams& cp, int B, cudaStream_t st,
                       bool source)
{
    if constexpr (N == 512 || N == 1024) {
        if ((variant == 2 || variant == 3) && E == 32) {
            const int w = N == 512 ? (variant == 2 ? 16 : 8) : (variant == 2 ? 8 : 4);
            const int hmode = sep ? (cp.first_order_cross ? 3 : cp.tiny_cross ? 2 : 1) : 0;
            cudaError_t e = col_pass_tma(N, w, conj, hmode, cp, B, st, source);
            if (e != cudaErrorNotSupported || source) return e;
        }
    }
    if (source) return cudaErrorNotSupported;
    if constexpr (N == 1024) {
        if (variant == 1 && E == 32) {
            if (sep) return conj ? col_launch_warp<N, true, true>(cp, B, st) : col_launch_warp<N, false, true>(cp, B, st);
            return conj ? col_launch_warp<N, true, false>(cp, B, st) : col_launch_warp<N, false, false>(cp, B, st);
        }
    }
#define TS_COLV(EE)                                                                                             \
    if (sep) return conj ? col_launch<N, EE, true, true>(cp, B, st) : col_launch<N, EE, false, true>(cp, B, st);  \
    return conj ? col_launch<N, EE, true, false>(cp, B, st) : col_launch<N, EE, false, false>(cp, B, st);
    if constexpr (N <= 256) {
        TS_COLV(16)
    } else {
        if (E == 16) {
            TS_COLV(16)
        }
        TS_COLV(32)
    }
#undef TS_COLV
}

template <int N>
cudaError_t prepare_prop_n()
{
    if constexpr (N <= 256) {
        return prepare_prop_for<N, 16>();
    } else {
        cudaError_t e = prepare_prop_for<N, 16>();
        if (e == cudaSuccess) e = prepare_prop_for<N, 32>();
        if constexpr (N == 1024) {
            if (e == cudaSuccess) e = row_attr_shared<N, 8>();
            if (e == cudaSuccess) e = row_attr_shared<N, 4>();
            if (e == cudaSuccess) e = row_attr_shared<N, 2>();
            const int ws = (int)ColWarpCfg<N>::smem;
            if (e == cudaSuccess) e = smem_attr(col_pass_warp_kernel<N, false, false>, ws);
            if (e == cudaSuccess) e = smem_attr(col_pass_warp_kernel<N, true, false>, ws);
            if (e == cudaSuccess) e = smem_attr(col_pass_warp_kernel<N, false, true>, ws);
            if (e == cudaSuccess) e = smem_attr(col_pass_warp_kernel<N, true, true>, ws);
        }
        return e;
    }
}

}  // namespace ts
