// ts_prop_decl.h -- parameter blocks and per-N entry points of the propagation passes.
#pragma once
#include <cuda_runtime.h>

#include "ts_internal.h"

namespace ts {

struct RowParams {
    float2* field;
    const float* phi;
    const float2* phasor;
    long long phi_set_stride;
    int phi_group;
    int phi_off;     // field b of this launch uses screen set (b + phi_off) / phi_group
    int src_off;     // field b of this launch starts as source (b + src_off) mod n_src
    float phase_sign;
    float* intensity;
    double* rows;
    const float2* tw;
    int n_src;
    float src_coef[kMaxSources];
    int* err;          // device error word (set when a bounded wait of a prefetching pass runs out)
    long long budget;  // clock64 cycles such a wait may take
    int stall;         // test hook: the prefetching pass skips its first copy (its first wait runs out)
};

struct ColParams {
    float2* field;
    const float2* tw;
    const float2* P;
    float dcoef;   // exact form: dz / (2 k^3)
    float ccross;  // separable form: dz / (4 k^3)
    float inv_k2;
    float dk;
    int* err;          // device error word (set when a bounded wait of a prefetching pass runs out)
    long long budget;  // clock64 cycles such a wait may take
    bool tiny_cross;   // separable form with the cross term e <= 0.01 rad: exp(-i e) to second order
    bool first_order_cross;  // ... and e <= 4.4e-4 rad: exp(-i e) = 1 - i e (error e^2 / 2 <= 1e-7 rad)
    int stall;         // test hook: the prefetching pass skips its first copy (its first wait runs out)
    // source mode of the prefetching column pass (the first step of a call with TS_PROP_SOURCE): the
    // input R0 = FFT_rows(U0) of field b is generated in registers as the rank-one product
    // src_fx[s][kx] * src_gy[s][y], s = (b + src_off) mod n_src
    const float2* src_fx;  // [kMaxSources][N] row DFTs of the sources' x profiles (FP64-built)
    const float* src_gy;   // [kMaxSources][N] the sources' y profiles exp(-(y - N/2)^2 dx^2 / w0^2), or 1
    int n_src, src_off;
};

// Per-N entry points, instantiated in ts_prop_n<N>.cu (one translation unit per N builds in parallel).
// variant 0: each CTA reads its own screen rows; variant 1 (N = 1024, E = 32, phasor screens): the
// CTA's fields share one screen set and its phasor rows are staged once in shared memory; variant 2
// (N = 512 / 1024, E = 32, phasor screens): persistent warps that prefetch their next rows and the
// screen phasor rows with bulk asynchronous copies
template <int N>
cudaError_t row_pass_n(int E, int variant, int flags, const RowParams& rp, int B, cudaStream_t st);
// variant 0: column lines shared by several warps (block synchronisation); variant 1 (N = 1024,
// E = 32): one warp per column, tile staged through shared memory; variant 2 (N = 512 / 1024, E = 32)
// and 3 (N = 1024, E = 32): persistent CTAs whose next 64 KiB / 32 KiB tile arrives by TMA while the
// current one is transformed
template <int N>
// source = true: the first column pass of a call that starts from the sources, generating its input
// (prefetching variants only; cudaErrorNotSupported otherwise, and the caller runs the first row pass)
cudaError_t col_pass_n(int E, int variant, bool conj, bool sep, const ColParams& cp, int B, cudaStream_t st,
                       bool source);
template <int N>
cudaError_t prepare_prop_n();

// The whole propagation of B fields of N = 1024 (first row pass, S column + row passes) in one
// persistent launch (ts_prop_fused.cu).  Field b (0-based in this launch) uses screen set
// (b + phi_off) / phi_group, whose screen s is the phasor row block phasor + s N^2 + set * set_stride.
struct FusedParams {
    float2* field;           // [B][N][N] complex64, in place
    const float2* tw;        // Stockham stage twiddles (32 points per thread)
    const float4* ht;        // [S][N] (P_s(m), ky(m)^2): the separable factor of H_s and ky^2
    const float2* phasor;    // exp(i phi): screen s of set g at phasor + s N^2 + g set_stride
    long long set_stride;
    int phi_group, phi_off;
    float phase_sign;
    int S, B;
    int source;              // phase 0 generates the sources instead of reading the field
    int src_off, n_src;      // field b starts as source (b + src_off) mod n_src
    int* done;               // [(2S+1) B + 1] completed tiles per (phase, field), then the work counter
    int* head;               // set by the launcher
    int* err;
    long long budget;
    int stall;               // test hook: no input copy is issued, so the first input wait runs out
    float inv_k2;
    float ccross[kMaxScreens];
    float dcoef[kMaxScreens];
    float src_coef[kMaxSources];
};
// cudaErrorNotSupported when the arguments do not fit the fused launch (alignment, sizes)
cudaError_t prop_fused_1024(int hmode, const FusedParams& fp, cudaStream_t st);
cudaError_t prepare_prop_fused_1024();
// ht[s][m] = (P[s][m], (dk kidx(m))^2) for N = 1024
cudaError_t build_ht_table(float4* ht, const float2* P, int S, double dk, cudaStream_t st);

// the TMA-prefetching passes (ts_prop_tma.cu), N = 512 and 1024 at 32 points per thread;
// cudaErrorNotSupported when the arguments do not fit them.  w = columns per CTA (N = 1024: 8, two
// CTAs per SM, or 4, four per SM; N = 512: 16)
cudaError_t col_pass_tma(int N, int w, bool conj, int hmode, const ColParams& cp, int B, cudaStream_t st,
                         bool source = false);
cudaError_t row_pass_tma(int N, int flags, const RowParams& rp, int B, cudaStream_t st);
cudaError_t prepare_prop_tma(int N);

}  // namespace ts
