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
    int stall;         // test hook: the prefetching pass skips its first copy (its first wait runs out)
};

// Per-N entry points, instantiated in ts_prop_n<N>.cu (one translation unit per N builds in parallel).
// variant 0: each CTA reads its own screen rows; variant 1 (N = 1024, E = 32, phasor screens): the
// CTA's fields share one screen set and its phasor rows are staged once in shared memory; variant 2
// (N = 1024, E = 32, phasor screens): persistent warps that prefetch their next row and the screen
// phasor row with bulk asynchronous copies
template <int N>
cudaError_t row_pass_n(int E, int variant, int flags, const RowParams& rp, int B, cudaStream_t st);
// variant 0: column lines shared by several warps (block synchronisation); variant 1 (N = 1024,
// E = 32): one warp per column, tile staged through shared memory; variant 2 (N = 1024, E = 32):
// persistent CTAs whose next 8-column tile arrives by TMA while the current one is transformed
template <int N>
cudaError_t col_pass_n(int E, int variant, bool conj, bool sep, const ColParams& cp, int B, cudaStream_t st);
template <int N>
cudaError_t prepare_prop_n();

// the TMA-prefetching passes (ts_prop_tma.cu); cudaErrorNotSupported when the arguments do not fit them
cudaError_t col_pass_tma_1024(bool conj, int hmode, const ColParams& cp, int B, cudaStream_t st);
cudaError_t row_pass_tma_1024(int flags, const RowParams& rp, int B, cudaStream_t st);
cudaError_t prepare_prop_tma_1024();

}  // namespace ts
