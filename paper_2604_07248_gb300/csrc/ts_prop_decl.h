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
};

struct ColParams {
    float2* field;
    const float2* tw;
    const float2* P;
    float dcoef;   // exact form: dz / (2 k^3)
    float ccross;  // separable form: dz / (4 k^3)
    float inv_k2;
    float dk;
};

// Per-N entry points, instantiated in ts_prop_n<N>.cu (one translation unit per N builds in parallel).
// variant 0: each CTA reads its own screen rows; variant 1 (N = 1024, E = 32, phasor screens): the
// CTA's fields share one screen set and its phasor rows are staged once in shared memory
template <int N>
cudaError_t row_pass_n(int E, int variant, int flags, const RowParams& rp, int B, cudaStream_t st);
// variant 0: column lines shared by several warps (block synchronisation); variant 1 (N = 1024,
// E = 32): one warp per column, tile staged through shared memory
template <int N>
cudaError_t col_pass_n(int E, int variant, bool conj, bool sep, const ColParams& cp, int B, cudaStream_t st);
template <int N>
cudaError_t prepare_prop_n();

}  // namespace ts
