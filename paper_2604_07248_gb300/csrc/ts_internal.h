// ts_internal.h -- plan layout and kernel launchers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/turbscreen.h"

namespace ts {

constexpr int kMaxScreens = 64;
constexpr int kMaxSources = 64;
constexpr int kShCoef = 27;     // 3 levels x 9 sub-grid cells (cell 4 = DC, unused)
constexpr int kShVectors = 7;   // V0, (Vc_p, Vs_p) for p = 1..3

// autotuner candidates of the propagation passes: (points per thread, column variant, row variant);
// variants other than 0 exist for N = 1024 at 32 points per thread
constexpr int kTuneCand = 8;
constexpr int kCandE[kTuneCand] = {16, 32, 32, 32, 32, 32, 32, 32};
constexpr int kCandCol[kTuneCand] = {0, 0, 1, 0, 2, 0, 2, 3};
constexpr int kCandRow[kTuneCand] = {0, 0, 0, 1, 0, 2, 2, 2};

struct Plan {
    int device = 0;
    int N = 0;
    int S = 0;
    int sh_levels = 0;
    int max_batch = 0;
    int screen_chunk = 0;  // screens per synthesis launch (workspace rows)
    double lambda = 0, n0 = 1, l0 = 0, L0 = 0, dx = 0, k = 0, dk = 0;
    double psd_alpha = 11.0 / 3.0;  // index PSD A Cn^2 (kappa^2 + kappa0^2)^(-alpha/2) exp(-kappa^2/kappa_m^2)
    double psd_A = 0.033;
    double dz[kMaxScreens] = {};
    double cn2[kMaxScreens] = {};
    int n_src = 0;
    float src_coef[kMaxSources] = {};  // dx^2 / w0^2, or -1 for a plane wave
    double loss_scale = 1.0;           // factor on the D2NN receiver loss and its gradients

    // device tables (FP64-built, FP32-stored unless noted)
    float2* tw = nullptr;      // Stockham stage twiddles, forward sign (default E for N)
    float2* tw16 = nullptr;    // the same for E = 16 (== tw when N <= 256)
    int fft_e = 32;            // points per thread of the propagation passes (16 or 32; 16 for N <= 256)
    bool split_bf16 = false;   // propagation passes on the tensor cores (split-BF16 DFTs, N = 1024)
    int* d_err = nullptr;      // device error word of the tensor-core passes (nonzero after a timeout)
    long long tc_budget = 0;   // clock64 cycles a bounded device wait may take (tensor-core and prefetching passes)
    bool test_stall = false;   // TS_PLAN_TEST_STALL: prefetching passes skip their first copy
    int tc_col_groups = 1;     // tensor-core column tiles: 1 = 4 columns (4 CTAs / SM), 2 = 8 columns (2 CTAs / SM)
    int col_variant = 0;       // column pass: 0 = lines shared by warps, 1 = one warp per column, 2 / 3 =
                               // persistent CTAs with TMA-prefetched wide / narrow tiles (N = 1024: 8 / 4
                               // columns, N = 512: 16 / 8; variant 1 at N = 1024 only; E = 32)
    int row_variant = 0;       // row pass: 0 = per-CTA screen rows, 1 = phasor rows shared by the CTA's fields,
                               // 2 = persistent warps with bulk-copy prefetch of rows and phasor rows
    float tune_us[8] = {};     // autotuner timings of one column + row pass per candidate (kCandE/Col/Row)
    int prop_groups = 1;       // field groups propagated concurrently on separate streams (1, 2 or 4)
    bool fused = false;        // ts_propagate runs the whole path as one persistent launch (N = 1024, E = 32)
    float tune_fused_us[2] = {0, 0};  // autotuner: one propagation through per-pass launches / fused launch
    float4* ht_all = nullptr;  // [S][N] (P_s, ky^2) for the fused launch (N = 1024)
    int* fused_ctr = nullptr;  // [(2S+1) max_batch + 1] completion counters and work counter of the fused launch
    float tune_group_us[3] = {0, 0, 0};  // autotuner timings for 1, 2, 4 groups
    float tune_col_us[2] = {0, 0};       // column variants 2 / 3 re-timed under the chosen field groups (0: not)
    cudaStream_t aux[3] = {nullptr, nullptr, nullptr};  // extra streams for the field groups
    cudaEvent_t fork = nullptr, join[3] = {nullptr, nullptr, nullptr};
    float2* P = nullptr;       // [S][N] exp(-i dz kappa^2 / 2k) / N (or the separable form, see sep_transfer)
    bool sep_transfer = false; // P includes the kappa^4 / 8k^3 term and kernels add the kx^2 ky^2 cross term
    bool tiny_cross = false;   // separable, and the cross term stays <= 0.01 rad on the whole grid
    bool first_order_cross = false;  // tiny_cross with e <= 4.4e-4 rad: exp(-i e) = 1 - i e (error <= 1e-7 rad)
    float* dcoef = nullptr;    // [S] dz / (2 k^3)  (non-paraxial phase correction)
    float* amp = nullptr;      // [S] sqrt(2 pi k^2 dz 0.033 Cn^2) dkappa
    float* g = nullptr;        // [N][N] (kappa^2 + kappa0^2)^(-11/12) exp(-kappa^2 / 2 kappa_m^2), g(0) = 0
    double2* shx = nullptr;    // [3][N] exp(i dkappa_p x_i), FP64
    float2* shy = nullptr;     // [3][N] (cos, sin)(dkappa_p y_j)
    double2* shy_mean = nullptr;  // [3] mean_j (cos, sin)(dkappa_p y_j), FP64
    double* shb = nullptr;     // [S][27] subharmonic amplitudes sqrt(Phi_phi) dkappa_p, FP64
    float2* tilt = nullptr;    // [2][N] AR translation factors (x then y), rebuilt per call
    float2* src_fx = nullptr;  // [kMaxSources][N] row DFT of each source's x profile (N = 512, 1024), FP64-built
    float* src_gy = nullptr;   // [kMaxSources][N] each source's y profile (N = 512, 1024), FP64-built

    // workspace
    float2* ws_y = nullptr;       // [screen_chunk][N][N] column-transformed screen spectra
    float* ws_shv = nullptr;      // [screen_chunk][7][N] subharmonic row vectors
    float* ws_shmean = nullptr;   // [screen_chunk] subharmonic piston
    double2* ws_sha = nullptr;    // [screen_chunk][27] subharmonic coefficients
    float2* ws_phi = nullptr;     // regenerated screens as exp(i phi) (phi == NULL paths): [max_batch][S][N][N]
                                  // when regen_all, else [max_batch][N][N] (one step at a time)
    bool regen_all = false;       // all S screens of a call synthesised in one launch (small workspaces)
    double* ws_rows = nullptr;    // [max_batch][N][2] per-row beam sums
    size_t bytes = 0;

    // optional per-kernel-kind event timing (kinds: 0 column pass, 1 row pass, 2 screen synthesis,
    // 3 fused propagation)
    bool timing = false;
    std::vector<cudaEvent_t> ev[4];
    int ev_used[4] = {0, 0, 0, 0};
};

// error plumbing
void set_error(const std::string& msg);
ts_status cuda_check(cudaError_t e, const char* where);

// ---- launchers (N dispatch inside) ----
// tables
cudaError_t build_tables(Plan& p);
cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int n, uint32_t* out, cudaStream_t st);
cudaError_t launch_twiddles(int N, float2* tw, cudaStream_t st);
cudaError_t launch_psd_shape(int N, float* g, double dk, double L0, double l0, cudaStream_t st);  // Kolmogorov
// one screen (no subharmonics) from caller-provided tables and intermediate buffer
cudaError_t launch_screen_raw(int N, const float2* tw, const float* g, const float* amp, float2* y, uint64_t seed,
                              int screen, uint32_t real, float* phi, cudaStream_t st);
cudaError_t build_tilt(Plan& p, double vx, double vy, double T, cudaStream_t st);

// propagation passes
enum RowFlags : int {
    RP_IN_SOURCE = 1,
    RP_IN_FREQ = 2,
    RP_PHASE = 4,
    RP_OUT_FREQ = 8,
    RP_INTENSITY = 16,
    RP_STORE = 32,
    RP_PHASOR = 64,  // modulation by precomputed exp(i phi) (complex64) instead of sincos(phi)
};
struct RowArgs {
    float2* field;
    const float* phi;          // screen s of set 0 (or nullptr)
    const float2* phasor;      // exp(i phi) of screen s of set 0 (or nullptr)
    long long phi_set_stride;  // elements between screen sets
    int phi_group;
    float phase_sign;
    const float* src_coef;     // device copy not needed: passed by value below
    float* intensity;
    double* rows;              // [B][N][2]
    int B;
    int b0;                    // index of this launch's first field in the caller's batch (sources, screen sets)
};
cudaError_t launch_row_pass(const Plan& p, int flags, const RowArgs& a, cudaStream_t st);
// split-BF16 tensor-core passes (N = 1024), see ts_tc_prop.cu
struct RowParams;
struct ColParams;
cudaError_t tc_row_pass(int flags, const RowParams& rp, int B, long long budget, int* err, cudaStream_t st);
cudaError_t tc_col_pass(int groups, bool conj, bool sep, const ColParams& cp, int B, long long budget, int* err,
                        cudaStream_t st);
cudaError_t prepare_tc_prop();
// source = true: the first column pass generates its input from the plan's sources (fields
// src_off + b), see ColParams; cudaErrorNotSupported where the kernels cannot, before any launch
cudaError_t launch_col_pass(const Plan& p, int step, bool conj, float2* field, int B, cudaStream_t st,
                            bool source = false, int src_off = 0);
cudaError_t prepare_prop_kernels(int N);
cudaError_t prepare_screen_kernels(int N);
cudaError_t launch_row_sums(const Plan& p, const double* rows, int B, double* out, cudaStream_t st);

// screens
enum ScreenMode : int { SC_INDEP = 0, SC_AR_INIT = 1, SC_AR_STEP = 2 };
struct ScreenArgs {
    uint64_t seed;
    int s_begin, s_count;      // screens s_begin .. s_begin + s_count - 1
    uint32_t r_begin;          // realizations r_begin + z / s_count
    int items;                 // s_count * realizations
    uint32_t t;                // AR step (noise tag)
    float alpha, beta;         // AR weights
    double alpha_d, beta_d;
    float2* spec;              // AR state [items][N][N]
    double2* sh_state;         // AR subharmonic state [items][27]
    float* phi;                // output [items][N][N] (or nullptr)
    float2* phasor;            // output exp(i phi) [items][N][N] (or nullptr)
    bool tilt;
    double vx, vy, T;
};
cudaError_t launch_screens(Plan& p, int mode, const ScreenArgs& a, cudaStream_t st);

// D2NN receiver
struct D2nnArgs {
    const float2* U;
    int B;
    const float* th1;
    const float* th2;
    double aperture;
    const float* Iref;
    int kind;
    float2* ws;      // [3][B][N][N]: Z1, W2, V
    float* I;
    double* loss;
    float* g_th1;
    float* g_th2;
    float2* gU;
};
cudaError_t launch_d2nn(const Plan& p, bool backward, const D2nnArgs& d, cudaStream_t st);
cudaError_t prepare_d2nn_kernels(int N);

// moments
cudaError_t launch_moments(const Plan& p, const float* I, int B, int G, int64_t count, double* mean, double* m2,
                           cudaStream_t st);
// per-group running beam sums: acc[g] (+)= sum over fields b = g mod G of (sum I, sum r^2 I)
cudaError_t launch_beam_acc(const double* beam_sums, int B, int G, bool first, double* acc, cudaStream_t st);
cudaError_t launch_moments_finalize(const Plan& p, const double* mean, const double* m2, int G, int64_t count,
                                    double* si_map, double* si_mean, double* si_center, cudaStream_t st);
// w_lt[g] = sqrt(2 acc[g][1] / acc[g][0])
cudaError_t launch_w_lt(const double* acc, int G, double* w_lt, cudaStream_t st);

}  // namespace ts
