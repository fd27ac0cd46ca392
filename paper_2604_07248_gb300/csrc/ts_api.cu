// ts_api.cu -- the C ABI (include/turbscreen.h): argument checks, plan construction and the
// launch sequences of the split-step path.  Every numeric step runs in the library's kernels; the
// host computes only per-plan scalars (amplitudes, limits) in FP64.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "ts_internal.h"
#include "ts_prop_decl.h"

namespace ts {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

ts_status cuda_check(cudaError_t e, const char* where)
{
    if (e == cudaSuccess) return TS_OK;
    set_error(std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return TS_ERR_CUDA;
}

namespace {

ts_status fail(ts_status st, const std::string& msg)
{
    set_error(msg);
    return st;
}

// Every call that launches work or touches the plan's memory runs on the device the plan was created
// on: the kernels receive raw pointers into that device's memory, so a call made while another device
// is current would hand them addresses they cannot reach.
ts_status check_device(const Plan& p, const char* where)
{
    int dev = -1;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, where);
    if (dev != p.device)
        return fail(TS_ERR_INVALID_ARG, std::string(where) + ": the plan lives on device " + std::to_string(p.device) +
                                            " but device " + std::to_string(dev) + " is current");
    return TS_OK;
}

bool supported_N(int N) { return N == 128 || N == 256 || N == 512 || N == 1024 || N == 2048; }

double wavenumber(const ts_medium* m) { return 2.0 * M_PI * m->n0 / m->lambda; }

// Phi_phi(kappa) = 2 pi k^2 dz A Cn^2 (kappa^2 + kappa0^2)^(-alpha/2) exp(-kappa^2 / kappa_m^2)
// (S14, S17; A = 0.033 and alpha = 11/3 for Kolmogorov, the power law of another medium per S12, S15)
double phase_psd(const Plan& p, double cn2, double dz, double k2)
{
    const double k0sq = (p.L0 > 0.0 && std::isfinite(p.L0)) ? std::pow(2.0 * M_PI / p.L0, 2.0) : 0.0;
    const double roll = p.l0 > 0.0 ? std::exp(-k2 / std::pow(2.0 * M_PI / p.l0, 2.0)) : 1.0;
    return 2.0 * M_PI * p.k * p.k * dz * p.psd_A * cn2 * std::pow(k2 + k0sq, -p.psd_alpha / 2.0) * roll;
}

template <class T>
cudaError_t dalloc(Plan& p, T** ptr, size_t count)
{
    const size_t bytes = sizeof(T) * (count > 0 ? count : 1);
    cudaError_t e = cudaMalloc((void**)ptr, bytes);
    if (e == cudaSuccess) p.bytes += bytes;
    return e;
}

void destroy_events(Plan* p)
{
    for (auto& v : p->ev) {
        for (cudaEvent_t e : v) cudaEventDestroy(e);
        v.clear();
    }
    for (int& u : p->ev_used) u = 0;
}

// Runs `launch` between two recorded events when timing is on and events remain for `kind`.
template <class F>
cudaError_t timed(Plan& p, int kind, cudaStream_t st, F&& launch)
{
    const int u = p.ev_used[kind];
    const bool on = p.timing && 2 * (u + 1) <= (int)p.ev[kind].size();
    if (on) cudaEventRecord(p.ev[kind][2 * u], st);
    cudaError_t e = launch();
    if (on) {
        cudaEventRecord(p.ev[kind][2 * u + 1], st);
        p.ev_used[kind] = u + 1;
    }
    return e;
}

void free_plan(Plan* p)
{
    destroy_events(p);
    for (int i = 0; i < 3; ++i) {
        if (p->aux[i]) cudaStreamDestroy(p->aux[i]);
        if (p->join[i]) cudaEventDestroy(p->join[i]);
    }
    if (p->fork) cudaEventDestroy(p->fork);
    void* ptrs[] = {p->tw,  p->P,    p->dcoef, p->amp,       p->g,         p->shx,      p->shy,    p->shy_mean,
                    p->shb, p->tilt, p->ws_y,  p->ws_shv,    p->ws_shmean, p->ws_sha,   p->ws_phi, p->ws_rows,
                    p->tw16 != p->tw ? p->tw16 : nullptr, p->d_err, p->ht_all, p->fused_ctr, p->src_fx, p->src_gy};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete p;
}

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// regenerate screen `s` of the G screen sets (realizations real_base .. real_base + G - 1) into ws_phi,
// or (s < 0, regen_all plans) all S screens of the G sets at once, ws_phi laid out [G][S][N][N]
ts_status regen_screen(Plan& p, uint64_t seed, uint32_t real_base, int G, int s, cudaStream_t st)
{
    ScreenArgs a{};
    a.seed = seed;
    a.s_begin = s < 0 ? 0 : s;
    a.s_count = s < 0 ? p.S : 1;
    a.r_begin = real_base;
    a.items = G * a.s_count;
    a.t = 0;
    a.phi = nullptr;
    a.phasor = p.ws_phi;
    return cuda_check(timed(p, 2, st, [&] { return launch_screens(p, SC_INDEP, a, st); }), "screen synthesis");
}

int rows_per_line(const Plan& p)
{
    const int T = p.N / (p.N <= 256 ? 16 : p.fft_e);
    return T > 32 ? T / 32 : 1;
}

// Eq. 1 over the plan's S steps for fields [b0, b0 + B) of the caller's batch U, on one stream.
ts_status prop_range(Plan& p, float2* U, int b0, int B, const float* phi, const void* phasor, int phi_group, int flags,
                     uint64_t seed, uint32_t real_base, float* intensity, double* rows, cudaStream_t st)
{
    const int N = p.N, S = p.S;
    const size_t N2 = (size_t)N * N;
    const int G = (B + phi_group - 1) / phi_group;
    float2* Ur = U + (size_t)b0 * N2;
    const size_t set0 = (size_t)(b0 / phi_group) * S * N2;  // first screen set of the range
    RowArgs ra{};
    ra.field = Ur;
    ra.phi_group = phi_group;
    ra.phase_sign = 1.0f;
    ra.B = B;
    ra.b0 = b0;
    const bool aligned = (reinterpret_cast<uintptr_t>(U) & 15) == 0 && (reinterpret_cast<uintptr_t>(phasor) & 15) == 0;
    if (p.fused && aligned && !(flags & TS_PROP_INTENSITY) && (phasor || (!phi && p.regen_all))) {
        // the whole path in one persistent launch
        const uint32_t rb = real_base + (uint32_t)(b0 / phi_group);
        FusedParams fp{};
        fp.field = Ur;
        fp.tw = p.tw;
        fp.ht = p.ht_all;
        if (phasor) {
            fp.phasor = reinterpret_cast<const float2*>(phasor) + set0;
            fp.phi_off = b0 % phi_group;
        } else {
            ts_status sr = regen_screen(p, seed, rb, G, -1, st);
            if (sr != TS_OK) return sr;
            fp.phasor = p.ws_phi;
            fp.phi_off = b0 % phi_group;
        }
        fp.set_stride = (long long)S * N2;
        fp.phi_group = phi_group;
        fp.phase_sign = 1.0f;
        fp.S = S;
        fp.B = B;
        fp.source = (flags & TS_PROP_SOURCE) ? 1 : 0;
        fp.src_off = b0;
        fp.n_src = p.n_src > 0 ? p.n_src : 1;
        fp.done = p.fused_ctr;
        fp.err = p.d_err;
        fp.budget = p.tc_budget;
        fp.stall = p.test_stall ? 1 : 0;
        fp.inv_k2 = (float)(1.0 / (p.k * p.k));
        for (int s = 0; s < S; ++s) {
            fp.ccross[s] = (float)(p.dz[s] / (4.0 * p.k * p.k * p.k));
            fp.dcoef[s] = (float)(p.dz[s] / (2.0 * p.k * p.k * p.k));
        }
        for (int i = 0; i < kMaxSources; ++i) fp.src_coef[i] = i < p.n_src ? p.src_coef[i] : -1.0f;
        const int hmode = p.sep_transfer ? (p.tiny_cross ? 2 : 1) : 0;
        cudaError_t e = cudaErrorNotSupported;
        ts_status sf = cuda_check(timed(p, 3, st, [&] { return e = prop_fused_1024(hmode, fp, st); }),
                                  "ts_propagate fused launch");
        if (e != cudaErrorNotSupported) return sf;
        set_error("");  // arguments the fused launch does not take: per-pass launches below
    }
    const int f0 = ((flags & TS_PROP_SOURCE) ? RP_IN_SOURCE : 0) | RP_OUT_FREQ | RP_STORE;
    // With sources, the prefetching column pass generates the row transform of each source in its
    // first step (a rank-one product), so the first row pass is not needed
    bool src_in_col = (flags & TS_PROP_SOURCE) && p.src_fx && !p.split_bf16 && p.fft_e == 32 &&
                      (p.col_variant == 2 || p.col_variant == 3) && (p.N == 512 || p.N == 1024) &&
                      (reinterpret_cast<uintptr_t>(Ur) & 15) == 0;
    ts_status stt = TS_OK;
    if (!src_in_col) {
        stt = cuda_check(timed(p, 1, st, [&] { return launch_row_pass(p, f0, ra, st); }), "ts_propagate first row pass");
        if (stt != TS_OK) return stt;
    }
    for (int s = 0; s < S; ++s) {
        const bool src = src_in_col && s == 0;
        cudaError_t ec = timed(p, 0, st, [&] { return launch_col_pass(p, s, false, Ur, B, st, src, b0); });
        if (src && ec == cudaErrorNotSupported) {  // the kernels could not take it after all: row pass first
            (void)cudaGetLastError();
            ec = timed(p, 1, st, [&] { return launch_row_pass(p, f0, ra, st); });
            if (ec == cudaSuccess) ec = timed(p, 0, st, [&] { return launch_col_pass(p, s, false, Ur, B, st); });
        }
        stt = cuda_check(ec, "ts_propagate column pass");
        if (stt != TS_OK) return stt;
        int rf = RP_IN_FREQ | RP_STORE;
        ra.phi = nullptr;
        ra.phasor = nullptr;
        ra.phi_set_stride = (long long)S * N2;
        if (phasor) {
            ra.phasor = reinterpret_cast<const float2*>(phasor) + set0 + (size_t)s * N2;
            rf |= RP_PHASOR;
        } else if (phi) {
            ra.phi = phi + set0 + (size_t)s * N2;
            rf |= RP_PHASE;
        } else {
            // regenerated screens: one per screen set of this range, realizations real_base + set index;
            // all S of them in one synthesis launch when the workspace holds them, else step by step
            const uint32_t rb = real_base + (uint32_t)(b0 / phi_group);
            if (p.regen_all) {
                if (s == 0 && (stt = regen_screen(p, seed, rb, G, -1, st)) != TS_OK) return stt;
                ra.phasor = p.ws_phi + (size_t)s * N2;
                ra.phi_set_stride = (long long)S * N2;
            } else {
                if ((stt = regen_screen(p, seed, rb, G, s, st)) != TS_OK) return stt;
                ra.phasor = p.ws_phi;
                ra.phi_set_stride = (long long)N2;
            }
            ra.b0 = b0 % phi_group;  // sets counted from this range's first set
            rf |= RP_PHASOR;
        }
        if (s < S - 1) {
            rf |= RP_OUT_FREQ;
        } else if (flags & TS_PROP_INTENSITY) {
            rf |= RP_INTENSITY;
            if (flags & TS_PROP_NO_FIELD) rf &= ~RP_STORE;
            ra.intensity = intensity + (size_t)b0 * N2;
            ra.rows = rows ? rows + (size_t)b0 * N * rows_per_line(p) * 2 : nullptr;
        }
        stt = cuda_check(timed(p, 1, st, [&] { return launch_row_pass(p, rf, ra, st); }), "ts_propagate row pass");
        ra.b0 = b0;
        if (stt != TS_OK) return stt;
    }
    return TS_OK;
}

// Eq. 1 for the whole batch.  With the screens given, the fields split into groups propagated
// concurrently on the plan's extra streams (fork / join through events, so the call stays asynchronous
// and capturable): one group's partial last waves overlap another's kernels.  Regenerated screens share
// one workspace, and the fused persistent launch fills the GPU by itself: no split.
ts_status propagate_groups(Plan& p, float2* U, int B, const float* phi, const void* phasor, int phi_group, int flags,
                           uint64_t seed, uint32_t real_base, float* intensity, double* rows, cudaStream_t st)
{
    const bool fused_call = p.fused && !(flags & TS_PROP_INTENSITY);
    const int groups = ((phi || phasor) && !fused_call) ? std::min(p.prop_groups, B) : 1;
    ts_status stt = TS_OK;
    if (groups <= 1) return prop_range(p, U, 0, B, phi, phasor, phi_group, flags, seed, real_base, intensity, rows, st);
    stt = cuda_check(cudaEventRecord(p.fork, st), "ts_propagate fork");
    for (int g = 1; g < groups && stt == TS_OK; ++g)
        stt = cuda_check(cudaStreamWaitEvent(p.aux[g - 1], p.fork, 0), "ts_propagate fork");
    const int per = (B + groups - 1) / groups;
    for (int g = 0; g < groups && stt == TS_OK; ++g) {
        const int b0 = g * per, bg = std::min(per, B - b0);
        if (bg <= 0) break;
        stt = prop_range(p, U, b0, bg, phi, phasor, phi_group, flags, seed, real_base, intensity, rows,
                         g == 0 ? st : p.aux[g - 1]);
    }
    for (int g = 1; g < groups && stt == TS_OK; ++g) {
        stt = cuda_check(cudaEventRecord(p.join[g - 1], p.aux[g - 1]), "ts_propagate join");
        if (stt == TS_OK) stt = cuda_check(cudaStreamWaitEvent(st, p.join[g - 1], 0), "ts_propagate join");
    }
    return stt;
}

// Autotuner: for N >= 512 the propagation passes exist with E = 16 and E = 32 points per thread
// (different register / occupancy / exchange trade-offs).  Each candidate runs one column pass and
// one middle row pass on B_t workspace fields (2 warm-up + 5 timed repetitions, CUDA events), in
// kTuneRounds interleaved rounds over the candidates; each candidate's fastest round counts, so a
// transient (clocks still ramping at the first launches, a co-tenant's burst) cannot decide the
// choice.  Results are cached per (device, N, B_t, transfer form); TS_FFT_E=16|32 forces a choice.
constexpr int kTuneRounds = 3;
// fields per timed pass in the first two stages: the plan's batch up to 32 (a plan for many fields,
// e.g. 64 Monte Carlo beams at N = 512, is timed at a batch that behaves like its own; the
// workspace holds screen_chunk >= this many fields)
constexpr int kTuneBatch = 32;
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tune_cache;

ts_status autotune(Plan& p)
{
    p.col_variant = 0;
    p.row_variant = 0;
    if (p.split_bf16) {
        p.fft_e = 32;  // the tensor-core passes have one configuration
        return TS_OK;
    }
    if (p.N <= 256) {
        p.fft_e = 16;
        return TS_OK;
    }
    // candidates (points per thread, column variant, row variant), filtered by TS_FFT_E / TS_COL_VARIANT /
    // TS_ROW_VARIANT; the variants other than 0 exist at 32 points per thread, for N = 1024 (and the
    // prefetching variants 2 for N = 512)
    int force_e = 0, force_v = -1, force_r = -1;
    if (const char* env = std::getenv("TS_FFT_E")) force_e = std::atoi(env);
    if (const char* env = std::getenv("TS_COL_VARIANT")) force_v = std::atoi(env);
    if (const char* env = std::getenv("TS_ROW_VARIANT")) force_r = std::atoi(env);
    constexpr int kCand = kTuneCand;
    const int *cand_e = kCandE, *cand_v = kCandCol, *cand_r = kCandRow;
    bool use[kCand];
    int n_use = 0, only = -1;
    for (int c = 0; c < kCand; ++c) {
        // column variant 1 and row variant 1 exist for N = 1024, the prefetching column variants 2 and 3
        // (wide and narrow tiles) and row variant 2 for N = 512 and 1024
        const bool avail_v = cand_v[c] == 0 || p.N == 1024 || ((cand_v[c] == 2 || cand_v[c] == 3) && p.N == 512);
        const bool avail_r = cand_r[c] == 0 || p.N == 1024 || (cand_r[c] == 2 && p.N == 512);
        use[c] = (force_e == 0 || force_e == cand_e[c]) && (force_v < 0 || force_v == cand_v[c]) &&
                 (force_r < 0 || force_r == cand_r[c]) && avail_v && avail_r;
        if (use[c]) {
            ++n_use;
            only = c;
        }
    }
    if (n_use == 0) {  // an unavailable forced combination: keep the forced points per thread
        p.fft_e = (force_e == 16 || force_e == 32) ? force_e : 32;
        return TS_OK;
    }
    if (n_use == 1) {
        p.fft_e = cand_e[only];
        p.col_variant = cand_v[only];
        p.row_variant = cand_r[only];
        return TS_OK;
    }
    const size_t N2 = (size_t)p.N * p.N;
    const int Bt = std::max(1, std::min(std::min(p.max_batch, p.screen_chunk), kTuneBatch));
    const auto key =
        std::make_tuple(p.device, p.N, Bt, (p.sep_transfer ? 1 : 0) + 2 * (force_e + 64 * (force_v + 1) + 256 * (force_r + 1)));
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            p.fft_e = cand_e[it->second];
            p.col_variant = cand_v[it->second];
            p.row_variant = cand_r[it->second];
            return TS_OK;
        }
    }
    cudaError_t e = cudaMemset(p.ws_y, 0, sizeof(float2) * N2 * Bt);
    if (e == cudaSuccess) e = cudaMemset(p.ws_phi, 0, sizeof(float2) * N2);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float t_min[kCand];
    for (int c = 0; c < kCand; ++c) t_min[c] = 1e30f;
    for (int rd = 0; rd < kTuneRounds && e == cudaSuccess; ++rd) {
        for (int c = 0; c < kCand && e == cudaSuccess; ++c) {
            if (!use[c]) continue;
            p.fft_e = cand_e[c];
            p.col_variant = cand_v[c];
            p.row_variant = cand_r[c];
            RowArgs ra{};
            ra.field = p.ws_y;
            ra.phasor = p.ws_phi;
            ra.phi_set_stride = 0;
            ra.phi_group = Bt;
            ra.phase_sign = 1.0f;
            ra.B = Bt;
            auto once = [&]() {
                cudaError_t x = launch_col_pass(p, 0, false, p.ws_y, Bt, nullptr);
                if (x == cudaSuccess)
                    x = launch_row_pass(p, RP_IN_FREQ | RP_PHASOR | RP_OUT_FREQ | RP_STORE, ra, nullptr);
                return x;
            };
            for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = once();
            if (e == cudaSuccess) e = cudaEventRecord(e0, nullptr);
            for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = once();
            if (e == cudaSuccess) e = cudaEventRecord(e1, nullptr);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess) t_min[c] = std::min(t_min[c], ms * 1000.0f / 5.0f);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_check(e, "ts_plan_create autotune");
    float best = 1e30f;
    int best_c = 1;
    for (int c = 0; c < kCand; ++c) {
        if (!use[c]) continue;
        p.tune_us[c] = t_min[c];
        if (t_min[c] < best) {
            best = t_min[c];
            best_c = c;
        }
    }
    p.fft_e = cand_e[best_c];
    p.col_variant = cand_v[best_c];
    p.row_variant = cand_r[best_c];
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best_c;
    return TS_OK;
}

// Second autotuner stage: how many field groups to propagate concurrently (1, 2 or 4 streams), timed
// as runs of four column + row pass pairs of B_t workspace fields per fork (the reported cost is per
// pair).  Then, when that is two or more groups at N = 512 or 1024 with a prefetching column variant
// (wide or narrow tiles: 16 / 8 columns at N = 512, 8 / 4 at 1024), both column variants are timed
// again the same way with that many groups: on one
// stream the two come within a few per cent of each other (so the first stage's pick between them
// follows noise), while under concurrent groups they differ, so the column variant is taken from
// this timing (the other one replaces the first stage's pick only when at least 1 % faster).  Cached
// like the first stage; TS_PROP_STREAMS=1|2|4 forces the group count and skips both timings,
// TS_COL_VARIANT skips the second.
struct GroupChoice {
    int groups;
    int col_variant;  // -1: the first stage's pick stands
    float us_cols[2];  // cost per pass pair of column variant 2 / 3 with `groups` groups (0: not timed)
};
std::map<std::tuple<int, int, int, int, int>, GroupChoice> g_group_cache;
constexpr int kTuneSteps = 4;  // column + row pass pairs per fork in the group timing

ts_status autotune_groups(Plan& p)
{
    p.prop_groups = 1;
    const int Bt = std::max(1, std::min(std::min(p.max_batch, p.screen_chunk), kTuneBatch));
    if (Bt < 2) return TS_OK;
    if (const char* env = std::getenv("TS_PROP_STREAMS")) {
        const int g = std::atoi(env);
        if (g == 1 || g == 2 || g == 4) {
            p.prop_groups = std::min(g, Bt);
            return TS_OK;
        }
    }
    const auto key = std::make_tuple(p.device, p.N, Bt, p.sep_transfer ? 1 : 0,
                                     p.split_bf16 ? -1 : p.fft_e + 1000 * p.col_variant + 2000 * p.row_variant);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_group_cache.find(key);
        if (it != g_group_cache.end()) {
            p.prop_groups = it->second.groups;
            if (it->second.col_variant >= 0) p.col_variant = it->second.col_variant;
            p.tune_col_us[0] = it->second.us_cols[0];  // the timings the cached choice was made on
            p.tune_col_us[1] = it->second.us_cols[1];
            return TS_OK;
        }
    }
    const size_t N2 = (size_t)p.N * p.N;
    cudaError_t e = cudaMemset(p.ws_y, 0, sizeof(float2) * N2 * Bt);
    if (e == cudaSuccess) e = cudaMemset(p.ws_phi, 0, sizeof(float2) * N2);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const int cand[3] = {1, 2, 4};
    float t_min[3] = {1e30f, 1e30f, 1e30f};
    // microseconds per column + row pass pair of `groups` concurrent groups (2 warm-up + 5 timed runs)
    auto time_groups = [&](int groups, float& us) {
        auto once = [&]() {
            cudaError_t x = cudaEventRecord(p.fork, nullptr);
            for (int g = 1; g < groups && x == cudaSuccess; ++g) x = cudaStreamWaitEvent(p.aux[g - 1], p.fork, 0);
            const int per = (Bt + groups - 1) / groups;
            for (int g = 0; g < groups && x == cudaSuccess; ++g) {
                const int b0 = g * per, bg = std::min(per, Bt - b0);
                if (bg <= 0) break;
                cudaStream_t st = g == 0 ? nullptr : p.aux[g - 1];
                RowArgs ra{};
                ra.field = p.ws_y + (size_t)b0 * N2;
                ra.phasor = p.ws_phi;
                ra.phi_group = Bt;
                ra.phase_sign = 1.0f;
                ra.B = bg;
                ra.b0 = b0;
                // a run of steps per fork, as in ts_propagate: the groups overlap in the steady state
                for (int s = 0; s < kTuneSteps && x == cudaSuccess; ++s) {
                    x = launch_col_pass(p, 0, false, ra.field, bg, st);
                    if (x == cudaSuccess) x = launch_row_pass(p, RP_IN_FREQ | RP_PHASOR | RP_OUT_FREQ | RP_STORE, ra, st);
                }
            }
            for (int g = 1; g < groups && x == cudaSuccess; ++g) {
                x = cudaEventRecord(p.join[g - 1], p.aux[g - 1]);
                if (x == cudaSuccess) x = cudaStreamWaitEvent(nullptr, p.join[g - 1], 0);
            }
            return x;
        };
        for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = once();
        if (e == cudaSuccess) e = cudaEventRecord(e0, nullptr);
        for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = once();
        if (e == cudaSuccess) e = cudaEventRecord(e1, nullptr);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess) us = std::min(us, ms * 1000.0f / (5.0f * kTuneSteps));
    };
    for (int rd = 0; rd < kTuneRounds * 3 && e == cudaSuccess; ++rd) {  // interleaved rounds, as above
        const int c = rd % 3;
        if (cand[c] <= Bt) time_groups(cand[c], t_min[c]);
    }
    float best = 1e30f;
    int best_g = 1;
    for (int c = 0; c < 3 && cand[c] <= Bt && e == cudaSuccess; ++c) {
        p.tune_group_us[c] = t_min[c];
        if (t_min[c] < best * 0.97f) {  // prefer fewer streams unless 3 % faster
            best = t_min[c];
            best_g = cand[c];
        }
    }
    p.prop_groups = best_g;
    // the column tiles under the chosen concurrency
    GroupChoice gc{best_g, -1, {0.0f, 0.0f}};
    const bool retime = e == cudaSuccess && best_g >= 2 && (p.N == 1024 || p.N == 512) && p.fft_e == 32 && !p.split_bf16 &&
                        (p.col_variant == 2 || p.col_variant == 3) && std::getenv("TS_COL_VARIANT") == nullptr;
    if (retime) {
        const int first = p.col_variant;
        float us[2] = {1e30f, 1e30f};
        for (int rd = 0; rd < kTuneRounds * 2 && e == cudaSuccess; ++rd) {
            p.col_variant = 2 + rd % 2;
            time_groups(best_g, us[rd % 2]);
        }
        const int other = first == 2 ? 3 : 2;
        p.col_variant = (e == cudaSuccess && us[other - 2] < 0.99f * us[first - 2]) ? other : first;
        if (e == cudaSuccess) gc = GroupChoice{best_g, p.col_variant, {us[0], us[1]}};
        p.tune_col_us[0] = gc.us_cols[0];
        p.tune_col_us[1] = gc.us_cols[1];
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_check(e, "ts_plan_create autotune (groups)");
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_group_cache[key] = gc;
    return TS_OK;
}

// Third autotuner stage (N = 1024, 32 points per thread, FP32 passes): one propagation of B_t
// workspace fields through the plan's S steps, by per-pass launches (the variants and field groups
// chosen above) or as one fused persistent launch; the fused launch is kept when it is faster.
// Cached like the other stages; TS_FUSED=0|1 forces a choice.
std::map<std::tuple<int, int, int, int, int, int>, int> g_fused_cache;

ts_status autotune_fused(Plan& p)
{
    p.fused = false;
    if (p.N != 1024 || p.fft_e != 32 || p.split_bf16 || !p.ht_all || !p.fused_ctr) return TS_OK;
    if (const char* env = std::getenv("TS_FUSED")) {
        p.fused = std::atoi(env) != 0;
        return TS_OK;
    }
    const int Bt = std::max(1, std::min(std::min(p.max_batch, p.screen_chunk), 8));
    const size_t N2 = (size_t)p.N * p.N;
    const auto key = std::make_tuple(p.device, p.N, Bt, p.S, (p.sep_transfer ? 1 : 0) + (p.tiny_cross ? 2 : 0),
                                     p.col_variant + 8 * p.row_variant + 64 * p.prop_groups);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_fused_cache.find(key);
        if (it != g_fused_cache.end()) {
            p.fused = it->second != 0;
            return TS_OK;
        }
    }
    // fields in ws_phi (>= max_batch N^2), the S phasor screens of one set in ws_y (>= S N^2)
    float2* U = p.ws_phi;
    const float2* ph = p.ws_y;
    cudaError_t e = cudaMemset(p.ws_y, 0, sizeof(float2) * N2 * p.S);
    if (e == cudaSuccess) e = cudaMemset(p.ws_phi, 0, sizeof(float2) * N2 * Bt);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_check(e, "ts_plan_create autotune (fused)");
    ts_status stt = TS_OK;
    p.tune_fused_us[0] = p.tune_fused_us[1] = 1e30f;
    for (int rd = 0; rd < kTuneRounds * 2 && stt == TS_OK; ++rd) {  // interleaved rounds, as above
        const int c = rd % 2;
        p.fused = c == 1;
        auto once = [&]() { return propagate_groups(p, U, Bt, nullptr, ph, Bt, 0, 0, 0, nullptr, nullptr, nullptr); };
        for (int w = 0; w < 2 && stt == TS_OK; ++w) stt = once();
        if (stt == TS_OK) stt = cuda_check(cudaEventRecord(e0, nullptr), "autotune (fused)");
        for (int r = 0; r < 5 && stt == TS_OK; ++r) stt = once();
        if (stt == TS_OK) stt = cuda_check(cudaEventRecord(e1, nullptr), "autotune (fused)");
        if (stt == TS_OK) stt = cuda_check(cudaEventSynchronize(e1), "autotune (fused)");
        float ms = 0.0f;
        if (stt == TS_OK) stt = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "autotune (fused)");
        if (stt == TS_OK) p.tune_fused_us[c] = std::min(p.tune_fused_us[c], ms * 1000.0f / 5.0f);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (stt != TS_OK) {
        p.fused = false;
        return stt;
    }
    {
        int code = 0;  // a fused launch whose bounded waits ran out is never chosen
        cudaError_t x = cudaMemcpy(&code, p.d_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (x == cudaSuccess && code != 0) x = cudaMemset(p.d_err, 0, sizeof(int));
        if (x != cudaSuccess) return cuda_check(x, "ts_plan_create autotune (fused)");
        p.fused = code == 0 && p.tune_fused_us[1] < p.tune_fused_us[0];
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_fused_cache[key] = p.fused ? 1 : 0;
    return TS_OK;
}

}  // namespace
}  // namespace ts

using namespace ts;

extern "C" {

const char* ts_status_string(ts_status s)
{
    switch (s) {
    case TS_OK: return "ok";
    case TS_ERR_INVALID_ARG: return "invalid argument";
    case TS_ERR_ALIASING: return "step exceeds the angular-spectrum aliasing limit (Eq. 7)";
    case TS_ERR_WORKSPACE: return "request exceeds the plan workspace";
    case TS_ERR_CUDA: return "CUDA error";
    case TS_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
    case TS_ERR_UNSUPPORTED: return "unsupported size or regime";
    }
    return "unknown status";
}

const char* ts_last_error(void) { return g_last_error.c_str(); }

double ts_max_step(const ts_medium* m, const ts_grid* g)
{
    if (!m || !g || g->N <= 0 || !(g->dx > 0.0) || !(m->lambda > 0.0) || !(m->n0 > 0.0)) return -1.0;
    const double k = wavenumber(m);
    const double kmax = M_PI / g->dx;
    if (kmax >= k) return 0.0;
    return 0.5 * g->N * g->dx * std::sqrt(k * k - kmax * kmax) / kmax;
}

double ts_power_law_constant(double alpha)
{
    if (!(alpha > 3.0 && alpha < 5.0)) return std::nan("");
    return std::tgamma(alpha - 1.0) * std::cos(M_PI * alpha / 2.0) / (4.0 * M_PI * M_PI);
}

ts_status ts_plan_create(ts_plan* out, const ts_medium* medium, const ts_grid* grid, const ts_path* path,
                         int sh_levels, int max_batch, int flags)
{
    return ts_plan_create_psd(out, medium, grid, path, sh_levels, max_batch, flags, 11.0 / 3.0, 0.033);
}

ts_status ts_plan_create_psd(ts_plan* out, const ts_medium* medium, const ts_grid* grid, const ts_path* path,
                             int sh_levels, int max_batch, int flags, double alpha, double A)
{
    set_error("");
    if (out) *out = nullptr;
    if (!(alpha > 3.0 && alpha < 5.0) || !(A > 0.0) || !std::isfinite(A))
        return fail(TS_ERR_INVALID_ARG, "power law alpha must lie in (3, 5) and A must be finite and > 0");
    if (!out || !medium || !grid || !path) return fail(TS_ERR_INVALID_ARG, "null pointer argument");
    *out = nullptr;
    if (!supported_N(grid->N)) return fail(TS_ERR_INVALID_ARG, "N must be one of 128, 256, 512, 1024, 2048");
    if (!(grid->dx > 0.0) || !(medium->lambda > 0.0) || !(medium->n0 > 0.0))
        return fail(TS_ERR_INVALID_ARG, "dx, lambda and n0 must be positive");
    if (path->n_screens < 1 || path->n_screens > kMaxScreens || !path->dz || !path->cn2)
        return fail(TS_ERR_INVALID_ARG, "path needs 1..64 screens with dz and cn2 arrays");
    if (sh_levels != 0 && sh_levels != 3) return fail(TS_ERR_INVALID_ARG, "sh_levels must be 0 or 3");
    if (max_batch < 1) return fail(TS_ERR_INVALID_ARG, "max_batch must be >= 1");
    if ((flags & TS_PLAN_SPLIT_BF16) && grid->N != 1024)
        return fail(TS_ERR_UNSUPPORTED, "TS_PLAN_SPLIT_BF16 is implemented for N = 1024 (32 x 32 tensor-core DFTs)");

    Plan tmp;
    tmp.psd_alpha = alpha;
    tmp.psd_A = A;
    tmp.N = grid->N;
    tmp.dx = grid->dx;
    tmp.S = path->n_screens;
    tmp.sh_levels = sh_levels;
    tmp.max_batch = max_batch;
    tmp.lambda = medium->lambda;
    tmp.n0 = medium->n0;
    tmp.l0 = medium->l0;
    tmp.L0 = medium->L0;
    tmp.k = wavenumber(medium);
    tmp.dk = 2.0 * M_PI / (grid->N * grid->dx);
    tmp.split_bf16 = (flags & TS_PLAN_SPLIT_BF16) != 0;
    const double dzmax = ts_max_step(medium, grid);
    const double kap2max = 2.0 * std::pow(M_PI / grid->dx, 2.0);
    for (int s = 0; s < tmp.S; ++s) {
        const double dz = path->dz[s], cn2 = path->cn2[s];
        if (!(dz > 0.0) || !(cn2 >= 0.0) || !std::isfinite(dz) || !std::isfinite(cn2))
            return fail(TS_ERR_INVALID_ARG, "dz must be > 0 and cn2 >= 0");
        if (!(flags & TS_PLAN_ALLOW_ALIASING) && dz > dzmax) {
            char buf[160];
            snprintf(buf, sizeof buf, "step %d: dz = %g m exceeds the Eq. 7 limit %g m", s, dz, dzmax);
            return fail(TS_ERR_ALIASING, buf);
        }
        if (kap2max >= tmp.k * tmp.k) return fail(TS_ERR_UNSUPPORTED, "grid reaches the evanescent region");
        const double root = std::sqrt(tmp.k * tmp.k - kap2max);
        const double delta = dz * kap2max * kap2max / (2.0 * tmp.k * (tmp.k + root) * (tmp.k + root));
        if (delta > 0.25)
            return fail(TS_ERR_UNSUPPORTED, "non-paraxial phase correction above 0.25 rad at the grid corner");
        tmp.dz[s] = dz;
        tmp.cn2[s] = cn2;
    }
    // separable transfer function when the dropped terms are negligible for every step:
    // dz kappa^6 / 16k^5 <= 1e-7 rad and the cross term dz kx^2 ky^2 / 4k^3 <= 0.05 rad
    {
        bool sep = true, tiny = true, first = true;
        const double kx2 = std::pow(M_PI / grid->dx, 2.0), k = tmp.k;
        for (int s = 0; s < tmp.S; ++s) {
            const double r6 = tmp.dz[s] * kap2max * kap2max * kap2max / (16.0 * std::pow(k, 5.0));
            const double ex = tmp.dz[s] * kx2 * kx2 / (4.0 * k * k * k);
            if (r6 > 1e-7 || ex > 0.05) sep = false;
            if (ex > 0.01) tiny = false;  // exp(-i e) to second order: error e^3 / 6 <= 1.7e-7 rad
            if (ex > 4.4e-4) first = false;  // exp(-i e) to first order: error e^2 / 2 <= 1e-7 rad
        }
        tmp.sep_transfer = sep;
        tmp.tiny_cross = sep && tiny;
        tmp.first_order_cross = sep && tiny && first;
    }

    Plan* p = new Plan(tmp);
    cudaError_t e = cudaGetDevice(&p->device);
    const int N = p->N, S = p->S;
    const size_t N2 = (size_t)N * N;
    // screens per synthesis launch: whole screen sets, about 256 MiB of complex workspace
    const int budget = (int)((256ull << 20) / (8 * N2));
    const int sets = std::max(1, std::min(max_batch, budget / S));
    p->screen_chunk = std::max(S * sets, std::min(max_batch, std::max(1, budget)));
    p->screen_chunk = ((p->screen_chunk + S - 1) / S) * S;
    auto ok = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    ok(dalloc(*p, &p->tw, 4 * (size_t)N));  // padded per-thread twiddle rows (FftCfg::tw_size <= 4 N)
    if (N >= 512) ok(dalloc(*p, &p->tw16, 4 * (size_t)N));
    else p->tw16 = p->tw;
    ok(dalloc(*p, &p->P, (size_t)S * N));
    ok(dalloc(*p, &p->amp, S));
    ok(dalloc(*p, &p->g, N2));
    ok(dalloc(*p, &p->tilt, 2 * (size_t)N));
    if (sh_levels) {
        ok(dalloc(*p, &p->shx, 3 * (size_t)N));
        ok(dalloc(*p, &p->shy, 3 * (size_t)N));
        ok(dalloc(*p, &p->shy_mean, 3));
        ok(dalloc(*p, &p->shb, (size_t)S * kShCoef));
        ok(dalloc(*p, &p->ws_shv, (size_t)p->screen_chunk * kShVectors * N));
        ok(dalloc(*p, &p->ws_shmean, p->screen_chunk));
        ok(dalloc(*p, &p->ws_sha, (size_t)p->screen_chunk * kShCoef));
    }
    ok(dalloc(*p, &p->ws_y, (size_t)p->screen_chunk * N2));
    // regenerated screens as exp(i phi): all S steps of a call at once when that takes <= 256 MiB
    p->regen_all = (size_t)max_batch * S * N2 * sizeof(float2) <= (256ull << 20);
    ok(dalloc(*p, &p->ws_phi, (size_t)max_batch * (p->regen_all ? S : 1) * N2));
    ok(dalloc(*p, &p->ws_rows, (size_t)max_batch * N * 4));
    if ((N == 512 || N == 1024) && !p->split_bf16) {
        ok(dalloc(*p, &p->src_fx, (size_t)kMaxSources * N));
        ok(dalloc(*p, &p->src_gy, (size_t)kMaxSources * N));
    }
    if (N == 1024 && !p->split_bf16) {
        ok(dalloc(*p, &p->ht_all, (size_t)S * N));
        ok(dalloc(*p, &p->fused_ctr, (size_t)(2 * S + 1) * max_batch + 1));
    }
    // device error word and wait budget of the passes with bounded waits (tensor-core and prefetching passes)
    ok(dalloc(*p, &p->d_err, 1));
    if (p->d_err) ok(cudaMemset(p->d_err, 0, sizeof(int)));
    {
        int khz = 0;
        ok(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, p->device));
        p->test_stall = (flags & TS_PLAN_TEST_STALL) != 0;
        const double seconds = p->test_stall ? 0.05 : 1.0;
        p->tc_budget = (long long)(seconds * (double)(khz > 0 ? khz : 2000000) * 1e3);
    }
    if (p->split_bf16) {
        // column tiles of 4 columns (one 128-vector group) unless TS_TC_COL_GROUPS=2 asks for 8
        const char* env = std::getenv("TS_TC_COL_GROUPS");
        p->tc_col_groups = (env && std::atoi(env) == 2) ? 2 : 1;
    }
    if (e != cudaSuccess) {
        ts_status st = cuda_check(e, "ts_plan_create allocation");
        free_plan(p);
        return st;
    }
    // per-screen amplitudes: s(kappa) = amp_s g(kappa), amp_s = sqrt(2 pi k^2 dz A Cn^2) dkappa
    float amp[kMaxScreens];
    for (int s = 0; s < S; ++s)
        amp[s] = (float)(std::sqrt(2.0 * M_PI * p->k * p->k * p->dz[s] * p->psd_A * p->cn2[s]) * p->dk);
    ok(cudaMemcpy(p->amp, amp, sizeof(float) * S, cudaMemcpyHostToDevice));
    if (sh_levels) {
        // b[p][q] = sqrt(Phi_phi(kappa_pq)) dkappa / 3^p, kappa_pq = (n', m') dkappa / 3^p   (Eq. 2)
        double shb[kMaxScreens * kShCoef];
        for (int s = 0; s < S; ++s)
            for (int lv = 1; lv <= 3; ++lv) {
                const double dkp = p->dk / std::pow(3.0, lv);
                for (int q = 0; q < 9; ++q) {
                    const int mp = q / 3 - 1, np = q % 3 - 1;
                    const double k2 = (np * dkp) * (np * dkp) + (mp * dkp) * (mp * dkp);
                    shb[s * kShCoef + (lv - 1) * 9 + q] = (q == 4) ? 0.0 : std::sqrt(phase_psd(*p, p->cn2[s], p->dz[s], k2)) * dkp;
                }
            }
        ok(cudaMemcpy(p->shb, shb, sizeof(double) * S * kShCoef, cudaMemcpyHostToDevice));
    }
    ok(build_tables(*p));
    if (p->ht_all) ok(build_ht_table(p->ht_all, p->P, S, p->dk, nullptr));
    ok(prepare_prop_kernels(N));
    if (p->split_bf16) ok(prepare_tc_prop());
    ok(prepare_screen_kernels(N));
    ok(prepare_d2nn_kernels(N));
    if (e != cudaSuccess) {
        ts_status st = cuda_check(e, "ts_plan_create tables");
        free_plan(p);
        return st;
    }
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) {
        ok(cudaStreamCreateWithFlags(&p->aux[i], cudaStreamNonBlocking));
        ok(cudaEventCreateWithFlags(&p->join[i], cudaEventDisableTiming));
    }
    ok(cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming));
    if (e != cudaSuccess) {
        ts_status st = cuda_check(e, "ts_plan_create streams");
        free_plan(p);
        return st;
    }
    {
        ts_status st = autotune(*p);
        if (st == TS_OK) st = autotune_groups(*p);
        if (st == TS_OK) st = autotune_fused(*p);
        if (st != TS_OK) {
            free_plan(p);
            return st;
        }
    }
    *out = reinterpret_cast<ts_plan>(p);
    return TS_OK;
}

ts_status ts_plan_destroy(ts_plan plan)
{
    if (!plan) return TS_OK;
    Plan* p = reinterpret_cast<Plan*>(plan);
    cudaError_t e = cudaDeviceSynchronize();
    free_plan(p);
    return cuda_check(e, "ts_plan_destroy");
}

size_t ts_plan_device_bytes(ts_plan plan) { return plan ? reinterpret_cast<Plan*>(plan)->bytes : 0; }

ts_status ts_plan_tuning(ts_plan plan, int* points_per_thread, float* us_e16, float* us_e32, int* streams,
                         float* us_streams, int* col_variant, float* us_e32_warp_columns, int* row_variant,
                         float* us_e32_shared_phasor_rows)
{
    if (!plan || !points_per_thread) return fail(TS_ERR_INVALID_ARG, "ts_plan_tuning: need plan and output");
    Plan* p = reinterpret_cast<Plan*>(plan);
    *points_per_thread = p->fft_e;
    if (us_e16) *us_e16 = p->tune_us[0];
    if (us_e32) *us_e32 = p->tune_us[1];
    if (streams) *streams = p->prop_groups;
    if (us_streams)
        for (int i = 0; i < 3; ++i) us_streams[i] = p->tune_group_us[i];
    if (col_variant) *col_variant = p->col_variant;
    if (us_e32_warp_columns) *us_e32_warp_columns = p->tune_us[2];
    if (row_variant) *row_variant = p->row_variant;
    if (us_e32_shared_phasor_rows) *us_e32_shared_phasor_rows = p->tune_us[3];
    return TS_OK;
}

ts_status ts_plan_tuning_candidates(ts_plan plan, int max, int* n, int* points_per_thread, int* col_variant,
                                    int* row_variant, float* us)
{
    if (!plan || !n) return fail(TS_ERR_INVALID_ARG, "ts_plan_tuning_candidates: need plan and n");
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    *n = kTuneCand;
    for (int c = 0; c < kTuneCand && c < max; ++c) {
        if (points_per_thread) points_per_thread[c] = kCandE[c];
        if (col_variant) col_variant[c] = kCandCol[c];
        if (row_variant) row_variant[c] = kCandRow[c];
        if (us) us[c] = p->tune_us[c];
    }
    return TS_OK;
}

ts_status ts_plan_tuning_columns(ts_plan plan, int* col_variant, float* us_variant2, float* us_variant3)
{
    if (!plan || !col_variant) return fail(TS_ERR_INVALID_ARG, "ts_plan_tuning_columns: need plan and output");
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    *col_variant = p->col_variant;
    if (us_variant2) *us_variant2 = p->tune_col_us[0];
    if (us_variant3) *us_variant3 = p->tune_col_us[1];
    return TS_OK;
}

ts_status ts_plan_tuning_fused(ts_plan plan, int* fused, float* us_per_pass, float* us_fused)
{
    if (!plan || !fused) return fail(TS_ERR_INVALID_ARG, "ts_plan_tuning_fused: need plan and output");
    const Plan* p = reinterpret_cast<const Plan*>(plan);
    *fused = p->fused ? 1 : 0;
    if (us_per_pass) *us_per_pass = p->tune_fused_us[0];
    if (us_fused) *us_fused = p->tune_fused_us[1];
    return TS_OK;
}

ts_status ts_plan_set_loss_scale(ts_plan plan, double scale)
{
    if (!plan || !(scale > 0.0) || !std::isfinite(scale))
        return fail(TS_ERR_INVALID_ARG, "ts_plan_set_loss_scale: need a plan and a finite scale > 0");
    reinterpret_cast<Plan*>(plan)->loss_scale = scale;
    return TS_OK;
}

ts_status ts_plan_device_status(ts_plan plan)
{
    if (!plan) return fail(TS_ERR_INVALID_ARG, "ts_plan_device_status: null plan");
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (ts_status sd = check_device(*p, "ts_plan_device_status"); sd != TS_OK) return sd;
    if (!p->d_err) return TS_OK;
    int code = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&code, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && code != 0) e = cudaMemset(p->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_check(e, "ts_plan_device_status");
    if (code != 0) return fail(TS_ERR_DEVICE_TIMEOUT, "a bounded device wait of the plan (tensor-core or prefetching pass) ran out of its budget");
    return TS_OK;
}

ts_status ts_plan_set_sources(ts_plan plan, int n, const double* w0)
{
    if (!plan || !w0 || n < 1 || n > kMaxSources) return fail(TS_ERR_INVALID_ARG, "need a plan and 1..64 source waists");
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (ts_status sd = check_device(*p, "ts_plan_set_sources"); sd != TS_OK) return sd;
    for (int i = 0; i < n; ++i) p->src_coef[i] = w0[i] > 0.0 ? (float)(p->dx * p->dx / (w0[i] * w0[i])) : -1.0f;
    p->n_src = n;
    if (p->src_fx) {
        // row DFT of each source's x profile and its y profile, FP64: the first column pass of a call
        // with sources starts from R0(kx, y) = Fx(kx) gy(y), the row transform of the separable source
        // U0 = exp(-(x^2 + y^2) dx^2 / w0^2) (pixel offsets from N/2; a plane wave has Fx = N delta)
        const int N = p->N;
        std::vector<float2> fx((size_t)n * N);
        std::vector<float> gy((size_t)n * N);
        std::vector<double> cs(N), g(N);
        for (int q = 0; q < N; ++q) cs[q] = std::cos(2.0 * M_PI * q / N);
        for (int i = 0; i < n; ++i) {
            const double c = w0[i] > 0.0 ? p->dx * p->dx / (w0[i] * w0[i]) : -1.0;
            for (int x = 0; x < N; ++x) g[x] = c < 0.0 ? 1.0 : std::exp(-(double)(x - N / 2) * (x - N / 2) * c);
            for (int y = 0; y < N; ++y) gy[(size_t)i * N + y] = (float)g[y];  // the same profile along y
            for (int k = 0; k < N; ++k) {
                // sum_x g(x) exp(-2 pi i k x / N) with g symmetric about N/2: (-1)^k sum_d g(N/2 + d) cos(2 pi k d / N)
                double re = 0.0;
                for (int x = 0; x < N; ++x) re += g[x] * cs[(size_t)((long long)k * ((x - N / 2 + N) % N) % N)];
                const double sgn = (k & 1) ? -1.0 : 1.0;
                fx[(size_t)i * N + k] = make_float2((float)(sgn * re), 0.0f);
            }
        }
        cudaError_t e = cudaDeviceSynchronize();  // no launch in flight still reads the previous table
        if (e == cudaSuccess) e = cudaMemcpy(p->src_fx, fx.data(), sizeof(float2) * fx.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p->src_gy, gy.data(), sizeof(float) * gy.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_check(e, "ts_plan_set_sources");
    }
    return TS_OK;
}

ts_status ts_make_sources(ts_plan plan, void* field, int B, void* stream)
{
    if (!plan || !field || B < 1) return fail(TS_ERR_INVALID_ARG, "ts_make_sources: need plan, field and B >= 1");
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (ts_status sd = check_device(*p, "ts_make_sources"); sd != TS_OK) return sd;
    if (p->n_src < 1) return fail(TS_ERR_INVALID_ARG, "ts_make_sources: no source table set");
    RowArgs ra{};
    ra.field = reinterpret_cast<float2*>(field);
    ra.phi_group = 1;
    ra.B = B;
    return cuda_check(launch_row_pass(*p, RP_IN_SOURCE | RP_STORE, ra, as_stream(stream)), "ts_make_sources");
}

ts_status ts_make_screens(ts_plan plan, uint64_t seed, uint32_t real_base, int n_real, float* phi, void* phasor,
                          void* stream)
{
    if (!plan || (!phi && !phasor) || n_real < 1)
        return fail(TS_ERR_INVALID_ARG, "ts_make_screens: need plan, phi or phasor, and n_real >= 1");
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (ts_status sd = check_device(*p, "ts_make_screens"); sd != TS_OK) return sd;
    ScreenArgs a{};
    a.seed = seed;
    a.s_begin = 0;
    a.s_count = p->S;
    a.r_begin = real_base;
    a.items = n_real * p->S;
    a.t = 0;
    a.phi = phi;
    a.phasor = reinterpret_cast<float2*>(phasor);
    cudaStream_t st = as_stream(stream);
    return cuda_check(timed(*p, 2, st, [&] { return launch_screens(*p, SC_INDEP, a, st); }), "ts_make_screens");
}

ts_status ts_evolve_screens(ts_plan plan, uint64_t seed, uint32_t real, uint32_t t, double alpha, double vx, double vy,
                            double T, void* spec, void* sh_state, float* phi, void* phasor, void* stream)
{
    if (!plan || !spec || (!phi && !phasor))
        return fail(TS_ERR_INVALID_ARG, "ts_evolve_screens: need plan, spec, and phi or phasor");
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (ts_status sd = check_device(*p, "ts_evolve_screens"); sd != TS_OK) return sd;
    if (p->sh_levels && !sh_state) return fail(TS_ERR_INVALID_ARG, "ts_evolve_screens: plan has subharmonics, sh_state needed");
    if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(TS_ERR_INVALID_ARG, "alpha must lie in [0, 1]");
    if (t > 0xFFFFFFu) return fail(TS_ERR_INVALID_ARG, "t must be below 2^24");
    cudaStream_t st = as_stream(stream);
    ScreenArgs a{};
    a.seed = seed;
    a.s_begin = 0;
    a.s_count = p->S;
    a.r_begin = real;
    a.items = p->S;
    a.t = t;
    a.alpha_d = alpha;
    a.beta_d = std::sqrt(1.0 - alpha * alpha);
    a.alpha = (float)a.alpha_d;
    a.beta = (float)a.beta_d;
    a.spec = reinterpret_cast<float2*>(spec);
    a.sh_state = reinterpret_cast<double2*>(sh_state);
    a.phi = phi;
    a.phasor = reinterpret_cast<float2*>(phasor);
    a.tilt = (t > 0) && T != 0.0 && (vx != 0.0 || vy != 0.0);
    a.vx = vx;
    a.vy = vy;
    a.T = T;
    if (a.tilt) {
        ts_status s0 = cuda_check(build_tilt(*p, vx, vy, T, st), "ts_evolve_screens tilt");
        if (s0 != TS_OK) return s0;
    }
    return cuda_check(timed(*p, 2, st, [&] { return launch_screens(*p, t == 0 ? SC_AR_INIT : SC_AR_STEP, a, st); }),
                      "ts_evolve_screens");
}

ts_status ts_propagate(ts_plan plan, void* field, int B, const float* phi, const void* phasor, int phi_group, int flags,
                       uint64_t seed, uint32_t real_base, float* intensity, double* beam_sums, void* stream)
{
    if (!plan || !field) return fail(TS_ERR_INVALID_ARG, "ts_propagate: need plan and field");
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (ts_status sd = check_device(*p, "ts_propagate"); sd != TS_OK) return sd;
    if (B < 1 || phi_group < 1) return fail(TS_ERR_INVALID_ARG, "ts_propagate: B and phi_group must be >= 1");
    if (B > p->max_batch) return fail(TS_ERR_WORKSPACE, "ts_propagate: B exceeds the plan's max_batch");
    if ((flags & TS_PROP_SOURCE) && p->n_src < 1) return fail(TS_ERR_INVALID_ARG, "ts_propagate: no source table set");
    if ((flags & TS_PROP_INTENSITY) && !intensity) return fail(TS_ERR_INVALID_ARG, "ts_propagate: intensity buffer needed");
    if (beam_sums && !(flags & TS_PROP_INTENSITY))
        return fail(TS_ERR_INVALID_ARG, "ts_propagate: beam_sums need TS_PROP_INTENSITY");
    if ((flags & TS_PROP_NO_FIELD) && !(flags & TS_PROP_INTENSITY))
        return fail(TS_ERR_INVALID_ARG, "ts_propagate: TS_PROP_NO_FIELD needs TS_PROP_INTENSITY");
    cudaStream_t st = as_stream(stream);
    float2* U = reinterpret_cast<float2*>(field);
    ts_status stt = propagate_groups(*p, U, B, phi, phasor, phi_group, flags, seed, real_base, intensity,
                                     beam_sums ? p->ws_rows : nullptr, st);
    if (stt != TS_OK) return stt;
    if (beam_sums) return cuda_check(launch_row_sums(*p, p->ws_rows, B, beam_sums, st), "ts_propagate beam sums");
    return TS_OK;
}

ts_status ts_propagate_backward(ts_plan plan, void* grad, int B, const float* phi, const void* phasor, int phi_group,
                                uint64_t seed, uint32_t real_base, void* stream)
{
    if (!plan || !grad) return fail(TS_ERR_INVALID_ARG, "ts_propagate_backward: need plan and grad");
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (ts_status sd = check_device(*p, "ts_propagate_backward"); sd != TS_OK) return sd;
    if (B < 1 || phi_group < 1) return fail(TS_ERR_INVALID_ARG, "ts_propagate_backward: B and phi_group must be >= 1");
    if (B > p->max_batch) return fail(TS_ERR_WORKSPACE, "ts_propagate_backward: B exceeds the plan's max_batch");
    cudaStream_t st = as_stream(stream);
    const int N = p->N, S = p->S;
    const size_t N2 = (size_t)N * N;
    const int G = (B + phi_group - 1) / phi_group;
    float2* g = reinterpret_cast<float2*>(grad);
    RowArgs ra{};
    ra.field = g;
    ra.phi_group = phi_group;
    ra.phase_sign = -1.0f;
    ra.B = B;
    ts_status stt = TS_OK;
    int phase_flag = RP_PHASOR;
    auto set_screen = [&](int s) -> ts_status {
        ra.phi = nullptr;
        ra.phasor = nullptr;
        ra.phi_set_stride = (long long)S * N2;
        if (phasor) {
            ra.phasor = reinterpret_cast<const float2*>(phasor) + (size_t)s * N2;
            phase_flag = RP_PHASOR;
            return TS_OK;
        }
        if (phi) {
            ra.phi = phi + (size_t)s * N2;
            phase_flag = RP_PHASE;
            return TS_OK;
        }
        phase_flag = RP_PHASOR;
        if (p->regen_all) {  // all S screens synthesised with the first (last-step) screen
            ra.phasor = p->ws_phi + (size_t)s * N2;
            ra.phi_set_stride = (long long)S * N2;
            return s == S - 1 ? regen_screen(*p, seed, real_base, G, -1, st) : TS_OK;
        }
        ra.phasor = p->ws_phi;
        ra.phi_set_stride = (long long)N2;
        return regen_screen(*p, seed, real_base, G, s, st);
    };
    if ((stt = set_screen(S - 1)) != TS_OK) return stt;
    stt = cuda_check(launch_row_pass(*p, phase_flag | RP_OUT_FREQ | RP_STORE, ra, st), "backward first row pass");
    if (stt != TS_OK) return stt;
    for (int s = S - 1; s >= 0; --s) {
        stt = cuda_check(launch_col_pass(*p, s, true, g, B, st), "backward column pass");
        if (stt != TS_OK) return stt;
        if (s > 0) {
            if ((stt = set_screen(s - 1)) != TS_OK) return stt;
            stt = cuda_check(launch_row_pass(*p, RP_IN_FREQ | phase_flag | RP_OUT_FREQ | RP_STORE, ra, st),
                             "backward row pass");
        } else {
            ra.phi = nullptr;
            ra.phasor = nullptr;
            stt = cuda_check(launch_row_pass(*p, RP_IN_FREQ | RP_STORE, ra, st), "backward last row pass");
        }
        if (stt != TS_OK) return stt;
    }
    return TS_OK;
}

ts_status ts_moments_accumulate(ts_plan plan, const float* intensity, int B, int n_groups, int64_t count, double* mean,
                                double* m2, const double* beam_sums, double* beam_acc, void* stream)
{
    if (!plan || !intensity || !mean || !m2) return fail(TS_ERR_INVALID_ARG, "ts_moments_accumulate: null pointer");
    if ((beam_sums == nullptr) != (beam_acc == nullptr))
        return fail(TS_ERR_INVALID_ARG, "ts_moments_accumulate: beam_sums and beam_acc go together");
    if (n_groups < 1 || B < n_groups || B % n_groups != 0 || count < 0)
        return fail(TS_ERR_INVALID_ARG, "ts_moments_accumulate: B must be a positive multiple of n_groups");
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (ts_status sd = check_device(*p, "ts_moments_accumulate"); sd != TS_OK) return sd;
    cudaStream_t st = as_stream(stream);
    if (beam_sums) {
        ts_status sb = cuda_check(launch_beam_acc(beam_sums, B, n_groups, count == 0, beam_acc, st),
                                  "ts_moments_accumulate beam sums");
        if (sb != TS_OK) return sb;
    }
    return cuda_check(launch_moments(*p, intensity, B, n_groups, count, mean, m2, st), "ts_moments_accumulate");
}

ts_status ts_moments_finalize(ts_plan plan, const double* mean, const double* m2, int n_groups, int64_t count,
                              const double* beam_acc, double* si_map, double* si_mean, double* si_center, double* w_lt,
                              void* stream)
{
    if (!plan || !mean || !m2 || n_groups < 1 || count < 1)
        return fail(TS_ERR_INVALID_ARG, "ts_moments_finalize: need moments with count >= 1");
    if (w_lt && !beam_acc) return fail(TS_ERR_INVALID_ARG, "ts_moments_finalize: w_lt needs beam_acc");
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (ts_status sd = check_device(*p, "ts_moments_finalize"); sd != TS_OK) return sd;
    cudaStream_t st = as_stream(stream);
    if (w_lt) {
        ts_status sw = cuda_check(launch_w_lt(beam_acc, n_groups, w_lt, st), "ts_moments_finalize w_lt");
        if (sw != TS_OK) return sw;
    }
    return cuda_check(launch_moments_finalize(*p, mean, m2, n_groups, count, si_map, si_mean, si_center, st),
                      "ts_moments_finalize");
}

ts_status ts_plan_timing(ts_plan plan, int enable, int capacity)
{
    if (!plan || capacity < 0) return fail(TS_ERR_INVALID_ARG, "ts_plan_timing: need a plan and capacity >= 0");
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (ts_status sd = check_device(*p, "ts_plan_timing"); sd != TS_OK) return sd;
    destroy_events(p);
    p->timing = enable != 0;
    if (!p->timing) return TS_OK;
    for (auto& v : p->ev) {
        v.resize(2 * (size_t)capacity);
        for (auto& e : v) {
            cudaError_t err = cudaEventCreate(&e);
            if (err != cudaSuccess) {
                e = nullptr;
                p->timing = false;
                return cuda_check(err, "ts_plan_timing");
            }
        }
    }
    return TS_OK;
}

ts_status ts_plan_timing_read(ts_plan plan, int kind, int* launches, double* total_ms)
{
    if (!plan || kind < 0 || kind > 3 || !launches || !total_ms)
        return fail(TS_ERR_INVALID_ARG, "ts_plan_timing_read: bad arguments");
    Plan* p = reinterpret_cast<Plan*>(plan);
    double tot = 0.0;
    for (int i = 0; i < p->ev_used[kind]; ++i) {
        cudaError_t e = cudaEventSynchronize(p->ev[kind][2 * i + 1]);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p->ev[kind][2 * i], p->ev[kind][2 * i + 1]);
        if (e != cudaSuccess) return cuda_check(e, "ts_plan_timing_read");
        tot += ms;
    }
    *launches = p->ev_used[kind];
    *total_ms = tot;
    return TS_OK;
}

ts_status ts_philox4x32_10(const uint32_t* ctr, uint32_t key0, uint32_t key1, int n, uint32_t* out, void* stream)
{
    if (!ctr || !out || n < 1) return fail(TS_ERR_INVALID_ARG, "ts_philox4x32_10: need ctr, out and n >= 1");
    return cuda_check(launch_philox(ctr, key0, key1, n, out, as_stream(stream)), "ts_philox4x32_10");
}

ts_status ts_d2nn_forward(ts_plan plan, const void* U, int B, const float* th1, const float* th2, double aperture,
                          const float* Iref, int kind, void* ws, float* intensity, double* loss, void* stream)
{
    if (!plan || !U || !th1 || !th2 || !Iref || !ws || !intensity || !loss)
        return fail(TS_ERR_INVALID_ARG, "ts_d2nn_forward: null pointer");
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (ts_status sd = check_device(*p, "ts_d2nn_forward"); sd != TS_OK) return sd;
    if (B < 1 || (kind != 0 && kind != 1) || !(aperture > 0.0))
        return fail(TS_ERR_INVALID_ARG, "ts_d2nn_forward: need B >= 1, kind 0/1 and aperture > 0");
    if (B > p->max_batch) return fail(TS_ERR_WORKSPACE, "ts_d2nn_forward: B exceeds the plan's max_batch");
    D2nnArgs d{};
    d.U = reinterpret_cast<const float2*>(U);
    d.B = B;
    d.th1 = th1;
    d.th2 = th2;
    d.aperture = aperture;
    d.Iref = Iref;
    d.kind = kind;
    d.ws = reinterpret_cast<float2*>(ws);
    d.I = intensity;
    d.loss = loss;
    return cuda_check(launch_d2nn(*p, false, d, as_stream(stream)), "ts_d2nn_forward");
}

ts_status ts_d2nn_backward(ts_plan plan, int B, const float* th1, const float* th2, double aperture, const float* Iref,
                           int kind, const void* ws, const float* intensity, float* g_th1, float* g_th2, void* gU,
                           void* stream)
{
    if (!plan || !th1 || !th2 || !Iref || !ws || !intensity || !g_th1 || !g_th2 || !gU)
        return fail(TS_ERR_INVALID_ARG, "ts_d2nn_backward: null pointer");
    Plan* p = reinterpret_cast<Plan*>(plan);
    if (ts_status sd = check_device(*p, "ts_d2nn_backward"); sd != TS_OK) return sd;
    if (B < 1 || (kind != 0 && kind != 1) || !(aperture > 0.0))
        return fail(TS_ERR_INVALID_ARG, "ts_d2nn_backward: need B >= 1, kind 0/1 and aperture > 0");
    if (B > p->max_batch) return fail(TS_ERR_WORKSPACE, "ts_d2nn_backward: B exceeds the plan's max_batch");
    D2nnArgs d{};
    d.B = B;
    d.th1 = th1;
    d.th2 = th2;
    d.aperture = aperture;
    d.Iref = Iref;
    d.kind = kind;
    d.ws = reinterpret_cast<float2*>(const_cast<void*>(ws));
    d.I = const_cast<float*>(intensity);
    d.g_th1 = g_th1;
    d.g_th2 = g_th2;
    d.gU = reinterpret_cast<float2*>(gU);
    return cuda_check(launch_d2nn(*p, true, d, as_stream(stream)), "ts_d2nn_backward");
}

}  // extern "C"
