/*
 * turbscreen.h -- C ABI of the GB300 (sm_103a) split-step optical-turbulence library.
 *
 * The library computes the data-parallel hot path of the split-step method of TurPy
 * (Greene et al., arXiv 2604.07248): FFT phase screens from a von Karman phase PSD with 3-level
 * subharmonics (Sec. 2.1-2.2, Eq. 2-3, App. B-C), AR(1) temporal evolution of the screens in the
 * Fourier domain (Sec. 2.3, Eq. 4-5), the propagate/modulate loop of Eq. 1 with the angular-spectrum
 * transfer function (Sec. 2.4), its adjoint, per-pixel intensity moments (S25) and the two-mask
 * dual-domain D2NN receiver (Sec. 2.5, 4.1).  Every step runs in hand-written CUDA kernels.
 *
 * Conventions used throughout:
 *   - complex fields are interleaved complex64 (float re, float im), row-major [N][N]
 *     (row j = y index, column i = x index); batches are [B][N][N], contiguous.
 *   - x = (i - N/2) dx for sources and apertures (beam centred on pixel (N/2, N/2)); screens use
 *     the DFT origin x = i dx.
 *   - spectral index f(n) = n for n < N/2, else n - N; kappa = 2 pi f / (N dx).
 *   - gradients follow the convention g = dL/dRe + i dL/dIm, so a linear map P back-propagates as P^H.
 *   - all device pointers are owned by the caller; a plan owns only its own tables and workspace
 *     (allocated once in ts_plan_create).  No call other than ts_plan_create / ts_plan_destroy
 *     allocates or frees device memory.
 *   - all work is enqueued asynchronously on the given CUDA stream (a cudaStream_t passed as
 *     void*; NULL = legacy default stream); a call may fan work out to the plan's own streams and
 *     joins them back into the caller's stream before returning.  Argument checks happen on the
 *     host before any launch; a failing check launches nothing.  One plan must not be used
 *     concurrently from two host threads or two unordered streams (it owns one workspace).
 *   - on error a call returns a non-zero ts_status and ts_last_error() gives a one-line detail.
 *   - a plan (and a batch) belongs to the CUDA device that was current when it was created; every
 *     call on it must be made with that device current and with buffers on that device.  A call
 *     made while another device is current returns TS_ERR_INVALID_ARG and launches nothing (the
 *     library cannot tell on which device a raw pointer lives, so matching the buffers is the
 *     caller's part; the Python binding checks them).
 */
#ifndef TURBSCREEN_H
#define TURBSCREEN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TS_OK = 0,
    TS_ERR_INVALID_ARG = 1,    /* a pointer, size or parameter is out of range                   */
    TS_ERR_ALIASING = 2,       /* a step dz exceeds the angular-spectrum aliasing limit (Eq. 7)   */
    TS_ERR_WORKSPACE = 3,      /* the plan's workspace cannot hold the request (batch too large)  */
    TS_ERR_CUDA = 4,           /* a CUDA runtime call failed (detail in ts_last_error())          */
    TS_ERR_DEVICE_TIMEOUT = 5, /* a bounded device-side wait gave up                              */
    TS_ERR_UNSUPPORTED = 6     /* a grid size or regime this build does not implement             */
} ts_status;

/* Medium (Fig. 1A inputs): vacuum wavelength [m], mean refractive index n0, inner scale l0 [m]
 * (<= 0: no inner-scale roll-off), outer scale L0 [m] (<= 0 or inf: no outer scale).
 * The refractive-index PSD is the modified von Karman form (S17 written through Cn^2, S18):
 *   Phi_n = 0.033 Cn^2 (kappa^2 + kappa0^2)^(-11/6) exp(-kappa^2 / kappa_m^2),
 *   kappa0 = 2 pi / L0, kappa_m = 2 pi / l0, and a screen covering dz has Phi_phi = 2 pi k^2 dz Phi_n (S14). */
typedef struct {
    double lambda;
    double n0;
    double l0;
    double L0;
} ts_medium;

/* Grid: N x N points (N in {128, 256, 512, 1024, 2048}), spacing dx [m]. */
typedef struct {
    int N;
    double dx;
} ts_grid;

/* Path (Fig. 1A "range samples" and "turbulence strength over path"): n_screens intervals; interval
 * s has length dz[s] [m] and structure constant cn2[s] [m^-2/3].  Both arrays are HOST pointers read
 * during ts_plan_create only.  Step s of Eq. 1 propagates dz[s] and then applies screen s. */
typedef struct {
    int n_screens;
    const double* dz;
    const double* cn2;
} ts_path;

typedef struct ts_plan_s* ts_plan;

/* ts_plan_create flags */
#define TS_PLAN_ALLOW_ALIASING 1 /* skip the Eq. 7 step-size check (caller accepts aliasing) */
#define TS_PLAN_SPLIT_BF16 2     /* propagation passes (column and row passes of Eq. 1, forward and adjoint)
                                    on the tensor cores: every line DFT is a 32 x 32 four-step DFT whose
                                    stages are BF16 GEMMs with FP32 accumulation, each factor split into
                                    BF16 hi + lo (products hi.hi + hi.lo + lo.hi, about 2^-16 relative
                                    error per stage).  N = 1024 only (else TS_ERR_UNSUPPORTED).  Screens,
                                    moments and the D2NN receiver stay FP32.  Not accepted by ts_batch. */
#define TS_PLAN_TEST_STALL 4     /* test hook: the prefetching passes (column / row variant 2) never issue their
                                  * first copy, so their first bounded wait runs out (budget 50 ms instead of
                                  * one second) and ts_plan_device_status reports TS_ERR_DEVICE_TIMEOUT */

/* Creates a plan for one medium, grid and path.  sh_levels is 0 or 3 (subharmonic levels, Eq. 2,
 * scale factor 3).  max_batch bounds the number of fields per ts_propagate / ts_propagate_backward
 * call and the number of realizations per ts_make_screens chunk.  The plan builds its FP64-derived
 * tables on the current CUDA device (twiddles, per-step transfer-function factors, PSD shape,
 * subharmonic basis) and allocates its workspace there; the call synchronises the device.
 * Errors: TS_ERR_INVALID_ARG (null pointers, N not supported, dx/lambda/dz <= 0, cn2 < 0,
 * sh_levels not 0/3, max_batch < 1), TS_ERR_ALIASING (some dz above the Eq. 7 limit
 * dz_max = (N dx / 2) sqrt(k^2 - kappa_max^2) / kappa_max with kappa_max = pi / dx, unless
 * TS_PLAN_ALLOW_ALIASING), TS_ERR_UNSUPPORTED (grid reaches the evanescent region, or
 * TS_PLAN_SPLIT_BF16 with N != 1024), TS_ERR_CUDA. */
ts_status ts_plan_create(ts_plan* plan, const ts_medium* medium, const ts_grid* grid, const ts_path* path,
                         int sh_levels, int max_batch, int flags);

/* ts_plan_create for another medium of Table S1: the refractive-index PSD is the power law
 *   Phi_n(kappa) = A Cn^2 (kappa^2 + kappa0^2)^(-alpha/2) exp(-kappa^2 / kappa_m^2)   (S12, S15, S17)
 * with alpha = beta + 3 (S11): atmosphere 11/3 (Kolmogorov; ts_plan_create uses alpha = 11/3,
 * A = 0.033), general atmosphere 3..4, oceanic 11/3..5, biological tissue 4.28..4.41.  The paper gives
 * the law up to its constant; ts_power_law_constant(alpha) returns the one for which Cn^2 is the
 * index structure constant (D_n(r) = Cn^2 r^(alpha - 3)).  Screens, subharmonics and AR evolution
 * all use this PSD.  Errors as ts_plan_create, plus TS_ERR_INVALID_ARG for alpha outside (3, 5) or
 * A not finite and > 0. */
ts_status ts_plan_create_psd(ts_plan* plan, const ts_medium* medium, const ts_grid* grid, const ts_path* path,
                             int sh_levels, int max_batch, int flags, double alpha, double A);

/* A(alpha) = Gamma(alpha - 1) cos(pi alpha / 2) / (4 pi^2) for 3 < alpha < 5 (0.0330 at 11/3), the
 * published non-Kolmogorov constant; NaN outside that range.  Host-only. */
double ts_power_law_constant(double alpha);

/* Device status of a plan: waits for all work on the device, then returns TS_ERR_DEVICE_TIMEOUT
 * (and clears the flag) if a bounded device wait of its passes ran out of its one-second budget since
 * the last call -- a tensor-core pass (TS_PLAN_SPLIT_BF16) waiting for its MMAs, or a prefetching
 * pass (column / row variant 2) waiting for its TMA copy; the pass then stopped early and its output
 * is incomplete -- else TS_OK.  A CTA (or warp) whose wait ran out waits once more, again bounded, for
 * its own copy in flight before it exits; if that second wait also runs out, the copy engine has not
 * delivered within two seconds and may still write into shared memory that a later CTA on that SM
 * reuses.  After TS_ERR_DEVICE_TIMEOUT, treat the plan's outputs and any later work on the device as
 * unreliable: destroy the plan and reset the device (cudaDeviceReset) before relying on it again. */
ts_status ts_plan_device_status(ts_plan plan);

/* Frees the plan's device memory (synchronises the device).  NULL is accepted. */
ts_status ts_plan_destroy(ts_plan plan);

/* Device bytes held by the plan (tables + workspace). */
size_t ts_plan_device_bytes(ts_plan plan);

/* Autotuner result of the plan (chosen once per device, N, batch and transfer form; cached):
 *  - the propagation passes run with `points_per_thread` FFT points per thread (16 or 32) and, for
 *    N = 1024 with 32 points, `col_variant` 0 (a column line spread over four warps, block-level
 *    exchanges) or 1 (one warp per column, the CTA's 8-column tile staged through shared memory);
 *    `row_variant` 0 (each CTA reads its rows of the screen phasor) or 1 (N = 1024, 32 points, phasor
 *    screens shared by 2, 4 or 8 fields: a CTA holds those fields' rows and stages the phasor rows
 *    once in shared memory); us_e16 / us_e32 / us_e32_warp_columns / us_e32_shared_phasor_rows
 *    receive the timed cost in microseconds of one column + one row pass of each candidate;
 *  - `streams` = number of field groups ts_propagate runs concurrently on the plan's own streams when
 *    the screens are given (1, 2 or 4; forked from and joined back to the caller's stream);
 *    us_streams[3] receives the timed cost for 1, 2 and 4 groups.
 * Each timing is the fastest of three interleaved rounds over the candidates (2 warm-up + 5 timed
 * repetitions each).  Outputs other than points_per_thread may be NULL; a 0 timing means not timed
 * (N <= 256, a cached result, or TS_FFT_E / TS_COL_VARIANT / TS_ROW_VARIANT / TS_PROP_STREAMS set in
 * the environment). */
ts_status ts_plan_tuning(ts_plan plan, int* points_per_thread, float* us_e16, float* us_e32, int* streams,
                         float* us_streams, int* col_variant, float* us_e32_warp_columns, int* row_variant,
                         float* us_e32_shared_phasor_rows);

/* The autotuner's whole candidate table: *n receives the number of candidates (8); for the first
 * min(max, *n) of them, points_per_thread[c] (16 or 32), col_variant[c] (0: a column line shared by
 * four warps; 1: one warp per column, tile staged through shared memory; 2 / 3: persistent CTAs whose
 * next tile arrives by TMA while the current one is transformed, wide / narrow tiles: 8 / 4 columns
 * (two / four CTAs per SM) at N = 1024, 16 / 8 columns at N = 512), row_variant[c] (0: each CTA
 * reads its screen rows; 1: phasor rows shared by the CTA's fields; 2: persistent warps that prefetch
 * their next field row and the screen phasor row with bulk asynchronous copies) and us[c], the timed
 * cost in microseconds of one column + one row pass (0 = not timed).  Column variants 2 and 3 and row
 * variant 2 exist for N = 512 and 1024, column variant 1 and row variant 1 for N = 1024, all at 32
 * points per thread.  Output arrays may be NULL.  Host-only; no device work. */
ts_status ts_plan_tuning_candidates(ts_plan plan, int max, int* n, int* points_per_thread, int* col_variant,
                                    int* row_variant, float* us);

/* The column tiles under concurrent field groups (N = 512 and 1024, 32 points per thread, FP32
 * passes): when the autotuner propagates two or more field groups concurrently and its first stage
 * picked a prefetching column pass (column variant 2 or 3: wide or narrow tiles), it times both again
 * as runs of column + row pass pairs on that many groups and keeps the faster (the other replaces the
 * first stage's pick only when at least 1 % faster).  *col_variant receives the column variant
 * ts_propagate uses; us_variant2 / us_variant3 the two costs in microseconds per pass pair (0 = not
 * timed: fewer than two groups, another variant, other N, or TS_COL_VARIANT / TS_PROP_STREAMS in the
 * environment; a choice cached from an earlier plan reports the timings it was made on).  Outputs
 * other than col_variant may be NULL.  Host-only. */
ts_status ts_plan_tuning_columns(ts_plan plan, int* col_variant, float* us_variant2, float* us_variant3);

/* The autotuner's last stage (N = 1024, 32 points per thread, FP32 passes): *fused = 1 when
 * ts_propagate runs the whole path of a call -- first row pass and S x (column pass, row pass) of
 * Eq. 1 -- as ONE persistent launch.  Its work items are (pass, field, 8-column or 8-row tile); an
 * item starts once every tile of the previous pass of its own field is done (bounded waits, error
 * word as in ts_plan_device_status), so one field's row pass runs while another's column pass
 * drains, and each CTA prefetches its next item's tile by TMA.  It serves calls whose screens are
 * given as phasors or regenerated from the seed (when the workspace holds all S screens) and that
 * store the field (no TS_PROP_INTENSITY); other calls use the per-pass launches.  us_per_pass /
 * us_fused receive the timed cost in microseconds of one propagation of min(max_batch, 8) fields
 * each way (0 = not timed: other N, a cached result, or TS_FUSED=0|1 in the environment).
 * Outputs other than `fused` may be NULL.  Host-only. */
ts_status ts_plan_tuning_fused(ts_plan plan, int* fused, float* us_per_pass, float* us_fused);

/* Aliasing-limited maximum step of Eq. 7 for this medium and grid (reading: kappa_max = pi/dx,
 * Nyquist spacing 2 pi / (N dx)); returns a negative value for invalid input. */
double ts_max_step(const ts_medium* medium, const ts_grid* grid);

/* Source table used by ts_propagate with TS_PROP_SOURCE: field b starts as source (b mod n).
 * w0[k] > 0: collimated Gaussian exp(-r^2 / w0^2) centred on pixel (N/2, N/2) (S22);
 * w0[k] <= 0: unit plane wave (Sec. 3.3).  w0 is a HOST array of n entries (n <= 64).  For N = 512
 * and 1024 it also builds, in FP64 on the host, each source's row transform (the sources are
 * separable), from which the first column pass of a call starts; it then waits for the device and
 * copies the tables synchronously, so call it outside stream capture and not while a ts_propagate of
 * the plan is in flight on another thread. */
ts_status ts_plan_set_sources(ts_plan plan, int n, const double* w0);

/* Source fields (S22; plane wave of Sec. 3.3): writes the plan's source table into field
 * (device complex64 [B][N][N]), field b = source (b mod n).  Requires ts_plan_set_sources. */
ts_status ts_make_sources(ts_plan plan, void* field, int B, void* stream);

/* Independent screens (Sec. 2.1, Fig. 1B-C; S16; Eq. 2-3): for realization r in
 * [real_base, real_base + n_real) and screen s in [0, S):
 *   phi = Re(sum_kappa s(kappa) c(kappa) exp(+i kappa.x)) + phi_SH - mean,
 * s(kappa) = sqrt(Phi_phi(kappa)) dkappa with s(0) = 0, c = Philox4x32-10 complex Gaussian noise.
 * phi: device float32 [n_real][S][N][N] and/or phasor: device complex64 [n_real][S][N][N] holding
 * exp(i phi) (either may be NULL, not both), written.  Counter layout of the noise:
 * key = (seed mod 2^32, seed >> 32), counter = (word0, s, r, (purpose << 24) | t) with t = 0;
 * grid bins (m, n) and (m + N/2, n) share word0 = m N + n (m < N/2); subharmonic cell q of level p
 * uses purpose 1 and word0 = (p - 1) 8 + q / 2. */
ts_status ts_make_screens(ts_plan plan, uint64_t seed, uint32_t real_base, int n_real, float* phi, void* phasor,
                          void* stream);

/* One screen without any device allocation.  The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc where they need a screen (for instance code running under
 * another framework's allocator or stream rules that forbid new device allocations, or a
 * latency-critical loop that cannot afford the implicit synchronisation of cudaMalloc/cudaFree).
 * It computes the same screen as ts_make_screens for a plan whose interval `screen` has length dz
 * and structure constant cn2 (no subharmonics): phi (device float32 [N][N], written) equals
 * ts_make_screens' phi[real][screen].  Its twiddles, PSD table and intermediate live in one
 * fixed-size file-scope device array (about 12 MiB) that every GPU on which the library's module is
 * loaded holds until the process exits: with lazy module loading (the CUDA default) the GPUs on
 * which a kernel of the library has run, with CUDA_MODULE_LOADING=EAGER every GPU the process opens.
 * Limits: N <= 1024 (N = 2048 returns TS_ERR_WORKSPACE), screen < 64.
 * Every call looks up the array's device address in the current context (cudaGetSymbolAddress: no
 * allocation, no synchronisation), so the address is right after cudaDeviceReset and under any
 * context the caller makes current; the first call in a context also sets kernel attributes and may
 * load the module, so make it before any CUDA stream capture.  All calls share the array and each
 * call overwrites it: calls that can overlap on the GPU (different streams without ordering between
 * them) race and produce wrong screens. */
ts_status ts_make_screen_noalloc(const ts_medium* medium, const ts_grid* grid, double dz, double cn2, uint64_t seed,
                                 uint32_t screen, uint32_t real, float* phi, void* stream);

/* AR(1) evolution of the S screens of realization `real` (Sec. 2.3, Eq. 4-5):
 *   t == 0: spec = s(kappa) c^(0)                                   (stationary start)
 *   t >= 1: spec = alpha exp(i theta) spec + sqrt(1 - alpha^2) s(kappa) c^(t),
 *           theta = -2 pi T (f_x vx + f_y vy)  (wind translation; T = 0 disables it),
 * then phi = Re(IDFT_unnormalised(spec)) + phi_SH - mean.  The subharmonic coefficients evolve
 * by the same rule with their own frequencies.
 * spec: device complex64 [S][N][N], read (t >= 1) and written.  sh_state: device complex128
 * [S][27] when the plan has subharmonics (else NULL), read/written likewise.  phi: device float32
 * [S][N][N] and/or phasor: device complex64 [S][N][N] = exp(i phi), written (either may be NULL,
 * not both).  0 <= alpha <= 1. */
ts_status ts_evolve_screens(ts_plan plan, uint64_t seed, uint32_t real, uint32_t t, double alpha, double vx,
                            double vy, double T, void* spec, void* sh_state, float* phi, void* phasor, void* stream);

/* ts_propagate flags */
#define TS_PROP_SOURCE 1    /* start from the plan's source table instead of reading `field`     */
#define TS_PROP_INTENSITY 2 /* write I = |U|^2 (float32 [B][N][N]) to `intensity`               */
#define TS_PROP_NO_FIELD 4  /* do not store the output field (only meaningful with INTENSITY)   */

/* Split-step propagation, Eq. 1, for s = 0..S-1:  U <- IFFT2(FFT2(U) H_s) exp(i phi_s), with
 *   H_s = exp(-i dz_s kappa^2 / (k + sqrt(k^2 - kappa^2)))  (H_as of Sec. 2.4 without its global
 *   piston exp(i k dz_s)), FFT2 unnormalised, IFFT2 with 1/N^2.
 * field: device complex64 [B][N][N], input (unless TS_PROP_SOURCE) and output.
 * phi: device float32 screens [G][S][N][N] with G = ceil(B / phi_group): field b uses screen set
 * b / phi_group.  phasor: the same screens as exp(i phi), device complex64 [G][S][N][N]; when given
 * it is used instead of phi (one complex multiply per point instead of a sincos, which pays off when
 * several fields share a screen).  Both NULL regenerates the screens from
 * (seed, real_base + b / phi_group) exactly as ts_make_screens does (plan workspace; no allocation).
 * intensity: device float32 [B][N][N] (TS_PROP_INTENSITY) else NULL.
 * beam_sums: device float64 [B][2] or NULL: per field sum I and sum r^2 I (r from pixel (N/2, N/2)).
 * Errors: TS_ERR_INVALID_ARG, TS_ERR_WORKSPACE (B > max_batch), TS_ERR_CUDA. */
ts_status ts_propagate(ts_plan plan, void* field, int B, const float* phi, const void* phasor, int phi_group, int flags,
                       uint64_t seed, uint32_t real_base, float* intensity, double* beam_sums, void* stream);

/* Adjoint of ts_propagate with respect to the input field: grad <- P^H grad, i.e. for s = S-1..0
 *   g <- g exp(-i phi_s);  g <- IFFT2(FFT2(g) conj(H_s)).
 * grad: device complex64 [B][N][N] in/out (dL/dU_out in, dL/dU_in out).  phi / phasor as in
 * ts_propagate; both NULL regenerates each screen from its seed (bit-identical to the forward
 * screens) one step at a time in the plan workspace instead of storing them. */
ts_status ts_propagate_backward(ts_plan plan, void* grad, int B, const float* phi, const void* phasor, int phi_group,
                                uint64_t seed, uint32_t real_base, void* stream);

/* Per-pixel intensity moments across realizations (S25 with Welford's algorithm, Sec. 3.3).
 * intensity: device float32 [B][N][N]; fields b with b mod n_groups == g form the chunk of group g
 * (B / n_groups fields each, B divisible by n_groups).  mean, m2: device float64 [n_groups][N][N]
 * holding `count` realizations per group before the call; the chunk is merged with the pairwise
 * (Chan et al.) update, so results do not depend on how realizations are split into calls.
 * After the call each group holds count + B / n_groups realizations.
 * beam_sums (device float64 [B][2], the per-field sums ts_propagate writes) and beam_acc (device
 * float64 [n_groups][2]) go together or are both NULL: beam_acc[g] receives (count == 0) or adds
 * (count > 0) the sums (sum I, sum r^2 I) of the group's fields, in increasing field order, FP64:
 * the zeroth and second moments of the long-term spot (S23 / S24) over all realizations. */
ts_status ts_moments_accumulate(ts_plan plan, const float* intensity, int B, int n_groups, int64_t count,
                                double* mean, double* m2, const double* beam_sums, double* beam_acc, void* stream);

/* Scintillation index map SI = (m2 / count) / mean^2 (S25, population variance), its plane
 * average and the on-axis value (pixel (N/2, N/2)), for n_groups groups; and the long-term beam
 * radius W_LT = sqrt(2 sum_r sum_x r^2 I / sum_r sum_x I) [m] (S23 / S24 as second moments, r from
 * pixel (N/2, N/2)) from the accumulated beam sums.  si_map: device float64 [n_groups][N][N] or
 * NULL; si_mean, si_center, w_lt: device float64 [n_groups] or NULL; beam_acc: the device float64
 * [n_groups][2] sums of ts_moments_accumulate (needed when w_lt is given, else may be NULL).
 * Asynchronous on `stream` like the other calls. */
ts_status ts_moments_finalize(ts_plan plan, const double* mean, const double* m2, int n_groups, int64_t count,
                              const double* beam_acc, double* si_map, double* si_mean, double* si_center, double* w_lt,
                              void* stream);

/* Factor applied to the D2NN receiver loss and to all its gradients (default 1): e.g. 1 / max(Iref)
 * for the MAE (kind 0) or 1 / max(Iref)^2 for the squared error normalises the intensities to the
 * reference's peak, which keeps the mask gradients of a unit-amplitude source in the range an Adam
 * optimiser with eps = 1e-8 resolves.  Host-side setting of the plan; later calls use it. */
ts_status ts_plan_set_loss_scale(ts_plan plan, double scale);

/* Two-mask dual-domain D2NN receiver (Sec. 2.5, 4.1), batch of B fields U (device complex64):
 *   Z1 = exp(i th1) A U;  W2 = exp(i th2) C(Z1);  V = C^-1(W2);  I = |V|^2,
 * C = fftshift o FFT2 o ifftshift / N (lens as a unitary centred DFT), A = disk of diameter
 * `aperture` [m] centred on pixel (N/2, N/2).  Loss against the reference intensity Iref
 * (device float32 [N][N]): kind 0 = mean |I - Iref| (MAE, Sec. 2.5), kind 1 = mean (I - Iref)^2,
 * mean over batch and pixels, times the plan's loss scale (ts_plan_set_loss_scale); written to loss
 * (device float64 [1]).
 * th1, th2: device float32 [N][N].  ws: device complex64 workspace [3][B][N][N] kept for the
 * backward call (Z1, W2, V); intensity: device float32 [B][N][N], written (also kept for the
 * backward call).  B <= max_batch.  N must be divisible by 4 (all supported N are). */
ts_status ts_d2nn_forward(ts_plan plan, const void* U, int B, const float* th1, const float* th2, double aperture,
                          const float* Iref, int kind, void* ws, float* intensity, double* loss, void* stream);

/* Adjoint of ts_d2nn_forward: writes dL/dth1, dL/dth2 (device float32 [N][N], sums over the
 * batch in increasing b) and dL/dU (device complex64 [B][N][N]) from the workspace and intensity of
 * the forward call (same th1, th2, aperture, Iref, kind).  The workspace is consumed: per-field
 * mask gradients overwrite Z1 and W2, so a second backward needs a new forward call.
 *   g_V = 2 V dL/dI; g_W2 = C(g_V); dL/dth2 = sum Im(g_W2 conj W2); g_Z1 = C^-1(exp(-i th2) g_W2);
 *   dL/dth1 = sum Im(g_Z1 conj Z1); dL/dU = A exp(-i th1) g_Z1. */
ts_status ts_d2nn_backward(ts_plan plan, int B, const float* th1, const float* th2, double aperture,
                           const float* Iref, int kind, const void* ws, const float* intensity, float* g_th1,
                           float* g_th2, void* gU, void* stream);

/* Kernel timing for roofline measurements.  While enabled, the plan records a CUDA event pair on
 * the launching stream around every launch of: kind 0 = propagation column pass, kind 1 =
 * propagation row pass, kind 2 = screen synthesis (column + row pass of one ts_make_screens /
 * ts_evolve_screens / regeneration call), kind 3 = fused propagation (one persistent launch that runs
 * all passes of a ts_propagate call, see ts_plan_tuning_fused).  `capacity` event pairs are created per kind (no device
 * memory); launches beyond it are not timed.  Enabling resets the counters.
 * ts_plan_timing_read waits for the recorded events and returns the number of timed launches of
 * `kind` and their summed device time in milliseconds. */
ts_status ts_plan_timing(ts_plan plan, int enable, int capacity);
ts_status ts_plan_timing_read(ts_plan plan, int kind, int* launches, double* total_ms);

/* Split-BF16 tensor-core 32-point DFT, the building block of the tensor-core DFT variant: for
 * v < nvec, X[v][q] = sum_j x[v][j] exp(sign 2 pi i j q / 32), computed as a BF16 GEMM with FP32
 * accumulation in tensor memory (tcgen05) from hi/lo BF16 splits of both factors
 * (hi.hi + hi.lo + lo.hi, about 2^-16 relative error).  x, X: device complex64 [nvec][32].
 * layout selects how the data operand is staged in shared memory: 0 = K-major, 1 = MN-major (the
 * form the tensor-core propagation passes use between their two DFT stages), 2 = MN-major with the
 * two descriptor strides exchanged (a check of the descriptor reading; its result is not a DFT).
 * err: device int, set to nonzero if the wait for the MMAs ran out of timeout_s. */
ts_status ts_tc_dft32(const void* x, void* X, int nvec, int sign, int layout, double timeout_s, int* err,
                      void* stream);

/* Adam step of the D2NN training loop (Sec. 2.5; Kingma & Ba 2015), elementwise over n device
 * floats: m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2; p <- p - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).
 * param, m, v: device float32 [n] in/out; grad: device float32 [n]; t >= 1 is the step number. */
ts_status ts_adam_step(float* param, const float* grad, float* m, float* v, long long n, double lr, double beta1,
                       double beta2, double eps, int t, void* stream);

/* ---- path planning (host functions, no GPU) ---------------------------------------------------- */

/* Hufnagel-Valley Cn^2 profile (S21) at n heights h [m] >= 0:
 *   cn2[i] = 0.00594 (V/27)^2 (1e-5 h)^10 exp(-h/1000) + 2.7e-16 exp(-h/1500) + A exp(-h/100),
 * V = wind speed [m/s], A = ground-level constant [m^-2/3] (HV5/7: V = 21, A = 1.7e-14).
 * h, cn2: host arrays of n doubles. */
ts_status ts_cn2_hufnagel_valley(const double* h, int n, double V, double A, double* cn2);

/* Rytov variance of the interval [z0, z1] of a sampled Cn^2 profile (S19):
 *   sigma^2 = 3.27 k^(7/6) dz^(5/6) int_0^dz Cn2(z0 + z) (1 - z/dz)^(5/3) dz,  k = 2 pi / lambda.
 * The profile (host arrays prof_z strictly increasing, prof_cn2 >= 0, n_prof >= 1) is linear
 * between samples and constant beyond the ends; the integral is evaluated in closed form on each
 * linear piece.  For a constant profile sigma^2 = 1.226 k^(7/6) Cn2 dz^(11/6). */
ts_status ts_rytov_interval(const double* prof_z, const double* prof_cn2, int n_prof, double lambda, double z0,
                            double z1, double* sigma2);

/* Screen placement (Sec. 2.4) over a path [0, L] of a sampled Cn^2 profile (as in ts_rytov_interval):
 *   1. start from the caller's interval boundaries init_bounds[0..n_init) (values inside (0, L);
 *      n_init = 0: one interval);
 *   2. split every interval whose Rytov variance (S19) exceeds rytov_limit at its midpoint until none
 *      does; 3. merge neighbours while the merged interval stays within the limit;
 *   4. final placement: a sweep from z = 0 extends each interval until its variance reaches the
 *      limit (lengths solved by linear interpolation of log sigma^2 against log dz); the sweep is kept
 *      when it needs no more intervals than steps 2-3;
 *   5. every interval longer than the Eq. 7 step limit of `grid` is split into equal parts.
 * Outputs (host arrays of max_screens doubles): dz_out[i] = interval length, cn2_out[i] = the
 * interval's path-integrated Cn^2 divided by its length (the strength its screen carries, S18),
 * rytov_out[i] = its Rytov variance (may be NULL); *n_out = number of intervals.  They can be
 * passed to ts_plan_create as a ts_path.  Errors: TS_ERR_INVALID_ARG, TS_ERR_WORKSPACE (more than
 * max_screens intervals needed; *n_out still holds the count). */
ts_status ts_place_screens(const double* prof_z, const double* prof_cn2, int n_prof, const ts_medium* medium,
                           const ts_grid* grid, double L, const double* init_bounds, int n_init, double rytov_limit,
                           int max_screens, double* dz_out, double* cn2_out, double* rytov_out, int* n_out);

/* Raw Philox4x32-10 words (Salmon et al., SC'11) of n counters, for bit-exact checks of the noise
 * generator used by the screens: out[4i..4i+3] = Philox4x32-10(ctr[4i..4i+3], key).  ctr and out
 * are device uint32 arrays of 4n words. */
ts_status ts_philox4x32_10(const uint32_t* ctr, uint32_t key0, uint32_t key1, int n, uint32_t* out, void* stream);

/* ---------------------------------------------------------------------------------------------- */
/* Uneven batches: independent instances of different grids and screen counts (Eq. 1 each),     */
/* propagated by one persistent kernel launch.                                                    */
/* ---------------------------------------------------------------------------------------------- */
typedef struct ts_batch_s* ts_batch;

typedef struct {
    ts_plan plan;       /* the instance's medium, grid and path (kept alive by the caller)          */
    void* field;        /* device complex64 [N][N]: input (unless source) and output                */
    const void* phasor; /* device complex64 [S][N][N] screens as exp(i phi), or NULL: the batch
                           synthesises them from (seed, real) exactly as ts_make_screens does      */
    uint64_t seed;
    uint32_t real;
    int source;         /* nonzero: start from the plan's source 0 (ts_plan_set_sources)            */
} ts_batch_instance;

#define TS_BATCH_TEST_STALL 1 /* test hook: instance 0 waits for a tile that never completes, so its
                                 dependency wait runs out and the batch reports TS_ERR_DEVICE_TIMEOUT */
#define TS_BATCH_NO_TUNE 2    /* keep the default tile shapes and item order (no autotuning)        */

/* Builds a batch: validates the instances (all plans on the current device, separable transfer
 * form), lays out the work list (instance, phase, tile) by increasing phase, allocates the screen
 * workspace for instances without screens, and captures the run (screen synthesis, counter reset,
 * one persistent launch) as a CUDA graph.  timeout_s bounds every device-side dependency wait.
 * Unless TS_BATCH_NO_TUNE (or the stall hook) is given, an autotuner first chooses the tile shape of
 * every grid size -- the points per thread of its line FFTs, hence the rows of a row tile and the
 * columns of a column tile: N = 512 and 2048 at 32 or 16, N = 1024 at 32, N <= 256 at 16 -- and the
 * order of instances within a phase (as given, or largest grids first), by timing whole replays of
 * the batch on scratch fields it allocates for the purpose and frees (the callers' fields are not
 * touched; without room for them the batch keeps the default configuration, untuned);
 * ts_batch_tuning reports the choices.  The call synchronises the device.
 * Copies `inst`; the plans, fields and screens must outlive the batch. */
ts_status ts_batch_create(ts_batch* batch, const ts_batch_instance* inst, int n, double timeout_s, int flags);

/* The batch autotuner's choices: for each distinct grid size of the batch (ascending, at most 5,
 * written to sizes[]) the points per thread of its tiles; the item order (0 = instances in the
 * caller's order within a phase, 1 = largest grids first); the number of configurations timed (0 when
 * not tuned); and the replay times (us) of the default configuration and of the chosen one.  Output
 * pointers may be NULL.  Host-only. */
ts_status ts_batch_tuning(ts_batch batch, int* n_sizes, int* sizes, int* points_per_thread, int* order,
                          int* candidates, float* us_default, float* us_chosen);

/* Launches the captured graph on `stream` (asynchronous). */
ts_status ts_batch_run(ts_batch batch, void* stream);

/* Synchronises `stream` and reads the batch's device error word: TS_OK, or TS_ERR_DEVICE_TIMEOUT if
 * a dependency wait ran out (the kernel then stopped taking work; the CUDA context stays usable). */
ts_status ts_batch_status(ts_batch batch, void* stream);

/* Work items, persistent grid size (CTAs) and device bytes of the batch. */
ts_status ts_batch_info(ts_batch batch, int* n_items, int* grid, size_t* device_bytes);

ts_status ts_batch_destroy(ts_batch batch);

const char* ts_status_string(ts_status status);

/* One-line detail of the last error raised on the calling host thread ("" if none). */
const char* ts_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TURBSCREEN_H */
