// ts_screens.cu -- phase-screen synthesis (S16, Eq. 2-3) and AR(1) evolution (Eq. 4-5).
//
// A screen is phi = Re(IDFT2_unnormalised(X)) + phi_SH - mean, X = s(kappa) c(kappa) (or the AR
// state).  Two passes:
//   column pass: draw Philox noise for the tile's bins in registers, form X (and the AR update),
//                store the AR state, inverse-transform each column, store Y (complex).
//   row pass:    inverse-transform each row of Y, keep the real part, add the subharmonic screen
//                (a rank-7 separable sum whose coefficients come from an FP64 kernel) minus its
//                piston, store phi (float32).
// The FFT part has zero mean exactly (s(0) = 0), so the only piston removed is the subharmonic
// one, computed in closed form from per-axis means.
#include <type_traits>

#include "ts_device.cuh"
#include "ts_internal.h"

namespace ts {

namespace {

struct ScreenColParams {
    const float2* tw;
    const float* g;
    const float* amp;
    float2* y;
    float2* spec;
    const float2* tilt;  // [2][N] or nullptr
    uint32_t k0, k1;
    int s_begin, s_count;
    uint32_t r_begin;
    uint32_t tag;
    float alpha, beta;
};

template <int N>
struct SColCfg {
    using C = FftCfg<N>;
    static constexpr int THREADS = 256;
    static constexpr int W = THREADS / C::T;
    static constexpr int LS = C::padded + (16 / W > 1 ? 16 / W : 1);
    static constexpr size_t smem = sizeof(float2) * (C::tw_smem + W * LS);
};

template <int N, int MODE>
__global__ void __launch_bounds__(SColCfg<N>::THREADS) screen_col_kernel(const ScreenColParams a)
{
    using C = FftCfg<N>;
    using CC = SColCfg<N>;
    constexpr int E = C::E, T = C::T, W = CC::W;
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % W, t = threadIdx.x / W;
    const int n = blockIdx.x * W + c;
    const int z = blockIdx.y;
    const int s = a.s_begin + z % a.s_count;
    const uint32_t r = a.r_begin + (uint32_t)(z / a.s_count);
    float2* tw = smem;
    float2* buf = smem + C::tw_smem + c * CC::LS;
    const float amp = __ldg(a.amp + s);
    stage_twiddles<N>(tw, a.tw);

    // The PSD shape and (AR step) the previous state are loaded first, so their latency overlaps the
    // Philox / Box-Muller arithmetic that follows; the arithmetic itself is unchanged.
    float2 v[E];
    float gv[E];
    float2* sp = a.spec + (size_t)z * N * N + n;
#pragma unroll
    for (int i = 0; i < E; ++i) gv[i] = __ldg(a.g + (size_t)(t + i * T) * N + n);
    if constexpr (MODE == SC_AR_STEP) {
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = sp[(size_t)(t + i * T) * N];
    }
    const float2 tx = (MODE == SC_AR_STEP && a.tilt) ? __ldg(a.tilt + n) : make_float2(1.0f, 0.0f);
    // bins (m, n) and (m + N/2, n) share one Philox call: registers i and i + E/2
#pragma unroll
    for (int i = 0; i < E / 2; ++i) {
        const int m = t + i * T;
        const u32x4 w = philox4x32_10(u32x4{(uint32_t)(m * N + n), (uint32_t)s, r, a.tag}, a.k0, a.k1);
        const float2 c0 = box_muller(w.a, w.b);
        const float2 c1 = box_muller(w.c, w.d);
        const float2 n0 = cscale(c0, amp * gv[i]);
        const float2 n1 = cscale(c1, amp * gv[i + E / 2]);
        if constexpr (MODE == SC_AR_STEP) {
            float2 o0 = v[i], o1 = v[i + E / 2];
            if (a.tilt) {
                o0 = cmul(o0, cmul(tx, __ldg(a.tilt + N + m)));
                o1 = cmul(o1, cmul(tx, __ldg(a.tilt + N + m + N / 2)));
            }
            v[i] = make_float2(fmaf(a.alpha, o0.x, a.beta * n0.x), fmaf(a.alpha, o0.y, a.beta * n0.y));
            v[i + E / 2] = make_float2(fmaf(a.alpha, o1.x, a.beta * n1.x), fmaf(a.alpha, o1.y, a.beta * n1.y));
        } else {
            v[i] = n0;
            v[i + E / 2] = n1;
        }
    }
    if constexpr (MODE != SC_INDEP) {
#pragma unroll
        for (int i = 0; i < E; ++i) sp[(size_t)(t + i * T) * N] = v[i];
    }
    __syncthreads();
    // the synthesis keeps the packed-add butterflies: the fused form measured slower here
    line_fft_c<FftCfg<N, 0, false>, +1>(v, buf, t, tw, BlockBar());
    float2* yo = a.y + (size_t)z * N * N + n;
#pragma unroll
    for (int i = 0; i < E; ++i) yo[(size_t)(t + i * T) * N] = v[i];
}

struct ScreenRowParams {
    const float2* tw;
    const float2* y;
    float* phi;       // float32 screen, or nullptr
    float2* phasor;   // exp(i phi), or nullptr
    const float* shv;      // [items][7][N]
    const float* shmean;   // [items]
    const float2* shy;     // [3][N]
};

template <int N>
struct SRowCfg {
    using C = FftCfg<N>;
    static constexpr int THREADS = 256;
    static constexpr int LPC = THREADS / C::T;
    static constexpr int LS = C::padded;
    static constexpr size_t smem = sizeof(float2) * (C::tw_smem + LPC * LS);
};

template <int N, bool SH>
__global__ void __launch_bounds__(SRowCfg<N>::THREADS) screen_row_kernel(const ScreenRowParams a)
{
    using C = FftCfg<N>;
    using RC = SRowCfg<N>;
    constexpr int E = C::E, T = C::T;
    extern __shared__ float2 smem[];
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int j = blockIdx.x * RC::LPC + line;
    const int z = blockIdx.y;
    float2* tw = smem;
    float2* buf = smem + C::tw_smem + line * RC::LS;
    using Bar = typename std::conditional<(T > 32), BlockBar, WarpBar>::type;

    const float2* yrow = a.y + ((size_t)z * N + j) * N;
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = yrow[t + i * T];
    stage_twiddles<N>(tw, a.tw);
    __syncthreads();
    line_fft_c<FftCfg<N, 0, false>, +1>(v, buf, t, tw, Bar());
    const size_t roff = ((size_t)z * N + j) * N;
    // phi in v[i].x, then stored as requested: float32 screen and/or its phasor exp(i phi)
    if constexpr (SH) {
        const float* V = a.shv + (size_t)z * kShVectors * N;
        const float2 e1 = __ldg(a.shy + j), e2 = __ldg(a.shy + N + j), e3 = __ldg(a.shy + 2 * N + j);
        const float pist = __ldg(a.shmean + z);
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int x = t + i * T;
            float sh = __ldg(V + x) - pist;
            sh = fmaf(e1.x, __ldg(V + N + x), sh);
            sh = fmaf(e1.y, __ldg(V + 2 * N + x), sh);
            sh = fmaf(e2.x, __ldg(V + 3 * N + x), sh);
            sh = fmaf(e2.y, __ldg(V + 4 * N + x), sh);
            sh = fmaf(e3.x, __ldg(V + 5 * N + x), sh);
            sh = fmaf(e3.y, __ldg(V + 6 * N + x), sh);
            v[i].x += sh;
        }
    }
    if (a.phi != nullptr) {
#pragma unroll
        for (int i = 0; i < E; ++i) a.phi[roff + t + i * T] = v[i].x;
    }
    if (a.phasor != nullptr) {
#pragma unroll
        for (int i = 0; i < E; ++i) a.phasor[roff + t + i * T] = expi_phase(v[i].x);
    }
}

// Subharmonic coefficients and row vectors, FP64 (Eq. 2).  One CTA per screen item.
//   a[p][q] = b[p][q] c[p][q]                                   (independent / AR start)
//   a[p][q] = alpha exp(i theta) a[p][q] + beta b[p][q] c^(t)   (AR step, Eq. 4-5)
//   A_p[m'](x) = sum_n' a[p][(m'+1)3 + n'+1] exp(i n' dkappa_p x)
//   phi_SH(x, y) = sum_p Re A_p[0] + cos(dk_p y) Re(A_p[1] + A_p[-1]) + sin(dk_p y) Im(A_p[-1] - A_p[1])
// Stored as V0 = sum_p Re A_p[0], Vc_p, Vs_p (float32) and the FP64 piston
//   mean = mean_x V0 + sum_p (mean_y cos) mean_x Vc_p + (mean_y sin) mean_x Vs_p.
struct ShParams {
    const double* shb;        // [S][27]
    const double2* shx;       // [3][N]
    const double2* shy_mean;  // [3]
    double2* sha;             // [items][27] (AR state or scratch)
    float* shv;               // [items][7][N]
    float* shmean;            // [items]
    uint32_t k0, k1;
    int s_begin, s_count;
    uint32_t r_begin;
    uint32_t t;
    int mode;
    double alpha, beta;
    double dk, vx, vy, T;
    int N;
};

__global__ void __launch_bounds__(256) sh_kernel(const ShParams a)
{
    const int z = blockIdx.x;
    const int s = a.s_begin + z % a.s_count;
    const uint32_t r = a.r_begin + (uint32_t)(z / a.s_count);
    const int N = a.N;
    __shared__ double2 coef[kShCoef];
    __shared__ double red[kShVectors][256];
    if (threadIdx.x < kShCoef) {
        const int idx = threadIdx.x, p = idx / 9 + 1, q = idx % 9;
        double2 out = make_double2(0.0, 0.0);
        if (q != 4) {
            const u32x4 w =
                philox4x32_10(u32x4{(uint32_t)((p - 1) * 8 + q / 2), (uint32_t)s, r, (1u << 24) | (a.t & 0xFFFFFFu)},
                              a.k0, a.k1);
            const double2 c = (q % 2 == 0) ? box_muller_d(w.a, w.b) : box_muller_d(w.c, w.d);
            const double b = a.shb[s * kShCoef + idx];
            if (a.mode == SC_AR_STEP) {
                const double2 old = a.sha[(size_t)z * kShCoef + idx];
                const double dkp = a.dk / pow(3.0, p);
                const double th = -a.T * (((q % 3) - 1) * dkp * a.vx + ((q / 3) - 1) * dkp * a.vy);
                double sn, cs;
                sincos(th, &sn, &cs);
                const double2 tl = make_double2(old.x * cs - old.y * sn, old.x * sn + old.y * cs);
                out = make_double2(a.alpha * tl.x + a.beta * b * c.x, a.alpha * tl.y + a.beta * b * c.y);
            } else {
                out = make_double2(b * c.x, b * c.y);
            }
        }
        coef[idx] = out;
        if (a.mode != SC_INDEP) a.sha[(size_t)z * kShCoef + idx] = out;
    }
    __syncthreads();
    double acc[kShVectors] = {0, 0, 0, 0, 0, 0, 0};
    float* V = a.shv + (size_t)z * kShVectors * N;
    for (int x = threadIdx.x; x < N; x += blockDim.x) {
        double v0 = 0.0;
        for (int p = 0; p < 3; ++p) {
            const double2 e = a.shx[p * N + x];  // exp(i dk_p x)
            double2 A[3];                        // m' = -1, 0, 1
            for (int mm = 0; mm < 3; ++mm) {
                const double2 cm = coef[p * 9 + mm * 3 + 0], c0 = coef[p * 9 + mm * 3 + 1], cp = coef[p * 9 + mm * 3 + 2];
                // cm e^{-i} + c0 + cp e^{+i}
                A[mm] = make_double2(c0.x + (cm.x * e.x + cm.y * e.y) + (cp.x * e.x - cp.y * e.y),
                                     c0.y + (cm.y * e.x - cm.x * e.y) + (cp.x * e.y + cp.y * e.x));
            }
            v0 += A[1].x;
            const double vc = A[2].x + A[0].x;
            const double vs = A[0].y - A[2].y;
            V[(1 + 2 * p) * N + x] = (float)vc;
            V[(2 + 2 * p) * N + x] = (float)vs;
            acc[1 + 2 * p] += vc;
            acc[2 + 2 * p] += vs;
        }
        V[x] = (float)v0;
        acc[0] += v0;
    }
    for (int k = 0; k < kShVectors; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < kShVectors; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double m = red[0][0] / N;
        for (int p = 0; p < 3; ++p) {
            const double2 ym = a.shy_mean[p];
            m += ym.x * red[1 + 2 * p][0] / N + ym.y * red[2 + 2 * p][0] / N;
        }
        a.shmean[z] = (float)m;
    }
}

template <int N, int MODE>
cudaError_t scol_launch(const ScreenColParams& cp, int items, cudaStream_t st)
{
    using CC = SColCfg<N>;
    dim3 grid(N / CC::W, items);
    screen_col_kernel<N, MODE><<<grid, CC::THREADS, CC::smem, st>>>(cp);
    return cudaGetLastError();
}

template <int N>
cudaError_t screens_for(Plan& p, int mode, const ScreenArgs& a, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    for (int z0 = 0; z0 < a.items; z0 += p.screen_chunk) {
        const int nz = (a.items - z0) < p.screen_chunk ? (a.items - z0) : p.screen_chunk;
        // item z0 + z maps to screen s_begin + (z0 + z) % s_count, realization r_begin + (z0 + z) / s_count;
        // chunks are multiples of s_count so each chunk restarts at screen s_begin.
        const uint32_t rb = a.r_begin + (uint32_t)(z0 / a.s_count);
        ScreenColParams cp;
        cp.tw = p.tw;
        cp.g = p.g;
        cp.amp = p.amp;
        cp.y = p.ws_y;
        cp.spec = a.spec ? a.spec + (size_t)z0 * N * N : nullptr;
        cp.tilt = a.tilt ? p.tilt : nullptr;
        cp.k0 = k0;
        cp.k1 = k1;
        cp.s_begin = a.s_begin;
        cp.s_count = a.s_count;
        cp.r_begin = rb;
        cp.tag = a.t & 0xFFFFFFu;
        cp.alpha = a.alpha;
        cp.beta = a.beta;
        if (mode == SC_INDEP) e = scol_launch<N, SC_INDEP>(cp, nz, st);
        else if (mode == SC_AR_INIT) e = scol_launch<N, SC_AR_INIT>(cp, nz, st);
        else e = scol_launch<N, SC_AR_STEP>(cp, nz, st);
        if (e != cudaSuccess) return e;
        const bool sh = p.sh_levels > 0;
        if (sh) {
            ShParams sp;
            sp.shb = p.shb;
            sp.shx = p.shx;
            sp.shy_mean = p.shy_mean;
            sp.sha = (mode == SC_INDEP) ? p.ws_sha : a.sh_state + (size_t)z0 * kShCoef;
            sp.shv = p.ws_shv;
            sp.shmean = p.ws_shmean;
            sp.k0 = k0;
            sp.k1 = k1;
            sp.s_begin = a.s_begin;
            sp.s_count = a.s_count;
            sp.r_begin = rb;
            sp.t = a.t;
            sp.mode = mode;
            sp.alpha = a.alpha_d;
            sp.beta = a.beta_d;
            sp.dk = p.dk;
            sp.vx = a.tilt ? a.vx : 0.0;
            sp.vy = a.tilt ? a.vy : 0.0;
            sp.T = a.tilt ? a.T : 0.0;
            sp.N = N;
            sh_kernel<<<nz, 256, 0, st>>>(sp);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        ScreenRowParams rp;
        rp.tw = p.tw;
        rp.y = p.ws_y;
        rp.phi = a.phi ? a.phi + (size_t)z0 * N * N : nullptr;
        rp.phasor = a.phasor ? a.phasor + (size_t)z0 * N * N : nullptr;
        rp.shv = p.ws_shv;
        rp.shmean = p.ws_shmean;
        rp.shy = p.shy;
        using RC = SRowCfg<N>;
        dim3 grid(N / RC::LPC, nz);
        if (sh) screen_row_kernel<N, true><<<grid, RC::THREADS, RC::smem, st>>>(rp);
        else screen_row_kernel<N, false><<<grid, RC::THREADS, RC::smem, st>>>(rp);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return e;
}

template <int N>
cudaError_t prepare_screens_for()
{
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    const int cs = (int)SColCfg<N>::smem, rs = (int)SRowCfg<N>::smem;
    chk(cudaFuncSetAttribute(screen_col_kernel<N, SC_INDEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs));
    chk(cudaFuncSetAttribute(screen_col_kernel<N, SC_AR_INIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs));
    chk(cudaFuncSetAttribute(screen_col_kernel<N, SC_AR_STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs));
    chk(cudaFuncSetAttribute(screen_row_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs));
    chk(cudaFuncSetAttribute(screen_row_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs));
    return e;
}

}  // namespace

cudaError_t launch_screens(Plan& p, int mode, const ScreenArgs& a, cudaStream_t st)
{
    switch (p.N) {
    case 128: return screens_for<128>(p, mode, a, st);
    case 256: return screens_for<256>(p, mode, a, st);
    case 512: return screens_for<512>(p, mode, a, st);
    case 1024: return screens_for<1024>(p, mode, a, st);
    case 2048: return screens_for<2048>(p, mode, a, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_screen_raw(int N, const float2* tw, const float* g, const float* amp, float2* y, uint64_t seed,
                              int screen, uint32_t real, float* phi, cudaStream_t st)
{
    ScreenColParams cp{};
    cp.tw = tw;
    cp.g = g;
    cp.amp = amp;
    cp.y = y;
    cp.spec = nullptr;
    cp.tilt = nullptr;
    cp.k0 = (uint32_t)seed;
    cp.k1 = (uint32_t)(seed >> 32);
    cp.s_begin = screen;
    cp.s_count = 1;
    cp.r_begin = real;
    cp.tag = 0;
    ScreenRowParams rp{};
    rp.tw = tw;
    rp.y = y;
    rp.phi = phi;
    rp.phasor = nullptr;
    cudaError_t e = cudaSuccess;
#define TS_RAW(NN)                                                                                    \
    case NN: {                                                                                        \
        e = scol_launch<NN, SC_INDEP>(cp, 1, st);                                                     \
        if (e != cudaSuccess) return e;                                                               \
        dim3 grid(NN / SRowCfg<NN>::LPC, 1);                                                          \
        screen_row_kernel<NN, false><<<grid, SRowCfg<NN>::THREADS, SRowCfg<NN>::smem, st>>>(rp);      \
        return cudaGetLastError();                                                                    \
    }
    switch (N) {
        TS_RAW(128)
        TS_RAW(256)
        TS_RAW(512)
        TS_RAW(1024)
        TS_RAW(2048)
    default: return cudaErrorInvalidValue;
    }
#undef TS_RAW
    return e;
}

cudaError_t prepare_screen_kernels(int N)
{
    switch (N) {
    case 128: return prepare_screens_for<128>();
    case 256: return prepare_screens_for<256>();
    case 512: return prepare_screens_for<512>();
    case 1024: return prepare_screens_for<1024>();
    case 2048: return prepare_screens_for<2048>();
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ts
