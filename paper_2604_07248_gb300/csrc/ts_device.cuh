// ts_device.cuh -- device building blocks for the split-step turbulence kernels (sm_103a).
//
//  * complex64 arithmetic on float2
//  * Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller
//  * fully unrolled in-register DFTs of radix 2..32 with compile-time twiddles
//  * a Stockham autosort line FFT: each thread keeps E points of a length-N line in registers,
//    stages of radix <= E exchange through padded shared memory (Govindaraju et al. formulation:
//    stage with sub-length Ns reads x[j + r N/R], twiddles by W_{Ns R}^{(j mod Ns) r}, writes
//    y[(j/Ns) Ns R + (j mod Ns) + r Ns]).  The last stage leaves output point t + i T in register i
//    of thread t, the same placement the first stage reads, so transforms chain without an
//    exchange.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ts {

// ----------------------------------------------------------------------------------------------
// complex helpers
// ----------------------------------------------------------------------------------------------
// Complex add / subtract as one packed FP32x2 operation each (sm_100+): per component identical to
// the scalar round-to-nearest add; a - b is b * (-1) + a with a single rounding.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// ----------------------------------------------------------------------------------------------
// Philox4x32-10 and Box-Muller.  Counter layout (shared definition with the host documentation):
//   key = (seed mod 2^32, seed >> 32), ctr = (word0, screen, realization, (purpose << 24) | t).
// ----------------------------------------------------------------------------------------------
struct u32x4 {
    uint32_t a, b, c, d;
};

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 ctr, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * ctr.a, hi0 = __umulhi(0xD2511F53u, ctr.a);
        const uint32_t lo1 = 0xCD9E8D57u * ctr.c, hi1 = __umulhi(0xCD9E8D57u, ctr.c);
        ctr = u32x4{hi1 ^ ctr.b ^ k0, lo1, hi0 ^ ctr.d ^ k1, lo0};
    }
    return ctr;
}

// ((w >> 8) + 0.5) * 2^-24, exact in binary32
__device__ __forceinline__ float u01f(uint32_t w) { return ((float)(w >> 8) + 0.5f) * 5.9604644775390625e-8f; }

// Box-Muller: radius sqrt(-2 ln ua), angle 2 pi ub.  The angle is taken as 2 pi (ub - 1/2) + pi, i.e.
// (cos, sin)(2 pi ub) = -(cos, sin)(2 pi (ub - 1/2)) with the argument in [-pi, pi), where the
// hardware sine / cosine approximations are accurate to about 4e-7 absolute (the sample's relative
// error stays near 1e-6, far below the screens' 1e-5 tolerance); the radius keeps the accurate log.
__device__ __forceinline__ float2 box_muller(uint32_t wa, uint32_t wb)
{
    const float rad = sqrtf(-2.0f * logf(u01f(wa)));
    float s, c;
    __sincosf(6.28318530717958648f * (u01f(wb) - 0.5f), &s, &c);
    return make_float2(-rad * c, -rad * s);
}

// exp(i phi) for a screen phase: phi reduced to [-pi, pi] by the nearest multiple of 2 pi with a
// two-part 2 pi (hi = fl(2 pi), lo = 2 pi - hi, so the reduction error stays below 1e-7 rad for
// |phi| < 1e4), then the hardware sine / cosine, accurate to about 4e-7 on that interval.  The screen
// synthesis (phasor screens) and the row pass (float screens) both use it, so the two give the same
// fields bit for bit.
__device__ __forceinline__ float2 expi_phase(float phi)
{
    const float kq = rintf(phi * 0.159154943091895336f);
    float r = fmaf(-kq, 6.28318548202514648f, phi);
    r = fmaf(-kq, -1.74845553e-7f, r);
    float s, c;
    __sincosf(r, &s, &c);
    return make_float2(c, s);
}

__device__ __forceinline__ double u01d(uint32_t w) { return ((double)(w >> 8) + 0.5) * 5.9604644775390625e-8; }

__device__ __forceinline__ double2 box_muller_d(uint32_t wa, uint32_t wb)
{
    const double rad = sqrt(-2.0 * log(u01d(wa)));
    double s, c;
    sincospi(2.0 * u01d(wb), &s, &c);
    return make_double2(rad * c, rad * s);
}

// ----------------------------------------------------------------------------------------------
// compile-time twiddles exp(SIGN 2 pi i k / 32) from the first octant of cos(2 pi k / 32)
// ----------------------------------------------------------------------------------------------
struct Oct {
    static constexpr double c[9] = {1.0,
                                    0.98078528040323043,
                                    0.92387953251128674,
                                    0.83146961230254524,
                                    0.70710678118654757,
                                    0.55557023301960229,
                                    0.38268343236508984,
                                    0.19509032201612833,
                                    0.0};
};
constexpr double cos32(int k)
{
    k &= 31;
    return k <= 8 ? Oct::c[k] : k <= 16 ? -Oct::c[16 - k] : k <= 24 ? -Oct::c[k - 16] : Oct::c[32 - k];
}
constexpr double sin32(int k)
{
    k &= 31;
    return k <= 8 ? Oct::c[8 - k] : k <= 16 ? Oct::c[k - 8] : k <= 24 ? -Oct::c[24 - k] : -Oct::c[k - 24];
}

// v * exp(SIGN 2 pi i K / R), with the trivial factors done without multiplications
template <int R, int K, int SIGN>
__device__ __forceinline__ float2 twiddle_const(float2 v)
{
    constexpr int k32 = (K * 32 / R) & 31;
    if constexpr (k32 == 0) {
        return v;
    } else if constexpr (k32 == 8) {  // SIGN * i
        return SIGN > 0 ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    } else if constexpr (k32 == 16) {
        return make_float2(-v.x, -v.y);
    } else if constexpr (k32 == 24) {  // -SIGN * i
        return SIGN > 0 ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
    } else {
        constexpr float c = (float)cos32(k32);
        constexpr float s = (float)(SIGN * sin32(k32));
        return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
    }
}

// In-register DFT of length R on a compact array x[0..R-1] (natural order in and out),
// X[k] = sum_n x[n] exp(SIGN 2 pi i n k / R).  Recursive radix-2 decimation in time; every index
// is a compile-time constant after unrolling, so x stays in registers.  In the butterflies, a twiddle
// of +-i becomes scalar adds with the sign folded in, and one of the odd multiples of pi/4 becomes
// t = (+-o.x -+ o.y, ...) followed by e +- t / sqrt(2) as packed FMAs (2 instructions saved each).
// Any other twiddle W: with FB, x[K] = e + W o as four FMAs (the product fused into the add) and
// x[K + R/2] = 2 e - x[K] as two, 6 FMA-pipe cycles per butterfly; without FB, W o (4) then a
// packed add and subtract (2 cycles each), 8 cycles.  The two differ only in rounding.  Without
// LEAF the first butterfly level (the pairs x[j], x[j + R/2]) is taken as already done by the caller.
template <int R, int SIGN, bool FB = true, bool LEAF = true>
struct Dft {
    __device__ __forceinline__ static void run(float2* x)
    {
        float2 e[R / 2], o[R / 2];
#pragma unroll
        for (int n = 0; n < R / 2; ++n) {
            e[n] = x[2 * n];
            o[n] = x[2 * n + 1];
        }
        Dft<R / 2, SIGN, FB, LEAF>::run(e);
        Dft<R / 2, SIGN, FB, LEAF>::run(o);
        combine<0>(x, e, o);
    }
    template <int K>
    __device__ __forceinline__ static void combine(float2* x, const float2* e, const float2* o)
    {
        if constexpr (K < R / 2) {
            constexpr int k32 = (K * 32 / R) & 31;
            if constexpr (k32 == 8 || k32 == 24) {
                // o * (+-i): scalar adds with the sign folded in
                constexpr float sg = (k32 == 8) == (SIGN > 0) ? 1.0f : -1.0f;  // o * (sg i) = (-sg o.y, sg o.x)
                x[K] = make_float2(e[K].x - sg * o[K].y, e[K].y + sg * o[K].x);
                x[K + R / 2] = make_float2(e[K].x + sg * o[K].y, e[K].y - sg * o[K].x);
            } else if constexpr ((k32 & 7) == 4) {
                // W = c (sr + i si), |c| = 1/sqrt(2): W o = c t, t = (sr o.x - si o.y, sr o.y + si o.x)
                constexpr double wr = cos32(k32), wi = SIGN * sin32(k32);
                constexpr float sr = wr > 0 ? 1.0f : -1.0f, si = wi > 0 ? 1.0f : -1.0f;
                constexpr float c = 0.70710678118654752f;
                const float2 t = make_float2(sr * o[K].x - si * o[K].y, sr * o[K].y + si * o[K].x);
                x[K] = __ffma2_rn(make_float2(c, c), t, e[K]);
                x[K + R / 2] = __ffma2_rn(make_float2(-c, -c), t, e[K]);
            } else if constexpr (k32 == 0 || !FB) {
                const float2 t = twiddle_const<R, K, SIGN>(o[K]);
                x[K] = cadd(e[K], t);
                x[K + R / 2] = csub(e[K], t);
            } else {
                constexpr float c = (float)cos32(k32);
                constexpr float s = (float)(SIGN * sin32(k32));
                const float re = fmaf(c, o[K].x, fmaf(-s, o[K].y, e[K].x));
                const float im = fmaf(c, o[K].y, fmaf(s, o[K].x, e[K].y));
                x[K] = make_float2(re, im);
                x[K + R / 2] = make_float2(fmaf(2.0f, e[K].x, -re), fmaf(2.0f, e[K].y, -im));
            }
            combine<K + 1>(x, e, o);
        }
    }
};

template <int SIGN, bool FB, bool LEAF>
struct Dft<2, SIGN, FB, LEAF> {
    __device__ __forceinline__ static void run(float2* x)
    {
        if constexpr (LEAF) {
            const float2 a = x[0], b = x[1];
            x[0] = cadd(a, b);
            x[1] = csub(a, b);
        }
    }
};

template <int SIGN, bool FB, bool LEAF>
struct Dft<1, SIGN, FB, LEAF> {
    __device__ __forceinline__ static void run(float2*) {}
};

// Strided wrapper: transforms v[0], v[S], ..., v[(R-1) S].
template <int R, int SIGN, int S, bool FB = true, bool LEAF = true>
__device__ __forceinline__ void dft_strided(float2* v)
{
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = v[r * S];
    Dft<R, SIGN, FB, LEAF>::run(x);
#pragma unroll
    for (int r = 0; r < R; ++r) v[r * S] = x[r];
}

// ----------------------------------------------------------------------------------------------
// Stockham line FFT configuration.  E points per thread (default 16 for N <= 256, else 32; a kernel
// may choose another power of two), T = N / E threads per line.  Stage k has sub-length
// Ns_k = E^k and radix R_k = min(E, N / Ns_k).  FB selects the butterfly form of the in-register
// DFTs (see Dft); TF folds the twiddles of radix-32 stages into the DFT's first butterfly level
// (see fft_stage_m; the persistent N = 1024 passes use it, the per-CTA tiles measured faster without).
// ----------------------------------------------------------------------------------------------
template <int N, int EE = 0, bool FB = true, bool TF = false>
struct FftCfg {
    static constexpr bool fused_butterflies = FB;
    static constexpr bool fold_twiddles = FB && TF;
    static constexpr int E = EE ? EE : ((N <= 256) ? 16 : 32);
    static constexpr int T = N / E;
    static constexpr int stages = (N <= E) ? 1 : (N <= E * E ? 2 : 3);
    static constexpr int Ns(int k) { return k == 0 ? 1 : (k == 1 ? E : E * E); }
    static constexpr int Rk(int k) { return (N / Ns(k)) < E ? (N / Ns(k)) : E; }
    // Stage k >= 1 twiddles are stored per jm (= j mod Ns) as a row of RP(k) float2: entries r = 1..R-1
    // at (r - 1), padded so that rows are 16-byte aligned and lanes with consecutive jm reading 16-byte
    // pairs hit distinct bank groups (row stride = 4 mod 32 words).  offset of stage k = sum Ns_k' RP(k').
    static constexpr int RP(int k) { return Rk(k) == 2 ? 1 : Rk(k) + 2; }  // radix 2: one twiddle, no pad
    static constexpr int tw_off(int k)
    {
        return k <= 1 ? 0 : Ns(1) * RP(1) + (k <= 2 ? 0 : Ns(2) * RP(2));
    }
    static constexpr int tw_size = tw_off(stages);
    // twiddle table footprint in shared memory, rounded to 16 float2 so the line buffers after it keep
    // the bank alignment the padding was designed for
    static constexpr int tw_smem = ((tw_size > 0 ? tw_size : 1) + 15) / 16 * 16;
    static_assert(tw_size <= 4 * N, "twiddle tables are allocated with 4 N entries");
    // padded index inside one line's exchange buffer (in float2 units)
    __host__ __device__ static constexpr int pad(int x) { return x + x / E; }
    static constexpr int padded = N + N / E;
};

// Exchange storage of one line: element x at buf[pad(x)] (a padded per-line buffer).
template <class C>
struct PadMap {
    float2* buf;
    __device__ __forceinline__ float2* operator()(int x) const { return buf + C::pad(x); }
};

// One Stockham stage.  v[i] holds point t + i T on entry (stage input ordering).  Non-final
// stages write to the line's exchange storage (element x at map(x)) and read back the next stage's
// inputs; `bar` synchronises all threads sharing the storage.
template <class C, int K, int SIGN, class Bar, class Map>
__device__ __forceinline__ void fft_stage_m(float2 (&v)[C::E], Map map, int t, const float2* tw, Bar bar)
{
    constexpr int E = C::E, T = C::T;
    constexpr int R = C::Rk(K), Ns = C::Ns(K), B = E / R;
    constexpr bool LAST = (K == C::stages - 1);
#pragma unroll
    for (int q = 0; q < B; ++q) {
        const int j = t + q * T;
        if constexpr (K > 0) {
            const int jm = j & (Ns - 1);
            if constexpr (R == 2) {
                const float2 wa = tw[C::tw_off(K) + jm];
                v[q + B] = SIGN < 0 ? cmul(v[q + B], wa) : cmulc(v[q + B], wa);
            } else if constexpr (C::fold_twiddles && R == 32) {
                // the stage twiddles fused into the DFT's first butterfly level: for each pair
                // (r, r + R/2), a = w_r v_r, then v_r = a + w v, v_(r+R/2) = 2 a - v_r (10 FMA-pipe
                // cycles per pair instead of 12; at radix 16 the separate multiplies measured faster)
                constexpr int H = R / 2;
                const float4* w4 = reinterpret_cast<const float4*>(tw + C::tw_off(K) + jm * C::RP(K));
                auto pair = [&](int ia, float2 wa, bool twa, int ib, float2 wb) {
                    float2 a = v[q + ia * B];
                    if (twa) a = SIGN < 0 ? cmul(a, wa) : cmulc(a, wa);
                    const float2 b = v[q + ib * B];
                    const float wr = wb.x, wi = SIGN < 0 ? wb.y : -wb.y;
                    const float re = fmaf(wr, b.x, fmaf(-wi, b.y, a.x));
                    const float im = fmaf(wr, b.y, fmaf(wi, b.x, a.y));
                    v[q + ia * B] = make_float2(re, im);
                    v[q + ib * B] = make_float2(fmaf(2.0f, a.x, -re), fmaf(2.0f, a.y, -im));
                };
#pragma unroll
                for (int p = 0; p < H / 2; ++p) {
                    const float4 lo = w4[p];          // twiddles 2p + 1, 2p + 2
                    const float4 hi = w4[p + H / 2];  // twiddles 2p + 1 + H, 2p + 2 + H (the last one padding)
                    pair(2 * p + 1, make_float2(lo.x, lo.y), true, 2 * p + 1 + H, make_float2(hi.x, hi.y));
                    if (p < H / 2 - 1)
                        pair(2 * p + 2, make_float2(lo.z, lo.w), true, 2 * p + 2 + H, make_float2(hi.z, hi.w));
                    else  // twiddle H pairs with the untwiddled point 0
                        pair(0, make_float2(0.0f, 0.0f), false, H, make_float2(lo.z, lo.w));
                }
                dft_strided<R, SIGN, B, true, false>(v + q);
                continue;
            } else {
            const float4* w4 = reinterpret_cast<const float4*>(tw + C::tw_off(K) + jm * C::RP(K));
#pragma unroll
            for (int r = 1; r < R; r += 2) {
                const float4 pr = w4[(r - 1) / 2];  // twiddles r and r + 1
                const float2 wa = make_float2(pr.x, pr.y);
                v[q + r * B] = SIGN < 0 ? cmul(v[q + r * B], wa) : cmulc(v[q + r * B], wa);
                if (r + 1 < R) {
                    const float2 wb = make_float2(pr.z, pr.w);
                    v[q + (r + 1) * B] = SIGN < 0 ? cmul(v[q + (r + 1) * B], wb) : cmulc(v[q + (r + 1) * B], wb);
                }
            }
            }
        }
        dft_strided<R, SIGN, B, C::fused_butterflies>(v + q);
    }
    if constexpr (!LAST) {
#pragma unroll
        for (int q = 0; q < B; ++q) {
            const int j = t + q * T;
            const int base = (j / Ns) * Ns * R + (j & (Ns - 1));
#pragma unroll
            for (int r = 0; r < R; ++r) *map(base + r * Ns) = v[q + r * B];
        }
        bar();
#pragma unroll
        for (int i = 0; i < E; ++i) v[i] = *map(t + i * T);
        bar();
    }
}

template <class C, int K, int SIGN, class Bar>
__device__ __forceinline__ void fft_stage_c(float2 (&v)[C::E], float2* buf, int t, const float2* tw, Bar bar)
{
    fft_stage_m<C, K, SIGN>(v, PadMap<C>{buf}, t, tw, bar);
}

// Full length-N transform of one line: X[k] = sum_n x[n] exp(SIGN 2 pi i n k / N), unnormalised.
template <class C, int SIGN, class Bar, class Map>
__device__ __forceinline__ void line_fft_m(float2 (&v)[C::E], Map map, int t, const float2* tw, Bar bar)
{
    fft_stage_m<C, 0, SIGN>(v, map, t, tw, bar);
    if constexpr (C::stages > 1) fft_stage_m<C, 1, SIGN>(v, map, t, tw, bar);
    if constexpr (C::stages > 2) fft_stage_m<C, 2, SIGN>(v, map, t, tw, bar);
}

template <class C, int SIGN, class Bar>
__device__ __forceinline__ void line_fft_c(float2 (&v)[C::E], float2* buf, int t, const float2* tw, Bar bar)
{
    line_fft_m<C, SIGN>(v, PadMap<C>{buf}, t, tw, bar);
}

template <int N, int SIGN, class Bar>
__device__ __forceinline__ void line_fft(float2 (&v)[FftCfg<N>::E], float2* buf, int t, const float2* tw, Bar bar)
{
    line_fft_c<FftCfg<N>, SIGN>(v, buf, t, tw, bar);
}

// Copies the stage twiddles into shared memory (all threads of the block; caller synchronises).
template <class C>
__device__ __forceinline__ void stage_twiddles_c(float2* dst, const float2* __restrict__ src)
{
    float4* d4 = reinterpret_cast<float4*>(dst);
    const float4* s4 = reinterpret_cast<const float4*>(src);
    for (int i = threadIdx.x; i < (C::tw_size + 1) / 2; i += blockDim.x) d4[i] = __ldg(s4 + i);
}

template <int N>
__device__ __forceinline__ void stage_twiddles(float2* dst, const float2* __restrict__ src)
{
    stage_twiddles_c<FftCfg<N>>(dst, src);
}

struct WarpBar {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct BlockBar {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
// The T threads of one line (whole consecutive warps) on named barrier `id` (1..15; 0 is the block
// barrier): lines of a CTA exchange independently of one another.
template <int T>
struct LineBar {
    int id;
    __device__ __forceinline__ void operator()() const { asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(T) : "memory"); }
};

// spectral index map f(n) = n for n < N/2, else n - N
__device__ __forceinline__ int kidx(int n, int N) { return n < (N >> 1) ? n : n - N; }

}  // namespace ts
