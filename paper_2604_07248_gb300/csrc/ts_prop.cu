// ts_prop.cu -- the propagate/modulate loop of Eq. 1 as two fused passes per step.
//
// The field is kept between steps in the "row-frequency" domain R = FFT_rows(U).  One step is
//   column pass:  C = IFFT_cols( H . FFT_cols(R) )          (H includes the 1/N^2 of IFFT2)
//   row pass:     U = IFFT_rows(C) . exp(i phi_s);  R = FFT_rows(U)   (next step)
// so each step reads and writes the field twice and reads the screen once (36 B per pixel).
// Row passes give each line of N points to T = N / E threads (E points per thread, registers);
// column passes load W adjacent columns per CTA so that every warp load touches W*8 contiguous
// bytes of each of 32 / W rows.
#include <type_traits>

#include "ts_device.cuh"
#include "ts_internal.h"

namespace ts {

namespace {

constexpr int kRowThreads = 256;

struct RowParams {
    float2* field;
    const float* phi;
    long long phi_set_stride;
    int phi_group;
    float phase_sign;
    float* intensity;
    double* rows;
    const float2* tw;
    int n_src;
    float src_coef[kMaxSources];
};

template <int N>
struct RowCfg {
    using C = FftCfg<N>;
    static constexpr int LPC = kRowThreads / C::T;  // lines per CTA
    static constexpr int LS = C::padded;            // line stride in shared memory (float2)
    static constexpr int WPL = C::T > 32 ? C::T / 32 : 1;  // warps per line
    static constexpr size_t smem = sizeof(float2) * LPC * LS;
};

template <int N, int FLAGS>
__global__ void __launch_bounds__(kRowThreads) row_pass_kernel(const RowParams a)
{
    using C = FftCfg<N>;
    using RC = RowCfg<N>;
    constexpr int E = C::E, T = C::T;
    extern __shared__ float2 smem[];
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int j = blockIdx.x * RC::LPC + line;
    const int b = blockIdx.y;
    float2* buf = smem + line * RC::LS;
    float2* row = a.field + ((size_t)b * N + j) * N;
    using Bar = typename std::conditional<(T > 32), BlockBar, WarpBar>::type;

    float2 v[E];
    if constexpr (FLAGS & RP_IN_SOURCE) {
        const float coef = a.src_coef[b % a.n_src];
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
    if constexpr (FLAGS & RP_IN_FREQ) line_fft<N, +1>(v, buf, t, a.tw, Bar());
    if constexpr (FLAGS & RP_PHASE) {
        if (a.phi != nullptr) {
            const float* ph = a.phi + (long long)(b / a.phi_group) * a.phi_set_stride + (size_t)j * N;
#pragma unroll
            for (int i = 0; i < E; ++i) {
                float s, c;
                sincosf(__ldg(ph + t + i * T), &s, &c);
                v[i] = cmul(v[i], make_float2(c, a.phase_sign * s));
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
    if constexpr (FLAGS & RP_OUT_FREQ) line_fft<N, -1>(v, buf, t, a.tw, Bar());
    if constexpr (FLAGS & RP_STORE) {
#pragma unroll
        for (int i = 0; i < E; ++i) row[t + i * T] = v[i];
    }
}

struct ColParams {
    float2* field;
    const float2* tw;
    const float2* P;
    float dcoef;
    float inv_k2;
    float dk;
};

template <int N>
struct ColCfg {
    using C = FftCfg<N>;
    static constexpr int THREADS = 256;
    static constexpr int W = THREADS / C::T;                        // columns per CTA
    static constexpr int LS = C::padded + (16 / W > 1 ? 16 / W : 1);  // conflict-free column stride
    static constexpr size_t smem = sizeof(float2) * W * LS;
};

// H(ky, kx) = P(kx) P(ky) exp(-i delta), delta = dz kappa^4 / (2k (k + sqrt(k^2 - kappa^2))^2), the
// exact angular-spectrum phase beyond its paraxial part; 0 in the evanescent region.
__device__ __forceinline__ float2 transfer(float2 px, float2 py, float k2, float inv_k2, float dcoef)
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

template <int N, bool CONJ>
__global__ void __launch_bounds__(ColCfg<N>::THREADS) col_pass_kernel(const ColParams a)
{
    using C = FftCfg<N>;
    using CC = ColCfg<N>;
    constexpr int E = C::E, T = C::T, W = CC::W;
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % W, t = threadIdx.x / W;
    const int col = blockIdx.x * W + c;
    float2* buf = smem + c * CC::LS;
    float2* base = a.field + (size_t)blockIdx.y * N * N + col;

    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = base[(size_t)(t + i * T) * N];
    line_fft<N, -1>(v, buf, t, a.tw, BlockBar());
    const float kx = a.dk * (float)kidx(col, N);
    const float2 px = __ldg(a.P + col);
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int m = t + i * T;
        const float ky = a.dk * (float)kidx(m, N);
        const float2 h = transfer(px, __ldg(a.P + m), fmaf(kx, kx, ky * ky), a.inv_k2, a.dcoef);
        v[i] = CONJ ? cmulc(v[i], h) : cmul(v[i], h);
    }
    line_fft<N, +1>(v, buf, t, a.tw, BlockBar());
#pragma unroll
    for (int i = 0; i < E; ++i) base[(size_t)(t + i * T) * N] = v[i];
}

// sum over rows (fixed order) of per-row beam sums; out[b] = (sum I, dx^2 sum r^2 I)
__global__ void row_sums_kernel(const double* rows, int B, int N, int wpl, double dx2, double* out)
{
    const int b = blockIdx.x;
    __shared__ double red[2][256];
    double s0 = 0.0, s1 = 0.0;
    for (int idx = threadIdx.x; idx < N * wpl; idx += blockDim.x) {
        s0 += rows[((size_t)b * N * wpl + idx) * 2];
        s1 += rows[((size_t)b * N * wpl + idx) * 2 + 1];
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * b] = red[0][0];
        out[2 * b + 1] = red[1][0] * dx2;
    }
}

template <int N, int FLAGS>
cudaError_t row_launch(const RowParams& rp, int B, cudaStream_t st)
{
    using RC = RowCfg<N>;
    dim3 grid(N / RC::LPC, B);
    row_pass_kernel<N, FLAGS><<<grid, kRowThreads, RC::smem, st>>>(rp);
    return cudaGetLastError();
}

template <int N>
cudaError_t row_dispatch(int flags, const RowParams& rp, int B, cudaStream_t st)
{
    switch (flags) {
    case RP_IN_SOURCE | RP_STORE: return row_launch<N, RP_IN_SOURCE | RP_STORE>(rp, B, st);
    case RP_IN_SOURCE | RP_OUT_FREQ | RP_STORE: return row_launch<N, RP_IN_SOURCE | RP_OUT_FREQ | RP_STORE>(rp, B, st);
    case RP_OUT_FREQ | RP_STORE: return row_launch<N, RP_OUT_FREQ | RP_STORE>(rp, B, st);
    case RP_PHASE | RP_OUT_FREQ | RP_STORE: return row_launch<N, RP_PHASE | RP_OUT_FREQ | RP_STORE>(rp, B, st);
    case RP_IN_FREQ | RP_PHASE | RP_OUT_FREQ | RP_STORE:
        return row_launch<N, RP_IN_FREQ | RP_PHASE | RP_OUT_FREQ | RP_STORE>(rp, B, st);
    case RP_IN_FREQ | RP_PHASE | RP_STORE: return row_launch<N, RP_IN_FREQ | RP_PHASE | RP_STORE>(rp, B, st);
    case RP_IN_FREQ | RP_PHASE | RP_INTENSITY | RP_STORE:
        return row_launch<N, RP_IN_FREQ | RP_PHASE | RP_INTENSITY | RP_STORE>(rp, B, st);
    case RP_IN_FREQ | RP_PHASE | RP_INTENSITY: return row_launch<N, RP_IN_FREQ | RP_PHASE | RP_INTENSITY>(rp, B, st);
    case RP_IN_FREQ | RP_STORE: return row_launch<N, RP_IN_FREQ | RP_STORE>(rp, B, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int N, bool CONJ>
cudaError_t col_launch(const ColParams& cp, int B, cudaStream_t st)
{
    using CC = ColCfg<N>;
    dim3 grid(N / CC::W, B);
    col_pass_kernel<N, CONJ><<<grid, CC::THREADS, CC::smem, st>>>(cp);
    return cudaGetLastError();
}

template <int N, int FLAGS>
cudaError_t row_attr()
{
    return cudaFuncSetAttribute(row_pass_kernel<N, FLAGS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)RowCfg<N>::smem);
}

template <int N>
cudaError_t prepare_prop_for()
{
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    chk(row_attr<N, RP_IN_SOURCE | RP_STORE>());
    chk(row_attr<N, RP_IN_SOURCE | RP_OUT_FREQ | RP_STORE>());
    chk(row_attr<N, RP_OUT_FREQ | RP_STORE>());
    chk(row_attr<N, RP_PHASE | RP_OUT_FREQ | RP_STORE>());
    chk(row_attr<N, RP_IN_FREQ | RP_PHASE | RP_OUT_FREQ | RP_STORE>());
    chk(row_attr<N, RP_IN_FREQ | RP_PHASE | RP_STORE>());
    chk(row_attr<N, RP_IN_FREQ | RP_PHASE | RP_INTENSITY | RP_STORE>());
    chk(row_attr<N, RP_IN_FREQ | RP_PHASE | RP_INTENSITY>());
    chk(row_attr<N, RP_IN_FREQ | RP_STORE>());
    chk(cudaFuncSetAttribute(col_pass_kernel<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ColCfg<N>::smem));
    chk(cudaFuncSetAttribute(col_pass_kernel<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ColCfg<N>::smem));
    return e;
}

template <int N>
int wpl_of()
{
    return RowCfg<N>::WPL;
}

}  // namespace

cudaError_t launch_row_pass(const Plan& p, int flags, const RowArgs& a, cudaStream_t st)
{
    RowParams rp;
    rp.field = a.field;
    rp.phi = a.phi;
    rp.phi_set_stride = a.phi_set_stride;
    rp.phi_group = a.phi_group > 0 ? a.phi_group : 1;
    rp.phase_sign = a.phase_sign;
    rp.intensity = a.intensity;
    rp.rows = a.rows;
    rp.tw = p.tw;
    rp.n_src = p.n_src > 0 ? p.n_src : 1;
    for (int i = 0; i < kMaxSources; ++i) rp.src_coef[i] = i < p.n_src ? p.src_coef[i] : -1.0f;
    switch (p.N) {
    case 128: return row_dispatch<128>(flags, rp, a.B, st);
    case 256: return row_dispatch<256>(flags, rp, a.B, st);
    case 512: return row_dispatch<512>(flags, rp, a.B, st);
    case 1024: return row_dispatch<1024>(flags, rp, a.B, st);
    case 2048: return row_dispatch<2048>(flags, rp, a.B, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_col_pass(const Plan& p, int step, bool conj, float2* field, int B, cudaStream_t st)
{
    ColParams cp;
    cp.field = field;
    cp.tw = p.tw;
    cp.P = p.P + (size_t)step * p.N;
    cp.dcoef = (float)(p.dz[step] / (2.0 * p.k * p.k * p.k));
    cp.inv_k2 = (float)(1.0 / (p.k * p.k));
    cp.dk = (float)p.dk;
#define TS_COL(NN) \
    case NN: return conj ? col_launch<NN, true>(cp, B, st) : col_launch<NN, false>(cp, B, st);
    switch (p.N) {
        TS_COL(128)
        TS_COL(256)
        TS_COL(512)
        TS_COL(1024)
        TS_COL(2048)
    default: return cudaErrorInvalidValue;
    }
#undef TS_COL
}

cudaError_t prepare_prop_kernels(int N)
{
    switch (N) {
    case 128: return prepare_prop_for<128>();
    case 256: return prepare_prop_for<256>();
    case 512: return prepare_prop_for<512>();
    case 1024: return prepare_prop_for<1024>();
    case 2048: return prepare_prop_for<2048>();
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_row_sums(const Plan& p, const double* rows, int B, double* out, cudaStream_t st)
{
    int wpl = 1;
    switch (p.N) {
    case 128: wpl = wpl_of<128>(); break;
    case 256: wpl = wpl_of<256>(); break;
    case 512: wpl = wpl_of<512>(); break;
    case 1024: wpl = wpl_of<1024>(); break;
    case 2048: wpl = wpl_of<2048>(); break;
    }
    row_sums_kernel<<<B, 256, 0, st>>>(rows, B, p.N, wpl, p.dx * p.dx, out);
    return cudaGetLastError();
}

}  // namespace ts
