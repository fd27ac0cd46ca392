// ts_d2nn.cu -- two-mask dual-domain D2NN receiver (Sec. 2.5, 4.1): forward and adjoint.
//
// With the checkerboard s(i, j) = (-1)^(i+j) and N divisible by 4, the centred unitary lens DFT is
//   C(x) = s . FFT2(s . x) / N,   C^-1(y) = s . IFFT2(s . y) / N   (IFFT2 unnormalised),
// pixel by pixel in the centred layout, so the receiver
//   Z1 = exp(i th1) A U,  W2 = exp(i th2) C(Z1),  V = C^-1(W2) = s . IFFT2(exp(i th2) FFT2(s Z1)) / N^2
// is one row pass, one column pass and one row pass, like a propagation step.  The adjoint
//   g_V = 2 V dL/dI,  g_W2 = C(g_V),  dth2 = sum_b Im(g_W2 conj W2),
//   g_Z1 = C^-1(exp(-i th2) g_W2) = s . IFFT2(exp(-i th2) FFT2(s g_V)) / N^2,
//   dth1 = sum_b Im(g_Z1 conj Z1),  g_U = A exp(-i th1) g_Z1
// has the same shape.  Per-field mask gradients are written in place of W2 / Z1 in the workspace and
// summed over the batch in a fixed order (deterministic).
#include <type_traits>

#include "ts_device.cuh"
#include "ts_internal.h"

namespace ts {

namespace {

struct D2Params {
    const float2* in;   // input field (forward row pass A) or workspace V (backward row pass A)
    float2* work;       // [B][N][N] transformed field
    float2* z1;         // [B][N][N] Z1 (forward: written; backward: read, then dth1 partial written)
    float2* w2;         // [B][N][N] W2 (forward: written; backward: read, then dth2 partial written)
    float2* v;          // [B][N][N] V
    float* I;           // [B][N][N]
    const float* Iref;  // [N][N]
    const float* th1;
    const float* th2;
    float2* gU;         // backward output
    double* rows;       // [B][N] loss partials
    const float2* tw;
    float r2ap;         // (aperture radius / dx)^2
    float inv_count;    // 1 / (B N^2)
    int kind;           // 0 MAE, 1 squared error
};

template <int N>
struct DRowCfg {
    using C = FftCfg<N>;
    static constexpr int THREADS = 256;
    static constexpr int LPC = THREADS / C::T;
    static constexpr int LS = C::padded;
    static constexpr size_t smem = sizeof(float2) * (C::tw_smem + LPC * LS);
};

template <int N>
struct DColCfg {
    using C = FftCfg<N>;
    static constexpr int THREADS = 256;
    static constexpr int W = THREADS / C::T;
    static constexpr int LS = C::padded + (16 / W > 1 ? 16 / W : 1);
    static constexpr size_t smem = sizeof(float2) * (C::tw_smem + W * LS);
};

__device__ __forceinline__ float checker(int i, int j) { return ((i + j) & 1) ? -1.0f : 1.0f; }

__device__ __forceinline__ float dldi(float I, float Iref, int kind, float inv_count)
{
    const float e = I - Iref;
    if (kind == 0) return (e > 0.0f ? 1.0f : (e < 0.0f ? -1.0f : 0.0f)) * inv_count;
    return 2.0f * e * inv_count;
}

// Forward row pass A: Z1 = exp(i th1) A U (stored), row FFT of s Z1 -> work.
// Backward row pass A: g_V = 2 V dL/dI (from V, I, Iref), row FFT of s g_V -> work.
template <int N, bool BACKWARD>
__global__ void __launch_bounds__(256) d2_row_a(const D2Params a)
{
    using C = FftCfg<N>;
    using RC = DRowCfg<N>;
    constexpr int E = C::E, T = C::T;
    extern __shared__ float2 smem[];
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int j = blockIdx.x * RC::LPC + line;
    const size_t rowoff = ((size_t)blockIdx.y * N + j) * N;
    float2* tw = smem;
    float2* buf = smem + C::tw_smem + line * RC::LS;
    stage_twiddles<N>(tw, a.tw);
    __syncthreads();
    using Bar = typename std::conditional<(T > 32), BlockBar, WarpBar>::type;
    const float y = (float)(j - N / 2);
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int x = t + i * T;
        if constexpr (!BACKWARD) {
            const float xf = (float)(x - N / 2);
            const float A = (xf * xf + y * y <= a.r2ap) ? 1.0f : 0.0f;
            float sn, cs;
            sincosf(__ldg(a.th1 + (size_t)j * N + x), &sn, &cs);
            const float2 z = cscale(cmul(a.in[rowoff + x], make_float2(cs, sn)), A);
            a.z1[rowoff + x] = z;
            v[i] = cscale(z, checker(x, j));
        } else {
            const float2 V = a.v[rowoff + x];
            const float g = 2.0f * dldi(a.I[rowoff + x], __ldg(a.Iref + (size_t)j * N + x), a.kind, a.inv_count);
            v[i] = cscale(V, g * checker(x, j));
        }
    }
    line_fft<N, -1>(v, buf, t, tw, Bar());
#pragma unroll
    for (int i = 0; i < E; ++i) a.work[rowoff + t + i * T] = v[i];
}

// Column pass: column FFT completes F = FFT2(s x); forward stores W2 = exp(i th2) s F / N and
// multiplies by exp(i th2) / N^2; backward forms g_W2 = s F / N, writes Im(g_W2 conj W2) over W2 and
// multiplies by exp(-i th2) / N^2.  Column IFFT -> work.
template <int N, bool BACKWARD>
__global__ void __launch_bounds__(256) d2_col(const D2Params a)
{
    using C = FftCfg<N>;
    using CC = DColCfg<N>;
    constexpr int E = C::E, T = C::T, W = CC::W;
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % W, t = threadIdx.x / W;
    const int col = blockIdx.x * W + c;
    float2* tw = smem;
    float2* buf = smem + C::tw_smem + c * CC::LS;
    stage_twiddles<N>(tw, a.tw);
    __syncthreads();
    const size_t base = (size_t)blockIdx.y * N * N + col;
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = a.work[base + (size_t)(t + i * T) * N];
    line_fft<N, -1>(v, buf, t, tw, BlockBar());
    const float invN = 1.0f / (float)N;
#pragma unroll
    for (int i = 0; i < E; ++i) {
        const int k = t + i * T;
        const size_t o = base + (size_t)k * N;
        float sn, cs;
        sincosf(__ldg(a.th2 + (size_t)k * N + col), &sn, &cs);
        const float2 F = cscale(v[i], checker(col, k) * invN);  // C(.) at pixel (k, col)
        if constexpr (!BACKWARD) {
            a.w2[o] = cmul(F, make_float2(cs, sn));
            v[i] = cmul(v[i], make_float2(cs * invN * invN, sn * invN * invN));
        } else {
            const float2 W2 = a.w2[o];
            a.w2[o] = make_float2(fmaf(F.y, W2.x, -F.x * W2.y), 0.0f);  // Im(g_W2 conj W2)
            v[i] = cmul(v[i], make_float2(cs * invN * invN, -sn * invN * invN));
        }
    }
    line_fft<N, +1>(v, buf, t, tw, BlockBar());
#pragma unroll
    for (int i = 0; i < E; ++i) a.work[base + (size_t)(t + i * T) * N] = v[i];
}

// Forward row pass B: V = s IFFT_rows(work); I = |V|^2; loss partial per row.
// Backward row pass B: g_Z1 = s IFFT_rows(work); Im(g_Z1 conj Z1) over Z1; g_U = A exp(-i th1) g_Z1.
template <int N, bool BACKWARD>
__global__ void __launch_bounds__(256) d2_row_b(const D2Params a)
{
    using C = FftCfg<N>;
    using RC = DRowCfg<N>;
    constexpr int E = C::E, T = C::T;
    extern __shared__ float2 smem[];
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int j = blockIdx.x * RC::LPC + line;
    const int b = blockIdx.y;
    const size_t rowoff = ((size_t)b * N + j) * N;
    float2* tw = smem;
    float2* buf = smem + C::tw_smem + line * RC::LS;
    stage_twiddles<N>(tw, a.tw);
    __syncthreads();
    using Bar = typename std::conditional<(T > 32), BlockBar, WarpBar>::type;
    float2 v[E];
#pragma unroll
    for (int i = 0; i < E; ++i) v[i] = a.work[rowoff + t + i * T];
    line_fft<N, +1>(v, buf, t, tw, Bar());
    const float y = (float)(j - N / 2);
    if constexpr (!BACKWARD) {
        double acc = 0.0;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int x = t + i * T;
            const float2 V = cscale(v[i], checker(x, j));
            const float I = V.x * V.x + V.y * V.y;
            a.v[rowoff + x] = V;
            a.I[rowoff + x] = I;
            const float e = I - __ldg(a.Iref + (size_t)j * N + x);
            acc += a.kind == 0 ? (double)fabsf(e) : (double)e * (double)e;
        }
        constexpr int width = T < 32 ? T : 32;
#pragma unroll
        for (int off = width / 2; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, width);
        if ((t % width) == 0) a.rows[((size_t)b * N + j) * (T > 32 ? T / 32 : 1) + t / 32] = acc;
    } else {
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int x = t + i * T;
            const float2 g = cscale(v[i], checker(x, j));
            const float2 Z1 = a.z1[rowoff + x];
            a.z1[rowoff + x] = make_float2(fmaf(g.y, Z1.x, -g.x * Z1.y), 0.0f);  // Im(g conj Z1)
            const float xf = (float)(x - N / 2);
            const float A = (xf * xf + y * y <= a.r2ap) ? 1.0f : 0.0f;
            float sn, cs;
            sincosf(__ldg(a.th1 + (size_t)j * N + x), &sn, &cs);
            a.gU[rowoff + x] = cscale(cmul(g, make_float2(cs, -sn)), A);
        }
    }
}

// out[p] = sum_b part[b][p].x in increasing b (deterministic batch sum of per-field mask gradients)
__global__ void batch_sum_kernel(const float2* __restrict__ part, int B, size_t npix, float* out)
{
    const size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (p >= npix) return;
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s += part[(size_t)b * npix + p].x;
    out[p] = s;
}

__global__ void loss_sum_kernel(const double* rows, int n, double scale, double* loss)
{
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += rows[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] * scale;
}

template <int N>
cudaError_t d2_for(const Plan& p, bool backward, const D2Params& a, int B, cudaStream_t st)
{
    using RC = DRowCfg<N>;
    using CC = DColCfg<N>;
    dim3 rg(N / RC::LPC, B), cg(N / CC::W, B);
    if (!backward) {
        d2_row_a<N, false><<<rg, 256, RC::smem, st>>>(a);
        d2_col<N, false><<<cg, 256, CC::smem, st>>>(a);
        d2_row_b<N, false><<<rg, 256, RC::smem, st>>>(a);
    } else {
        d2_row_a<N, true><<<rg, 256, RC::smem, st>>>(a);
        d2_col<N, true><<<cg, 256, CC::smem, st>>>(a);
        d2_row_b<N, true><<<rg, 256, RC::smem, st>>>(a);
    }
    return cudaGetLastError();
}

template <int N>
cudaError_t prepare_d2_for()
{
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    const int rs = (int)DRowCfg<N>::smem, cs = (int)DColCfg<N>::smem;
    chk(cudaFuncSetAttribute(d2_row_a<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs));
    chk(cudaFuncSetAttribute(d2_row_a<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs));
    chk(cudaFuncSetAttribute(d2_row_b<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs));
    chk(cudaFuncSetAttribute(d2_row_b<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, rs));
    chk(cudaFuncSetAttribute(d2_col<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs));
    chk(cudaFuncSetAttribute(d2_col<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, cs));
    return e;
}

}  // namespace

cudaError_t prepare_d2nn_kernels(int N)
{
    switch (N) {
    case 128: return prepare_d2_for<128>();
    case 256: return prepare_d2_for<256>();
    case 512: return prepare_d2_for<512>();
    case 1024: return prepare_d2_for<1024>();
    case 2048: return prepare_d2_for<2048>();
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_d2nn(const Plan& p, bool backward, const D2nnArgs& d, cudaStream_t st)
{
    const int N = p.N;
    const size_t N2 = (size_t)N * N;
    D2Params a;
    a.in = backward ? nullptr : d.U;
    a.z1 = d.ws;
    a.w2 = d.ws + (size_t)d.B * N2;
    a.v = d.ws + 2 * (size_t)d.B * N2;
    a.work = a.v;  // transformed field shares the V slot (each pass reads and writes its own rows/columns)
    a.I = d.I;
    a.Iref = d.Iref;
    a.th1 = d.th1;
    a.th2 = d.th2;
    a.gU = d.gU;
    a.rows = p.ws_rows;
    a.tw = p.tw;
    const double rad = 0.5 * d.aperture / p.dx;
    a.r2ap = (float)(rad * rad);
    a.inv_count = (float)(p.loss_scale / ((double)d.B * (double)N2));
    a.kind = d.kind;
    cudaError_t e = cudaSuccess;
    switch (N) {
    case 128: e = d2_for<128>(p, backward, a, d.B, st); break;
    case 256: e = d2_for<256>(p, backward, a, d.B, st); break;
    case 512: e = d2_for<512>(p, backward, a, d.B, st); break;
    case 1024: e = d2_for<1024>(p, backward, a, d.B, st); break;
    case 2048: e = d2_for<2048>(p, backward, a, d.B, st); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (!backward) {
        const int per_row = (N == 2048) ? 2 : 1;  // one partial per warp of a line
        loss_sum_kernel<<<1, 256, 0, st>>>(p.ws_rows, d.B * N * per_row, p.loss_scale / ((double)d.B * (double)N2),
                                           d.loss);
    } else {
        const unsigned grid = (unsigned)((N2 + 255) / 256);
        batch_sum_kernel<<<grid, 256, 0, st>>>(a.z1, d.B, N2, d.g_th1);
        batch_sum_kernel<<<grid, 256, 0, st>>>(a.w2, d.B, N2, d.g_th2);
    }
    return cudaGetLastError();
}

}  // namespace ts
