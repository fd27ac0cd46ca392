// ts_tables.cu -- per-plan tables, computed on the GPU in double precision and stored in the
// precision the kernels read them in.
#include "ts_device.cuh"
#include "ts_internal.h"

namespace ts {

namespace {

// Stockham stage twiddles exp(-2 pi i jm r / (Ns R)) for stages k >= 1 (forward sign).
template <class C>
__global__ void twiddle_kernel(float2* tw)
{
    for (int k = 1; k < C::stages; ++k) {
        const int R = C::Rk(k), Ns = C::Ns(k), RP = C::RP(k);
        for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < RP * Ns; idx += gridDim.x * blockDim.x) {
            const int jm = idx / RP, r = idx % RP + 1;
            float2 w = make_float2(0.0f, 0.0f);  // padding entries
            if (r < R) {
                double s, c;
                sincospi(-2.0 * (double)jm * (double)r / (double)(Ns * R), &s, &c);
                w = make_float2((float)c, (float)s);
            }
            tw[C::tw_off(k) + idx] = w;
        }
    }
}

// P[s][n] = exp(-i dz_s (kappa_n^2 / 2k [+ kappa_n^4 / 8k^3])) / N: the per-axis factors of H (Sec. 2.4;
// 1/N per axis).  The quartic term is included when the kernels use the separable form.
__global__ void paraxial_kernel(float2* P, const double* dz, int S, int N, double dk, double k, int quartic)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < S * N; idx += gridDim.x * blockDim.x) {
        const int s = idx / N, n = idx % N;
        const double kap = dk * (double)kidx(n, N);
        const double k2 = kap * kap;
        const double ph = -dz[s] * (k2 / (2.0 * k) + (quartic ? k2 * k2 / (8.0 * k * k * k) : 0.0));
        double sn, cs;
        sincos(ph, &sn, &cs);
        P[idx] = make_float2((float)(cs / N), (float)(sn / N));
    }
}

// PSD shape g = (kappa^2 + kappa0^2)^expo exp(-kappa^2 / (2 kappa_m^2)), g(0) = 0, expo = -alpha/4
// (-11/12 for Kolmogorov), so that s(kappa) = sqrt(Phi_phi) dkappa = amp_s g (S14, S16, S17; power
// law of Table S1 / S15).
__global__ void psd_shape_kernel(float* g, int N, double dk, double k0sq, double inv_kmsq, double expo)
{
    const size_t total = (size_t)N * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(idx / N), n = (int)(idx % N);
        const double kx = dk * kidx(n, N), ky = dk * kidx(m, N);
        const double k2 = kx * kx + ky * ky;
        double v = 0.0;
        if (m != 0 || n != 0) v = pow(k2 + k0sq, expo) * exp(-0.5 * k2 * inv_kmsq);
        g[idx] = (float)v;
    }
}

// Subharmonic bases: shx[p][i] = exp(i dkappa_p i dx) (FP64), shy[p][j] = (cos, sin)(dkappa_p j dx),
// shy_mean[p] = mean over j of (cos, sin)(dkappa_p j dx), dkappa_p = dkappa / 3^p.
__global__ void sh_basis_kernel(double2* shx, float2* shy, double2* shy_mean, int N, double dk, double dx)
{
    __shared__ double red[2][256];
    for (int p = 0; p < 3; ++p) {
        const double dkp = dk / pow(3.0, p + 1);
        double sc = 0.0, ss = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            double sn, cs;
            sincos(dkp * (double)i * dx, &sn, &cs);
            shx[p * N + i] = make_double2(cs, sn);
            shy[p * N + i] = make_float2((float)cs, (float)sn);
            sc += cs;
            ss += sn;
        }
        red[0][threadIdx.x] = sc;
        red[1][threadIdx.x] = ss;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) {
                red[0][threadIdx.x] += red[0][threadIdx.x + w];
                red[1][threadIdx.x] += red[1][threadIdx.x + w];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) shy_mean[p] = make_double2(red[0][0] / N, red[1][0] / N);
        __syncthreads();
    }
}

// AR translation factors (Eq. 4): tilt[0][n] = exp(-i T vx kappa_n), tilt[1][m] = exp(-i T vy kappa_m).
__global__ void tilt_kernel(float2* tilt, int N, double dk, double vx, double vy, double T)
{
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 2 * N; idx += gridDim.x * blockDim.x) {
        const int axis = idx / N, n = idx % N;
        const double v = axis == 0 ? vx : vy;
        double sn, cs;
        sincos(-T * v * dk * (double)kidx(n, N), &sn, &cs);
        tilt[idx] = make_float2((float)cs, (float)sn);
    }
}

__global__ void philox_kernel(const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1, int n, uint32_t* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const u32x4 w = philox4x32_10(u32x4{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]}, k0, k1);
    out[4 * i] = w.a;
    out[4 * i + 1] = w.b;
    out[4 * i + 2] = w.c;
    out[4 * i + 3] = w.d;
}

template <int N>
cudaError_t twiddles_for(float2* tw)
{
    twiddle_kernel<FftCfg<N>><<<8, 256>>>(tw);
    return cudaGetLastError();
}

template <int N>
cudaError_t twiddles16_for(float2* tw)
{
    twiddle_kernel<FftCfg<N, 16>><<<8, 256>>>(tw);
    return cudaGetLastError();
}

}  // namespace

cudaError_t build_tables(Plan& p)
{
    cudaError_t e = cudaSuccess;
    switch (p.N) {
    case 128: e = twiddles_for<128>(p.tw); break;
    case 256: e = twiddles_for<256>(p.tw); break;
    case 512: e = twiddles_for<512>(p.tw); break;
    case 1024: e = twiddles_for<1024>(p.tw); break;
    case 2048: e = twiddles_for<2048>(p.tw); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    if (p.tw16 != p.tw) {
        switch (p.N) {
        case 512: e = twiddles16_for<512>(p.tw16); break;
        case 1024: e = twiddles16_for<1024>(p.tw16); break;
        case 2048: e = twiddles16_for<2048>(p.tw16); break;
        default: break;
        }
        if (e != cudaSuccess) return e;
    }

    double* dz_d = nullptr;
    e = cudaMalloc(&dz_d, sizeof(double) * p.S);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(dz_d, p.dz, sizeof(double) * p.S, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        paraxial_kernel<<<64, 256>>>(p.P, dz_d, p.S, p.N, p.dk, p.k, p.sep_transfer ? 1 : 0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(dz_d);
    if (e != cudaSuccess) return e;

    const double k0sq = (p.L0 > 0.0 && isfinite(p.L0)) ? (2.0 * M_PI / p.L0) * (2.0 * M_PI / p.L0) : 0.0;
    const double inv_kmsq = p.l0 > 0.0 ? 1.0 / ((2.0 * M_PI / p.l0) * (2.0 * M_PI / p.l0)) : 0.0;
    psd_shape_kernel<<<1024, 256>>>(p.g, p.N, p.dk, k0sq, inv_kmsq, -p.psd_alpha / 4.0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (p.sh_levels > 0) {
        sh_basis_kernel<<<1, 256>>>(p.shx, p.shy, p.shy_mean, p.N, p.dk, p.dx);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaDeviceSynchronize();
}

cudaError_t launch_twiddles(int N, float2* tw, cudaStream_t st)
{
    switch (N) {
    case 128: twiddle_kernel<FftCfg<128>><<<8, 256, 0, st>>>(tw); break;
    case 256: twiddle_kernel<FftCfg<256>><<<8, 256, 0, st>>>(tw); break;
    case 512: twiddle_kernel<FftCfg<512>><<<8, 256, 0, st>>>(tw); break;
    case 1024: twiddle_kernel<FftCfg<1024>><<<8, 256, 0, st>>>(tw); break;
    case 2048: twiddle_kernel<FftCfg<2048>><<<8, 256, 0, st>>>(tw); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_psd_shape(int N, float* g, double dk, double L0, double l0, cudaStream_t st)
{
    const double k0sq = (L0 > 0.0 && isfinite(L0)) ? (2.0 * M_PI / L0) * (2.0 * M_PI / L0) : 0.0;
    const double inv_kmsq = l0 > 0.0 ? 1.0 / ((2.0 * M_PI / l0) * (2.0 * M_PI / l0)) : 0.0;
    psd_shape_kernel<<<1024, 256, 0, st>>>(g, N, dk, k0sq, inv_kmsq, -11.0 / 12.0);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int n, uint32_t* out, cudaStream_t st)
{
    philox_kernel<<<(n + 255) / 256, 256, 0, st>>>(ctr, k0, k1, n, out);
    return cudaGetLastError();
}

cudaError_t build_tilt(Plan& p, double vx, double vy, double T, cudaStream_t st)
{
    tilt_kernel<<<(2 * p.N + 255) / 256, 256, 0, st>>>(p.tilt, p.N, p.dk, vx, vy, T);
    return cudaGetLastError();
}

}  // namespace ts
