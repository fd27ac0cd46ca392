// ts_moments.cu -- per-pixel intensity moments across realizations in FP64 (S25, Welford), and the
// long-term beam radius W_LT from the accumulated beam sums (S23 / S24).
//
// Each call merges one chunk (the fields of a group) into running (count, mean, M2) with the
// pairwise update of Chan, Golub and LeVeque: the chunk's own mean and M2 are formed in FP64 by two
// passes over its intensities (read from L2 the second time), then
//   delta = mean_c - mean;  mean += delta n_c / n;  M2 += M2_c + delta^2 count n_c / n.
// The weights are host-computed FP64 scalars, so the kernel has no per-pixel division.
#include "ts_device.cuh"
#include "ts_internal.h"

namespace ts {

namespace {

__global__ void __launch_bounds__(256) moments_kernel(const float* __restrict__ I, int B, int G, size_t npix,
                                                      double inv_nc, double w_mean, double w_m2, bool first,
                                                      double* __restrict__ mean, double* __restrict__ m2)
{
    const size_t pix = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const int g = blockIdx.y;
    if (pix >= npix) return;
    double sum = 0.0;
    for (int b = g; b < B; b += G) sum += (double)__ldg(I + (size_t)b * npix + pix);
    const double mc = sum * inv_nc;
    double mc2 = 0.0;
    for (int b = g; b < B; b += G) {
        const double d = (double)__ldg(I + (size_t)b * npix + pix) - mc;
        mc2 = fma(d, d, mc2);
    }
    const size_t o = (size_t)g * npix + pix;
    if (first) {
        mean[o] = mc;
        m2[o] = mc2;
    } else {
        const double ma = mean[o];
        const double d = mc - ma;
        mean[o] = fma(d, w_mean, ma);
        m2[o] = m2[o] + mc2 + d * d * w_m2;
    }
}

__global__ void __launch_bounds__(256) si_kernel(const double* __restrict__ mean, const double* __restrict__ m2,
                                                 size_t npix, double inv_count, double* si_map, double* si_mean,
                                                 double* si_center, size_t center)
{
    const int g = blockIdx.x;
    __shared__ double red[256];
    double acc = 0.0;
    for (size_t pix = threadIdx.x; pix < npix; pix += blockDim.x) {
        const size_t o = (size_t)g * npix + pix;
        const double mu = mean[o];
        const double si = (m2[o] * inv_count) / (mu * mu);
        if (si_map) si_map[o] = si;
        acc += si;
        if (si_center && pix == center) si_center[g] = si;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0 && si_mean) si_mean[g] = red[0] / (double)npix;
}

// Beam sums of one chunk, per group, in increasing field order (FP64): the long-term spot's zeroth
// and second moments accumulated over realizations (S23 / S24).
__global__ void beam_acc_kernel(const double* __restrict__ sums, int B, int G, bool first, double* __restrict__ acc)
{
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        double s0 = 0.0, s1 = 0.0;
        for (int b = g; b < B; b += G) {
            s0 += sums[2 * b];
            s1 += sums[2 * b + 1];
        }
        acc[2 * g] = first ? s0 : acc[2 * g] + s0;
        acc[2 * g + 1] = first ? s1 : acc[2 * g + 1] + s1;
    }
}

// second-moment radius of the long-term spot, W_LT^2 = 2 sum r^2 I / sum I (S23 / S24 reading)
__global__ void w_lt_kernel(const double* __restrict__ acc, int G, double* __restrict__ w)
{
    for (int g = threadIdx.x; g < G; g += blockDim.x) w[g] = sqrt(2.0 * acc[2 * g + 1] / acc[2 * g]);
}

}  // namespace

cudaError_t launch_beam_acc(const double* beam_sums, int B, int G, bool first, double* acc, cudaStream_t st)
{
    beam_acc_kernel<<<1, 128, 0, st>>>(beam_sums, B, G, first, acc);
    return cudaGetLastError();
}

cudaError_t launch_w_lt(const double* acc, int G, double* w_lt, cudaStream_t st)
{
    w_lt_kernel<<<1, 128, 0, st>>>(acc, G, w_lt);
    return cudaGetLastError();
}

cudaError_t launch_moments(const Plan& p, const float* I, int B, int G, int64_t count, double* mean, double* m2,
                           cudaStream_t st)
{
    const size_t npix = (size_t)p.N * p.N;
    const double nc = (double)(B / G), na = (double)count, n = na + nc;
    dim3 grid((unsigned)((npix + 255) / 256), G);
    moments_kernel<<<grid, 256, 0, st>>>(I, B, G, npix, 1.0 / nc, nc / n, na * nc / n, count == 0, mean, m2);
    return cudaGetLastError();
}

cudaError_t launch_moments_finalize(const Plan& p, const double* mean, const double* m2, int G, int64_t count,
                                    double* si_map, double* si_mean, double* si_center, cudaStream_t st)
{
    const size_t npix = (size_t)p.N * p.N;
    const size_t center = (size_t)(p.N / 2) * p.N + p.N / 2;
    si_kernel<<<G, 256, 0, st>>>(mean, m2, npix, 1.0 / (double)count, si_map, si_mean, si_center, center);
    return cudaGetLastError();
}

}  // namespace ts
