// ts_train.cu -- the optimiser step of the D2NN training loop (Sec. 2.5): Adam on the phase masks.
//
// Adam (Kingma & Ba, 2015) for step t >= 1 with gradient g:
//   m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
//   p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
// The bias corrections are computed on the host in FP64 and passed as scalars.
#include <cmath>

#include "ts_internal.h"

namespace ts {

namespace {

// omb1 = 1 - b1 and omb2 = 1 - b2 come from the host in FP64 (1 - 0.999f in FP32 is off by 1e-5)
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float omb1, float omb2,
                            float eps, float c1, float c2)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], omb1 * gi);
        const float vi = fmaf(b2, v[i], omb2 * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

}  // namespace

}  // namespace ts

extern "C" ts_status ts_adam_step(float* param, const float* grad, float* m, float* v, long long n, double lr,
                                  double beta1, double beta2, double eps, int t, void* stream)
{
    if (!param || !grad || !m || !v || n < 1 || t < 1 || !(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) ||
        !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0)) {
        ts::set_error("ts_adam_step: need param, grad, m, v, n >= 1, t >= 1, lr >= 0, 0 <= beta < 1, eps > 0");
        return TS_ERR_INVALID_ARG;
    }
    const double c1 = 1.0 / (1.0 - std::pow(beta1, (double)t));
    const double c2 = 1.0 / (1.0 - std::pow(beta2, (double)t));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (n + 255) / 256;
    const int blocks = (int)std::min<long long>(want, (long long)(sms > 0 ? sms : 1) * 8);
    ts::adam_kernel<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        param, grad, m, v, n, (float)lr, (float)beta1, (float)beta2, (float)(1.0 - beta1), (float)(1.0 - beta2),
        (float)eps, (float)c1, (float)c2);
    return ts::cuda_check(cudaGetLastError(), "ts_adam_step");
}
