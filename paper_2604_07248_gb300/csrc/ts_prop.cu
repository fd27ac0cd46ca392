// ts_prop.cu -- entry points of the propagation passes: argument packing and N dispatch.
#include "ts_prop_decl.h"

namespace ts {

namespace {
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
}  // namespace

cudaError_t launch_row_pass(const Plan& p, int flags, const RowArgs& a, cudaStream_t st)
{
    RowParams rp{};
    rp.field = a.field;
    rp.phi = a.phi;
    rp.phasor = a.phasor;
    rp.phi_set_stride = a.phi_set_stride;
    rp.phi_group = a.phi_group > 0 ? a.phi_group : 1;
    rp.phi_off = a.b0 % rp.phi_group;
    rp.src_off = a.b0;
    rp.phase_sign = a.phase_sign;
    rp.intensity = a.intensity;
    rp.rows = a.rows;
    rp.tw = p.tw;
    rp.n_src = p.n_src > 0 ? p.n_src : 1;
    for (int i = 0; i < kMaxSources; ++i) rp.src_coef[i] = i < p.n_src ? p.src_coef[i] : -1.0f;
    rp.tw = p.fft_e == 16 ? p.tw16 : p.tw;
    rp.err = p.d_err;
    rp.budget = p.tc_budget;
    rp.stall = p.test_stall ? 1 : 0;
    if (p.split_bf16) return tc_row_pass(flags, rp, a.B, p.tc_budget, p.d_err, st);
    switch (p.N) {
    case 128: return row_pass_n<128>(p.fft_e, p.row_variant, flags, rp, a.B, st);
    case 256: return row_pass_n<256>(p.fft_e, p.row_variant, flags, rp, a.B, st);
    case 512: return row_pass_n<512>(p.fft_e, p.row_variant, flags, rp, a.B, st);
    case 1024: return row_pass_n<1024>(p.fft_e, p.row_variant, flags, rp, a.B, st);
    case 2048: return row_pass_n<2048>(p.fft_e, p.row_variant, flags, rp, a.B, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_col_pass(const Plan& p, int step, bool conj, float2* field, int B, cudaStream_t st, bool source,
                            int src_off)
{
    ColParams cp{};
    cp.field = field;
    cp.tw = p.tw;
    cp.P = p.P + (size_t)step * p.N;
    cp.dcoef = (float)(p.dz[step] / (2.0 * p.k * p.k * p.k));
    cp.ccross = (float)(p.dz[step] / (4.0 * p.k * p.k * p.k));
    cp.inv_k2 = (float)(1.0 / (p.k * p.k));
    cp.dk = (float)p.dk;
    cp.tw = p.fft_e == 16 ? p.tw16 : p.tw;
    cp.err = p.d_err;
    cp.budget = p.tc_budget;
    cp.tiny_cross = p.tiny_cross;
    cp.first_order_cross = p.first_order_cross;
    cp.stall = p.test_stall ? 1 : 0;
    cp.src_fx = p.src_fx;
    cp.src_gy = p.src_gy;
    cp.n_src = p.n_src;
    cp.src_off = src_off;
    if (source && (p.split_bf16 || p.src_fx == nullptr || p.n_src < 1)) return cudaErrorNotSupported;
    if (p.split_bf16) return tc_col_pass(p.tc_col_groups, conj, p.sep_transfer, cp, B, p.tc_budget, p.d_err, st);
    switch (p.N) {
    case 128: return col_pass_n<128>(p.fft_e, p.col_variant, conj, p.sep_transfer, cp, B, st, source);
    case 256: return col_pass_n<256>(p.fft_e, p.col_variant, conj, p.sep_transfer, cp, B, st, source);
    case 512: return col_pass_n<512>(p.fft_e, p.col_variant, conj, p.sep_transfer, cp, B, st, source);
    case 1024: return col_pass_n<1024>(p.fft_e, p.col_variant, conj, p.sep_transfer, cp, B, st, source);
    case 2048: return col_pass_n<2048>(p.fft_e, p.col_variant, conj, p.sep_transfer, cp, B, st, source);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t prepare_prop_kernels(int N)
{
    if (N == 512 || N == 1024) {
        cudaError_t e = prepare_prop_tma(N);
        if (e == cudaSuccess && N == 1024) e = prepare_prop_fused_1024();
        if (e != cudaSuccess) return e;
    }
    switch (N) {
    case 128: return prepare_prop_n<128>();
    case 256: return prepare_prop_n<256>();
    case 512: return prepare_prop_n<512>();
    case 1024: return prepare_prop_n<1024>();
    case 2048: return prepare_prop_n<2048>();
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_row_sums(const Plan& p, const double* rows, int B, double* out, cudaStream_t st)
{
    const int T = p.N / (p.N <= 256 ? 16 : p.fft_e);
    const int wpl = T > 32 ? T / 32 : 1;
    row_sums_kernel<<<B, 256, 0, st>>>(rows, B, p.N, wpl, p.dx * p.dx, out);
    return cudaGetLastError();
}

}  // namespace ts
