// ts_noalloc.cu -- one phase screen for callers that cannot allocate device memory.
//
// ts_plan_create allocates a plan's tables and workspace with cudaMalloc.  Some callers cannot do
// that where they need a screen: code that runs inside another framework's allocator or stream
// discipline that forbids new device allocations, or a latency-critical loop in which the implicit
// device synchronisation of cudaMalloc / cudaFree would stall the pipeline.  ts_make_screen_noalloc
// serves them: it takes the medium, grid and one interval directly, and keeps its FFT twiddles, PSD
// shape table and column-transformed intermediate in one file-scope device array of fixed size,
// so it allocates nothing.  It launches the same screen-synthesis kernels as ts_make_screens.
//
// The array lives in this file's module: every GPU on which the library's module is loaded holds it
// (kNoAllocBytes, about 12 MiB) until the process exits.  With lazy module loading (the CUDA default)
// that is every GPU on which a kernel of the library has run; with CUDA_MODULE_LOADING=EAGER it is
// every GPU the process opens.  Host code cannot use the array's name as a device address, so every
// call looks the address up in the current context with cudaGetSymbolAddress (a host-side query: no
// allocation, no synchronisation), which stays correct after cudaDeviceReset or under a context the
// caller made current through the driver API.  The first call in a context also sets the synthesis
// kernels' shared-memory limits; contexts are told apart by their process-unique id.
#include <cuda.h>

#include <cmath>
#include <mutex>
#include <utility>
#include <string>

#include "ts_internal.h"

namespace ts {

namespace {

constexpr int kNoAllocMaxN = 1024;
constexpr size_t kAlign = 256;
constexpr size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kOffY = 0;                                                               // float2 [N][N]
constexpr size_t kOffG = kOffY + round_up(sizeof(float2) * kNoAllocMaxN * kNoAllocMaxN);  // float [N][N]
constexpr size_t kOffTw = kOffG + round_up(sizeof(float) * kNoAllocMaxN * kNoAllocMaxN);  // float2 [4N]
constexpr size_t kOffAmp = kOffTw + round_up(sizeof(float2) * 4 * kNoAllocMaxN);          // float [64]
constexpr size_t kNoAllocBytes = kOffAmp + round_up(sizeof(float) * kMaxScreens);

static __device__ __align__(256) unsigned char ts_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
constexpr int kMaxContexts = 64;
unsigned long long g_ready[kMaxContexts] = {};  // ids of the contexts whose kernel limits are set
int g_n_ready = 0;

__global__ void store_amplitude(float* amp, int s, float v) { amp[s] = v; }

// The process-unique id of the current context (cuCtxGetCurrent + cuCtxGetId, reached through the
// runtime's driver entry-point query), or 0 when it cannot be read.
unsigned long long current_context_id()
{
    using GetCurrentFn = CUresult (*)(CUcontext*);
    using GetIdFn = CUresult (*)(CUcontext, unsigned long long*);
    static const auto fns = []() {
        void* a = nullptr;
        void* b = nullptr;
        cudaDriverEntryPointQueryResult qa = cudaDriverEntryPointSymbolNotFound, qb = qa;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
            qa != cudaDriverEntryPointSuccess)
            a = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
            qb != cudaDriverEntryPointSuccess)
            b = nullptr;
        return std::make_pair(reinterpret_cast<GetCurrentFn>(a), reinterpret_cast<GetIdFn>(b));
    }();
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!fns.first || !fns.second || fns.first(&ctx) != CUDA_SUCCESS || !ctx || fns.second(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// The device address of the array in the current context, and (first call in a context) the
// shared-memory limits of the synthesis kernels.
ts_status scratch_for_current_context(unsigned char** out)
{
    void* ptr = nullptr;  // also brings up the current device's primary context if none is current
    ts_status st =
        cuda_check(cudaGetSymbolAddress(&ptr, ts_noalloc_scratch), "ts_make_screen_noalloc: cudaGetSymbolAddress");
    if (st != TS_OK) return st;
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lock(g_mu);
    bool ready = false;
    for (int i = 0; i < g_n_ready && id != 0; ++i) ready = ready || g_ready[i] == id;
    if (!ready) {
        for (int n = 128; n <= kNoAllocMaxN; n *= 2) {
            st = cuda_check(prepare_screen_kernels(n), "ts_make_screen_noalloc: kernel attributes");
            if (st != TS_OK) return st;
        }
        if (id != 0 && g_n_ready < kMaxContexts) g_ready[g_n_ready++] = id;
    }
    *out = static_cast<unsigned char*>(ptr);
    return TS_OK;
}

}  // namespace
}  // namespace ts

using namespace ts;

extern "C" ts_status ts_make_screen_noalloc(const ts_medium* medium, const ts_grid* grid, double dz, double cn2,
                                            uint64_t seed, uint32_t screen, uint32_t real, float* phi, void* stream)
{
    if (!medium || !grid || !phi) {
        set_error("ts_make_screen_noalloc: null pointer argument");
        return TS_ERR_INVALID_ARG;
    }
    const int N = grid->N;
    if (N != 128 && N != 256 && N != 512 && N != 1024 && N != 2048) {
        set_error("ts_make_screen_noalloc: N must be one of 128, 256, 512, 1024, 2048");
        return TS_ERR_INVALID_ARG;
    }
    if (N > kNoAllocMaxN) {
        set_error("ts_make_screen_noalloc: N = " + std::to_string(N) + " exceeds the static scratch (N <= 1024)");
        return TS_ERR_WORKSPACE;
    }
    if (!(grid->dx > 0.0) || !(medium->lambda > 0.0) || !(medium->n0 > 0.0) || !(dz > 0.0) || !(cn2 >= 0.0) ||
        !std::isfinite(dz) || !std::isfinite(cn2)) {
        set_error("ts_make_screen_noalloc: dx, lambda, n0, dz must be > 0 and cn2 >= 0");
        return TS_ERR_INVALID_ARG;
    }
    if (screen >= (uint32_t)kMaxScreens) {
        set_error("ts_make_screen_noalloc: screen index must be below 64");
        return TS_ERR_INVALID_ARG;
    }
    unsigned char* base = nullptr;
    ts_status st = scratch_for_current_context(&base);
    if (st != TS_OK) return st;
    float2* y = reinterpret_cast<float2*>(base + kOffY);
    float* g = reinterpret_cast<float*>(base + kOffG);
    float2* tw = reinterpret_cast<float2*>(base + kOffTw);
    float* amp = reinterpret_cast<float*>(base + kOffAmp);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const double k = 2.0 * M_PI * medium->n0 / medium->lambda;
    const double dk = 2.0 * M_PI / (N * grid->dx);
    // s(kappa) = amp g(kappa), amp = sqrt(2 pi k^2 dz 0.033 Cn^2) dkappa   (S14, S16, S17)
    const float a = (float)(std::sqrt(2.0 * M_PI * k * k * dz * 0.033 * cn2) * dk);
    // every region the kernels read is rewritten first in stream order, so nothing needs zeroing
    cudaError_t e = launch_twiddles(N, tw, s);
    if (e == cudaSuccess) e = launch_psd_shape(N, g, dk, medium->L0, medium->l0, s);
    if (e == cudaSuccess) {
        store_amplitude<<<1, 1, 0, s>>>(amp, (int)screen, a);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_screen_raw(N, tw, g, amp, y, seed, (int)screen, real, phi, s);
    return cuda_check(e, "ts_make_screen_noalloc");
}
