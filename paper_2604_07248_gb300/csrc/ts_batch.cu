// ts_batch.cu -- uneven batches: many independent split-step instances of different N and screen
// counts propagated by ONE persistent kernel launch (captured, with the screen synthesis, in a CUDA
// graph).
//
// Work items are (instance, phase, tile) with phase 0 = first row pass, 2s+1 = column pass of step s,
// 2s+2 = row pass of step s.  The host lists them by increasing phase (instances and tiles
// interleaved), CTAs take them from a global counter, and an item of phase k waits until every tile
// of phase k-1 of its own instance is done (per-instance completion counters, release/acquire at GPU
// scope).  Because items are handed out in that order, every item a CTA waits on was taken earlier
// by a running CTA, so the schedule cannot deadlock whatever the grid size.  All waits are bounded by
// a clock64 budget: a CTA that gives up sets the error word, every CTA then stops taking work, and the
// host reads the status with ts_batch_status.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "ts_prop_impl.cuh"

namespace ts {

namespace {

constexpr int kBatchThreads = 256;

struct BInst {
    int N, S, src;
    int tiles_row, tiles_col;
    int ctr_base;
    int extra_need;  // test hook: added to the phase-1 dependency of this instance (never satisfied)
    float src_coef;
    float dk;
    float2* field;
    const float2* phasor;  // [S][N][N]
    const float2* tw;      // twiddles for the default points-per-thread of N
    const float2* P;       // [S][N] separable per-axis transfer factors
    const float* ccross;   // [S] dz / (4 k^3)
};

struct BatchParams {
    const BInst* inst;
    const int4* items;  // (instance, phase, tile, unused)
    int n_items;
    int* head;
    int* done;
    int* err;
    long long budget;  // clock64 cycles per wait
};

__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int N>
__device__ __noinline__ void batch_row(const BInst& I, int phase, int tile, float2* smem, bool stage)
{
    RowParams a{};
    a.field = I.field;
    a.phi_group = 1;
    a.phase_sign = 1.0f;
    a.tw = I.tw;
    a.n_src = 1;
    a.src_coef[0] = I.src_coef;
    if (phase == 0) {
        if (I.src) row_tile<N, 0, RP_IN_SOURCE | RP_OUT_FREQ | RP_STORE>(a, tile, 0, smem, stage);
        else row_tile<N, 0, RP_OUT_FREQ | RP_STORE>(a, tile, 0, smem, stage);
        return;
    }
    const int s = phase / 2 - 1;
    a.phasor = I.phasor + (size_t)s * N * N;
    if (s < I.S - 1) row_tile<N, 0, RP_IN_FREQ | RP_PHASOR | RP_OUT_FREQ | RP_STORE>(a, tile, 0, smem, stage);
    else row_tile<N, 0, RP_IN_FREQ | RP_PHASOR | RP_STORE>(a, tile, 0, smem, stage);
}

template <int N>
__device__ __noinline__ void batch_col(const BInst& I, int phase, int tile, float2* smem, bool stage)
{
    const int s = (phase - 1) / 2;
    ColParams c{};
    c.field = I.field;
    c.tw = I.tw;
    c.P = I.P + (size_t)s * N;
    c.ccross = I.ccross[s];
    c.dk = I.dk;
    col_tile<N, 0, false, true>(c, tile, 0, smem, stage);
}

__global__ void __launch_bounds__(kBatchThreads, 2) batch_kernel(const BatchParams bp)
{
    extern __shared__ float2 smem[];
    __shared__ int s_item;
    int lastN = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            int it = atomicAdd(bp.head, 1);
            bool stop = it >= bp.n_items || ld_relaxed(bp.err) != 0;
            if (!stop) {
                const int4 w = bp.items[it];
                if (w.y > 0) {
                    const BInst& I = bp.inst[w.x];
                    const int prev = w.y - 1;
                    const int need = ((prev & 1) ? I.tiles_col : I.tiles_row) + (w.y == 1 ? I.extra_need : 0);
                    const int* ctr = bp.done + I.ctr_base + prev;
                    const long long t0 = clock64();
                    while (ld_acquire(ctr) < need) {
                        if (ld_relaxed(bp.err) != 0) {
                            stop = true;
                            break;
                        }
                        if (clock64() - t0 > bp.budget) {
                            atomicExch(bp.err, 2);  // this CTA's wait ran out
                            stop = true;
                            break;
                        }
                        __nanosleep(128);
                    }
                }
            }
            s_item = stop ? -1 : it;
        }
        __syncthreads();
        const int it = s_item;
        if (it < 0) break;
        const int4 w = bp.items[it];
        const BInst& I = bp.inst[w.x];
        const bool stage = I.N != lastN;  // twiddles depend only on N (same points per thread)
        lastN = I.N;
        const bool colpass = (w.y & 1) != 0;
        switch (I.N) {
        case 128: colpass ? batch_col<128>(I, w.y, w.z, smem, stage) : batch_row<128>(I, w.y, w.z, smem, stage); break;
        case 256: colpass ? batch_col<256>(I, w.y, w.z, smem, stage) : batch_row<256>(I, w.y, w.z, smem, stage); break;
        case 512: colpass ? batch_col<512>(I, w.y, w.z, smem, stage) : batch_row<512>(I, w.y, w.z, smem, stage); break;
        case 1024: colpass ? batch_col<1024>(I, w.y, w.z, smem, stage) : batch_row<1024>(I, w.y, w.z, smem, stage); break;
        default: colpass ? batch_col<2048>(I, w.y, w.z, smem, stage) : batch_row<2048>(I, w.y, w.z, smem, stage); break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(bp.done + I.ctr_base + w.y, 1);
        }
    }
}

template <int N>
constexpr size_t batch_smem_n()
{
    return RowCfg<N, 0>::smem > ColCfg<N, 0>::smem ? RowCfg<N, 0>::smem : ColCfg<N, 0>::smem;
}

}  // namespace

struct Batch {
    int device = 0;
    int n = 0;
    int n_items = 0;
    int grid = 0;
    size_t smem = 0;
    std::vector<Plan*> plans;
    std::vector<BInst> host_inst;
    BInst* inst = nullptr;
    int4* items = nullptr;
    int* counters = nullptr;  // [head][err][done...]
    int n_counters = 0;
    float* ccross = nullptr;
    float2* screens = nullptr;  // generated screens (phasors) of instances without their own
    std::vector<size_t> screen_off;
    std::vector<int> gen;        // instance needs generated screens
    std::vector<uint64_t> seed;
    std::vector<uint32_t> real;
    long long budget = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    size_t bytes = 0;
};

}  // namespace ts

using namespace ts;

namespace {

ts_status bfail(ts_status s, const std::string& m)
{
    set_error(m);
    return s;
}

void free_batch(Batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    void* ptrs[] = {b->inst, b->items, b->counters, b->ccross, b->screens};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete b;
}

// the launch sequence captured into the batch's graph: screen synthesis, counter reset, one launch
cudaError_t record_batch(Batch& b, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < b.n && e == cudaSuccess; ++i) {
        if (!b.gen[i]) continue;
        Plan& p = *b.plans[i];
        ScreenArgs a{};
        a.seed = b.seed[i];
        a.s_begin = 0;
        a.s_count = p.S;
        a.r_begin = b.real[i];
        a.items = p.S;
        a.phasor = b.screens + b.screen_off[i];
        e = launch_screens(p, SC_INDEP, a, st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(b.counters, 0, sizeof(int) * b.n_counters, st);
    if (e == cudaSuccess) {
        BatchParams bp;
        bp.inst = b.inst;
        bp.items = b.items;
        bp.n_items = b.n_items;
        bp.head = b.counters;
        bp.err = b.counters + 1;
        bp.done = b.counters + 2;
        bp.budget = b.budget;
        batch_kernel<<<b.grid, kBatchThreads, b.smem, st>>>(bp);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace

extern "C" {

ts_status ts_batch_create(ts_batch* out, const ts_batch_instance* inst, int n, double timeout_s, int flags)
{
    if (!out || !inst || n < 1) return bfail(TS_ERR_INVALID_ARG, "ts_batch_create: need instances");
    *out = nullptr;
    if (!(timeout_s > 0.0)) return bfail(TS_ERR_INVALID_ARG, "ts_batch_create: timeout must be positive");
    Batch* b = new Batch();
    b->n = n;
    cudaError_t e = cudaGetDevice(&b->device);
    size_t screen_elems = 0;
    int ctr = 0;
    std::vector<int4> items;
    int max_phase = 0;
    std::vector<float> ccross;
    std::vector<size_t> cc_off;
    for (int i = 0; i < n; ++i) {
        Plan* p = reinterpret_cast<Plan*>(inst[i].plan);
        if (!p || !inst[i].field) {
            free_batch(b);
            return bfail(TS_ERR_INVALID_ARG, "ts_batch_create: instance " + std::to_string(i) + " needs plan and field");
        }
        if (p->device != b->device) {
            free_batch(b);
            return bfail(TS_ERR_INVALID_ARG, "ts_batch_create: all plans must live on the current device");
        }
        if (p->split_bf16) {
            free_batch(b);
            return bfail(TS_ERR_UNSUPPORTED, "ts_batch_create: instance " + std::to_string(i) +
                                                 " uses the split-BF16 passes (the persistent batch kernel is FP32)");
        }
        if (!p->sep_transfer) {
            free_batch(b);
            return bfail(TS_ERR_UNSUPPORTED, "ts_batch_create: instance " + std::to_string(i) +
                                                 " needs the exact (non-separable) transfer function");
        }
        if (inst[i].source && p->n_src < 1) {
            free_batch(b);
            return bfail(TS_ERR_INVALID_ARG, "ts_batch_create: instance " + std::to_string(i) + " has no source set");
        }
        b->plans.push_back(p);
        const int N = p->N;
        BInst bi{};
        bi.N = N;
        bi.S = p->S;
        bi.src = inst[i].source ? 1 : 0;
        const int T = N / (N <= 256 ? 16 : 32);
        bi.tiles_row = N / (kBatchThreads / T);
        bi.tiles_col = N / (kBatchThreads / T);
        bi.ctr_base = ctr;
        ctr += 2 * p->S + 1;
        bi.extra_need = ((flags & TS_BATCH_TEST_STALL) && i == 0) ? 1 : 0;
        bi.src_coef = p->src_coef[0];
        bi.dk = (float)p->dk;
        bi.field = reinterpret_cast<float2*>(inst[i].field);
        bi.tw = p->tw;
        bi.P = p->P;
        bi.phasor = reinterpret_cast<const float2*>(inst[i].phasor);
        b->gen.push_back(inst[i].phasor ? 0 : 1);
        b->seed.push_back(inst[i].seed);
        b->real.push_back(inst[i].real);
        b->screen_off.push_back(screen_elems);
        if (!inst[i].phasor) screen_elems += (size_t)p->S * N * N;
        cc_off.push_back(ccross.size());
        for (int s = 0; s < p->S; ++s) ccross.push_back((float)(p->dz[s] / (4.0 * p->k * p->k * p->k)));
        b->host_inst.push_back(bi);
        max_phase = std::max(max_phase, 2 * p->S);
    }
    // Items by increasing phase, instances and tiles interleaved within a phase (a topological order,
    // so the schedule cannot deadlock).  Staggering instances by a few phases was measured slower.
    for (int k = 0; k <= max_phase; ++k)
        for (int i = 0; i < n; ++i) {
            const BInst& bi = b->host_inst[i];
            if (k > 2 * bi.S) continue;
            const int tiles = (k & 1) ? bi.tiles_col : bi.tiles_row;
            for (int t = 0; t < tiles; ++t) items.push_back(make_int4(i, k, t, 0));
        }
    b->n_items = (int)items.size();
    b->n_counters = 2 + ctr;
    // shared memory: the largest tile of any instance
    size_t smem = 0;
    for (int i = 0; i < n; ++i) {
        switch (b->host_inst[i].N) {
        case 128: smem = std::max(smem, batch_smem_n<128>()); break;
        case 256: smem = std::max(smem, batch_smem_n<256>()); break;
        case 512: smem = std::max(smem, batch_smem_n<512>()); break;
        case 1024: smem = std::max(smem, batch_smem_n<1024>()); break;
        default: smem = std::max(smem, batch_smem_n<2048>()); break;
        }
    }
    b->smem = smem;
    auto ok = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    ok(cudaMalloc(&b->inst, sizeof(BInst) * n));
    ok(cudaMalloc(&b->items, sizeof(int4) * items.size()));
    ok(cudaMalloc(&b->counters, sizeof(int) * b->n_counters));
    ok(cudaMalloc(&b->ccross, sizeof(float) * std::max<size_t>(1, ccross.size())));
    if (screen_elems) ok(cudaMalloc(&b->screens, sizeof(float2) * screen_elems));
    if (e == cudaSuccess) {
        for (int i = 0; i < n; ++i) {
            BInst& bi = b->host_inst[i];
            bi.ccross = b->ccross + cc_off[i];
            if (!bi.phasor) bi.phasor = b->screens + b->screen_off[i];
        }
        ok(cudaMemcpy(b->inst, b->host_inst.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice));
        ok(cudaMemcpy(b->items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
        ok(cudaMemcpy(b->ccross, ccross.data(), sizeof(float) * ccross.size(), cudaMemcpyHostToDevice));
        ok(cudaMemset(b->counters, 0, sizeof(int) * b->n_counters));
    }
    b->bytes = sizeof(BInst) * n + sizeof(int4) * items.size() + sizeof(int) * b->n_counters +
               sizeof(float) * ccross.size() + sizeof(float2) * screen_elems;
    // grid: as many CTAs as fit at once (one per SM at this shared-memory size and up to the limit)
    int sms = 0, per_sm = 0, clock_khz = 0;
    ok(cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    ok(cudaFuncSetAttribute(batch_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    ok(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
    ok(cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, b->device));
    ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, kBatchThreads, b->smem));
    b->grid = std::max(1, sms * std::max(1, per_sm));
    b->budget = (long long)(timeout_s * (double)std::max(clock_khz, 1000000) * 1e3);
    // capture the whole run as one graph on a private stream
    ok(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    if (e == cudaSuccess) {
        e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t er = record_batch(*b, b->cap);
            e = cudaStreamEndCapture(b->cap, &b->graph);
            if (e == cudaSuccess) e = er;
        }
    }
    ok(b->graph ? cudaGraphInstantiate(&b->exec, b->graph, 0) : cudaErrorInvalidValue);
    if (e != cudaSuccess) {
        ts_status st = cuda_check(e, "ts_batch_create");
        free_batch(b);
        return st;
    }
    *out = reinterpret_cast<ts_batch>(b);
    return TS_OK;
}

ts_status ts_batch_run(ts_batch batch, void* stream)
{
    if (!batch) return bfail(TS_ERR_INVALID_ARG, "ts_batch_run: null batch");
    Batch* b = reinterpret_cast<Batch*>(batch);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device)
        return bfail(TS_ERR_INVALID_ARG, "ts_batch_run: the batch lives on device " + std::to_string(b->device) +
                                             ", which must be current");
    return cuda_check(cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream)), "ts_batch_run");
}

ts_status ts_batch_status(ts_batch batch, void* stream)
{
    if (!batch) return bfail(TS_ERR_INVALID_ARG, "ts_batch_status: null batch");
    Batch* b = reinterpret_cast<Batch*>(batch);
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, b->counters + 1, sizeof(int), cudaMemcpyDeviceToHost,
                                    reinterpret_cast<cudaStream_t>(stream));
    if (e == cudaSuccess) e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_check(e, "ts_batch_status");
    if (err != 0) return bfail(TS_ERR_DEVICE_TIMEOUT, "ts_batch_status: a dependency wait ran out of its budget");
    return TS_OK;
}

ts_status ts_batch_info(ts_batch batch, int* n_items, int* grid, size_t* device_bytes)
{
    if (!batch) return bfail(TS_ERR_INVALID_ARG, "ts_batch_info: null batch");
    Batch* b = reinterpret_cast<Batch*>(batch);
    if (n_items) *n_items = b->n_items;
    if (grid) *grid = b->grid;
    if (device_bytes) *device_bytes = b->bytes;
    return TS_OK;
}

ts_status ts_batch_destroy(ts_batch batch)
{
    if (!batch) return TS_OK;
    Batch* b = reinterpret_cast<Batch*>(batch);
    cudaError_t e = cudaDeviceSynchronize();
    free_batch(b);
    return cuda_check(e, "ts_batch_destroy");
}

}  // extern "C"
