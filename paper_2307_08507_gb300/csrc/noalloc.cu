// mdot_dual_eval_noalloc: the fp32-entry dual evaluation for callers that cannot allocate device
// memory.  Its scratch lives in one static __device__ array compiled into the library; the host
// side only ever holds that array's device address (looked up once per device).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "mdot.h"
#include "launch.h"
#include "solver_kernels.cuh"

namespace {

using namespace mdot;

constexpr int kMaxN = MDOT_NOALLOC_MAX_N;
constexpr int kMaxG = 160;                                  // CTAs (one per SM), capped
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch layout (byte offsets): barrier/state, column partials, per-column and per-row
// constants, column scales, per-CTA reductions.
constexpr size_t kOffState = 0;
constexpr size_t kOffColpart = align256(kOffState + sizeof(State));
constexpr size_t kOffHh = align256(kOffColpart + (size_t)kMaxG * kMaxN * sizeof(float));
constexpr size_t kOffWc = align256(kOffHh + (size_t)kMaxN * sizeof(float));
constexpr size_t kOffFh = align256(kOffWc + (size_t)kMaxN * sizeof(float));
constexpr size_t kOffWr = align256(kOffFh + (size_t)kMaxN * sizeof(float));
constexpr size_t kOffA = align256(kOffWr + (size_t)kMaxN * sizeof(float));
constexpr size_t kOffScratch = align256(kOffA + (size_t)kMaxN * sizeof(int));
constexpr size_t kOffBlockred = align256(kOffScratch + (size_t)kMaxG * 8 * sizeof(double));
constexpr size_t kBytes = align256(kOffBlockred + (size_t)kMaxG * kNRed * sizeof(double));

// About 2.6 MiB; every device that loads the library holds it for the life of the process.
__device__ __align__(256) unsigned char g_noalloc_scratch[kBytes];

struct DeviceSetup {
    bool done = false;
    unsigned char* base = nullptr;    // device address of g_noalloc_scratch on this device
    int G = 0;
};

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

// The message mdot_last_error() returns (the library's per-thread error text).
mdot_status fail(mdot_status st, const char* what, cudaError_t e = cudaSuccess)
{
    char msg[256];
    if (e != cudaSuccess)
        snprintf(msg, sizeof msg, "mdot_dual_eval_noalloc: %s: %s", what, cudaGetErrorString(e));
    else
        snprintf(msg, sizeof msg, "mdot_dual_eval_noalloc: %s", what);
    set_last_error(msg);
    return st;
}

// Once per device, with that device current: the scratch's device address and the grid size.
cudaError_t setup_device(int dev, DeviceSetup** out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& s = g_setup[dev];
    if (!s.done) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        const int G = std::min(sms, kMaxG);
        const size_t smem = kSmemLimit;        // the largest layout any n up to kMaxN takes
        e = raise_smem_limit((const void*)dual_eval_kernel<TIER_F32, COST_DENSE>, smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)dual_eval_kernel<TIER_F32, COST_DENSE>,
                                                          kStageThreads, smem);
        if (e != cudaSuccess) return e;
        if (nb < 1) return cudaErrorCooperativeLaunchTooLarge;
        s.base = static_cast<unsigned char*>(ptr);
        s.G = G;
        s.done = true;
    }
    *out = &s;
    return cudaSuccess;
}

}  // namespace

extern "C" mdot_status mdot_dual_eval_noalloc(const double* u, const double* v, double gamma,
                                              const float* C, int64_t n, const double* ref_log_rP,
                                              double* log_rP, double* log_cP, void* stream)
{
    if (!u || !v || !C || !log_rP || !log_cP || n < 1 || !(gamma > 0.0) || !std::isfinite(gamma))
        return fail(MDOT_ERR_INVALID_ARG, "null pointer, n < 1 or gamma not positive and finite");
    if (n > kMaxN) {
        char what[128];
        snprintf(what, sizeof what, "n = %lld exceeds MDOT_NOALLOC_MAX_N = %d", (long long)n, kMaxN);
        return fail(MDOT_ERR_INVALID_ARG, what);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(MDOT_ERR_CUDA, "cudaGetDevice", e);
    if (dev < 0 || dev >= kMaxDevices) return fail(MDOT_ERR_CUDA, "device index beyond the set-up table");
    DeviceSetup* s = nullptr;
    e = setup_device(dev, &s);
    if (e != cudaSuccess) return fail(MDOT_ERR_CUDA, "set-up (scratch address, kernel attributes)", e);
    cudaStream_t st = (cudaStream_t)stream;

    WS ws{};
    ws.n = (int)n;
    ws.G = s->G;
    ws.C = C;
    ws.st = reinterpret_cast<State*>(s->base + kOffState);
    ws.colpart = reinterpret_cast<float*>(s->base + kOffColpart);
    ws.Hh = reinterpret_cast<float*>(s->base + kOffHh);
    ws.Wc = reinterpret_cast<float*>(s->base + kOffWc);
    ws.Fh = reinterpret_cast<float*>(s->base + kOffFh);
    ws.Wr = reinterpret_cast<float*>(s->base + kOffWr);
    ws.A = reinterpret_cast<int*>(s->base + kOffA);
    ws.scratch = reinterpret_cast<double*>(s->base + kOffScratch);
    ws.blockred = reinterpret_cast<double*>(s->base + kOffBlockred);
    ws.lrtr = log_rP;          // results go straight to the caller's buffers
    ws.lcout = log_cP;

    EvalArgs a{};
    a.gamma = gamma;
    a.G64 = gamma * kLog2e;
    a.u = u;
    a.v = v;
    a.ref = ref_log_rP;

    // the barrier and status must start at zero; everything else is overwritten by the call
    e = cudaMemsetAsync(ws.st, 0, sizeof(State), st);
    if (e != cudaSuccess) return fail(MDOT_ERR_CUDA, "clearing the scratch state", e);
    WS wk = ws;
    EvalArgs ak = a;
    void* args[] = {(void*)&wk, (void*)&ak};
    const size_t smem = smem_layout((int)n, s->G, TIER_F32, kStageThreads, true).bytes;
    e = cudaLaunchCooperativeKernel((const void*)dual_eval_kernel<TIER_F32, COST_DENSE>, dim3(s->G), dim3(kStageThreads),
                                    args, smem, st);
    if (e != cudaSuccess) return fail(MDOT_ERR_CUDA, "kernel launch", e);
    int status = 0;
    e = cudaMemcpyAsync(&status, &ws.st->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(MDOT_ERR_CUDA, "reading the status", e);
    const mdot_status out = status_of(status);       // the device status, one to one
    if (out != MDOT_OK) return fail(out, "the evaluation kernel reported a failure");
    return MDOT_OK;
}
