// Instantiation and cooperative launch of the rounding, lower-bound and validation kernels.
#include <algorithm>

#include "launch.h"
#include "round_kernels.cuh"

namespace mdot {

cudaError_t configure_stage_kernels(int max_n, int G, int* min_blocks);

size_t round_smem_bytes(int n, int G) { return round_smem(n, G, kThreads).bytes; }
size_t lb_smem_bytes(int n, int G) { return (size_t)((n + G - 1) / G + 1) * sizeof(double); }

static cudaError_t coop(const void* kernel, int G, size_t smem, cudaStream_t s, void** args)
{
    return cudaLaunchCooperativeKernel(kernel, dim3(G), dim3(kThreads), args, smem, s);
}

static const void* round_fn(int kind)
{
    return kind == COST_SQEUCLID ? (const void*)round_kernel<COST_SQEUCLID>
         : kind == COST_L1       ? (const void*)round_kernel<COST_L1>
                                 : (const void*)round_kernel<COST_DENSE>;
}

static const void* lb_fn(int kind)
{
    return kind == COST_SQEUCLID ? (const void*)lower_bound_kernel<COST_SQEUCLID>
         : kind == COST_L1       ? (const void*)lower_bound_kernel<COST_L1>
                                 : (const void*)lower_bound_kernel<COST_DENSE>;
}

cudaError_t launch_round(const WS& ws, const RoundArgs& a, cudaStream_t s)
{
    WS w = ws;
    RoundArgs aa = a;
    void* args[] = {(void*)&w, (void*)&aa};
    return coop(round_fn(ws.ckind), ws.G, round_smem_bytes(ws.n, ws.G), s, args);
}

cudaError_t launch_lower_bound(const WS& ws, const LbArgs& a, cudaStream_t s)
{
    WS w = ws;
    LbArgs aa = a;
    void* args[] = {(void*)&w, (void*)&aa};
    return coop(lb_fn(ws.ckind), ws.G, lb_smem_bytes(ws.n, ws.G), s, args);
}

cudaError_t launch_validate(const WS& ws, double* out, cudaStream_t s)
{
    WS w = ws;
    double* o = out;
    void* args[] = {(void*)&w, (void*)&o};
    return coop((const void*)validate_kernel, ws.G, 0, s, args);
}

cudaError_t configure_kernels(int max_n, int G, int* min_blocks_per_sm)
{
    int mb = 1 << 30;
    cudaError_t e = configure_stage_kernels(max_n, G, &mb);
    if (e != cudaSuccess) return e;
    struct K { const void* f; size_t smem; } ks[] = {
        {round_fn(COST_DENSE), round_smem_bytes(max_n, G)},
        {round_fn(COST_SQEUCLID), round_smem_bytes(max_n, G)},
        {round_fn(COST_L1), round_smem_bytes(max_n, G)},
        {lb_fn(COST_DENSE), lb_smem_bytes(max_n, G)},
        {lb_fn(COST_SQEUCLID), lb_smem_bytes(max_n, G)},
        {lb_fn(COST_L1), lb_smem_bytes(max_n, G)},
        {(const void*)validate_kernel, 0}};
    for (auto& k : ks) {
        e = raise_smem_limit(k.f, k.smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k.f, kThreads, k.smem);
        if (e != cudaSuccess) return e;
        mb = std::min(mb, nb);
    }
    *min_blocks_per_sm = mb;
    return cudaSuccess;
}

}  // namespace mdot
