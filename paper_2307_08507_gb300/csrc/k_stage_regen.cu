// Instantiation and cooperative launch of the stage and dual-evaluation kernels with the cost
// regenerated from coordinates (squared Euclidean and L1).
#include <algorithm>

#include "launch.h"
#include "solver_kernels.cuh"

namespace mdot {

template <int COST>
static cudaError_t launch_stage_kind(int tier, const WS& ws, const StageArgs& a, cudaStream_t s)
{
    WS w = ws;
    StageArgs aa = a;
    void* args[] = {(void*)&w, (void*)&aa};
    const size_t smem = stage_smem_bytes(ws.n, ws.G, tier);
    const void* f = tier == TIER_F64 ? (const void*)stage_kernel<TIER_F64, COST>
                  : tier == TIER_F32A ? (const void*)stage_kernel_flag<TIER_F32A, COST>
                                      : (const void*)stage_kernel_flag<TIER_F32, COST>;
    return cudaLaunchCooperativeKernel(f, dim3(ws.G), dim3(kStageThreads), args, smem, s);
}

template <int COST>
static cudaError_t launch_eval_kind(int tier, const WS& ws, const EvalArgs& a, cudaStream_t s)
{
    WS w = ws;
    EvalArgs aa = a;
    void* args[] = {(void*)&w, (void*)&aa};
    const size_t smem = eval_smem_bytes(ws.n, ws.G, tier);
    const void* f = tier == TIER_F64 ? (const void*)dual_eval_kernel<TIER_F64, COST>
                  : tier == TIER_F32A ? (const void*)dual_eval_kernel<TIER_F32A, COST>
                                      : (const void*)dual_eval_kernel<TIER_F32, COST>;
    return cudaLaunchCooperativeKernel(f, dim3(ws.G), dim3(kStageThreads), args, smem, s);
}

template <int COST>
static cudaError_t launch_sinkhorn_kind(int tier, const WS& ws, const StageArgs& a, cudaStream_t s)
{
    WS w = ws;
    StageArgs aa = a;
    void* args[] = {(void*)&w, (void*)&aa};
    const size_t smem = stage_smem_bytes(ws.n, ws.G, tier);
    const void* f = tier == TIER_F64 ? (const void*)sinkhorn_kernel<TIER_F64, COST>
                  : tier == TIER_F32A ? (const void*)sinkhorn_kernel<TIER_F32A, COST>
                                      : (const void*)sinkhorn_kernel<TIER_F32, COST>;
    return cudaLaunchCooperativeKernel(f, dim3(ws.G), dim3(kStageThreads), args, smem, s);
}

cudaError_t launch_sinkhorn_regen(int tier, const WS& ws, const StageArgs& a, cudaStream_t s)
{
    return ws.ckind == COST_L1 ? launch_sinkhorn_kind<COST_L1>(tier, ws, a, s)
                               : launch_sinkhorn_kind<COST_SQEUCLID>(tier, ws, a, s);
}

cudaError_t launch_stage_regen(int tier, const WS& ws, const StageArgs& a, cudaStream_t s)
{
    return ws.ckind == COST_L1 ? launch_stage_kind<COST_L1>(tier, ws, a, s)
                               : launch_stage_kind<COST_SQEUCLID>(tier, ws, a, s);
}

cudaError_t launch_dual_eval_regen(int tier, const WS& ws, const EvalArgs& a, cudaStream_t s)
{
    return ws.ckind == COST_L1 ? launch_eval_kind<COST_L1>(tier, ws, a, s)
                               : launch_eval_kind<COST_SQEUCLID>(tier, ws, a, s);
}

cudaError_t configure_regen_kernels(int max_n, int G, int* min_blocks)
{
    struct K { const void* f; int tier; } ks[] = {
        {(const void*)stage_kernel_flag<TIER_F32, COST_SQEUCLID>, TIER_F32},
        {(const void*)stage_kernel<TIER_F64, COST_SQEUCLID>, TIER_F64},
        {(const void*)stage_kernel_flag<TIER_F32A, COST_SQEUCLID>, TIER_F32A},
        {(const void*)stage_kernel_flag<TIER_F32, COST_L1>, TIER_F32},
        {(const void*)stage_kernel<TIER_F64, COST_L1>, TIER_F64},
        {(const void*)stage_kernel_flag<TIER_F32A, COST_L1>, TIER_F32A},
        {(const void*)dual_eval_kernel<TIER_F32, COST_SQEUCLID>, TIER_F32},
        {(const void*)dual_eval_kernel<TIER_F64, COST_SQEUCLID>, TIER_F64},
        {(const void*)dual_eval_kernel<TIER_F32A, COST_SQEUCLID>, TIER_F32A},
        {(const void*)dual_eval_kernel<TIER_F32, COST_L1>, TIER_F32},
        {(const void*)dual_eval_kernel<TIER_F64, COST_L1>, TIER_F64},
        {(const void*)dual_eval_kernel<TIER_F32A, COST_L1>, TIER_F32A},
        {(const void*)sinkhorn_kernel<TIER_F32, COST_SQEUCLID>, TIER_F32},
        {(const void*)sinkhorn_kernel<TIER_F64, COST_SQEUCLID>, TIER_F64},
        {(const void*)sinkhorn_kernel<TIER_F32A, COST_SQEUCLID>, TIER_F32A},
        {(const void*)sinkhorn_kernel<TIER_F32, COST_L1>, TIER_F32},
        {(const void*)sinkhorn_kernel<TIER_F64, COST_L1>, TIER_F64},
        {(const void*)sinkhorn_kernel<TIER_F32A, COST_L1>, TIER_F32A}};
    for (auto& k : ks) {
        const size_t smem = stage_smem_bytes(max_n, G, k.tier);
        // the limit goes to the largest layout any n may take (fewer rows per CTA leave room for
        // more ring slots), not just to the layout of max_n
        (void)smem;
        cudaError_t e = raise_smem_limit(k.f, kSmemLimit);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k.f, kStageThreads, kSmemLimit);
        if (e != cudaSuccess) return e;
        *min_blocks = std::min(*min_blocks, nb);
    }
    return cudaSuccess;
}

}  // namespace mdot
