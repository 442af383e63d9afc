// Instantiation and cooperative launch of the barrier-synchronised stage kernel for the fp32-entry
// tiers, which carries the diagonal-Hessian direction (Eq. (16)): the stages of a solve with
// precond = 1 run here (the fp64 tier uses the same kernel from k_stage.cu).
#include <algorithm>

#include "launch.h"
#include "solver_kernels.cuh"

namespace mdot {

template <int COST>
static const void* precond_fn(int tier)
{
    return tier == TIER_F32A ? (const void*)stage_kernel<TIER_F32A, COST> : (const void*)stage_kernel<TIER_F32, COST>;
}

static const void* precond_kernel(int tier, int ckind)
{
    return ckind == COST_DENSE ? precond_fn<COST_DENSE>(tier)
         : ckind == COST_L1    ? precond_fn<COST_L1>(tier)
                               : precond_fn<COST_SQEUCLID>(tier);
}

cudaError_t launch_stage_precond(int tier, const WS& ws, const StageArgs& a, cudaStream_t s)
{
    WS w = ws;
    StageArgs aa = a;
    void* args[] = {(void*)&w, (void*)&aa};
    const size_t smem = stage_smem_bytes(ws.n, ws.G, tier);
    return cudaLaunchCooperativeKernel(precond_kernel(tier, ws.ckind), dim3(ws.G), dim3(kStageThreads), args,
                                       smem, s);
}

cudaError_t configure_precond_kernels(int G, int* min_blocks)
{
    (void)G;
    for (int ck : {COST_DENSE, COST_SQEUCLID, COST_L1})
        for (int tier : {TIER_F32, TIER_F32A}) {
            const void* f = precond_kernel(tier, ck);
            cudaError_t e = raise_smem_limit(f, kSmemLimit);
            if (e != cudaSuccess) return e;
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kStageThreads, kSmemLimit);
            if (e != cudaSuccess) return e;
            *min_blocks = std::min(*min_blocks, nb);
        }
    return cudaSuccess;
}

}  // namespace mdot
