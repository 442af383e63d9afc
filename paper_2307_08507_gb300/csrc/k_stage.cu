// Instantiation and cooperative launch of the stage and dual-evaluation kernels.
#include <algorithm>
#include <cstring>
#include "launch.h"
#include "solver_kernels.cuh"

namespace mdot {

size_t stage_smem_bytes(int n, int G, int tier) { return smem_layout(n, G, tier, kStageThreads).bytes; }
// the standalone dual evaluation (wide column merge)
size_t eval_smem_bytes(int n, int G, int tier) { return smem_layout(n, G, tier, kStageThreads, true).bytes; }
// the flag-synchronised stage kernel with dense C (its own block size, the published-state copy)
static size_t flag_smem_bytes(int n, int G, int tier)
{
    return smem_layout(n, G, tier, kFlagDenseThreads, false, true).bytes;
}

template <typename K>
static cudaError_t coop(K kernel, int G, size_t smem, cudaStream_t s, void** args, int threads = kStageThreads)
{
    return cudaLaunchCooperativeKernel((const void*)kernel, dim3(G), dim3(threads), args, smem, s);
}

cudaError_t launch_stage_regen(int tier, const WS& ws, const StageArgs& a, cudaStream_t s);
cudaError_t launch_dual_eval_regen(int tier, const WS& ws, const EvalArgs& a, cudaStream_t s);
cudaError_t configure_regen_kernels(int max_n, int G, int* min_blocks);

cudaError_t launch_stage_precond(int tier, const WS& ws, const StageArgs& a, cudaStream_t s);
cudaError_t configure_precond_kernels(int G, int* min_blocks);

cudaError_t launch_stage(int tier, const WS& ws, const StageArgs& a, cudaStream_t s)
{
    // the diagonal-Hessian direction lives in the barrier-synchronised kernel (fp32 tiers: own unit)
    if (a.precond && tier != TIER_F64) return launch_stage_precond(tier, ws, a, s);
    if (ws.ckind != COST_DENSE) return launch_stage_regen(tier, ws, a, s);
    WS w = ws;
    StageArgs aa = a;
    void* args[] = {(void*)&w, (void*)&aa};
    if (tier == TIER_F64) return coop(stage_kernel<TIER_F64, COST_DENSE>, ws.G, stage_smem_bytes(ws.n, ws.G, tier), s, args);
    // the flag-synchronised kernel streams dense C through its TMA ring only: other C (n not a
    // multiple of 4, C not 16-byte aligned, no room for two ring slots) takes the
    // barrier-synchronised kernel, same arithmetic
    if ((ws.n & 3) != 0 || (reinterpret_cast<uintptr_t>(ws.C) & 15) != 0 ||
        smem_layout(ws.n, ws.G, tier, kFlagDenseThreads, false, true).stages < 2)
        return launch_stage_precond(tier, ws, a, s);
    const size_t smem = flag_smem_bytes(ws.n, ws.G, tier);
    if (tier == TIER_F32A)
        return coop(stage_kernel_flag<TIER_F32A, COST_DENSE>, ws.G, smem, s, args, kFlagDenseThreads);
    return coop(stage_kernel_flag<TIER_F32, COST_DENSE>, ws.G, smem, s, args, kFlagDenseThreads);
}

cudaError_t launch_sinkhorn_regen(int tier, const WS& ws, const StageArgs& a, cudaStream_t s);

cudaError_t launch_sinkhorn(int tier, const WS& ws, const StageArgs& a, cudaStream_t s)
{
    if (ws.ckind != COST_DENSE) return launch_sinkhorn_regen(tier, ws, a, s);
    WS w = ws;
    StageArgs aa = a;
    void* args[] = {(void*)&w, (void*)&aa};
    const size_t smem = stage_smem_bytes(ws.n, ws.G, tier);
    if (tier == TIER_F64) return coop(sinkhorn_kernel<TIER_F64, COST_DENSE>, ws.G, smem, s, args);
    if (tier == TIER_F32A) return coop(sinkhorn_kernel<TIER_F32A, COST_DENSE>, ws.G, smem, s, args);
    return coop(sinkhorn_kernel<TIER_F32, COST_DENSE>, ws.G, smem, s, args);
}

cudaError_t launch_dual_eval(int tier, const WS& ws, const EvalArgs& a, cudaStream_t s)
{
    if (ws.ckind != COST_DENSE) return launch_dual_eval_regen(tier, ws, a, s);
    WS w = ws;
    EvalArgs aa = a;
    void* args[] = {(void*)&w, (void*)&aa};
    const size_t smem = eval_smem_bytes(ws.n, ws.G, tier);
    if (tier == TIER_F64) return coop(dual_eval_kernel<TIER_F64, COST_DENSE>, ws.G, smem, s, args);
    if (tier == TIER_F32A) return coop(dual_eval_kernel<TIER_F32A, COST_DENSE>, ws.G, smem, s, args);
    return coop(dual_eval_kernel<TIER_F32, COST_DENSE>, ws.G, smem, s, args);
}

cudaError_t configure_stage_kernels(int max_n, int G, int* min_blocks)
{
    struct K { const void* f; int tier; int threads; } ks[] = {
        {(const void*)stage_kernel_flag<TIER_F32, COST_DENSE>, TIER_F32, kFlagDenseThreads},
        {(const void*)stage_kernel<TIER_F64, COST_DENSE>, TIER_F64, kStageThreads},
        {(const void*)stage_kernel_flag<TIER_F32A, COST_DENSE>, TIER_F32A, kFlagDenseThreads},
        {(const void*)dual_eval_kernel<TIER_F32, COST_DENSE>, TIER_F32, kStageThreads},
        {(const void*)dual_eval_kernel<TIER_F64, COST_DENSE>, TIER_F64, kStageThreads},
        {(const void*)dual_eval_kernel<TIER_F32A, COST_DENSE>, TIER_F32A, kStageThreads},
        {(const void*)sinkhorn_kernel<TIER_F32, COST_DENSE>, TIER_F32, kStageThreads},
        {(const void*)sinkhorn_kernel<TIER_F64, COST_DENSE>, TIER_F64, kStageThreads},
        {(const void*)sinkhorn_kernel<TIER_F32A, COST_DENSE>, TIER_F32A, kStageThreads}};
    for (auto& k : ks) {
        // the limit goes to the largest layout any n may take (fewer rows per CTA leave room for
        // more ring slots), not just to the layout of max_n
        (void)max_n;
        cudaError_t e = raise_smem_limit(k.f, kSmemLimit);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k.f, k.threads, kSmemLimit);
        if (e != cudaSuccess) return e;
        *min_blocks = std::min(*min_blocks, nb);
    }
    cudaError_t e = configure_regen_kernels(max_n, G, min_blocks);
    if (e != cudaSuccess) return e;
    return configure_precond_kernels(G, min_blocks);
}

}  // namespace mdot

extern "C" mdot_status mdot_phase_timers(uint64_t* out, int32_t max_ctas, int32_t clear)
{
    using namespace mdot;
    if (!out || max_ctas < 1) return MDOT_ERR_INVALID_ARG;
#ifdef MDOT_PHASE_TIMERS
    static unsigned long long h[kPhaseCtas][kPhases + 1];
    if (cudaMemcpyFromSymbol(h, g_phase, sizeof(h)) != cudaSuccess) return MDOT_ERR_CUDA;
    const int m = std::min(max_ctas, kPhaseCtas);
    for (int b = 0; b < m; ++b)
        for (int k = 0; k <= kPhases; ++k) out[(size_t)b * (kPhases + 1) + k] = h[b][k];
    if (clear) {
        memset(h, 0, sizeof(h));
        if (cudaMemcpyToSymbol(g_phase, h, sizeof(h)) != cudaSuccess) return MDOT_ERR_CUDA;
    }
    return MDOT_OK;
#else
    (void)clear;
    return MDOT_NOT_READY;
#endif
}
