// Host-side launchers of the cooperative kernels (defined in k_stage.cu / k_round.cu).
#pragma once

#include <cuda_runtime.h>

#include <mutex>

#include "mdot.h"
#include "mdot_device.cuh"

namespace mdot {

struct BatchArgs;

// The library's per-thread error text (what mdot_last_error returns) and the mapping of a device
// status (SolveStatus) to mdot_status; both defined in capi.cu.
void set_last_error(const char* msg);
mdot_status status_of(int st);

// Raise (never lower) a kernel's dynamic shared-memory limit: handles of different sizes, the
// serving runtime and the no-allocation entry share the kernels of one process.
inline cudaError_t raise_smem_limit(const void* f, size_t bytes)
{
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    if ((long long)bytes <= (long long)fa.maxDynamicSharedSizeBytes) return cudaSuccess;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

size_t stage_smem_bytes(int n, int G, int tier);
size_t eval_smem_bytes(int n, int G, int tier);
size_t round_smem_bytes(int n, int G);
size_t lb_smem_bytes(int n, int G);
// Raise the dynamic shared-memory limit of every kernel to what max_n needs; returns the number
// of co-resident CTAs per SM the cooperative kernels can have (0 if one does not fit).
cudaError_t configure_kernels(int max_n, int G, int* min_blocks_per_sm);

cudaError_t launch_stage(int tier, const WS& ws, const StageArgs& a, cudaStream_t s);
cudaError_t launch_sinkhorn(int tier, const WS& ws, const StageArgs& a, cudaStream_t s);
// one stage's projection: PNCG (projector 0) or Sinkhorn (1)
inline cudaError_t launch_projection(int projector, int tier, const WS& ws, const StageArgs& a, cudaStream_t s)
{
    return projector == 1 ? launch_sinkhorn(tier, ws, a, s) : launch_stage(tier, ws, a, s);
}
cudaError_t launch_dual_eval(int tier, const WS& ws, const EvalArgs& a, cudaStream_t s);
cudaError_t launch_round(const WS& ws, const RoundArgs& a, cudaStream_t s);
cudaError_t launch_lower_bound(const WS& ws, const LbArgs& a, cudaStream_t s);
cudaError_t launch_validate(const WS& ws, double* out, cudaStream_t s);

// Are all 3n coordinates of X and Y integers of magnitude <= 255 (the tensor-core form of the
// squared-Euclidean cost)?  Synchronises st; d_flag: one device word of scratch, h_flag: pinned.
cudaError_t check_grid_points(const float* X, const float* Y, int n, unsigned int* d_flag, unsigned int* h_flag,
                              cudaStream_t st, bool* grid);

// batched solver (k_batch.cu): blocks_per_sm has one entry per tile variant (kBatchVariants)
cudaError_t configure_batch_kernels(int* blocks_per_sm);
cudaError_t launch_batch(int kind, int variant, int grid, const BatchArgs& a, cudaStream_t s);

}  // namespace mdot
