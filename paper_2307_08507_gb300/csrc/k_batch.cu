// Instantiation and launch of the batched solver (one persistent launch for many problems), in
// its tile variants (batch_threads).
#include <algorithm>

#include "batch_kernels.cuh"
#include "launch.h"

namespace mdot {

size_t batch_smem_bytes(int variant) { return batch_smem(batch_threads(variant)).bytes; }
size_t batch_slot_doubles() { return kSlotDoubles; }
int batch_max_n() { return kBatchMaxN; }

template <int COST>
static const void* batch_fn_cost(int variant)
{
    return variant == 1 ? (const void*)batch_kernel<COST, 128> : (const void*)batch_kernel<COST, 256>;
}

static const void* batch_fn(int kind, int variant)
{
    return kind == COST_SQEUCLID ? batch_fn_cost<COST_SQEUCLID>(variant)
         : kind == COST_L1       ? batch_fn_cost<COST_L1>(variant)
                                 : batch_fn_cost<COST_DENSE>(variant);
}

// blocks_per_sm[v]: co-resident CTAs per SM of variant v (the smallest over the cost forms)
cudaError_t configure_batch_kernels(int* blocks_per_sm)
{
    for (int v = 0; v < kBatchVariants; ++v) {
        int mb = 1 << 30;
        for (int k = 0; k < 3; ++k) {
            cudaError_t e = raise_smem_limit(batch_fn(k, v), batch_smem_bytes(v));
            if (e != cudaSuccess) return e;
            int nb = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_fn(k, v), batch_threads(v), batch_smem_bytes(v));
            if (e != cudaSuccess) return e;
            mb = std::min(mb, nb);
        }
        blocks_per_sm[v] = mb;
    }
    return cudaSuccess;
}

cudaError_t launch_batch(int kind, int variant, int grid, const BatchArgs& a, cudaStream_t s)
{
    BatchArgs aa = a;
    void* args[] = {(void*)&aa};
    return cudaLaunchKernel(batch_fn(kind, variant), dim3(grid), dim3(batch_threads(variant)), args,
                            batch_smem_bytes(variant), s);
}

}  // namespace mdot
