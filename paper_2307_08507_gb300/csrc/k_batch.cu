// Instantiation and launch of the batched solver (one persistent launch for many problems).
#include <algorithm>

#include "batch_kernels.cuh"
#include "launch.h"

namespace mdot {

size_t batch_smem_bytes() { return batch_smem().bytes; }
size_t batch_slot_doubles() { return kSlotDoubles; }
int batch_max_n() { return kBatchMaxN; }

static const void* batch_fn(int kind)
{
    return kind == COST_SQEUCLID ? (const void*)batch_kernel<COST_SQEUCLID>
         : kind == COST_L1       ? (const void*)batch_kernel<COST_L1>
                                 : (const void*)batch_kernel<COST_DENSE>;
}

cudaError_t configure_batch_kernels(int* blocks_per_sm)
{
    int mb = 1 << 30;
    for (int k = 0; k < 3; ++k) {
        cudaError_t e = raise_smem_limit(batch_fn(k), batch_smem_bytes());
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_fn(k), kBatchThreads, batch_smem_bytes());
        if (e != cudaSuccess) return e;
        mb = std::min(mb, nb);
    }
    *blocks_per_sm = mb;
    return cudaSuccess;
}

cudaError_t launch_batch(int kind, int grid, const BatchArgs& a, cudaStream_t s)
{
    BatchArgs aa = a;
    void* args[] = {(void*)&aa};
    return cudaLaunchKernel(batch_fn(kind), dim3(grid), dim3(kBatchThreads), args, batch_smem_bytes(), s);
}

}  // namespace mdot
