// mdot_read_probe: a streaming read of a device buffer with 128-bit loads, for measuring the
// read rate of the memory level a buffer lives in (L2 when it fits, HBM when it does not).  The
// benchmark states the roofline of the n = 4096 evaluation, whose 64 MiB cost matrix stays in L2,
// against this rate.
#include <cuda_runtime.h>

#include "launch.h"
#include "mdot.h"

namespace {

__global__ void __launch_bounds__(512) read_probe_kernel(const float4* __restrict__ buf, long long n4, int reps,
                                                         float* out)
{
    float acc = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        // four independent 16-byte loads in flight per thread per step
        long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        for (; i + 3 * stride < n4; i += 4 * stride) {
            const float4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride);
            const float4 c = __ldcg(buf + i + 2 * stride), d = __ldcg(buf + i + 3 * stride);
            acc += ((a.x + b.y) + (c.z + d.w)) + ((a.w + b.x) + (c.y + d.z));
        }
        for (; i < n4; i += stride) {
            const float4 a = __ldcg(buf + i);
            acc += (a.x + a.w);
        }
    }
    // one atomic per warp keeps the loads live without adding traffic
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

}  // namespace

extern "C" mdot_status mdot_read_probe(const float* buf, int64_t n_floats, int32_t reps, float* out, void* stream)
{
    if (!buf || !out || n_floats < 4 || (n_floats & 3) != 0 || reps < 1 ||
        (reinterpret_cast<uintptr_t>(buf) & 15) != 0)
        return MDOT_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, sizeof(float), (cudaStream_t)stream);
    if (e != cudaSuccess) {
        mdot::set_last_error(cudaGetErrorString(e));
        return MDOT_ERR_CUDA;
    }
    read_probe_kernel<<<4 * sms, 512, 0, (cudaStream_t)stream>>>(reinterpret_cast<const float4*>(buf), n_floats / 4,
                                                                   reps, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        mdot::set_last_error(cudaGetErrorString(e));
        return MDOT_ERR_CUDA;
    }
    return MDOT_OK;
}
