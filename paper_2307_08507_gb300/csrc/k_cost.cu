// The regenerated cost outside the solver: the check that selects the tensor-core form (integer
// points, |coordinate| <= 255) and mdot_cost_matrix, which writes C with the arithmetic the
// passes use (tensor cores for such points with the squared-Euclidean cost, fp32 operations in
// the fixed order of point_cost otherwise).
#include <cuda_runtime.h>

#include "launch.h"
#include "mdot.h"
#include "solver_kernels.cuh"

namespace mdot {

namespace {

__device__ __forceinline__ bool small_integer(float v) { return fabsf(v) <= 255.0f && v == rintf(v); }

__global__ void grid_points_kernel(const float* __restrict__ X, const float* __restrict__ Y, long long m,
                                   unsigned int* bad)
{
    bool ok = true;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (long long)gridDim.x * blockDim.x)
        ok = ok && small_integer(__ldg(X + q)) && small_integer(__ldg(Y + q));
    if (!__all_sync(0xffffffffu, ok) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}

// One warp per 16 x 32 tile of C (tensor-core form) or per 32 columns of 16 rows (fp32 form).
template <bool TC, int KIND>
__global__ void __launch_bounds__(256) cost_matrix_kernel(const float* __restrict__ X, const float* __restrict__ Y,
                                                          float s, int n, float* __restrict__ C)
{
    constexpr int NT = 4;
    const int lane = threadIdx.x & 31;
    const long long tile = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int tiles_c = (n + 8 * NT - 1) / (8 * NT);
    const long long tiles = (long long)((n + 15) / 16) * tiles_c;
    if (tile >= tiles) return;                     // a whole warp leaves together
    const int i0 = (int)(tile / tiles_c) * 16, j0 = (int)(tile % tiles_c) * 8 * NT;
    if (TC) {
        const int g = lane >> 2, t = lane & 3;
        const int ia = i0 + g, ib = i0 + g + 8;
        unsigned int a0 = 0u, a1 = 0u, a2 = 0u, a3 = 0u;
        if (ia < n) tc_a_regs(X[3 * (size_t)ia], X[3 * (size_t)ia + 1], X[3 * (size_t)ia + 2], t, a0, a2);
        if (ib < n) tc_a_regs(X[3 * (size_t)ib], X[3 * (size_t)ib + 1], X[3 * (size_t)ib + 2], t, a1, a3);
        const float2 S = pk(s), Z = pk(-(s * 0.0f));
#pragma unroll
        for (int q = 0; q < NT; ++q) {
            const int jb = j0 + 8 * q + g;
            unsigned int b0 = 0u, b1 = 0u;
            if (jb < n) tc_b_regs(Y[3 * (size_t)jb], Y[3 * (size_t)jb + 1], Y[3 * (size_t)jb + 2], t, b0, b1);
            float d[4];
            mma_bf16_16816(d, a0, a1, a2, a3, b0, b1);
            const float2 c0 = fma2(make_float2(d[0], d[1]), S, Z);
            const float2 c1 = fma2(make_float2(d[2], d[3]), S, Z);
            const int j = j0 + 8 * q + 2 * t;
            if (ia < n) {
                if (j < n) C[(size_t)ia * n + j] = c0.x;
                if (j + 1 < n) C[(size_t)ia * n + j + 1] = c0.y;
            }
            if (ib < n) {
                if (j < n) C[(size_t)ib * n + j] = c1.x;
                if (j + 1 < n) C[(size_t)ib * n + j + 1] = c1.y;
            }
        }
    } else {
        const int j = j0 + lane;
        if (j >= n) return;
        const float y0 = Y[3 * (size_t)j], y1 = Y[3 * (size_t)j + 1], y2 = Y[3 * (size_t)j + 2];
        for (int i = i0; i < min(i0 + 16, n); ++i)
            C[(size_t)i * n + j] = point_cost<KIND>(X[3 * (size_t)i], X[3 * (size_t)i + 1], X[3 * (size_t)i + 2], y0,
                                                    y1, y2, s);
    }
}

}  // namespace

cudaError_t check_grid_points(const float* X, const float* Y, int n, unsigned int* d_flag, unsigned int* h_flag,
                              cudaStream_t st, bool* grid)
{
    cudaError_t e = cudaMemsetAsync(d_flag, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    const long long m = 3LL * n;
    const int blocks = (int)std::min<long long>((m + 255) / 256, 1024);
    grid_points_kernel<<<blocks, 256, 0, st>>>(X, Y, m, d_flag);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_flag, d_flag, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) *grid = (*h_flag == 0u);
    return e;
}

}  // namespace mdot

extern "C" mdot_status mdot_cost_matrix(const float* x, const float* y, int32_t cost_kind, float scale, int64_t n,
                                        float* C_out, void* stream)
{
    using namespace mdot;
    if (!x || !y || !C_out || n < 1 || n > (1 << 20) || !(scale > 0.0f) || !std::isfinite(scale) ||
        (cost_kind != MDOT_COST_SQEUCLID && cost_kind != MDOT_COST_L1))
        return MDOT_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned int* d_flag = nullptr;
    unsigned int h_flag = 0;
    bool grid = false;
    cudaError_t e = cudaSuccess;
    if (cost_kind == MDOT_COST_SQEUCLID) {
        e = cudaMallocAsync((void**)&d_flag, sizeof(unsigned int), st);
        if (e == cudaSuccess) e = check_grid_points(x, y, (int)n, d_flag, &h_flag, st, &grid);
        if (d_flag) cudaFreeAsync(d_flag, st);
    }
    if (e == cudaSuccess) {
        const long long tiles = (long long)((n + 15) / 16) * ((n + 31) / 32);
        const int blocks = (int)((tiles + 7) / 8);
        if (cost_kind == MDOT_COST_L1)
            cost_matrix_kernel<false, COST_L1><<<blocks, 256, 0, st>>>(x, y, scale, (int)n, C_out);
        else if (grid)
            cost_matrix_kernel<true, COST_SQEUCLID><<<blocks, 256, 0, st>>>(x, y, scale, (int)n, C_out);
        else
            cost_matrix_kernel<false, COST_SQEUCLID><<<blocks, 256, 0, st>>>(x, y, scale, (int)n, C_out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        return MDOT_ERR_CUDA;
    }
    return MDOT_OK;
}
