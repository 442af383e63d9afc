// Rounding (Alg. 3) of P = exp(u 1^T + 1 v^T - gamma C) onto U(r, c), its cost <G, C> without
// forming G (optionally writing G), the c-transform lower bound on the OT value, and the input
// validation / entropy reduction.  Entries of P use the fp32 exponent of the F32 tier; every
// sum over entries is accumulated in fp64, so the written G has marginals r and c to fp64
// rounding and the cost is consistent with it.
#pragma once

#include "solver_kernels.cuh"

namespace mdot {


enum RoundMode { RM_ROWSUM = 0, RM_COLSUM = 1, RM_ROWFINAL = 2, RM_WRITE = 3 };

// One pass over the CTA's rows.  sRowX: per local row x_i 2^{A_i} (fp64); sAcc: per-warp row sums
// [warp][3][nloc] fp64 (each slot written by one lane: no atomics, fixed order).
template <int MODE, int RG, int COST>
__device__ __forceinline__ void pass_round(const WS& ws, const float* __restrict__ C, int n, int r0, int r1,
                                           const float* Hh, const float* Wc, const float* sFh,
                                           const float* sWr, const double* sRowX, float G32, float Glo,
                                           const double* Y, const double* EC, const double* ER,
                                           double inv_e1, double* sAcc, int nloc,
                                           double* colpart_b, double* G_out)
{
    constexpr int KR = 2;   // float4 groups per thread per sweep
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int BN = 4 * KR * T;
    double* wAcc = sAcc + (size_t)warp * 3 * nloc;
    for (int cb = 0; cb < n; cb += BN) {
        float hh[KR][4], wc[KR][4];
        double yv[KR][4], ev[KR][4], ca[KR][4];
        int jk[KR];
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            jk[k] = cb + 4 * (tid + k * T);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = jk[k] + e;
                const bool ok = j < n;
                hh[k][e] = ok ? __ldcg(Hh + j) : 0.0f;
                wc[k][e] = ok ? __ldcg(Wc + j) : kPadW;
                yv[k][e] = (MODE >= RM_ROWFINAL && ok) ? __ldcg(Y + j) : 0.0;
                ev[k][e] = ((MODE == RM_ROWFINAL || MODE == RM_WRITE) && ok) ? __ldcg(EC + j) : 0.0;
                ca[k][e] = 0.0;
            }
        }
        for (int rg = r0; rg < r1; rg += RG) {
            double a0[RG], a1[RG], a2[RG];
#pragma unroll
            for (int ii = 0; ii < RG; ++ii) {
                a0[ii] = 0.0; a1[ii] = 0.0; a2[ii] = 0.0;
                const int i = rg + ii;
                if (i < r1) {
                    const float fh = sFh[i - r0], wr = sWr[i - r0];
                    const double xs = sRowX[i - r0];
                    const float* Crow = C + (size_t)i * (size_t)n;
                    double er_i = 0.0;
                    if (MODE == RM_WRITE) er_i = __ldcg(ER + i) * inv_e1;
#pragma unroll
                    for (int k = 0; k < KR; ++k) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int j = jk[k] + e;
                            const float cv = (j < n) ? cost_at<COST>(ws, Crow, i, j) : 0.0f;
                            const float d = (fh + hh[k][e]) - cv;
                            const float t = fmaf(Glo, d, fmaf(G32, d, wr + wc[k][e]));
                            const double E = (double)ex2f(t);
                            if (MODE == RM_ROWSUM) {
                                a0[ii] += E;
                            } else if (MODE == RM_COLSUM) {
                                ca[k][e] = fma(xs, E, ca[k][e]);
                            } else if (MODE == RM_ROWFINAL) {
                                const double Ey = E * yv[k][e];
                                a0[ii] += Ey;
                                a1[ii] = fma(Ey, (double)cv, a1[ii]);
                                a2[ii] = fma((double)cv, ev[k][e], a2[ii]);
                            } else {
                                if (j < n) G_out[(size_t)i * n + j] = fma(xs * E, yv[k][e], er_i * ev[k][e]);
                            }
                        }
                    }
                }
            }
            if (MODE == RM_ROWSUM || MODE == RM_ROWFINAL) {
                butterfly<RG>(a0, lane);
                if (MODE == RM_ROWFINAL) {
                    butterfly<RG>(a1, lane);
                    butterfly<RG>(a2, lane);
                }
                const int il = rg + (lane % RG);
                if (lane < RG && il < r1) {
                    wAcc[il - r0] += a0[0];
                    if (MODE == RM_ROWFINAL) {
                        wAcc[nloc + il - r0] += a1[0];
                        wAcc[2 * nloc + il - r0] += a2[0];
                    }
                }
            }
        }
        if (MODE == RM_COLSUM) {
#pragma unroll
            for (int k = 0; k < KR; ++k)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (jk[k] + e < n) colpart_b[jk[k] + e] = ca[k][e];
        }
    }
}

// Smem: sFh, sWr (float), sRowX (double), sA (int), sAcc (3 x nloc doubles), merge scratch.
struct RoundSmem {
    int nloc_max;
    size_t off_fh, off_wr, off_x, off_A, off_acc, off_merge, bytes;
};

__host__ __device__ inline RoundSmem round_smem(int n, int G, int nthreads)
{
    RoundSmem L;
    L.nloc_max = (n + G - 1) / G + 1;
    size_t o = 0;
    L.off_fh = o;    o += (size_t)L.nloc_max * 4;        o = (o + 15) & ~(size_t)15;
    L.off_wr = o;    o += (size_t)L.nloc_max * 4;        o = (o + 15) & ~(size_t)15;
    L.off_x = o;     o += (size_t)L.nloc_max * 8;        o = (o + 15) & ~(size_t)15;
    L.off_A = o;     o += (size_t)L.nloc_max * 4;        o = (o + 15) & ~(size_t)15;
    L.off_acc = o;   o += (size_t)(nthreads / 32) * 3 * L.nloc_max * 8;    o = (o + 15) & ~(size_t)15;
    L.off_merge = o; o += (size_t)32 * (nthreads / 32) * 8; o = (o + 15) & ~(size_t)15;
    L.bytes = o;
    return L;
}

template <int COST>
__global__ void __launch_bounds__(kThreads, 1) round_kernel(WS ws, RoundArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double red_smem[32 * kNRed];
    __shared__ int s_flag[2];
    __shared__ unsigned int s_gen;
    const int n = ws.n, G = ws.G, b = blockIdx.x, T = blockDim.x, tid = threadIdx.x;
    const RoundSmem L = round_smem(n, G, T);
    int r0, r1, c0, c1;
    row_range(n, G, b, r0, r1);
    row_range(n, G, b, c0, c1);
    const int nloc = L.nloc_max;
    State* S = ws.st;
    float* sFh = reinterpret_cast<float*>(sm + L.off_fh);
    float* sWr = reinterpret_cast<float*>(sm + L.off_wr);
    double* sX = reinterpret_cast<double*>(sm + L.off_x);
    int* sA = reinterpret_cast<int*>(sm + L.off_A);
    double* sAcc = reinterpret_cast<double*>(sm + L.off_acc);
    const float G32 = (float)a.G64;
    const float Glo = (float)(a.G64 - (double)G32);
    double x[kNRed];
    double e1 = 0.0, cost = 0.0;
    if (tid == 0) s_gen = ld_acquire(&S->bar.gen);
    __syncthreads();
    unsigned int gen = s_gen;

    for (int j = c0 + tid; j < c1; j += T) {
        float gh, wl;
        split_cost_unit(a.v[j] / a.gamma, gh, wl, a.G64);
        ws.Hh[j] = gh;
        ws.Wc[j] = wl;
    }
    if (a.ref == nullptr) {
        if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;
        const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
        for (int i = r0 + warp; i < r1; i += nw) {
            float fh, wl;
            split_cost_unit(a.u[i] / a.gamma, fh, wl, a.G64);
            float m = -INFINITY;
            const float* Crow = ws.C + (size_t)i * n;
            for (int j = lane; j < n; j += 32)
                m = fmaxf(m, fmaf(G32, (fh + __ldcg(ws.Hh + j)) - cost_at<COST>(ws, Crow, i, j), wl + __ldcg(ws.Wc + j)));
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) sA[i - r0] = (int)fmin(fmax(ceil((double)m), -1.0e6), 1.0e6);
        }
    } else {
        for (int i = r0 + tid; i < r1; i += T) sA[i - r0] = (int)fmin(fmax(rint(a.ref[i] * kLog2e), -1.0e6), 1.0e6);
    }
    __syncthreads();
    for (int i = r0 + tid; i < r1; i += T) {
        const int il = i - r0;
        float fh, wl;
        split_cost_unit(a.u[i] / a.gamma - (double)sA[il] / a.G64, fh, wl, a.G64);
        sFh[il] = fh;
        sWr[il] = wl;
    }
    for (int x0 = tid; x0 < (T >> 5) * 3 * nloc; x0 += T) sAcc[x0] = 0.0;
    if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;

    // pass 1: r(P)_i = 2^{A_i} sum_j E_ij ; x_i = min(r_i / r(P)_i, 1)  (Alg. 3)
    pass_round<RM_ROWSUM, 4, COST>(ws, ws.C, n, r0, r1, ws.Hh, ws.Wc, sFh, sWr, sX, G32, Glo, nullptr, nullptr,
                              nullptr, 0.0, sAcc, nloc, nullptr, nullptr);
    __syncthreads();
    for (int i = r0 + tid; i < r1; i += T) {
        const int il = i - r0;
        double acc = 0.0;
        for (int w = 0; w < (T >> 5); ++w) acc += sAcc[(size_t)w * 3 * nloc + il];
        const double rP = ldexp(acc, sA[il]);
        const double xi = (rP > 0.0) ? fmin(a.r[i] / rP, 1.0) : 1.0;
        sX[il] = ldexp(xi, sA[il]);     // x_i 2^{A_i}: scale of row i of F = X P
    }
    __syncthreads();
    // pass 2: c(F)_j = sum_i x_i P_ij  (Alg. 3)
    pass_round<RM_COLSUM, 4, COST>(ws, ws.C, n, r0, r1, ws.Hh, ws.Wc, sFh, sWr, sX, G32, Glo, nullptr, nullptr,
                              nullptr, 0.0, sAcc, nloc, ws.colpartd + (size_t)b * n, nullptr);
    if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;
    for (int j0 = c0; j0 < c1; j0 += 32) {
        const double cF = merge_cols_f64(ws.colpartd, n, G, j0, c1, reinterpret_cast<double*>(sm + L.off_merge));
        const int j = j0 + tid;
        if (tid < 32 && j < c1) {
            const double yj = (cF > 0.0) ? fmin(a.c[j] / cF, 1.0) : 1.0;     // y = c / c(F) ^ 1
            a.Y[j] = yj;
            a.EC[j] = a.c[j] - cF * yj;                                        // err_c
        }
    }
    for (int x0 = tid; x0 < (T >> 5) * 3 * nloc; x0 += T) sAcc[x0] = 0.0;
    if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;
    // pass 3: r(F')_i, <F', C> by rows, (C err_c)_i   (Alg. 3)
    pass_round<RM_ROWFINAL, 4, COST>(ws, ws.C, n, r0, r1, ws.Hh, ws.Wc, sFh, sWr, sX, G32, Glo, a.Y, a.EC,
                               nullptr, 0.0, sAcc, nloc, nullptr, nullptr);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kNRed; ++q) x[q] = 0.0;
    for (int i = r0 + tid; i < r1; i += T) {
        const int il = i - r0;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int w = 0; w < (T >> 5); ++w) {
            const double* wa = sAcc + (size_t)w * 3 * nloc;
            s0 += wa[il];
            s1 += wa[nloc + il];
            s2 += wa[2 * nloc + il];
        }
        const double rF = sX[il] * s0;
        const double er = a.r[i] - rF;
        a.ER[i] = er;
        x[0] += sX[il] * s1;                   // <F', C> row i
        x[1] += fabs(er);                      // ||err_r||_1
        x[2] += er * s2;                       // err_r^T C err_c
    }
    block_reduce_nred(x, red_smem);
    if (tid == 0)
        for (int q = 0; q < kNRed; ++q) ws.blockred[(size_t)b * kNRed + q] = x[q];
    if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;
    {
        const int lane = tid & 31, warp = tid >> 5;
        if (warp < 3) {
            double s = 0.0;
            for (int bb = lane; bb < G; bb += 32) s += __ldcg(ws.blockred + (size_t)bb * kNRed + warp);
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) red_smem[warp] = s;
        }
        __syncthreads();
        const double costF = red_smem[0];
        e1 = red_smem[1];
        const double ecc = red_smem[2];
        cost = costF + ((e1 > 0.0) ? ecc / e1 : 0.0);
        if (b == 0 && tid == 0) {
            a.out[0] = cost;
            a.out[1] = e1;
            a.out[2] = ecc;
            a.out[3] = costF;
        }
    }
    if (a.G_out != nullptr) {
        // G = F' + err_r err_c^T / ||err_r||_1 (Alg. 3), written row-major in fp64
        pass_round<RM_WRITE, 4, COST>(ws, ws.C, n, r0, r1, ws.Hh, ws.Wc, sFh, sWr, sX, G32, Glo, a.Y, a.EC,
                                 a.ER, (e1 > 0.0) ? 1.0 / e1 : 0.0, sAcc, nloc, nullptr, a.G_out);
    }
    return;
timeout:
    if (tid == 0) atomicMax(&S->status, (int)ST_TIMEOUT);
}

// ---------------------------------------------------------------------------------------------
// c-transform lower bound: g'_j = min_i (C_ij - f_i), f'_i = min_j (C_ij - g'_j), fp64
// ---------------------------------------------------------------------------------------------

template <int COST>
__global__ void __launch_bounds__(kThreads, 1) lower_bound_kernel(WS ws, LbArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double red_smem[32 * kNRed];
    __shared__ int s_flag[2];
    __shared__ unsigned int s_gen;
    const int n = ws.n, G = ws.G, b = blockIdx.x, T = blockDim.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    int r0, r1, c0, c1;
    row_range(n, G, b, r0, r1);
    row_range(n, G, b, c0, c1);
    State* S = ws.st;
    double x[kNRed];
    if (tid == 0) s_gen = ld_acquire(&S->bar.gen);
    __syncthreads();
    unsigned int gen = s_gen;
    double* sf = reinterpret_cast<double*>(sm);
    for (int i = r0 + tid; i < r1; i += T) sf[i - r0] = a.u[i] / a.gamma;      // f = u / gamma
    __syncthreads();
    // column minima over own rows: thread owns columns j = tid, tid + T, ...
    for (int j = tid; j < n; j += T) {
        double m = INFINITY;
        for (int i = r0; i < r1; ++i) m = fmin(m, (double)cost_elem<COST>(ws, i, j) - sf[i - r0]);
        ws.colpartd[(size_t)b * n + j] = m;
    }
    if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;
    for (int j = c0 + tid; j < c1; j += T) {
        double m = INFINITY;
        for (int bb = 0; bb < G; ++bb) m = fmin(m, __ldcg(ws.colpartd + (size_t)bb * n + j));
        a.gp[j] = m;
    }
    if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;
#pragma unroll
    for (int q = 0; q < kNRed; ++q) x[q] = 0.0;
    // row minima f'_i = min_j (C_ij - g'_j), one warp per row
    for (int i = r0 + warp; i < r1; i += nw) {
        double m = INFINITY;
        const float* Crow = ws.C + (size_t)i * n;
        for (int j = lane; j < n; j += 32) m = fmin(m, (double)cost_at<COST>(ws, Crow, i, j) - __ldcg(a.gp + j));
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) x[0] += m * a.r[i];
    }
    for (int j = c0 + tid; j < c1; j += T) x[1] += __ldcg(a.gp + j) * a.c[j];
    block_reduce_nred(x, red_smem);
    if (tid == 0) ws.blockred[(size_t)b * kNRed] = x[0] + x[1];
    if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;
    if (b == 0 && tid == 0) {
        double s = 0.0;
        for (int bb = 0; bb < G; ++bb) s += __ldcg(ws.blockred + (size_t)bb * kNRed);
        a.out[0] = s;
    }
    return;
timeout:
    if (tid == 0) atomicMax(&S->status, (int)ST_TIMEOUT);
}

// ---------------------------------------------------------------------------------------------
// validation / entropy: out = {sum r, sum c, H(r), H(c), min r, min c, #non-finite}
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1) validate_kernel(WS ws, double* out)
{
    __shared__ double red_smem[32 * kNRed];
    __shared__ double s_min[2][32];
    __shared__ int s_flag[2];
    __shared__ unsigned int s_gen;
    const int n = ws.n, G = ws.G, b = blockIdx.x, T = blockDim.x, tid = threadIdx.x;
    State* S = ws.st;
    int r0, r1;
    row_range(n, G, b, r0, r1);
    double x[kNRed];
#pragma unroll
    for (int q = 0; q < kNRed; ++q) x[q] = 0.0;
    double mr = INFINITY, mc = INFINITY;
    if (tid == 0) s_gen = ld_acquire(&S->bar.gen);
    __syncthreads();
    unsigned int gen = s_gen;
    for (int i = r0 + tid; i < r1; i += T) {
        const double ri = ws.r[i], ci = ws.c[i];
        x[0] += ri;
        x[1] += ci;
        if (ri > 0.0) x[2] -= ri * log(ri);
        if (ci > 0.0) x[3] -= ci * log(ci);
        x[4] += (isfinite(ri) && isfinite(ci)) ? 0.0 : 1.0;
        mr = fmin(mr, ri);
        mc = fmin(mc, ci);
    }
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        mr = fmin(mr, __shfl_xor_sync(0xffffffffu, mr, o));
        mc = fmin(mc, __shfl_xor_sync(0xffffffffu, mc, o));
    }
    if ((tid & 31) == 0) { s_min[0][tid >> 5] = mr; s_min[1][tid >> 5] = mc; }
    block_reduce_nred(x, red_smem);
    if (tid == 0) {
        for (int w = 0; w < (T >> 5); ++w) { mr = fmin(mr, s_min[0][w]); mc = fmin(mc, s_min[1][w]); }
        for (int q = 0; q < 5; ++q) ws.blockred[(size_t)b * kNRed + q] = x[q];
        ws.scratch[(size_t)b * 8 + 0] = mr;
        ws.scratch[(size_t)b * 8 + 1] = mc;
    }
    if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;
    if (b == 0 && tid == 0) {
        double t[5] = {0, 0, 0, 0, 0};
        double m0 = INFINITY, m1 = INFINITY;
        for (int bb = 0; bb < G; ++bb) {
            for (int q = 0; q < 5; ++q) t[q] += __ldcg(ws.blockred + (size_t)bb * kNRed + q);
            m0 = fmin(m0, __ldcg(ws.scratch + (size_t)bb * 8 + 0));
            m1 = fmin(m1, __ldcg(ws.scratch + (size_t)bb * 8 + 1));
        }
        out[0] = t[0]; out[1] = t[1]; out[2] = t[2]; out[3] = t[3];
        out[4] = m0; out[5] = m1; out[6] = t[4];
    }
    return;
timeout:
    if (tid == 0) atomicMax(&S->status, (int)ST_TIMEOUT);
}

}  // namespace mdot
