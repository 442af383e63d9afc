// Device-side building blocks of the MDOT-PNCG library (sm_103a).
//
// One dual evaluation (the two reductions of Alg. 2) is one pass over the n x n cost matrix.  A cooperative
// grid of G CTAs (one per SM) splits the ROWS evenly: CTA b owns rows [r0_b, r1_b) and sweeps all
// columns in blocks of 4*K*T.  Per entry it forms the log2 of P_ij relative to a per-row scale
// 2^{A_i}, takes ONE exp2, and adds the result both into the row sum (complete inside the CTA) and,
// scaled by 2^{A_i - Aglob}, into a per-CTA column partial.  A second phase merges the G column
// partials of the columns each CTA owns.  Rows and columns of the O(n) epilogue (gradient,
// Sinkhorn direction, phi', beta terms; Eq. (4), (17), (18), (26)) are finished by their owners.
//
// fp32 entries ("F32 tier"): with f_i = u_i/gamma - A_i/(gamma log2 e) and g_j = v_j/gamma split
// into a part quantised to 2^-21 and a remainder, the cost-unit difference (fh_i + gh_j) - C_ij is
// exact (Sterbenz), so
//     log2 P_ij - A_i = G * ((fh_i + gh_j) - C_ij) + G*(fl_i + gl_j),   G = gamma log2 e,
// is formed with relative error ~2^-24 of its own (small) value instead of ~2^-24 of gamma.
// fp64 entries ("F64 tier") evaluate u_i + v_j - gamma C_ij and exp() in double.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mdot {

constexpr double kLog2e = 1.4426950408889634074;
constexpr double kLn2 = 0.69314718055994530942;
constexpr double kQuant = 2097152.0;          // 2^21: quantum of the exact part of f, g
constexpr int kNRed = 6;                       // scalars reduced per evaluation
constexpr int kThreads = 256;                  // CTA size of the cooperative kernels
constexpr int kK = 4;                          // float4 column groups per thread per sweep

enum Tier { TIER_F32 = 0, TIER_F64 = 1 };
enum EvalKind { KIND_INIT = 0, KIND_TRIAL = 1, KIND_FORCE = 2 };
enum Phase { PH_RUN = 0, PH_DONE = 1 };
enum SolveStatus { ST_OK = 0, ST_CAP = 1, ST_LSFAIL = 2, ST_NUMERIC = 3, ST_TIMEOUT = 4 };

struct GridBar {
    unsigned int count;
    unsigned int gen;
    unsigned int abort;
    unsigned int pad;
};

// Scalar state of one projection (one MDOT stage) plus cumulative counters.
struct State {
    double alpha;          // step of the evaluation in flight
    double lo, hi, dlo, dhi, d0;   // line-search bracket (App. B) and phi'(0)
    double beta;           // beta applied at the next commit (Eq. (18))
    double alpha_commit;   // step committed at the next commit
    double gnorm;          // ||grad g||_1 at the current point
    int kind;              // EvalKind of the evaluation in flight
    int accept;            // the last evaluation was accepted
    int trials;            // phi' evaluations in the current line search
    int k;                 // PNCG iterations in this stage
    int phase;             // Phase
    int status;            // SolveStatus (sticky, worst wins)
    int pad0, pad1;
    long long evals, evals64, iters, ls_trials;
    GridBar bar;
};

struct WS {
    int n, G;
    const float* C;
    const double *r, *c;              // original marginals
    double *rt, *ct, *lrt, *lct;      // smoothed marginals and logs (Alg. 1)
    double *u, *v, *pu, *pv, *uprev, *vprev;
    double *gr, *gc;                  // gradient at the current point
    double *grt, *gct, *srt, *sct;    // gradient and Sinkhorn direction at the trial point
    double *lr, *lrtr;                // log r(P) at the current / trial point
    double *lcout;                    // log c(P) at the trial point
    float *Fh, *Wr, *Hh, *Wc;         // fp32 per-row / per-column constants of the trial
    double *Fd, *Hd;                  // fp64 per-row / per-column constants of the trial
    int* A;                           // per-row log2 scales
    float* colpart;                   // [G][n] fp32 column partials
    double* colpartd;                 // [G][n] fp64 column partials
    double* blockred;                 // [G][kNRed]
    double* scratch;                  // [G][8] misc per-CTA values
    State* st;
};

struct StageArgs {
    double gamma, G64, tol, w, ratio, c1, c2;
    int first, warm_start, tier, ls_max_trials, max_iter, Aglob;
};

// Arguments of the standalone dual evaluation (mdot_dual_eval).
struct EvalArgs {
    double gamma, G64;
    const double* u;
    const double* v;
    const double* ref;   // nullable
};

// Arguments of the rounding kernel (Alg. 3).
struct RoundArgs {
    double gamma, G64;
    const double *u, *v, *r, *c;
    const double* ref;     // nullable: estimate of log r(P) for the row scales
    double* Y;             // [n] y_j
    double* EC;            // [n] err_c
    double* ER;            // [n] err_r
    double* G_out;         // nullable, n*n
    double* out;           // [8] results: cost, ||err_r||_1, <err_r, C err_c>, <F', C>
};

// Arguments of the c-transform lower bound.
struct LbArgs {
    double gamma;
    const double *u, *r, *c;
    double* gp;     // [n] g'
    double* out;    // [1]
};

// ---------------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float4 ldg4(const float* p)
{
    return __ldg(reinterpret_cast<const float4*>(p));
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ float pow2f_int(int e)
{
    if (e < -126) return 0.0f;
    if (e > 127) return __int_as_float(0x7f800000);
    return __int_as_float((e + 127) << 23);
}

__device__ __forceinline__ void row_range(int n, int G, int b, int& r0, int& r1)
{
    r0 = (int)(((long long)b * n) / G);
    r1 = (int)(((long long)(b + 1) * n) / G);
}

// Kahan-compensated fp32 accumulation.
__device__ __forceinline__ void kahan_add(float& s, float& comp, float x)
{
    float y = x - comp;
    float t = s + y;
    comp = (t - s) - y;
    s = t;
}

// Reduce N values held by every lane across the 32 lanes of a warp; afterwards lane l holds in
// v[0] the warp total of value (l mod N).  N = 32, 16 or 8.  Fixed shuffle tree: deterministic.
template <int N, typename T>
__device__ __forceinline__ void butterfly(T (&v)[N], int lane)
{
#pragma unroll
    for (int o = 16; o >= N; o >>= 1) {
#pragma unroll
        for (int q = 0; q < N; ++q) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    }
#pragma unroll
    for (int o = N / 2; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int q = 0; q < o; ++q) {
            T send = upper ? v[q] : v[q + o];
            T keep = upper ? v[q + o] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
}

// Block-wide sum of kNRed doubles; result valid in thread 0.  red_smem: >= 32 * kNRed doubles.
__device__ __forceinline__ void block_reduce_nred(double (&x)[kNRed], double* red_smem)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < kNRed; ++q)
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) x[q] += __shfl_xor_sync(0xffffffffu, x[q], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < kNRed; ++q) red_smem[warp * kNRed + q] = x[q];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < kNRed; ++q) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += red_smem[w * kNRed + q];
            x[q] = s;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// grid barrier with a bounded wait: a CTA that waits longer than the limit raises `abort`, every
// waiter leaves, and the kernel returns with ST_TIMEOUT instead of hanging.
// ---------------------------------------------------------------------------------------------
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;   // 2 s

// s_flag points at two ints in shared memory: [0] "last to arrive", [1] "wait succeeded" (kept
// apart so that a thread still reading one cannot see the other being rewritten).
__device__ __forceinline__ bool bar_arrive(GridBar* gb, unsigned int nblocks, int* s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned int prev = atomicAdd(&gb->count, 1u);
        s_flag[0] = (prev == nblocks - 1u);
    }
    __syncthreads();
    return s_flag[0] != 0;
}

__device__ __forceinline__ void bar_release(GridBar* gb, unsigned int target)
{
    // thread 0 of the last CTA
    gb->count = 0u;
    __threadfence();
    atomicExch(&gb->gen, target);
}

__device__ __forceinline__ bool bar_wait(GridBar* gb, unsigned int target, int* s_flag)
{
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long t0 = globaltimer();
        unsigned int spins = 0;
        while (true) {
            unsigned int g = ld_acquire(&gb->gen);
            if ((int)(g - target) >= 0) break;
            if (ld_acquire(&gb->abort)) { ok = 0; break; }
            if (++spins > 64u) __nanosleep(64);
            if ((spins & 255u) == 0u && globaltimer() - t0 > kBarrierTimeoutNs) {
                atomicExch(&gb->abort, 1u);
                ok = 0;
                break;
            }
        }
        __threadfence();
        s_flag[1] = ok;
    }
    __syncthreads();
    return s_flag[1] != 0;
}

// Full barrier: arrive + (last CTA releases) + wait.
__device__ __forceinline__ bool grid_sync(GridBar* gb, unsigned int nblocks, unsigned int& gen, int* s_flag)
{
    ++gen;
    bool last = bar_arrive(gb, nblocks, s_flag);
    if (last && threadIdx.x == 0) bar_release(gb, gen);
    return bar_wait(gb, gen, s_flag);
}

// ---------------------------------------------------------------------------------------------
// per-row / per-column constants of an evaluation at u + alpha p_u, v + alpha p_v
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void split_cost_unit(double x, float& hi, float& lo, double G64)
{
    const double h = rint(x * kQuant) / kQuant;   // exact in fp32 while |x| < 8
    hi = (float)h;
    lo = (float)(G64 * (x - h));
}

// Row scale A_i = round(log2 of the predicted row sum).  Not clamped to the fp32 exponent range:
// the row sum is formed relative to 2^{A_i} for any A_i; only the column weight 2^{A_i - Aglob}
// flushes to 0 below 2^-126 (see pow2f_int).
__device__ __forceinline__ int row_scale(double log_r_pred)
{
    double a = rint(log_r_pred * kLog2e);
    a = fmin(fmax(a, -1.0e6), 1.0e6);
    return (int)a;
}

// ---------------------------------------------------------------------------------------------
// Phase A: one pass over the rows [r0, r1) of C.  Row sums go to sRow[warp][local row]
// (accumulated, fp32 or fp64), column partials to colpart_b[j].
// ---------------------------------------------------------------------------------------------
template <bool VEC4>
__device__ __forceinline__ void pass_f32(const float* __restrict__ C, int n, int r0, int r1,
                                         const float* Hh, const float* Wc,
                                         const float* sFh, const float* sWr, const float* sS,
                                         float G32, float Glo, float* sRow, int nloc,
                                         float* colpart_b)
{
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int BN = 4 * kK * T;
    for (int cb = 0; cb < n; cb += BN) {
        float hh[kK][4], wc[kK][4], ca[kK][4];
        int jk[kK];
#pragma unroll
        for (int k = 0; k < kK; ++k) {
            jk[k] = cb + 4 * (tid + k * T);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = jk[k] + e;
                const bool ok = j < n;
                // per-trial constants are rewritten inside the launch: read through L2, never the
                // non-coherent path
                hh[k][e] = ok ? __ldcg(Hh + j) : 0.0f;
                wc[k][e] = ok ? __ldcg(Wc + j) : -INFINITY;     // invalid column: exp2(-inf) = 0
                ca[k][e] = 0.0f;
            }
        }
        for (int rg = r0; rg < r1; rg += 32) {
            float rp[32];
#pragma unroll
            for (int ii = 0; ii < 32; ++ii) {
                rp[ii] = 0.0f;
                const int i = rg + ii;
                if (i < r1) {
                    const float fh = sFh[i - r0], wr = sWr[i - r0], s = sS[i - r0];
                    const float* Crow = C + (size_t)i * (size_t)n;
#pragma unroll
                    for (int k = 0; k < kK; ++k) {
                        float cv[4];
                        if (VEC4) {
                            if (jk[k] < n) {
                                float4 t4 = ldg4(Crow + jk[k]);
                                cv[0] = t4.x; cv[1] = t4.y; cv[2] = t4.z; cv[3] = t4.w;
                            } else {
                                cv[0] = cv[1] = cv[2] = cv[3] = 0.0f;
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e) cv[e] = (jk[k] + e < n) ? __ldg(Crow + jk[k] + e) : 0.0f;
                        }
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float d = (fh + hh[k][e]) - cv[e];
                            const float t = fmaf(Glo, d, fmaf(G32, d, wr + wc[k][e]));
                            const float E = ex2f(t);
                            rp[ii] += E;
                            ca[k][e] = fmaf(E, s, ca[k][e]);
                        }
                    }
                }
            }
            butterfly<32>(rp, lane);
            const int il = rg + lane;
            if (il < r1) sRow[warp * nloc + (il - r0)] += rp[0];
        }
#pragma unroll
        for (int k = 0; k < kK; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (jk[k] + e < n) colpart_b[jk[k] + e] = ca[k][e];
    }
}

__device__ __forceinline__ void pass_f64(const float* __restrict__ C, int n, int r0, int r1,
                                         const double* Hd, const double* sFd,
                                         const double* sS, double gamma, double* sRow, int nloc,
                                         double* colpart_b)
{
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int BN = 4 * kK * T;
    for (int cb = 0; cb < n; cb += BN) {
        double hd[kK][4], ca[kK][4];
        int jk[kK];
#pragma unroll
        for (int k = 0; k < kK; ++k) {
            jk[k] = cb + 4 * (tid + k * T);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = jk[k] + e;
                hd[k][e] = (j < n) ? __ldcg(Hd + j) : -INFINITY;
                ca[k][e] = 0.0;
            }
        }
        for (int rg = r0; rg < r1; rg += 16) {
            double rp[16];
#pragma unroll
            for (int ii = 0; ii < 16; ++ii) {
                rp[ii] = 0.0;
                const int i = rg + ii;
                if (i < r1) {
                    const double fd = sFd[i - r0], s = sS[i - r0];
                    const float* Crow = C + (size_t)i * (size_t)n;
#pragma unroll
                    for (int k = 0; k < kK; ++k) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int j = jk[k] + e;
                            const double cv = (j < n) ? (double)__ldg(Crow + j) : 0.0;
                            const double E = exp((fd + hd[k][e]) - gamma * cv);
                            rp[ii] += E;
                            ca[k][e] = fma(E, s, ca[k][e]);
                        }
                    }
                }
            }
            butterfly<16>(rp, lane);
            const int il = rg + (lane & 15);
            if (lane < 16 && il < r1) sRow[warp * nloc + (il - r0)] += rp[0];
        }
#pragma unroll
        for (int k = 0; k < kK; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (jk[k] + e < n) colpart_b[jk[k] + e] = ca[k][e];
    }
}

// Two-scale pass of the generic dual evaluation: the row sum of row i uses exponents relative to
// the row scale A_i (folded into the row constants sFh/sWr), the column sum of column j uses
// exponents relative to the column scale B_j (folded into the column constants Hh2/Wc2), so both
// log-sum-exps stay exact for potentials of any spread.  Two exp2 per entry.
template <bool VEC4>
__device__ __forceinline__ void pass2_f32(const float* __restrict__ C, int n, int r0, int r1,
                                          const float* Hh, const float* Wc, const float* Hh2,
                                          const float* Wc2, const float* sFh, const float* sWr,
                                          const float* sFh2, const float* sWr2, float G32, float Glo,
                                          float* sRow, int nloc, float* colpart_b)
{
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int K2 = 2;
    const int BN = 4 * K2 * T;
    for (int cb = 0; cb < n; cb += BN) {
        float hh[K2][4], wc[K2][4], hh2[K2][4], wc2[K2][4], ca[K2][4];
        int jk[K2];
#pragma unroll
        for (int k = 0; k < K2; ++k) {
            jk[k] = cb + 4 * (tid + k * T);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = jk[k] + e;
                const bool ok = j < n;
                hh[k][e] = ok ? __ldcg(Hh + j) : 0.0f;
                wc[k][e] = ok ? __ldcg(Wc + j) : -INFINITY;
                hh2[k][e] = ok ? __ldcg(Hh2 + j) : 0.0f;
                wc2[k][e] = ok ? __ldcg(Wc2 + j) : -INFINITY;
                ca[k][e] = 0.0f;
            }
        }
        for (int rg = r0; rg < r1; rg += 32) {
            float rp[32];
#pragma unroll
            for (int ii = 0; ii < 32; ++ii) {
                rp[ii] = 0.0f;
                const int i = rg + ii;
                if (i < r1) {
                    const float fh = sFh[i - r0], wr = sWr[i - r0], fh2 = sFh2[i - r0], wr2 = sWr2[i - r0];
                    const float* Crow = C + (size_t)i * (size_t)n;
#pragma unroll
                    for (int k = 0; k < K2; ++k) {
                        float cv[4];
                        if (VEC4) {
                            if (jk[k] < n) {
                                float4 t4 = ldg4(Crow + jk[k]);
                                cv[0] = t4.x; cv[1] = t4.y; cv[2] = t4.z; cv[3] = t4.w;
                            } else {
                                cv[0] = cv[1] = cv[2] = cv[3] = 0.0f;
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e) cv[e] = (jk[k] + e < n) ? __ldg(Crow + jk[k] + e) : 0.0f;
                        }
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float d = (fh + hh[k][e]) - cv[e];
                            rp[ii] += ex2f(fmaf(Glo, d, fmaf(G32, d, wr + wc[k][e])));
                            const float d2 = (fh2 + hh2[k][e]) - cv[e];
                            ca[k][e] += ex2f(fmaf(Glo, d2, fmaf(G32, d2, wr2 + wc2[k][e])));
                        }
                    }
                }
            }
            butterfly<32>(rp, lane);
            const int il = rg + lane;
            if (il < r1) sRow[warp * nloc + (il - r0)] += rp[0];
        }
#pragma unroll
        for (int k = 0; k < K2; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (jk[k] + e < n) colpart_b[jk[k] + e] = ca[k][e];
    }
}

__device__ __forceinline__ void pass2_f64(const float* __restrict__ C, int n, int r0, int r1,
                                          const double* Hd, const double* Bd, const double* sFd,
                                          const double* sAd, double gamma, double* sRow, int nloc,
                                          double* colpart_b)
{
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int K2 = 2;
    const int BN = 4 * K2 * T;
    for (int cb = 0; cb < n; cb += BN) {
        double hd[K2][4], bd[K2][4], ca[K2][4];
        int jk[K2];
#pragma unroll
        for (int k = 0; k < K2; ++k) {
            jk[k] = cb + 4 * (tid + k * T);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = jk[k] + e;
                hd[k][e] = (j < n) ? __ldcg(Hd + j) : -INFINITY;
                bd[k][e] = (j < n) ? __ldcg(Bd + j) : 0.0;
                ca[k][e] = 0.0;
            }
        }
        for (int rg = r0; rg < r1; rg += 16) {
            double rp[16];
#pragma unroll
            for (int ii = 0; ii < 16; ++ii) {
                rp[ii] = 0.0;
                const int i = rg + ii;
                if (i < r1) {
                    const double fd = sFd[i - r0], ad = sAd[i - r0];
                    const float* Crow = C + (size_t)i * (size_t)n;
#pragma unroll
                    for (int k = 0; k < K2; ++k) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int j = jk[k] + e;
                            const double cv = (j < n) ? (double)__ldg(Crow + j) : 0.0;
                            const double z = (fd + hd[k][e]) - gamma * cv;   // u_i + v_j - gamma C_ij
                            rp[ii] += exp(z - ad);
                            ca[k][e] += exp(z - bd[k][e]);
                        }
                    }
                }
            }
            butterfly<16>(rp, lane);
            const int il = rg + (lane & 15);
            if (lane < 16 && il < r1) sRow[warp * nloc + (il - r0)] += rp[0];
        }
#pragma unroll
        for (int k = 0; k < K2; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (jk[k] + e < n) colpart_b[jk[k] + e] = ca[k][e];
    }
}

// Sum of the G column partials of column j (fp32 partials, Kahan per warp, warps combined in
// fp64).  Called by all threads of the CTA for the 32 columns [j0, j0 + 32); the result for
// column j0 + lane is returned in warp 0.  sm: >= 2 * 32 * nwarps floats.
__device__ __forceinline__ double merge_cols_f32(const float* colpart, int n, int G,
                                                 int j0, int j1, float* sm)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int j = j0 + lane;
    float s = 0.0f, comp = 0.0f;
    if (j < j1)
        for (int b = warp; b < G; b += nw) kahan_add(s, comp, __ldcg(colpart + (size_t)b * n + j));
    sm[warp * 32 + lane] = s;
    sm[(nw + warp) * 32 + lane] = -comp;
    __syncthreads();
    double tot = 0.0;
    if (warp == 0)
        for (int w = 0; w < nw; ++w) tot += (double)sm[w * 32 + lane] + (double)sm[(nw + w) * 32 + lane];
    __syncthreads();
    return tot;
}

__device__ __forceinline__ double merge_cols_f64(const double* colpart, int n, int G,
                                                 int j0, int j1, double* sm)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int j = j0 + lane;
    double s = 0.0;
    if (j < j1)
        for (int b = warp; b < G; b += nw) s += __ldcg(colpart + (size_t)b * n + j);
    sm[warp * 32 + lane] = s;
    __syncthreads();
    double tot = 0.0;
    if (warp == 0)
        for (int w = 0; w < nw; ++w) tot += sm[w * 32 + lane];
    __syncthreads();
    return tot;
}

}  // namespace mdot
