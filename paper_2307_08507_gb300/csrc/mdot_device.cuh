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
// the barrier-synchronised stage kernel adds three for the diagonal-Hessian direction (Eq. (16)):
// <y, -s_h>, <s_h, grad g> and the count of ratios r~ / r(P) outside [0.01, 100]
constexpr int kNRedP = 9;
constexpr int kStallIters = 400;               // accepted iterations without 1 % progress end a stage
                                               // (||grad g||_1 is not monotone along PNCG: a last-resort guard)
constexpr int kThreads = 256;                  // CTA size of the cooperative kernels
constexpr int kK = 4;                          // float4 column groups per thread per sweep
constexpr int kRG = 4;                         // rows per group in the passes (keeps the loop body small)

enum Tier { TIER_F32 = 0, TIER_F64 = 1, TIER_F32A = 2 };
// Cost source: a dense row-major matrix, or regenerated from coordinates x_i, y_j (n x 3 each)
// inside the pass: squared Euclidean or L1 distance times a scale s (App. C point clouds; grids
// use z = 0).  Both regenerated forms round every operation in a fixed order, so the value equals
// the one a caller would materialise with the same fp32 operations.
enum CostKind { COST_DENSE = 0, COST_SQEUCLID = 1, COST_L1 = 2 };   // F32A: fp32 with an accurate exponent and exp2
enum EvalKind { KIND_INIT = 0, KIND_TRIAL = 1, KIND_FORCE = 2 };
enum Phase { PH_RUN = 0, PH_DONE = 1 };
enum SolveStatus { ST_OK = 0, ST_CAP = 1, ST_LSFAIL = 2, ST_NUMERIC = 3, ST_TIMEOUT = 4 };

struct GridBar {
    unsigned int count;
    unsigned int gen;
    unsigned int abort;
    unsigned int limit_us;     // limit of every bounded wait in microseconds (0: kBarrierTimeoutNs)
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
    int since_best;        // accepted iterations since ||grad g||_1 last improved by 1 %
    int stalls;            // stages ended by the stall rule (cumulative)
    int hess;              // the direction committed next uses the diagonal-Hessian form (Eq. (16))
    double best_gnorm;     // smallest ||grad g||_1 seen in this stage
    long long evals, evals64, iters, ls_trials;
    GridBar bar;
};

// Noise floor of ||grad g||_1 per entry tier: twice the largest relative error of one entry of P
// (ex2.approx 2^-22.7; the accurate fp32 tier 1.1e-7, measured on 4e6 points per gamma; fp64 the
// 1e-13 resolution floor of the stage tolerance).  The stall rule (a last-resort end of a stage
// that stops improving) is armed only for stages whose tolerance is below 4x this floor; above it
// the stage runs to its tolerance or to max_iter.
__host__ __device__ inline double stall_floor(int tier)
{
    return 4.0 * (tier == TIER_F64 ? 1e-13 : tier == TIER_F32A ? 2.2e-7 : 3.0e-7);
}

struct WS {
    int n, G;
    const float* C;
    const float* X;                   // n x 3 source coordinates (regenerated cost)
    const float* Y;                   // n x 3 target coordinates
    float cscale;                     // s = 1 / max distance
    int ckind;                        // CostKind
    int tc;                           // squared-Euclidean cost of integer points |x_k| <= 255: on the
                                      // tensor cores (pass_f32_regen_tc)
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
    double* blockred;                 // [G][kNRedP]
    double* scratch;                  // [G][8] misc per-CTA values
    State* st;
    // flags of the stage kernel: [2][G] evaluation tags (column partials written; column state
    // published), and the tag base, which grows over the workspace's life
    unsigned int* flags;
    unsigned int* epoch;
    unsigned long long* tsp;          // [G][2 kNRed] tagged per-CTA scalar partials (fp64 halves)
    float4* pub;                      // [n] published column state (see col_publish)
};

struct StageArgs {
    double gamma, G64, tol, w, ratio, c1, c2;
    double stall_below;    // the stall rule applies only when tol < stall_below (see stall_floor)
    int first, warm_start, tier, ls_max_trials, max_iter, Aglob;
    int precond;           // 1: diagonal-Hessian direction (Eq. (16)) where every ratio allows it
    int ls_init;           // 1: first trial step = previous accepted step clamped to [1/2, 2]
};

// Arguments of the standalone dual evaluation (mdot_dual_eval).
struct EvalArgs {
    double gamma, G64;
    const double* u;
    const double* v;
    const double* ref;   // nullable
    // the dual objective g(u, v; gamma, r, c) of Eq. (4) into *g_out (device) when g_out is not
    // null (r, c then given): sum_i r(P)_i - <u, r> - <v, c>, fp64 sums in a fixed order
    const double* r;
    const double* c;
    double* g_out;
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
// Exponent remainder of a padding column (j >= n): large and finite, so that both exponent paths
// (ex2.approx and exp2_acc, whose range reduction would turn -inf into inf - inf) give exactly 0.
constexpr float kPadW = -1.0e30f;

__device__ __forceinline__ float ex2f(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Accurate tier: 2^(G d + W) with G = G32 + Glo (gamma log2 e split in two floats), d the exact
// cost-unit difference and W the row + column remainders.  k = rint(G32 d + W) is taken from one
// rounded fma (1.5 * 2^23 added and subtracted leaves the nearest integer); the reduced argument
// x = (G32 d - k) + W + Glo d is then formed with the product exact inside the fma, so its error is
// a few 2^-25 whatever the size of G d.  2^x on [-1/2, 1/2] by a degree-6 relative-minimax
// polynomial with p(0) = 1 (Remez exchange, csrc/exp2_poly_fit.py: level 1.98e-9; 1.57e-8 with the
// coefficients rounded to fp32 as written here), 2^k by ex2.approx on the
// integer k (exact there; 0 below 2^-126 and inf above 2^127, so no clamping is needed).  Relative
// error ~1 ulp and unbiased, unlike ex2.approx on a general argument, whose error on this GPU
// averages -5e-8.
__device__ __forceinline__ float exp2_acc(float d, float G32, float Glo, float W)
{
    const float th = fmaf(G32, d, W);
    const float t = th + 12582912.0f;
    const float kf = t - 12582912.0f;
    float x = fmaf(G32, d, -kf);
    x = fmaf(Glo, d, x + W);
    float p = 1.53458124e-4f;
    p = fmaf(p, x, 1.33999309e-3f);
    p = fmaf(p, x, 9.61848907e-3f);
    p = fmaf(p, x, 5.55032864e-2f);
    p = fmaf(p, x, 2.40226462e-1f);
    p = fmaf(p, x, 6.93147182e-1f);
    p = fmaf(p, x, 1.0f);
    return p * ex2f(kf);
}

// C_ij regenerated from coordinates: d_k = x_ik - y_jk, D = (d0 d0 + d1 d1) + d2 d2 (or
// (|d0| + |d1|) + |d2|), C = D s, every operation rounded to fp32 in that order (no contraction).
template <int KIND>
__device__ __forceinline__ float point_cost(float x0, float x1, float x2, float y0, float y1, float y2, float s)
{
    const float d0 = __fsub_rn(x0, y0), d1 = __fsub_rn(x1, y1), d2 = __fsub_rn(x2, y2);
    float D;
    if (KIND == COST_SQEUCLID)
        D = __fadd_rn(__fadd_rn(__fmul_rn(d0, d0), __fmul_rn(d1, d1)), __fmul_rn(d2, d2));
    else
        D = __fadd_rn(__fadd_rn(fabsf(d0), fabsf(d1)), fabsf(d2));
    return __fmul_rn(D, s);
}

// Packed fp32 pairs: one instruction computes two entries on this GPU; every component is
// rounded exactly as the scalar operation it stands for (round to nearest), so the packed passes
// give the same bits as the scalar forms above.  Written as PTX with an explicit rounding mode:
// such adds and multiplies are never contracted into an fma by the compiler (the regenerated
// cost must round every product and sum on its own).
__device__ __forceinline__ unsigned long long pk_bits(float2 a)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 unpk_bits(unsigned long long r)
{
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 pk(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b with one rounding: b * (-1) is exact inside the fma
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return fma2(b, make_float2(-1.0f, -1.0f), a); }

// exp2_acc on a pair.  -k = 1.5 * 2^23 - t is exact (t lies within a factor 2 of 1.5 * 2^23), and
// the fma with it rounds as the scalar fmaf(G32, d, -k) does.
__device__ __forceinline__ float2 exp2_acc2(float2 d, float2 G32, float2 Glo, float2 W)
{
    const float2 M = pk(12582912.0f);
    const float2 th = fma2(G32, d, W);
    const float2 t = add2(th, M);
    const float2 nk = sub2(M, t);
    float2 x = fma2(G32, d, nk);
    x = fma2(Glo, d, add2(x, W));
    float2 p = pk(1.53458124e-4f);
    p = fma2(p, x, pk(1.33999309e-3f));
    p = fma2(p, x, pk(9.61848907e-3f));
    p = fma2(p, x, pk(5.55032864e-2f));
    p = fma2(p, x, pk(2.40226462e-1f));
    p = fma2(p, x, pk(6.93147182e-1f));
    p = fma2(p, x, pk(1.0f));
    return mul2(p, make_float2(ex2f(-nk.x), ex2f(-nk.y)));
}

// Two entries of one row: E = 2^(G ((fh + hh) - C) + wr + wc), as the scalar passes compute it.
template <bool ACC>
__device__ __forceinline__ float2 entry2(float2 fh, float2 wr, float2 hh, float2 wc, float2 cv, float2 G32, float2 Glo)
{
    const float2 d = sub2(add2(fh, hh), cv);
    const float2 W = add2(wr, wc);
    if (ACC) return exp2_acc2(d, G32, Glo, W);
    const float2 a = fma2(Glo, d, fma2(G32, d, W));
    return make_float2(ex2f(a.x), ex2f(a.y));
}

// The four entries of one row in a float4 column group: the row sum takes them in column order,
// the column partials ca += E s.
template <bool ACC>
__device__ __forceinline__ void entry4(float fh, float wr, float s, const float2 (&hh)[2], const float2 (&wc)[2],
                                       float2 c01, float2 c23, float2 G32, float2 Glo, float& rp, float2 (&ca)[2])
{
    const float2 FH = pk(fh), WR = pk(wr), S = pk(s);
    const float2 E0 = entry2<ACC>(FH, WR, hh[0], wc[0], c01, G32, Glo);
    const float2 E1 = entry2<ACC>(FH, WR, hh[1], wc[1], c23, G32, Glo);
    rp += E0.x;
    rp += E0.y;
    rp += E1.x;
    rp += E1.y;
    ca[0] = fma2(E0, S, ca[0]);
    ca[1] = fma2(E1, S, ca[1]);
}

// point_cost on a pair of columns (same row).  The code generator fuses a packed multiply into a
// following packed add even when both carry an explicit rounding mode (and turns an fma with a
// constant -0 back into a multiply): measured, 18 % of the regenerated costs then differed from
// the scalar form.  So every product is an fma whose addend z is a -0 the generator cannot see
// (computed at run time by the caller, e.g. -(s * 0)): exact, since adding -0 changes no product,
// and an fma is never fused into the next addition.
template <int KIND>
__device__ __forceinline__ float2 point_cost2(float2 x0, float2 x1, float2 x2, float2 y0, float2 y1, float2 y2,
                                              float2 s, float2 z)
{
    const float2 d0 = sub2(x0, y0), d1 = sub2(x1, y1), d2 = sub2(x2, y2);
    float2 D;
    if (KIND == COST_SQEUCLID)
        D = add2(add2(fma2(d0, d0, z), fma2(d1, d1, z)), fma2(d2, d2, z));
    else
        D = add2(add2(make_float2(fabsf(d0.x), fabsf(d0.y)), make_float2(fabsf(d1.x), fabsf(d1.y))),
                 make_float2(fabsf(d2.x), fabsf(d2.y)));
    return fma2(D, s, z);
}

// column constants of a float4 group as pairs, and the pairs of column partials back to a float4
template <int KK>
__device__ __forceinline__ void to_pairs(const float (&a)[KK][4], float2 (&b)[KK][2])
{
#pragma unroll
    for (int k = 0; k < KK; ++k) {
        b[k][0] = make_float2(a[k][0], a[k][1]);
        b[k][1] = make_float2(a[k][2], a[k][3]);
    }
}
__device__ __forceinline__ void from_pairs(const float2 (&b)[2], float (&a)[4])
{
    a[0] = b[0].x; a[1] = b[0].y; a[2] = b[1].x; a[3] = b[1].y;
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
// v[0] the warp total of value (l mod N).  N a power of two <= 32.  Fixed shuffle tree: deterministic.
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

// Block-wide sum of NR doubles; result valid in thread 0.  red_smem: >= 32 * NR doubles.
// Fixed reduction tree (deterministic); the last step runs on NR lanes in parallel.
template <int NR>
__device__ __forceinline__ void block_reduce_nred(double (&x)[NR], double* red_smem)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NR; ++q)
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) x[q] += __shfl_xor_sync(0xffffffffu, x[q], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NR; ++q) red_smem[warp * NR + q] = x[q];
    __syncthreads();
    if (warp == 0) {
        double s = 0.0;
        if (lane < NR)
            for (int w = 0; w < nw; ++w) s += red_smem[w * NR + lane];
        // move lane q's total into x[q] of thread 0
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            const double t = __shfl_sync(0xffffffffu, s, q);
            if (lane == 0) x[q] = t;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// grid barrier with a bounded wait: a CTA that waits longer than the limit raises `abort`, every
// waiter leaves, and the kernel returns with ST_TIMEOUT instead of hanging.
// ---------------------------------------------------------------------------------------------
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;   // 2 s: default wait limit

__device__ __forceinline__ unsigned long long wait_limit_ns(const GridBar* gb)
{
    // set by the host before the launch and never written by a kernel: a read-only (L1-cached)
    // load, so that starting a wait does not cost a round trip to L2
    const unsigned int us = __ldg(&gb->limit_us);
    return us ? 1000ull * us : kBarrierTimeoutNs;
}

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
        const unsigned long long t0 = globaltimer(), lim = wait_limit_ns(gb);
        unsigned int spins = 0;
        while (true) {
            unsigned int g = ld_acquire(&gb->gen);
            if ((int)(g - target) >= 0) break;
            if (ld_acquire(&gb->abort)) { ok = 0; break; }
            if (++spins > 64u) __nanosleep(64);
            // the clock is read at every poll for the first 64, then every 64th
            if ((spins <= 64u || (spins & 63u) == 0u) && globaltimer() - t0 > lim) {
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

// Tagged 64-bit words: a 32-bit value in the low half and the evaluation's tag in the high half,
// written and read as single 64-bit accesses (each is single-copy atomic), so a reader that sees
// the tag also sees the value: the word is its own ready flag.
__device__ __forceinline__ unsigned long long tag_pack(unsigned int v, unsigned int tag)
{
    return ((unsigned long long)tag << 32) | (unsigned long long)v;
}
__device__ __forceinline__ unsigned int tag_of(unsigned long long w) { return (unsigned int)(w >> 32); }
__device__ __forceinline__ void st_tag(unsigned long long* p, unsigned long long w)
{
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(w) : "memory");
}
__device__ __forceinline__ void ld_tag2(const unsigned long long* p, unsigned long long& a, unsigned long long& b)
{
    asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}

// One step of a bounded wait on flags written by other CTAs: back off, and give up (raising the
// shared abort flag gb->abort) once the wait has lasted longer than the limit (gb->limit_us,
// default kBarrierTimeoutNs) or when another CTA has raised the flag.  deadline = 0 on the first
// call (it is then set from the clock and the limit).  Returns false to give up.
__device__ __forceinline__ bool wait_backoff(unsigned int& spins, unsigned long long& deadline, GridBar* gb)
{
    ++spins;
    // poll without sleeping at first: a flag poll is a handful of loads by one warp, and the
    // sleep's granularity would add to every hand-off
    if (spins > 4096u) __nanosleep(64);
    // the clock is read at every poll for the first 64 (a register read), then with the abort
    // flag (a load from L2) at every 64th
    const bool every64 = (spins & 63u) == 0u;
    if (spins <= 64u || every64) {
        if (every64 && ld_acquire(&gb->abort)) return false;
        const unsigned long long now = globaltimer();
        if (deadline == 0ull) {
            deadline = now + wait_limit_ns(gb);
        } else if (now > deadline) {
            atomicExch(&gb->abort, 1u);
            return false;
        }
    }
    return true;
}

// Column constants and column partials of one pass over C (plain arrays; a grid barrier or the
// stage kernel's flags order them).  Other sources (e.g. constants computed in place) supply the
// same calls: load_seg (the constants of all of a thread's column groups of a segment at once, so
// every load is in flight before any arithmetic) and store4.
struct ColPlain {
    const float* Hh;
    const float* Wc;
    float* out;                       // this CTA's row of column partials
    __device__ __forceinline__ bool load4(int j0, int n, float hh[4], float wc[4]) const
    {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = j0 + e;
            const bool ok = j < n;
            // per-trial constants are rewritten inside the launch: read through L2, never the
            // non-coherent path
            hh[e] = ok ? __ldcg(Hh + j) : 0.0f;
            wc[e] = ok ? __ldcg(Wc + j) : kPadW;     // padding column: its entry is exactly 0
        }
        return true;
    }
    template <int KK>
    __device__ __forceinline__ bool load_seg(const int (&jk)[KK], int n, float (&hh)[KK][4], float (&wc)[KK][4]) const
    {
#pragma unroll
        for (int k = 0; k < KK; ++k) load4(jk[k], n, hh[k], wc[k]);
        return true;
    }
    __device__ __forceinline__ void store4(int j0, int n, const float ca[4]) const
    {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (j0 + e < n) out[j0 + e] = ca[e];
    }
    // the constants of column j (tensor-core pass, staged in shared memory) and the partials of
    // columns j0, j0 + 1
    __device__ __forceinline__ void load1(int j, int n, float& hh, float& wc) const
    {
        hh = (j < n) ? __ldcg(Hh + j) : 0.0f;
        wc = (j < n) ? __ldcg(Wc + j) : kPadW;
    }
    __device__ __forceinline__ void store2(int j0, int n, float2 ca) const
    {
        if (j0 < n) out[j0] = ca.x;
        if (j0 + 1 < n) out[j0 + 1] = ca.y;
    }
};


// ---------------------------------------------------------------------------------------------
// Double-float arithmetic (a value as an unevaluated sum hi + lo of two floats, ~48 bits): Knuth's
// TwoSum, the fast variant for |a| >= |b|, and products through the fma's exact error term.
// Every operation is an explicitly rounded intrinsic, so no contraction can change the results.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return make_float2(s, e);
}
__device__ __forceinline__ float2 df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b)
{
    const float2 s = df_two_sum(a.x, b.x);
    return df_fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(a.y, b.y)));
}
// a * b for a double-float a and a float b
__device__ __forceinline__ float2 df_mul_f(float2 a, float b)
{
    const float p = __fmul_rn(a.x, b);
    const float e = __fmaf_rn(a.y, b, __fmaf_rn(a.x, b, -p));
    return df_fast_two_sum(p, e);
}
// a * b for double-floats a and b
__device__ __forceinline__ float2 df_mul(float2 a, float2 b)
{
    const float p = __fmul_rn(a.x, b.x);
    const float e = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, __fmaf_rn(a.x, b.x, -p)));
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ float2 df_from_double(double x)
{
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}
__device__ __forceinline__ double df_to_double(float2 a) { return (double)a.x + (double)a.y; }
// a + b for a double-float a and a float b (TwoSum, then renormalise)
__device__ __forceinline__ float2 df_add_f(float2 a, float b)
{
    const float2 s = df_two_sum(a.x, b);
    return df_fast_two_sum(s.x, __fadd_rn(s.y, a.y));
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
// a * 2^e for a double-float a and -126 <= e <= 127 (exact unless a component leaves the normal
// range)
__device__ __forceinline__ float2 df_ldexp(float2 a, int e)
{
    const float m = __int_as_float((e + 127) << 23);
    return make_float2(__fmul_rn(a.x, m), __fmul_rn(a.y, m));
}
__device__ __forceinline__ float2 df_shfl_xor(float2 a, int o)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
}

// Decision of one evaluation as every thread of the stage kernel sees it: commit (v += alpha_c p,
// p = s + beta p) when accepted, then the trial point v + alpha p.  Steps are fp32 numbers (the
// line search rounds them), so the same arithmetic on the same inputs gives the same bits in
// every CTA.
struct ColStep {
    int accept;
    float alpha_c, beta, alpha;
};

// Commit of one column's (v, p) (double-floats) for a decision.
__device__ __forceinline__ void col_commit(const ColStep& d, float2& v, float2& p, float s)
{
    if (d.accept) {
        v = df_add(v, df_mul_f(p, d.alpha_c));                 // (u, v) += alpha p (Alg. 2)
        p = df_add(df_mul_f(p, d.beta), make_float2(s, 0.0f));  // p = s + beta p (Alg. 2, Eq. (18))
    }
}

// Published state of one column for the next pass, computed by the column's owner from its
// committed v, p (double-floats) and the new direction s:
//   x = v / gamma in cost units, split into a part quantised to 2^-21 (hb, exact in fp32 while
//   |x| < 8) and the remainder in exponent units (rb = gamma log2 e (x - hb));
//   P = log2 e p and S = log2 e s, the directions in exponent units (gamma log2 e / gamma = log2 e).
// Any trial point of the next pass, v + k1 p + k2 s, then has the column constants
//   hh = hb,  wc = rb + k1 P + k2 S,
// two fmas per column and consumer (see ColDelta).  The step terms carry the fp32 rounding of
// k1 P + k2 S (relative 2^-24 of a term that is small near convergence); the committed (v, p)
// stay exact double-floats in the owner.
__device__ __forceinline__ float4 col_publish(float2 v, float2 p, float s, float2 inv_gamma, float G32, float Glo)
{
    const float2 x = df_mul(v, inv_gamma);
    const float h = __fmul_rn(rintf(__fmul_rn(x.x, 2097152.0f)), 1.0f / 2097152.0f);
    const float lo = __fadd_rn(__fsub_rn(x.x, h), x.y);       // x.x - h is exact
    const float rb = __fmaf_rn(lo, G32, __fmul_rn(lo, Glo));
    return make_float4(h, rb, (float)(kLog2e * df_to_double(p)), (float)(kLog2e * (double)s));
}

// The (k1, k2) of the next trial point v + k1 p + k2 s for a decision: after an accepted step the
// owner commits v <- v + alpha_c p, p <- s + beta p, and the trial is v + alpha p of those, i.e.
// k1 = alpha_c + alpha beta, k2 = alpha; otherwise the trial is v + alpha p (k1 = alpha, k2 = 0).
__device__ __forceinline__ float2 col_step_coeffs(const ColStep& d)
{
    return d.accept ? make_float2(__fmaf_rn(d.alpha, d.beta, d.alpha_c), d.alpha) : make_float2(d.alpha, 0.0f);
}

// Column constants of a pass derived in place by every consumer thread from the owners'
// published state (col_publish) and the decision: no hand-off of constants between CTAs.
// Partials go to plain arrays.
struct ColDelta {
    const float4* pub;
    float* out;
    float k1, k2;
    // the published state of a thread's column groups: it does not depend on the decision, so the
    // stage kernel loads it while the decision is being taken (load_pub), then derives (derive)
    template <int KK>
    __device__ __forceinline__ void load_pub(const int (&jk)[KK], int n, float4 (&q)[KK][4]) const
    {
#pragma unroll
        for (int k = 0; k < KK; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = jk[k] + e;
                q[k][e] = (j < n) ? __ldcg(pub + j) : make_float4(0.0f, kPadW, 0.0f, 0.0f);
            }
    }
    template <int KK>
    __device__ __forceinline__ void derive(const float4 (&q)[KK][4], const int (&jk)[KK], int n, float (&hh)[KK][4],
                                           float (&wc)[KK][4]) const
    {
#pragma unroll
        for (int k = 0; k < KK; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                hh[k][e] = q[k][e].x;
                wc[k][e] = (jk[k] + e < n) ? __fmaf_rn(k1, q[k][e].z, __fmaf_rn(k2, q[k][e].w, q[k][e].y)) : kPadW;
            }
    }
    template <int KK>
    __device__ __forceinline__ bool load_seg(const int (&jk)[KK], int n, float (&hh)[KK][4], float (&wc)[KK][4]) const
    {
        float4 q[KK][4];
        load_pub(jk, n, q);
        derive(q, jk, n, hh, wc);
        return true;
    }
    __device__ __forceinline__ void store4(int j0, int n, const float ca[4]) const
    {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (j0 + e < n) out[j0 + e] = ca[e];
    }
    __device__ __forceinline__ void load1(int j, int n, float& hh, float& wc) const
    {
        const float4 q = (j < n) ? __ldcg(pub + j) : make_float4(0.0f, kPadW, 0.0f, 0.0f);
        hh = q.x;
        wc = (j < n) ? __fmaf_rn(k1, q.z, __fmaf_rn(k2, q.w, q.y)) : kPadW;
    }
    __device__ __forceinline__ void store2(int j0, int n, float2 ca) const
    {
        if (j0 < n) out[j0] = ca.x;
        if (j0 + 1 < n) out[j0 + 1] = ca.y;
    }
};

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
// Column partials over many rows: a thread's fp32 chain of E_ij s_i over the rows of its CTA is
// folded every kFoldRows rows into a compensated (TwoSum) pair, so that a long chain (up to 4096
// rows in the batched form) adds ~1 ulp of error instead of ~sqrt(rows) ulp; the result is
// rounded to fp32 once.  (The spread such sums leave in the marginals sets the smallest
// ||grad g||_1 fp32 entries can resolve.)
// ---------------------------------------------------------------------------------------------
constexpr int kFoldRows = 16;

__device__ __forceinline__ void fold1(float& hi, float& lo, float& ca)
{
    const float s = __fadd_rn(hi, ca);
    const float bb = __fsub_rn(s, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(ca, bb)));
    hi = s;
    ca = 0.0f;
}
__device__ __forceinline__ void fold2(float2& hi, float2& lo, float2& ca)
{
    fold1(hi.x, lo.x, ca.x);
    fold1(hi.y, lo.y, ca.y);
}
// the folded total (the open chain included), rounded once
__device__ __forceinline__ float2 fold_total(float2 hi, float2 lo, float2 ca)
{
    fold2(hi, lo, ca);
    return make_float2(__fadd_rn(hi.x, lo.x), __fadd_rn(hi.y, lo.y));
}

// ---------------------------------------------------------------------------------------------
// Phase A: one pass over the rows [r0, r1) of C.  Row sums go to sRow[warp][local row]
// (accumulated, fp32 or fp64), column partials to colpart_b[j].
// ---------------------------------------------------------------------------------------------
template <bool VEC4, bool ACC, class IO>
__device__ __forceinline__ void pass_f32(const float* __restrict__ C, int n, int r0, int r1, const IO& io,
                                         const float* sFh, const float* sWr, const float* sS,
                                         float G32, float Glo, float* sRow, int nloc)
{
    const float2 G32p = pk(G32), Glop = pk(Glo);
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int BN = 4 * kK * T;
    for (int cb = 0; cb < n; cb += BN) {
        float hh[kK][4], wc[kK][4];
        float2 hh2[kK][2], wc2[kK][2], ca2[kK][2], fh2[kK][2], fl2[kK][2];
        int jk[kK];
#pragma unroll
        for (int k = 0; k < kK; ++k) {
            jk[k] = cb + 4 * (tid + k * T);
            ca2[k][0] = ca2[k][1] = fh2[k][0] = fh2[k][1] = fl2[k][0] = fl2[k][1] = make_float2(0.0f, 0.0f);
        }
        io.load_seg(jk, n, hh, wc);
        to_pairs(hh, hh2);
        to_pairs(wc, wc2);
        for (int rg = r0; rg < r1; rg += kRG) {
            float rp[kRG];
#pragma unroll
            for (int ii = 0; ii < kRG; ++ii) {
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
                        entry4<ACC>(fh, wr, s, hh2[k], wc2[k], make_float2(cv[0], cv[1]), make_float2(cv[2], cv[3]),
                                    G32p, Glop, rp[ii], ca2[k]);
                    }
                }
            }
            butterfly<kRG>(rp, lane);
            const int il = rg + lane;
            if (lane < kRG && il < r1) sRow[warp * nloc + (il - r0)] += rp[0];
            if (((rg - r0 + kRG) % kFoldRows) == 0) {
#pragma unroll
                for (int k = 0; k < kK; ++k) {
                    fold2(fh2[k][0], fl2[k][0], ca2[k][0]);
                    fold2(fh2[k][1], fl2[k][1], ca2[k][1]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kK; ++k) {
            float2 tot[2] = {fold_total(fh2[k][0], fl2[k][0], ca2[k][0]), fold_total(fh2[k][1], fl2[k][1], ca2[k][1])};
            float ca[4];
            from_pairs(tot, ca);
            io.store4(jk[k], n, ca);
        }
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
        for (int rg = r0; rg < r1; rg += kRG) {
            double rp[kRG];
#pragma unroll
            for (int ii = 0; ii < kRG; ++ii) {
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
            butterfly<kRG>(rp, lane);
            const int il = rg + lane;
            if (lane < kRG && il < r1) sRow[warp * nloc + (il - r0)] += rp[0];
        }
#pragma unroll
        for (int k = 0; k < kK; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (jk[k] + e < n) colpart_b[jk[k] + e] = ca[k][e];
    }
}

// ---------------------------------------------------------------------------------------------
// TMA-fed pass (fp32 entries): one producer warp streams row segments C[i, cb : cb + 4096) into a
// ring of kStages shared-memory slots with cp.async.bulk (completion counted on a per-slot "full"
// mbarrier); the 8 consumer warps read each slot with 128-bit shared loads and release it on a
// per-slot "empty" mbarrier.  Every wait is bounded; a wait that gives up sets *abort and the
// pass drains what it issued (bounded as well) before returning.
// ---------------------------------------------------------------------------------------------
constexpr int kConsumerThreads = 256;
constexpr int kStageThreads = kConsumerThreads + 32;    // + one producer warp
constexpr int kStages = 12;                            // ring slots at most (fewer if smem is short)
constexpr size_t kSmemLimit = 223 * 1024;      // dynamic shared memory of a CTA (227 KB less room
                                                // for the kernels' static shared memory)
constexpr int kSegFloats = 4 * kK * kConsumerThreads;   // 4096 floats = 16 KiB per slot
constexpr unsigned int kWaitSpins = 1u << 24;           // bounded mbarrier wait (with backoff)

__device__ __forceinline__ unsigned int smem_u32(const void* p)
{
    return (unsigned int)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned int bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned int parity)
{
    unsigned int ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned int parity)
{
    for (unsigned int it = 0; it < kWaitSpins; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 32) __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void tma_load_1d(void* dst_smem, const void* src_gmem, unsigned int bytes,
                                            unsigned long long* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst_smem)), "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// Requires n % 4 == 0 and C 16-byte aligned.  ring: kStages * kSegFloats floats (16-byte aligned);
// bars: 2 * kStages mbarriers (full, empty).  Block = kStageThreads threads.
template <bool ACC, class IO>
__device__ __forceinline__ void pass_f32_tma(const float* __restrict__ C, int n, int r0, int r1, const IO& io,
                                             const float* sFh, const float* sWr, const float* sS, float G32,
                                             float Glo, float* sRow, int nloc, float* ring, int nst,
                                             unsigned long long* bars, int* s_issued, unsigned int* abort)
{
    const float2 G32p = pk(G32), Glop = pk(Glo);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nrows = r1 - r0;
    const int ncb = (n + kSegFloats - 1) / kSegFloats;
    const int items = nrows * ncb;
    unsigned long long* full = bars;
    unsigned long long* empty = bars + kStages;
    if (tid == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerThreads / 32);
        }
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == kConsumerThreads / 32) {
        // ------------------------------ producer warp ------------------------------
        if (lane == 0) {
            bool ok = true;
            int q = 0, s = 0, ph = 0, cbi = 0, il = 0;       // slot, parity of its current use, item
            for (; q < items && ok; ++q) {
                if (q >= nst) ok = mbar_wait(&empty[s], ph ^ 1);
                if (!ok) break;
                const int i = r0 + il;
                const int cb = cbi * kSegFloats;
                const unsigned int bytes = (unsigned int)(min(kSegFloats, n - cb) * 4);
                mbar_arrive_expect_tx(&full[s], bytes);
                tma_load_1d(ring + (size_t)s * kSegFloats, C + (size_t)i * n + cb, bytes, &full[s]);
                if (++s == nst) { s = 0; ph ^= 1; }
                if (++il == nrows) { il = 0; ++cbi; }
            }
            *s_issued = q;
            if (!ok) atomicExch(abort, 1u);
        }
        __syncwarp();
    } else {
        // ------------------------------ consumer warps ------------------------------
        int q = 0, sl = 0, ph = 0;
        bool ok = true;
        for (int cbi = 0; cbi < ncb; ++cbi) {
            const int cb = cbi * kSegFloats;
            float hh[kK][4], wc[kK][4];
            float2 hh2[kK][2], wc2[kK][2], ca2[kK][2];
            int jk[kK];
#pragma unroll
            for (int k = 0; k < kK; ++k) {
                jk[k] = cb + 4 * (tid + k * kConsumerThreads);
                ca2[k][0] = ca2[k][1] = make_float2(0.0f, 0.0f);
            }
            // a constant that never arrives (timeout) turns this consumer into a pass-through: it
            // still releases every ring slot so that the producer can finish
            if (!io.load_seg(jk, n, hh, wc)) ok = false;
            to_pairs(hh, hh2);
            to_pairs(wc, wc2);
            for (int rg = r0; rg < r1; rg += kRG) {
                float rp[kRG];
#pragma unroll
                for (int ii = 0; ii < kRG; ++ii) {
                    rp[ii] = 0.0f;
                    const int i = rg + ii;
                    if (i < r1) {
                        const int s = sl;
                        if (ok) ok = mbar_wait(&full[s], ph);
                        const float fh = sFh[i - r0], wr = sWr[i - r0], sc = sS[i - r0];
                        const float4* seg = reinterpret_cast<const float4*>(ring + (size_t)s * kSegFloats);
#pragma unroll
                        for (int k = 0; k < kK; ++k) {
                            float cv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                            if (ok && jk[k] < n) {
                                const float4 t4 = seg[tid + k * kConsumerThreads];
                                cv[0] = t4.x; cv[1] = t4.y; cv[2] = t4.z; cv[3] = t4.w;
                            }
                            entry4<ACC>(fh, wr, sc, hh2[k], wc2[k], make_float2(cv[0], cv[1]), make_float2(cv[2], cv[3]),
                                        G32p, Glop, rp[ii], ca2[k]);
                        }
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&empty[s]);
                        ++q;
                        if (++sl == nst) { sl = 0; ph ^= 1; }
                    }
                }
                butterfly<kRG>(rp, lane);
                const int il = rg + lane;
                if (lane < kRG && il < r1) sRow[warp * nloc + (il - r0)] += rp[0];
            }
#pragma unroll
            for (int k = 0; k < kK; ++k) {
                float ca[4];
                from_pairs(ca2[k], ca);
                io.store4(jk[k], n, ca);
            }
        }
        if (!ok && lane == 0) atomicExch(abort, 1u);
    }
    __syncthreads();
    if (tid == 0 && *reinterpret_cast<volatile unsigned int*>(abort)) {
        // a wait gave up: let every copy that may still be in flight land (bounded) before the
        // shared memory is reused or the CTA exits
        const int issued = *s_issued;
        for (int q = max(0, issued - nst); q < issued; ++q) mbar_wait(&full[q % nst], (q / nst) & 1);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------------------
// TMA ring that persists over the passes of one launch (stage kernel): C does not change within a
// stage, so the producer never stops: while the CTA is in its epilogue and hand-offs it already
// holds the first rows of the next pass.  Items are numbered over all passes; item Q is row
// (Q mod items) % nrows, segment (Q mod items) / nrows, in slot Q % nst with parity (Q / nst) & 1.
// ---------------------------------------------------------------------------------------------
struct RingGeom {
    const float* C;
    int n, r0, nrows, ncb, nst;
    float* ring;
    unsigned long long* full;     // [kStages]
    unsigned long long* empty;    // [kStages]
    __device__ __forceinline__ int items() const { return nrows * ncb; }
};

// CONS: consumer threads (the producer is the next warp)
template <int CONS>
__device__ __forceinline__ void ring_init(const RingGeom& g)
{
    if (threadIdx.x == 0) {
        for (int s = 0; s < g.nst; ++s) {
            mbar_init(&g.full[s], 1);
            mbar_init(&g.empty[s], CONS / 32);
        }
        mbar_fence_init();
    }
}

// Producer thread: issue items up to (not including) `upto`; false if a slot never came free.
// (Slot, parity, row and segment advance incrementally: no integer division per item.)
__device__ __forceinline__ bool ring_issue(const RingGeom& g, int& issued, int upto)
{
    const int items = g.items();
    if (items == 0 || issued >= upto) return true;
    int s = issued % g.nst, ph = (issued / g.nst) & 1;
    const int loc = issued % items;
    int il = loc % g.nrows, cbi = loc / g.nrows;
    for (; issued < upto; ++issued) {
        if (issued >= g.nst && !mbar_wait(&g.empty[s], ph ^ 1)) return false;
        const int cb = cbi * kSegFloats;
        const unsigned int bytes = (unsigned int)(min(kSegFloats, g.n - cb) * 4);
        mbar_arrive_expect_tx(&g.full[s], bytes);
        tma_load_1d(g.ring + (size_t)s * kSegFloats, g.C + (size_t)(g.r0 + il) * g.n + cb, bytes, &g.full[s]);
        if (++s == g.nst) { s = 0; ph ^= 1; }
        if (++il == g.nrows) {
            il = 0;
            if (++cbi == g.ncb) cbi = 0;
        }
    }
    return true;
}

// Before the CTA exits: every issued copy lands (bounded) so that none writes shared memory late.
__device__ __forceinline__ void ring_drain(const RingGeom& g, int consumed, int issued)
{
    for (int Q = max(consumed, issued - g.nst); Q < issued; ++Q) mbar_wait(&g.full[Q % g.nst], (Q / g.nst) & 1);
}

// One row of a ring slot for this thread's column groups: the row sum (column order) and the
// column partials.
template <bool ACC, int KK, int CONS>
__device__ __forceinline__ float ring_row(const float4* seg, bool ok, const int (&jk)[KK], int n, int tid, float fh,
                                          float wr, float sc, const float2 (&hh2)[KK][2], const float2 (&wc2)[KK][2],
                                          float2 G32p, float2 Glop, float2 (&ca2)[KK][2])
{
    float rp = 0.0f;
#pragma unroll
    for (int k = 0; k < KK; ++k) {
        float4 t4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (ok && jk[k] < n) t4 = seg[tid + k * CONS];
        entry4<ACC>(fh, wr, sc, hh2[k], wc2[k], make_float2(t4.x, t4.y), make_float2(t4.z, t4.w), G32p, Glop, rp,
                    ca2[k]);
    }
    return rp;
}

// One pass over the CTA's rows through the persistent ring (same arithmetic as pass_f32_tma).
// consumed: items consumed before this pass (identical in every thread); issued: the producer
// thread's count.  Both advance here.
// sPub (nullable): the published column state of segment 0 being copied into shared memory (float4
// per column, in column order) by a bulk copy that completes on pub_bar with parity pub_parity.
// CONS consumer threads (kSegFloats / (4 CONS) float4 column groups each per segment), the producer
// warp after them.
template <bool ACC, int CONS, class IO>
__device__ __forceinline__ void pass_f32_ring(const RingGeom& g, int r1, const IO& io, const float4* sPub,
                                              unsigned long long* pub_bar, unsigned int pub_parity,
                                              const float* sFh, const float* sWr,
                                              const float* sS, float G32, float Glo, float* sRow, int nloc,
                                              int& consumed, int& issued, unsigned int* abort)
{
    constexpr int KK = kSegFloats / (4 * CONS);
    static_assert(KK * 4 * CONS == kSegFloats, "a segment splits evenly over the consumer threads");
    const float2 G32p = pk(G32), Glop = pk(Glo);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = g.n, r0 = g.r0, items = g.items();
    if (warp == CONS / 32) {
        // ------------------------------ producer warp ------------------------------
        if (lane == 0 && !ring_issue(g, issued, consumed + items + g.nst)) atomicExch(abort, 1u);
        __syncwarp();
    } else {
        // ------------------------------ consumer warps ------------------------------
        int sl = consumed % g.nst, ph = (consumed / g.nst) & 1;   // slot and parity of the next item
        bool ok = true;
        for (int cbi = 0; cbi < g.ncb; ++cbi) {
            const int cb = cbi * kSegFloats;
            float hh[KK][4], wc[KK][4];
            float2 hh2[KK][2], wc2[KK][2], ca2[KK][2];
            int jk[KK];
#pragma unroll
            for (int k = 0; k < KK; ++k) {
                jk[k] = cb + 4 * (tid + k * CONS);
                ca2[k][0] = ca2[k][1] = make_float2(0.0f, 0.0f);
            }
            if (sPub != nullptr && cbi == 0) {
                if (ok) ok = mbar_wait(pub_bar, pub_parity);
                float4 q[KK][4];
#pragma unroll
                for (int k = 0; k < KK; ++k)
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        q[k][e] = (jk[k] + e < n) ? sPub[jk[k] + e] : make_float4(0.0f, kPadW, 0.0f, 0.0f);
                io.derive(q, jk, n, hh, wc);
            } else {
                io.load_seg(jk, n, hh, wc);
            }
            to_pairs(hh, hh2);
            to_pairs(wc, wc2);
            for (int rg = r0; rg < r1; rg += kRG) {
                float rp[kRG];
#pragma unroll
                for (int ii = 0; ii < kRG; ii += 2) {
                    rp[ii] = 0.0f;
                    rp[ii + 1] = 0.0f;
                    const int i = rg + ii;
                    if (i < r1) {
                        // two rows (ring slots) at a time when both exist: their entries are
                        // independent, so the two instruction streams interleave; each row's sum
                        // and the column partials keep their order
                        const bool two = i + 1 < r1;
                        const int sA = sl, pA = ph;
                        if (++sl == g.nst) { sl = 0; ph ^= 1; }
                        const int sB = sl, pB = ph;
                        if (two && ++sl == g.nst) { sl = 0; ph ^= 1; }
                        if (ok) ok = mbar_wait(&g.full[sA], pA);
                        if (two && ok) ok = mbar_wait(&g.full[sB], pB);
                        const float4* segA = reinterpret_cast<const float4*>(g.ring + (size_t)sA * kSegFloats);
                        rp[ii] = ring_row<ACC, KK, CONS>(segA, ok, jk, n, tid, sFh[i - r0], sWr[i - r0], sS[i - r0], hh2, wc2,
                                               G32p, Glop, ca2);
                        if (two) {
                            const float4* segB = reinterpret_cast<const float4*>(g.ring + (size_t)sB * kSegFloats);
                            rp[ii + 1] = ring_row<ACC, KK, CONS>(segB, ok, jk, n, tid, sFh[i + 1 - r0], sWr[i + 1 - r0],
                                                       sS[i + 1 - r0], hh2, wc2, G32p, Glop, ca2);
                        }
                        __syncwarp();
                        if (lane == 0) {
                            mbar_arrive(&g.empty[sA]);
                            if (two) mbar_arrive(&g.empty[sB]);
                        }
                    }
                }
                butterfly<kRG>(rp, lane);
                const int il = rg + lane;
                if (lane < kRG && il < r1) sRow[warp * nloc + (il - r0)] += rp[0];
            }
#pragma unroll
            for (int k = 0; k < KK; ++k) {
                float ca[4];
                from_pairs(ca2[k], ca);
                io.store4(jk[k], n, ca);
            }
        }
        if (!ok && lane == 0) atomicExch(abort, 1u);
    }
    consumed += items;
    __syncthreads();
}

// One row of the regenerated-cost pass for this thread's column groups: the row sum (column order)
// and the column partials.
template <bool ACC, int KIND, int KR>
__device__ __forceinline__ float regen_row(const float* sX, int il, const float* sFh, const float* sWr,
                                           const float* sS, const float2 (&y0)[KR][2], const float2 (&y1)[KR][2],
                                           const float2 (&y2)[KR][2], const float2 (&hh2)[KR][2],
                                           const float2 (&wc2)[KR][2], float2 CS, float2 Z, float2 G32p, float2 Glop,
                                           float2 (&ca2)[KR][2])
{
    const float fh = sFh[il], wr = sWr[il], sc = sS[il];
    const float2 x0 = pk(sX[3 * il]), x1 = pk(sX[3 * il + 1]), x2 = pk(sX[3 * il + 2]);
    float rp = 0.0f;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
        const float2 c01 = point_cost2<KIND>(x0, x1, x2, y0[k][0], y1[k][0], y2[k][0], CS, Z);
        const float2 c23 = point_cost2<KIND>(x0, x1, x2, y0[k][1], y1[k][1], y2[k][1], CS, Z);
        entry4<ACC>(fh, wr, sc, hh2[k], wc2[k], c01, c23, G32p, Glop, rp, ca2[k]);
    }
    return rp;
}

// Pass over the CTA's rows with C regenerated from coordinates (no C in memory): same structure
// as pass_f32 with two float4 column groups per thread; the row coordinates come from shared
// memory (sX: 3 floats per local row), the column coordinates sit in registers per sweep.
// ---------------------------------------------------------------------------------------------
// Squared-Euclidean cost between integer grid points on the tensor cores.  For points with integer
// coordinates |x_k| <= 255, D_ij = |x_i|^2 + |y_j|^2 - 2 <x_i, y_j> is one contraction of length
// 9 of bf16 vectors that hold every value exactly:
//   A_i = [x0, x1, x2, a2, a1, a0, 1, 1, 1, 0 ...]   (a2 a1 a0: base-256 digits of |x_i|^2)
//   B_j = [-2y0, -2y1, -2y2, 2^16, 2^8, 1, b2 2^16, b1 2^8, b0, 0 ...]
// Every product is an integer below 2^18 and every partial sum an integer below 2^20, so the fp32
// accumulation of the tensor cores is exact: D is the exact integer, and C = fl32(D s) has the bits
// of the fp32 cost (d0 d0 + d1 d1) + d2 d2 times s that the FMA pass and the host generator form.
// (A contraction of length 9 uses a tiny share of the tensor pipe: what it removes is the ALU work
// of the cost, about half of the fp32 operations of an entry.)
// ---------------------------------------------------------------------------------------------
// two floats (exact in bf16) as one bf16x2 register; `lo` in the low half (the smaller k)
__device__ __forceinline__ unsigned int bf16x2(float lo, float hi)
{
    unsigned int d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// D = A B (m16n8k16, bf16 inputs, fp32 accumulation from zero).  Fragments as the PTX ISA lays
// them out: lane = 4 g + t; a0/a1: rows g / g + 8, k = 2t, 2t + 1; a2/a3: the same rows,
// k = 8 + 2t, 9 + 2t; b0/b1: column g, k = 2t, 2t + 1 / 8 + 2t, 9 + 2t; d0, d1: row g, columns
// 2t, 2t + 1; d2, d3: row g + 8, the same columns.
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], unsigned int a0, unsigned int a1, unsigned int a2,
                                               unsigned int a3, unsigned int b0, unsigned int b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%10, %10, %10, %10};"
                 : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(0.0f));
}

// |x|^2 of an integer point, as its base-256 digits (d2, d1, d0)
__device__ __forceinline__ void sq_digits(float x0, float x1, float x2, float& d2, float& d1, float& d0)
{
    const int s = (int)x0 * (int)x0 + (int)x1 * (int)x1 + (int)x2 * (int)x2;
    d2 = (float)(s >> 16);
    d1 = (float)((s >> 8) & 255);
    d0 = (float)(s & 255);
}

// This lane's two A registers (k = 2t, 2t + 1 and k = 8 + 2t, 9 + 2t) of a row point.
__device__ __forceinline__ void tc_a_regs(float x0, float x1, float x2, int t, unsigned int& klo, unsigned int& khi)
{
    float d2, d1, d0;
    sq_digits(x0, x1, x2, d2, d1, d0);
    const float e0 = t == 0 ? x0 : t == 1 ? x2 : t == 2 ? d1 : 1.0f;
    const float e1 = t == 0 ? x1 : t == 1 ? d2 : t == 2 ? d0 : 1.0f;
    klo = bf16x2(e0, e1);
    khi = t == 0 ? bf16x2(1.0f, 0.0f) : 0u;
}

// This lane's two B registers of a column point.
__device__ __forceinline__ void tc_b_regs(float y0, float y1, float y2, int t, unsigned int& b0, unsigned int& b1)
{
    float d2, d1, d0;
    sq_digits(y0, y1, y2, d2, d1, d0);
    const float e0 = t == 0 ? -2.0f * y0 : t == 1 ? -2.0f * y2 : t == 2 ? 256.0f : d2 * 65536.0f;
    const float e1 = t == 0 ? -2.0f * y1 : t == 1 ? 65536.0f : t == 2 ? 1.0f : d1 * 256.0f;
    b0 = bf16x2(e0, e1);
    b1 = t == 0 ? bf16x2(d0, 0.0f) : 0u;
}

// Pass over the CTA's rows with the squared-Euclidean cost of integer grid points formed on the
// tensor cores (see above); same outputs as pass_f32_regen.  The columns go in blocks of
// kTcSubs x 32 columns per warp: the CTA first stages a block's column constants and coordinates in
// shared memory (stage: kTcStageFloats per column, tc_stage_floats(warps) floats), then every warp
// takes kTcSubs sub-blocks of 32 columns and sweeps the CTA's rows in tiles of 16: per tile four
// mma.sync give the costs, every lane forms its 2 rows x 8 columns of entries (the exponent and the
// sums as in entry2), the row partials are added over the 4 lanes of a row, and the column
// partials, folded every kFoldRows rows (fold2), over the 8 row groups at the end of the sweep.
constexpr int kTcSubs = 16;            // 32-column sub-blocks per warp and column block
constexpr int kTcStageFloats = 5;      // hh, wc, y0, y1, y2 per staged column
__host__ __device__ constexpr int tc_block_cols(int warps) { return warps * kTcSubs * 32; }
__host__ __device__ constexpr int tc_stage_floats(int warps) { return kTcStageFloats * tc_block_cols(warps); }

// One 16-row tile of a tensor-core sweep for this lane: the costs of its rows g, g + 8 and its
// 2 NT columns, the entries, the row partials (added into rp0 / rp1) and the column partials.
template <bool ACC, int NT>
__device__ __forceinline__ void tc_tile(unsigned int a0, unsigned int a1, unsigned int a2, unsigned int a3,
                                        const unsigned int (&b0)[NT], const unsigned int (&b1)[NT],
                                        float fh0, float wr0, float s0, float fh1, float wr1, float s1,
                                        const float2 (&hh2)[NT], const float2 (&wc2)[NT], float2 CS, float2 Z,
                                        float2 G32p, float2 Glop, float& rp0, float& rp1, float2 (&ca2)[NT])
{
    const float2 FH0 = pk(fh0), WR0 = pk(wr0), S0 = pk(s0), FH1 = pk(fh1), WR1 = pk(wr1), S1 = pk(s1);
#pragma unroll
    for (int q = 0; q < NT; ++q) {
        float d[4];
        mma_bf16_16816(d, a0, a1, a2, a3, b0[q], b1[q]);
        // C = fl32(D s): an fma with a -0 addend the generator cannot fold (see point_cost2)
        const float2 c0 = fma2(make_float2(d[0], d[1]), CS, Z);
        const float2 c1 = fma2(make_float2(d[2], d[3]), CS, Z);
        const float2 E0 = entry2<ACC>(FH0, WR0, hh2[q], wc2[q], c0, G32p, Glop);
        const float2 E1 = entry2<ACC>(FH1, WR1, hh2[q], wc2[q], c1, G32p, Glop);
        rp0 += E0.x;
        rp0 += E0.y;
        rp1 += E1.x;
        rp1 += E1.y;
        ca2[q] = fma2(E0, S0, ca2[q]);
        ca2[q] = fma2(E1, S1, ca2[q]);
    }
}

template <bool ACC, class IO>
__device__ __forceinline__ void pass_f32_regen_tc(const float* __restrict__ Y, float cs, int n, int r0, int r1,
                                                  const IO& io, const float* sFh, const float* sWr,
                                                  const float* sS, const float* sX, float G32, float Glo,
                                                  float* sRow, int nloc, float* stage, uint2* sA4)
{
    constexpr int NT = 4;
    const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int nrows = r1 - r0;
    const int BW = tc_block_cols(nw);
    float* stH = stage;                 // staged block: hh, wc, y0, y1, y2 (BW each)
    float* stW = stage + BW;
    float* stY = stage + 2 * BW;        // 3 BW, column-major per coordinate
    const float2 G32p = pk(G32), Glop = pk(Glo), CS = pk(cs);
    const float2 Z = pk(-(cs * 0.0f));          // -0, opaque to the code generator (see point_cost2)
    // the A registers of every row and lane position t, once per pass (when there is room)
    if (sA4 != nullptr)
        for (int q = tid; q < 4 * nrows; q += T) {
            const int il = q >> 2, tt = q & 3;
            uint2 v;
            tc_a_regs(sX[3 * il], sX[3 * il + 1], sX[3 * il + 2], tt, v.x, v.y);
            sA4[q] = v;
        }
    for (int cb0 = 0; cb0 < n; cb0 += BW) {
        __syncthreads();                        // the previous block is no longer read
        for (int q = tid; q < BW; q += T) {
            const int j = cb0 + q;
            float hh, wc;
            io.load1(j, n, hh, wc);
            stH[q] = hh;
            stW[q] = wc;
            const bool ok = j < n;
            stY[q] = ok ? __ldg(Y + 3 * (size_t)j) : 0.0f;
            stY[BW + q] = ok ? __ldg(Y + 3 * (size_t)j + 1) : 0.0f;
            stY[2 * BW + q] = ok ? __ldg(Y + 3 * (size_t)j + 2) : 0.0f;
        }
        __syncthreads();
        for (int sb = 0; sb < kTcSubs; ++sb) {
            const int lb = (warp * kTcSubs + sb) * 32;          // sub-block offset in the block
            if (cb0 + lb >= n) break;                           // warp-uniform
            unsigned int b0[NT], b1[NT];
            float2 hh2[NT], wc2[NT], ca2[NT], fh2[NT], fl2[NT];
#pragma unroll
            for (int q = 0; q < NT; ++q) {
                const int jb = lb + 8 * q + g;                  // the column this lane feeds into B
                if (cb0 + jb < n) {
                    tc_b_regs(stY[jb], stY[BW + jb], stY[2 * BW + jb], t, b0[q], b1[q]);
                } else {
                    b0[q] = 0u;
                    b1[q] = 0u;
                }
                const int jc = lb + 8 * q + 2 * t;              // this lane's two cost columns
                hh2[q] = make_float2(stH[jc], stH[jc + 1]);
                wc2[q] = make_float2(stW[jc], stW[jc + 1]);
                ca2[q] = fh2[q] = fl2[q] = make_float2(0.0f, 0.0f);
            }
            // two row tiles per step, in one basic block so that their instruction streams
            // interleave (a tile past the last row is all padding: its entries are 0)
            for (int rt = 0; rt < nrows; rt += 32) {
                float rp[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int base = rt + 16 * h;
                    const int il0 = base + g, il1 = base + g + 8;
                    // rows past the last are padding: read the last row and select zero A registers
                    // and constants whose entries are 0 (selects, no divergent branches)
                    const bool ok0 = il0 < nrows, ok1 = il1 < nrows;
                    const int ic0 = ok0 ? il0 : nrows - 1, ic1 = ok1 ? il1 : nrows - 1;
                    unsigned int a0, a1, a2, a3;
                    if (sA4 != nullptr) {
                        const uint2 v0 = sA4[4 * ic0 + t], v1 = sA4[4 * ic1 + t];
                        a0 = v0.x; a2 = v0.y; a1 = v1.x; a3 = v1.y;
                    } else {
                        tc_a_regs(sX[3 * ic0], sX[3 * ic0 + 1], sX[3 * ic0 + 2], t, a0, a2);
                        tc_a_regs(sX[3 * ic1], sX[3 * ic1 + 1], sX[3 * ic1 + 2], t, a1, a3);
                    }
                    a0 = ok0 ? a0 : 0u; a2 = ok0 ? a2 : 0u; a1 = ok1 ? a1 : 0u; a3 = ok1 ? a3 : 0u;
                    const float fh0 = ok0 ? sFh[ic0] : 0.0f, wr0 = ok0 ? sWr[ic0] : kPadW, s0 = ok0 ? sS[ic0] : 0.0f;
                    const float fh1 = ok1 ? sFh[ic1] : 0.0f, wr1 = ok1 ? sWr[ic1] : kPadW, s1 = ok1 ? sS[ic1] : 0.0f;
                    tc_tile<ACC, NT>(a0, a1, a2, a3, b0, b1, fh0, wr0, s0, fh1, wr1, s1, hh2, wc2, CS, Z, G32p, Glop,
                                     rp[2 * h], rp[2 * h + 1], ca2);
                }
                // the four lanes of a row group hold the same rows
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    rp[k] += __shfl_xor_sync(0xffffffffu, rp[k], 1);
                    rp[k] += __shfl_xor_sync(0xffffffffu, rp[k], 2);
                }
                if (t == 0) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int il = rt + 16 * (k >> 1) + 8 * (k & 1) + g;
                        if (il < nrows) sRow[warp * nloc + il] += rp[k];
                    }
                }
                if (((rt + 32) % (8 * kFoldRows)) == 0) {        // 2 rows per tile and lane
#pragma unroll
                    for (int q = 0; q < NT; ++q) fold2(fh2[q], fl2[q], ca2[q]);
                }
            }
            // column partials: the eight row groups of the warp (lanes with the same t) hold the
            // same two columns of each tile
#pragma unroll
            for (int q = 0; q < NT; ++q) {
                float2 c = fold_total(fh2[q], fl2[q], ca2[q]);
#pragma unroll
                for (int o = 4; o <= 16; o <<= 1) {
                    c.x += __shfl_xor_sync(0xffffffffu, c.x, o);
                    c.y += __shfl_xor_sync(0xffffffffu, c.y, o);
                }
                if (g == 0) io.store2(cb0 + lb + 8 * q + 2 * t, n, c);
            }
        }
    }
}

template <bool ACC, int KIND, class IO>
__device__ __forceinline__ void pass_f32_regen(const float* __restrict__ Y, float cs, int n, int r0, int r1,
                                               const IO& io, const float* sFh,
                                               const float* sWr, const float* sS, const float* sX,
                                               float G32, float Glo, float* sRow, int nloc)
{
    constexpr int KR = 2;
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int BN = 4 * KR * T;
    const float2 G32p = pk(G32), Glop = pk(Glo), CS = pk(cs);
    const float2 Z = pk(-(cs * 0.0f));          // -0, opaque to the code generator (see point_cost2)
    for (int cb = 0; cb < n; cb += BN) {
        float hh[KR][4], wc[KR][4];
        float2 hh2[KR][2], wc2[KR][2], ca2[KR][2], y0[KR][2], y1[KR][2], y2[KR][2], fh2[KR][2], fl2[KR][2];
        int jk[KR];
#pragma unroll
        for (int k = 0; k < KR; ++k) jk[k] = cb + 4 * (tid + k * T);
        io.load_seg(jk, n, hh, wc);
        to_pairs(hh, hh2);
        to_pairs(wc, wc2);
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            float yv[3][4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = jk[k] + e;
                const bool ok = j < n;
#pragma unroll
                for (int a = 0; a < 3; ++a) yv[a][e] = ok ? __ldg(Y + 3 * (size_t)j + a) : 0.0f;
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                y0[k][q] = make_float2(yv[0][2 * q], yv[0][2 * q + 1]);
                y1[k][q] = make_float2(yv[1][2 * q], yv[1][2 * q + 1]);
                y2[k][q] = make_float2(yv[2][2 * q], yv[2][2 * q + 1]);
            }
            ca2[k][0] = ca2[k][1] = fh2[k][0] = fh2[k][1] = fl2[k][0] = fl2[k][1] = make_float2(0.0f, 0.0f);
        }
        for (int rg = r0; rg < r1; rg += kRG) {
            float rp[kRG];
#pragma unroll
            for (int ii = 0; ii < kRG; ii += 2) {
                rp[ii] = 0.0f;
                rp[ii + 1] = 0.0f;
                const int i = rg + ii;
                // two rows in one block when both exist, so that their instruction streams
                // interleave (row sums and column partials keep their order)
                if (i + 1 < r1) {
                    rp[ii] = regen_row<ACC, KIND, KR>(sX, i - r0, sFh, sWr, sS, y0, y1, y2, hh2, wc2, CS, Z, G32p,
                                                      Glop, ca2);
                    rp[ii + 1] = regen_row<ACC, KIND, KR>(sX, i + 1 - r0, sFh, sWr, sS, y0, y1, y2, hh2, wc2, CS, Z,
                                                          G32p, Glop, ca2);
                } else if (i < r1) {
                    rp[ii] = regen_row<ACC, KIND, KR>(sX, i - r0, sFh, sWr, sS, y0, y1, y2, hh2, wc2, CS, Z, G32p,
                                                      Glop, ca2);
                }
            }
            butterfly<kRG>(rp, lane);
            const int il = rg + lane;
            if (lane < kRG && il < r1) sRow[warp * nloc + (il - r0)] += rp[0];
            if (((rg - r0 + kRG) % kFoldRows) == 0) {
#pragma unroll
                for (int k = 0; k < KR; ++k) {
                    fold2(fh2[k][0], fl2[k][0], ca2[k][0]);
                    fold2(fh2[k][1], fl2[k][1], ca2[k][1]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            float2 tot[2] = {fold_total(fh2[k][0], fl2[k][0], ca2[k][0]), fold_total(fh2[k][1], fl2[k][1], ca2[k][1])};
            float ca[4];
            from_pairs(tot, ca);
            io.store4(jk[k], n, ca);
        }
    }
}

// fp64 entries with the regenerated cost (the fp32 cost value promoted, as the dense tier does)
template <int KIND>
__device__ __forceinline__ void pass_f64_regen(const float* __restrict__ Y, float cs, int n, int r0, int r1,
                                               const double* Hd, const double* sFd, const double* sS,
                                               const float* sX, double gamma, double* sRow, int nloc,
                                               double* colpart_b)
{
    constexpr int KR = 2;
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int BN = 4 * KR * T;
    for (int cb = 0; cb < n; cb += BN) {
        double hd[KR][4], ca[KR][4];
        float y0[KR][4], y1[KR][4], y2[KR][4];
        int jk[KR];
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            jk[k] = cb + 4 * (tid + k * T);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = jk[k] + e;
                const bool ok = j < n;
                hd[k][e] = ok ? __ldcg(Hd + j) : -INFINITY;
                y0[k][e] = ok ? __ldg(Y + 3 * (size_t)j) : 0.0f;
                y1[k][e] = ok ? __ldg(Y + 3 * (size_t)j + 1) : 0.0f;
                y2[k][e] = ok ? __ldg(Y + 3 * (size_t)j + 2) : 0.0f;
                ca[k][e] = 0.0;
            }
        }
        for (int rg = r0; rg < r1; rg += kRG) {
            double rp[kRG];
#pragma unroll
            for (int ii = 0; ii < kRG; ++ii) {
                rp[ii] = 0.0;
                const int i = rg + ii;
                if (i < r1) {
                    const int il = i - r0;
                    const double fd = sFd[il], s = sS[il];
                    const float x0 = sX[3 * il], x1 = sX[3 * il + 1], x2 = sX[3 * il + 2];
#pragma unroll
                    for (int k = 0; k < KR; ++k) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const double cv = (double)point_cost<KIND>(x0, x1, x2, y0[k][e], y1[k][e], y2[k][e], cs);
                            const double E = exp((fd + hd[k][e]) - gamma * cv);
                            rp[ii] += E;
                            ca[k][e] = fma(E, s, ca[k][e]);
                        }
                    }
                }
            }
            butterfly<kRG>(rp, lane);
            const int il = rg + lane;
            if (lane < kRG && il < r1) sRow[warp * nloc + (il - r0)] += rp[0];
        }
#pragma unroll
        for (int k = 0; k < KR; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (jk[k] + e < n) colpart_b[jk[k] + e] = ca[k][e];
    }
}

// C_ij inside the generic passes: a dense row pointer, or regenerated (scalar loads; the generic
// evaluation is not on the solver's hot path).
template <int COST>
__device__ __forceinline__ float cost_at(const WS& ws, const float* Crow, int i, int j)
{
    if (COST == COST_DENSE) return __ldg(Crow + j);
    return point_cost<COST>(__ldg(ws.X + 3 * (size_t)i), __ldg(ws.X + 3 * (size_t)i + 1), __ldg(ws.X + 3 * (size_t)i + 2),
                            __ldg(ws.Y + 3 * (size_t)j), __ldg(ws.Y + 3 * (size_t)j + 1), __ldg(ws.Y + 3 * (size_t)j + 2),
                            ws.cscale);
}

// Two-scale pass of the generic dual evaluation: the row sum of row i uses exponents relative to
// the row scale A_i (folded into the row constants sFh/sWr), the column sum of column j uses
// exponents relative to the column scale B_j (folded into the column constants Hh2/Wc2), so both
// log-sum-exps stay exact for potentials of any spread.  Two exp2 per entry.
template <bool VEC4, bool ACC, int COST>
__device__ __forceinline__ void pass2_f32(const WS& ws, const float* __restrict__ C, int n, int r0, int r1,
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
                wc[k][e] = ok ? __ldcg(Wc + j) : kPadW;
                hh2[k][e] = ok ? __ldcg(Hh2 + j) : 0.0f;
                wc2[k][e] = ok ? __ldcg(Wc2 + j) : kPadW;
                ca[k][e] = 0.0f;
            }
        }
        for (int rg = r0; rg < r1; rg += kRG) {
            float rp[kRG];
#pragma unroll
            for (int ii = 0; ii < kRG; ++ii) {
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
                            for (int e = 0; e < 4; ++e)
                                cv[e] = (jk[k] + e < n) ? cost_at<COST>(ws, Crow, i, jk[k] + e) : 0.0f;
                        }
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float d = (fh + hh[k][e]) - cv[e];
                            const float d2 = (fh2 + hh2[k][e]) - cv[e];
                            if (ACC) {
                                rp[ii] += exp2_acc(d, G32, Glo, wr + wc[k][e]);
                                ca[k][e] += exp2_acc(d2, G32, Glo, wr2 + wc2[k][e]);
                            } else {
                                rp[ii] += ex2f(fmaf(Glo, d, fmaf(G32, d, wr + wc[k][e])));
                                ca[k][e] += ex2f(fmaf(Glo, d2, fmaf(G32, d2, wr2 + wc2[k][e])));
                            }
                        }
                    }
                }
            }
            butterfly<kRG>(rp, lane);
            const int il = rg + lane;
            if (lane < kRG && il < r1) sRow[warp * nloc + (il - r0)] += rp[0];
        }
#pragma unroll
        for (int k = 0; k < K2; ++k)
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (jk[k] + e < n) colpart_b[jk[k] + e] = ca[k][e];
    }
}

template <int COST>
__device__ __forceinline__ void pass2_f64(const WS& ws, const float* __restrict__ C, int n, int r0, int r1,
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
        for (int rg = r0; rg < r1; rg += kRG) {
            double rp[kRG];
#pragma unroll
            for (int ii = 0; ii < kRG; ++ii) {
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
                            const double cv = (j < n) ? (double)cost_at<COST>(ws, Crow, i, j) : 0.0;
                            const double z = (fd + hd[k][e]) - gamma * cv;   // u_i + v_j - gamma C_ij
                            rp[ii] += exp(z - ad);
                            ca[k][e] += exp(z - bd[k][e]);
                        }
                    }
                }
            }
            butterfly<kRG>(rp, lane);
            const int il = rg + lane;
            if (lane < kRG && il < r1) sRow[warp * nloc + (il - r0)] += rp[0];
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
// column j0 + lane is returned in warp 0.  Each warp issues all of its partial loads before
// summing them (independent loads in flight instead of a dependent chain).  sm: >= 2 * 32 * nwarps
// floats.  Requires G <= 24 * nwarps.
// merge_cols_f32 with the total as a double-float (the fp32 stage kernel's epilogue avoids fp64:
// on this GPU an fp64 warp instruction holds the SM's small fp64 pipe for many cycles).
__device__ __forceinline__ float2 merge_cols_f32_df(const float* colpart, int n, int G, int j0, int j1, float* sm)
{
    constexpr int kMaxPer = 24;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int j = j0 + lane;
    float vals[kMaxPer];
#pragma unroll
    for (int k = 0; k < kMaxPer; ++k) {
        const int b = warp + k * nw;
        vals[k] = (j < j1 && b < G) ? __ldcg(colpart + (size_t)b * n + j) : 0.0f;
    }
    float s = 0.0f, comp = 0.0f;
#pragma unroll
    for (int k = 0; k < kMaxPer; ++k) kahan_add(s, comp, vals[k]);
    sm[warp * 32 + lane] = s;
    sm[(nw + warp) * 32 + lane] = -comp;
    __syncthreads();
    float2 tot = make_float2(0.0f, 0.0f);
    if (warp == 0)
        for (int w = 0; w < nw; ++w) tot = df_add_f(df_add_f(tot, sm[w * 32 + lane]), sm[(nw + w) * 32 + lane]);
    __syncthreads();
    return tot;
}

__device__ __forceinline__ double merge_cols_f32(const float* colpart, int n, int G,
                                                 int j0, int j1, float* sm)
{
    constexpr int kMaxPer = 24;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int j = j0 + lane;
    float vals[kMaxPer];
#pragma unroll
    for (int k = 0; k < kMaxPer; ++k) {
        const int b = warp + k * nw;
        vals[k] = (j < j1 && b < G) ? __ldcg(colpart + (size_t)b * n + j) : 0.0f;
    }
    float s = 0.0f, comp = 0.0f;
#pragma unroll
    for (int k = 0; k < kMaxPer; ++k) kahan_add(s, comp, vals[k]);
    sm[warp * 32 + lane] = s;
    sm[(nw + warp) * 32 + lane] = -comp;
    __syncthreads();
    double tot = 0.0;
    if (warp == 0)
        for (int w = 0; w < nw; ++w) tot += (double)sm[w * 32 + lane] + (double)sm[(nw + w) * 32 + lane];
    __syncthreads();
    return tot;
}

// merge_cols_f32 for up to 32 MC columns [j0, j1) in one round trip: every load of every column
// group is in flight before any addition; the column totals (fp64) go to out[j - j0].
template <int MC>
__device__ __forceinline__ void merge_cols_f32_wide(const float* colpart, int n, int G, int j0, int j1, float* sm,
                                                    double* out)
{
    constexpr int kMaxPer = 24;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float vals[MC][kMaxPer];
#pragma unroll
    for (int m = 0; m < MC; ++m) {
        const int j = j0 + lane + 32 * m;
#pragma unroll
        for (int k = 0; k < kMaxPer; ++k) {
            const int b = warp + k * nw;
            vals[m][k] = (j < j1 && b < G) ? __ldcg(colpart + (size_t)b * n + j) : 0.0f;
        }
    }
#pragma unroll
    for (int m = 0; m < MC; ++m) {
        float s = 0.0f, comp = 0.0f;
#pragma unroll
        for (int k = 0; k < kMaxPer; ++k) kahan_add(s, comp, vals[m][k]);
        sm[(m * nw + warp) * 32 + lane] = s;
        sm[((MC + m) * nw + warp) * 32 + lane] = -comp;
    }
    __syncthreads();
    if (warp < MC) {
        double tot = 0.0;
        for (int w = 0; w < nw; ++w)
            tot += (double)sm[(warp * nw + w) * 32 + lane] + (double)sm[((MC + warp) * nw + w) * 32 + lane];
        out[warp * 32 + lane] = tot;
    }
    __syncthreads();
}

__device__ __forceinline__ double merge_cols_f64(const double* colpart, int n, int G,
                                                 int j0, int j1, double* sm)
{
    constexpr int kMaxPer = 24;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int j = j0 + lane;
    double vals[kMaxPer];
#pragma unroll
    for (int k = 0; k < kMaxPer; ++k) {
        const int b = warp + k * nw;
        vals[k] = (j < j1 && b < G) ? __ldcg(colpart + (size_t)b * n + j) : 0.0;
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kMaxPer; ++k) s += vals[k];
    sm[warp * 32 + lane] = s;
    __syncthreads();
    double tot = 0.0;
    if (warp == 0)
        for (int w = 0; w < nw; ++w) tot += sm[w * 32 + lane];
    __syncthreads();
    return tot;
}

}  // namespace mdot
