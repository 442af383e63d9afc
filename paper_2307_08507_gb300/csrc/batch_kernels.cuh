// Batched MDOT-PNCG: one persistent launch solves many problems of uneven n (up to kBatchMaxN).
// Each CTA takes the next problem from an atomic work queue (problems ordered by decreasing n)
// and runs the whole solve of Alg. 1 on it with block-level synchronisation only: validation and
// entropies, the gamma schedule, every stage's PNCG projection with the App. B line search (same
// decide() as the cooperative path), rounding (Alg. 3) and the c-transform bound.  All reductions
// run in a fixed order, so a problem's result does not depend on which CTA solves it or on what
// else is in the batch.
#pragma once

#include "solver_kernels.cuh"

namespace mdot {

constexpr int kBatchMaxN = 8192;
constexpr int kBatchThreads = 256;     // threads of the default ("wide") variant
constexpr int kRowChunk = 4096;        // rows whose per-warp partial sums sit in shared memory at once

// Tile variants of the batched kernel, chosen per problem-size bucket by mdot_tune_batch:
// 0 ("wide"): 256 threads, one CTA (problem) per SM; 1 ("narrow"): 128 threads, two CTAs
// (problems) per SM -- half the warps per problem, twice the problems in flight.
constexpr int kBatchVariants = 2;
__host__ __device__ constexpr int batch_threads(int variant) { return variant == 1 ? 128 : 256; }
// problem-size buckets of the tuning table: n < 512, < 1024, < 2048, < 4096, <= kBatchMaxN
constexpr int kBatchBuckets = 5;
__host__ __device__ inline int batch_bucket(int n) { return n < 512 ? 0 : n < 1024 ? 1 : n < 2048 ? 2 : n < 4096 ? 3 : 4; }

struct BatchProblem {
    int n, kind;               // size, CostKind
    float scale;               // cost scale (regenerated cost)
    int pad;
    double eps, gamma_f;       // target gap (gamma_f <= 0: from eps, Prop. 2) or gamma_f
    const double *r, *c;
    const float *C, *X, *Y;
    double *u_out, *v_out;     // nullable
    double* slot;              // nullable: this problem's workspace (else the CTA's slot)
    int slot_stride;           // vector stride of that workspace (>= n), see batch_slot_doubles
    int pad2;
};

// Doubles of a workspace whose vectors have the given stride (18 fp64 and 7 fp32/int32 vectors).
__host__ __device__ inline size_t batch_slot_doubles(int stride)
{
    return (size_t)19 * stride + ((size_t)7 * stride + 1) / 2;
}

struct BatchResult {
    int status, stages;
    long long evals, iters;
    double cost, lower_bound, grad_l1, gamma_f, H_min;
    int stalls, pad;
};

struct BatchArgs {
    int nprob;
    const BatchProblem* probs;
    BatchResult* results;
    const int* order;          // solve order (indices into probs)
    unsigned int* next;        // work-queue counter (zeroed by the host)
    int* done;                 // nullable: done[i] = 1 once results[i] is written (may be host memory)
    double* slots;             // per-CTA workspace, slot_doubles each
    size_t slot_doubles;
    // parameters of Alg. 1 / App. B
    double gamma_i, p, q, c1, c2, fp32_floor, final_tol;
    int ls_max_trials, max_iter, warm_start, precision, smoothing, ls_init;
    int tensor_cores;          // 1: integer-point squared-Euclidean costs on the tensor cores
    int polish_iters;          // fp64 iterations at most that finish a stalled last stage
};

// slot layout (vectors of `stride` elements): 18 fp64 vectors, then 7 fp32 / int32 vectors
enum SlotVec { SV_U = 0, SV_V, SV_PU, SV_PV, SV_UP, SV_VP, SV_GR, SV_GC, SV_RT, SV_CT, SV_GRT, SV_GCT,
               SV_SRT, SV_SCT, SV_LR, SV_Y, SV_EC, SV_RS, SV_COUNT };
enum SlotF32 { SF_HH = 0, SF_WC, SF_COL, SF_FH, SF_WR, SF_S, SF_A, SF_COUNT };
static_assert(SV_COUNT <= 19 && SF_COUNT <= 7, "batch_slot_doubles covers the slot layout");
constexpr size_t kSlotDoubles = (size_t)SV_COUNT * kBatchMaxN + ((size_t)SF_COUNT * kBatchMaxN + 1) / 2;

struct BatchSmem {
    size_t off_row, off_stage, bytes;
};

__host__ __device__ inline BatchSmem batch_smem(int threads)
{
    BatchSmem L;
    L.off_row = 0;
    L.off_stage = (size_t)(threads / 32) * kRowChunk * 4;            // per-warp row partials of one chunk
    L.bytes = L.off_stage + (size_t)tc_stage_floats(threads / 32) * 4;    // tensor-core column blocks
    return L;
}

// Column partials of a row chunk added to the sums of the earlier chunks (the same thread owns
// column j in every chunk, so the order is fixed).
struct ColAccum {
    const float* Hh;
    const float* Wc;
    float* out;
    bool first;
    template <int KK>
    __device__ __forceinline__ bool load_seg(const int (&jk)[KK], int n, float (&hh)[KK][4], float (&wc)[KK][4]) const
    {
        return ColPlain{Hh, Wc, out}.load_seg(jk, n, hh, wc);
    }
    __device__ __forceinline__ void store4(int j0, int n, const float ca[4]) const
    {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (j0 + e < n) out[j0 + e] = first ? ca[e] : out[j0 + e] + ca[e];
    }
    __device__ __forceinline__ void load1(int j, int n, float& hh, float& wc) const
    {
        ColPlain{Hh, Wc, out}.load1(j, n, hh, wc);
    }
    __device__ __forceinline__ void store2(int j0, int n, float2 ca) const
    {
        if (j0 < n) out[j0] = first ? ca.x : out[j0] + ca.x;
        if (j0 + 1 < n) out[j0 + 1] = first ? ca.y : out[j0 + 1] + ca.y;
    }
};

// One pass over all n rows (the CTA owns the whole problem), in chunks of kRowChunk rows: the
// fp64 row sums (relative to 2^{A_i}) go to rowsum, the complete column sums to colsum.
// tc: the squared-Euclidean cost of integer points on the tensor cores (pass_f32_regen_tc).
template <bool ACC, int COST>
__device__ __forceinline__ void batch_pass(const BatchProblem& P, const float* Hh, const float* Wc,
                                           const float* Fh, const float* Wr, const float* S,
                                           float G32, float Glo, float* sRow, float* colsum, double* rowsum,
                                           bool tc, float* stage)
{
    const int n = P.n, nw = blockDim.x >> 5;
    for (int r0 = 0; r0 < n; r0 += kRowChunk) {
        const int r1 = min(n, r0 + kRowChunk), nc = r1 - r0;
        for (int x = threadIdx.x; x < nw * nc; x += blockDim.x) sRow[x] = 0.0f;
        __syncthreads();
        const ColAccum io{Hh, Wc, colsum, r0 == 0};
        if (COST == COST_SQEUCLID && tc)
            pass_f32_regen_tc<ACC>(P.Y, P.scale, n, r0, r1, io, Fh + r0, Wr + r0, S + r0, P.X + 3 * (size_t)r0,
                                   G32, Glo, sRow, nc, stage, nullptr);
        else if (COST != COST_DENSE)
            pass_f32_regen<ACC, COST>(P.Y, P.scale, n, r0, r1, io, Fh + r0, Wr + r0, S + r0, P.X + 3 * (size_t)r0,
                                      G32, Glo, sRow, nc);
        else if ((n & 3) == 0 && (reinterpret_cast<uintptr_t>(P.C) & 15) == 0)
            pass_f32<true, ACC>(P.C, n, r0, r1, io, Fh + r0, Wr + r0, S + r0, G32, Glo, sRow, nc);
        else
            pass_f32<false, ACC>(P.C, n, r0, r1, io, Fh + r0, Wr + r0, S + r0, G32, Glo, sRow, nc);
        __syncthreads();
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += (double)sRow[w * nc + (i - r0)];
            rowsum[i] = t;
        }
        __syncthreads();
    }
}

template <int COST>
__device__ __forceinline__ float batch_cost(const BatchProblem& P, int i, int j)
{
    if (COST == COST_DENSE) return __ldg(P.C + (size_t)i * P.n + j);
    return point_cost<COST>(__ldg(P.X + 3 * (size_t)i), __ldg(P.X + 3 * (size_t)i + 1), __ldg(P.X + 3 * (size_t)i + 2),
                            __ldg(P.Y + 3 * (size_t)j), __ldg(P.Y + 3 * (size_t)j + 1), __ldg(P.Y + 3 * (size_t)j + 2),
                            P.scale);
}

// Per-row constants of an evaluation at ua with row scale A (fp32 tiers).
__device__ __forceinline__ void batch_prep_row(double ua, int A, double inv_gamma, double G64, float* sFh,
                                               float* sWr, float* sS, int* sA, int i)
{
    float fh, wl;
    split_cost_unit((ua - (double)A * kLn2) * inv_gamma, fh, wl, G64);
    sFh[i] = fh;
    sWr[i] = wl;
    sS[i] = pow2f_int(A);
    sA[i] = A;
}

// Per-row constants of an fp64-entry evaluation at ua with row scale A: E_ij = exp(fd_i + v_j -
// gamma C_ij) relative to 2^{A_i}, weighted by 2^{A_i} into the column sums.
__device__ __forceinline__ void batch_prep_row64(double ua, int A, double* fd, double* s64, int* sA, int i)
{
    fd[i] = ua - (double)A * kLn2;
    s64[i] = ldexp(1.0, A);
    sA[i] = A;
}

// One fp64-entry pass over all n rows (the polish of the last stage) in chunks of kRowChunk / 2 rows,
// whose per-warp fp64 row partials fill the shared memory of the fp32 passes' chunks: row sums
// (relative to 2^{A_i}) to rowsum, the complete column sums to colsum (a later chunk's partials go
// through tmp and are added in a fixed order).
template <int COST>
__device__ __forceinline__ void batch_pass64(const BatchProblem& P, const double* hd, const double* fd,
                                             const double* s64, double gamma, double* sRow, double* colsum,
                                             double* tmp, double* rowsum)
{
    constexpr int kChunk = kRowChunk / 2;
    const int n = P.n, nw = blockDim.x >> 5;
    for (int r0 = 0; r0 < n; r0 += kChunk) {
        const int r1 = min(n, r0 + kChunk), nc = r1 - r0;
        double* part = (r0 == 0) ? colsum : tmp;
        for (int x = threadIdx.x; x < nw * nc; x += blockDim.x) sRow[x] = 0.0;
        __syncthreads();
        if (COST == COST_DENSE)
            pass_f64(P.C, n, r0, r1, hd, fd + r0, s64 + r0, gamma, sRow, nc, part);
        else
            pass_f64_regen<COST>(P.Y, P.scale, n, r0, r1, hd, fd + r0, s64 + r0, P.X + 3 * (size_t)r0, gamma,
                                 sRow, nc, part);
        __syncthreads();
        if (r0 > 0)
            for (int j = threadIdx.x; j < n; j += blockDim.x) colsum[j] += tmp[j];
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += sRow[w * nc + (i - r0)];
            rowsum[i] = t;
        }
        __syncthreads();
    }
}

template <int COST, int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS == 128 ? 2 : 1) batch_kernel(BatchArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double red_smem[32 * kNRed];
    __shared__ double s_bc[8];
    __shared__ State st;
    __shared__ int s_prob;
    const BatchSmem L = batch_smem(THREADS);
    float* sRow = reinterpret_cast<float*>(sm + L.off_row);
    float* sStage = reinterpret_cast<float*>(sm + L.off_stage);
    const int tid = threadIdx.x, T = blockDim.x, nw = T >> 5, lane = tid & 31, warp = tid >> 5;
    double* const cta_slot = a.slots + (size_t)blockIdx.x * a.slot_doubles;

    for (;;) {
        if (tid == 0) s_prob = (int)atomicAdd(a.next, 1u);
        __syncthreads();
        const int pidx = s_prob;
        __syncthreads();
        if (pidx >= a.nprob) break;
        const int pi = a.order[pidx];
        const BatchProblem P = a.probs[pi];
        const int n = P.n;
        // workspace: the problem's own slot if it has one, else this CTA's
        double* slot = P.slot ? P.slot : cta_slot;
        const size_t sd = P.slot ? (size_t)P.slot_stride : (size_t)kBatchMaxN;
        double* V[SV_COUNT];
        for (int k = 0; k < SV_COUNT; ++k) V[k] = slot + (size_t)k * sd;
        float* F32 = reinterpret_cast<float*>(slot + (size_t)SV_COUNT * sd);
        float* Hh = F32 + (size_t)SF_HH * sd;
        float* Wc = F32 + (size_t)SF_WC * sd;
        float* colsum = F32 + (size_t)SF_COL * sd;
        float* sFh = F32 + (size_t)SF_FH * sd;      // per-row constants (read through L1)
        float* sWr = F32 + (size_t)SF_WR * sd;
        float* sS = F32 + (size_t)SF_S * sd;
        int* sA = reinterpret_cast<int*>(F32 + (size_t)SF_A * sd);
        // the fp64 polish of the last stage reuses vectors that are idle by then: the warm-start
        // history (row and column constants), the rounding's error vector (column sums), the fp32
        // column constants (row scales 2^A) and the fp32 column sums with the row constants (a row
        // chunk's column partials); the per-warp row partials take the fp32 passes' shared memory
        double* fd64 = V[SV_UP];
        double* hd64 = V[SV_VP];
        double* col64 = V[SV_EC];
        double* s64 = reinterpret_cast<double*>(Hh);        // Hh, Wc: 2 sd floats
        double* tmp64 = reinterpret_cast<double*>(colsum);  // colsum, sFh: 2 sd floats
        double* sRow64 = reinterpret_cast<double*>(sm + L.off_row);
        BatchResult res;
        memset(&res, 0, sizeof(res));

        // ---- validation and H_min (entropies in fp64 sums of fp32 logs) ----
        double x[kNRed];
#pragma unroll
        for (int q = 0; q < kNRed; ++q) x[q] = 0.0;
        for (int i = tid; i < n; i += T) {
            const double ri = P.r[i], ci = P.c[i];
            x[0] += ri;
            x[1] += ci;
            if (ri > 0.0) x[2] -= ri * (double)__logf((float)ri);
            if (ci > 0.0) x[3] -= ci * (double)__logf((float)ci);
            x[4] += (isfinite(ri) && isfinite(ci) && ri >= 0.0 && ci >= 0.0) ? 0.0 : 1.0;
        }
        block_reduce_nred(x, red_smem);
        if (tid == 0) {
            const bool bad = x[4] != 0.0 || !(fabs(x[0] - 1.0) <= 1e-9) || !(fabs(x[1] - 1.0) <= 1e-9) || n < 1 ||
                             n > kBatchMaxN;
            const double H = fmax(fmin(x[2], x[3]), 1e-12);
            double gf = P.gamma_f;
            if (!(gf > 0.0)) {
                const double target = pow(5.0 * H / (2.0 * P.eps), 1.0 / a.p);       // Prop. 2
                gf = a.gamma_i;
                while (gf < target * (1.0 - 1e-12)) gf *= a.q;
            }
            s_bc[0] = H;
            s_bc[1] = gf;
            s_bc[2] = bad ? 1.0 : 0.0;
        }
        __syncthreads();
        const double H = s_bc[0], gf = s_bc[1];
        // squared-Euclidean cost of integer points (|coordinate| <= 255): the tensor-core form
        bool tc = false;
        if (COST == COST_SQEUCLID && a.tensor_cores && s_bc[2] == 0.0) {
            bool ok = true;
            for (int q = tid; q < 3 * n; q += T) {
                const float xv = __ldg(P.X + q), yv = __ldg(P.Y + q);
                ok = ok && fabsf(xv) <= 255.0f && xv == rintf(xv) && fabsf(yv) <= 255.0f && yv == rintf(yv);
            }
            tc = __syncthreads_and(ok ? 1 : 0) != 0;
        }
        if (s_bc[2] != 0.0) {
            if (tid == 0) {
                res.status = ST_NUMERIC + 10;          // invalid problem
                a.results[pi] = res;
                if (a.done) {
                    __threadfence_system();
                    reinterpret_cast<volatile int*>(a.done)[pi] = 1;
                }
            }
            __syncthreads();
            continue;
        }

        // ---- MDOT (Alg. 1): stage after stage ----
        if (tid == 0) memset(&st, 0, sizeof(State));
        __syncthreads();
        double gamma = fmin(a.gamma_i, gf), dgamma_prev = gamma, ratio = 0.0, tol_last = 0.0;
        int stages = 0;
        for (int t = 1;; ++t) {
            const double eps_d = H / pow(gamma, a.p);
            const double w = (a.smoothing == 1) ? H / pow(gf, a.p) : eps_d;    // smoothing weight (Alg. 1)
            double tol = fmax(eps_d / 2.0, 1e-13 + 1e-15 * gamma);
            const bool last = (gamma == gf);
            if (last && a.final_tol > 0.0) tol = a.final_tol;
            const bool acc = a.precision == 3 || (a.precision == 0 && tol < 2e-6);
            StageArgs sa{};
            sa.gamma = gamma;
            sa.G64 = gamma * kLog2e;
            sa.tol = fmax(tol, a.fp32_floor);
            sa.c1 = a.c1;
            sa.c2 = a.c2;
            sa.ls_max_trials = a.ls_max_trials;
            sa.ls_init = a.ls_init;
            sa.max_iter = a.max_iter;
            sa.tier = acc ? TIER_F32A : TIER_F32;
            sa.stall_below = stall_floor(sa.tier);
            const double inv_gamma = 1.0 / gamma, G64 = sa.G64;
            const float G32 = (float)G64, Glo = (float)(G64 - (double)G32);
            // prologue: smoothing, rank-one start or warm start (Eq. (13)), constants at alpha = 0
            for (int i = tid; i < n; i += T) {
                const double rt = (1.0 - w / 4.0) * P.r[i] + w / (4.0 * n);
                const double lrt = log(rt);
                double u = V[SV_U][i];
                if (t == 1) { u = lrt; V[SV_UP][i] = u; }
                else if (a.warm_start == 0) { const double z = u; u = z + ratio * (z - V[SV_UP][i]); V[SV_UP][i] = z; }
                else if (a.warm_start == 1) { u = ratio * u; }
                V[SV_U][i] = u; V[SV_PU][i] = 0.0; V[SV_GR][i] = 0.0; V[SV_RT][i] = rt; V[SV_LR][i] = lrt;
                batch_prep_row(u, row_scale(lrt), inv_gamma, G64, sFh, sWr, sS, sA, i);
            }
            for (int j = tid; j < n; j += T) {
                const double ct = (1.0 - w / 4.0) * P.c[j] + w / (4.0 * n);
                double v = V[SV_V][j];
                if (t == 1) { v = log(ct); V[SV_VP][j] = v; }
                else if (a.warm_start == 0) { const double z = v; v = z + ratio * (z - V[SV_VP][j]); V[SV_VP][j] = z; }
                else if (a.warm_start == 1) { v = ratio * v; }
                V[SV_V][j] = v; V[SV_PV][j] = 0.0; V[SV_GC][j] = 0.0; V[SV_CT][j] = ct;
                float gh, wl;
                split_cost_unit(v * inv_gamma, gh, wl, G64);
                Hh[j] = gh;
                Wc[j] = wl;
            }
            if (tid == 0) {
                st.alpha = 0.0; st.kind = KIND_INIT; st.accept = 0; st.trials = 0; st.k = 0;
                st.phase = PH_RUN; st.beta = 0.0; st.alpha_commit = 0.0;
            }
            __syncthreads();
            // one PNCG projection (Alg. 2 with the App. B line search) at this gamma, from the
            // constants already prepared: fp32 entries, or fp64 entries for the polish below
            auto project = [&](const StageArgs& sx, bool f64) {
                for (;;) {
                    if (f64)      batch_pass64<COST>(P, hd64, fd64, s64, gamma, sRow64, col64, tmp64, V[SV_RS]);
                    else if (acc) batch_pass<true, COST>(P, Hh, Wc, sFh, sWr, sS, G32, Glo, sRow, colsum, V[SV_RS], tc, sStage);
                    else          batch_pass<false, COST>(P, Hh, Wc, sFh, sWr, sS, G32, Glo, sRow, colsum, V[SV_RS], tc, sStage);
#pragma unroll
                    for (int q = 0; q < kNRed; ++q) x[q] = 0.0;
                    for (int i = tid; i < n; i += T) {
                        const double sum = V[SV_RS][i];
                        if (!(sum > 0.0) || !isfinite(sum)) { x[5] += 1.0; continue; }
                        const double rt = V[SV_RT][i];
                        const double g = ldexp(sum, sA[i]) - rt;
                        const double s = -(double)log1pf((float)g / (float)rt);     // Eq. (17)
                        const double p = V[SV_PU][i], y = g - V[SV_GR][i];
                        x[0] += p * g; x[1] += fabs(g); x[2] += y * (-s); x[3] += y * p; x[4] += s * g;
                        V[SV_GRT][i] = g;
                        V[SV_SRT][i] = s;
                        V[SV_Y][i] = ((double)__log2f((float)sum) + (double)sA[i]) * kLn2;   // log r(P), scale only
                    }
                    for (int j = tid; j < n; j += T) {
                        const double cs = f64 ? col64[j] : (double)colsum[j];
                        if (!(cs > 0.0) || !isfinite(cs)) { x[5] += 1.0; continue; }
                        const double ct = V[SV_CT][j];
                        const double g = cs - ct;
                        const double s = -(double)log1pf((float)g / (float)ct);
                        const double p = V[SV_PV][j], y = g - V[SV_GC][j];
                        x[0] += p * g; x[1] += fabs(g); x[2] += y * (-s); x[3] += y * p; x[4] += s * g;
                        V[SV_GCT][j] = g;
                        V[SV_SCT][j] = s;
                    }
                    block_reduce_nred(x, red_smem);
                    if (tid == 0) {
                        decide(&st, x, sx);
                        s_bc[0] = st.alpha; s_bc[1] = st.alpha_commit; s_bc[2] = st.beta;
                        s_bc[3] = (double)st.accept; s_bc[4] = (double)st.phase;
                    }
                    __syncthreads();
                    const double alpha = s_bc[0], acommit = s_bc[1], beta = s_bc[2];
                    const bool accept = s_bc[3] != 0.0, done = s_bc[4] != 0.0;
                    for (int i = tid; i < n; i += T) {
                        double u = V[SV_U][i], p = V[SV_PU][i];
                        if (accept) {
                            u += acommit * p;
                            V[SV_U][i] = u;
                            V[SV_GR][i] = V[SV_GRT][i];
                            V[SV_LR][i] = V[SV_Y][i];
                            p = V[SV_SRT][i] + beta * p;
                            V[SV_PU][i] = p;
                        }
                        if (done) continue;
                        const int A = row_scale(V[SV_LR][i] + alpha * p);
                        if (f64) batch_prep_row64(u + alpha * p, A, fd64, s64, sA, i);
                        else     batch_prep_row(u + alpha * p, A, inv_gamma, G64, sFh, sWr, sS, sA, i);
                    }
                    for (int j = tid; j < n; j += T) {
                        double v = V[SV_V][j], p = V[SV_PV][j];
                        if (accept) {
                            v += acommit * p;
                            V[SV_V][j] = v;
                            V[SV_GC][j] = V[SV_GCT][j];
                            p = V[SV_SCT][j] + beta * p;
                            V[SV_PV][j] = p;
                        }
                        if (done) continue;
                        if (f64) {
                            hd64[j] = v + alpha * p;
                        } else {
                            float gh, wl;
                            split_cost_unit((v + alpha * p) * inv_gamma, gh, wl, G64);
                            Hh[j] = gh;
                            Wc[j] = wl;
                        }
                    }
                    __syncthreads();
                    if (done) break;
                }
            };
            project(sa, false);
            ++stages;
            tol_last = sa.tol;
            // a last stage whose fp32 part ended by the stall rule above its tolerance (which is
            // floored at fp32_floor here, see mdot_solve_batch) continues in fp64 entries from the
            // fp32 iterate, same gamma and smoothing, for at most polish_iters iterations: an fp64
            // evaluation on one SM costs ~5 ns per entry (fp64 runs at 1/64 of the fp32 rate on
            // this GPU), so a problem that needs more reports MDOT_ERR_NOT_CONVERGED with its best
            // iterate instead of holding its SM
            if (last && a.precision == 0 && a.polish_iters > 0 && st.status == ST_OK && !(st.gnorm <= sa.tol)) {
                StageArgs sb = sa;
                sb.tier = TIER_F64;
                sb.stall_below = stall_floor(TIER_F64);
                sb.max_iter = min(a.max_iter, a.polish_iters);
                for (int i = tid; i < n; i += T) {
                    V[SV_PU][i] = 0.0;
                    V[SV_GR][i] = 0.0;
                    batch_prep_row64(V[SV_U][i], row_scale(V[SV_LR][i]), fd64, s64, sA, i);
                }
                for (int j = tid; j < n; j += T) {
                    V[SV_PV][j] = 0.0;
                    V[SV_GC][j] = 0.0;
                    hd64[j] = V[SV_V][j];
                }
                if (tid == 0) {
                    st.alpha = 0.0; st.kind = KIND_INIT; st.accept = 0; st.trials = 0; st.k = 0;
                    st.phase = PH_RUN; st.beta = 0.0; st.alpha_commit = 0.0;
                }
                __syncthreads();
                project(sb, true);
                tol_last = sb.tol;
            }
            if (last || st.status >= ST_LSFAIL) break;
            double dg = (a.q - 1.0) * gamma;
            const double gnext = fmin(gamma + dg, gf);
            dg = gnext - gamma;
            ratio = (a.warm_start == 1) ? gnext / gamma : dg / dgamma_prev;
            dgamma_prev = dg;
            gamma = gnext;
        }

        // ---- rounding (Alg. 3) at gamma_f, cost <G, C> ----
        {
            const double inv_gamma = 1.0 / gf, G64 = gf * kLog2e;
            const float G32 = (float)G64, Glo = (float)(G64 - (double)G32);
            for (int i = tid; i < n; i += T) batch_prep_row(V[SV_U][i], row_scale(V[SV_LR][i]), inv_gamma, G64, sFh, sWr, sS, sA, i);
            for (int j = tid; j < n; j += T) {
                float gh, wl;
                split_cost_unit(V[SV_V][j] * inv_gamma, gh, wl, G64);
                Hh[j] = gh;
                Wc[j] = wl;
            }
            __syncthreads();
            // r(P) and x = min(r / r(P), 1); the column pass then weights row i by x_i 2^{A_i}
            batch_pass<true, COST>(P, Hh, Wc, sFh, sWr, sS, G32, Glo, sRow, colsum, V[SV_RS], tc, sStage);
            for (int i = tid; i < n; i += T) {
                const double rP = ldexp(V[SV_RS][i], sA[i]);
                const double xi = (rP > 0.0) ? fmin(P.r[i] / rP, 1.0) : 1.0;
                V[SV_GRT][i] = xi;
                sS[i] = (float)ldexp(xi, sA[i]);
            }
            __syncthreads();
            batch_pass<true, COST>(P, Hh, Wc, sFh, sWr, sS, G32, Glo, sRow, colsum, V[SV_RS], tc, sStage);   // colsum = c(F)
            for (int j = tid; j < n; j += T) {
                const double cF = (double)colsum[j];
                const double yj = (cF > 0.0) ? fmin(P.c[j] / cF, 1.0) : 1.0;
                V[SV_Y][j] = yj;
                V[SV_EC][j] = P.c[j] - cF * yj;
            }
            __syncthreads();
            // rows of F' = X P Y: r(F')_i, <F', C>_i and (C err_c)_i, one warp per row (fixed order)
#pragma unroll
            for (int q = 0; q < kNRed; ++q) x[q] = 0.0;
            for (int i = warp; i < n; i += nw) {
                const float fh = sFh[i], wr = sWr[i];
                double a0 = 0.0, a1 = 0.0, a2 = 0.0;
                for (int j = lane; j < n; j += 32) {
                    const float cv = batch_cost<COST>(P, i, j);
                    const float d = (fh + Hh[j]) - cv;
                    const double Ey = (double)exp2_acc(d, G32, Glo, wr + Wc[j]) * V[SV_Y][j];
                    a0 += Ey;
                    a1 = fma(Ey, (double)cv, a1);
                    a2 = fma((double)cv, V[SV_EC][j], a2);
                }
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) {
                    a0 += __shfl_xor_sync(0xffffffffu, a0, o);
                    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
                    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
                }
                if (lane == 0) {
                    const double xs = ldexp(V[SV_GRT][i], sA[i]);
                    const double er = P.r[i] - xs * a0;
                    x[0] += xs * a1;
                    x[1] += fabs(er);
                    x[2] += er * a2;
                }
            }
            block_reduce_nred(x, red_smem);
            if (tid == 0) res.cost = x[0] + ((x[1] > 0.0) ? x[2] / x[1] : 0.0);
        }

        // ---- c-transform lower bound from f = u / gamma_f, fp64 throughout (the gap estimate) ----
        {
            const double inv_gamma = 1.0 / gf;
            double* fv = V[SV_SRT];                      // free once the stages are over
            double* gv = V[SV_SCT];
            for (int i = tid; i < n; i += T) fv[i] = V[SV_U][i] * inv_gamma;
            __syncthreads();
            for (int j = tid; j < n; j += T) {           // g'_j = min_i (C_ij - f_i)
                double m = INFINITY;
                for (int i = 0; i < n; ++i) m = fmin(m, (double)batch_cost<COST>(P, i, j) - fv[i]);
                gv[j] = m;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kNRed; ++q) x[q] = 0.0;
            for (int i = warp; i < n; i += nw) {         // f'_i = min_j (C_ij - g'_j)
                double m = INFINITY;
                for (int j = lane; j < n; j += 32) m = fmin(m, (double)batch_cost<COST>(P, i, j) - gv[j]);
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (lane == 0) x[0] += m * P.r[i];
            }
            for (int j = tid; j < n; j += T) x[1] += gv[j] * P.c[j];
            block_reduce_nred(x, red_smem);
            if (tid == 0) res.lower_bound = x[0] + x[1];
        }
        for (int i = tid; i < n; i += T) {
            if (P.u_out) P.u_out[i] = V[SV_U][i];
            if (P.v_out) P.v_out[i] = V[SV_V][i];
        }
        __syncthreads();           // every output is written before the result (and done flag)
        if (tid == 0) {
            // a last stage that ended above its tolerance (by the stall rule) has not converged
            res.status = (st.status == ST_OK && !(st.gnorm <= tol_last)) ? (int)ST_CAP : st.status;
            res.stages = stages;
            res.evals = st.evals;
            res.iters = st.iters;
            res.grad_l1 = st.gnorm;
            res.gamma_f = gf;
            res.H_min = H;
            res.stalls = st.stalls;
            a.results[pi] = res;
            if (a.done) {
                __threadfence_system();
                reinterpret_cast<volatile int*>(a.done)[pi] = 1;
            }
        }
        __syncthreads();
    }
}

}  // namespace mdot
