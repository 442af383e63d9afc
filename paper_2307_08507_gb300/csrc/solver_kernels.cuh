// Cooperative kernels of the MDOT-PNCG solve: one launch runs one MDOT stage of Alg. 1
// (smoothing, warm start, then the PNCG projection of Alg. 2 with the App. B line search) entirely
// on the device.  Per evaluation: phase A (pass over C, row epilogue) -> grid barrier -> phase B
// (column merge, column epilogue, per-CTA partial sums) -> arrive; the last CTA reduces the
// partials in a fixed order and takes the line-search / PNCG decision -> phase C (commit the
// accepted step, new direction, constants of the next trial) -> grid barrier.
#pragma once

#include <cstddef>

#include "mdot_device.cuh"

namespace mdot {

// ---------------------------------------------------------------------------------------------
// decision of one evaluation (thread 0 of the last CTA).  tot = {phi', ||grad||_1,
// <y, -s>, <y, p>, <s, grad>, #bad}, y = grad_trial - grad_current (Eq. (18)).
// ---------------------------------------------------------------------------------------------
static __device__ void decide(State* S, const double* tot, const StageArgs& a)
{
    const double phi = tot[0], gn = tot[1], den = tot[3];
    // Sinkhorn direction (Eq. (17)), or the diagonal-Hessian one (Eq. (16)) when asked for and
    // every ratio allows it; tot[6..8] exist only where precond can be set
    const bool hess = a.precond && tot[8] == 0.0;
    const double num = hess ? tot[6] : tot[2], S1 = hess ? tot[7] : tot[4];
    const bool bad = tot[5] > 0.0 || !isfinite(phi) || !isfinite(gn);
    S->evals += 1;
    if (a.tier == TIER_F64) S->evals64 += 1;
    bool accept = false;
    if (S->kind == KIND_INIT) {
        if (bad) {
            S->status = max((int)S->status, (int)ST_NUMERIC);
            S->phase = PH_DONE;
            S->accept = 0;
            return;
        }
        accept = true;
    } else {
        S->ls_trials += 1;
        S->trials += 1;
        if (S->kind == KIND_FORCE) {
            accept = !bad;
            if (bad) {
                S->status = max((int)S->status, (int)ST_NUMERIC);
                S->phase = PH_DONE;
                S->accept = 0;
                return;
            }
        } else if (bad) {
            // overshoot into overflow: treat as an upper end and bisect (App. B reading)
            S->hi = S->alpha;
            S->dhi = INFINITY;
            S->alpha = 0.5 * (S->lo + S->hi);
        } else if (phi <= (2.0 * a.c1 - 1.0) * S->d0 && phi >= a.c2 * S->d0) {
            accept = true;                                      // Eq. (24)
        } else {
            if (phi < a.c2 * S->d0) { S->lo = S->alpha; S->dlo = phi; }
            else                    { S->hi = S->alpha; S->dhi = phi; }
            if (isinf(S->hi)) {
                S->alpha = 2.0 * S->alpha;
            } else if (isinf(S->dhi)) {
                S->alpha = 0.5 * (S->lo + S->hi);
            } else {
                const double a_sec = (S->lo * S->dhi - S->hi * S->dlo) / (S->dhi - S->dlo);  // Eq. (25)
                S->alpha = 0.5 * a_sec + 0.5 * (0.5 * (S->lo + S->hi));
            }
        }
        if (!accept && S->trials >= a.ls_max_trials) {
            if (S->lo > 0.0) {
                S->alpha = S->lo;
                S->kind = KIND_FORCE;
            } else {
                S->status = max((int)S->status, (int)ST_LSFAIL);
                S->phase = PH_DONE;
                S->accept = 0;
                return;
            }
        }
    }
    S->accept = accept ? 1 : 0;
    if (!accept) return;
    S->hess = hess ? 1 : 0;

    const bool was_init = (S->kind == KIND_INIT);
    S->alpha_commit = was_init ? 0.0 : S->alpha;
    if (!was_init) { S->k += 1; S->iters += 1; }
    S->gnorm = gn;
    if (gn <= a.tol) { S->phase = PH_DONE; S->beta = 0.0; return; }
    // stall rule: a stage whose tolerance lies within 4x of the noise floor of its arithmetic
    // (a.stall_below = stall_floor(tier)) stops after kStallIters accepted iterations without 1 %
    // progress; the host then continues from the iterate (the next stage, the fp64 polish of the
    // last stage) or reports MDOT_ERR_NOT_CONVERGED
    if (was_init || gn < 0.99 * S->best_gnorm) {
        S->best_gnorm = gn;
        S->since_best = 0;
    } else if (++S->since_best >= kStallIters && a.tol < a.stall_below) {
        S->stalls += 1;
        S->phase = PH_DONE;
        S->beta = 0.0;
        return;
    }
    if (S->k >= a.max_iter) {
        S->status = max((int)S->status, (int)ST_CAP);
        S->phase = PH_DONE;
        S->beta = 0.0;
        return;
    }
    // next direction p = s + beta p (Alg. 2, Eq. (18)), reset to s if not a descent direction
    double beta = 0.0;
    if (!was_init) {
        const double q = num / den;
        beta = (den != 0.0 && isfinite(q)) ? q : 0.0;
    }
    double pg = S1 + beta * phi;     // <s + beta p, grad> ; phi = <p_old, grad>
    if (pg >= 0.0) { beta = 0.0; pg = S1; }
    S->beta = beta;
    if (!(pg < 0.0)) {
        S->status = max((int)S->status, (int)ST_LSFAIL);
        S->phase = PH_DONE;
        return;
    }
    S->d0 = pg;
    S->lo = 0.0; S->dlo = pg; S->hi = INFINITY; S->dhi = INFINITY;
    // first trial step: 1, or the step just accepted clamped to [1/2, 2] (App. B leaves it open)
    S->alpha = (a.ls_init && !was_init) ? fmin(fmax(S->alpha_commit, 0.5), 2.0) : 1.0;
    S->trials = 0;
    S->kind = KIND_TRIAL;
}

// ---------------------------------------------------------------------------------------------
// shared-memory layout of the stage / dual-eval kernels
// ---------------------------------------------------------------------------------------------
struct SmemLayout {
    int nloc_max;
    size_t off_row, off_c0, off_c1, off_s, off_A, off_x, off_merge, off_ring, off_bars, off_misc,
        off_rstate, off_cstate, off_xc, off_pub, bytes;
    int stages;        // TMA ring slots (fp32 entries)
    bool pub;          // room for a copy of the published column state at off_pub
};

// per-row / per-column state of the CTA's own rows and columns, kept in shared memory for a stage
enum RowState { RS_U = 0, RS_P, RS_G, RS_T, RS_LT, RS_L, RS_GT, RS_ST, RS_LTR, RS_COUNT };
enum ColState { CS_V = 0, CS_P, CS_G, CS_T, CS_GT, CS_ST, CS_COUNT };

constexpr int kMergeGroups = 4;        // 32-column groups merged in one round trip by dual_eval_kernel

// Threads of the flag-synchronised stage kernel: 8 consumer warps (16 columns of a 4096-column
// ring segment each with dense C) and the producer warp.  (16 consumer warps with 8 columns each,
// at most 96 registers a thread, measured slower: 30.6 against 29.0 us per evaluation at n = 4096.)
constexpr int kFlagDenseThreads = kStageThreads;
__host__ __device__ constexpr int flag_threads(int cost) { return cost == COST_DENSE ? kFlagDenseThreads : kStageThreads; }

// wide: the merge scratch of merge_cols_f32_wide (standalone dual evaluation); pub_copy: room for
// the flag-synchronised stage kernel's copy of the published column state (dense C)
__host__ __device__ inline SmemLayout smem_layout(int n, int G, int tier, int nthreads, bool wide = false,
                                                  bool pub_copy = false)
{
    SmemLayout L;
    const int nw = nthreads / 32;
    L.nloc_max = (n + G - 1) / G + 1;
    const size_t el = (tier == TIER_F64) ? 8 : 4;
    size_t o = 0;
    L.off_row = o;   o += (size_t)nw * L.nloc_max * el;          o = (o + 15) & ~(size_t)15;
    L.off_c0 = o;    o += (size_t)L.nloc_max * el;               o = (o + 15) & ~(size_t)15;
    L.off_c1 = o;    o += (size_t)L.nloc_max * 4;                o = (o + 15) & ~(size_t)15;
    L.off_s = o;     o += (size_t)L.nloc_max * el;               o = (o + 15) & ~(size_t)15;
    L.off_A = o;     o += (size_t)L.nloc_max * 4;                o = (o + 15) & ~(size_t)15;
    L.off_x = o;     o += (size_t)L.nloc_max * 8;                o = (o + 15) & ~(size_t)15;
    // merge scratch: one 32-column group (stage kernels) or kMergeGroups of them plus their totals
    // (standalone evaluation, merge_cols_f32_wide)
    L.off_merge = o; o += !wide ? (size_t)2 * 32 * nw * 8
                                : (size_t)2 * kMergeGroups * 32 * nw * 4 + (size_t)kMergeGroups * 32 * 8;
    o = (o + 15) & ~(size_t)15;
    L.off_rstate = o; o += (size_t)RS_COUNT * L.nloc_max * 8;   o = (o + 15) & ~(size_t)15;
    L.off_cstate = o; o += (size_t)CS_COUNT * L.nloc_max * 8;   o = (o + 15) & ~(size_t)15;
    L.off_xc = o;    o += (size_t)3 * L.nloc_max * 4;           o = (o + 15) & ~(size_t)15;
    L.off_misc = o;  o += 16;
    L.off_bars = o;  o += (tier != TIER_F64) ? (size_t)2 * kStages * 8 : 0;   o = (o + 127) & ~(size_t)127;
    // stage kernels, fp32 entries, one ring segment: a copy of the published column state (float4
    // per column) that the flag-synchronised stage kernel fills while the decision is taken
    L.pub = pub_copy && !wide && tier != TIER_F64 && n <= kSegFloats;
    L.off_pub = o;   o += L.pub ? (size_t)kSegFloats * 16 : 0;
    L.off_ring = o;
    L.stages = 0;
    if (tier != TIER_F64) {
        const size_t room = (o < kSmemLimit) ? (kSmemLimit - o) / ((size_t)kSegFloats * 4) : 0;
        L.stages = (int)(room < (size_t)kStages ? room : (size_t)kStages);
        o += (size_t)L.stages * kSegFloats * 4;
    }
    L.bytes = o;
    return L;
}

// C_ij for the non-streaming passes (max passes, lower bound): dense load or regenerated.
template <int COST>
__device__ __forceinline__ float cost_elem(const WS& ws, int i, int j)
{
    if (COST == COST_DENSE) return __ldg(ws.C + (size_t)i * ws.n + j);
    return point_cost<COST>(__ldg(ws.X + 3 * (size_t)i), __ldg(ws.X + 3 * (size_t)i + 1), __ldg(ws.X + 3 * (size_t)i + 2),
                            __ldg(ws.Y + 3 * (size_t)j), __ldg(ws.Y + 3 * (size_t)j + 1), __ldg(ws.Y + 3 * (size_t)j + 2),
                            ws.cscale);
}

// coordinates of the CTA's rows into shared memory (regenerated cost)
template <int COST>
__device__ __forceinline__ void load_row_coords(const WS& ws, int r0, int r1, unsigned char* sm, size_t off)
{
    if (COST == COST_DENSE) return;
    float* sX = reinterpret_cast<float*>(sm + off);
    for (int q = threadIdx.x; q < 3 * (r1 - r0); q += blockDim.x) sX[q] = __ldg(ws.X + 3 * (size_t)r0 + q);
}

// Row prep of an evaluation at potential ua (already u + alpha p_u) with row scale A.
template <int TIER>
__device__ __forceinline__ void prep_row(double ua, int A, int Aglob, double gamma, double G64,
                                         unsigned char* sm, const SmemLayout& L, int il)
{
    if (TIER != TIER_F64) {
        float fh, wl;
        // (u - A ln2) / gamma, with the division replaced by a product with 1/gamma (exact to
        // fp64 rounding; fp64 division is slow on this GPU)
        split_cost_unit((ua - (double)A * kLn2) * (1.0 / gamma), fh, wl, G64);
        reinterpret_cast<float*>(sm + L.off_c0)[il] = fh;
        reinterpret_cast<float*>(sm + L.off_c1)[il] = wl;
        reinterpret_cast<float*>(sm + L.off_s)[il] = pow2f_int(A - Aglob);
    } else {
        reinterpret_cast<double*>(sm + L.off_c0)[il] = ua - (double)A * kLn2;
        reinterpret_cast<double*>(sm + L.off_s)[il] = ldexp(1.0, A - Aglob);
    }
    reinterpret_cast<int*>(sm + L.off_A)[il] = A;
}

template <int TIER>
__device__ __forceinline__ void prep_col(const WS& ws, int j, double va, double gamma, double G64)
{
    if (TIER != TIER_F64) {
        float gh, wl;
        split_cost_unit(va * (1.0 / gamma), gh, wl, G64);
        ws.Hh[j] = gh;
        ws.Wc[j] = wl;
    } else {
        ws.Hd[j] = va;
    }
}

// Phase A for the CTA's rows: pass over C (streamed or regenerated), row sums into sRow.
// io: where the column constants come from and the column partials go (plain arrays ordered by
// grid barriers, or tagged words).
template <int TIER, int COST, class IO>
__device__ __forceinline__ void phase_A(const WS& ws, const IO& io, int r0, int r1, double gamma, double G64,
                                        unsigned char* sm, const SmemLayout& L)
{
    const int n = ws.n, nloc = r1 - r0, nw = blockDim.x >> 5;
    const int b = blockIdx.x;
    if (TIER != TIER_F64) {
        float* sRow = reinterpret_cast<float*>(sm + L.off_row);
        for (int x = threadIdx.x; x < nw * L.nloc_max; x += blockDim.x) sRow[x] = 0.0f;
        __syncthreads();
        const float G32 = (float)G64;
        const float Glo = (float)(G64 - (double)G32);
        const float* sFh = reinterpret_cast<const float*>(sm + L.off_c0);
        const float* sWr = reinterpret_cast<const float*>(sm + L.off_c1);
        const float* sS = reinterpret_cast<const float*>(sm + L.off_s);
        // the tensor-core form stages its column blocks, and the A registers of its rows when there
        // is room, in the (unused) ring region
        const size_t room = (size_t)L.stages * kSegFloats, need = (size_t)tc_stage_floats(nw);
        if (COST == COST_SQEUCLID && ws.tc && room >= need)
            pass_f32_regen_tc<TIER == TIER_F32A>(
                ws.Y, ws.cscale, n, r0, r1, io, sFh, sWr, sS, reinterpret_cast<const float*>(sm + L.off_xc), G32,
                Glo, sRow, L.nloc_max, reinterpret_cast<float*>(sm + L.off_ring),
                room >= need + 8 * (size_t)L.nloc_max ? reinterpret_cast<uint2*>(sm + L.off_ring + 4 * need) : nullptr);
        else if (COST != COST_DENSE)
            pass_f32_regen<TIER == TIER_F32A, COST>(ws.Y, ws.cscale, n, r0, r1, io, sFh, sWr, sS,
                                                    reinterpret_cast<const float*>(sm + L.off_xc), G32, Glo,
                                                    sRow, L.nloc_max);
        else if ((n & 3) == 0 && (reinterpret_cast<uintptr_t>(ws.C) & 15) == 0 && blockDim.x == kStageThreads &&
            L.stages >= 2)
            pass_f32_tma<TIER == TIER_F32A>(ws.C, n, r0, r1, io, sFh, sWr, sS, G32, Glo, sRow, L.nloc_max,
                         reinterpret_cast<float*>(sm + L.off_ring), L.stages,
                         reinterpret_cast<unsigned long long*>(sm + L.off_bars),
                         reinterpret_cast<int*>(sm + L.off_misc), &ws.st->bar.abort);
        else if ((n & 3) == 0)
            pass_f32<true, TIER == TIER_F32A>(ws.C, n, r0, r1, io, sFh, sWr, sS, G32, Glo, sRow, L.nloc_max);
        else
            pass_f32<false, TIER == TIER_F32A>(ws.C, n, r0, r1, io, sFh, sWr, sS, G32, Glo, sRow, L.nloc_max);
    } else {
        double* sRow = reinterpret_cast<double*>(sm + L.off_row);
        for (int x = threadIdx.x; x < nw * L.nloc_max; x += blockDim.x) sRow[x] = 0.0;
        __syncthreads();
        if (COST != COST_DENSE)
            pass_f64_regen<COST>(ws.Y, ws.cscale, n, r0, r1, ws.Hd, reinterpret_cast<const double*>(sm + L.off_c0),
                                 reinterpret_cast<const double*>(sm + L.off_s),
                                 reinterpret_cast<const float*>(sm + L.off_xc), gamma, sRow, L.nloc_max,
                                 ws.colpartd + (size_t)b * n);
        else
            pass_f64(ws.C, n, r0, r1, ws.Hd, reinterpret_cast<const double*>(sm + L.off_c0),
                     reinterpret_cast<const double*>(sm + L.off_s), gamma, sRow, L.nloc_max,
                     ws.colpartd + (size_t)b * n);
    }
    __syncthreads();
    (void)nloc;
}

template <int TIER>
__device__ __forceinline__ double row_total(const unsigned char* sm, const SmemLayout& L, int il)
{
    const int nw = blockDim.x >> 5;
    double s = 0.0;
    if (TIER != TIER_F64) {
        const float* sRow = reinterpret_cast<const float*>(sm + L.off_row);
        for (int w = 0; w < nw; ++w) s += (double)sRow[w * L.nloc_max + il];
    } else {
        const double* sRow = reinterpret_cast<const double*>(sm + L.off_row);
        for (int w = 0; w < nw; ++w) s += sRow[w * L.nloc_max + il];
    }
    return s;
}

// Eq. (16): the diagonal-Hessian direction s_h = r~ / r(P) - 1 = exp(s) - 1 with s of Eq. (17),
// taken where every ratio r~ / r(P), c~ / c(P) lies in [0.01, 100] (otherwise s itself)
constexpr double kLogRatioLo = -4.605170185988091;     // log 0.01
constexpr double kLogRatioHi = 4.605170185988091;      // log 100
__device__ __forceinline__ double hess_dir(double s) { return (double)expm1f((float)s); }
__device__ __forceinline__ double dir_of(double s, bool hess) { return hess ? hess_dir(s) : s; }
__device__ __forceinline__ void hess_terms(double s, double g, double y, double (&x)[kNRedP])
{
    const double sh = hess_dir(s);
    x[6] += y * (-sh);
    x[7] += sh * g;
    if (!(s >= kLogRatioLo && s <= kLogRatioHi)) x[8] += 1.0;
}

// ---------------------------------------------------------------------------------------------
// the stage kernel
// ---------------------------------------------------------------------------------------------
// words of State before the grid barrier (the part the decision reads and writes)
constexpr int kStateWords = (int)(offsetof(State, bar) / 8);

template <int TIER, int COST>
__global__ void __launch_bounds__(kStageThreads, 1) stage_kernel(WS ws, StageArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double red_smem[32 * kNRedP];
    __shared__ double s_bc[8];
    __shared__ int s_flag[2];
    __shared__ unsigned int s_gen;

    const int n = ws.n, G = ws.G, b = blockIdx.x, T = blockDim.x, tid = threadIdx.x;
    const SmemLayout L = smem_layout(n, G, TIER, T);
    int r0, r1, c0, c1;
    row_range(n, G, b, r0, r1);
    row_range(n, G, b, c0, c1);
    const int NL = L.nloc_max;
    double* R = reinterpret_cast<double*>(sm + L.off_rstate);     // R[k * NL + local row]
    double* Q = reinterpret_cast<double*>(sm + L.off_cstate);     // Q[k * NL + local column]
    const double gamma = a.gamma, G64 = a.G64, w = a.w;
    State* S = ws.st;

    if (tid == 0) s_gen = ld_acquire(&S->bar.gen);
    load_row_coords<COST>(ws, r0, r1, sm, L.off_xc);
    __syncthreads();
    unsigned int gen = s_gen;

    // ---- prologue (Alg. 1): smoothing, rank-one start or warm start, constants at alpha = 0 ----
    for (int i = r0 + tid; i < r1; i += T) {
        const int il = i - r0;
        const double rt = (1.0 - w / 4.0) * ws.r[i] + w / (4.0 * n);
        const double lrt = log(rt);
        double u = ws.u[i];
        if (a.first) {
            u = lrt;
            ws.uprev[i] = u;
        } else if (a.warm_start == 0) {
            const double z = u;
            u = z + a.ratio * (z - ws.uprev[i]);             // Eq. (13)
            ws.uprev[i] = z;
        } else if (a.warm_start == 1) {
            u = a.ratio * u;                                    // eps-scaling
        }
        R[RS_U * NL + il] = u;
        R[RS_P * NL + il] = 0.0;
        R[RS_G * NL + il] = 0.0;
        R[RS_T * NL + il] = rt;
        R[RS_LT * NL + il] = lrt;
        R[RS_L * NL + il] = lrt;
        prep_row<TIER>(u, row_scale(lrt), a.Aglob, gamma, G64, sm, L, il);
    }
    for (int j = c0 + tid; j < c1; j += T) {
        const int jl = j - c0;
        const double ct = (1.0 - w / 4.0) * ws.c[j] + w / (4.0 * n);
        double v = ws.v[j];
        if (a.first) {
            v = log(ct);
            ws.vprev[j] = v;
        } else if (a.warm_start == 0) {
            const double z = v;
            v = z + a.ratio * (z - ws.vprev[j]);
            ws.vprev[j] = z;
        } else if (a.warm_start == 1) {
            v = a.ratio * v;
        }
        Q[CS_V * NL + jl] = v;
        Q[CS_P * NL + jl] = 0.0;
        Q[CS_G * NL + jl] = 0.0;
        Q[CS_T * NL + jl] = ct;
        prep_col<TIER>(ws, j, v, gamma, G64);
    }
    if (b == 0 && tid == 0) {
        S->alpha = 0.0;
        S->kind = KIND_INIT;
        S->accept = 0;
        S->trials = 0;
        S->k = 0;
        S->phase = PH_RUN;
        S->beta = 0.0;
        S->alpha_commit = 0.0;
    }
    if (!grid_sync(&S->bar, G, gen, s_flag)) goto finish;

    for (;;) {
        // ---------------- phase A: pass over own rows, row epilogue ----------------
        phase_A<TIER, COST>(ws, ColPlain{ws.Hh, ws.Wc, ws.colpart + (size_t)b * n}, r0, r1, gamma, G64, sm, L);
        double x[kNRedP];
#pragma unroll
        for (int q = 0; q < kNRedP; ++q) x[q] = 0.0;
        {
            const int* sA = reinterpret_cast<const int*>(sm + L.off_A);
            for (int i = r0 + tid; i < r1; i += T) {
                const int il = i - r0;
                const double sum = row_total<TIER>(sm, L, il);
                if (!(sum > 0.0) || !isfinite(sum)) { x[5] += 1.0; continue; }
                const double rt = R[RS_T * NL + il];
                const double g = ldexp(sum, sA[il]) - rt;
                // Eq. (17): s = log r~ - log r(P) = -log1p(g / r~); this form keeps the sign of s
                // opposite to g, so <s, grad> < 0 (Sec. 4) holds numerically.  s is a search
                // direction: fp32 accuracy suffices (fp64 transcendentals cost ~16 cycles per warp
                // instruction on this GPU); the gradient g and every dot product stay fp64.
                const double s = -(double)log1pf((float)g / (float)rt);
                const double p = R[RS_P * NL + il];
                const double y = g - R[RS_G * NL + il];
                x[0] += p * g;
                x[1] += fabs(g);
                x[2] += y * (-s);
                x[3] += y * p;
                x[4] += s * g;
                if (a.precond) hess_terms(s, g, y, x);
                R[RS_GT * NL + il] = g;
                R[RS_ST * NL + il] = s;
                R[RS_LTR * NL + il] = ((double)__log2f((float)sum) + (double)sA[il]) * kLn2;   // scale only
            }
        }
        if (!grid_sync(&S->bar, G, gen, s_flag)) goto finish;

        // ---------------- phase B: column merge and epilogue ----------------
        for (int j0 = c0; j0 < c1; j0 += 32) {
            double colsum;
            if (TIER != TIER_F64)
                colsum = merge_cols_f32(ws.colpart, n, G, j0, c1, reinterpret_cast<float*>(sm + L.off_merge));
            else
                colsum = merge_cols_f64(ws.colpartd, n, G, j0, c1, reinterpret_cast<double*>(sm + L.off_merge));
            const int j = j0 + tid;
            if (tid < 32 && j < c1) {
                if (!(colsum > 0.0) || !isfinite(colsum)) { x[5] += 1.0; continue; }
                const int jl = j - c0;
                const double ct = Q[CS_T * NL + jl];
                const double g = ldexp(colsum, a.Aglob) - ct;
                const double s = -(double)log1pf((float)g / (float)ct);   // Eq. (17), see rows
                const double p = Q[CS_P * NL + jl];
                const double y = g - Q[CS_G * NL + jl];
                x[0] += p * g;
                x[1] += fabs(g);
                x[2] += y * (-s);
                x[3] += y * p;
                x[4] += s * g;
                if (a.precond) hess_terms(s, g, y, x);
                Q[CS_GT * NL + jl] = g;
                Q[CS_ST * NL + jl] = s;
            }
        }
        block_reduce_nred(x, red_smem);
        if (tid == 0) {
#pragma unroll
            for (int q = 0; q < kNRedP; ++q) ws.blockred[(size_t)b * kNRedP + q] = x[q];
        }

        // ---------------- reduction + decision by the last CTA ----------------
        ++gen;
        if (bar_arrive(&S->bar, G, s_flag)) {
            __threadfence();
            // warp q sums scalar q over the G CTAs in a fixed order; all loads issued first
            const int lane = tid & 31, warp = tid >> 5;
            if (warp < (a.precond ? kNRedP : kNRed)) {
                double v8[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int bb = lane + 32 * k;
                    v8[k] = (bb < G) ? __ldcg(ws.blockred + (size_t)bb * kNRedP + warp) : 0.0;
                }
                double sacc = 0.0;
#pragma unroll
                for (int k = 0; k < 8; ++k) sacc += v8[k];
#pragma unroll
                for (int o = 16; o >= 1; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
                if (lane == 0) red_smem[warp] = sacc;
            }
            __syncthreads();
            if (tid == 0) {
                double tot[kNRedP];
                for (int q = 0; q < kNRedP; ++q) tot[q] = a.precond ? red_smem[q] : (q < kNRed ? red_smem[q] : 0.0);
                // decide on a local copy: one pipelined load and one store of the state words
                State loc;
                unsigned long long* lw = reinterpret_cast<unsigned long long*>(&loc);
                const volatile unsigned long long* sw = reinterpret_cast<const volatile unsigned long long*>(S);
#pragma unroll
                for (int k = 0; k < kStateWords; ++k) lw[k] = sw[k];
                decide(&loc, tot, a);
                volatile unsigned long long* dw = reinterpret_cast<volatile unsigned long long*>(S);
#pragma unroll
                for (int k = 0; k < kStateWords; ++k) dw[k] = lw[k];
                bar_release(&S->bar, gen);
            }
        }
        if (!bar_wait(&S->bar, gen, s_flag)) goto finish;
        if (tid == 0) {
            const volatile State* vS = S;
            const double d0 = vS->alpha, d1 = vS->alpha_commit, d2 = vS->beta;
            const int i3 = vS->accept, i4 = vS->phase, i5 = vS->hess;
            s_bc[0] = d0;
            s_bc[1] = d1;
            s_bc[2] = d2;
            s_bc[3] = (double)i3;
            s_bc[4] = (double)i4;
            s_bc[5] = (double)i5;
        }
        __syncthreads();
        const double alpha = s_bc[0], acommit = s_bc[1], beta = s_bc[2];
        const bool accept = s_bc[3] != 0.0, done = s_bc[4] != 0.0, hess = s_bc[5] != 0.0;

        // ---------------- phase C: commit, new direction, next trial constants ----------------
        for (int i = r0 + tid; i < r1; i += T) {
            const int il = i - r0;
            double u = R[RS_U * NL + il], p = R[RS_P * NL + il];
            if (accept) {
                u = u + acommit * p;                            // (u, v) += alpha p (Alg. 2)
                R[RS_U * NL + il] = u;
                R[RS_G * NL + il] = R[RS_GT * NL + il];
                R[RS_L * NL + il] = R[RS_LTR * NL + il];
                p = dir_of(R[RS_ST * NL + il], hess) + beta * p;   // p = s + beta p, beta = 0 on reset (Alg. 2)
                R[RS_P * NL + il] = p;
            }
            if (!done) prep_row<TIER>(u + alpha * p, row_scale(R[RS_L * NL + il] + alpha * p), a.Aglob,
                                      gamma, G64, sm, L, il);
        }
        for (int j = c0 + tid; j < c1; j += T) {
            const int jl = j - c0;
            double v = Q[CS_V * NL + jl], p = Q[CS_P * NL + jl];
            if (accept) {
                v = v + acommit * p;
                Q[CS_V * NL + jl] = v;
                Q[CS_G * NL + jl] = Q[CS_GT * NL + jl];
                p = dir_of(Q[CS_ST * NL + jl], hess) + beta * p;
                Q[CS_P * NL + jl] = p;
            }
            if (!done) prep_col<TIER>(ws, j, v + alpha * p, gamma, G64);
        }
        if (done) break;
        if (!grid_sync(&S->bar, G, gen, s_flag)) goto finish;
    }
finish:
    // the stage's iterate (also on a timeout: the best iterate so far) goes back to global memory
    __syncthreads();
    for (int i = r0 + tid; i < r1; i += T) {
        ws.u[i] = R[RS_U * NL + i - r0];
        ws.lr[i] = R[RS_L * NL + i - r0];
    }
    for (int j = c0 + tid; j < c1; j += T) ws.v[j] = Q[CS_V * NL + j - c0];
    if (tid == 0 && *reinterpret_cast<volatile unsigned int*>(&S->bar.abort)) {
        atomicMax(&S->status, (int)ST_TIMEOUT);
        S->phase = PH_DONE;
    }
}

// ---------------------------------------------------------------------------------------------
// the stage kernel without grid barriers (fp32-entry tiers): the same evaluation sequence as
// stage_kernel with two hand-offs per evaluation, neither through a central counter or a last
// arriver:
//   fcp[b]: a per-CTA flag, CTA b's column partials are written (read by every column owner);
//   tsp[b]: CTA b's partial sums of the six scalars as tagged words (each word is its own ready
//           flag), read by every CTA, with fpub[b]: CTA b's column state is published (the
//           committed (v, p) and the new direction s of its columns), awaited in parallel.
// Each CTA reduces the G scalar partials in the same fixed order and takes the line-search /
// PNCG decision on its own copy of the stage state, so all copies stay identical.  Every consumer
// thread then derives the next trial's constants of its own columns from the published column
// state and that decision (double-float arithmetic, identical in every CTA), so the column
// constants never travel between CTAs.  The fp64 epilogues stay packed into as few warps as
// possible: on this GPU an fp64 warp instruction holds the SM's fp64 pipe for ~16 cycles however
// few of its lanes are active.
// ---------------------------------------------------------------------------------------------

// Publish `tag` in flag (thread 0, after a __syncthreads that follows the CTA's data writes): a
// release store, so every write the CTA made before the barrier is visible to a reader that
// observes the tag.
__device__ __forceinline__ void post_flag(unsigned int* flag, unsigned int tag)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(flag), "r"(tag) : "memory");
}

// One warp waits (bounded) until every flags[0..G) has reached tag; false if it gave up.
__device__ __forceinline__ bool wait_flags(const unsigned int* flags, int G, unsigned int tag, GridBar* gb)
{
    const int lane = threadIdx.x & 31;
    unsigned int spins = 0;
    unsigned long long deadline = 0;
    for (;;) {
        bool ready = true;
        for (int b = lane; b < G; b += 32) {
            unsigned int f;
            asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(f) : "l"(flags + b) : "memory");
            ready = ready && (int)(f - tag) >= 0;
        }
        if (__all_sync(0xffffffffu, ready)) {
            asm volatile("fence.acq_rel.gpu;" ::: "memory");     // acquire for the relaxed polls
            return true;
        }
        const bool go_on = wait_backoff(spins, deadline, gb);
        if (!__all_sync(0xffffffffu, go_on)) return false;
    }
}

// Warp 0 waits on the flags; the whole CTA learns the outcome (s_ok) after a __syncthreads.
__device__ __forceinline__ bool cta_wait_flags(const unsigned int* flags, int G, unsigned int tag,
                                               GridBar* gb, int* s_ok)
{
    if (threadIdx.x < 32) {
        const bool ok = wait_flags(flags, G, tag, gb);
        if (threadIdx.x == 0 && !ok) *s_ok = 0;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Row constants of a trial point u + alpha p in the fp32-entry stage kernel, from the row's
// double-float state (the arithmetic of col_publish, no fp64): the row scale A from the predicted
// log r(P) (log_r + alpha p), then x = (u + alpha p - A ln 2) / gamma in cost units split into a
// part quantised to 2^-21 (fh) and the remainder in exponent units (wr).
__device__ __forceinline__ void prep_row_df(float2 u, float2 p, float alpha, float log_r, int Aglob,
                                            float2 inv_gamma, float G32, float Glo, unsigned char* sm,
                                            const SmemLayout& L, int il)
{
    const float2 ua = df_add(u, df_mul_f(p, alpha));
    float a = rintf(__fmul_rn(__fmaf_rn(alpha, p.x, log_r), (float)kLog2e));
    a = fminf(fmaxf(a, -1.0e6f), 1.0e6f);
    const int A = (int)a;
    // A ln 2 as a double-float: the product with ln 2's leading float is exact inside the fma
    const float l2h = (float)kLn2, l2l = (float)(kLn2 - (double)(float)kLn2);
    const float ph = __fmul_rn(a, l2h);
    const float2 aln2 = df_fast_two_sum(ph, __fmaf_rn(a, l2l, __fmaf_rn(a, l2h, -ph)));
    const float2 x = df_mul(df_add(ua, df_neg(aln2)), inv_gamma);
    const float h = __fmul_rn(rintf(__fmul_rn(x.x, 2097152.0f)), 1.0f / 2097152.0f);
    const float lo = __fadd_rn(__fsub_rn(x.x, h), x.y);       // x.x - h is exact
    reinterpret_cast<float*>(sm + L.off_c0)[il] = h;
    reinterpret_cast<float*>(sm + L.off_c1)[il] = __fmaf_rn(lo, G32, __fmul_rn(lo, Glo));
    reinterpret_cast<float*>(sm + L.off_s)[il] = pow2f_int(A - Aglob);
    reinterpret_cast<int*>(sm + L.off_A)[il] = A;
}

// Epilogue of one row or column in the fp32-entry stage kernel, without fp64 (an fp64 warp
// instruction holds this GPU's small fp64 pipe for many cycles, and these epilogues sit on the
// critical path of every evaluation).  sum: the fp32 row (column) sum as a double-float, A its
// power-of-two scale, t the smoothed marginal r~_i (c~_j) as a double-float, p the direction,
// gprev the gradient entry at the current point.  The marginal sum 2^A and the gradient entry
// g = r(P)_i - r~_i are formed in double-float (the difference is exact), the Sinkhorn direction
// s = -log1p(g / r~) (Eq. (17); the sign of s is opposite to that of g, Sec. 4) in fp32, and the
// five terms of the evaluation's scalars (<p, grad>, ||grad||_1, <y, -s>, <y, p>, <s, grad>,
// y = grad - grad_prev, Eq. (18)) are fp32 products added into double-float sums.  The fp32
// rounding of a term (2^-24 relative) is below the error the fp32 entries already leave in the
// marginal.  Returns false for a row (column) whose sum is not positive and finite.
__device__ __forceinline__ bool epi_entry(float2 sum, int A, float2 t, float p, float gprev, float2 (&xs)[kNRed],
                                          float& g_out, float& s_out)
{
    if (!(sum.x > 0.0f) || !isfinite(sum.x)) {
        xs[5] = df_add_f(xs[5], 1.0f);
        return false;
    }
    const float2 m = (A >= -126 && A <= 127) ? df_ldexp(sum, A)
                                             : make_float2((float)ldexp((double)sum.x, A), 0.0f);
    const float g = df_add(m, df_neg(t)).x;
    const float sdir = -log1pf(g / t.x);
    const float y = __fsub_rn(g, gprev);
    xs[0] = df_add_f(xs[0], __fmul_rn(p, g));
    xs[1] = df_add_f(xs[1], fabsf(g));
    xs[2] = df_add_f(xs[2], __fmul_rn(y, -sdir));
    xs[3] = df_add_f(xs[3], __fmul_rn(y, p));
    xs[4] = df_add_f(xs[4], __fmul_rn(sdir, g));
    g_out = g;
    s_out = sdir;
    return true;
}

// Phase timers of stage_kernel_flag (diagnostic; only in a library built with
// -DMDOT_PHASE_TIMERS, read by mdot_phase_timers): thread 0 of every CTA adds the SM cycles
// since its previous mark to the phase's counter.  Phases: 0 loop top, 1 pass, 2 row epilogue,
// 3 wait for the column partials, 4 merge and column epilogue, 5 CTA reduction and publication,
// 6 wait for the scalar partials, 7 decision, 8 commit and next row constants; counter 9 counts
// the evaluations.
constexpr int kPhases = 9;
constexpr int kPhaseCtas = 160;
#ifdef MDOT_PHASE_TIMERS
static __device__ unsigned long long g_phase[kPhaseCtas][kPhases + 1];
#define MDOT_PHASE(k)                                                                        \
    do {                                                                                     \
        if (threadIdx.x == 0 && blockIdx.x < kPhaseCtas) {                                   \
            const unsigned long long t_ = clock64();                                         \
            g_phase[blockIdx.x][k] += t_ - ph_last;                                          \
            ph_last = t_;                                                                    \
        }                                                                                    \
    } while (0)
#else
#define MDOT_PHASE(k) do { } while (0)
#endif

template <int TIER, int COST>
__global__ void __launch_bounds__(flag_threads(COST), 1) stage_kernel_flag(WS ws, StageArgs a)
{
    static_assert(TIER != TIER_F64, "the flag-synchronised stage kernel carries fp32 partials");
    constexpr int kCons = flag_threads(COST) - 32;      // consumer threads; the producer warp follows
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ float2 red_smem[32 * kNRed];
    __shared__ double tot_smem[kNRed];
    __shared__ State sst;                 // this CTA's copy of the stage state
    __shared__ ColStep s_step;            // the last decision, as the column arithmetic uses it
    __shared__ unsigned int s_base;
    __shared__ int s_ok;

    const int n = ws.n, G = ws.G, b = blockIdx.x, T = blockDim.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const SmemLayout L = smem_layout(n, G, TIER, T, false, COST == COST_DENSE);
    int r0, r1, c0, c1;
    row_range(n, G, b, r0, r1);
    row_range(n, G, b, c0, c1);
    const int NL = L.nloc_max, nrl = r1 - r0;
    double* R = reinterpret_cast<double*>(sm + L.off_rstate);     // R[k * NL + local row]
    double* Q = reinterpret_cast<double*>(sm + L.off_cstate);     // Q[k * NL + local column]
    float2* QV = reinterpret_cast<float2*>(Q + CS_V * NL);        // column v and p as double-floats
    float2* QP = reinterpret_cast<float2*>(Q + CS_P * NL);
    // float views of the state slots: gradients (RS_G, RS_GT, CS_G, CS_GT) and directions (RS_ST,
    // CS_ST) as floats, the smoothed marginals (RS_T, CS_T) as double-floats
    float* RF = reinterpret_cast<float*>(R);
    float* QF = reinterpret_cast<float*>(Q);
    float2* RT = reinterpret_cast<float2*>(R + RS_T * NL);
    float2* QT = reinterpret_cast<float2*>(Q + CS_T * NL);
    // rows mirror the columns: u and p as double-floats, log r(P) as floats
    float2* RU = reinterpret_cast<float2*>(R + RS_U * NL);
    float2* RP = reinterpret_cast<float2*>(R + RS_P * NL);
    const double gamma = a.gamma, G64 = a.G64, w = a.w;
    const float G32 = (float)G64, Glo = (float)(G64 - (double)G32);
    const float2 inv_gamma = df_from_double(1.0 / gamma);
    unsigned int* abort = &ws.st->bar.abort;
    unsigned int* fcp = ws.flags;
    unsigned int* fpub = ws.flags + G;      // the column state is published (prologue included)
    // warps holding epilogue sums: rows sit in threads 0 .. nrl - 1, columns in warp 0
    const int red_warps = max(1, min((nrl + 31) / 32, T / 32));
    unsigned int t = 0;                   // evaluations of this launch so far
    // dense C streamed through a TMA ring that stays alive over the launch (see pass_f32_ring)
    const bool use_ring = COST == COST_DENSE && (n & 3) == 0 && (reinterpret_cast<uintptr_t>(ws.C) & 15) == 0 &&
                          T == flag_threads(COST) && L.stages >= 2;
    RingGeom ring{ws.C, n, r0, nrl, (n + kSegFloats - 1) / kSegFloats, L.stages,
                  reinterpret_cast<float*>(sm + L.off_ring), reinterpret_cast<unsigned long long*>(sm + L.off_bars),
                  reinterpret_cast<unsigned long long*>(sm + L.off_bars) + kStages};
    int consumed = 0, issued = 0;
    // the owners' published column state (one segment: n <= kSegFloats) is bulk-copied into shared
    // memory as soon as its flags are seen, while the scalar partials are awaited and the decision
    // is taken; the next pass derives its column constants from that copy
    float4* sPub = reinterpret_cast<float4*>(sm + L.off_pub);
    __shared__ __align__(8) unsigned long long s_pub_bar;
    __shared__ unsigned int s_pub_issued;            // copies issued (written by the issuing lane only)
    const bool prefetch = use_ring && L.pub;
    unsigned int pub_used = 0;                       // copies consumed by passes (uniform in the CTA)

    if (tid == 0) {
        s_base = *reinterpret_cast<volatile unsigned int*>(ws.epoch);
        const volatile unsigned long long* src = reinterpret_cast<const volatile unsigned long long*>(ws.st);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sst);
        for (int k = 0; k < kStateWords; ++k) dst[k] = src[k];
        sst.alpha = 0.0;
        sst.kind = KIND_INIT;
        sst.accept = 0;
        sst.trials = 0;
        sst.k = 0;
        sst.phase = PH_RUN;
        sst.beta = 0.0;
        sst.alpha_commit = 0.0;
        s_step = ColStep{0, 0.0f, 0.0f, 0.0f};
        s_ok = 1;
    }
    if (use_ring) ring_init<kCons>(ring);
    if (prefetch && tid == 0) {
        mbar_init(&s_pub_bar, 1);
        mbar_fence_init();
    }
    if (tid == 0) s_pub_issued = 0;
    load_row_coords<COST>(ws, r0, r1, sm, L.off_xc);
    __syncthreads();
    const unsigned int base = s_base;
    // the first rows of the first pass load while the prologue runs
    if (use_ring && tid == kCons && !ring_issue(ring, issued, ring.nst)) atomicExch(abort, 1u);

    // ---- prologue (Alg. 1): smoothing, rank-one start or warm start, constants at alpha = 0 ----
    for (int i = r0 + tid; i < r1; i += T) {
        const int il = i - r0;
        const double rt = (1.0 - w / 4.0) * ws.r[i] + w / (4.0 * n);
        const double lrt = log(rt);
        double u = ws.u[i];
        if (a.first) {
            u = lrt;
            ws.uprev[i] = u;
        } else if (a.warm_start == 0) {
            const double z = u;
            u = z + a.ratio * (z - ws.uprev[i]);             // Eq. (13)
            ws.uprev[i] = z;
        } else if (a.warm_start == 1) {
            u = a.ratio * u;                                    // eps-scaling
        }
        RU[il] = df_from_double(u);
        RP[il] = make_float2(0.0f, 0.0f);
        RF[RS_G * 2 * NL + il] = 0.0f;                 // gradients: floats
        RT[il] = df_from_double(rt);                    // r~ as a double-float
        RF[RS_L * 2 * NL + il] = (float)lrt;
        prep_row_df(RU[il], RP[il], 0.0f, (float)lrt, a.Aglob, inv_gamma, G32, Glo, sm, L, il);
    }
    for (int j = c0 + tid; j < c1; j += T) {
        const int jl = j - c0;
        const double ct = (1.0 - w / 4.0) * ws.c[j] + w / (4.0 * n);
        double v = ws.v[j];
        if (a.first) {
            v = log(ct);
            ws.vprev[j] = v;
        } else if (a.warm_start == 0) {
            const double z = v;
            v = z + a.ratio * (z - ws.vprev[j]);
            ws.vprev[j] = z;
        } else if (a.warm_start == 1) {
            v = a.ratio * v;
        }
        QV[jl] = df_from_double(v);
        QP[jl] = make_float2(0.0f, 0.0f);
        QF[CS_G * 2 * NL + jl] = 0.0f;
        QT[jl] = df_from_double(ct);                    // c~ as a double-float
        QF[CS_ST * 2 * NL + jl] = 0.0f;
        ws.pub[j] = col_publish(QV[jl], QP[jl], 0.0f, inv_gamma, G32, Glo);
    }
    // tags: base + 1 for this prologue, base + 2 + t for evaluation t (flags start at 0, and every
    // tag of an earlier launch is at most its base + t + 3 <= this base)
    __syncthreads();
    if (tid == 0) post_flag(fpub + b, base + 1u);
    cta_wait_flags(fpub, G, base + 1u, &ws.st->bar, &s_ok);

#ifdef MDOT_PHASE_TIMERS
    unsigned long long ph_last = clock64();
#endif
    for (; s_ok; ++t) {
        const unsigned int tag = base + 2u + t;
#ifdef MDOT_PHASE_TIMERS
        if (tid == 0 && b < kPhaseCtas) g_phase[b][kPhases] += 1;
#endif
        MDOT_PHASE(0);
        // ---------------- phase A: pass over own rows; column constants derived in place ----------------
        {
            const float2 kk = col_step_coeffs(s_step);
            const ColDelta io{ws.pub, ws.colpart + (size_t)b * n, kk.x, kk.y};
            if (use_ring) {
                float* sRow = reinterpret_cast<float*>(sm + L.off_row);
                for (int x = tid; x < (T >> 5) * NL; x += T) sRow[x] = 0.0f;
                __syncthreads();
                const bool from_copy = pub_used < s_pub_issued;   // read after a barrier
                pass_f32_ring<TIER == TIER_F32A, kCons>(ring, r1, io, from_copy ? sPub : nullptr, &s_pub_bar,
                                                 pub_used & 1u,
                                                 reinterpret_cast<const float*>(sm + L.off_c0),
                                                 reinterpret_cast<const float*>(sm + L.off_c1),
                                                 reinterpret_cast<const float*>(sm + L.off_s), G32, Glo, sRow, NL,
                                                 consumed, issued, abort);
                if (from_copy) ++pub_used;
            } else if (COST != COST_DENSE) {
                phase_A<TIER, COST>(ws, io, r0, r1, gamma, G64, sm, L);
            }
            // (dense C that the ring cannot stream -- n not a multiple of 4, C not 16-byte aligned,
            // no room for two slots -- is solved by the barrier-synchronised stage kernel instead:
            // flag_stage_ok below)
        }
        MDOT_PHASE(1);
        if (tid == 0) post_flag(fcp + b, tag);             // phase_A ends with a __syncthreads
        float2 x[kNRed];
#pragma unroll
        for (int q = 0; q < kNRed; ++q) x[q] = make_float2(0.0f, 0.0f);
        {
            const int* sA = reinterpret_cast<const int*>(sm + L.off_A);
            const float* sRow = reinterpret_cast<const float*>(sm + L.off_row);
            for (int i = r0 + tid; i < r1; i += T) {
                const int il = i - r0;
                float2 sum = make_float2(0.0f, 0.0f);           // the warps' partials, double-float
                for (int w = 0; w < (T >> 5); ++w) sum = df_add_f(sum, sRow[w * NL + il]);   // every warp's slot
                float g, sd;
                if (!epi_entry(sum, sA[il], RT[il], RP[il].x, RF[RS_G * 2 * NL + il], x, g, sd))
                    continue;
                RF[RS_GT * 2 * NL + il] = g;
                RF[RS_ST * 2 * NL + il] = sd;
                // log r(P), for the next row scale only
                RF[RS_LTR * 2 * NL + il] = __fmul_rn(__log2f(sum.x) + (float)sA[il], (float)kLn2);
            }
        }

        MDOT_PHASE(2);
        // ---------------- phase B: column merge and epilogue; publish the column state ----------------
        if (!cta_wait_flags(fcp, G, tag, &ws.st->bar, &s_ok)) break;
        MDOT_PHASE(3);
        for (int j0 = c0; j0 < c1; j0 += 32) {
            const float2 colsum = merge_cols_f32_df(ws.colpart, n, G, j0, c1, reinterpret_cast<float*>(sm + L.off_merge));
            const int j = j0 + tid;
            if (tid < 32 && j < c1) {
                const int jl = j - c0;
                float g, sf = 0.0f;
                if (epi_entry(colsum, a.Aglob, QT[jl], QP[jl].x, QF[CS_G * 2 * NL + jl], x, g, sf))
                    QF[CS_GT * 2 * NL + jl] = g;
                else
                    sf = 0.0f;
                QF[CS_ST * 2 * NL + jl] = sf;
                ws.pub[j] = col_publish(QV[jl], QP[jl], sf, inv_gamma, G32, Glo);
            }
        }
        MDOT_PHASE(4);
        // CTA partial sums (double-floats): only the warps that hold rows (columns sit in warp 0)
        if (red_warps == 1) {
            // every partial sits in warp 0 (at most 32 own rows): it reduces them, writes the tagged
            // words and publishes its column state itself, with no barrier of the whole CTA
            if (warp == 0) {
#pragma unroll
                for (int q = 0; q < kNRed; ++q)
#pragma unroll
                    for (int o = 16; o >= 1; o >>= 1) x[q] = df_add(x[q], df_shfl_xor(x[q], o));
                float2 acc = x[0];
#pragma unroll
                for (int q = 1; q < kNRed; ++q)
                    if (lane == q) acc = x[q];
                if (lane < kNRed) {
                    unsigned long long* dst = ws.tsp + (size_t)b * 2 * kNRed + 2 * lane;
                    st_tag(dst, tag_pack(__float_as_uint(acc.y), tag));
                    st_tag(dst + 1, tag_pack(__float_as_uint(acc.x), tag));
                }
                // the lanes' column-state writes are ordered before the release by the warp barrier
                __syncwarp();
                if (lane == 0) post_flag(fpub + b, tag);
            }
        } else {
            if (warp < red_warps) {
#pragma unroll
                for (int q = 0; q < kNRed; ++q)
#pragma unroll
                    for (int o = 16; o >= 1; o >>= 1) x[q] = df_add(x[q], df_shfl_xor(x[q], o));
                if (lane == 0)
#pragma unroll
                    for (int q = 0; q < kNRed; ++q) red_smem[warp * kNRed + q] = x[q];
            }
            __syncthreads();
            if (tid < kNRed) {
                // the CTA's partial sum as two tagged words: the double-float's high and low floats
                float2 acc = make_float2(0.0f, 0.0f);
                for (int ww = 0; ww < red_warps; ++ww) acc = df_add(acc, red_smem[ww * kNRed + tid]);
                unsigned long long* dst = ws.tsp + (size_t)b * 2 * kNRed + 2 * tid;
                st_tag(dst, tag_pack(__float_as_uint(acc.y), tag));
                st_tag(dst + 1, tag_pack(__float_as_uint(acc.x), tag));
            }
            // the column state written in phase B is published by a thread with nothing else to do:
            // the release store waits for those writes, and only this thread waits with it
            if (tid == kCons) post_flag(fpub + b, tag);
        }

        MDOT_PHASE(5);
        // ---------------- every CTA: the G partials in a fixed order, then the decision ----------------
        bool ok = true;
        if (warp < kNRed) {
            float2 v5[5];
            unsigned int spins = 0;
            unsigned long long deadline = 0;
            for (;;) {
                bool ready = true;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const int bb = lane + 32 * k;
                    v5[k] = make_float2(0.0f, 0.0f);
                    if (bb < G) {
                        unsigned long long lo, hi;
                        ld_tag2(ws.tsp + (size_t)bb * 2 * kNRed + 2 * warp, lo, hi);
                        ready = ready && tag_of(lo) == tag && tag_of(hi) == tag;
                        v5[k] = make_float2(__uint_as_float((unsigned int)hi), __uint_as_float((unsigned int)lo));
                    }
                }
                if (__all_sync(0xffffffffu, ready)) break;
                const bool go_on = wait_backoff(spins, deadline, &ws.st->bar);
                if (!__all_sync(0xffffffffu, go_on)) {      // the warp gives up together
                    ok = false;
                    break;
                }
            }
            float2 sacc = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int k = 0; k < 5; ++k) sacc = df_add(sacc, v5[k]);
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) sacc = df_add(sacc, df_shfl_xor(sacc, o));
            if (lane == 0) tot_smem[warp] = df_to_double(sacc);
        } else if (warp == kNRed) {
            // the next pass reads every owner's column state (published before its scalar words):
            // once all of it is visible, one lane starts its bulk copy into shared memory
            ok = wait_flags(fpub, G, tag, &ws.st->bar);
            if (ok && prefetch && lane == 0) {
                // the state was acquired through the generic proxy; the copy reads it through the
                // async proxy, and overwrites a copy the last pass read through the generic proxy
                asm volatile("fence.proxy.async.global;" ::: "memory");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                const unsigned int bytes = (unsigned int)n * 16u;
                mbar_arrive_expect_tx(&s_pub_bar, bytes);
                for (unsigned int o = 0; o < bytes; o += 16384u)
                    tma_load_1d(reinterpret_cast<unsigned char*>(sPub) + o,
                                reinterpret_cast<const unsigned char*>(ws.pub) + o, min(16384u, bytes - o), &s_pub_bar);
                s_pub_issued += 1u;
            }
        }
        if (!ok) s_ok = 0;
        __syncthreads();
        if (!s_ok) break;
        MDOT_PHASE(6);
        if (tid == 0) {
            double tot[kNRed];
            for (int q = 0; q < kNRed; ++q) tot[q] = tot_smem[q];
            State loc = sst;                   // decide on registers, one copy in and out
            decide(&loc, tot, a);
            // steps as fp32 numbers: the column arithmetic uses them exactly, rows too
            loc.alpha = (double)(float)loc.alpha;
            loc.beta = (double)(float)loc.beta;
            sst = loc;
            s_step = ColStep{loc.accept, (float)loc.alpha_commit, (float)loc.beta, (float)loc.alpha};
        }
        __syncthreads();
        MDOT_PHASE(7);
        const bool accept = sst.accept != 0, done = sst.phase != PH_RUN;

        // ---------------- phase C: commit, new direction, next trial constants (rows) ----------------
        for (int i = r0 + tid; i < r1; i += T) {
            const int il = i - r0;
            float2 u = RU[il], p = RP[il];
            if (accept) {
                RF[RS_G * 2 * NL + il] = RF[RS_GT * 2 * NL + il];
                RF[RS_L * 2 * NL + il] = RF[RS_LTR * 2 * NL + il];
                // (u, v) += alpha p and p = s + beta p (Alg. 2, Eq. (18)), as for the columns
                col_commit(s_step, u, p, RF[RS_ST * 2 * NL + il]);
                RU[il] = u;
                RP[il] = p;
            }
            if (!done) prep_row_df(u, p, s_step.alpha, RF[RS_L * 2 * NL + il], a.Aglob, inv_gamma, G32, Glo, sm, L, il);
        }
        // own columns: the same commit every consumer applies to the published state
        for (int j = c0 + tid; j < c1; j += T) {
            const int jl = j - c0;
            if (accept) QF[CS_G * 2 * NL + jl] = QF[CS_GT * 2 * NL + jl];
            col_commit(s_step, QV[jl], QP[jl], QF[CS_ST * 2 * NL + jl]);
        }
        if (done) break;
        __syncthreads();
        MDOT_PHASE(8);
    }
    // the stage's iterate (also on a timeout: the best iterate so far) goes back to global memory
    __syncthreads();
    for (int i = r0 + tid; i < r1; i += T) {
        ws.u[i] = df_to_double(RU[i - r0]);
        ws.lr[i] = (double)RF[RS_L * 2 * NL + i - r0];
    }
    for (int j = c0 + tid; j < c1; j += T) ws.v[j] = df_to_double(QV[j - c0]);
    // rows prefetched for a pass that never came, and a copy of the column state that no pass
    // consumed, must land before the CTA exits
    if (use_ring && tid == kCons) ring_drain(ring, consumed, issued);
    if (prefetch && tid == 0 && pub_used < s_pub_issued) mbar_wait(&s_pub_bar, pub_used & 1u);
    if (tid == 0) {
        // the next launch's tags start above every tag this one may have posted
        atomicMax(ws.epoch, base + t + 3u);
        if (b == 0) {
            if (!s_ok || *reinterpret_cast<volatile unsigned int*>(abort)) {
                sst.status = max((int)sst.status, (int)ST_TIMEOUT);
                sst.phase = PH_DONE;
            }
            volatile unsigned long long* dw = reinterpret_cast<volatile unsigned long long*>(ws.st);
            const unsigned long long* lw = reinterpret_cast<const unsigned long long*>(&sst);
            for (int k = 0; k < kStateWords; ++k) dw[k] = lw[k];
        }
    }
}

// ---------------------------------------------------------------------------------------------
// MDOT-Sinkhorn stage (Alg. 4 as the projector of Alg. 1): alternate exact row and column
// normalisations in the log domain until ||r(P) - r~||_1 <= tol (after a column update c(P) = c~
// exactly, so this is ||grad g||_1).  Each half step is one fused pass over C of which one
// reduction is used: the row update needs r(P) at (u, v), the column update c(P) at the new u.
// ---------------------------------------------------------------------------------------------
template <int TIER, int COST>
__global__ void __launch_bounds__(kStageThreads, 1) sinkhorn_kernel(WS ws, StageArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double red_smem[32 * kNRed];
    __shared__ int s_flag[2];
    __shared__ unsigned int s_gen;
    __shared__ double s_gn;

    const int n = ws.n, G = ws.G, b = blockIdx.x, T = blockDim.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const SmemLayout L = smem_layout(n, G, TIER, T);
    int r0, r1, c0, c1;
    row_range(n, G, b, r0, r1);
    row_range(n, G, b, c0, c1);
    const int NL = L.nloc_max;
    double* R = reinterpret_cast<double*>(sm + L.off_rstate);
    double* Q = reinterpret_cast<double*>(sm + L.off_cstate);
    const double gamma = a.gamma, G64 = a.G64, w = a.w;
    State* S = ws.st;
    long long evals = 0, iters = 0;
    int status = ST_OK;
    double gn = INFINITY;

    if (tid == 0) s_gen = ld_acquire(&S->bar.gen);
    load_row_coords<COST>(ws, r0, r1, sm, L.off_xc);
    __syncthreads();
    unsigned int gen = s_gen;

    // ---- prologue (Alg. 1): smoothing, rank-one start or warm start ----
    for (int i = r0 + tid; i < r1; i += T) {
        const int il = i - r0;
        const double rt = (1.0 - w / 4.0) * ws.r[i] + w / (4.0 * n);
        const double lrt = log(rt);
        double u = ws.u[i];
        if (a.first) {
            u = lrt;
            ws.uprev[i] = u;
        } else if (a.warm_start == 0) {
            const double z = u;
            u = z + a.ratio * (z - ws.uprev[i]);             // Eq. (13)
            ws.uprev[i] = z;
        } else if (a.warm_start == 1) {
            u = a.ratio * u;
        }
        R[RS_U * NL + il] = u;
        R[RS_T * NL + il] = rt;
        R[RS_LT * NL + il] = lrt;
        R[RS_L * NL + il] = lrt;
        prep_row<TIER>(u, row_scale(lrt), a.Aglob, gamma, G64, sm, L, il);
    }
    for (int j = c0 + tid; j < c1; j += T) {
        const int jl = j - c0;
        const double ct = (1.0 - w / 4.0) * ws.c[j] + w / (4.0 * n);
        double v = ws.v[j];
        if (a.first) {
            v = log(ct);
            ws.vprev[j] = v;
        } else if (a.warm_start == 0) {
            const double z = v;
            v = z + a.ratio * (z - ws.vprev[j]);
            ws.vprev[j] = z;
        } else if (a.warm_start == 1) {
            v = a.ratio * v;
        }
        Q[CS_V * NL + jl] = v;
        Q[CS_T * NL + jl] = ct;
        prep_col<TIER>(ws, j, v, gamma, G64);
    }
    if (!grid_sync(&S->bar, G, gen, s_flag)) goto finish;

    for (;;) {
        // ---- half step 1: r(P) at (u, v); ||r(P) - r~||_1; the row update u += log r~ - log r(P) ----
        phase_A<TIER, COST>(ws, ColPlain{ws.Hh, ws.Wc, ws.colpart + (size_t)b * n}, r0, r1, gamma, G64, sm, L);
        ++evals;
        {
            double x = 0.0, bad = 0.0;
            const int* sA = reinterpret_cast<const int*>(sm + L.off_A);
            for (int i = r0 + tid; i < r1; i += T) {
                const int il = i - r0;
                const double sum = row_total<TIER>(sm, L, il);
                if (!(sum > 0.0) || !isfinite(sum)) { bad += 1.0; continue; }
                const double lrP = log(sum) + (double)sA[il] * kLn2;
                x += fabs(exp(lrP) - R[RS_T * NL + il]);
                R[RS_ST * NL + il] = R[RS_LT * NL + il] - lrP;      // the row update (Alg. 4)
                R[RS_L * NL + il] = lrP;
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                x += __shfl_xor_sync(0xffffffffu, x, o);
                bad += __shfl_xor_sync(0xffffffffu, bad, o);
            }
            if (lane == 0) { red_smem[2 * warp] = x; red_smem[2 * warp + 1] = bad; }
            __syncthreads();
            if (tid == 0) {
                double tx = 0.0, tb = 0.0;
                for (int ww = 0; ww < (T >> 5); ++ww) { tx += red_smem[2 * ww]; tb += red_smem[2 * ww + 1]; }
                ws.blockred[(size_t)b * kNRed] = tx;
                ws.blockred[(size_t)b * kNRed + 1] = tb;
            }
        }
        if (!grid_sync(&S->bar, G, gen, s_flag)) goto finish;
        if (warp == 0) {
            // every CTA sums the G partials in the same fixed order
            double x = 0.0, bad = 0.0;
            for (int k = 0; k < 5; ++k) {
                const int bb = lane + 32 * k;
                if (bb < G) {
                    x += __ldcg(ws.blockred + (size_t)bb * kNRed);
                    bad += __ldcg(ws.blockred + (size_t)bb * kNRed + 1);
                }
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                x += __shfl_xor_sync(0xffffffffu, x, o);
                bad += __shfl_xor_sync(0xffffffffu, bad, o);
            }
            if (lane == 0) s_gn = (bad > 0.0) ? -1.0 : x;
        }
        __syncthreads();
        gn = s_gn;
        if (gn < 0.0) { status = ST_NUMERIC; break; }
        if (gn <= a.tol) break;                                  // (u, v) meets the stage tolerance
        if (iters >= a.max_iter) { status = ST_CAP; break; }
        ++iters;
        for (int i = r0 + tid; i < r1; i += T) {
            const int il = i - r0;
            const double u = R[RS_U * NL + il] + R[RS_ST * NL + il];
            R[RS_U * NL + il] = u;
            R[RS_L * NL + il] = R[RS_LT * NL + il];             // r(P) = r~ after the row update
            prep_row<TIER>(u, row_scale(R[RS_LT * NL + il]), a.Aglob, gamma, G64, sm, L, il);
        }
        __syncthreads();

        // ---- half step 2: c(P) at the new u; the column update v += log c~ - log c(P) ----
        phase_A<TIER, COST>(ws, ColPlain{ws.Hh, ws.Wc, ws.colpart + (size_t)b * n}, r0, r1, gamma, G64, sm, L);
        ++evals;
        if (!grid_sync(&S->bar, G, gen, s_flag)) goto finish;
        for (int j0 = c0; j0 < c1; j0 += 32) {
            double colsum;
            if (TIER != TIER_F64)
                colsum = merge_cols_f32(ws.colpart, n, G, j0, c1, reinterpret_cast<float*>(sm + L.off_merge));
            else
                colsum = merge_cols_f64(ws.colpartd, n, G, j0, c1, reinterpret_cast<double*>(sm + L.off_merge));
            const int j = j0 + tid;
            if (tid < 32 && j < c1) {
                const int jl = j - c0;
                double v = Q[CS_V * NL + jl];
                if (colsum > 0.0 && isfinite(colsum))
                    v += log(Q[CS_T * NL + jl]) - (log(colsum) + (double)a.Aglob * kLn2);
                Q[CS_V * NL + jl] = v;
                prep_col<TIER>(ws, j, v, gamma, G64);
            }
        }
        if (!grid_sync(&S->bar, G, gen, s_flag)) goto finish;
    }
finish:
    __syncthreads();
    for (int i = r0 + tid; i < r1; i += T) {
        ws.u[i] = R[RS_U * NL + i - r0];
        ws.lr[i] = R[RS_L * NL + i - r0];
    }
    for (int j = c0 + tid; j < c1; j += T) ws.v[j] = Q[CS_V * NL + j - c0];
    if (b == 0 && tid == 0) {
        if (*reinterpret_cast<volatile unsigned int*>(&S->bar.abort)) status = ST_TIMEOUT;
        S->evals += evals;
        if (TIER == TIER_F64) S->evals64 += evals;
        S->iters += iters;
        S->gnorm = gn;
        S->status = max((int)S->status, status);
        S->phase = PH_DONE;
    }
}

// ---------------------------------------------------------------------------------------------
// standalone dual evaluation (mdot_dual_eval): optional max pass for the row scales, one pass,
// merge.  Writes log r(P) to ws.lrtr and log c(P) to ws.lcout.
// ---------------------------------------------------------------------------------------------

template <int TIER, int COST>
__global__ void __launch_bounds__(kStageThreads, 1) dual_eval_kernel(WS ws, EvalArgs a)
{
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ double red_g[32];
    __shared__ int s_flag[2];
    __shared__ unsigned int s_gen;
    const int n = ws.n, G = ws.G, b = blockIdx.x, T = blockDim.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    const SmemLayout L = smem_layout(n, G, TIER, T, true);
    int r0, r1, c0, c1;
    row_range(n, G, b, r0, r1);
    row_range(n, G, b, c0, c1);
    State* S = ws.st;
    if (tid == 0) s_gen = ld_acquire(&S->bar.gen);
    load_row_coords<COST>(ws, r0, r1, sm, L.off_xc);
    __syncthreads();
    unsigned int gen = s_gen;
    int* sA = reinterpret_cast<int*>(sm + L.off_A);
    double* sM = reinterpret_cast<double*>(sm + L.off_x);
    const float G32 = (float)a.G64;

    // column constants without scale (row view / max pass)
    for (int j = c0 + tid; j < c1; j += T) {
        float gh, wl;
        split_cost_unit(a.v[j] / a.gamma, gh, wl, a.G64);
        ws.Hh[j] = gh;
        ws.Wc[j] = wl;
        if (TIER == TIER_F64) ws.Hd[j] = a.v[j];
    }
    if (a.ref != nullptr) {
        // ---- one-scale path (the solver's): row scales from the estimate, one exp2 per entry;
        // column weights relative to the largest row scale Aglob (grid max) ----
        {
            int am = -2000000;
            for (int i = r0 + tid; i < r1; i += T) {
                const int A = row_scale(a.ref[i]);
                sA[i - r0] = A;
                am = max(am, A);
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) am = max(am, __shfl_xor_sync(0xffffffffu, am, o));
            __shared__ int s_am[32];
            if (lane == 0) s_am[warp] = am;
            __syncthreads();
            if (tid == 0) {
                for (int w = 1; w < nw; ++w) am = max(am, s_am[w]);
                reinterpret_cast<volatile int*>(ws.scratch)[b] = max(am, s_am[0]);
            }
        }
        if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;
        {
            __shared__ int s_ag;
            if (tid == 0) {
                int m = -2000000;
                for (int bb = 0; bb < G; ++bb) m = max(m, reinterpret_cast<const volatile int*>(ws.scratch)[bb]);
                s_ag = m;
            }
            __syncthreads();
            const int Aglob = s_ag;
            for (int i = r0 + tid; i < r1; i += T)
                prep_row<TIER>(a.u[i], sA[i - r0], Aglob, a.gamma, a.G64, sm, L, i - r0);
            __syncthreads();
            phase_A<TIER, COST>(ws, ColPlain{ws.Hh, ws.Wc, ws.colpart + (size_t)b * n}, r0, r1, a.gamma, a.G64, sm, L);
            for (int i = r0 + tid; i < r1; i += T) {
                const int il = i - r0;
                ws.lrtr[i] = log(row_total<TIER>(sm, L, il)) + (double)sA[il] * kLn2;
            }
            if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;
            if (TIER != TIER_F64) {
                // up to kMergeGroups x 32 columns per round trip
                float* msm = reinterpret_cast<float*>(sm + L.off_merge);
                double* tot = reinterpret_cast<double*>(msm + 2 * kMergeGroups * 32 * nw);
                for (int j0 = c0; j0 < c1; j0 += 32 * kMergeGroups) {
                    merge_cols_f32_wide<kMergeGroups>(ws.colpart, n, G, j0, c1, msm, tot);
                    const int j = j0 + tid;
                    if (tid < 32 * kMergeGroups && j < c1) ws.lcout[j] = log(tot[tid]) + (double)Aglob * kLn2;
                    __syncthreads();
                }
            } else {
                for (int j0 = c0; j0 < c1; j0 += 32) {
                    const double colsum = merge_cols_f64(ws.colpartd, n, G, j0, c1,
                                                         reinterpret_cast<double*>(sm + L.off_merge));
                    const int j = j0 + tid;
                    if (tid < 32 && j < c1) ws.lcout[j] = log(colsum) + (double)Aglob * kLn2;
                }
            }
        }
        goto dual_value;
    }
    // ---- two-scale path: max pass for row and column scales, then both LSEs exactly ----
    // unscaled row constants (they are also the column-view row constants)
    for (int i = r0 + tid; i < r1; i += T) {
        float fh, wl;
        split_cost_unit(a.u[i] / a.gamma, fh, wl, a.G64);
        reinterpret_cast<float*>(sm + L.off_s)[i - r0] = fh;
        reinterpret_cast<float*>(sm + L.off_A)[i - r0] = wl;
    }
    if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;
    {
        const float* f2 = reinterpret_cast<const float*>(sm + L.off_s);
        const float* w2 = reinterpret_cast<const float*>(sm + L.off_A);
        // row maxima (one warp per row) in log2 units (F32) or natural-log units (F64)
        for (int i = r0 + warp; i < r1; i += nw) {
            double m = -INFINITY;
            if (TIER != TIER_F64) {
                const float fh = f2[i - r0], wl = w2[i - r0];
                float mf = -INFINITY;
                for (int j = lane; j < n; j += 32)
                    mf = fmaxf(mf, fmaf(G32, (fh + __ldcg(ws.Hh + j)) - cost_elem<COST>(ws, i, j), wl + __ldcg(ws.Wc + j)));
                m = (double)mf;
            } else {
                const double ui = a.u[i];
                for (int j = lane; j < n; j += 32)
                    m = fmax(m, (ui + __ldcg(ws.Hd + j)) - a.gamma * (double)cost_elem<COST>(ws, i, j));
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) sM[i - r0] = m;
        }
        // column maxima over own rows (thread per column), CTA partials
        for (int j = tid; j < n; j += T) {
            if (TIER != TIER_F64) {
                const float gh = __ldcg(ws.Hh + j), wc = __ldcg(ws.Wc + j);
                float mf = -INFINITY;
                for (int i = r0; i < r1; ++i)
                    mf = fmaxf(mf, fmaf(G32, (f2[i - r0] + gh) - cost_elem<COST>(ws, i, j), w2[i - r0] + wc));
                ws.colpart[(size_t)b * n + j] = mf;
            } else {
                const double vj = __ldcg(ws.Hd + j);
                double md = -INFINITY;
                for (int i = r0; i < r1; ++i)
                    md = fmax(md, (a.u[i] + vj) - a.gamma * (double)cost_elem<COST>(ws, i, j));
                ws.colpartd[(size_t)b * n + j] = md;
            }
        }
    }
    if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;
    // column scales and column-view constants (own columns)
    for (int j = c0 + tid; j < c1; j += T) {
        double m = -INFINITY;
        if (TIER != TIER_F64) {
            for (int bb = 0; bb < G; ++bb) m = fmax(m, (double)__ldcg(ws.colpart + (size_t)bb * n + j));
            const double B = fmin(fmax(ceil(m), -1.0e7), 1.0e7);
            float gh, wl;
            split_cost_unit(a.v[j] / a.gamma - B / a.G64, gh, wl, a.G64);
            ws.Fh[j] = gh;          // column-view constants (reuse of the fp32 row arrays)
            ws.Wr[j] = wl;
            ws.A[j] = (int)B;
        } else {
            for (int bb = 0; bb < G; ++bb) m = fmax(m, __ldcg(ws.colpartd + (size_t)bb * n + j));
            ws.Fd[j] = m;
        }
    }
    // row scales and both row constants (own rows)
    for (int i = r0 + tid; i < r1; i += T) {
        const int il = i - r0;
        if (TIER != TIER_F64) {
            const double A = fmin(fmax(ceil(sM[il]), -1.0e7), 1.0e7);
            float fh, wl;
            split_cost_unit(a.u[i] / a.gamma - A / a.G64, fh, wl, a.G64);
            reinterpret_cast<float*>(sm + L.off_c0)[il] = fh;
            reinterpret_cast<float*>(sm + L.off_c1)[il] = wl;
            sM[il] = A;
        } else {
            reinterpret_cast<double*>(sm + L.off_c0)[il] = a.u[i];
            reinterpret_cast<double*>(sm + L.off_s)[il] = sM[il];
        }
    }
    if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;
    {
        const int nwl = T >> 5;
        if (TIER != TIER_F64) {
            float* sRow = reinterpret_cast<float*>(sm + L.off_row);
            for (int x = tid; x < nwl * L.nloc_max; x += T) sRow[x] = 0.0f;
            __syncthreads();
            const float Glo = (float)(a.G64 - (double)G32);
            const float* f1 = reinterpret_cast<const float*>(sm + L.off_c0);
            const float* w1 = reinterpret_cast<const float*>(sm + L.off_c1);
            const float* f2 = reinterpret_cast<const float*>(sm + L.off_s);
            const float* w2 = reinterpret_cast<const float*>(sm + L.off_A);
            if ((n & 3) == 0 && COST == COST_DENSE)
                pass2_f32<true, TIER == TIER_F32A, COST>(ws, ws.C, n, r0, r1, ws.Hh, ws.Wc, ws.Fh, ws.Wr, f1, w1, f2, w2, G32, Glo, sRow,
                                L.nloc_max, ws.colpart + (size_t)b * n);
            else
                pass2_f32<false, TIER == TIER_F32A, COST>(ws, ws.C, n, r0, r1, ws.Hh, ws.Wc, ws.Fh, ws.Wr, f1, w1, f2, w2, G32, Glo, sRow,
                                 L.nloc_max, ws.colpart + (size_t)b * n);
        } else {
            double* sRow = reinterpret_cast<double*>(sm + L.off_row);
            for (int x = tid; x < nwl * L.nloc_max; x += T) sRow[x] = 0.0;
            __syncthreads();
            pass2_f64<COST>(ws, ws.C, n, r0, r1, ws.Hd, ws.Fd, reinterpret_cast<const double*>(sm + L.off_c0),
                      reinterpret_cast<const double*>(sm + L.off_s), a.gamma, sRow, L.nloc_max,
                      ws.colpartd + (size_t)b * n);
        }
        __syncthreads();
        for (int i = r0 + tid; i < r1; i += T) {
            const int il = i - r0;
            const double sum = row_total<TIER>(sm, L, il);
            ws.lrtr[i] = log(sum) + (TIER != TIER_F64 ? sM[il] * kLn2 : sM[il]);
        }
    }
    if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;
    for (int j0 = c0; j0 < c1; j0 += 32) {
        double colsum;
        if (TIER != TIER_F64)
            colsum = merge_cols_f32(ws.colpart, n, G, j0, c1, reinterpret_cast<float*>(sm + L.off_merge));
        else
            colsum = merge_cols_f64(ws.colpartd, n, G, j0, c1, reinterpret_cast<double*>(sm + L.off_merge));
        const int j = j0 + tid;
        if (tid < 32 && j < c1)
            ws.lcout[j] = log(colsum) + (TIER != TIER_F64 ? (double)__ldcg(ws.A + j) * kLn2 : __ldcg(ws.Fd + j));
    }
dual_value:
    // Eq. (4): g = sum_i r(P)_i - <u, r> - <v, c>.  Each CTA sums its own rows (log r(P)_i was
    // written by the same thread above) and its own columns, then CTA 0 adds the G partials in
    // CTA order after one more barrier.
    if (a.g_out != nullptr) {
        double x[1] = {0.0};
        for (int i = r0 + tid; i < r1; i += T) x[0] += exp(ws.lrtr[i]) - a.u[i] * a.r[i];
        for (int j = c0 + tid; j < c1; j += T) x[0] -= a.v[j] * a.c[j];
        block_reduce_nred<1>(x, red_g);
        if (tid == 0) reinterpret_cast<volatile double*>(ws.scratch)[G + b] = x[0];
        if (!grid_sync(&S->bar, G, gen, s_flag)) goto timeout;
        if (b == 0 && tid == 0) {
            double g = 0.0;
            for (int bb = 0; bb < G; ++bb) g += reinterpret_cast<const volatile double*>(ws.scratch)[G + bb];
            *a.g_out = g;
        }
    }
    return;
timeout:
    if (tid == 0) atomicMax(&S->status, (int)ST_TIMEOUT);
}

}  // namespace mdot
