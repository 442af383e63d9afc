// C ABI of the MDOT-PNCG library (declared in include/mdot.h): handle and workspace management,
// argument validation, the host side of MDOT (Alg. 1: the gamma schedule, stage tolerances and
// warm-start ratios) and the launch sequence of the device stages, rounding and lower bound.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "batch_kernels.cuh"
#include "launch.h"
#include "mdot.h"

using namespace mdot;

namespace {

thread_local char g_err[512] = "";
constexpr int kTraceMax = 512;          // launches recorded by a profiled solve

struct Deleter {
    std::vector<void*> dev, host;
    ~Deleter()
    {
        for (void* p : dev) cudaFree(p);
        for (void* p : host) cudaFreeHost(p);
    }
};

}  // namespace

struct mdot_handle {
    int dev = 0, sms = 0, G = 0;
    cudaStream_t stream = nullptr;
    int64_t max_n = 0;
    Deleter mem;
    WS ws{};
    double* d_out = nullptr;       // [16] device results
    double* h_out = nullptr;       // [16] pinned
    State* h_state = nullptr;      // pinned copy of the state
    unsigned int* h_limit = nullptr;   // pinned: the wait limit copied into the state of a solve
    double *Y = nullptr, *EC = nullptr, *ER = nullptr, *gp = nullptr;
    // device buffers of mdot_solve_host
    double *d_r = nullptr, *d_c = nullptr, *d_u = nullptr, *d_v = nullptr;
    float* d_C = nullptr;
    int64_t host_n = 0;
    // batched solver workspace (allocated on first use) and its tile-variant table per size bucket
    double* b_slots = nullptr;
    int b_grid[kBatchVariants] = {0, 0};
    int b_variant[kBatchBuckets] = {0, 0, 0, 0, 0};
    BatchProblem* b_probs = nullptr;
    BatchResult* b_results = nullptr;
    int* b_order = nullptr;
    unsigned int* b_next = nullptr;
    int b_cap = 0;
    double* b_uv = nullptr;        // potentials of batched problems that asked for none (finish)
    size_t b_uv_cap = 0;           // doubles
    // evaluation tags consumed by the stage kernel's flags since they were last cleared (an upper
    // bound, from the evaluation counts); cleared well before the 32-bit tag could wrap
    unsigned long long tags_used = 0;
    size_t flag_bytes = 0;
    // per-launch rows of the last profiled solve (mdot_solve_trace)
    long long* h_trace_evals = nullptr;     // pinned [kTraceMax]
    std::vector<mdot_trace_row> trace;
    // device time of the last standalone dual-evaluation kernel (events around its launch)
    cudaEvent_t de_ev[2] = {nullptr, nullptr};
    double de_ms = -1.0;
    ~mdot_handle()
    {
        if (de_ev[0]) cudaEventDestroy(de_ev[0]);
        if (de_ev[1]) cudaEventDestroy(de_ev[1]);
        cudaFree(d_r); cudaFree(d_c); cudaFree(d_u); cudaFree(d_v); cudaFree(d_C);
        cudaFree(b_slots); cudaFree(b_probs); cudaFree(b_results); cudaFree(b_order); cudaFree(b_next);
        cudaFree(b_uv);
    }
};

namespace mdot {

}

#define CKR(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            snprintf(g_err, sizeof g_err, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),        \
                     __FILE__, __LINE__);                                                          \
            return MDOT_ERR_CUDA;                                                                  \
        }                                                                                          \
    } while (0)

extern "C" {

void mdot_default_params(mdot_params* prm)
{
    if (!prm) return;
    memset(prm, 0, sizeof(*prm));
    prm->gamma_i = 16.0;                 // Sec. 5.2
    prm->gamma_f = 0.0;                  // derived from eps_target (Prop. 2)
    prm->p = 1.5;                        // Sec. 5.2
    prm->q = std::cbrt(2.0);             // Sec. 5.2
    prm->ls_c1 = 0.1;                    // App. B leaves 0 < c1 < c2 < 1 open (reading)
    prm->ls_c2 = 0.5;
    prm->ls_max_trials = 50;
    prm->max_iter = 100000;
    prm->precision = MDOT_PREC_AUTO;
    prm->warm_start = 0;
    prm->final_tol = 0.0;
    prm->fp32_floor = 2e-7;
    prm->profile = 0;
    prm->ls_init = 1;                    // App. B leaves the first trial step open (see mdot.h)
    prm->wait_limit_us = 0;              // bounded device waits: the 2 s default
    prm->tensor_cores = 0;               // grid costs in fp32 operations (measured faster)
    prm->polish_iters = 64;              // batched form: fp64 iterations repairing a stalled last stage
    prm->reserved = 0;
}

const char* mdot_status_string(int32_t s)
{
    switch (s) {
    case MDOT_OK: return "MDOT_OK";
    case MDOT_ERR_INVALID_ARG: return "MDOT_ERR_INVALID_ARG";
    case MDOT_ERR_NOT_CONVERGED: return "MDOT_ERR_NOT_CONVERGED";
    case MDOT_ERR_NUMERIC: return "MDOT_ERR_NUMERIC";
    case MDOT_ERR_TIMEOUT: return "MDOT_ERR_TIMEOUT";
    case MDOT_ERR_OOM: return "MDOT_ERR_OOM";
    case MDOT_ERR_CUDA: return "MDOT_ERR_CUDA";
    case MDOT_NOT_READY: return "MDOT_NOT_READY";
    default: return "MDOT_UNKNOWN_STATUS";
    }
}

const char* mdot_last_error(void) { return g_err; }

mdot_status mdot_create(mdot_handle** out, int64_t max_n, void* stream)
{
    if (!out || max_n < 1 || max_n > (int64_t)1 << 20) return MDOT_ERR_INVALID_ARG;
    *out = nullptr;
    mdot_handle* h = new mdot_handle();
    h->stream = (cudaStream_t)stream;
    h->max_n = max_n;
    cudaError_t e = cudaGetDevice(&h->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->dev);
    if (e != cudaSuccess) {
        snprintf(g_err, sizeof g_err, "device query: %s", cudaGetErrorString(e));
        delete h;
        return MDOT_ERR_CUDA;
    }
    h->G = std::min(h->sms, 160);        // one CTA per SM (cooperative, persistent per launch); the
                                         // fixed-order reductions handle at most 160 CTAs
    int mb = 0;
    e = configure_kernels((int)max_n, h->G, &mb);
    if (e != cudaSuccess || mb < 1) {
        snprintf(g_err, sizeof g_err, "kernel configuration: %s (blocks/SM %d)",
                 e != cudaSuccess ? cudaGetErrorString(e) : "does not fit", mb);
        delete h;
        return e != cudaSuccess ? MDOT_ERR_CUDA : MDOT_ERR_INVALID_ARG;
    }
    const size_t n = (size_t)max_n, G = (size_t)h->G;
    auto dalloc = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
        h->mem.dev.push_back(p);
        return p;
    };
    const int nvec = 25;
    double* vec = (double*)dalloc(nvec * n * sizeof(double));
    float* f32 = (float*)dalloc(4 * n * sizeof(float));
    int* A = (int*)dalloc(n * sizeof(int));
    float* colpart = (float*)dalloc(G * n * sizeof(float));
    double* colpartd = (double*)dalloc(G * n * sizeof(double));
    double* blockred = (double*)dalloc(G * kNRedP * sizeof(double));
    double* scratch = (double*)dalloc(G * 8 * sizeof(double));
    State* st = (State*)dalloc(sizeof(State));
    // stage-kernel flags [2][G] and the tag base; published column state (hb, rb, P, S per column)
    const size_t flag_words = 2 * G + 1;
    unsigned int* flagw = (unsigned int*)dalloc(flag_words * sizeof(unsigned int));
    float* pubw = (float*)dalloc(4 * n * sizeof(float));
    unsigned long long* tspw = (unsigned long long*)dalloc(G * 2 * kNRed * sizeof(unsigned long long));
    h->d_out = (double*)dalloc(16 * sizeof(double));
    void* hp = nullptr;
    if (cudaMallocHost(&hp, 16 * sizeof(double) + sizeof(State) + 16 + kTraceMax * sizeof(long long)) == cudaSuccess)
        h->mem.host.push_back(hp);
    if (!vec || !f32 || !A || !colpart || !colpartd || !blockred || !scratch || !st || !flagw || !pubw || !tspw || !h->d_out || !hp) {
        snprintf(g_err, sizeof g_err, "workspace allocation failed for max_n = %lld", (long long)max_n);
        delete h;
        return MDOT_ERR_OOM;
    }
    h->h_out = (double*)hp;
    h->h_state = (State*)((char*)hp + 16 * sizeof(double));
    h->h_limit = (unsigned int*)((char*)hp + 16 * sizeof(double) + sizeof(State));
    h->h_trace_evals = (long long*)((char*)hp + 16 * sizeof(double) + sizeof(State) + 16);
    WS& w = h->ws;
    double* p = vec;
    auto take = [&]() { double* q = p; p += n; return q; };
    w.rt = take(); w.ct = take(); w.lrt = take(); w.lct = take();
    w.u = take(); w.v = take(); w.pu = take(); w.pv = take(); w.uprev = take(); w.vprev = take();
    w.gr = take(); w.gc = take(); w.grt = take(); w.gct = take(); w.srt = take(); w.sct = take();
    w.lr = take(); w.lrtr = take(); w.lcout = take(); w.Fd = take(); w.Hd = take();
    h->Y = take(); h->EC = take(); h->ER = take(); h->gp = take();
    w.Fh = f32; w.Wr = f32 + n; w.Hh = f32 + 2 * n; w.Wc = f32 + 3 * n;
    w.A = A;
    w.colpart = colpart;
    w.colpartd = colpartd;
    w.blockred = blockred;
    w.scratch = scratch;
    w.st = st;
    w.flags = flagw;
    w.epoch = flagw + 2 * G;
    w.tsp = tspw;
    w.pub = reinterpret_cast<float4*>(pubw);
    h->flag_bytes = flag_words * sizeof(unsigned int);
    w.G = h->G;
    if (cudaMemsetAsync(st, 0, sizeof(State), h->stream) != cudaSuccess ||
        cudaMemsetAsync(flagw, 0, h->flag_bytes, h->stream) != cudaSuccess ||
        cudaMemsetAsync(tspw, 0, G * 2 * kNRed * sizeof(unsigned long long), h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        snprintf(g_err, sizeof g_err, "state initialisation failed");
        delete h;
        return MDOT_ERR_CUDA;
    }
    *out = h;
    return MDOT_OK;
}

mdot_status mdot_destroy(mdot_handle* h)
{
    if (h) {
        cudaStreamSynchronize(h->stream);
        delete h;
    }
    return MDOT_OK;
}

}  // extern "C"

namespace mdot {

// Shared with the serving runtime (server.cu).
mdot_status params_valid(const mdot_params& P);
mdot_status status_of(int st);
void set_last_error(const char* msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

}  // namespace mdot

namespace {

mdot_status params_ok(const mdot_params& P)
{
    if (!(P.gamma_i > 0.0) || !(P.p >= 1.0) || !(P.q > 1.0) || !(P.ls_c1 > 0.0) ||
        !(P.ls_c2 > P.ls_c1) || !(P.ls_c2 < 1.0) || P.ls_max_trials < 1 || P.max_iter < 1 ||
        P.precision < 0 || P.precision > 3 || P.warm_start < 0 || P.warm_start > 2 ||
        P.smoothing < 0 || P.smoothing > 1 || P.projector < 0 || P.projector > 1 || P.stop_entropy < 0 ||
        P.stop_entropy > 1 || P.precond < 0 || P.precond > 1 || P.ls_init < 0 || P.ls_init > 1 ||
        !(P.fp32_floor >= 0.0) || !std::isfinite(P.gamma_f) || P.tensor_cores < 0 || P.tensor_cores > 1 ||
        P.polish_iters < 0)
        return MDOT_ERR_INVALID_ARG;
    return MDOT_OK;
}

mdot_status map_status(int st)
{
    switch (st) {
    case ST_OK: return MDOT_OK;
    case ST_CAP:
    case ST_LSFAIL: return MDOT_ERR_NOT_CONVERGED;
    case ST_NUMERIC: return MDOT_ERR_NUMERIC;
    default: return MDOT_ERR_TIMEOUT;
    }
}

}  // namespace

namespace mdot {
mdot_status params_valid(const mdot_params& P) { return params_ok(P); }
mdot_status status_of(int st) { return map_status(st); }

// Run the handle's cooperative kernels on G CTAs instead of one per SM (the serving runtime
// gives large requests a share of the GPU); the workspace was sized for more.
mdot_status handle_set_grid(mdot_handle* h, int G)
{
    if (!h || G < 1 || G > std::min(h->sms, 160)) return MDOT_ERR_INVALID_ARG;
    int mb = 0;
    cudaError_t e = configure_kernels((int)h->max_n, G, &mb);
    if (e != cudaSuccess || mb < 1) return MDOT_ERR_CUDA;
    h->G = G;
    h->ws.G = G;
    return MDOT_OK;
}
}  // namespace mdot

namespace {

// Optional per-launch timing with CUDA events on the handle's stream; after each launch the
// cumulative evaluation count of the state is copied into a pinned slot (the solve trace).
struct Timer {
    bool on = false;
    cudaStream_t s = nullptr;
    const long long* dev_evals = nullptr;     // State::evals on the device
    long long* host_evals = nullptr;          // pinned, kTraceMax slots
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    std::vector<int> kind;
    void begin(int k)
    {
        if (!on) return;
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
        ev.push_back({a, b});
        kind.push_back(k);
    }
    void end()
    {
        if (!on) return;
        cudaEventRecord(ev.back().second, s);
        if (host_evals && ev.size() <= (size_t)kTraceMax)
            cudaMemcpyAsync(host_evals + ev.size() - 1, dev_evals, sizeof(long long), cudaMemcpyDeviceToHost, s);
    }
    // call after the stream is synchronised; sums[k] += ms; the per-launch rows go to trace
    void collect(double* sums, std::vector<mdot_trace_row>* trace = nullptr)
    {
        if (trace) trace->clear();
        long long prev = 0;
        for (size_t q = 0; q < ev.size(); ++q) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, ev[q].first, ev[q].second);
            sums[kind[q]] += ms;
            if (trace && host_evals && q < (size_t)kTraceMax) {
                const long long e = host_evals[q];
                trace->push_back(mdot_trace_row{kind[q], 0, (double)ms, e - prev});
                prev = e;
            }
            cudaEventDestroy(ev[q].first);
            cudaEventDestroy(ev[q].second);
        }
        ev.clear();
        kind.clear();
    }
    ~Timer() { double d[8] = {0}; collect(d); }
};

// Reset the barrier and counters before a new call (also clears an aborted barrier); limit_us > 0
// sets the limit of the call's bounded waits (0: the default of the device code).
cudaError_t reset_state(mdot_handle* h, int limit_us = 0)
{
    cudaError_t e = cudaMemsetAsync(h->ws.st, 0, sizeof(State), h->stream);
    if (e != cudaSuccess || limit_us <= 0) return e;
    *h->h_limit = (unsigned int)limit_us;      // pinned; the call synchronises before it returns
    return cudaMemcpyAsync(&h->ws.st->bar.limit_us, h->h_limit, sizeof(unsigned int), cudaMemcpyHostToDevice,
                           h->stream);
}

double gamma_f_for_eps(double H, double eps, double gi, double q, double p)
{
    // Prop. 2: gamma_f = (5 H_min / (2 eps))^(1/p), rounded up onto gamma_i q^k
    const double target = std::pow(5.0 * H / (2.0 * eps), 1.0 / p);
    double g = gi;
    while (g < target * (1.0 - 1e-12)) g *= q;
    return g;
}

// Validate r, c on the device; returns H_min in *H.
mdot_status check_marginals(mdot_handle* h, const WS& ws, double* H)
{
    CKR(reset_state(h));
    CKR(launch_validate(ws, h->d_out, h->stream));
    CKR(cudaMemcpyAsync(h->h_out, h->d_out, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CKR(cudaStreamSynchronize(h->stream));
    const double* o = h->h_out;
    if (o[6] != 0.0 || !(o[4] >= 0.0) || !(o[5] >= 0.0) || !(std::fabs(o[0] - 1.0) <= 1e-9) ||
        !(std::fabs(o[1] - 1.0) <= 1e-9)) {
        snprintf(g_err, sizeof g_err, "marginals invalid: sum r %.17g sum c %.17g min r %g min c %g nonfinite %g",
                 o[0], o[1], o[4], o[5], o[6]);
        return MDOT_ERR_INVALID_ARG;
    }
    // H_min floored at 1e-12: a point-mass marginal keeps a positive smoothing weight (Alg. 1)
    *H = std::max(std::min(o[2], o[3]), 1e-12);
    return MDOT_OK;
}

// The squared-Euclidean cost of integer points (|coordinate| <= 255) runs on the tensor cores
// when the caller allows it (exact: see pass_f32_regen_tc); one check of the coordinates per call.
cudaError_t select_cost_form(mdot_handle* h, WS& ws, bool allow)
{
    ws.tc = 0;
    if (ws.ckind != COST_SQEUCLID || !allow) return cudaSuccess;
    bool grid = false;
    cudaError_t e = check_grid_points(ws.X, ws.Y, ws.n, reinterpret_cast<unsigned int*>(h->d_out + 14),
                                      reinterpret_cast<unsigned int*>(h->h_out + 14), h->stream, &grid);
    ws.tc = grid ? 1 : 0;
    return e;
}

// Where C comes from: a dense matrix, or coordinates (n x 3 each) with a kind and a scale.
struct CostSpec {
    const float* C = nullptr;
    const float* X = nullptr;
    const float* Y = nullptr;
    int kind = COST_DENSE;
    float scale = 1.0f;
    bool valid() const
    {
        if (kind == COST_DENSE) return C != nullptr;
        return (kind == COST_SQEUCLID || kind == COST_L1) && X && Y && std::isfinite(scale) && scale > 0.0f;
    }
    void apply(WS& ws) const
    {
        ws.C = C;
        ws.X = X;
        ws.Y = Y;
        ws.ckind = kind;
        ws.cscale = scale;
    }
};

mdot_status solve_core(mdot_handle* h, const double* r, const double* c, const CostSpec& cs, int64_t n,
                       double eps_target, const mdot_params* prm, double* u_out, double* v_out,
                       double* cost_out, double* gap_out, mdot_info* info)
{
    if (!h || !r || !c || !cs.valid() || !u_out || !v_out || n < 1 || n > h->max_n) return MDOT_ERR_INVALID_ARG;
    mdot_params P;
    if (prm) P = *prm; else mdot_default_params(&P);
    if (params_ok(P) != MDOT_OK) return MDOT_ERR_INVALID_ARG;
    if (!(P.gamma_f > 0.0) && !(eps_target > 0.0 && std::isfinite(eps_target))) return MDOT_ERR_INVALID_ARG;
    WS ws = h->ws;
    ws.n = (int)n;
    ws.r = r;
    ws.c = c;
    cs.apply(ws);
    double H = 0.0;
    mdot_status ms = check_marginals(h, ws, &H);
    if (ms != MDOT_OK) return ms;
    CKR(select_cost_form(h, ws, P.tensor_cores != 0));
    const double gf = (P.gamma_f > 0.0) ? P.gamma_f : gamma_f_for_eps(H, eps_target, P.gamma_i, P.q, P.p);
    // precision tiers: fp64 entries for small n; otherwise fp32 entries with ex2.approx while the
    // stage tolerance is loose, the accurate fp32 tier (double-float exponent, polynomial exp2)
    // once it is below kAccSwitch, and an fp64 polish of the last stage if even that tolerance is
    // below the accurate tier's noise floor (fp32_floor)
    constexpr double kAccSwitch = 2e-6;
    const bool all64 = P.precision == MDOT_PREC_FP64 || (P.precision == MDOT_PREC_AUTO && n <= 512);
    const bool polish = P.precision == MDOT_PREC_AUTO && !all64;
    CKR(reset_state(h, P.wait_limit_us));
    if (h->tags_used > (1ull << 31)) {
        // restart the stage kernel's tags from zero long before the 32-bit tag could wrap
        CKR(cudaMemsetAsync(h->ws.flags, 0, h->flag_bytes, h->stream));
        CKR(cudaMemsetAsync(h->ws.tsp, 0, (size_t)h->G * 2 * kNRed * sizeof(unsigned long long), h->stream));
        h->tags_used = 0;
    }
    Timer tm;
    tm.on = P.profile != 0;
    tm.s = h->stream;
    tm.dev_evals = &ws.st->evals;
    tm.host_evals = h->h_trace_evals;
    int launches = 1, launches32 = 0;
    double tol_last = 0.0;           // tolerance the last stage launch was asked for
    // Alg. 1: gamma schedule, stage by stage (same arithmetic as the paper's loop)
    double gamma = std::min(P.gamma_i, gf);
    double dgamma_prev = gamma;      // stage 0 is gamma = 0 (Prop. 1): the first step is gamma_1
    double ratio = 0.0;
    int stages = 0;
    for (int t = 1;; ++t) {
        // stopping tolerance (Alg. 1); App. C's comparison puts log n in place of H_min
        const double eps_d = (P.stop_entropy == 1 ? std::log((double)n) : H) / std::pow(gamma, P.p);
        // projection tolerance eps_d / 2, floored at the fp64 resolution of the marginals (~2e-16 gamma relative noise)
        double tol = std::max(eps_d / 2.0, 1e-13 + 1e-15 * gamma);
        const bool last = (gamma == gf);
        if (last && P.final_tol > 0.0) tol = P.final_tol;
        StageArgs a{};
        a.gamma = gamma;
        a.G64 = gamma * kLog2e;
        // smoothing weight: eps_d of the stage (Alg. 1), or fixed at its gamma_f value (ablation)
        a.w = (P.smoothing == 1) ? H / std::pow(gf, P.p) : eps_d;
        a.ratio = ratio;
        a.c1 = P.ls_c1;
        a.c2 = P.ls_c2;
        a.first = (t == 1);
        a.warm_start = P.warm_start;
        a.ls_max_trials = P.ls_max_trials;
        a.ls_init = P.ls_init;
        a.max_iter = P.max_iter;
        a.Aglob = 0;
        a.precond = P.precond;
        if (all64) {
            a.tier = TIER_F64;
            a.tol = tol;
            a.stall_below = stall_floor(TIER_F64);
            tm.begin(1);
            CKR(launch_projection(P.projector, TIER_F64, ws, a, h->stream));
            tm.end();
            ++launches;
            tol_last = a.tol;
        } else {
            int tier = TIER_F32;
            if (P.precision == MDOT_PREC_FP32A || (P.precision == MDOT_PREC_AUTO && tol < kAccSwitch)) tier = TIER_F32A;
            a.tier = tier;
            a.tol = std::max(tol, (double)P.fp32_floor);
            a.stall_below = stall_floor(tier);
            tm.begin(0);
            CKR(launch_projection(P.projector, tier, ws, a, h->stream));
            tm.end();
            ++launches;
            ++launches32;
            tol_last = a.tol;
            bool polish_now = last && polish && tol < P.fp32_floor;
            if (last && polish && !polish_now) {
                // the last fp32 stage may have ended by the stall rule above its tolerance: read
                // its outcome (one synchronisation per solve) and polish in fp64 if so
                CKR(cudaMemcpyAsync(h->h_state, ws.st, sizeof(State), cudaMemcpyDeviceToHost, h->stream));
                CKR(cudaStreamSynchronize(h->stream));
                polish_now = h->h_state->status == ST_OK && !(h->h_state->gnorm <= a.tol);
            }
            if (polish_now) {
                // final stage below the fp32 noise floor, or stalled above its tolerance: continue
                // in fp64 entries from the fp32 iterate (same gamma, same smoothing, no warm start)
                StageArgs b = a;
                b.tier = TIER_F64;
                b.tol = tol;
                b.first = 0;
                b.warm_start = 2;
                b.stall_below = stall_floor(TIER_F64);
                tm.begin(1);
                CKR(launch_projection(P.projector, TIER_F64, ws, b, h->stream));
                tm.end();
                ++launches;
                tol_last = b.tol;
            }
        }
        ++stages;
        if (last) break;                                                   // exit at gamma_f
        double dg = (P.q - 1.0) * gamma;                                   // gamma <- min(q gamma, gamma_f)
        const double gnext = std::min(gamma + dg, gf);
        dg = gnext - gamma;
        ratio = (P.warm_start == 1) ? gnext / gamma : dg / dgamma_prev;    // warm start, Eq. (13)
        dgamma_prev = dg;
        gamma = gnext;
        if (stages > 100000) return MDOT_ERR_INVALID_ARG;
    }
    // Alg. 1, final step: round P(u, v; gamma_f) onto U(r, c); then the lower bound
    RoundArgs ra{};
    ra.gamma = gf;
    ra.G64 = gf * kLog2e;
    ra.u = ws.u;
    ra.v = ws.v;
    ra.r = r;
    ra.c = c;
    ra.ref = ws.lr;
    ra.Y = h->Y;
    ra.EC = h->EC;
    ra.ER = h->ER;
    ra.G_out = nullptr;
    ra.out = h->d_out;
    tm.begin(2);
    CKR(launch_round(ws, ra, h->stream));
    tm.end();
    LbArgs la{};
    la.gamma = gf;
    la.u = ws.u;
    la.r = r;
    la.c = c;
    la.gp = h->gp;
    la.out = h->d_out + 8;
    tm.begin(3);
    CKR(launch_lower_bound(ws, la, h->stream));
    tm.end();
    launches += 2;
    CKR(cudaMemcpyAsync(u_out, ws.u, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CKR(cudaMemcpyAsync(v_out, ws.v, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CKR(cudaMemcpyAsync(h->h_out, h->d_out, 16 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CKR(cudaMemcpyAsync(h->h_state, ws.st, sizeof(State), cudaMemcpyDeviceToHost, h->stream));
    CKR(cudaStreamSynchronize(h->stream));
    const State& S = *h->h_state;
    h->tags_used += (unsigned long long)S.evals + 4ull * (unsigned long long)(launches + 1);
    double tsum[8] = {0};
    tm.collect(tsum, tm.on ? &h->trace : nullptr);
    const double cost = h->h_out[0], lb = h->h_out[8];
    if (cost_out) *cost_out = cost;
    if (gap_out) *gap_out = cost - lb;
    mdot_status out = map_status(S.status);
    if (out == MDOT_OK && !(std::isfinite(cost) && std::isfinite(lb))) out = MDOT_ERR_NUMERIC;
    // the last stage must have reached the tolerance it was asked for (a stage that stalled above
    // it and could not be polished leaves the best iterate in the outputs)
    if (out == MDOT_OK && !(S.gnorm <= tol_last)) out = MDOT_ERR_NOT_CONVERGED;
    if (info) {
        memset(info, 0, sizeof(*info));
        info->status = out;
        info->stages = stages;
        info->evals = S.evals;
        info->evals_fp64 = S.evals64;
        info->iters = S.iters;
        info->ls_trials = S.ls_trials;
        info->grad_l1 = S.gnorm;
        info->gamma_f = gf;
        info->H_min = H;
        info->cost = cost;
        info->lower_bound = lb;
        info->gap_cert = cost - lb;
        info->t_stage_fp32_ms = tsum[0];
        info->t_stage_fp64_ms = tsum[1];
        info->t_round_ms = tsum[2];
        info->t_bound_ms = tsum[3];
        info->launches = launches;
        info->stalls = S.stalls;
        info->stage_launches_fp32 = launches32;
        info->tensor_cores = ws.tc;
    }
    return out;
}

}  // namespace

extern "C" {

mdot_status mdot_solve(mdot_handle* h, const double* r, const double* c, const float* C, int64_t n,
                       double eps_target, const mdot_params* prm, double* u_out, double* v_out,
                       double* cost_out, double* gap_out, mdot_info* info)
{
    CostSpec cs;
    cs.C = C;
    return solve_core(h, r, c, cs, n, eps_target, prm, u_out, v_out, cost_out, gap_out, info);
}

mdot_status mdot_solve_points(mdot_handle* h, const double* r, const double* c, const float* x, const float* y,
                              int32_t cost_kind, float scale, int64_t n, double eps_target,
                              const mdot_params* prm, double* u_out, double* v_out, double* cost_out,
                              double* gap_out, mdot_info* info)
{
    CostSpec cs;
    cs.X = x;
    cs.Y = y;
    cs.kind = cost_kind;
    cs.scale = scale;
    if (cost_kind == COST_DENSE) return MDOT_ERR_INVALID_ARG;
    return solve_core(h, r, c, cs, n, eps_target, prm, u_out, v_out, cost_out, gap_out, info);
}

mdot_status mdot_solve_host(mdot_handle* h, const double* r_host, const double* c_host, const float* C_host,
                            int64_t n, double eps_target, const mdot_params* prm, double* u_host,
                            double* v_host, double* cost_out, double* gap_out, mdot_info* info)
{
    if (!h || !r_host || !c_host || !C_host || !u_host || !v_host || n < 1 || n > h->max_n)
        return MDOT_ERR_INVALID_ARG;
    if (h->host_n < n) {
        cudaFree(h->d_r); cudaFree(h->d_c); cudaFree(h->d_u); cudaFree(h->d_v); cudaFree(h->d_C);
        h->d_r = h->d_c = h->d_u = h->d_v = nullptr;
        h->d_C = nullptr;
        h->host_n = 0;
        if (cudaMalloc(&h->d_r, n * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h->d_c, n * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h->d_u, n * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h->d_v, n * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h->d_C, (size_t)n * n * sizeof(float)) != cudaSuccess) {
            snprintf(g_err, sizeof g_err, "host-path buffers for n = %lld", (long long)n);
            return MDOT_ERR_OOM;
        }
        h->host_n = n;
    }
    CKR(cudaMemcpyAsync(h->d_r, r_host, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CKR(cudaMemcpyAsync(h->d_c, c_host, n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CKR(cudaMemcpyAsync(h->d_C, C_host, (size_t)n * n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CostSpec cs;
    cs.C = h->d_C;
    mdot_status s = solve_core(h, h->d_r, h->d_c, cs, n, eps_target, prm, h->d_u, h->d_v,
                               cost_out, gap_out, info);
    if (s == MDOT_ERR_INVALID_ARG || s == MDOT_ERR_CUDA) return s;
    CKR(cudaMemcpyAsync(u_host, h->d_u, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CKR(cudaMemcpyAsync(v_host, h->d_v, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CKR(cudaStreamSynchronize(h->stream));
    return s;
}

static mdot_status dual_eval_core(mdot_handle* h, const double* u, const double* v, double gamma,
                                  const CostSpec& cs, int64_t n, const double* ref_log_rP, int32_t precision,
                                  double* log_rP, double* log_cP, const double* r, const double* c,
                                  double* g_out)
{
    const int32_t tier_bits = precision & ~MDOT_PREC_TENSOR_CORES;
    if (!h || !u || !v || !cs.valid() || !log_rP || !log_cP || n < 1 || n > h->max_n || !(gamma > 0.0) ||
        !std::isfinite(gamma) || tier_bits < 0 || tier_bits > 3 || (g_out && (!r || !c)))
        return MDOT_ERR_INVALID_ARG;
    WS ws = h->ws;
    ws.n = (int)n;
    cs.apply(ws);
    CKR(select_cost_form(h, ws, (precision & MDOT_PREC_TENSOR_CORES) != 0));
    precision &= ~MDOT_PREC_TENSOR_CORES;
    EvalArgs a{};
    a.gamma = gamma;
    a.G64 = gamma * kLog2e;
    a.u = u;
    a.v = v;
    a.ref = ref_log_rP;
    if (g_out) {
        a.r = r;
        a.c = c;
        a.g_out = h->d_out + 15;
    }
    const int tier = (precision == MDOT_PREC_FP64) ? TIER_F64 : (precision == MDOT_PREC_FP32A) ? TIER_F32A : TIER_F32;
    CKR(reset_state(h));
    if (!h->de_ev[0]) {
        CKR(cudaEventCreate(&h->de_ev[0]));
        CKR(cudaEventCreate(&h->de_ev[1]));
    }
    h->de_ms = -1.0;
    CKR(cudaEventRecord(h->de_ev[0], h->stream));
    CKR(launch_dual_eval(tier, ws, a, h->stream));
    CKR(cudaEventRecord(h->de_ev[1], h->stream));
    CKR(cudaMemcpyAsync(log_rP, ws.lrtr, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CKR(cudaMemcpyAsync(log_cP, ws.lcout, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CKR(cudaMemcpyAsync(h->h_state, ws.st, sizeof(State), cudaMemcpyDeviceToHost, h->stream));
    if (g_out) CKR(cudaMemcpyAsync(h->h_out + 15, h->d_out + 15, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CKR(cudaStreamSynchronize(h->stream));
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, h->de_ev[0], h->de_ev[1]) == cudaSuccess) h->de_ms = ms;
    if (h->h_state->status != ST_OK) return map_status(h->h_state->status);
    if (g_out) *g_out = h->h_out[15];
    return MDOT_OK;
}

}  // extern "C"

namespace {

// mdot_problem -> BatchProblem; INVALID_ARG if malformed
mdot_status batch_problems(int32_t nprob, const mdot_problem* probs, std::vector<BatchProblem>& bp)
{
    bp.assign(nprob, BatchProblem{});
    for (int k = 0; k < nprob; ++k) {
        const mdot_problem& q = probs[k];
        BatchProblem& b = bp[k];
        memset(&b, 0, sizeof(b));
        const bool dense = q.C != nullptr;
        if (q.n < 1 || q.n > MDOT_BATCH_MAX_N || !q.r || !q.c ||
            (!dense && (!q.x || !q.y || (q.cost_kind != MDOT_COST_SQEUCLID && q.cost_kind != MDOT_COST_L1) ||
                        !(q.scale > 0.0f) || !std::isfinite(q.scale))) ||
            (!(q.gamma_f > 0.0) && !(q.eps_target > 0.0 && std::isfinite(q.eps_target))))
            return MDOT_ERR_INVALID_ARG;
        b.n = (int)q.n;
        b.kind = dense ? COST_DENSE : q.cost_kind;
        b.scale = q.scale;
        b.eps = q.eps_target;
        b.gamma_f = q.gamma_f;
        b.r = q.r; b.c = q.c; b.C = q.C; b.X = q.x; b.Y = q.y;
        b.u_out = q.u_out; b.v_out = q.v_out;
    }
    return MDOT_OK;
}

mdot_status batch_params(const mdot_params* prm, mdot_params& P)
{
    if (prm) P = *prm; else mdot_default_params(&P);
    if (params_ok(P) != MDOT_OK || P.precision == MDOT_PREC_FP64 || P.projector != 0 || P.stop_entropy != 0 ||
        P.precond != 0)
        return MDOT_ERR_INVALID_ARG;
    return MDOT_OK;
}

// The batched solve of bp: one persistent launch per (cost form, tile variant) -- the variant of a
// problem is the handle's table entry for its size bucket, or `forced` (>= 0) for every problem;
// inside a launch, problems by decreasing n.  *ms (nullable): device time of all launches.
mdot_status batch_core(mdot_handle* h, const std::vector<BatchProblem>& bp, const mdot_params& P,
                       std::vector<BatchResult>& br, int forced, double* ms)
{
    const int nprob = (int)bp.size();
    if (!h->b_slots) {
        int bps[kBatchVariants] = {0, 0};
        CKR(configure_batch_kernels(bps));
        int grid_max = 0;
        for (int v = 0; v < kBatchVariants; ++v) {
            if (bps[v] < 1) return MDOT_ERR_INVALID_ARG;
            h->b_grid[v] = h->sms * bps[v];
            grid_max = std::max(grid_max, h->b_grid[v]);
        }
        if (cudaMalloc(&h->b_slots, (size_t)grid_max * kSlotDoubles * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&h->b_next, 4 * sizeof(unsigned int)) != cudaSuccess) {
            snprintf(g_err, sizeof g_err, "batch workspace allocation failed");
            return MDOT_ERR_OOM;
        }
    }
    if (h->b_cap < nprob) {
        cudaFree(h->b_probs); cudaFree(h->b_results); cudaFree(h->b_order);
        h->b_probs = nullptr; h->b_results = nullptr; h->b_order = nullptr; h->b_cap = 0;
        if (cudaMalloc(&h->b_probs, nprob * sizeof(BatchProblem)) != cudaSuccess ||
            cudaMalloc(&h->b_results, nprob * sizeof(BatchResult)) != cudaSuccess ||
            cudaMalloc(&h->b_order, nprob * sizeof(int)) != cudaSuccess) {
            snprintf(g_err, sizeof g_err, "batch descriptor allocation failed");
            return MDOT_ERR_OOM;
        }
        h->b_cap = nprob;
    }
    br.assign(nprob, BatchResult{});
    CKR(cudaMemcpyAsync(h->b_probs, bp.data(), nprob * sizeof(BatchProblem), cudaMemcpyHostToDevice, h->stream));
    if (!h->de_ev[0]) {
        CKR(cudaEventCreate(&h->de_ev[0]));
        CKR(cudaEventCreate(&h->de_ev[1]));
    }
    double total_ms = 0.0;
    for (int kind = 0; kind < 3; ++kind) {
        for (int v = 0; v < kBatchVariants; ++v) {
            std::vector<int> order;
            for (int k = 0; k < nprob; ++k) {
                const int vk = forced >= 0 ? forced : h->b_variant[batch_bucket(bp[k].n)];
                if (bp[k].kind == kind && vk == v) order.push_back(k);
            }
            if (order.empty()) continue;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return bp[x].n > bp[y].n; });
            CKR(cudaMemcpyAsync(h->b_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice,
                                h->stream));
            CKR(cudaMemsetAsync(h->b_next, 0, sizeof(unsigned int), h->stream));
            BatchArgs a{};
            a.nprob = (int)order.size();
            a.probs = h->b_probs;
            a.results = h->b_results;
            a.order = h->b_order;
            a.next = h->b_next;
            a.slots = h->b_slots;
            a.slot_doubles = kSlotDoubles;
            a.gamma_i = P.gamma_i; a.p = P.p; a.q = P.q; a.c1 = P.ls_c1; a.c2 = P.ls_c2;
            a.fp32_floor = P.fp32_floor; a.final_tol = P.final_tol;
            a.ls_max_trials = P.ls_max_trials; a.max_iter = P.max_iter; a.warm_start = P.warm_start;
            a.precision = P.precision;
            a.smoothing = P.smoothing;
            a.ls_init = P.ls_init;
            a.tensor_cores = P.tensor_cores;
            a.polish_iters = P.polish_iters;
            CKR(cudaEventRecord(h->de_ev[0], h->stream));
            CKR(launch_batch(kind, v, std::min(h->b_grid[v], a.nprob), a, h->stream));
            CKR(cudaEventRecord(h->de_ev[1], h->stream));
            CKR(cudaStreamSynchronize(h->stream));     // the order buffer is reused by the next launch
            float t = 0.0f;
            CKR(cudaEventElapsedTime(&t, h->de_ev[0], h->de_ev[1]));
            total_ms += t;
        }
    }
    CKR(cudaMemcpyAsync(br.data(), h->b_results, nprob * sizeof(BatchResult), cudaMemcpyDeviceToHost, h->stream));
    CKR(cudaStreamSynchronize(h->stream));
    if (ms) *ms = total_ms;
    return MDOT_OK;
}

// Finish one batched problem whose last stage the batch kernel left above its tolerance (its fp32
// part stalled and the fp64 polish on its one SM did not get there): the single-problem solver's
// fp64 stage on every SM of the handle, from the batch's potentials (q.u_out, q.v_out), at the
// same gamma_f, smoothing and floored tolerance, then rounding (Alg. 3) and the bound as in
// solve_core.  The result record is updated in place (evaluation counts added).
mdot_status batch_finish(mdot_handle* h, const BatchProblem& q, const mdot_params& P, BatchResult& br)
{
    const int n = q.n;
    WS ws = h->ws;
    ws.n = n;
    ws.r = q.r;
    ws.c = q.c;
    CostSpec cs;
    cs.kind = q.kind;
    cs.C = q.C;
    cs.X = q.X;
    cs.Y = q.Y;
    cs.scale = q.scale;
    cs.apply(ws);
    CKR(select_cost_form(h, ws, P.tensor_cores != 0));
    CKR(reset_state(h, P.wait_limit_us));
    CKR(cudaMemcpyAsync(ws.u, q.u_out, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CKR(cudaMemcpyAsync(ws.v, q.v_out, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    const double gf = br.gamma_f;
    const double eps_d = br.H_min / std::pow(gf, P.p);      // the batch's last stage: gamma = gamma_f
    double tol = std::max(eps_d / 2.0, 1e-13 + 1e-15 * gf);
    if (P.final_tol > 0.0) tol = P.final_tol;
    tol = std::max(tol, (double)P.fp32_floor);             // the batched form's floor
    StageArgs a{};
    a.gamma = gf;
    a.G64 = gf * kLog2e;
    a.w = eps_d;                                           // smoothing 0 or 1: the same at gamma_f
    a.ratio = 0.0;
    a.c1 = P.ls_c1;
    a.c2 = P.ls_c2;
    a.first = 0;
    a.warm_start = 2;                                      // continue from the given potentials
    a.ls_max_trials = P.ls_max_trials;
    a.ls_init = P.ls_init;
    a.max_iter = P.max_iter;
    a.Aglob = 0;
    a.precond = 0;
    a.tier = TIER_F64;
    a.tol = tol;
    a.stall_below = stall_floor(TIER_F64);
    CKR(launch_projection(0, TIER_F64, ws, a, h->stream));
    RoundArgs ra{};
    ra.gamma = gf;
    ra.G64 = gf * kLog2e;
    ra.u = ws.u;
    ra.v = ws.v;
    ra.r = q.r;
    ra.c = q.c;
    ra.ref = ws.lr;
    ra.Y = h->Y;
    ra.EC = h->EC;
    ra.ER = h->ER;
    ra.G_out = nullptr;
    ra.out = h->d_out;
    CKR(launch_round(ws, ra, h->stream));
    LbArgs la{};
    la.gamma = gf;
    la.u = ws.u;
    la.r = q.r;
    la.c = q.c;
    la.gp = h->gp;
    la.out = h->d_out + 8;
    CKR(launch_lower_bound(ws, la, h->stream));
    CKR(cudaMemcpyAsync(q.u_out, ws.u, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CKR(cudaMemcpyAsync(q.v_out, ws.v, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CKR(cudaMemcpyAsync(h->h_out, h->d_out, 16 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CKR(cudaMemcpyAsync(h->h_state, ws.st, sizeof(State), cudaMemcpyDeviceToHost, h->stream));
    CKR(cudaStreamSynchronize(h->stream));
    const State& S = *h->h_state;
    br.cost = h->h_out[0];
    br.lower_bound = h->h_out[8];
    br.grad_l1 = S.gnorm;
    br.evals += S.evals;
    br.iters += S.iters;
    br.status = (S.status != ST_OK) ? S.status : (S.gnorm <= tol ? (int)ST_OK : (int)ST_CAP);
    return MDOT_OK;
}

}  // namespace

extern "C" {

mdot_status mdot_solve_batch(mdot_handle* h, int32_t nprob, const mdot_problem* probs, const mdot_params* prm,
                             mdot_result* results)
{
    if (!h || nprob < 0 || (nprob > 0 && (!probs || !results))) return MDOT_ERR_INVALID_ARG;
    if (nprob == 0) return MDOT_OK;
    mdot_params P;
    if (batch_params(prm, P) != MDOT_OK) return MDOT_ERR_INVALID_ARG;
    std::vector<BatchProblem> bp;
    if (batch_problems(nprob, probs, bp) != MDOT_OK) return MDOT_ERR_INVALID_ARG;
    // with precision AUTO a problem the batch leaves above its tolerance is finished on every SM
    // (batch_finish), which starts from its potentials: problems that asked for none get some in
    // the handle's scratch (problems larger than the handle's max_n cannot be finished)
    const bool finish = P.precision == MDOT_PREC_AUTO && P.polish_iters > 0;
    if (finish) {
        size_t need = 0;
        for (const BatchProblem& q : bp)
            if ((!q.u_out || !q.v_out) && q.n <= h->max_n) need += 2 * (size_t)q.n;
        if (need > h->b_uv_cap) {
            cudaFree(h->b_uv);
            h->b_uv = nullptr;
            h->b_uv_cap = 0;
            if (cudaMalloc(&h->b_uv, need * sizeof(double)) != cudaSuccess) {
                snprintf(g_err, sizeof g_err, "batch potential scratch allocation failed");
                return MDOT_ERR_OOM;
            }
            h->b_uv_cap = need;
        }
        size_t o = 0;
        for (BatchProblem& q : bp)
            if ((!q.u_out || !q.v_out) && q.n <= h->max_n) {
                // only the missing output is replaced: the caller still receives the one it asked for
                if (!q.u_out) q.u_out = h->b_uv + o;
                if (!q.v_out) q.v_out = h->b_uv + o + q.n;
                o += 2 * (size_t)q.n;
            }
    }
    std::vector<BatchResult> br;
    mdot_status st = batch_core(h, bp, P, br, -1, nullptr);
    if (st != MDOT_OK) return st;
    if (finish)
        for (int k = 0; k < nprob; ++k)
            if (br[k].status == ST_CAP && bp[k].n <= h->max_n) {
                st = batch_finish(h, bp[k], P, br[k]);
                if (st != MDOT_OK) return st;
            }
    for (int k = 0; k < nprob; ++k) {
        const BatchResult& b = br[k];
        mdot_result& r = results[k];
        memset(&r, 0, sizeof(r));
        r.status = (b.status >= 10) ? MDOT_ERR_INVALID_ARG : map_status(b.status);
        if (r.status == MDOT_OK && !(std::isfinite(b.cost) && std::isfinite(b.lower_bound))) r.status = MDOT_ERR_NUMERIC;
        r.stages = b.stages;
        r.evals = b.evals;
        r.iters = b.iters;
        r.cost = b.cost;
        r.lower_bound = b.lower_bound;
        r.gap_cert = b.cost - b.lower_bound;
        r.grad_l1 = b.grad_l1;
        r.gamma_f = b.gamma_f;
        r.H_min = b.H_min;
    }
    return MDOT_OK;
}

mdot_status mdot_tune_batch(mdot_handle* h, int32_t nprob, const mdot_problem* probs, const mdot_params* prm,
                            int32_t sample, mdot_batch_tuning* out)
{
    if (!h || nprob < 1 || !probs || !out || sample < 1) return MDOT_ERR_INVALID_ARG;
    mdot_params P;
    if (batch_params(prm, P) != MDOT_OK) return MDOT_ERR_INVALID_ARG;
    std::vector<BatchProblem> bp;
    if (batch_problems(nprob, probs, bp) != MDOT_OK) return MDOT_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    // the timing batch: up to `sample` problems evenly spaced in size order, no potentials written,
    // stopped at gamma_f <= 2^12 (the tables' relative speed is that of the per-evaluation work and
    // of the packing, not of the schedule's length)
    std::vector<int> order(nprob);
    for (int k = 0; k < nprob; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return bp[x].n < bp[y].n; });
    const int m = std::min(sample, nprob);
    std::vector<BatchProblem> pick;
    for (int k = 0; k < m; ++k) {
        BatchProblem q = bp[order[(size_t)k * nprob / m]];
        q.u_out = nullptr;
        q.v_out = nullptr;
        if (!(q.gamma_f > 0.0) || q.gamma_f > 4096.0) q.gamma_f = 4096.0;
        pick.push_back(q);
    }
    int saved[kBatchBuckets];
    for (int b = 0; b < kBatchBuckets; ++b) saved[b] = h->b_variant[b];
    int best_k = 0;
    double best = -1.0;
    for (int k = 0; k <= kBatchBuckets; ++k) {
        for (int b = 0; b < kBatchBuckets; ++b) h->b_variant[b] = (b < k) ? 1 : 0;
        std::vector<BatchResult> br;
        double ms = 0.0;
        const mdot_status st = batch_core(h, pick, P, br, -1, &ms);
        if (st != MDOT_OK) {
            for (int b = 0; b < kBatchBuckets; ++b) h->b_variant[b] = saved[b];
            return st;
        }
        out->seconds[k] = ms / 1e3;
        if (best < 0.0 || ms < best) {
            best = ms;
            best_k = k;
        }
    }
    for (int b = 0; b < kBatchBuckets; ++b) h->b_variant[b] = out->variant[b] = (b < best_k) ? 1 : 0;
    out->narrow_below = best_k;
    return MDOT_OK;
}

mdot_status mdot_set_batch_tuning(mdot_handle* h, const mdot_batch_tuning* t)
{
    if (!h || !t) return MDOT_ERR_INVALID_ARG;
    for (int b = 0; b < kBatchBuckets; ++b)
        if (t->variant[b] < 0 || t->variant[b] >= kBatchVariants) return MDOT_ERR_INVALID_ARG;
    for (int b = 0; b < kBatchBuckets; ++b) h->b_variant[b] = t->variant[b];
    return MDOT_OK;
}

mdot_status mdot_dual_eval(mdot_handle* h, const double* u, const double* v, double gamma, const float* C,
                           int64_t n, const double* ref_log_rP, int32_t precision, double* log_rP,
                           double* log_cP, const double* r, const double* c, double* g_out)
{
    CostSpec cs;
    cs.C = C;
    return dual_eval_core(h, u, v, gamma, cs, n, ref_log_rP, precision, log_rP, log_cP, r, c, g_out);
}

mdot_status mdot_solve_trace(const mdot_handle* h, int32_t max_rows, mdot_trace_row* rows, int32_t* count)
{
    if (!h || !count || max_rows < 0 || (max_rows > 0 && !rows)) return MDOT_ERR_INVALID_ARG;
    *count = (int32_t)h->trace.size();
    for (int32_t k = 0; k < max_rows && k < *count; ++k) rows[k] = h->trace[k];
    return h->trace.empty() ? MDOT_NOT_READY : MDOT_OK;
}

mdot_status mdot_dual_eval_time(const mdot_handle* h, double* ms_out)
{
    if (!h || !ms_out) return MDOT_ERR_INVALID_ARG;
    *ms_out = h->de_ms;
    return h->de_ms >= 0.0 ? MDOT_OK : MDOT_NOT_READY;
}

mdot_status mdot_dual_eval_points(mdot_handle* h, const double* u, const double* v, double gamma,
                                  const float* x, const float* y, int32_t cost_kind, float scale, int64_t n,
                                  const double* ref_log_rP, int32_t precision, double* log_rP, double* log_cP,
                                  const double* r, const double* c, double* g_out)
{
    CostSpec cs;
    cs.X = x;
    cs.Y = y;
    cs.kind = cost_kind;
    cs.scale = scale;
    if (cost_kind == COST_DENSE) return MDOT_ERR_INVALID_ARG;
    return dual_eval_core(h, u, v, gamma, cs, n, ref_log_rP, precision, log_rP, log_cP, r, c, g_out);
}

mdot_status mdot_round(mdot_handle* h, const double* u, const double* v, double gamma, const float* C,
                       const double* r, const double* c, int64_t n, double* cost_out, double* G_out)
{
    if (!h || !u || !v || !C || !r || !c || !cost_out || n < 1 || n > h->max_n || !(gamma > 0.0) ||
        !std::isfinite(gamma))
        return MDOT_ERR_INVALID_ARG;
    WS ws = h->ws;
    ws.n = (int)n;
    ws.C = C;
    RoundArgs ra{};
    ra.gamma = gamma;
    ra.G64 = gamma * kLog2e;
    ra.u = u;
    ra.v = v;
    ra.r = r;
    ra.c = c;
    ra.ref = nullptr;
    ra.Y = h->Y;
    ra.EC = h->EC;
    ra.ER = h->ER;
    ra.G_out = G_out;
    ra.out = h->d_out;
    CKR(reset_state(h));
    CKR(launch_round(ws, ra, h->stream));
    CKR(cudaMemcpyAsync(h->h_out, h->d_out, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CKR(cudaMemcpyAsync(h->h_state, ws.st, sizeof(State), cudaMemcpyDeviceToHost, h->stream));
    CKR(cudaStreamSynchronize(h->stream));
    *cost_out = h->h_out[0];
    if (h->h_state->status != ST_OK) return MDOT_ERR_TIMEOUT;
    return std::isfinite(h->h_out[0]) ? MDOT_OK : MDOT_ERR_NUMERIC;
}

mdot_status mdot_lower_bound(mdot_handle* h, const double* u, double gamma, const float* C, const double* r,
                             const double* c, int64_t n, double* lb_out)
{
    if (!h || !u || !C || !r || !c || !lb_out || n < 1 || n > h->max_n || !(gamma > 0.0)) return MDOT_ERR_INVALID_ARG;
    WS ws = h->ws;
    ws.n = (int)n;
    ws.C = C;
    LbArgs la{};
    la.gamma = gamma;
    la.u = u;
    la.r = r;
    la.c = c;
    la.gp = h->gp;
    la.out = h->d_out + 8;
    CKR(reset_state(h));
    CKR(launch_lower_bound(ws, la, h->stream));
    CKR(cudaMemcpyAsync(h->h_out, h->d_out, 16 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CKR(cudaMemcpyAsync(h->h_state, ws.st, sizeof(State), cudaMemcpyDeviceToHost, h->stream));
    CKR(cudaStreamSynchronize(h->stream));
    *lb_out = h->h_out[8];
    return h->h_state->status == ST_OK ? MDOT_OK : MDOT_ERR_TIMEOUT;
}

}  // extern "C"
