// Serving runtime (declared in include/mdot.h): a request loop with continuous batching on one
// GPU.  Requests up to big_n are admitted in arrival order as soon as their workspace fits the
// pool (the HBM budget given at creation); every admission round becomes one persistent batched
// launch (one CTA per problem, the solver of batch_kernels.cuh) on one of a few streams, so
// launches admitted while others still run overlap on the device and take SMs as earlier problems
// finish.  Each problem reports completion through a flag in mapped host memory, so its workspace
// returns to the pool (and the next request is admitted) without waiting for the rest of its
// launch.  Larger requests would hold one SM for a long time; they go to a few "big lanes", each
// a cooperative solve (the stage kernels of the single-problem solver) on a share of the SMs.
// The SMs are partitioned so that every resident CTA fits at once: batched problems in flight
// <= SMs - lanes x CTAs per lane - 8.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch_kernels.cuh"
#include "launch.h"
#include "mdot.h"

namespace mdot {
mdot_status params_valid(const mdot_params& P);
mdot_status status_of(int st);
void set_last_error(const char* msg);
}  // namespace mdot

using namespace mdot;

namespace {

constexpr int kLanes = 4;            // streams the launches rotate over
constexpr int kRecords = 32;         // launches in flight at most
constexpr int kRecordCap = 256;      // problems per launch at most
constexpr int kStrideAlign = 32;     // workspace vector stride granularity (elements)
constexpr int kMaxBigLanes = 16;     // concurrent cooperative solves at most

// First-fit allocator over the workspace pool (offsets and lengths in doubles).
struct Pool {
    std::map<size_t, size_t> free_blocks;
    size_t total = 0, used = 0;
    void init(size_t n)
    {
        free_blocks.clear();
        free_blocks[0] = n;
        total = n;
        used = 0;
    }
    bool alloc(size_t len, size_t& off)
    {
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second < len) continue;
            off = it->first;
            const size_t rest = it->second - len;
            free_blocks.erase(it);
            if (rest) free_blocks[off + len] = rest;
            used += len;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t len)
    {
        used -= len;
        auto it = free_blocks.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_blocks.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_blocks.erase(nx);
        }
        if (it != free_blocks.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_blocks.erase(it);
            }
        }
    }
};

// One launch: its device descriptor arrays, mapped result/flag arrays and bookkeeping.
struct Record {
    bool busy = false;
    int m = 0, remaining = 0;
    BatchProblem* d_probs = nullptr;
    int* d_order = nullptr;
    unsigned int* d_next = nullptr;
    BatchProblem* h_probs = nullptr;     // pinned staging of the descriptors
    int* h_order = nullptr;
    BatchResult* h_res = nullptr;        // mapped pinned memory, written by the kernel
    int* h_done = nullptr;
    BatchResult* d_res = nullptr;        // device aliases of the two
    int* d_done = nullptr;
    cudaEvent_t ev = nullptr;
    uint64_t ticket[kRecordCap];
    size_t off[kRecordCap], len[kRecordCap];
    bool reported[kRecordCap];
};

struct Request {
    uint64_t ticket;
    mdot_problem p;
    size_t len;          // workspace doubles
    int stride;
    int kind;
};

int cost_kind_of(const mdot_problem& q) { return q.C ? COST_DENSE : q.cost_kind; }

bool problem_ok(const mdot_problem& q)
{
    const bool dense = q.C != nullptr;
    return q.n >= 1 && q.n <= MDOT_BATCH_MAX_N && q.r && q.c &&
           (dense || (q.x && q.y && (q.cost_kind == MDOT_COST_SQEUCLID || q.cost_kind == MDOT_COST_L1) &&
                      q.scale > 0.0f && std::isfinite(q.scale))) &&
           ((q.gamma_f > 0.0 && std::isfinite(q.gamma_f)) || (q.eps_target > 0.0 && std::isfinite(q.eps_target)));
}

// A big lane: one cooperative solver handle on a share of the SMs, served by its own thread.
struct BigLane {
    mdot_handle* h = nullptr;
    cudaStream_t stream = nullptr;
    double *u = nullptr, *v = nullptr;   // potentials when the request has no output buffers
    std::thread thread;
};

}  // namespace

namespace mdot {
mdot_status handle_set_grid(mdot_handle* h, int G);
}

struct mdot_server {
    int dev = 0;
    mdot_params prm{};
    cudaStream_t lanes[kLanes] = {};
    int next_lane = 0;
    double* pool_mem = nullptr;
    Pool pool;
    Record rec[kRecords];
    std::mutex mu;
    std::condition_variable cv_work;     // wakes the worker
    std::condition_variable cv_done;     // wakes waiters
    std::deque<Request> pending;         // batched route
    std::deque<Request> big_pending;     // big lanes
    BigLane big[kMaxBigLanes];
    int64_t big_n = 2048;
    int big_lanes = 0;
    int batch_inflight = 0, batch_cap = 0;
    std::unordered_map<uint64_t, int> state;          // 0 queued, 1 running, 2 finished
    std::unordered_map<uint64_t, mdot_result> finished;
    uint64_t next_ticket = 1;
    bool stop = false;
    cudaError_t fatal = cudaSuccess;
    std::thread worker;
};

namespace {

mdot_result to_result(const BatchResult& b)
{
    mdot_result r;
    memset(&r, 0, sizeof(r));
    r.status = (b.status >= 10) ? MDOT_ERR_INVALID_ARG : status_of(b.status);
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
    return r;
}

// Completed problems (flags in host memory): results out, workspace back to the pool.
// Called with the lock held.  Returns whether any launch is still in flight.
bool collect(mdot_server* s)
{
    bool inflight = false;
    for (Record& r : s->rec) {
        if (!r.busy) continue;
        for (int i = 0; i < r.m; ++i) {
            if (r.reported[i] || reinterpret_cast<volatile int*>(r.h_done)[i] == 0) continue;
            std::atomic_thread_fence(std::memory_order_acquire);
            BatchResult b;
            memcpy(&b, reinterpret_cast<const void*>(const_cast<const BatchResult*>(r.h_res + i)), sizeof(b));
            s->finished[r.ticket[i]] = to_result(b);
            s->state[r.ticket[i]] = 2;
            s->pool.release(r.off[i], r.len[i]);
            --s->batch_inflight;
            r.reported[i] = true;
            --r.remaining;
            s->cv_done.notify_all();
        }
        // the descriptor arrays are reusable once the launch itself has finished
        if (r.remaining == 0 && cudaEventQuery(r.ev) == cudaSuccess) r.busy = false;
        if (r.busy) inflight = true;
    }
    return inflight;
}

// Admit queued requests in arrival order while they fit; one launch per admission round (the
// requests of one round share the cost form of the first one).  Lock held.
cudaError_t admit(mdot_server* s)
{
    while (!s->pending.empty()) {
        Record* r = nullptr;
        for (Record& x : s->rec)
            if (!x.busy) { r = &x; break; }
        if (!r) return cudaSuccess;
        const int kind = s->pending.front().kind;
        int m = 0;
        while (!s->pending.empty() && m < kRecordCap && s->pending.front().kind == kind &&
               s->batch_inflight < s->batch_cap) {
            Request& q = s->pending.front();
            size_t off = 0;
            if (!s->pool.alloc(q.len, off)) break;          // strict arrival order: wait for room
            ++s->batch_inflight;
            BatchProblem& b = r->h_probs[m];
            memset(&b, 0, sizeof(b));
            b.n = (int)q.p.n;
            b.kind = kind;
            b.scale = q.p.scale;
            b.eps = q.p.eps_target;
            b.gamma_f = q.p.gamma_f;
            b.r = q.p.r; b.c = q.p.c; b.C = q.p.C; b.X = q.p.x; b.Y = q.p.y;
            b.u_out = q.p.u_out; b.v_out = q.p.v_out;
            b.slot = s->pool_mem + off;
            b.slot_stride = q.stride;
            r->ticket[m] = q.ticket;
            r->off[m] = off;
            r->len[m] = q.len;
            r->reported[m] = false;
            r->h_done[m] = 0;
            s->state[q.ticket] = 1;
            s->pending.pop_front();
            ++m;
        }
        if (m == 0) return cudaSuccess;
        // largest problems first inside the launch
        for (int i = 0; i < m; ++i) r->h_order[i] = i;
        std::stable_sort(r->h_order, r->h_order + m, [&](int x, int y) { return r->h_probs[x].n > r->h_probs[y].n; });
        r->busy = true;
        r->m = m;
        r->remaining = m;
        cudaStream_t st = s->lanes[s->next_lane];
        s->next_lane = (s->next_lane + 1) % kLanes;
        cudaError_t e = cudaMemcpyAsync(r->d_probs, r->h_probs, m * sizeof(BatchProblem), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(r->d_order, r->h_order, m * sizeof(int), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(r->d_next, 0, sizeof(unsigned int), st);
        if (e != cudaSuccess) return e;
        BatchArgs a{};
        a.nprob = m;
        a.probs = r->d_probs;
        a.results = r->d_res;
        a.order = r->d_order;
        a.next = r->d_next;
        a.done = r->d_done;
        a.slots = s->pool_mem;            // every problem brings its own workspace
        a.slot_doubles = 0;
        const mdot_params& P = s->prm;
        a.gamma_i = P.gamma_i; a.p = P.p; a.q = P.q; a.c1 = P.ls_c1; a.c2 = P.ls_c2;
        a.fp32_floor = P.fp32_floor; a.final_tol = P.final_tol;
        a.ls_max_trials = P.ls_max_trials; a.max_iter = P.max_iter; a.warm_start = P.warm_start;
        a.precision = P.precision;
        a.smoothing = P.smoothing;
        a.ls_init = P.ls_init;
        a.tensor_cores = P.tensor_cores;
        a.polish_iters = P.polish_iters;
        e = launch_batch(kind, 0, m, a, st);       // the wide variant: one problem per SM
        if (e == cudaSuccess) e = cudaEventRecord(r->ev, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void fail_all(mdot_server* s)
{
    // a CUDA failure: every request not yet finished ends with MDOT_ERR_CUDA
    for (auto& kv : s->state) {
        if (kv.second == 2) continue;
        mdot_result r;
        memset(&r, 0, sizeof(r));
        r.status = MDOT_ERR_CUDA;
        s->finished[kv.first] = r;
        kv.second = 2;
    }
    s->pending.clear();
    s->big_pending.clear();
    for (Record& r : s->rec) r.busy = false;
    s->cv_done.notify_all();
}

void worker_loop(mdot_server* s)
{
    cudaSetDevice(s->dev);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool inflight = false;
        if (s->fatal == cudaSuccess) {
            inflight = collect(s);
            const cudaError_t e = admit(s);
            if (e != cudaSuccess) {
                s->fatal = e;
                fail_all(s);
            }
            for (const Record& r : s->rec) inflight = inflight || r.busy;
        }
        if (s->stop && s->pending.empty() && !inflight) break;
        if (inflight) {
            // poll the completion flags at a fine interval while work is on the GPU
            s->cv_work.wait_for(lk, std::chrono::microseconds(20));
        } else {
            s->cv_work.wait(lk, [&] { return s->stop || (!s->pending.empty() && s->fatal == cudaSuccess); });
        }
    }
}

mdot_result solve_big(mdot_server* s, BigLane& L, const Request& q)
{
    mdot_params P = s->prm;
    if (q.p.gamma_f > 0.0) P.gamma_f = q.p.gamma_f;
    const double eps = q.p.eps_target > 0.0 ? q.p.eps_target : 1.0;     // unused when gamma_f is set
    double* u = q.p.u_out ? q.p.u_out : L.u;
    double* v = q.p.v_out ? q.p.v_out : L.v;
    double cost = 0.0, gap = 0.0;
    mdot_info info;
    memset(&info, 0, sizeof(info));
    // A cooperative launch is refused (not queued) while the SMs it needs are busy; the SM
    // partition makes that rare, and the solve is then simply started again a moment later.
    mdot_status st = MDOT_ERR_CUDA;
    for (int attempt = 0; attempt < 2000; ++attempt) {
        st = q.p.C ? mdot_solve(L.h, q.p.r, q.p.c, q.p.C, q.p.n, eps, &P, u, v, &cost, &gap, &info)
                   : mdot_solve_points(L.h, q.p.r, q.p.c, q.p.x, q.p.y, q.p.cost_kind, q.p.scale, q.p.n, eps, &P, u,
                                       v, &cost, &gap, &info);
        if (st != MDOT_ERR_CUDA || cudaGetLastError() != cudaErrorCooperativeLaunchTooLarge) break;
        cudaStreamSynchronize(L.stream);
        std::this_thread::sleep_for(std::chrono::microseconds(500));
    }
    if (st == MDOT_ERR_CUDA)
        fprintf(stderr, "mdot server: cooperative solve of n = %lld failed: %s\n", (long long)q.p.n,
                mdot_last_error());
    mdot_result r;
    memset(&r, 0, sizeof(r));
    r.status = st;
    r.stages = info.stages;
    r.evals = info.evals;
    r.iters = info.iters;
    r.cost = cost;
    r.lower_bound = info.lower_bound;
    r.gap_cert = gap;
    r.grad_l1 = info.grad_l1;
    r.gamma_f = info.gamma_f;
    r.H_min = info.H_min;
    return r;
}

void big_loop(mdot_server* s, int lane)
{
    cudaSetDevice(s->dev);
    BigLane& L = s->big[lane];
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        s->cv_work.wait(lk, [&] { return s->stop || !s->big_pending.empty(); });
        if (s->big_pending.empty()) {
            if (s->stop) break;
            continue;
        }
        const Request q = s->big_pending.front();
        s->big_pending.pop_front();
        s->state[q.ticket] = 1;
        lk.unlock();
        const mdot_result r = solve_big(s, L, q);
        lk.lock();
        s->finished[q.ticket] = r;
        s->state[q.ticket] = 2;
        s->cv_done.notify_all();
    }
}

void destroy_records(mdot_server* s)
{
    for (Record& r : s->rec) {
        cudaFree(r.d_probs); cudaFree(r.d_order); cudaFree(r.d_next);
        cudaFreeHost(r.h_probs); cudaFreeHost(r.h_order); cudaFreeHost(r.h_res); cudaFreeHost(r.h_done);
        if (r.ev) cudaEventDestroy(r.ev);
    }
}

}  // namespace

extern "C" {

mdot_status mdot_server_create(mdot_server** out, uint64_t workspace_bytes, const mdot_params* prm,
                               const mdot_server_config* cfg)
{
    if (!out) return MDOT_ERR_INVALID_ARG;
    *out = nullptr;
    mdot_params P;
    if (prm) P = *prm; else mdot_default_params(&P);
    if (params_valid(P) != MDOT_OK || P.precision == MDOT_PREC_FP64 || P.projector != 0 || P.stop_entropy != 0 ||
        P.precond != 0)
        return MDOT_ERR_INVALID_ARG;
    const size_t pool_doubles = (size_t)(workspace_bytes / sizeof(double));
    if (pool_doubles < batch_slot_doubles(kStrideAlign)) return MDOT_ERR_INVALID_ARG;
    mdot_server* s = new mdot_server();
    s->prm = P;
    int bps[kBatchVariants] = {0, 0};
    cudaError_t e = cudaGetDevice(&s->dev);
    if (e == cudaSuccess) e = configure_batch_kernels(bps);
    if (e == cudaSuccess && bps[0] < 1) e = cudaErrorInvalidConfiguration;
    for (int i = 0; i < kLanes && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&s->lanes[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s->pool_mem, pool_doubles * sizeof(double));
    for (Record& r : s->rec) {
        if (e != cudaSuccess) break;
        e = cudaMalloc(&r.d_probs, kRecordCap * sizeof(BatchProblem));
        if (e == cudaSuccess) e = cudaMalloc(&r.d_order, kRecordCap * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&r.d_next, sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaHostAlloc(&r.h_probs, kRecordCap * sizeof(BatchProblem), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaHostAlloc(&r.h_order, kRecordCap * sizeof(int), cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaHostAlloc(&r.h_res, kRecordCap * sizeof(BatchResult), cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostAlloc(&r.h_done, kRecordCap * sizeof(int), cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&r.d_res, r.h_res, 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(&r.d_done, r.h_done, 0);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming);
    }
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->dev);
    const int gmax = std::min(sms, 160);
    // defaults measured on the serving trace (200 requests, n log-uniform on [128, 8192], gaps
    // 1e-4 .. 1e-7, requests above n = 2048 holding ~90 % of the work): three lanes of 29 % of the
    // SMs each for n > 2048 served 5.50 problems/s, against 5.19 with two lanes of 64 SMs, 4.74 with
    // four of 32, 4.58 with four of 32 from n > 1024 and 3.25 with two lanes of a quarter of the SMs
    s->big_n = (cfg && cfg->big_n > 0) ? cfg->big_n : 2048;
    s->big_lanes = cfg ? cfg->big_lanes : 3;
    const int share = (cfg && cfg->lane_ctas > 0) ? cfg->lane_ctas : std::max(1, gmax * 29 / 100);
    if (s->big_lanes < 0 || s->big_lanes > kMaxBigLanes || share > gmax || s->big_lanes * share > gmax - 8) {
        destroy_records(s);
        cudaFree(s->pool_mem);
        for (auto& l : s->lanes)
            if (l) cudaStreamDestroy(l);
        delete s;
        return MDOT_ERR_INVALID_ARG;
    }
    mdot_status hs = MDOT_OK;
    for (int li = 0; li < s->big_lanes; ++li) {
        BigLane& L = s->big[li];
        if (e != cudaSuccess || hs != MDOT_OK) break;
        e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMalloc(&L.u, MDOT_BATCH_MAX_N * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&L.v, MDOT_BATCH_MAX_N * sizeof(double));
        if (e == cudaSuccess) hs = mdot_create(&L.h, MDOT_BATCH_MAX_N, L.stream);
        if (e == cudaSuccess && hs == MDOT_OK) hs = handle_set_grid(L.h, share);
    }
    if (e == cudaSuccess && hs != MDOT_OK) e = cudaErrorInvalidConfiguration;
    // a few SMs of slack: a batched CTA that has reported its problem may not have left its SM yet
    s->batch_cap = std::max(1, sms - s->big_lanes * share - 8);
    if (e != cudaSuccess) {
        set_last_error(cudaGetErrorString(e));
        for (BigLane& L : s->big) {
            if (L.h) mdot_destroy(L.h);
            cudaFree(L.u);
            cudaFree(L.v);
            if (L.stream) cudaStreamDestroy(L.stream);
        }
        destroy_records(s);
        cudaFree(s->pool_mem);
        for (auto& l : s->lanes)
            if (l) cudaStreamDestroy(l);
        delete s;
        return e == cudaErrorMemoryAllocation ? MDOT_ERR_OOM : MDOT_ERR_CUDA;
    }
    s->pool.init(pool_doubles);
    s->worker = std::thread(worker_loop, s);
    for (int i = 0; i < s->big_lanes; ++i) s->big[i].thread = std::thread(big_loop, s, i);
    *out = s;
    return MDOT_OK;
}

mdot_status mdot_server_submit(mdot_server* s, const mdot_problem* prob, uint64_t* ticket)
{
    if (!s || !prob || !ticket || !problem_ok(*prob)) return MDOT_ERR_INVALID_ARG;
    Request q;
    q.p = *prob;
    q.kind = cost_kind_of(*prob);
    q.stride = (int)(((prob->n + kStrideAlign - 1) / kStrideAlign) * kStrideAlign);
    q.len = batch_slot_doubles(q.stride);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal != cudaSuccess) return MDOT_ERR_CUDA;
    const bool big = s->big_lanes > 0 && prob->n > s->big_n;
    if (!big && q.len > s->pool.total) return MDOT_ERR_INVALID_ARG;     // could never be admitted
    q.ticket = s->next_ticket++;
    s->state[q.ticket] = 0;
    (big ? s->big_pending : s->pending).push_back(q);
    *ticket = q.ticket;
    s->cv_work.notify_all();
    return MDOT_OK;
}

mdot_status mdot_server_poll(mdot_server* s, uint64_t ticket, mdot_result* out)
{
    if (!s || !out) return MDOT_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->state.find(ticket);
    if (it == s->state.end()) return MDOT_ERR_INVALID_ARG;
    if (it->second != 2) return MDOT_NOT_READY;
    *out = s->finished[ticket];
    s->finished.erase(ticket);
    s->state.erase(it);
    return MDOT_OK;
}

mdot_status mdot_server_wait(mdot_server* s, uint64_t ticket, double timeout_s, mdot_result* out)
{
    if (!s || !out || !(timeout_s >= 0.0)) return MDOT_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto done = [&] {
        auto it = s->state.find(ticket);
        return it == s->state.end() || it->second == 2;
    };
    s->cv_done.wait_for(lk, std::chrono::duration<double>(std::min(timeout_s, 1e6)), done);
    auto it = s->state.find(ticket);
    if (it == s->state.end()) return MDOT_ERR_INVALID_ARG;
    if (it->second != 2) return MDOT_NOT_READY;
    *out = s->finished[ticket];
    s->finished.erase(ticket);
    s->state.erase(it);
    return MDOT_OK;
}

mdot_status mdot_server_destroy(mdot_server* s)
{
    if (!s) return MDOT_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();      // every admitted and queued request finishes
    for (auto& l : s->lanes) {
        cudaStreamSynchronize(l);
        cudaStreamDestroy(l);
    }
    for (BigLane& L : s->big) {
        if (L.thread.joinable()) L.thread.join();
        if (L.h) mdot_destroy(L.h);
        cudaFree(L.u);
        cudaFree(L.v);
        if (L.stream) cudaStreamDestroy(L.stream);
    }
    destroy_records(s);
    cudaFree(s->pool_mem);
    delete s;
    return MDOT_OK;
}

}  // extern "C"
