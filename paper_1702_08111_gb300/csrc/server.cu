// Continuous-batching solve server (host C++).
//
// Requests (problem parameters + caller-owned device charge/result arrays)
// are queued by mlc_server_enqueue.  A worker thread forms batches from the
// queue: every request whose plan is free joins the next batch (up to
// max_batch requests), and the batch runs as one batched launch sequence
// (batch.cu): the per-patch steps of all its requests share launches, grouped
// by patch geometry and tier, and the per-request coarse steps run on
// parallel branches.  Up to kLanes batches are in flight at once, each on its
// own lane (stream, launch streams, item tables and local-convolution
// scratch), so requests that arrive while batches run are admitted into the
// next one as soon as a lane is free -- continuous batching, not a queue of
// whole solves.
// Plans (DGF tables, kernel spectra, basis tables, per-patch arrays) stay
// resident in a cache keyed by the problem parameters and are reused; the
// local-convolution scratch belongs to the lanes, not to the plans.  Idle
// plans are evicted only when the memory budget needs the room.
//
// Batches are formed by estimated cost (points x a per-tier weight from the
// measured tier rates): the requests of a batch complete together, so a
// request whose estimate is above kHeavyMs runs as a batch of its own, light
// requests are batched up to kBatchMs of estimated work, and the last lane
// takes light batches only, so light requests never wait behind two heavy
// solves.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "mlc_internal.h"

using namespace mlc;

namespace {

using Clock = std::chrono::steady_clock;
constexpr int kLanes = 3;           // lanes 0 .. kLanes-2 take any batch, the last light batches only
constexpr double kHeavyMs = 20.0;   // estimated solve time above which a request runs alone
constexpr double kBatchMs = 10.0;   // estimated work of a light batch

// Estimated solve time (ms): N^3 points at the measured rate of each tier at
// 256^3 on one GB300 (split 2700, split-DF 3600, double-float 1100, FP64 270
// Mpoints/s).
double estimate_ms(const mlc_params &p) {
    const double pts = (double)p.N * p.N * p.N;
    const int t = p.tier < 0 ? MLC_TIER_FP64 : p.tier;
    const double rate = t == MLC_TIER_SPLIT ? 2700.0 : (t == MLC_TIER_SPLIT_DF ? 3600.0 : (t == MLC_TIER_DF ? 1100.0 : 270.0));
    return pts / (rate * 1e3);
}

struct Key {
    int v[15];
    bool operator<(const Key &o) const { return std::memcmp(v, o.v, sizeof(v)) < 0; }
};

Key key_of(const mlc_params &p) {
    Key k;
    const int v[15] = {p.N, p.n, p.s, p.C, p.P, p.Q, p.g_beta, p.b, p.tier, p.mode, p.dgf_nD, p.dgf_zeta,
                       p.conv_chunk, p.levels, p.coarse_s};
    std::memcpy(k.v, v, sizeof(v));
    return k;
}

struct Pending {
    uint64_t ticket;
    mlc_request req;
    Clock::time_point t_enq;
    size_t est;      // device bytes of its plan (bound)
    double est_ms;   // estimated solve time
};

// Upper bound of the device bytes a plan with these parameters holds (its
// per-patch arrays and tables; the shared DGF table and the lanes' scratch
// are not counted).
size_t estimate_bytes(const mlc_params &p) {
    const long N = p.N, n = p.n, s = p.s;
    if (n <= 0 || N <= 0 || N % n) return 0;
    const long rb = conv_real_bytes(p.tier < 0 ? MLC_TIER_FP64 : p.tier);
    long M = 1;
    while (M < 2 * (n + s)) M <<= 1;
    const long Mh = M / 2 + 1, W = n + 2 * s + 1, np = N / n, NP = np * np * np;
    const long nc = (n + 2 * s) / 4 + 1;
    long bytes = NP * (nc * nc * nc + 6 * W * W) * rb;        // coarse lattice, face planes
    bytes += NP * (6 * W * W + 64) * 8;                       // residuals, moments
    const long nf = N / 4 + 2 * (s / 4 + 4);                  // coarse extents (bound)
    long Mc = 1;
    while (Mc < 2 * nf) Mc <<= 1;
    bytes += 3L * nf * Mc * (Mc / 2 + 1) * 16 + 2L * nf * nf * nf * 8;
    bytes += 3L * (np + 1) * (N + 1) * (N + 1) * 8;           // boundary planes
    bytes += (Mh * Mh * Mh + (Mc / 2 + 1) * (Mc / 2 + 1) * (Mc / 2 + 1)) * 12;
    if (rb == 4) {  // split tiers: ring terms of one face-plane axis for the ring GEMM
        const long gb = p.g_beta >= 0 ? p.g_beta : (p.Q == 4 ? n : (9 * n + 7) / 8);
        const long wbx = n + 2 * gb + 1, npb = (n + 2 * gb) / n + 2;
        bytes += NP * ((npb * wbx * wbx + 127) / 128 * 128) * 4;
    }
    if (n > 24) bytes += NP * (n - 1) * (n - 1) * (n - 1) * 8;  // Dirichlet workspace
    if (p.Q == 10 && n > 16) bytes += NP * 2 * (n - 1) * (n - 1) * (n - 1) * 8;  // two-layer Dirichlet arrays
    if (p.Q == 10 && n > 16 && n <= 24) bytes += NP * (n - 1) * (n - 1) * (n - 1) * 8;
    if (p.Q == 10)  // the second boundary layer: off-face local fields and residuals, planes
        bytes += NP * 12 * W * W * (rb + 8) + 6L * (np + 1) * (N + 1) * (N + 1) * 8 +
                 6L * (np + 1) * (nf + 4) * (N + 1) * 8;
    if (p.levels > 2) {
        // the next coarser level: its own plan (with its local-convolution
        // scratch, allocated at creation) and its charge and result arrays
        const long gb = p.g_beta >= 0 ? p.g_beta : (p.Q == 4 ? n : (9 * n + 7) / 8);
        const long b = p.b >= 0 ? p.b : (p.Q == 4 ? 2 : (p.Q == 6 ? 3 : 4));
        const long span = N / 4 + 2 * (gb / 4 + b + 2);
        mlc_params c = p;
        c.N = (int)(n * ((span + n - 1) / n));
        c.levels = p.levels - 1;
        if (c.coarse_s > 0) c.s = c.coarse_s;
        const long Nc = c.N, npc = Nc / n, NPc = npc * npc * npc;
        const long chunk = std::min<long>(p.conv_chunk > 0 ? p.conv_chunk : 1024, NPc);
        bytes += (long)estimate_bytes(c) + Nc * Nc * Nc * 12 +
                 chunk * (Mh * (n + 1) * (n + 1) + W * Mh * W) * 2 * rb;
    }
    bytes += 32L << 20;                                        // basis tables, index maps, slack
    return (size_t)bytes;
}

// One lane: a batch in flight and the resources it runs with.
struct Lane {
    cudaStream_t st = nullptr;
    BatchStreams S;
    cudaEvent_t done = nullptr;
    int2 *d_items = nullptr, *h_items = nullptr;   // device / pinned host item tables
    PlanPtrs *d_recs = nullptr, *h_recs = nullptr;
    size_t cap_items = 0, cap_recs = 0;
    std::vector<void *> scratch;      // per group: local-convolution scratch
    std::vector<size_t> scratch_cap;
    size_t scratch_total = 0;
    // the batch in flight
    bool busy = false;
    std::vector<Pending> reqs;
    std::vector<mlc_plan_t> plans;
    std::vector<Key> keys;
    std::vector<size_t> bytes;
    Clock::time_point t_start;
    mlc_status launch_status = MLC_OK;
};

}  // namespace

struct mlc_server_s {
    size_t budget;
    int max_batch;
    int device;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Pending> queue;
    std::map<uint64_t, mlc_result> results;
    std::multimap<Key, std::pair<mlc_plan_t, size_t>> idle;  // resident idle plans
    std::map<Key, int> nplans;                                // resident plans per key
    size_t used = 0;  // bytes of plans (idle or in a batch) and lane scratch
    uint64_t next_ticket = 1;
    bool stop = false;
    Lane lanes[kLanes];
    std::thread worker;

    void run();
    bool form_and_launch(Lane &ln, bool heavy_ok, std::unique_lock<std::mutex> &lk);
    void retire(Lane &ln);
    cudaError_t launch(Lane &ln);
};

// Take requests from the queue (in arrival order, skipping those whose plans
// are all busy) into a batch for lane ln and launch it.  Plans come from the
// idle cache; a key with no resident plan, or with room in the budget for a
// second one, gets a new plan (idle plans of other keys are evicted first if
// the budget needs it).
bool mlc_server_s::form_and_launch(Lane &ln, bool heavy_ok, std::unique_lock<std::mutex> &lk) {
    ln.reqs.clear();
    ln.plans.clear();
    ln.keys.clear();
    ln.bytes.clear();
    std::vector<size_t> taken;
    double cost = 0.0;
    for (size_t i = 0; i < queue.size() && (int)ln.reqs.size() < max_batch; ++i) {
        Pending &pd = queue[i];
        const bool heavy = pd.est_ms > kHeavyMs;
        if (heavy && (!heavy_ok || !ln.reqs.empty())) continue;   // heavy: alone, on a heavy lane
        if (!ln.reqs.empty() && cost + pd.est_ms > kBatchMs) continue;
        const Key k = key_of(pd.req.params);
        mlc_plan_t plan = nullptr;
        size_t bytes = 0;
        auto it = idle.find(k);
        if (it != idle.end()) {
            plan = it->second.first;
            bytes = it->second.second;
            idle.erase(it);
        } else {
            const int have = nplans[k];
            if (have >= kLanes) continue;                       // all its plans are busy
            if (have > 0 && used + pd.est > budget) continue;   // a second plan only if it fits
            while (used + pd.est > budget && !idle.empty()) {   // make room
                auto ev = idle.begin();
                used -= ev->second.second;
                nplans[ev->first] -= 1;
                lk.unlock();
                mlc_plan_destroy(ev->second.first);
                lk.lock();
                idle.erase(ev);
            }
            if (used + pd.est > budget) continue;  // wait for running batches to finish
            used += pd.est;
            nplans[k] += 1;
            lk.unlock();
            mlc_status st = mlc_plan_create_ex(&pd.req.params, &plan);
            lk.lock();
            if (st != MLC_OK) {
                used -= pd.est;
                nplans[k] -= 1;
                results[pd.ticket] = mlc_result{st, 0.0, 0.0};
                taken.push_back(i);
                cv_done.notify_all();
                continue;
            }
            bytes = pd.est;
        }
        ln.reqs.push_back(pd);
        ln.plans.push_back(plan);
        ln.keys.push_back(k);
        ln.bytes.push_back(bytes);
        taken.push_back(i);
        cost += pd.est_ms;
        if (heavy) break;
    }
    for (size_t j = taken.size(); j-- > 0;) queue.erase(queue.begin() + (long)taken[j]);
    if (ln.reqs.empty()) return false;
    ln.busy = true;
    ln.t_start = Clock::now();
    const cudaError_t e = launch(ln);
    ln.launch_status = e == cudaSuccess ? MLC_OK : (e == cudaErrorMemoryAllocation ? MLC_ERR_OOM : MLC_ERR_CUDA);
    cudaEventRecord(ln.done, ln.st);
    return true;
}

// Enqueue the batch of lane ln on its stream: item tables from pinned host
// buffers, scratch per geometry group, the batched launch sequence.
cudaError_t mlc_server_s::launch(Lane &ln) {
    const int count = (int)ln.reqs.size();
    std::vector<const void *> f(count);
    std::vector<void *> phi(count);
    for (int k = 0; k < count; ++k) {
        f[k] = ln.reqs[k].req.f;
        phi[k] = ln.reqs[k].req.phi;
    }
    BatchLayout L;
    batch_layout(count, ln.plans.data(), f.data(), phi.data(), L);
    cudaError_t e = cudaSuccess;
    // item tables: the pinned host copies are rewritten only while the lane is idle
    if (L.items.size() > ln.cap_items) {
        if (ln.d_items) cudaFreeAsync(ln.d_items, ln.st);
        if (ln.h_items) cudaFreeHost(ln.h_items);
        ln.cap_items = std::max(L.items.size(), (size_t)1 << 20);
        e = cudaMallocAsync((void **)&ln.d_items, ln.cap_items * sizeof(int2), ln.st);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&ln.h_items, ln.cap_items * sizeof(int2), 0);
        if (e != cudaSuccess) { ln.cap_items = 0; ln.d_items = nullptr; ln.h_items = nullptr; return e; }
    }
    if (L.recs.size() > ln.cap_recs) {
        if (ln.d_recs) cudaFreeAsync(ln.d_recs, ln.st);
        if (ln.h_recs) cudaFreeHost(ln.h_recs);
        ln.cap_recs = std::max(L.recs.size(), (size_t)64);
        e = cudaMallocAsync((void **)&ln.d_recs, ln.cap_recs * sizeof(PlanPtrs), ln.st);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&ln.h_recs, ln.cap_recs * sizeof(PlanPtrs), 0);
        if (e != cudaSuccess) { ln.cap_recs = 0; ln.d_recs = nullptr; ln.h_recs = nullptr; return e; }
    }
    std::memcpy(ln.h_items, L.items.data(), L.items.size() * sizeof(int2));
    std::memcpy(ln.h_recs, L.recs.data(), L.recs.size() * sizeof(PlanPtrs));
    e = cudaMemcpyAsync(ln.d_items, ln.h_items, L.items.size() * sizeof(int2), cudaMemcpyHostToDevice, ln.st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ln.d_recs, ln.h_recs, L.recs.size() * sizeof(PlanPtrs), cudaMemcpyHostToDevice, ln.st);
    if (e != cudaSuccess) return e;
    // local-convolution scratch per group, grown in stream order
    if (ln.scratch.size() < L.groups.size()) {
        ln.scratch.resize(L.groups.size(), nullptr);
        ln.scratch_cap.resize(L.groups.size(), 0);
    }
    for (size_t g = 0; g < L.groups.size(); ++g) {
        const Geom &G = L.groups[g].rep->g;
        const long nit = std::min<long>(G.chunk, L.groups[g].nitems);
        const size_t need = conv_scratch_bytes(G, nit);
        if (need > ln.scratch_cap[g]) {
            if (ln.scratch[g]) cudaFreeAsync(ln.scratch[g], ln.st);
            ln.scratch_total -= ln.scratch_cap[g];
            used -= ln.scratch_cap[g];
            ln.scratch_cap[g] = 0;
            e = cudaMallocAsync(&ln.scratch[g], need, ln.st);
            if (e != cudaSuccess) { ln.scratch[g] = nullptr; return e; }
            ln.scratch_cap[g] = need;
            ln.scratch_total += need;
            used += need;
        }
        L.groups[g].a1 = ln.scratch[g];
        L.groups[g].a4 = (char *)ln.scratch[g] + conv_scratch_a4_offset(G, nit);
    }
    return batch_enqueue(ln.plans, L, ln.d_items, ln.d_recs, ln.S, std::min(4, count), 0, ln.st);
}

void mlc_server_s::retire(Lane &ln) {
    const cudaError_t q = cudaEventQuery(ln.done);
    const auto now = Clock::now();
    for (size_t k = 0; k < ln.reqs.size(); ++k) {
        mlc_result r{};
        r.status = ln.launch_status != MLC_OK ? ln.launch_status : (q == cudaSuccess ? MLC_OK : MLC_ERR_CUDA);
        r.latency_ms = std::chrono::duration<double, std::milli>(now - ln.reqs[k].t_enq).count();
        r.queue_ms = std::chrono::duration<double, std::milli>(ln.t_start - ln.reqs[k].t_enq).count();
        results[ln.reqs[k].ticket] = r;
        idle.insert({ln.keys[k], {ln.plans[k], ln.bytes[k]}});
    }
    ln.reqs.clear();
    ln.plans.clear();
    ln.busy = false;
}

void mlc_server_s::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        bool any_busy = false;
        for (Lane &ln : lanes) any_busy |= ln.busy;
        if (stop && queue.empty() && !any_busy) break;
        // retire finished batches
        bool retired = false;
        for (Lane &ln : lanes)
            if (ln.busy && cudaEventQuery(ln.done) != cudaErrorNotReady) {
                retire(ln);
                retired = true;
            }
        if (retired) cv_done.notify_all();
        // fill free lanes with the next batches
        for (int l = 0; l < kLanes; ++l)
            if (!lanes[l].busy && !queue.empty()) form_and_launch(lanes[l], l < kLanes - 1, lk);
        any_busy = false;
        for (Lane &ln : lanes) any_busy |= ln.busy;
        if (!any_busy && queue.empty()) {
            cv_work.wait(lk, [&] { return stop || !queue.empty(); });
        } else {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

extern "C" {

mlc_status mlc_server_create(size_t hbm_budget_bytes, int max_batch, mlc_server_t *out) {
    if (!out || max_batch < 1 || max_batch > 64 || hbm_budget_bytes == 0) return MLC_ERR_INVALID_ARG;
    mlc_server_s *s = new (std::nothrow) mlc_server_s();
    if (!s) return MLC_ERR_OOM;
    s->budget = hbm_budget_bytes;
    s->max_batch = max_batch;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return MLC_ERR_CUDA;
    }
    for (Lane &ln : s->lanes)
        if (cudaStreamCreateWithFlags(&ln.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ln.done, cudaEventDisableTiming) != cudaSuccess) {
            delete s;
            return MLC_ERR_CUDA;
        }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return MLC_OK;
}

mlc_status mlc_server_destroy(mlc_server_t s) {
    if (!s) return MLC_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaDeviceSynchronize();
    for (auto &kv : s->idle) mlc_plan_destroy(kv.second.first);
    for (Lane &ln : s->lanes) {
        for (void *p : ln.scratch) if (p) cudaFree(p);
        if (ln.d_items) cudaFree(ln.d_items);
        if (ln.d_recs) cudaFree(ln.d_recs);
        if (ln.h_items) cudaFreeHost(ln.h_items);
        if (ln.h_recs) cudaFreeHost(ln.h_recs);
        ln.S.release();
        if (ln.done) cudaEventDestroy(ln.done);
        if (ln.st) cudaStreamDestroy(ln.st);
    }
    delete s;
    return MLC_OK;
}

mlc_status mlc_server_enqueue(mlc_server_t s, const mlc_request *req, uint64_t *ticket) {
    if (!s || !req || !ticket || !req->f || !req->phi) return MLC_ERR_INVALID_ARG;
    const mlc_params &p = req->params;
    if (p.N <= 0 || p.n <= 0 || p.N % p.n || p.n % 4 || p.s % 4 || (p.Q != 4 && p.Q != 6 && p.Q != 10) || p.C != 4 ||
        (p.tier >= 0 && !tier_valid(p.tier)))
        return MLC_ERR_INVALID_ARG;
    const size_t est = estimate_bytes(p);
    if (est > s->budget) return MLC_ERR_ADMISSION;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return MLC_ERR_INVALID_ARG;
    Pending pd{s->next_ticket++, *req, Clock::now(), est, estimate_ms(p)};
    *ticket = pd.ticket;
    s->queue.push_back(pd);
    s->cv_work.notify_all();
    return MLC_OK;
}

mlc_status mlc_server_wait(mlc_server_t s, uint64_t ticket, int timeout_ms, mlc_result *res) {
    if (!s || !res) return MLC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] { return s->results.count(ticket) > 0; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, ready);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        return MLC_ERR_TIMEOUT;
    }
    *res = s->results[ticket];
    s->results.erase(ticket);
    return MLC_OK;
}

}  // extern "C"
