// Continuous-batching solve server (host C++).
//
// Requests (problem parameters + caller-owned device charge/result arrays)
// are queued by mlc_server_enqueue.  A worker thread admits queued requests
// whenever a slot and enough of the device-memory budget are free, runs each
// admitted request on its own stream from a pool so that the kernels of
// requests in flight overlap on the GPU, and retires requests as their
// completion events fire -- new requests are admitted while others are still
// running.  Plans (DGF tables, kernel spectra, basis tables, workspace) stay
// resident in a cache keyed by the problem parameters and are reused; idle
// plans are evicted only when the budget needs the room.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "mlc_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Key {
    int v[12];
    bool operator<(const Key &o) const { return std::memcmp(v, o.v, sizeof(v)) < 0; }
};

Key key_of(const mlc_params &p) {
    Key k;
    const int v[12] = {p.N, p.n, p.s, p.C, p.P, p.Q, p.g_beta, p.b, p.tier, p.mode, p.dgf_nD, p.dgf_zeta};
    std::memcpy(k.v, v, sizeof(v));
    return k;
}

struct Pending {
    uint64_t ticket;
    mlc_request req;
    Clock::time_point t_enq;
    size_t est;
};

struct Active {
    uint64_t ticket;
    mlc_plan_t plan;
    Key key;
    int slot;
    cudaEvent_t done;
    Clock::time_point t_enq, t_start;
    size_t bytes;
    mlc_status launch_status;
};

// Upper bound of the device bytes a plan with these parameters holds
// (workspace and per-plan tables; the shared DGF table is not counted).
size_t estimate_bytes(const mlc_params &p) {
    const long N = p.N, n = p.n, s = p.s;
    if (n <= 0 || N <= 0 || N % n) return 0;
    const long rb = mlc::conv_real_bytes(p.tier < 0 ? MLC_TIER_FP64 : p.tier);
    long M = 1;
    while (M < 2 * (n + s)) M <<= 1;
    const long Mh = M / 2 + 1, nb = n + 1, W = n + 2 * s + 1, np = N / n, NP = np * np * np;
    const long nc = (n + 2 * s) / 4 + 1;
    long bytes = NP * (nb * nb * Mh + W * W * Mh) * 2 * rb;   // spectra workspace
    bytes += NP * (nc * nc * nc + 6 * W * W) * rb;            // coarse lattice, face planes
    bytes += NP * (6 * W * W + 64) * 8;                       // residuals, moments
    const long nf = N / 4 + 2 * (s / 4 + 4);                  // coarse extents (bound)
    long Mc = 1;
    while (Mc < 2 * nf) Mc <<= 1;
    bytes += 3L * nf * Mc * (Mc / 2 + 1) * 16 + 2L * nf * nf * nf * 8;
    bytes += 3L * (np + 1) * (N + 1) * (N + 1) * 8;           // boundary planes
    bytes += (Mh * Mh * Mh + (Mc / 2 + 1) * (Mc / 2 + 1) * (Mc / 2 + 1)) * 12;
    bytes += 2 * N * N * N * 8;                               // host-path staging (if used)
    bytes += 32L << 20;                                        // basis tables, index maps, slack
    return (size_t)bytes;
}

}  // namespace

struct mlc_server_s {
    size_t budget;
    int max_batch;
    int device;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Pending> queue;
    std::vector<Active> active;
    std::map<uint64_t, mlc_result> results;
    std::multimap<Key, std::pair<mlc_plan_t, size_t>> idle;  // resident idle plans
    size_t used = 0;  // bytes of plans in use or idle
    uint64_t next_ticket = 1;
    bool stop = false;
    std::vector<cudaStream_t> streams;
    std::vector<bool> slot_busy;
    std::thread worker;

    void run();
    bool admit_locked(std::unique_lock<std::mutex> &lk);
};

bool mlc_server_s::admit_locked(std::unique_lock<std::mutex> &lk) {
    bool any = false;
    while (!queue.empty() && (int)active.size() < max_batch) {
        Pending &pd = queue.front();
        const Key k = key_of(pd.req.params);
        mlc_plan_t plan = nullptr;
        size_t bytes = 0;
        auto it = idle.find(k);
        if (it != idle.end()) {
            plan = it->second.first;
            bytes = it->second.second;
            idle.erase(it);
        } else {
            // make room: evict idle plans until the estimate fits
            while (used + pd.est > budget && !idle.empty()) {
                auto ev = idle.begin();
                used -= ev->second.second;
                mlc_plan_destroy(ev->second.first);
                idle.erase(ev);
            }
            if (used + pd.est > budget) break;  // wait for running requests to finish
            lk.unlock();
            mlc_status st = mlc_plan_create_ex(&pd.req.params, &plan);
            size_t ws = 0;
            if (st == MLC_OK) mlc_plan_workspace_bytes(plan, &ws);
            lk.lock();
            if (st != MLC_OK) {
                mlc_result r{st, 0.0, 0.0};
                results[pd.ticket] = r;
                queue.pop_front();
                cv_done.notify_all();
                continue;
            }
            bytes = std::max(pd.est, ws);
            used += bytes;
        }
        int slot = 0;
        while (slot_busy[slot]) ++slot;
        slot_busy[slot] = true;
        Active a{};
        a.ticket = pd.ticket;
        a.plan = plan;
        a.key = k;
        a.slot = slot;
        a.t_enq = pd.t_enq;
        a.t_start = Clock::now();
        a.bytes = bytes;
        cudaEventCreateWithFlags(&a.done, cudaEventDisableTiming);
        a.launch_status = mlc_solve(plan, pd.req.f, pd.req.phi, streams[slot]);
        cudaEventRecord(a.done, streams[slot]);
        active.push_back(a);
        queue.pop_front();
        any = true;
    }
    return any;
}

void mlc_server_s::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        if (stop && queue.empty() && active.empty()) break;
        admit_locked(lk);
        // retire finished requests
        bool retired = false;
        for (size_t i = 0; i < active.size();) {
            Active &a = active[i];
            cudaError_t q = cudaEventQuery(a.done);
            if (q == cudaErrorNotReady) {
                ++i;
                continue;
            }
            const auto now = Clock::now();
            mlc_result r{};
            r.status = a.launch_status != MLC_OK ? a.launch_status : (q == cudaSuccess ? MLC_OK : MLC_ERR_CUDA);
            r.latency_ms = std::chrono::duration<double, std::milli>(now - a.t_enq).count();
            r.queue_ms = std::chrono::duration<double, std::milli>(a.t_start - a.t_enq).count();
            results[a.ticket] = r;
            cudaEventDestroy(a.done);
            slot_busy[a.slot] = false;
            idle.insert({a.key, {a.plan, a.bytes}});
            active.erase(active.begin() + (long)i);
            retired = true;
        }
        if (retired) cv_done.notify_all();
        if (active.empty() && queue.empty()) {
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
    s->streams.resize(max_batch);
    s->slot_busy.assign(max_batch, false);
    for (auto &st : s->streams)
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
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
    for (auto &kv : s->idle) mlc_plan_destroy(kv.second.first);
    for (auto &st : s->streams) cudaStreamDestroy(st);
    delete s;
    return MLC_OK;
}

mlc_status mlc_server_enqueue(mlc_server_t s, const mlc_request *req, uint64_t *ticket) {
    if (!s || !req || !ticket || !req->f || !req->phi) return MLC_ERR_INVALID_ARG;
    const mlc_params &p = req->params;
    if (p.N <= 0 || p.n <= 0 || p.N % p.n || p.n % 4 || p.s % 4 || (p.Q != 4 && p.Q != 6) || p.C != 4)
        return MLC_ERR_INVALID_ARG;
    const size_t est = estimate_bytes(p);
    if (est > s->budget) return MLC_ERR_ADMISSION;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return MLC_ERR_INVALID_ARG;
    Pending pd{s->next_ticket++, *req, Clock::now(), est};
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
