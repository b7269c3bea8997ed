// mlc_batch_solve: many independent problems with the same patch geometry in
// one pass.  The per-patch steps (moments, local convolutions, residuals,
// Dirichlet solves) of all problems run in shared launches over an item table
// of (problem, patch) pairs; the per-problem coarse steps (F^H assembly,
// coarse solve, boundary values) run on parallel branches, the moments beside
// the local convolutions and the residuals beside the coarse steps.  The sequence is
// captured once as a CUDA graph per (plans, f, phi) set and replayed; the
// number of parallel branches is picked by timing the candidates on the
// first call (autotuning).
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "mlc_internal.h"

using namespace mlc;

namespace {

struct BatchCtx {
    std::vector<mlc_plan_t> plans;
    int2 *d_items = nullptr;
    PlanPtrs *d_plans = nullptr;
    int nitems = 0;
    cudaGraphExec_t exec = nullptr;
    int branches = 0;
    int persist = 0;
    float tuned_ms = 0.f;
};

std::mutex g_mu;
std::map<std::vector<uintptr_t>, BatchCtx *> g_cache;

#define TRYE(x)                            \
    do {                                   \
        cudaError_t _e = (x);              \
        if (_e != cudaSuccess) return _e;  \
    } while (0)

cudaError_t capture(BatchCtx &c, int branches, int persist, cudaGraphExec_t *out) {
    cudaStream_t cap;
    TRYE(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    std::vector<cudaStream_t> side(branches + 1);  // coarse branches, then the moments / residual stream
    std::vector<cudaEvent_t> ev(branches + 4);
    for (auto &s : side) cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (auto &e : ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    cudaStream_t aux = side[branches];
    cudaEvent_t ev_start = ev[branches], ev_mom = ev[branches + 1], ev_conv = ev[branches + 2],
                ev_res = ev[branches + 3];
    const mlc_plan_s *rep = c.plans[0];
    Items it{c.d_items, c.d_plans, c.nitems};
    it.persist = persist;
    cudaError_t err = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    g_capturing = true;
    // moments beside the local convolutions; residuals beside the coarse steps
    if (err == cudaSuccess) err = cudaEventRecord(ev_start, cap);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(aux, ev_start, 0);
    if (err == cudaSuccess) err = launch_moments(rep, it, aux);
    if (err == cudaSuccess) err = cudaEventRecord(ev_mom, aux);
    if (err == cudaSuccess) err = launch_patch_conv(rep, it, cap);
    if (err == cudaSuccess) err = cudaEventRecord(ev_conv, cap);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(aux, ev_conv, 0);
    if (err == cudaSuccess) err = launch_resid(rep, it, aux);
    if (err == cudaSuccess) err = cudaEventRecord(ev_res, aux);
    for (int b = 0; b < branches && err == cudaSuccess; ++b) {
        err = cudaStreamWaitEvent(side[b], ev_conv, 0);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(side[b], ev_mom, 0);
    }
    // per branch: the coarse charges and coarse solves of its problems, then
    // (after the residuals) their boundary values
    for (size_t k = 0; k < c.plans.size() && err == cudaSuccess; ++k) {
        cudaStream_t s = side[k % branches];
        err = launch_assemble(c.plans[k], s);
        if (err == cudaSuccess) err = launch_coarse(c.plans[k], s);
    }
    for (int b = 0; b < branches && err == cudaSuccess; ++b) err = cudaStreamWaitEvent(side[b], ev_res, 0);
    for (size_t k = 0; k < c.plans.size() && err == cudaSuccess; ++k)
        err = launch_boundary(c.plans[k], side[k % branches]);
    for (int b = 0; b < branches && err == cudaSuccess; ++b) {
        err = cudaEventRecord(ev[b], side[b]);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(cap, ev[b], 0);
    }
    if (err == cudaSuccess) err = launch_dirichlet(rep, it, cap);
    g_capturing = false;
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (err == cudaSuccess) err = e2;
    if (err == cudaSuccess) err = cudaGraphInstantiate(out, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    for (auto &s : side) cudaStreamDestroy(s);
    for (auto &e : ev) cudaEventDestroy(e);
    cudaStreamDestroy(cap);
    return err;
}

// Time a few replays of each candidate (parallel branches for the coarse
// steps x persistent or one-CTA-per-slab local convolutions) and keep the
// fastest.
cudaError_t build_and_tune(BatchCtx &c, cudaStream_t st) {
    const int nplans = (int)c.plans.size();
    std::vector<std::pair<int, int>> cand;
    for (int b : {1, 4, 16})
        if (b == 1 || b <= nplans)
            for (int ps : {0, 1}) cand.push_back({b, ps});
    cudaEvent_t e0, e1;
    TRYE(cudaEventCreate(&e0));
    TRYE(cudaEventCreate(&e1));
    cudaError_t err = cudaSuccess;
    for (auto bp : cand) {
        const int b = bp.first;
        cudaGraphExec_t ex = nullptr;
        err = capture(c, b, bp.second, &ex);
        if (err != cudaSuccess) break;
        float best = 1e30f;
        for (int r = 0; r < 4 && err == cudaSuccess; ++r) {
            cudaEventRecord(e0, st);
            err = cudaGraphLaunch(ex, st);
            cudaEventRecord(e1, st);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0 && ms < best) best = ms;  // first replay is a warm-up
        }
        if (err != cudaSuccess) {
            cudaGraphExecDestroy(ex);
            break;
        }
        if (!c.exec || best < c.tuned_ms) {
            if (c.exec) cudaGraphExecDestroy(c.exec);
            c.exec = ex;
            c.branches = b;
            c.persist = bp.second;
            c.tuned_ms = best;
        } else {
            cudaGraphExecDestroy(ex);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return err;
}

bool same_patch_geometry(const Geom &a, const Geom &b) {
    return a.n == b.n && a.s == b.s && a.Q == b.Q && a.P == b.P && a.b == b.b && a.ga == b.ga &&
           a.gb == b.gb && a.tier == b.tier && a.M == b.M;
}

}  // namespace

extern "C" mlc_status mlc_batch_solve(int count, const mlc_plan_t *plans, const void *const *f,
                                      void *const *phi, void *stream) {
    if (count < 0 || (count > 0 && (!plans || !f || !phi))) return MLC_ERR_INVALID_ARG;
    if (count == 0) return MLC_OK;
    for (int k = 0; k < count; ++k) {
        if (!plans[k] || !f[k] || !phi[k] || f[k] == phi[k]) return MLC_ERR_INVALID_ARG;
        if (!same_patch_geometry(plans[k]->g, plans[0]->g)) return MLC_ERR_INVALID_ARG;
        for (int j = 0; j < k; ++j)
            if (plans[j] == plans[k]) return MLC_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<uintptr_t> key;
    for (int k = 0; k < count; ++k) {
        key.push_back((uintptr_t)plans[k]);
        key.push_back((uintptr_t)f[k]);
        key.push_back((uintptr_t)phi[k]);
    }
    std::lock_guard<std::mutex> lk(g_mu);
    BatchCtx *c = nullptr;
    auto found = g_cache.find(key);
    if (found != g_cache.end()) {
        c = found->second;
    } else {
        c = new BatchCtx();
        c->plans.assign(plans, plans + count);
        std::vector<int2> items;
        std::vector<PlanPtrs> recs;
        for (int k = 0; k < count; ++k) {
            PlanPtrs r = plans[k]->hptrs;
            r.f = f[k];
            r.phi = (double *)phi[k];
            recs.push_back(r);
            for (int p = 0; p < plans[k]->g.NP; ++p) items.push_back(make_int2(k, p));
        }
        c->nitems = (int)items.size();
        cudaError_t e = cudaMalloc((void **)&c->d_items, items.size() * sizeof(int2));
        if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_plans, recs.size() * sizeof(PlanPtrs));
        if (e == cudaSuccess)
            e = cudaMemcpy(c->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->d_plans, recs.data(), recs.size() * sizeof(PlanPtrs), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = build_and_tune(*c, st);
        if (e != cudaSuccess) {
            if (c->exec) cudaGraphExecDestroy(c->exec);
            cudaFree(c->d_items);
            cudaFree(c->d_plans);
            delete c;
            return e == cudaErrorMemoryAllocation ? MLC_ERR_OOM : MLC_ERR_CUDA;
        }
        g_cache[key] = c;
    }
    cudaError_t e = cudaGraphLaunch(c->exec, st);
    return e == cudaSuccess ? MLC_OK : MLC_ERR_CUDA;
}

// Release the cached batch graphs that reference `plan` (called on destroy).
void mlc_batch_forget(mlc_plan_t plan) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_cache.begin(); it != g_cache.end();) {
        bool uses = false;
        for (auto *p : it->second->plans) uses |= (p == plan);
        if (uses) {
            BatchCtx *c = it->second;
            if (c->exec) cudaGraphExecDestroy(c->exec);
            cudaFree(c->d_items);
            cudaFree(c->d_plans);
            delete c;
            it = g_cache.erase(it);
        } else {
            ++it;
        }
    }
}

// Configuration the autotuner chose for the batch of `plans` solved with these
// arrays: parallel branches * 2 + persistent flag (0 if the batch is unknown).
extern "C" int mlc_debug_batch_choice(int count, const mlc_plan_t *plans, const void *const *f,
                                      void *const *phi) {
    std::vector<uintptr_t> key;
    for (int k = 0; k < count; ++k) {
        key.push_back((uintptr_t)plans[k]);
        key.push_back((uintptr_t)f[k]);
        key.push_back((uintptr_t)phi[k]);
    }
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    return it == g_cache.end() ? 0 : it->second->branches * 2 + it->second->persist;
}
