// mlc_batch_solve: many independent problems in one pass.  Problems are
// grouped by patch geometry and tier (n, s, Q, P, b, g_alpha, g_beta, M,
// tier); the per-patch steps (moments, local convolutions, residuals,
// Dirichlet solves) of all problems of a group run in shared launches over an
// item table of (problem, patch) pairs, the groups on concurrent streams; the
// per-problem coarse steps (F^H assembly, coarse solve, boundary values) run
// on parallel branches, the moments beside the local convolutions and the
// residuals beside the coarse steps.  The sequence is captured once as a CUDA
// graph per (plans, f, phi) set and replayed; the number of parallel branches
// and the slab launch shape are picked by timing the candidates on the first
// call (autotuning).  The same launch sequence runs uncaptured for the
// continuous-batching server (batch_enqueue).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "mlc_internal.h"

using namespace mlc;

namespace mlc {

bool same_patch_geometry(const Geom &a, const Geom &b) {
    return a.n == b.n && a.s == b.s && a.Q == b.Q && a.P == b.P && a.b == b.b && a.ga == b.ga &&
           a.gb == b.gb && a.tier == b.tier && a.M == b.M;
}

void batch_layout(int count, const mlc_plan_t *plans, const void *const *f, void *const *phi,
                  BatchLayout &L) {
    L.order.clear();
    L.plan_group.clear();
    L.groups.clear();
    L.items.clear();
    L.recs.clear();
    // groups in order of first appearance; problems keep their order inside a group
    std::vector<int> gof(count, -1);
    std::vector<int> reps;
    for (int k = 0; k < count; ++k) {
        for (size_t g = 0; g < reps.size(); ++g)
            if (same_patch_geometry(plans[reps[g]]->g, plans[k]->g)) {
                gof[k] = (int)g;
                break;
            }
        if (gof[k] < 0) {
            gof[k] = (int)reps.size();
            reps.push_back(k);
        }
    }
    for (size_t g = 0; g < reps.size(); ++g) {
        BatchLayout::Group G;
        G.rep = plans[reps[g]];
        G.item0 = (int)L.items.size();
        for (int k = 0; k < count; ++k) {
            if (gof[k] != (int)g) continue;
            const int slot = (int)L.recs.size();
            PlanPtrs r = plans[k]->hptrs;
            r.f = f[k];
            r.phi = (double *)phi[k];
            L.recs.push_back(r);
            L.order.push_back(k);
            L.plan_group.push_back((int)g);
            for (int p = 0; p < plans[k]->g.NP; ++p) L.items.push_back(make_int2(slot, p));
        }
        G.nitems = (int)L.items.size() - G.item0;
        L.groups.push_back(G);
    }
}

cudaError_t BatchStreams::ensure(int ngroups, int nbranches) {
    auto mk_s = [](std::vector<cudaStream_t> &v, size_t n) -> cudaError_t {
        while (v.size() < n) {
            cudaStream_t s;
            cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            if (e != cudaSuccess) return e;
            v.push_back(s);
        }
        return cudaSuccess;
    };
    auto mk_e = [](std::vector<cudaEvent_t> &v, size_t n) -> cudaError_t {
        while (v.size() < n) {
            cudaEvent_t e;
            cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
            if (r != cudaSuccess) return r;
            v.push_back(e);
        }
        return cudaSuccess;
    };
    cudaError_t e = mk_s(conv, ngroups);
    if (e == cudaSuccess) e = mk_s(aux, ngroups);
    if (e == cudaSuccess) e = mk_s(side, nbranches);
    if (e == cudaSuccess) e = mk_e(ev, 1 + 4 * (size_t)ngroups + nbranches);
    return e;
}

void BatchStreams::release() {
    for (auto v : {&conv, &aux, &side})
        for (auto s : *v) cudaStreamDestroy(s);
    for (auto e : ev) cudaEventDestroy(e);
    conv.clear();
    aux.clear();
    side.clear();
    ev.clear();
}

cudaError_t batch_enqueue(const std::vector<mlc_plan_t> &plans, const BatchLayout &L, const int2 *d_items,
                          const PlanPtrs *d_recs, BatchStreams &S, int branches, int persist,
                          cudaStream_t st, int chunk) {
    const int G = (int)L.groups.size();
    cudaError_t err = S.ensure(G, branches);
    if (err != cudaSuccess) return err;
    cudaEvent_t ev_start = S.ev[0];
    auto ev_mom = [&](int g) { return S.ev[1 + 4 * g]; };
    auto ev_conv = [&](int g) { return S.ev[2 + 4 * g]; };
    auto ev_res = [&](int g) { return S.ev[3 + 4 * g]; };
    auto ev_dir = [&](int g) { return S.ev[4 + 4 * g]; };
    auto ev_br = [&](int b) { return S.ev[1 + 4 * G + b]; };
#define TRYE(x)                              \
    do {                                     \
        err = (x);                           \
        if (err != cudaSuccess) return err;  \
    } while (0)
    TRYE(cudaEventRecord(ev_start, st));
    // per group: moments beside the local convolutions, then the residuals
    for (int g = 0; g < G; ++g) {
        const BatchLayout::Group &gr = L.groups[g];
        Items it{d_items + gr.item0, d_recs, gr.nitems};
        it.persist = persist;
        it.chunk = chunk;
        it.a1 = gr.a1;
        it.a4 = gr.a4;
        TRYE(cudaStreamWaitEvent(S.aux[g], ev_start, 0));
        TRYE(cudaStreamWaitEvent(S.conv[g], ev_start, 0));
        TRYE(launch_moments(gr.rep, it, S.aux[g]));
        TRYE(cudaEventRecord(ev_mom(g), S.aux[g]));
        TRYE(launch_patch_conv(gr.rep, it, S.conv[g]));
        TRYE(cudaEventRecord(ev_conv(g), S.conv[g]));
        TRYE(cudaStreamWaitEvent(S.aux[g], ev_conv(g), 0));
        TRYE(launch_resid(gr.rep, it, S.aux[g]));
        TRYE(cudaEventRecord(ev_res(g), S.aux[g]));
    }
    // per branch: the coarse charges and coarse solves of its problems, then
    // (after the residuals of their groups) their boundary values
    const int P = (int)plans.size();
    for (int j = 0; j < P; ++j) {
        cudaStream_t s = S.side[j % branches];
        const int g = L.plan_group[j];
        TRYE(cudaStreamWaitEvent(s, ev_conv(g), 0));
        TRYE(cudaStreamWaitEvent(s, ev_mom(g), 0));
        TRYE(launch_assemble(plans[L.order[j]], s));
        TRYE(launch_coarse(plans[L.order[j]], s));
    }
    for (int j = 0; j < P; ++j) {
        cudaStream_t s = S.side[j % branches];
        TRYE(cudaStreamWaitEvent(s, ev_res(L.plan_group[j]), 0));
        TRYE(launch_boundary(plans[L.order[j]], s));
    }
    const int nb = std::min(branches, P);
    for (int b = 0; b < nb; ++b) TRYE(cudaEventRecord(ev_br(b), S.side[b]));
    // Dirichlet solves of each group after every boundary step; join into st
    for (int g = 0; g < G; ++g) {
        const BatchLayout::Group &gr = L.groups[g];
        Items it{d_items + gr.item0, d_recs, gr.nitems};
        for (int b = 0; b < nb; ++b) TRYE(cudaStreamWaitEvent(S.conv[g], ev_br(b), 0));
        TRYE(launch_dirichlet(gr.rep, it, S.conv[g]));
        TRYE(cudaEventRecord(ev_dir(g), S.conv[g]));
        TRYE(cudaStreamWaitEvent(st, ev_dir(g), 0));
    }
#undef TRYE
    return cudaSuccess;
}

}  // namespace mlc

namespace {

struct BatchCtx {
    std::vector<mlc_plan_t> plans;  // in call order
    BatchLayout L;
    int2 *d_items = nullptr;
    PlanPtrs *d_plans = nullptr;
    std::vector<void *> scratch;  // per group: local-convolution scratch of one launch group
    cudaGraphExec_t exec = nullptr;
    int branches = 0;
    int persist = 0;
    int chunk = 0;                // patches per local-convolution launch group (tuned)
    float tuned_ms = 0.f;
    // the arrays the device records point at; a call with other arrays for
    // the same plans rewrites the records (stream-ordered) and replays the
    // same graph: no new capture and no new tuning
    std::vector<uintptr_t> bufs;
    PlanPtrs *h_recs = nullptr;   // pinned staging of the records
    cudaEvent_t done = nullptr;   // after the last replay
    cudaEvent_t copied = nullptr; // after the last record upload
};

void free_ctx(BatchCtx *c) {
    if (c->exec) cudaGraphExecDestroy(c->exec);
    cudaFree(c->d_items);
    cudaFree(c->d_plans);
    for (void *p : c->scratch) cudaFree(p);
    if (c->h_recs) cudaFreeHost(c->h_recs);
    if (c->done) cudaEventDestroy(c->done);
    if (c->copied) cudaEventDestroy(c->copied);
    delete c;
}

std::mutex g_mu;
std::map<std::vector<uintptr_t>, BatchCtx *> g_cache;
constexpr int kBatchMaxChunk = 2048;  // largest local-convolution launch group the tuner tries

cudaError_t capture(BatchCtx &c, int branches, int persist, int chunk, cudaGraphExec_t *out) {
    cudaStream_t cap;
    cudaError_t err = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (err != cudaSuccess) return err;
    BatchStreams S;
    err = S.ensure((int)c.L.groups.size(), branches);
    if (err == cudaSuccess) err = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    const bool began = err == cudaSuccess;
    g_capturing = true;
    if (err == cudaSuccess) err = batch_enqueue(c.plans, c.L, c.d_items, c.d_plans, S, branches, persist, cap, chunk);
    g_capturing = false;
    cudaGraph_t graph = nullptr;
    if (began) {
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (err == cudaSuccess) err = e2;
    }
    if (err == cudaSuccess) err = cudaGraphInstantiate(out, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    S.release();
    cudaStreamDestroy(cap);
    return err;
}

// Time a few replays of each candidate (parallel branches for the coarse
// steps x persistent or one-CTA-per-slab slab launches x patches per
// local-convolution launch group, the batch of pencils one launch
// transforms) and keep the fastest.
cudaError_t build_and_tune(BatchCtx &c, cudaStream_t st) {
    const int nplans = (int)c.plans.size();
    int maxitems = 0;
    for (auto &gr : c.L.groups) maxitems = std::max(maxitems, gr.nitems);
    struct Cand { int b, ps, chunk; };
    std::vector<Cand> cand;
    for (int b : {1, 4, 16})
        if (b == 1 || b <= nplans)
            for (int ps : {0, 1})
                for (int ch : {512, 1024, kBatchMaxChunk})
                    if (ch == 1024 || ch / 2 < maxitems) cand.push_back({b, ps, ch});
    cudaEvent_t e0, e1;
    cudaError_t err = cudaEventCreate(&e0);
    if (err != cudaSuccess) return err;
    err = cudaEventCreate(&e1);
    if (err != cudaSuccess) return err;
    for (auto bp : cand) {
        const int b = bp.b;
        cudaGraphExec_t ex = nullptr;
        err = capture(c, b, bp.ps, bp.chunk, &ex);
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
            c.persist = bp.ps;
            c.chunk = bp.chunk;
            c.tuned_ms = best;
        } else {
            cudaGraphExecDestroy(ex);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return err;
}

}  // namespace

extern "C" mlc_status mlc_batch_solve(int count, const mlc_plan_t *plans, const void *const *f,
                                      void *const *phi, void *stream) {
    if (count < 0 || (count > 0 && (!plans || !f || !phi))) return MLC_ERR_INVALID_ARG;
    if (count == 0) return MLC_OK;
    for (int k = 0; k < count; ++k) {
        if (!plans[k] || !f[k] || !phi[k] || f[k] == phi[k]) return MLC_ERR_INVALID_ARG;
        if (plans[k]->device != plans[0]->device) return MLC_ERR_INVALID_ARG;
        for (int j = 0; j < k; ++j)
            if (plans[j] == plans[k]) return MLC_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<uintptr_t> key, bufs;
    for (int k = 0; k < count; ++k) {
        key.push_back((uintptr_t)plans[k]);
        bufs.push_back((uintptr_t)f[k]);
        bufs.push_back((uintptr_t)phi[k]);
    }
    std::lock_guard<std::mutex> lk(g_mu);
    BatchCtx *c = nullptr;
    auto found = g_cache.find(key);
    if (found != g_cache.end()) {
        c = found->second;
        if (c->bufs != bufs) {  // same plans, other arrays: new records, same graph
            BatchLayout L;
            batch_layout(count, plans, f, phi, L);
            cudaError_t e = cudaStreamWaitEvent(st, c->done, 0);  // replays still reading them
            if (e == cudaSuccess) e = cudaEventSynchronize(c->copied);  // the staging buffer is free
            if (e == cudaSuccess) {
                std::memcpy(c->h_recs, L.recs.data(), L.recs.size() * sizeof(PlanPtrs));
                e = cudaMemcpyAsync(c->d_plans, c->h_recs, L.recs.size() * sizeof(PlanPtrs),
                                    cudaMemcpyHostToDevice, st);
            }
            if (e == cudaSuccess) e = cudaEventRecord(c->copied, st);
            if (e != cudaSuccess) return MLC_ERR_CUDA;
            c->bufs = bufs;
        }
    } else {
        c = new BatchCtx();
        c->plans.assign(plans, plans + count);
        batch_layout(count, plans, f, phi, c->L);
        const auto &items = c->L.items;
        const auto &recs = c->L.recs;
        cudaError_t e = cudaMalloc((void **)&c->d_items, items.size() * sizeof(int2));
        if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_plans, recs.size() * sizeof(PlanPtrs));
        for (auto &gr : c->L.groups) {
            if (e != cudaSuccess) break;
            const Geom &G = gr.rep->g;
            const long nit = std::min<long>(kBatchMaxChunk, gr.nitems);  // room for every candidate group size
            void *p = nullptr;
            e = cudaMalloc(&p, conv_scratch_bytes(G, nit));
            if (e != cudaSuccess) break;
            c->scratch.push_back(p);
            gr.a1 = p;
            gr.a4 = (char *)p + conv_scratch_a4_offset(G, nit);
        }
        if (e == cudaSuccess)
            e = cudaMemcpy(c->d_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(c->d_plans, recs.data(), recs.size() * sizeof(PlanPtrs), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_recs, recs.size() * sizeof(PlanPtrs));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->copied, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(c->copied, st);
        if (e == cudaSuccess) e = build_and_tune(*c, st);
        if (e != cudaSuccess) {
            free_ctx(c);
            return e == cudaErrorMemoryAllocation ? MLC_ERR_OOM : MLC_ERR_CUDA;
        }
        c->bufs = bufs;
        g_cache[key] = c;
    }
    cudaError_t e = cudaGraphLaunch(c->exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(c->done, st);
    return e == cudaSuccess ? MLC_OK : MLC_ERR_CUDA;
}

// Release the cached batch graphs that reference `plan` (called on destroy).
void mlc_batch_forget(mlc_plan_t plan) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_cache.begin(); it != g_cache.end();) {
        bool uses = false;
        for (auto *p : it->second->plans) uses |= (p == plan);
        if (uses) {
            free_ctx(it->second);
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
    (void)f;
    (void)phi;  // a batch is tuned once per set of plans, whatever arrays it solves
    std::vector<uintptr_t> key;
    for (int k = 0; k < count; ++k) key.push_back((uintptr_t)plans[k]);
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    return it == g_cache.end() ? 0 : it->second->branches * 2 + it->second->persist;
}

// Patches per local-convolution launch group the autotuner chose for this
// batch (0 if the batch is unknown).
extern "C" int mlc_debug_batch_chunk(int count, const mlc_plan_t *plans, const void *const *f,
                                     void *const *phi) {
    (void)f;
    (void)phi;  // a batch is tuned once per set of plans, whatever arrays it solves
    std::vector<uintptr_t> key;
    for (int k = 0; k < count; ++k) key.push_back((uintptr_t)plans[k]);
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    return it == g_cache.end() ? 0 : it->second->chunk;
}
