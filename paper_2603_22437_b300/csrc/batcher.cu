// Batching runtime around the evaluator: CUDA-graph capture of a whole
// evaluation, and a batcher that queues uneven windows (different frame
// counts, different users), groups them by (frames, key set), cuts the groups
// into batches and replays one captured graph per (frames, keys, batch size)
// from graph-owned staging buffers.  Plans (one per frame count) and graphs
// are cached least-recently-used under device-memory budgets.
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <map>
#include <memory>
#include <new>
#include <tuple>
#include <utility>
#include <vector>

#include "circuits.h"
#include "handles.h"
#include "internal.h"

using namespace mmfhe;

namespace {

mmfhe_status bfail(Context *c, mmfhe_status code, const char *msg) {
    if (c) c->last_error = msg;
    return code;
}

#define B_TRY try {
#define B_CATCH(ctxp)                                                                          \
    }                                                                                          \
    catch (const Error &e) { return bfail(ctxp, e.code, e.what()); }                           \
    catch (const std::bad_alloc &) { return bfail(ctxp, MMFHE_ERR_OUT_OF_MEMORY, "host allocation failed"); } \
    catch (const std::exception &e) { return bfail(ctxp, MMFHE_ERR_CUDA, e.what()); }          \
    catch (...) { return bfail(ctxp, MMFHE_ERR_CUDA, "unknown error"); }                       \
    return MMFHE_OK;

// The context allocates from `mine` for the lifetime of this object.
struct PoolSwap {
    Context &c;
    std::unique_ptr<Pool> &mine;
    PoolSwap(Context &c_, std::unique_ptr<Pool> &m) : c(c_), mine(m) { std::swap(c.pool, mine); }
    ~PoolSwap() { std::swap(c.pool, mine); }
};

// Profiling and tracing off for the lifetime of this object.
struct QuietLaunches {
    Context &c;
    bool prof, trace;
    explicit QuietLaunches(Context &c_) : c(c_), prof(c_.profiling), trace(c_.tracing) {
        c.profiling = false;
        c.tracing = false;
    }
    ~QuietLaunches() {
        c.profiling = prof;
        c.tracing = trace;
    }
};

struct StreamOwner {
    cudaStream_t s = nullptr;
    StreamOwner() { CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)); }
    ~StreamOwner() { cudaStreamDestroy(s); }
};

}  // namespace

struct mmfhe_graph {
    Context *c = nullptr;
    std::unique_ptr<Pool> pool;   // every intermediate of the captured evaluation
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels = 0;
    ~mmfhe_graph() {
        if (exec) cudaGraphExecDestroy(exec);
    }
    uint64_t bytes() const { return pool ? pool->bytes_held() : 0; }
};

namespace {

std::unique_ptr<mmfhe_graph> capture_eval(Context &c, const Plan &p, const Keys *const *keys,
                                          const uint64_t *const *ins, size_t B, uint64_t *const *outs) {
    if (B == 0) throw Error(MMFHE_ERR_BAD_ARG, "graph of an empty batch");
    for (size_t w = 0; w < B; w++)
        if (!ins[w] || !outs[w] || is_host_ptr(ins[w]) || is_host_ptr(outs[w]))
            throw Error(MMFHE_ERR_BAD_ARG, "graph capture needs device buffers");
    std::unique_ptr<mmfhe_graph> g(new mmfhe_graph());
    g->c = &c;
    g->pool.reset(new Pool(c.device));
    StreamOwner cs;
    CK(cudaDeviceSynchronize());   // keys and plan uploads may be pending on other streams
    PoolSwap swap(c, g->pool);
    QuietLaunches quiet(c);
    // first run: fills the graph's pool with exactly the buffers the recorded run takes
    eval_windows(c, p, keys, ins, B, outs, cs.s);
    CK(cudaStreamSynchronize(cs.s));
    const uint64_t l0 = c.launches;
    CK(cudaStreamBeginCapture(cs.s, cudaStreamCaptureModeRelaxed));
    cudaGraph_t graph = nullptr;
    try {
        eval_windows(c, p, keys, ins, B, outs, cs.s);
    } catch (...) {
        cudaStreamEndCapture(cs.s, &graph);
        if (graph) cudaGraphDestroy(graph);
        c.launches = l0;
        throw;
    }
    CK(cudaStreamEndCapture(cs.s, &graph));
    g->kernels = c.launches - l0;
    c.launches = l0;   // recording launched nothing
    const cudaError_t e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    CK(e);
    return g;
}

void graph_launch(mmfhe_graph &g, cudaStream_t st) {
    CK(cudaGraphLaunch(g.exec, st));
    g.c->launches += g.kernels;
}

}  // namespace

// ---------------------------------------------------------------------------
// batcher
// ---------------------------------------------------------------------------
struct mmfhe_batcher {
    Context *c = nullptr;
    mmfhe_circuit_config base{};
    mmfhe_batcher_config cfg{};
    uint64_t clock = 0;

    struct PlanEntry {
        std::unique_ptr<mmfhe_plan> h;
        uint64_t bytes = 0, last_use = 0;
        size_t in_words = 0, out_words = 0;
    };
    std::map<uint32_t, PlanEntry> plans;   // by frame count

    struct GraphEntry {
        std::unique_ptr<mmfhe_graph> g;
        uint64_t *stage_in = nullptr, *stage_out = nullptr;
        size_t in_bytes = 0, out_bytes = 0;
        int device = 0;
        uint64_t bytes = 0, last_use = 0;
        ~GraphEntry() {
            g.reset();
            dev_free(device, stage_in, in_bytes);
            dev_free(device, stage_out, out_bytes);
        }
    };
    using GraphKey = std::tuple<uint32_t, const Keys *, uint32_t>;   // frames, keys, batch size
    std::map<GraphKey, std::unique_ptr<GraphEntry>> graphs;

    struct Req {
        const Keys *k;
        uint32_t frames;
        const uint64_t *in;
        uint64_t *out;
    };
    std::vector<Req> pending;
    mmfhe_batcher_stats st{};

    uint64_t plan_bytes() const {
        uint64_t s = 0;
        for (auto &kv : plans) s += kv.second.bytes;
        return s;
    }
    uint64_t graph_bytes() const {
        uint64_t s = 0;
        for (auto &kv : graphs) s += kv.second->bytes;
        return s;
    }

    void drop_graphs_if(const std::function<bool(const GraphKey &)> &pred) {
        bool any = false;
        for (auto &kv : graphs) any |= pred(kv.first);
        if (!any) return;
        CK(cudaDeviceSynchronize());   // replays in flight finish before their buffers go
        for (auto it = graphs.begin(); it != graphs.end();) {
            if (pred(it->first)) {
                it = graphs.erase(it);
                st.graphs_evicted++;
            } else {
                ++it;
            }
        }
    }

    PlanEntry &plan_for(uint32_t frames) {
        auto it = plans.find(frames);
        if (it == plans.end()) {
            mmfhe_circuit_config cc = base;
            cc.frames = frames;
            std::unique_ptr<mmfhe_plan> h(new mmfhe_plan{create_plan(*c, cc)});
            plan_encode_consts(*h->p, 0);
            CK(cudaDeviceSynchronize());
            PlanEntry e;
            for (const PtDev &pt : h->p->consts) e.bytes += pt.buf.words() * 8;
            e.in_words = (size_t)h->p->n_in * c->ct_words(c->L);
            for (int l : h->p->out_levels) e.out_words += c->ct_words(l);
            e.h = std::move(h);
            it = plans.emplace(frames, std::move(e)).first;
            st.plans_created++;
            evict_plans(frames);
        }
        it->second.last_use = ++clock;
        return it->second;
    }

    // Least recently used plans (never `keep`) go until the budget holds.
    void evict_plans(uint32_t keep) {
        if (!cfg.plan_budget_bytes) return;
        bool freed = false;
        while (plan_bytes() > cfg.plan_budget_bytes && plans.size() > 1) {
            auto victim = plans.end();
            for (auto it = plans.begin(); it != plans.end(); ++it)
                if (it->first != keep && (victim == plans.end() || it->second.last_use < victim->second.last_use))
                    victim = it;
            if (victim == plans.end()) break;
            const uint32_t f = victim->first;
            drop_graphs_if([f](const GraphKey &k) { return std::get<0>(k) == f; });
            CK(cudaDeviceSynchronize());
            delete victim->second.h->p;
            plans.erase(victim);
            st.plans_evicted++;
            freed = true;
        }
        if (freed) c->pool->trim();
    }

    GraphEntry &graph_for(uint32_t frames, const Keys *k, uint32_t b, PlanEntry &pe) {
        const GraphKey key{frames, k, b};
        auto it = graphs.find(key);
        if (it == graphs.end()) {
            std::unique_ptr<GraphEntry> e(new GraphEntry());
            e->device = c->device;
            e->in_bytes = std::max<size_t>(8, b * pe.in_words * 8);
            e->out_bytes = std::max<size_t>(8, b * pe.out_words * 8);
            e->stage_in = (uint64_t *)dev_alloc(c->device, e->in_bytes);
            if (!e->stage_in) throw Error(MMFHE_ERR_OUT_OF_MEMORY, "batcher staging allocation failed");
            e->stage_out = (uint64_t *)dev_alloc(c->device, e->out_bytes);
            if (!e->stage_out) throw Error(MMFHE_ERR_OUT_OF_MEMORY, "batcher staging allocation failed");
            CK(cudaMemset(e->stage_in, 0, b * pe.in_words * 8));
            std::vector<const uint64_t *> ins(b);
            std::vector<uint64_t *> outs(b);
            std::vector<const Keys *> ks(b, k);
            for (uint32_t w = 0; w < b; w++) {
                ins[w] = e->stage_in + w * pe.in_words;
                outs[w] = e->stage_out + w * pe.out_words;
            }
            e->g = capture_eval(*c, *pe.h->p, ks.data(), ins.data(), b, outs.data());
            e->bytes = e->g->bytes() + b * (pe.in_words + pe.out_words) * 8;
            it = graphs.emplace(key, std::move(e)).first;
            st.graphs_captured++;
            evict_graphs(key);
        }
        it->second->last_use = ++clock;
        return *it->second;
    }

    void evict_graphs(const GraphKey &keep) {
        if (!cfg.graph_budget_bytes) return;
        while (graph_bytes() > cfg.graph_budget_bytes && graphs.size() > 1) {
            auto victim = graphs.end();
            for (auto it = graphs.begin(); it != graphs.end(); ++it)
                if (it->first != keep && (victim == graphs.end() || it->second->last_use < victim->second->last_use))
                    victim = it;
            if (victim == graphs.end()) break;
            const GraphKey vk = victim->first;
            drop_graphs_if([&vk](const GraphKey &k) { return k == vk; });
        }
    }

    void flush(cudaStream_t s) {
        if (pending.empty()) return;
        // groups of equal (frames, keys), in order of first submission
        std::vector<std::pair<std::pair<uint32_t, const Keys *>, std::vector<size_t>>> groups;
        std::map<std::pair<uint32_t, const Keys *>, size_t> gi;
        for (size_t i = 0; i < pending.size(); i++) {
            auto key = std::make_pair(pending[i].frames, pending[i].k);
            auto it = gi.find(key);
            if (it == gi.end()) {
                it = gi.emplace(key, groups.size()).first;
                groups.push_back({key, {}});
            }
            groups[it->second].second.push_back(i);
        }
        bool host = false;
        for (auto &g : groups) {
            const uint32_t frames = g.first.first;
            const Keys *k = g.first.second;
            PlanEntry &pe = plan_for(frames);
            const auto &idx = g.second;
            for (size_t s0 = 0; s0 < idx.size(); s0 += cfg.max_batch) {
                const uint32_t b = (uint32_t)std::min<size_t>(cfg.max_batch, idx.size() - s0);
                if (!cfg.use_graphs) {
                    std::vector<const uint64_t *> ins(b);
                    std::vector<uint64_t *> outs(b);
                    std::vector<const Keys *> ks(b, k);
                    for (uint32_t w = 0; w < b; w++) {
                        ins[w] = pending[idx[s0 + w]].in;
                        outs[w] = pending[idx[s0 + w]].out;
                    }
                    eval_windows(*c, *pe.h->p, ks.data(), ins.data(), b, outs.data(), s);
                } else {
                    GraphEntry &ge = graph_for(frames, k, b, pe);
                    for (uint32_t w = 0; w < b; w++)
                        CK(cudaMemcpyAsync(ge.stage_in + w * pe.in_words, pending[idx[s0 + w]].in, pe.in_words * 8,
                                           cudaMemcpyDefault, s));
                    graph_launch(*ge.g, s);
                    st.graph_replays++;
                    for (uint32_t w = 0; w < b; w++)
                        CK(cudaMemcpyAsync(pending[idx[s0 + w]].out, ge.stage_out + w * pe.out_words,
                                           pe.out_words * 8, cudaMemcpyDefault, s));
                }
                for (uint32_t w = 0; w < b; w++) host |= is_host_ptr(pending[idx[s0 + w]].out);
                st.batches++;
                st.windows += b;
            }
        }
        pending.clear();
        if (host) CK(cudaStreamSynchronize(s));
        CK(cudaGetLastError());
    }
};

extern "C" {

mmfhe_status mmfhe_graph_capture(mmfhe_ctx *ctx, const mmfhe_plan *plan, mmfhe_keys *const *keys,
                                 const uint64_t *const *in_cts, size_t batch, uint64_t *const *out_cts,
                                 mmfhe_graph **out) {
    Context *c = nullptr;
    B_TRY
    if (!ctx || !ctx->c) throw Error(MMFHE_ERR_BAD_ARG, "null context");
    c = ctx->c;
    CK(cudaSetDevice(c->device));
    if (!plan || !plan->p || plan->p->ctx != c) throw Error(MMFHE_ERR_BAD_ARG, "plan of another context");
    if (!out || !keys || !in_cts || !out_cts) throw Error(MMFHE_ERR_BAD_ARG, "null argument");
    std::vector<const Keys *> ks(batch);
    for (size_t w = 0; w < batch; w++) {
        if (!keys[w] || keys[w]->k.ctx != c) throw Error(MMFHE_ERR_BAD_ARG, "keys of another context");
        ks[w] = &keys[w]->k;
    }
    *out = capture_eval(*c, *plan->p, ks.data(), in_cts, batch, out_cts).release();
    B_CATCH(c)
}

mmfhe_status mmfhe_graph_launch(mmfhe_graph *graph, void *stream) {
    Context *c = nullptr;
    B_TRY
    if (!graph || !graph->exec) throw Error(MMFHE_ERR_BAD_ARG, "null graph");
    c = graph->c;
    CK(cudaSetDevice(c->device));
    graph_launch(*graph, (cudaStream_t)stream);
    B_CATCH(c)
}

mmfhe_status mmfhe_graph_info(const mmfhe_graph *graph, uint64_t *kernels, uint64_t *bytes) {
    if (!graph) return bfail(nullptr, MMFHE_ERR_BAD_ARG, "null graph");
    if (kernels) *kernels = graph->kernels;
    if (bytes) *bytes = graph->bytes();
    return MMFHE_OK;
}

mmfhe_status mmfhe_graph_destroy(mmfhe_graph *graph) {
    if (!graph) return MMFHE_OK;
    cudaSetDevice(graph->c->device);
    cudaDeviceSynchronize();
    delete graph;
    return MMFHE_OK;
}

mmfhe_status mmfhe_batcher_create(mmfhe_ctx *ctx, const mmfhe_circuit_config *base, size_t base_size,
                                  const mmfhe_batcher_config *cfg, mmfhe_batcher **out) {
    Context *c = nullptr;
    B_TRY
    if (!ctx || !ctx->c) throw Error(MMFHE_ERR_BAD_ARG, "null context");
    c = ctx->c;
    if (!base || base_size != sizeof(mmfhe_circuit_config) || !cfg || !out)
        throw Error(MMFHE_ERR_BAD_ARG, "bad batcher arguments");
    if (cfg->max_batch < 1 || cfg->max_batch > 256) throw Error(MMFHE_ERR_BAD_ARG, "max_batch must be 1..256");
    std::unique_ptr<mmfhe_batcher> b(new mmfhe_batcher());
    b->c = c;
    b->base = *base;
    b->cfg = *cfg;
    *out = b.release();
    B_CATCH(c)
}

mmfhe_status mmfhe_batcher_plan(mmfhe_batcher *b, uint32_t frames, const mmfhe_plan **out) {
    Context *c = nullptr;
    B_TRY
    if (!b || !out) throw Error(MMFHE_ERR_BAD_ARG, "null argument");
    c = b->c;
    CK(cudaSetDevice(c->device));
    *out = b->plan_for(frames).h.get();
    B_CATCH(c)
}

mmfhe_status mmfhe_batcher_submit(mmfhe_batcher *b, mmfhe_keys *keys, uint32_t frames, const uint64_t *in,
                                  uint64_t *out) {
    Context *c = nullptr;
    B_TRY
    if (!b || !keys || !in || !out) throw Error(MMFHE_ERR_BAD_ARG, "null argument");
    c = b->c;
    if (keys->k.ctx != c) throw Error(MMFHE_ERR_PARAM_MISMATCH, "keys of another context");
    if (frames < 2) throw Error(MMFHE_ERR_BAD_ARG, "window shorter than two frames");
    b->pending.push_back(mmfhe_batcher::Req{&keys->k, frames, in, out});
    B_CATCH(c)
}

mmfhe_status mmfhe_batcher_flush(mmfhe_batcher *b, void *stream) {
    Context *c = nullptr;
    B_TRY
    if (!b) throw Error(MMFHE_ERR_BAD_ARG, "null batcher");
    c = b->c;
    CK(cudaSetDevice(c->device));
    try {
        b->flush((cudaStream_t)stream);
    } catch (...) {
        b->pending.clear();   // a failed flush drops its windows
        throw;
    }
    B_CATCH(c)
}

mmfhe_status mmfhe_batcher_forget_keys(mmfhe_batcher *b, const mmfhe_keys *keys) {
    Context *c = nullptr;
    B_TRY
    if (!b || !keys) throw Error(MMFHE_ERR_BAD_ARG, "null argument");
    c = b->c;
    CK(cudaSetDevice(c->device));
    const Keys *k = &keys->k;
    b->drop_graphs_if([k](const mmfhe_batcher::GraphKey &g) { return std::get<1>(g) == k; });
    B_CATCH(c)
}

mmfhe_status mmfhe_batcher_stats_get(const mmfhe_batcher *b, mmfhe_batcher_stats *out) {
    if (!b || !out) return bfail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    *out = b->st;
    out->plan_bytes = b->plan_bytes();
    out->graph_bytes = b->graph_bytes();
    return MMFHE_OK;
}

mmfhe_status mmfhe_batcher_destroy(mmfhe_batcher *b) {
    if (!b) return MMFHE_OK;
    cudaSetDevice(b->c->device);
    cudaDeviceSynchronize();
    b->graphs.clear();
    for (auto &kv : b->plans) delete kv.second.h->p;
    b->plans.clear();
    delete b;
    return MMFHE_OK;
}

}  // extern "C"
