// Serving loop: windows from many users arrive on any thread; one worker
// thread admits them into batches of equal frame count (users mixed, each
// window switched with its own keys) whenever one of the stream slots is free, runs each batch on the slot's stream with the slot's
// private memory pool (so batches on different slots overlap on the device
// and never share scratch), and keeps users' keys resident under a device
// budget, reloading evicted users from their registered words.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "circuits.h"
#include "engine.h"
#include "handles.h"
#include "internal.h"

using namespace mmfhe;
using Clock = std::chrono::steady_clock;

struct mmfhe_server {
    Context *c = nullptr;
    mmfhe_circuit_config base{};
    mmfhe_server_config cfg{};

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread worker;

    struct User {
        const uint64_t *relin = nullptr;
        std::vector<std::pair<int32_t, const uint64_t *>> galois;
        std::unique_ptr<Keys> keys;   // resident when set (worker thread only)
        uint64_t bytes = 0, last_use = 0;
        int pins = 0;                 // running batches (worker thread only)
    };
    std::map<uint64_t, User> users;   // structure guarded by mu

    enum State { QUEUED, RUNNING, DONE, FAILED };
    struct Req {
        uint64_t user;
        uint32_t frames;
        const uint64_t *in;
        uint64_t *out;
        Clock::time_point t_submit, t_done;
        State state = QUEUED;
        mmfhe_status status = MMFHE_OK;
    };
    std::map<uint64_t, Req> reqs;     // guarded by mu
    std::deque<uint64_t> queue;       // guarded by mu
    uint64_t next_ticket = 1;

    struct Slot {
        cudaStream_t st = nullptr;
        cudaEvent_t done = nullptr;
        std::unique_ptr<Pool> pool;
        bool busy = false;
        std::vector<uint64_t> tickets;
        std::vector<User *> users;   // distinct users of the running batch (pinned)
    };
    std::vector<Slot> slots;
    std::map<uint32_t, std::unique_ptr<Plan>> plans;   // worker thread creates; count read under mu
    std::map<uint32_t, std::vector<double>> fc_layers; // learned layers applied to every plan (guarded by mu)
    // caller-encoded constants: frame count -> constant index -> coefficient-form words; set before the
    // first submit (guarded by mu), read-only afterwards
    std::map<uint32_t, std::map<uint32_t, std::vector<uint64_t>>> const_words;

    // statistics (guarded by mu)
    uint64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, batches = 0, batch_windows = 0;
    uint64_t key_loads = 0, key_evictions = 0;
    std::vector<double> lat_ms;
    Clock::time_point t_first{}, t_last{};
    bool any_submit = false;
    uint64_t clock = 0;

    uint64_t key_set_bytes(const User &u) const {
        return (uint64_t)(1 + u.galois.size()) * c->dnum * 2 * (c->num_q + c->num_p) * c->n * 8;
    }
    uint64_t resident_bytes() const {
        uint64_t s = 0;
        for (auto &kv : users)
            if (kv.second.keys) s += kv.second.bytes;
        return s;
    }

    const Plan &plan_for(uint32_t frames) {
        auto it = plans.find(frames);
        if (it == plans.end()) {
            mmfhe_circuit_config cc = base;
            cc.frames = frames;
            std::unique_ptr<Plan> p(create_plan(*c, cc));
            if (base.kind != MMFHE_CIRCUIT_FC) plan_encode_consts(*p, 0);
            std::map<uint32_t, std::vector<double>> layers;
            {
                std::lock_guard<std::mutex> g(mu);
                layers = fc_layers;
            }
            for (auto &kv : layers) plan_set_fc_layer(*p, kv.first, kv.second.data());
            const std::map<uint32_t, std::vector<uint64_t>> *words = nullptr;
            {
                std::lock_guard<std::mutex> g(mu);
                auto f = const_words.find(frames);
                if (f != const_words.end()) words = &f->second;
            }
            if (words) {
                for (auto &kv : *words) {
                    if (kv.first >= p->keys.size()) throw Error(MMFHE_ERR_BAD_ARG, "server constant index out of range");
                    if (kv.second.size() != (size_t)(p->keys[kv.first].level + 1) * c->n)
                        throw Error(MMFHE_ERR_BAD_ARG, "server constant size does not match the plan's constant");
                    plan_set_const(*p, kv.first, kv.second.data(), 0);
                }
                CK(cudaStreamSynchronize(0));
            }
            std::lock_guard<std::mutex> g(mu);
            it = plans.emplace(frames, std::move(p)).first;
        }
        return *it->second;
    }

    // True if u registered every key plan p needs.
    bool covers(const User &u, const Plan &p) const {
        std::vector<int32_t> have;
        for (auto &rg : u.galois) have.push_back(norm_rot(*c, rg.first));
        for (int32_t r : p.rotations)
            if (std::find(have.begin(), have.end(), norm_rot(*c, r)) == have.end()) return false;
        return u.relin != nullptr;
    }

    // Make u's keys resident; false if the budget cannot be met now (every
    // other resident user has a running batch).
    bool ensure_keys(User &u) {
        u.last_use = ++clock;
        if (u.keys) return true;
        const uint64_t need = key_set_bytes(u);
        if (cfg.key_budget_bytes) {
            if (need > cfg.key_budget_bytes) throw Error(MMFHE_ERR_OUT_OF_MEMORY, "key budget below one key set");
            std::lock_guard<std::mutex> g(mu);
            while (resident_bytes() + need > cfg.key_budget_bytes) {
                User *victim = nullptr;
                for (auto &kv : users)
                    if (kv.second.keys && kv.second.pins == 0 && &kv.second != &u &&
                        (!victim || kv.second.last_use < victim->last_use))
                        victim = &kv.second;
                if (!victim) return false;
                victim->keys.reset();   // no running batch reads these words
                key_evictions++;
            }
        }
        std::unique_ptr<Keys> k(new Keys());
        k->ctx = c;
        k->rlk = load_key(*c, u.relin);
        for (auto &rg : u.galois) k->gk[norm_rot(*c, rg.first)] = load_key(*c, rg.second);
        std::lock_guard<std::mutex> g(mu);
        u.keys = std::move(k);
        u.bytes = need;
        key_loads++;
        return true;
    }

    void finish(Slot &s, bool ok, mmfhe_status code) {
        const auto now = Clock::now();
        {
            std::lock_guard<std::mutex> g(mu);
            for (uint64_t t : s.tickets) {
                Req &r = reqs[t];
                r.t_done = now;
                if (ok) {
                    r.state = DONE;
                    completed++;
                    lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r.t_submit).count());
                    t_last = now;
                } else {
                    r.state = FAILED;
                    r.status = code;
                    failed++;
                }
            }
        }
        for (User *u : s.users) u->pins--;
        s.users.clear();
        s.tickets.clear();
        s.busy = false;
        cv_done.notify_all();
    }

    // True when a batch should go now: max_batch windows of the oldest
    // window's frame count are queued, or the oldest has waited batch_wait_us.
    bool batch_ready() {
        std::lock_guard<std::mutex> g(mu);
        if (queue.empty()) return false;
        if (cfg.batch_wait_us == 0 || stop) return true;
        const Req &first = reqs[queue.front()];
        if (Clock::now() - first.t_submit >= std::chrono::microseconds(cfg.batch_wait_us)) return true;
        uint32_t n = 0;
        for (uint64_t t : queue)
            if (reqs[t].frames == first.frames && ++n >= cfg.max_batch) return true;
        return false;
    }

    // Take queued windows of the oldest window's frame count, up to
    // max_batch: the oldest window first, then windows whose users' keys are
    // resident, then the others, in queue order, as long as the distinct
    // users' key sets fit the key budget together.  Users of a batch may
    // differ (each window keeps its own keys).
    bool take_batch(std::vector<uint64_t> &tickets, uint32_t &frames, std::vector<User *> &batch_users,
                    std::vector<User *> &window_users) {
        std::lock_guard<std::mutex> g(mu);
        if (queue.empty()) return false;
        frames = reqs[queue.front()].frames;
        uint64_t bytes = 0;
        auto take = [&](bool resident_only, bool first_only) {
            for (auto it = queue.begin(); it != queue.end() && tickets.size() < cfg.max_batch;) {
                Req &r = reqs[*it];
                User *u = &users[r.user];
                if (r.frames != frames || (resident_only && !u->keys)) {
                    ++it;
                    continue;
                }
                const bool known = std::find(batch_users.begin(), batch_users.end(), u) != batch_users.end();
                if (!known) {
                    const uint64_t need = key_set_bytes(*u);
                    if (cfg.key_budget_bytes && !batch_users.empty() && bytes + need > cfg.key_budget_bytes) {
                        ++it;
                        continue;
                    }
                    bytes += need;
                    batch_users.push_back(u);
                }
                tickets.push_back(*it);
                window_users.push_back(u);
                r.state = RUNNING;
                it = queue.erase(it);
                if (first_only) return;
            }
        };
        take(false, true);    // the oldest window always goes
        take(true, false);    // windows that need no key upload
        take(false, false);   // the rest, budget permitting
        return true;
    }

    void requeue_front(const std::vector<uint64_t> &tickets) {
        std::lock_guard<std::mutex> g(mu);
        for (auto it = tickets.rbegin(); it != tickets.rend(); ++it) {
            reqs[*it].state = QUEUED;
            queue.push_front(*it);
        }
    }

    void dispatch(Slot &s, const std::vector<uint64_t> &tickets, const std::vector<User *> &window_users,
                  uint32_t frames) {
        const Plan &p = plan_for(frames);
        size_t out_words = 0;
        for (int l : p.out_levels) out_words += c->ct_words(l);
        const size_t b = tickets.size();
        std::vector<const uint64_t *> ins(b);
        std::vector<uint64_t *> user_outs(b), outs(b);
        std::vector<const Keys *> ks(b);
        for (size_t w = 0; w < b; w++) ks[w] = window_users[w]->keys.get();
        {
            std::lock_guard<std::mutex> g(mu);
            for (size_t w = 0; w < b; w++) {
                ins[w] = reqs[tickets[w]].in;
                user_outs[w] = reqs[tickets[w]].out;
            }
        }
        std::swap(c->pool, s.pool);   // this batch allocates from the slot's pool
        try {
            Buf stage(c->pool.get(), b * out_words);   // reused only by later work on this slot's stream
            for (size_t w = 0; w < b; w++) outs[w] = stage.get() + w * out_words;
            eval_windows(*c, p, ks.data(), ins.data(), b, outs.data(), s.st, true);
            for (size_t w = 0; w < b; w++)
                CK(cudaMemcpyAsync(user_outs[w], outs[w], out_words * 8, cudaMemcpyDefault, s.st));
            CK(cudaEventRecord(s.done, s.st));
        } catch (...) {
            std::swap(c->pool, s.pool);
            throw;
        }
        std::swap(c->pool, s.pool);
        s.tickets = tickets;
        s.busy = true;
        std::lock_guard<std::mutex> g(mu);
        batches++;
        batch_windows += b;
    }

    void run() {
        CK(cudaSetDevice(c->device));
        for (;;) {
            bool progressed = false;
            // retire finished batches
            for (Slot &s : slots) {
                if (!s.busy) continue;
                const cudaError_t e = cudaEventQuery(s.done);
                if (e == cudaErrorNotReady) continue;
                if (e == cudaSuccess) {
                    finish(s, true, MMFHE_OK);
                } else {
                    cudaGetLastError();
                    finish(s, false, MMFHE_ERR_CUDA);
                }
                progressed = true;
            }
            // admit the next batch into a free slot
            Slot *free_slot = nullptr;
            for (Slot &s : slots)
                if (!s.busy) {
                    free_slot = &s;
                    break;
                }
            if (free_slot) {
                std::vector<uint64_t> tickets;
                uint32_t frames = 0;
                std::vector<User *> bu, wu;
                if (batch_ready() && take_batch(tickets, frames, bu, wu)) {
                    try {
                        // windows whose user lacks a key the plan needs fail alone
                        const Plan &p = plan_for(frames);
                        std::vector<uint64_t> bad;
                        for (size_t i = 0; i < tickets.size();) {
                            if (covers(*wu[i], p)) {
                                ++i;
                                continue;
                            }
                            bad.push_back(tickets[i]);
                            tickets.erase(tickets.begin() + i);
                            wu.erase(wu.begin() + i);
                        }
                        if (!bad.empty()) {
                            Slot tmp;
                            tmp.tickets = bad;
                            finish(tmp, false, MMFHE_ERR_NOT_FOUND);
                            bu.clear();
                            for (User *u : wu)
                                if (std::find(bu.begin(), bu.end(), u) == bu.end()) bu.push_back(u);
                            progressed = true;
                            if (tickets.empty()) continue;
                        }
                        // keys of every user of the batch resident and pinned
                        bool ok = true;
                        for (User *u : bu) {
                            if (!ensure_keys(*u)) {
                                ok = false;
                                break;
                            }
                            u->pins++;
                            free_slot->users.push_back(u);
                        }
                        if (!ok) {
                            for (User *u : free_slot->users) u->pins--;
                            free_slot->users.clear();
                            requeue_front(tickets);   // waits for a running batch to release keys
                        } else {
                            dispatch(*free_slot, tickets, wu, frames);
                            progressed = true;
                        }
                    } catch (const Error &e) {
                        free_slot->tickets = tickets;
                        finish(*free_slot, false, e.code);
                        progressed = true;
                    } catch (...) {
                        free_slot->tickets = tickets;
                        finish(*free_slot, false, MMFHE_ERR_CUDA);
                        progressed = true;
                    }
                }
            }
            if (progressed) continue;
            bool busy = false;
            for (Slot &s : slots) busy |= s.busy;
            std::unique_lock<std::mutex> lk(mu);
            if (stop && queue.empty() && !busy) break;
            // running or filling a batch: poll; idle: sleep until a submission
            if (busy || !queue.empty())
                cv_work.wait_for(lk, std::chrono::microseconds(50));
            else
                cv_work.wait_for(lk, std::chrono::milliseconds(20), [this] { return stop || !queue.empty(); });
        }
    }
};

namespace {

mmfhe_status sfail(Context *c, mmfhe_status code, const char *msg) {
    if (c) c->last_error = msg;
    return code;
}

}  // namespace

extern "C" {

mmfhe_status mmfhe_server_create(mmfhe_ctx *ctx, const mmfhe_circuit_config *base, size_t base_size,
                                 const mmfhe_server_config *cfg, mmfhe_server **out) {
    Context *c = nullptr;
    try {
        if (!ctx || !ctx->c) throw Error(MMFHE_ERR_BAD_ARG, "null context");
        c = ctx->c;
        if (!base || base_size != sizeof(mmfhe_circuit_config) || !cfg || !out)
            throw Error(MMFHE_ERR_BAD_ARG, "bad server arguments");
        if (cfg->max_batch < 1 || cfg->max_batch > 256 || cfg->streams < 1 || cfg->streams > 8)
            throw Error(MMFHE_ERR_BAD_ARG, "max_batch must be 1..256 and streams 1..8");
        CK(cudaSetDevice(c->device));
        std::unique_ptr<mmfhe_server> s(new mmfhe_server());
        s->c = c;
        s->base = *base;
        s->cfg = *cfg;
        s->slots.resize(cfg->streams);
        for (auto &sl : s->slots) {
            CK(cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
            sl.pool.reset(new Pool(c->device));
        }
        CK(cudaDeviceSynchronize());
        mmfhe_server *raw = s.get();
        s->worker = std::thread([raw] {
            try {
                raw->run();
            } catch (...) {
                std::lock_guard<std::mutex> g(raw->mu);
                raw->stop = true;
            }
        });
        *out = s.release();
    } catch (const Error &e) {
        return sfail(c, e.code, e.what());
    } catch (const std::exception &e) {
        return sfail(c, MMFHE_ERR_CUDA, e.what());
    }
    return MMFHE_OK;
}

mmfhe_status mmfhe_server_add_user(mmfhe_server *s, uint64_t user_id, const uint64_t *relin, const int32_t *rotations,
                                   const uint64_t *const *galois, uint32_t n_rot) {
    if (!s || !relin || (n_rot && (!rotations || !galois))) return sfail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    std::lock_guard<std::mutex> g(s->mu);
    if (s->users.count(user_id)) return sfail(s->c, MMFHE_ERR_BAD_ARG, "user already registered");
    mmfhe_server::User &u = s->users[user_id];
    u.relin = relin;
    for (uint32_t i = 0; i < n_rot; i++) {
        if (!galois[i]) return sfail(s->c, MMFHE_ERR_BAD_ARG, "null Galois key");
        u.galois.push_back({rotations[i], galois[i]});
    }
    return MMFHE_OK;
}

mmfhe_status mmfhe_server_set_fc_layer(mmfhe_server *s, uint32_t layer, const double *W, size_t count) {
    if (!s || !W) return sfail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    const mmfhe_circuit_config &b = s->base;
    size_t want = 0;
    if (b.kind == MMFHE_CIRCUIT_FC && layer < b.taps) want = (size_t)b.bins * b.bins;
    if (b.kind == MMFHE_CIRCUIT_GESTURE && layer < 3)
        want = layer == 0 ? (size_t)b.fc_width * (b.fc_dims[0] + 1) : (size_t)b.fc_width * b.fc_width;
    if (!want) return sfail(s->c, MMFHE_ERR_BAD_ARG, "the server's circuit has no such learned layer");
    if (count != want) return sfail(s->c, MMFHE_ERR_BAD_ARG, "wrong layer size");
    std::lock_guard<std::mutex> g(s->mu);
    if (!s->plans.empty() || s->submitted) return sfail(s->c, MMFHE_ERR_BUSY, "layers are set before the first submit");
    s->fc_layers[layer].assign(W, W + count);
    return MMFHE_OK;
}

mmfhe_status mmfhe_server_set_const(mmfhe_server *s, uint32_t frames, uint32_t index, const uint64_t *words,
                                    size_t count) {
    if (!s || !words || !count) return sfail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    std::lock_guard<std::mutex> g(s->mu);
    if (!s->plans.empty() || s->submitted) return sfail(s->c, MMFHE_ERR_BUSY, "constants are set before the first submit");
    s->const_words[frames][index].assign(words, words + count);
    return MMFHE_OK;
}

mmfhe_status mmfhe_server_submit(mmfhe_server *s, uint64_t user_id, uint32_t frames, const uint64_t *in,
                                 uint64_t *out, uint64_t *ticket) {
    if (!s || !in || !out || !ticket) return sfail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (!s->users.count(user_id)) return sfail(s->c, MMFHE_ERR_NOT_FOUND, "unknown user");
        if (s->stop) return sfail(s->c, MMFHE_ERR_BUSY, "server stopping");
        const uint64_t t = s->next_ticket++;
        mmfhe_server::Req &r = s->reqs[t];
        r.user = user_id;
        r.frames = frames;
        r.in = in;
        r.out = out;
        r.t_submit = Clock::now();
        if (!s->any_submit) {
            s->any_submit = true;
            s->t_first = r.t_submit;
        }
        s->submitted++;
        s->queue.push_back(t);
        *ticket = t;
    }
    s->cv_work.notify_one();
    return MMFHE_OK;
}

mmfhe_status mmfhe_server_cancel(mmfhe_server *s, uint64_t ticket) {
    if (!s) return sfail(nullptr, MMFHE_ERR_BAD_ARG, "null server");
    {
        std::lock_guard<std::mutex> g(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return sfail(s->c, MMFHE_ERR_NOT_FOUND, "unknown ticket");
        mmfhe_server::Req &r = it->second;
        if (r.state != mmfhe_server::QUEUED) return sfail(s->c, MMFHE_ERR_BUSY, "the window is running or complete");
        auto q = std::find(s->queue.begin(), s->queue.end(), ticket);
        if (q == s->queue.end()) return sfail(s->c, MMFHE_ERR_BUSY, "the window is being dispatched");
        s->queue.erase(q);
        r.state = mmfhe_server::FAILED;
        r.status = MMFHE_ERR_CANCELLED;
        r.t_done = Clock::now();
        s->cancelled++;
    }
    s->cv_done.notify_all();
    return MMFHE_OK;
}

mmfhe_status mmfhe_server_wait(mmfhe_server *s, uint64_t ticket, uint32_t timeout_ms, double *latency_ms) {
    if (!s) return sfail(nullptr, MMFHE_ERR_BAD_ARG, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return sfail(s->c, MMFHE_ERR_NOT_FOUND, "unknown ticket");
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        return it->second.state == mmfhe_server::DONE || it->second.state == mmfhe_server::FAILED;
    });
    if (!ok) return MMFHE_ERR_TIMEOUT;
    if (latency_ms)
        *latency_ms = std::chrono::duration<double, std::milli>(it->second.t_done - it->second.t_submit).count();
    return it->second.state == mmfhe_server::DONE ? MMFHE_OK : it->second.status;
}

mmfhe_status mmfhe_server_drain(mmfhe_server *s, uint32_t timeout_ms) {
    if (!s) return sfail(nullptr, MMFHE_ERR_BAD_ARG, "null server");
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                        [&] { return s->completed + s->failed + s->cancelled == s->submitted; });
    return ok ? MMFHE_OK : MMFHE_ERR_TIMEOUT;
}

mmfhe_status mmfhe_server_stats_get(mmfhe_server *s, mmfhe_server_stats *out) {
    if (!s || !out) return sfail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    std::lock_guard<std::mutex> g(s->mu);
    *out = mmfhe_server_stats{};
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->failed = s->failed;
    out->cancelled = s->cancelled;
    out->batches = s->batches;
    out->key_loads = s->key_loads;
    out->key_evictions = s->key_evictions;
    for (auto &kv : s->users)
        if (kv.second.keys) {
            out->keys_resident++;
            out->key_bytes += kv.second.bytes;
        }
    out->mean_batch = s->batches ? (double)s->batch_windows / (double)s->batches : 0.0;
    if (!s->lat_ms.empty()) {
        std::vector<double> v = s->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&v](double p) {
            const size_t i = (size_t)std::min<double>(v.size() - 1, std::ceil(p * v.size()) - 1);
            return v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
        out->windows_per_s = span > 0 ? (double)s->completed / span : 0.0;
    }
    return MMFHE_OK;
}

mmfhe_status mmfhe_server_destroy(mmfhe_server *s) {
    if (!s) return MMFHE_OK;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->c->device);
    cudaDeviceSynchronize();
    for (auto &sl : s->slots) {
        sl.pool.reset();
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    s->plans.clear();
    s->users.clear();
    delete s;
    return MMFHE_OK;
}

}  // extern "C"
