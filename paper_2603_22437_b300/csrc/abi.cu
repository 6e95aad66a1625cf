// extern "C" entry points of libmmfhe (declared in include/mmfhe.h).
// Every call catches all exceptions and returns a status code.
#include <cuda_runtime.h>

#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <set>
#include <thread>

#include "circuits.h"
#include "engine.h"
#include "handles.h"
#include "hostmath.h"

using namespace mmfhe;

namespace mmfhe {
Context *create_context(const mmfhe_params &p, int device);
void destroy_context(Context *c);
mmfhe_status params_select(uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, uint32_t, mmfhe_params *);
}  // namespace mmfhe

static thread_local std::string g_last_error;

void mmfhe::set_thread_error(const std::string &msg) { g_last_error = msg; }

static mmfhe_status fail(Context *c, mmfhe_status code, const char *msg) {
    g_last_error = msg;
    if (c) c->last_error = msg;
    return code;
}

#define ABI_TRY try {
#define ABI_CATCH(ctxptr)                                                        \
    }                                                                            \
    catch (const Error &e) { return fail(ctxptr, e.code, e.what()); }            \
    catch (const std::bad_alloc &) { return fail(ctxptr, MMFHE_ERR_OUT_OF_MEMORY, "host allocation failed"); } \
    catch (const std::exception &e) { return fail(ctxptr, MMFHE_ERR_CUDA, e.what()); } \
    catch (...) { return fail(ctxptr, MMFHE_ERR_CUDA, "unknown error"); }       \
    return MMFHE_OK;

static Context *ctx_of(mmfhe_ctx *c) {
    if (!c || !c->c) throw Error(MMFHE_ERR_BAD_ARG, "null context");
    CK(cudaSetDevice(c->c->device));
    return c->c;
}

bool mmfhe::is_host_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged;
}

static void check_ptr(const void *p, const char *what) {
    if (!p) throw Error(MMFHE_ERR_BAD_ARG, std::string("null pointer: ") + what);
    if (!is_host_ptr(p) && ((uintptr_t)p & 15)) throw Error(MMFHE_ERR_BAD_ARG, std::string("device pointer not 16-byte aligned: ") + what);
}

static void check_level(const Context &c, uint32_t level) {
    if ((int)level > c.L) throw Error(MMFHE_ERR_LEVEL_MISMATCH, "level above the top level");
}

// Load B ciphertexts (coefficient form) from per-window pointers into the evaluation domain.
static CtB load_cts(Context &c, const uint64_t *const *ptrs, size_t offset_words, int B, int level, double scale,
                    cudaStream_t st) {
    CtB r = ct_new(c, B, level, scale);
    const size_t w = c.ct_words(level);
    for (int b = 0; b < B; b++)
        CK(cudaMemcpyAsync(r.ptr() + b * w, ptrs[b] + offset_words, w * 8, cudaMemcpyDefault, st));
    ntt_q_blocks(c, r.ptr(), (size_t)B * 2, level + 1, false, st);
    return r;
}

// Store a batch back in coefficient form; returns true if any destination is host memory.
static bool store_cts(Context &c, const CtB &a, uint64_t *const *ptrs, size_t offset_words, cudaStream_t st) {
    const int nl = a.level + 1;
    const size_t w = c.ct_words(a.level);
    Buf tmp(c.pool.get(), (size_t)a.B * w);
    std::vector<int> pids(nl);
    for (int i = 0; i < nl; i++) pids[i] = i;
    RowsView src{a.ptr(), make_map(nl, nl, pids), (size_t)a.B * 2 * nl};
    RowsView dst{tmp.get(), make_map(nl, nl, pids), (size_t)a.B * 2 * nl};
    launch_ntt(c, src, dst, true, st);
    bool host = false;
    for (int b = 0; b < a.B; b++) {
        host |= is_host_ptr(ptrs[b]);
        CK(cudaMemcpyAsync(ptrs[b] + offset_words, tmp.get() + b * w, w * 8, cudaMemcpyDefault, st));
    }
    if (host) CK(cudaStreamSynchronize(st));
    return host;
}

static std::vector<const uint64_t *> contiguous(const uint64_t *base, size_t B, size_t stride) {
    std::vector<const uint64_t *> v(B);
    for (size_t b = 0; b < B; b++) v[b] = base + b * stride;
    return v;
}

static std::vector<uint64_t *> contiguous_out(uint64_t *base, size_t B, size_t stride) {
    std::vector<uint64_t *> v(B);
    for (size_t b = 0; b < B; b++) v[b] = base + b * stride;
    return v;
}

// Evaluate a plan on `batch` windows; windows with the same key set form one
// batch (every launch covers all of them).  Pointers may be host or device.
void mmfhe::eval_windows(Context &c, const Plan &p, const Keys *const *keys, const uint64_t *const *in_cts,
                         size_t batch, uint64_t *const *out_cts, cudaStream_t st, bool mix_users, double in_scale,
                         std::vector<double> *out_scales) {
    // groups of windows evaluated together, with the key set they run under
    std::vector<std::pair<const Keys *, std::vector<size_t>>> groups;
    std::vector<std::unique_ptr<Keys>> mixed;   // per-window key views of mixed batches
    // a gesture batch holds every pair of every window: one key set per batch
    if (p.cfg.kind == MMFHE_CIRCUIT_GESTURE) mix_users = false;
    for (size_t w = 0; w < batch; w++) {
        check_ptr(in_cts[w], "window input");
        check_ptr(out_cts[w], "window output");
    }
    if (!mix_users) {
        std::map<const Keys *, size_t> gi;
        for (size_t w = 0; w < batch; w++) {
            auto it = gi.find(keys[w]);
            if (it == gi.end()) {
                it = gi.emplace(keys[w], groups.size()).first;
                groups.push_back({keys[w], {}});
            }
            groups[it->second].second.push_back(w);
        }
    } else {
        for (size_t w0 = 0; w0 < batch; w0 += MAX_KEY_WINDOWS) {
            const size_t nb = std::min<size_t>(MAX_KEY_WINDOWS, batch - w0);
            std::vector<size_t> idx(nb);
            bool same = true;
            for (size_t i = 0; i < nb; i++) {
                idx[i] = w0 + i;
                same &= keys[w0 + i] == keys[w0];
            }
            if (same) {
                groups.push_back({keys[w0], idx});
                continue;
            }
            std::unique_ptr<Keys> view(new Keys());
            view->ctx = &c;
            for (size_t i = 0; i < nb; i++) view->windows.push_back(keys[w0 + i]);
            groups.push_back({view.get(), idx});
            mixed.push_back(std::move(view));
        }
    }
    const size_t in_w = c.ct_words(c.L);
    std::vector<size_t> out_off(p.out_levels.size());
    size_t off = 0;
    for (size_t o = 0; o < p.out_levels.size(); o++) {
        out_off[o] = off;
        off += c.ct_words(p.out_levels[o]);
    }
    bool host_out = false;
    for (auto &g : groups) {
        const Keys &K = *g.first;
        const int B = (int)g.second.size();
        std::vector<const uint64_t *> ins(B);
        std::vector<uint64_t *> outs(B);
        for (int b = 0; b < B; b++) {
            ins[b] = in_cts[g.second[b]];
            outs[b] = out_cts[g.second[b]];
        }
        std::vector<CtB> in;
        if (p.cfg.kind == MMFHE_CIRCUIT_GESTURE && p.cfg.complex_slots) {
            // one complex-slot ciphertext per pair, window-major
            std::vector<const uint64_t *> z((size_t)B * p.pairs);
            for (int b = 0; b < B; b++)
                for (int j = 0; j < p.pairs; j++) z[(size_t)b * p.pairs + j] = ins[b] + (size_t)j * in_w;
            in.push_back(load_cts(c, z.data(), 0, B * p.pairs, c.L, in_scale, st));
        } else if (p.cfg.kind == MMFHE_CIRCUIT_GESTURE) {
            // Re and Im of all pairs of all windows, window-major
            std::vector<const uint64_t *> re((size_t)B * p.pairs), im((size_t)B * p.pairs);
            for (int b = 0; b < B; b++)
                for (int j = 0; j < p.pairs; j++) {
                    re[(size_t)b * p.pairs + j] = ins[b] + (size_t)(2 * j) * in_w;
                    im[(size_t)b * p.pairs + j] = ins[b] + (size_t)(2 * j + 1) * in_w;
                }
            in.push_back(load_cts(c, re.data(), 0, B * p.pairs, c.L, in_scale, st));
            in.push_back(load_cts(c, im.data(), 0, B * p.pairs, c.L, in_scale, st));
        } else {
            for (int i = 0; i < p.n_in; i++) in.push_back(load_cts(c, ins.data(), i * in_w, B, c.L, in_scale, st));
        }
        std::vector<CtB> res = run_plan(c, p, K, in, st);
        in.clear();
        if (out_scales) {
            out_scales->clear();
            for (auto &r : res) out_scales->push_back(r.scale);
        }
        for (size_t o = 0; o < res.size(); o++) host_out |= store_cts(c, res[o], outs.data(), out_off[o], st);
    }
    if (host_out) CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
}

static const Keys &keys_of(const mmfhe_keys *k, const Context *c) {
    if (!k) throw Error(MMFHE_ERR_BAD_ARG, "null keys");
    if (k->k.ctx != c) throw Error(MMFHE_ERR_PARAM_MISMATCH, "keys belong to another context");
    return k->k;
}

Buf mmfhe::load_key(Context &c, const uint64_t *words) {
    check_ptr(words, "key words");
    const int rows = c.num_q + c.num_p;
    const size_t total = (size_t)c.dnum * 2 * rows * c.n;
    // the context pool reuses a freed buffer at once, which is safe only in
    // stream order; evaluations may run on a caller's stream, so wait for
    // all device work before this set-up step allocates from the pool
    CK(cudaDeviceSynchronize());
    Buf b(c.pool.get(), total);
    CK(cudaMemcpy(b.get(), words, total * 8, cudaMemcpyDefault));
    std::vector<int> pids(rows);
    for (int i = 0; i < rows; i++) pids[i] = i;
    RowsView v{b.get(), make_map(rows, rows, pids), (size_t)c.dnum * 2 * rows};
    launch_ntt(c, v, v, false, 0);
    k_launch_mont_convert(c, v, true, 0);   // keys are kept in Montgomery form (key inner product)
    CK(cudaStreamSynchronize(0));
    return b;
}

extern "C" {

mmfhe_status mmfhe_params_select(uint32_t log_n, uint32_t num_q, uint32_t q0_bits, uint32_t q_bits, uint32_t num_p,
                                 uint32_t p_bits, uint32_t dnum, mmfhe_params *out) {
    ABI_TRY
    if (!out) throw Error(MMFHE_ERR_BAD_ARG, "null output");
    params_select(log_n, num_q, q0_bits, q_bits, num_p, p_bits, dnum, out);
    ABI_CATCH(nullptr)
}

mmfhe_status mmfhe_ctx_create(const mmfhe_params *params, size_t params_size, int device, mmfhe_ctx **out) {
    ABI_TRY
    if (!params || !out || params_size != sizeof(mmfhe_params)) throw Error(MMFHE_ERR_BAD_ARG, "bad parameter struct");
    *out = nullptr;
    Context *c = create_context(*params, device);
    *out = new mmfhe_ctx{c};
    ABI_CATCH(nullptr)
}

mmfhe_status mmfhe_ctx_destroy(mmfhe_ctx *ctx) {
    ABI_TRY
    if (!ctx) return MMFHE_OK;
    destroy_context(ctx->c);
    delete ctx;
    ABI_CATCH(nullptr)
}

const char *mmfhe_last_error(const mmfhe_ctx *ctx) {
    if (ctx && ctx->c) return ctx->c->last_error.c_str();
    return g_last_error.c_str();
}

mmfhe_status mmfhe_sync(mmfhe_ctx *ctx, void *stream, uint32_t timeout_ms) {
    Context *c = nullptr;
    ABI_TRY
    c = ctx_of(ctx);
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery((cudaStream_t)stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) CK(e);
        auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
        if (ms >= (long long)timeout_ms) throw Error(MMFHE_ERR_TIMEOUT, "stream still busy after timeout");
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    ABI_CATCH(c)
}

mmfhe_status mmfhe_launch_count(const mmfhe_ctx *ctx, uint64_t *out) {
    if (!ctx || !ctx->c || !out) return fail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    *out = ctx->c->launches;
    return MMFHE_OK;
}

mmfhe_status mmfhe_mem_stats_get(const mmfhe_ctx *ctx, mmfhe_mem_stats *out) {
    if (!ctx || !ctx->c || !out) return fail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    Context *c = ctx->c;
    mem_stats(c->device, &out->device_bytes, &out->peak_bytes, &out->allocations);
    out->pool_bytes = c->pool ? c->pool->bytes_held() : 0;
    out->pool_free_bytes = c->pool ? c->pool->bytes_free() : 0;
    return MMFHE_OK;
}

mmfhe_status mmfhe_mem_peak_reset(mmfhe_ctx *ctx) {
    if (!ctx || !ctx->c) return fail(nullptr, MMFHE_ERR_BAD_ARG, "null context");
    mem_peak_reset(ctx->c->device);
    return MMFHE_OK;
}

mmfhe_status mmfhe_debug_fail_allocations(int64_t after) {
    set_fail_after(after);
    return MMFHE_OK;
}

mmfhe_status mmfhe_trace_enable(mmfhe_ctx *ctx, int enable) {
    if (!ctx || !ctx->c) return fail(nullptr, MMFHE_ERR_BAD_ARG, "null context");
    ctx->c->tracing = enable != 0;
    if (enable) ctx->c->trace.clear();
    return MMFHE_OK;
}

mmfhe_status mmfhe_trace_get(const mmfhe_ctx *ctx, char *buf, size_t capacity, size_t *length) {
    if (!ctx || !ctx->c || !length) return fail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    std::string s;
    for (const std::string &l : ctx->c->trace) {
        s += l;
        s += '\n';
    }
    *length = s.size();
    if (buf && capacity) {
        size_t n = std::min(capacity - 1, s.size());
        memcpy(buf, s.data(), n);
        buf[n] = 0;
    }
    return MMFHE_OK;
}

mmfhe_status mmfhe_profile_enable(mmfhe_ctx *ctx, int enable) {
    Context *c = nullptr;
    ABI_TRY
    c = ctx_of(ctx);
    if (enable) {
        CK(cudaDeviceSynchronize());
        c->prof.clear();
        c->event_next = 0;
    }
    c->profiling = enable != 0;
    ABI_CATCH(c)
}

mmfhe_status mmfhe_profile_get(mmfhe_ctx *ctx, mmfhe_kernel_stat *out, uint32_t capacity, uint32_t *count) {
    Context *c = nullptr;
    ABI_TRY
    c = ctx_of(ctx);
    if (!count) throw Error(MMFHE_ERR_BAD_ARG, "null count");
    CK(cudaDeviceSynchronize());
    std::map<std::string, mmfhe_kernel_stat> agg;
    std::vector<std::string> order;
    for (const auto &r : c->prof) {
        if (!r.name || !r.stop) continue;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, r.start, r.stop));
        auto it = agg.find(r.name);
        if (it == agg.end()) {
            mmfhe_kernel_stat s{};
            snprintf(s.name, sizeof s.name, "%s", r.name);
            it = agg.emplace(r.name, s).first;
            order.push_back(r.name);
        }
        it->second.launches++;
        it->second.total_ms += ms;
        it->second.bytes += r.bytes;
        it->second.butterflies += r.butterflies;
        it->second.macs += r.macs;
    }
    *count = (uint32_t)agg.size();
    if (out)
        for (uint32_t i = 0; i < capacity && i < order.size(); i++) out[i] = agg[order[i]];
    ABI_CATCH(c)
}

mmfhe_status mmfhe_measure_butterfly_peak(mmfhe_ctx *ctx, double *bf64_per_s, double *bf32_per_s) {
    Context *c = nullptr;
    ABI_TRY
    c = ctx_of(ctx);
    if (!bf64_per_s || !bf32_per_s) throw Error(MMFHE_ERR_BAD_ARG, "null output");
    CK(cudaSetDevice(c->device));
    measure_butterfly_peak(*c, bf64_per_s, bf32_per_s);
    ABI_CATCH(c)
}

mmfhe_status mmfhe_measure_mac_peak(mmfhe_ctx *ctx, double *mac64_per_s) {
    Context *c = nullptr;
    ABI_TRY
    c = ctx_of(ctx);
    if (!mac64_per_s) throw Error(MMFHE_ERR_BAD_ARG, "null output");
    CK(cudaSetDevice(c->device));
    *mac64_per_s = measure_mac_peak(*c);
    ABI_CATCH(c)
}

// ---- keys ----
mmfhe_status mmfhe_keys_create(mmfhe_ctx *ctx, uint64_t user_id, mmfhe_keys **out) {
    Context *c = nullptr;
    ABI_TRY
    c = ctx_of(ctx);
    if (!out) throw Error(MMFHE_ERR_BAD_ARG, "null output");
    mmfhe_keys *k = new mmfhe_keys();
    k->k.ctx = c;
    k->k.user = user_id;
    *out = k;
    ABI_CATCH(c)
}

mmfhe_status mmfhe_keys_set_relin(mmfhe_keys *keys, const uint64_t *words) {
    Context *c = nullptr;
    ABI_TRY
    if (!keys || !keys->k.ctx) throw Error(MMFHE_ERR_BAD_ARG, "null keys");
    c = keys->k.ctx;
    CK(cudaSetDevice(c->device));
    keys->k.rlk = load_key(*c, words);
    ABI_CATCH(c)
}

mmfhe_status mmfhe_keys_set_galois(mmfhe_keys *keys, int32_t rotation, const uint64_t *words) {
    Context *c = nullptr;
    ABI_TRY
    if (!keys || !keys->k.ctx) throw Error(MMFHE_ERR_BAD_ARG, "null keys");
    c = keys->k.ctx;
    CK(cudaSetDevice(c->device));
    int32_t r = norm_rot(*c, rotation);
    if (r == 0) throw Error(MMFHE_ERR_BAD_ARG, "rotation by 0 needs no key");
    keys->k.gk[r] = load_key(*c, words);
    ABI_CATCH(c)
}

mmfhe_status mmfhe_keys_unload(mmfhe_keys *keys) {
    ABI_TRY
    if (!keys) return MMFHE_OK;
    if (keys->k.ctx) {
        CK(cudaSetDevice(keys->k.ctx->device));
        CK(cudaDeviceSynchronize());
    }
    delete keys;
    ABI_CATCH(nullptr)
}

// ---- primitives ----
mmfhe_status mmfhe_ntt(mmfhe_ctx *ctx, uint64_t *rows, const uint32_t *prime_idx, size_t num_rows, int inverse,
                       void *stream) {
    Context *c = nullptr;
    ABI_TRY
    c = ctx_of(ctx);
    if (num_rows == 0) return MMFHE_OK;
    check_ptr(rows, "rows");
    if (!prime_idx) throw Error(MMFHE_ERR_BAD_ARG, "null prime_idx");
    cudaStream_t st = (cudaStream_t)stream;
    const int np = c->num_q + c->num_p;
    for (size_t r = 0; r < num_rows; r++)
        if ((int)prime_idx[r] >= np) throw Error(MMFHE_ERR_BAD_ARG, "prime index out of range");
    Buf d(c->pool.get(), num_rows * c->n);
    CK(cudaMemcpyAsync(d.get(), rows, num_rows * c->n * 8, cudaMemcpyDefault, st));
    for (size_t r = 0; r < num_rows; r++) {
        RowsView v{d.get() + r * c->n, make_map(1, 1, {(int)prime_idx[r]}), 1};
        launch_ntt(*c, v, v, inverse != 0, st);
    }
    CK(cudaMemcpyAsync(rows, d.get(), num_rows * c->n * 8, cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    ABI_CATCH(c)
}

mmfhe_status mmfhe_ntt_batch(mmfhe_ctx *ctx, uint64_t *rows, size_t blocks, uint32_t limbs, int inverse,
                             void *stream) {
    Context *c = nullptr;
    ABI_TRY
    c = ctx_of(ctx);
    if (blocks == 0) return MMFHE_OK;
    if (!rows || is_host_ptr(rows) || ((uintptr_t)rows & 15)) throw Error(MMFHE_ERR_BAD_ARG, "rows must be 16-byte aligned device memory");
    if (limbs < 1 || (int)limbs > c->num_q) throw Error(MMFHE_ERR_BAD_ARG, "limbs must be 1..num_q");
    CK(cudaSetDevice(c->device));
    ntt_q_blocks(*c, rows, blocks, (int)limbs, inverse != 0, (cudaStream_t)stream);
    CK(cudaGetLastError());
    ABI_CATCH(c)
}

mmfhe_status mmfhe_poly_mul(mmfhe_ctx *ctx, uint64_t *out, const uint64_t *a, const uint64_t *b,
                            const uint32_t *prime_idx, size_t num_rows, void *stream) {
    Context *c = nullptr;
    ABI_TRY
    c = ctx_of(ctx);
    if (num_rows == 0) return MMFHE_OK;
    check_ptr(out, "out");
    check_ptr(a, "a");
    check_ptr(b, "b");
    if (!prime_idx) throw Error(MMFHE_ERR_BAD_ARG, "null prime_idx");
    if (num_rows > (size_t)MAXROWMAP) throw Error(MMFHE_ERR_BAD_ARG, "at most 64 rows per call");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> pids(num_rows);
    PidList pl{};
    for (size_t r = 0; r < num_rows; r++) {
        if ((int)prime_idx[r] >= c->num_q + c->num_p) throw Error(MMFHE_ERR_BAD_ARG, "prime index out of range");
        pids[r] = (int)prime_idx[r];
        pl.pid[r] = (uint8_t)prime_idx[r];
    }
    Buf da(c->pool.get(), num_rows * c->n), db(c->pool.get(), num_rows * c->n);
    CK(cudaMemcpyAsync(da.get(), a, num_rows * c->n * 8, cudaMemcpyDefault, st));
    CK(cudaMemcpyAsync(db.get(), b, num_rows * c->n * 8, cudaMemcpyDefault, st));
    RowsView va{da.get(), make_map((uint32_t)num_rows, (uint32_t)num_rows, pids), num_rows};
    RowsView vb{db.get(), make_map((uint32_t)num_rows, (uint32_t)num_rows, pids), num_rows};
    launch_ntt(*c, va, va, false, st);
    launch_ntt(*c, vb, vb, false, st);
    // point-wise product: b plays the plaintext covering all rows
    k_launch_mul_plain(*c, da.get(), da.get(), db.get(), num_rows, pl, (uint32_t)num_rows, false, st);
    launch_ntt(*c, va, va, true, st);
    CK(cudaMemcpyAsync(out, da.get(), num_rows * c->n * 8, cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    ABI_CATCH(c)
}

#define PRIM_SETUP(level_)                                  \
    c = ctx_of(ctx);                                        \
    check_level(*c, level_);                                \
    cudaStream_t st = (cudaStream_t)stream;                 \
    const size_t W = c->ct_words(level_);                   \
    (void)W;

mmfhe_status mmfhe_ct_add(mmfhe_ctx *ctx, uint64_t *out, const uint64_t *a, const uint64_t *b, size_t batch,
                          uint32_t level, void *stream) {
    Context *c = nullptr;
    ABI_TRY
    PRIM_SETUP(level)
    if (!batch) return MMFHE_OK;
    check_ptr(out, "out"); check_ptr(a, "a"); check_ptr(b, "b");
    CtB A = load_cts(*c, contiguous(a, batch, W).data(), 0, (int)batch, (int)level, 1.0, st);
    CtB Bc = load_cts(*c, contiguous(b, batch, W).data(), 0, (int)batch, (int)level, 1.0, st);
    ct_addsub(*c, A, A, Bc, false, st);
    store_cts(*c, A, contiguous_out(out, batch, W).data(), 0, st);
    CK(cudaStreamSynchronize(st));
    ABI_CATCH(c)
}

mmfhe_status mmfhe_ct_mul_plain(mmfhe_ctx *ctx, uint64_t *out, const uint64_t *ct, const uint64_t *pt, size_t batch,
                                uint32_t level, void *stream) {
    Context *c = nullptr;
    ABI_TRY
    PRIM_SETUP(level)
    if (!batch) return MMFHE_OK;
    check_ptr(out, "out"); check_ptr(ct, "ct"); check_ptr(pt, "pt");
    CtB A = load_cts(*c, contiguous(ct, batch, W).data(), 0, (int)batch, (int)level, 1.0, st);
    PtDev P = pt_new(*c, (int)level, 1.0);
    CK(cudaMemcpyAsync(P.buf.get(), pt, (size_t)(level + 1) * c->n * 8, cudaMemcpyDefault, st));
    ntt_q_blocks(*c, P.buf.get(), 1, (int)level + 1, false, st);
    ct_mul_plain(*c, A, A, P, false, st);
    store_cts(*c, A, contiguous_out(out, batch, W).data(), 0, st);
    CK(cudaStreamSynchronize(st));
    ABI_CATCH(c)
}

mmfhe_status mmfhe_ct_mul_relin(mmfhe_ctx *ctx, const mmfhe_keys *keys, uint64_t *out, const uint64_t *a,
                                const uint64_t *b, size_t batch, uint32_t level, void *stream) {
    Context *c = nullptr;
    ABI_TRY
    PRIM_SETUP(level)
    const Keys &K = keys_of(keys, c);
    if (!batch) return MMFHE_OK;
    check_ptr(out, "out"); check_ptr(a, "a"); check_ptr(b, "b");
    CtB A = load_cts(*c, contiguous(a, batch, W).data(), 0, (int)batch, (int)level, 1.0, st);
    CtB Bc = load_cts(*c, contiguous(b, batch, W).data(), 0, (int)batch, (int)level, 1.0, st);
    TensorB t = tensor_new(*c, (int)batch, (int)level);
    tensor_acc(*c, t, A, Bc, 1, true, st);
    CtB r = relin(*c, K, t, st);
    store_cts(*c, r, contiguous_out(out, batch, W).data(), 0, st);
    CK(cudaStreamSynchronize(st));
    ABI_CATCH(c)
}

mmfhe_status mmfhe_ct_rescale(mmfhe_ctx *ctx, uint64_t *out, const uint64_t *in, size_t batch, uint32_t level,
                              void *stream) {
    Context *c = nullptr;
    ABI_TRY
    PRIM_SETUP(level)
    if (level < 1) throw Error(MMFHE_ERR_LEVEL_MISMATCH, "rescale needs level >= 1");
    if (!batch) return MMFHE_OK;
    check_ptr(out, "out"); check_ptr(in, "in");
    CtB A = load_cts(*c, contiguous(in, batch, W).data(), 0, (int)batch, (int)level, 1.0, st);
    CtB r = rescale(*c, A, st);
    store_cts(*c, r, contiguous_out(out, batch, c->ct_words(level - 1)).data(), 0, st);
    CK(cudaStreamSynchronize(st));
    ABI_CATCH(c)
}

mmfhe_status mmfhe_ct_rotate_hoisted(mmfhe_ctx *ctx, const mmfhe_keys *keys, uint64_t *const *outs,
                                     const uint64_t *in, size_t batch, uint32_t level, const int32_t *ks,
                                     size_t num_k, void *stream) {
    Context *c = nullptr;
    ABI_TRY
    PRIM_SETUP(level)
    const Keys &K = keys_of(keys, c);
    if (!batch || !num_k) return MMFHE_OK;
    if (!outs || !ks) throw Error(MMFHE_ERR_BAD_ARG, "null outputs");
    check_ptr(in, "in");
    for (size_t i = 0; i < num_k; i++) check_ptr(outs[i], "out");
    CtB A = load_cts(*c, contiguous(in, batch, W).data(), 0, (int)batch, (int)level, 1.0, st);
    std::vector<CtB> r = rotate_hoisted(*c, K, A, std::vector<int32_t>(ks, ks + num_k), st);
    for (size_t i = 0; i < num_k; i++) store_cts(*c, r[i], contiguous_out(outs[i], batch, W).data(), 0, st);
    CK(cudaStreamSynchronize(st));
    ABI_CATCH(c)
}

mmfhe_status mmfhe_ct_rotate(mmfhe_ctx *ctx, const mmfhe_keys *keys, uint64_t *out, const uint64_t *in, size_t batch,
                             uint32_t level, int32_t k, void *stream) {
    uint64_t *outs[1] = {out};
    return mmfhe_ct_rotate_hoisted(ctx, keys, outs, in, batch, level, &k, 1, stream);
}

mmfhe_status mmfhe_modup(mmfhe_ctx *ctx, uint64_t *out, const uint64_t *d, size_t batch, uint32_t level, void *stream) {
    Context *c = nullptr;
    ABI_TRY
    PRIM_SETUP(level)
    if (!batch) return MMFHE_OK;
    check_ptr(out, "out"); check_ptr(d, "d");
    const int nl = (int)level + 1, nre = nl + c->num_p;
    Buf dd(c->pool.get(), batch * nl * c->n);
    CK(cudaMemcpyAsync(dd.get(), d, batch * nl * c->n * 8, cudaMemcpyDefault, st));
    ntt_q_blocks(*c, dd.get(), batch, nl, false, st);
    DigitsB dg = modup(*c, dd.get(), (size_t)nl, (int)batch, (int)level, st);
    digits_fill_own(*c, dg, st);
    std::vector<int> pids(nre);
    for (int t = 0; t < nre; t++) pids[t] = t <= (int)level ? t : c->num_q + (t - nl);
    RowsView v{dg.buf.get(), make_map(nre, nre, pids), batch * dg.beta * nre};
    launch_ntt(*c, v, v, true, st);
    CK(cudaMemcpyAsync(out, dg.buf.get(), batch * dg.beta * nre * c->n * 8, cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    ABI_CATCH(c)
}

mmfhe_status mmfhe_keyswitch(mmfhe_ctx *ctx, const mmfhe_keys *keys, int which, int32_t rotation, uint64_t *out,
                             const uint64_t *d, size_t batch, uint32_t level, void *stream) {
    Context *c = nullptr;
    ABI_TRY
    PRIM_SETUP(level)
    const Keys &K = keys_of(keys, c);
    if (!batch) return MMFHE_OK;
    check_ptr(out, "out"); check_ptr(d, "d");
    const int nl = (int)level + 1;
    const KeyPtrs key = which == 0 ? relin_key(K) : galois_key(K, norm_rot(*c, rotation));
    Buf dd(c->pool.get(), batch * nl * c->n);
    CK(cudaMemcpyAsync(dd.get(), d, batch * nl * c->n * 8, cudaMemcpyDefault, st));
    ntt_q_blocks(*c, dd.get(), batch, nl, false, st);
    DigitsB dg = modup(*c, dd.get(), (size_t)nl, (int)batch, (int)level, st);
    CtB r = keyswitch_moddown(*c, dg, key, 1, nullptr, nullptr, 0, 1.0, st);
    store_cts(*c, r, contiguous_out(out, batch, W).data(), 0, st);
    CK(cudaStreamSynchronize(st));
    ABI_CATCH(c)
}

mmfhe_status mmfhe_ct_rotsum(mmfhe_ctx *ctx, const mmfhe_keys *keys, uint64_t *out, const uint64_t *in, size_t batch,
                             uint32_t level, int32_t stride, uint32_t span, void *stream) {
    Context *c = nullptr;
    ABI_TRY
    PRIM_SETUP(level)
    const Keys &K = keys_of(keys, c);
    if (!batch) return MMFHE_OK;
    if (span == 0 || (span & (span - 1))) throw Error(MMFHE_ERR_BAD_ARG, "span must be a power of two");
    check_ptr(out, "out"); check_ptr(in, "in");
    CtB A = load_cts(*c, contiguous(in, batch, W).data(), 0, (int)batch, (int)level, 1.0, st);
    CtB r = rotsum(*c, K, A, stride, span, st);
    store_cts(*c, r, contiguous_out(out, batch, W).data(), 0, st);
    CK(cudaStreamSynchronize(st));
    ABI_CATCH(c)
}

mmfhe_status mmfhe_ct_bsgs(mmfhe_ctx *ctx, const mmfhe_keys *keys, uint64_t *out, const uint64_t *in, size_t batch,
                           uint32_t level, int32_t stride, uint32_t n1, const uint32_t *deltas,
                           const uint64_t *const *diags, size_t num_diags, void *stream) {
    Context *c = nullptr;
    ABI_TRY
    PRIM_SETUP(level)
    const Keys &K = keys_of(keys, c);
    if (!batch) return MMFHE_OK;
    if (!num_diags || !deltas || !diags || n1 == 0) throw Error(MMFHE_ERR_BAD_ARG, "no diagonals");
    check_ptr(out, "out"); check_ptr(in, "in");
    CtB A = load_cts(*c, contiguous(in, batch, W).data(), 0, (int)batch, (int)level, 1.0, st);
    std::vector<PtDev> pts(num_diags);
    std::set<int> need;
    for (size_t i = 0; i < num_diags; i++) {
        check_ptr(diags[i], "diagonal");
        pts[i] = pt_new(*c, (int)level, 1.0);
        CK(cudaMemcpyAsync(pts[i].buf.get(), diags[i], (size_t)(level + 1) * c->n * 8, cudaMemcpyDefault, st));
        ntt_q_blocks(*c, pts[i].buf.get(), 1, (int)level + 1, false, st);
        pt_to_mont(*c, pts[i], st);
        need.insert((int)(deltas[i] % n1));
    }
    BsgsTerm t;
    std::vector<int32_t> rr;
    for (int b : need) {
        t.baby_idx.push_back(b);
        rr.push_back(b * stride);
    }
    std::vector<CtB> babies = rotate_hoisted(*c, K, A, rr, st);
    t.baby = &babies;
    for (size_t i = 0; i < num_diags; i++) t.diags.push_back({(int)deltas[i], &pts[i]});
    CtB r = bsgs(*c, K, {t}, (int)n1, stride, st);
    store_cts(*c, r, contiguous_out(out, batch, W).data(), 0, st);
    CK(cudaStreamSynchronize(st));
    ABI_CATCH(c)
}

mmfhe_status mmfhe_ct_bsgs_dh(mmfhe_ctx *ctx, const mmfhe_keys *keys, uint64_t *out, const uint64_t *in, size_t batch,
                              uint32_t level, int32_t stride, uint32_t n1, uint32_t num_sets, const int32_t *offsets,
                              const uint32_t *set_of, const uint32_t *deltas, const uint64_t *const *diags,
                              size_t num_diags, void *stream) {
    Context *c = nullptr;
    ABI_TRY
    PRIM_SETUP(level)
    const Keys &K = keys_of(keys, c);
    if (!batch) return MMFHE_OK;
    if (!num_diags || !deltas || !diags || !set_of || n1 == 0) throw Error(MMFHE_ERR_BAD_ARG, "no diagonals");
    if (num_sets == 0 || num_sets > 64 || !offsets) throw Error(MMFHE_ERR_BAD_ARG, "1..64 baby sets");
    check_ptr(out, "out"); check_ptr(in, "in");
    CtB A = load_cts(*c, contiguous(in, batch, W).data(), 0, (int)batch, (int)level, 1.0, st);
    std::vector<PtDev> pts;
    pts.reserve(num_diags);
    std::vector<BsgsSet> sets(num_sets);
    for (uint32_t s = 0; s < num_sets; s++) {
        sets[s].x = &A;
        sets[s].offset = offsets[s];
    }
    for (size_t i = 0; i < num_diags; i++) {
        check_ptr(diags[i], "diagonal");
        if (set_of[i] >= num_sets) throw Error(MMFHE_ERR_BAD_ARG, "diagonal of an unknown baby set");
        pts.push_back(pt_qp_from_coeffs(*c, diags[i], (int)level, 1.0, st));
    }
    for (size_t i = 0; i < num_diags; i++) sets[set_of[i]].diags.push_back({(int)deltas[i], &pts[i]});
    CtB r = bsgs_dh(*c, K, sets, (int)n1, stride, st);
    store_cts(*c, r, contiguous_out(out, batch, W).data(), 0, st);
    CK(cudaStreamSynchronize(st));
    ABI_CATCH(c)
}

// ---- plans ----
mmfhe_status mmfhe_plan_create(mmfhe_ctx *ctx, const mmfhe_circuit_config *cfg, size_t cfg_size, mmfhe_plan **out) {
    Context *c = nullptr;
    ABI_TRY
    c = ctx_of(ctx);
    if (!cfg || !out || cfg_size != sizeof(mmfhe_circuit_config)) throw Error(MMFHE_ERR_BAD_ARG, "bad config struct");
    *out = new mmfhe_plan{create_plan(*c, *cfg)};
    ABI_CATCH(c)
}

mmfhe_status mmfhe_plan_destroy(mmfhe_plan *plan) {
    ABI_TRY
    if (!plan) return MMFHE_OK;
    if (plan->p) {
        CK(cudaSetDevice(plan->p->ctx->device));
        CK(cudaDeviceSynchronize());
    }
    delete plan->p;
    delete plan;
    ABI_CATCH(nullptr)
}

mmfhe_status mmfhe_plan_num_consts(const mmfhe_plan *plan, uint32_t *count) {
    if (!plan || !plan->p || !count) return fail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    *count = (uint32_t)plan->p->keys.size();
    return MMFHE_OK;
}

mmfhe_status mmfhe_plan_const_key(const mmfhe_plan *plan, uint32_t i, mmfhe_const_key *out) {
    if (!plan || !plan->p || !out) return fail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    if (i >= plan->p->keys.size()) return fail(plan->p->ctx, MMFHE_ERR_BAD_ARG, "constant index out of range");
    *out = plan->p->keys[i];
    return MMFHE_OK;
}

mmfhe_status mmfhe_plan_set_const(mmfhe_plan *plan, uint32_t i, const uint64_t *words) {
    Context *c = nullptr;
    ABI_TRY
    if (!plan || !plan->p) throw Error(MMFHE_ERR_BAD_ARG, "null plan");
    c = plan->p->ctx;
    CK(cudaSetDevice(c->device));
    check_ptr(words, "words");
    plan_set_const(*plan->p, i, words, 0);
    CK(cudaStreamSynchronize(0));
    ABI_CATCH(c)
}

mmfhe_status mmfhe_plan_get_const(const mmfhe_plan *plan, uint32_t i, uint64_t *words) {
    Context *c = nullptr;
    ABI_TRY
    if (!plan || !plan->p) throw Error(MMFHE_ERR_BAD_ARG, "null plan");
    c = plan->p->ctx;
    CK(cudaSetDevice(c->device));
    check_ptr(words, "words");
    if (i >= plan->p->keys.size()) throw Error(MMFHE_ERR_BAD_ARG, "constant index out of range");
    const PtDev &pt = plan->p->consts[i];
    if (!pt.buf.get()) throw Error(MMFHE_ERR_NOT_FOUND, "constant not set");
    const int nl = pt.level + 1;
    Buf tmp(c->pool.get(), (size_t)nl * c->n);
    std::vector<int> pids(nl);
    for (int k = 0; k < nl; k++) pids[k] = k;
    CK(cudaMemcpyAsync(tmp.get(), pt.buf.get(), (size_t)nl * c->n * 8, cudaMemcpyDeviceToDevice, 0));
    RowsView tv{tmp.get(), make_map(nl, nl, pids), (size_t)nl};
    if (pt.mont) k_launch_mont_convert(*c, tv, false, 0);
    launch_ntt(*c, tv, tv, true, 0);
    CK(cudaMemcpy(words, tmp.get(), (size_t)nl * c->n * 8, cudaMemcpyDefault));
    ABI_CATCH(c)
}

mmfhe_status mmfhe_plan_encode_consts(mmfhe_plan *plan) {
    Context *c = nullptr;
    ABI_TRY
    if (!plan || !plan->p) throw Error(MMFHE_ERR_BAD_ARG, "null plan");
    c = plan->p->ctx;
    CK(cudaSetDevice(c->device));
    plan_encode_consts(*plan->p, 0);
    ABI_CATCH(c)
}

mmfhe_status mmfhe_plan_num_scalars(const mmfhe_plan *plan, uint32_t *count) {
    if (!plan || !plan->p || !count) return fail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    *count = (uint32_t)plan->p->scalars.size();
    return MMFHE_OK;
}

mmfhe_status mmfhe_plan_get_scalars(const mmfhe_plan *plan, double *out, uint32_t capacity) {
    if (!plan || !plan->p || !out) return fail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    const auto &v = plan->p->scalars;
    if (capacity < v.size()) return fail(plan->p->ctx, MMFHE_ERR_BAD_ARG, "capacity too small");
    std::copy(v.begin(), v.end(), out);
    return MMFHE_OK;
}

mmfhe_status mmfhe_plan_set_scalars(mmfhe_plan *plan, const double *values, uint32_t count) {
    Context *c = nullptr;
    ABI_TRY
    if (!plan || !plan->p || !values) throw Error(MMFHE_ERR_BAD_ARG, "null argument");
    c = plan->p->ctx;
    plan_set_scalars(*plan->p, values, count);
    ABI_CATCH(c)
}

mmfhe_status mmfhe_plan_set_fc_layer(mmfhe_plan *plan, uint32_t layer, const double *W) {
    Context *c = nullptr;
    ABI_TRY
    if (!plan || !plan->p || !W) throw Error(MMFHE_ERR_BAD_ARG, "null argument");
    c = plan->p->ctx;
    CK(cudaSetDevice(c->device));
    plan_set_fc_layer(*plan->p, layer, W);
    ABI_CATCH(c)
}

mmfhe_status mmfhe_plan_rotations(const mmfhe_plan *plan, int32_t *out, uint32_t capacity, uint32_t *count) {
    if (!plan || !plan->p || !count) return fail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    const auto &r = plan->p->rotations;
    *count = (uint32_t)r.size();
    if (out) {
        if (capacity < r.size()) return fail(plan->p->ctx, MMFHE_ERR_BAD_ARG, "capacity too small");
        std::copy(r.begin(), r.end(), out);
    }
    return MMFHE_OK;
}

mmfhe_status mmfhe_plan_io(const mmfhe_plan *plan, uint32_t *n_in, uint32_t *n_out, uint32_t *out_levels) {
    if (!plan || !plan->p || !n_in || !n_out) return fail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    *n_in = (uint32_t)plan->p->n_in;
    *n_out = (uint32_t)plan->p->out_levels.size();
    if (out_levels) {
        if (plan->p->out_levels.size() > 16) return fail(plan->p->ctx, MMFHE_ERR_BAD_ARG, "more than 16 outputs");
        for (size_t i = 0; i < plan->p->out_levels.size(); i++) out_levels[i] = (uint32_t)plan->p->out_levels[i];
    }
    return MMFHE_OK;
}

mmfhe_status mmfhe_plan_readout(const mmfhe_plan *plan, uint32_t *out_index, uint32_t *slot, uint32_t capacity,
                                uint32_t *count) {
    if (!plan || !plan->p || !count) return fail(nullptr, MMFHE_ERR_BAD_ARG, "null argument");
    const Plan &p = *plan->p;
    if (p.cfg.kind != MMFHE_CIRCUIT_VITAL) {
        *count = 0;
        return MMFHE_OK;
    }
    const uint32_t rc = (uint32_t)p.r_c;
    const uint32_t idx[6] = {0, 0, 1, 1, 2, 2};
    const uint32_t pos[6] = {0, rc, 0, (uint32_t)p.span[0] * rc, 1, (uint32_t)p.span[1] * rc + 1};
    *count = 6;
    if (capacity < 6 || !out_index || !slot) return fail(p.ctx, MMFHE_ERR_BAD_ARG, "readout needs room for 6 entries");
    for (int i = 0; i < 6; i++) {
        out_index[i] = idx[i];
        slot[i] = pos[i];
    }
    return MMFHE_OK;
}

mmfhe_status mmfhe_eval(mmfhe_ctx *ctx, const mmfhe_plan *plan, mmfhe_keys *const *keys,
                        const uint64_t *const *in_cts, size_t batch, uint64_t *const *out_cts, void *stream) {
    Context *c = nullptr;
    ABI_TRY
    c = ctx_of(ctx);
    if (!plan || !plan->p) throw Error(MMFHE_ERR_BAD_ARG, "null plan");
    if (plan->p->ctx != c) throw Error(MMFHE_ERR_PARAM_MISMATCH, "plan belongs to another context");
    if (batch == 0) return MMFHE_OK;
    if (!keys || !in_cts || !out_cts) throw Error(MMFHE_ERR_BAD_ARG, "null window arrays");
    std::vector<const Keys *> ks(batch);
    for (size_t w = 0; w < batch; w++) ks[w] = &keys_of(keys[w], c);
    eval_windows(*c, *plan->p, ks.data(), in_cts, batch, out_cts, (cudaStream_t)stream);
    ABI_CATCH(c)
}

mmfhe_status mmfhe_eval_vital(mmfhe_ctx *ctx, const mmfhe_plan *plan, mmfhe_keys *const *keys,
                              const uint64_t *const *in_cts, size_t batch, uint64_t *const *out_cts, void *stream) {
    if (!plan || !plan->p ||
        (plan->p->cfg.kind != MMFHE_CIRCUIT_VITAL && plan->p->cfg.kind != MMFHE_CIRCUIT_VITAL_PER_FRAME))
        return fail(ctx ? ctx->c : nullptr, MMFHE_ERR_BAD_ARG, "plan is not a vital-sign circuit");
    return mmfhe_eval(ctx, plan, keys, in_cts, batch, out_cts, stream);
}

// ---- host helpers ----
mmfhe_status mmfhe_pack_window(uint32_t log_n, uint32_t frames, uint32_t bins, const double *values, double *out) {
    ABI_TRY
    if (!values || !out || log_n < 2 || log_n > 20 || frames == 0 || bins == 0) throw Error(MMFHE_ERR_BAD_ARG, "bad arguments");
    uint32_t n = 1u << (log_n - 1), fp = 1;
    while (fp < frames) fp <<= 1;
    if (fp > n) throw Error(MMFHE_ERR_BAD_ARG, "window longer than the slot count");
    uint32_t rc = n / fp, G = (bins + rc - 1) / rc;
    memset(out, 0, sizeof(double) * (size_t)G * n);
    for (uint32_t t = 0; t < frames; t++)
        for (uint32_t r = 0; r < bins; r++) out[(size_t)(r / rc) * n + t * rc + (r % rc)] = values[(size_t)t * bins + r];
    ABI_CATCH(nullptr)
}

mmfhe_status mmfhe_encode(const mmfhe_params *params, const double *slots, double scale, uint32_t level, uint64_t *out) {
    ABI_TRY
    if (!params || !slots || !out || level >= params->num_q || params->log_n < 10 || params->log_n > 16)
        throw Error(MMFHE_ERR_BAD_ARG, "bad arguments");
    encode_slots(*params, slots, scale, (int)level, out);
    ABI_CATCH(nullptr)
}

}  // extern "C"
