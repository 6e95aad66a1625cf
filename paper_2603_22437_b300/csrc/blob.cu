// Serialized evaluation keys and plans, the per-ciphertext header, and the
// header-checked evaluation entry point.
//
// The paper's cloud receives the client's ciphertexts and its public
// evaluation keys (rlk and one Galois key per rotation) and never sees the
// secret key (Sec. "System Design", threat model).  What crosses that trust
// boundary is checked here before any of it reaches the GPU: blobs carry the
// fingerprint of the parameter set they were made for, their sizes, a
// checksum, and residues that must lie below their primes; every ciphertext
// carries its level, scale and parameter fingerprint.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "circuits.h"
#include "engine.h"
#include "handles.h"
#include "internal.h"

using namespace mmfhe;

namespace {

constexpr uint64_t kBlobMagic = 0x424C424548464D4Dull;   // bytes "MMFHEBLB"
constexpr uint32_t kBlobVersion = 1;
constexpr uint64_t kFnvOffset = 0xcbf29ce484222325ull;
constexpr uint64_t kFnvPrime = 0x100000001b3ull;
constexpr size_t kHeaderWords = 4;   // magic, version|kind, params hash, body words

mmfhe_status bfail(Context *c, mmfhe_status code, const std::string &msg) {
    set_thread_error(msg);
    if (c) c->last_error = msg;
    return code;
}

#define BLOB_TRY try {
#define BLOB_CATCH(ctxptr)                                                             \
    }                                                                                  \
    catch (const Error &e) { return bfail(ctxptr, e.code, e.what()); }                 \
    catch (const std::bad_alloc &) { return bfail(ctxptr, MMFHE_ERR_OUT_OF_MEMORY, "host allocation failed"); } \
    catch (const std::exception &e) { return bfail(ctxptr, MMFHE_ERR_CUDA, e.what()); } \
    catch (...) { return bfail(ctxptr, MMFHE_ERR_CUDA, "unknown error"); }            \
    return MMFHE_OK;

// Word-wise FNV-1a: h = (h xor w) * 0x100000001b3 over 64-bit words, from the
// FNV-1a offset basis.
uint64_t fnv_words(const uint64_t *w, size_t n, uint64_t h = kFnvOffset) {
    for (size_t i = 0; i < n; i++) h = (h ^ w[i]) * kFnvPrime;
    return h;
}

uint64_t params_hash(const mmfhe_params &p) {
    std::vector<uint64_t> w = {p.log_n, p.num_q, p.num_p, p.dnum};
    for (uint32_t i = 0; i < p.num_q && i < MMFHE_MAX_Q; i++) w.push_back(p.q[i]);
    for (uint32_t k = 0; k < p.num_p && k < MMFHE_MAX_P; k++) w.push_back(p.p[k]);
    return fnv_words(w.data(), w.size());
}

void check_params_shape(const mmfhe_params &p) {
    if (p.log_n < 10 || p.log_n > 16 || p.num_q < 1 || p.num_q > MMFHE_MAX_Q || p.num_p < 1 ||
        p.num_p > MMFHE_MAX_P || p.dnum < 1 || p.dnum > p.num_q)
        throw Error(MMFHE_ERR_BAD_ARG, "parameter set out of range");
}

size_t key_words(const mmfhe_params &p) { return (size_t)p.dnum * 2 * (p.num_q + p.num_p) << p.log_n; }

// Every residue of a switching key ([dnum][2][L+1+K][N]) below its prime.
void check_key_residues(const mmfhe_params &p, const uint64_t *w, const char *what) {
    const size_t N = 1ull << p.log_n, rows = p.num_q + p.num_p;
    for (size_t blk = 0; blk < (size_t)p.dnum * 2; blk++)
        for (size_t r = 0; r < rows; r++) {
            const uint64_t q = r < p.num_q ? p.q[r] : p.p[r - p.num_q];
            const uint64_t *row = w + (blk * rows + r) * N;
            for (size_t i = 0; i < N; i++)
                if (row[i] >= q)
                    throw Error(MMFHE_ERR_BAD_BLOB, std::string(what) + ": residue not below its prime (row " +
                                                        std::to_string(r) + ")");
        }
}

// Every residue of a polynomial at `level` ([level+1][N]) below its prime.
void check_poly_residues(const mmfhe_params &p, const uint64_t *w, uint32_t level, const char *what) {
    const size_t N = 1ull << p.log_n;
    for (uint32_t r = 0; r <= level; r++)
        for (size_t i = 0; i < N; i++)
            if (w[r * N + i] >= p.q[r])
                throw Error(MMFHE_ERR_BAD_BLOB, std::string(what) + ": residue not below its prime (row " +
                                                    std::to_string(r) + ")");
}

// A parsed blob: header fields and the body's words (pointers into the blob).
struct BlobView {
    uint32_t kind = 0;
    uint64_t hash = 0;
    const uint64_t *body = nullptr;
    size_t body_words = 0;
};

// Header, size and checksum of a blob; the body is parsed by the caller.
BlobView parse_blob(const void *blob, size_t size) {
    if (!blob) throw Error(MMFHE_ERR_BAD_ARG, "null blob");
    if ((uintptr_t)blob & 7) throw Error(MMFHE_ERR_BAD_ARG, "blob not 8-byte aligned");
    if (!is_host_ptr(blob)) throw Error(MMFHE_ERR_BAD_ARG, "blobs are read from host memory");
    if (size % 8 || size < (kHeaderWords + 1) * 8) throw Error(MMFHE_ERR_BAD_BLOB, "blob truncated or misaligned");
    const uint64_t *w = (const uint64_t *)blob;
    if (w[0] != kBlobMagic) throw Error(MMFHE_ERR_BAD_BLOB, "not an mmfhe blob");
    if ((uint32_t)w[1] != kBlobVersion) throw Error(MMFHE_ERR_BAD_BLOB, "unsupported blob version");
    BlobView v;
    v.kind = (uint32_t)(w[1] >> 32);
    v.hash = w[2];
    v.body_words = (size_t)w[3];
    if (v.body_words != size / 8 - kHeaderWords - 1) throw Error(MMFHE_ERR_BAD_BLOB, "blob size does not match its header");
    if (fnv_words(w, kHeaderWords + v.body_words) != w[kHeaderWords + v.body_words])
        throw Error(MMFHE_ERR_BAD_BLOB, "blob checksum mismatch");
    v.body = w + kHeaderWords;
    return v;
}

// Body of an evaluation-key blob: count, words per key, ids[count], keys.
struct KeysBody {
    size_t count = 0;
    const int64_t *ids = nullptr;
    const uint64_t *words = nullptr;
};

KeysBody parse_keys(const mmfhe_params &p, const BlobView &v) {
    if (v.kind != MMFHE_BLOB_KEYS) throw Error(MMFHE_ERR_BAD_BLOB, "not an evaluation-key blob");
    if (v.body_words < 2) throw Error(MMFHE_ERR_BAD_BLOB, "key blob truncated");
    KeysBody k;
    k.count = (size_t)v.body[0];
    if (v.body[1] != key_words(p)) throw Error(MMFHE_ERR_BAD_BLOB, "key size does not match the parameter set");
    if (k.count == 0 || k.count > 4096) throw Error(MMFHE_ERR_BAD_BLOB, "bad key count");
    if (v.body_words != 2 + k.count + k.count * key_words(p)) throw Error(MMFHE_ERR_BAD_BLOB, "key blob truncated");
    k.ids = (const int64_t *)(v.body + 2);
    k.words = v.body + 2 + k.count;
    const int64_t slots = 1ll << (p.log_n - 1);
    for (size_t i = 0; i < k.count; i++) {
        const int64_t id = k.ids[i];
        const bool ok = i == 0 ? id == 0 : (id == (int64_t)MMFHE_ROT_CONJ || (id > 0 && id < slots));
        if (!ok) throw Error(MMFHE_ERR_BAD_BLOB, "bad key id (the relinearization key first, then rotations in [1, N/2))");
    }
    for (size_t i = 0; i < k.count; i++) check_key_residues(p, k.words + i * key_words(p), "key blob");
    return k;
}

// Body of a plan blob: config bytes, count, levels[count], constants.
struct PlanBody {
    mmfhe_circuit_config cfg{};
    size_t count = 0;
    const uint64_t *levels = nullptr;
    const uint64_t *words = nullptr;
};

constexpr size_t kCfgWords = (sizeof(mmfhe_circuit_config) + 7) / 8;

PlanBody parse_plan(const mmfhe_params &p, const BlobView &v) {
    if (v.kind != MMFHE_BLOB_PLAN) throw Error(MMFHE_ERR_BAD_BLOB, "not a plan blob");
    if (v.body_words < 2 + kCfgWords) throw Error(MMFHE_ERR_BAD_BLOB, "plan blob truncated");
    if (v.body[0] != sizeof(mmfhe_circuit_config)) throw Error(MMFHE_ERR_BAD_BLOB, "circuit configuration of another size");
    PlanBody b;
    memcpy(&b.cfg, v.body + 1, sizeof(mmfhe_circuit_config));
    b.count = (size_t)v.body[1 + kCfgWords];
    if (b.count > (1u << 20)) throw Error(MMFHE_ERR_BAD_BLOB, "bad constant count");
    const size_t head = 2 + kCfgWords + b.count;
    if (v.body_words < head) throw Error(MMFHE_ERR_BAD_BLOB, "plan blob truncated");
    b.levels = v.body + 2 + kCfgWords;
    const size_t N = 1ull << p.log_n;
    size_t total = 0;
    for (size_t i = 0; i < b.count; i++) {
        if (b.levels[i] >= p.num_q) throw Error(MMFHE_ERR_BAD_BLOB, "constant level above the top level");
        total += (size_t)(b.levels[i] + 1) * N;
    }
    if (v.body_words != head + total) throw Error(MMFHE_ERR_BAD_BLOB, "plan blob truncated");
    b.words = v.body + head;
    size_t off = 0;
    for (size_t i = 0; i < b.count; i++) {
        check_poly_residues(p, b.words + off, (uint32_t)b.levels[i], "plan blob");
        off += (size_t)(b.levels[i] + 1) * N;
    }
    return b;
}

// Write header + body + checksum into out (capacity bytes); *size gets the
// total.  out == nullptr: size only.
mmfhe_status finish_blob(uint32_t kind, uint64_t hash, const std::vector<std::pair<const uint64_t *, size_t>> &parts,
                         void *out, size_t capacity, size_t *size) {
    size_t body = 0;
    for (auto &pt : parts) body += pt.second;
    const size_t total = (kHeaderWords + body + 1) * 8;
    if (size) *size = total;
    if (!out) return MMFHE_OK;
    if (capacity < total) throw Error(MMFHE_ERR_BAD_ARG, "blob capacity too small");
    if ((uintptr_t)out & 7) throw Error(MMFHE_ERR_BAD_ARG, "blob buffer not 8-byte aligned");
    uint64_t *w = (uint64_t *)out;
    w[0] = kBlobMagic;
    w[1] = (uint64_t)kBlobVersion | ((uint64_t)kind << 32);
    w[2] = hash;
    w[3] = body;
    size_t off = kHeaderWords;
    for (auto &pt : parts) {
        memcpy(w + off, pt.first, pt.second * 8);
        off += pt.second;
    }
    w[off] = fnv_words(w, off);
    return MMFHE_OK;
}

Context *ctx_checked(mmfhe_ctx *ctx) {
    if (!ctx || !ctx->c) throw Error(MMFHE_ERR_BAD_ARG, "null context");
    CK(cudaSetDevice(ctx->c->device));
    return ctx->c;
}

}  // namespace

extern "C" {

mmfhe_status mmfhe_params_hash(const mmfhe_params *params, uint64_t *out) {
    BLOB_TRY
    if (!params || !out) throw Error(MMFHE_ERR_BAD_ARG, "null argument");
    check_params_shape(*params);
    *out = params_hash(*params);
    BLOB_CATCH(nullptr)
}

mmfhe_status mmfhe_ct_header_make(const mmfhe_params *params, uint32_t level, double scale, mmfhe_ct_header *out) {
    BLOB_TRY
    if (!params || !out) throw Error(MMFHE_ERR_BAD_ARG, "null argument");
    check_params_shape(*params);
    if (level >= params->num_q) throw Error(MMFHE_ERR_LEVEL_MISMATCH, "level above the top level");
    if (!(scale > 0) || !std::isfinite(scale)) throw Error(MMFHE_ERR_BAD_ARG, "scale must be positive");
    memset(out, 0, sizeof *out);
    out->magic = MMFHE_CT_MAGIC;
    out->version = 1;
    out->level = level;
    out->log2_scale = std::log2(scale);
    out->params_hash = params_hash(*params);
    BLOB_CATCH(nullptr)
}

mmfhe_status mmfhe_keys_blob_write(const mmfhe_params *params, const uint64_t *relin, uint32_t n_rot,
                                   const int32_t *rotations, const uint64_t *const *galois, void *out, size_t capacity,
                                   size_t *size) {
    BLOB_TRY
    if (!params || !relin || (n_rot && (!rotations || !galois))) throw Error(MMFHE_ERR_BAD_ARG, "null argument");
    check_params_shape(*params);
    const size_t kw = key_words(*params);
    const int64_t slots = 1ll << (params->log_n - 1);
    std::vector<uint64_t> head = {(uint64_t)(1 + n_rot), (uint64_t)kw};
    head.push_back(0);   // id of the relinearization key
    for (uint32_t i = 0; i < n_rot; i++) {
        int64_t r = rotations[i];
        if (r != (int64_t)MMFHE_ROT_CONJ) r = ((r % slots) + slots) % slots;
        if (r == 0) throw Error(MMFHE_ERR_BAD_ARG, "rotation by 0 needs no key");
        head.push_back((uint64_t)r);
        if (!galois[i]) throw Error(MMFHE_ERR_BAD_ARG, "null Galois key");
    }
    std::vector<std::pair<const uint64_t *, size_t>> parts = {{head.data(), head.size()}, {relin, kw}};
    for (uint32_t i = 0; i < n_rot; i++) parts.push_back({galois[i], kw});
    if (out) {
        check_key_residues(*params, relin, "relinearization key");
        for (uint32_t i = 0; i < n_rot; i++) check_key_residues(*params, galois[i], "Galois key");
    }
    finish_blob(MMFHE_BLOB_KEYS, params_hash(*params), parts, out, capacity, size);
    BLOB_CATCH(nullptr)
}

mmfhe_status mmfhe_plan_blob_write(const mmfhe_params *params, const mmfhe_circuit_config *cfg, size_t cfg_size,
                                   uint32_t count, const uint32_t *levels, const uint64_t *const *consts, void *out,
                                   size_t capacity, size_t *size) {
    BLOB_TRY
    if (!params || !cfg || (count && (!levels || !consts))) throw Error(MMFHE_ERR_BAD_ARG, "null argument");
    if (cfg_size != sizeof(mmfhe_circuit_config)) throw Error(MMFHE_ERR_BAD_ARG, "bad config struct");
    check_params_shape(*params);
    const size_t N = 1ull << params->log_n;
    std::vector<uint64_t> head(2 + kCfgWords + count, 0);
    head[0] = sizeof(mmfhe_circuit_config);
    memcpy(head.data() + 1, cfg, sizeof(mmfhe_circuit_config));
    head[1 + kCfgWords] = count;
    std::vector<std::pair<const uint64_t *, size_t>> parts;
    for (uint32_t i = 0; i < count; i++) {
        if (levels[i] >= params->num_q) throw Error(MMFHE_ERR_LEVEL_MISMATCH, "constant level above the top level");
        if (!consts[i]) throw Error(MMFHE_ERR_BAD_ARG, "null constant");
        head[2 + kCfgWords + i] = levels[i];
    }
    parts.push_back({head.data(), head.size()});
    for (uint32_t i = 0; i < count; i++) {
        if (out) check_poly_residues(*params, consts[i], levels[i], "constant");
        parts.push_back({consts[i], (size_t)(levels[i] + 1) * N});
    }
    finish_blob(MMFHE_BLOB_PLAN, params_hash(*params), parts, out, capacity, size);
    BLOB_CATCH(nullptr)
}

mmfhe_status mmfhe_blob_check(const mmfhe_params *params, const void *blob, size_t size, uint32_t *kind) {
    BLOB_TRY
    if (!params) throw Error(MMFHE_ERR_BAD_ARG, "null parameters");
    check_params_shape(*params);
    BlobView v = parse_blob(blob, size);
    if (v.hash != params_hash(*params)) throw Error(MMFHE_ERR_PARAM_MISMATCH, "blob made for another parameter set");
    if (v.kind == MMFHE_BLOB_KEYS)
        parse_keys(*params, v);
    else if (v.kind == MMFHE_BLOB_PLAN)
        parse_plan(*params, v);
    else
        throw Error(MMFHE_ERR_BAD_BLOB, "unknown blob kind");
    if (kind) *kind = v.kind;
    BLOB_CATCH(nullptr)
}

mmfhe_status mmfhe_keys_load(mmfhe_ctx *ctx, uint64_t user_id, const void *blob, size_t size, mmfhe_keys **out) {
    Context *c = nullptr;
    BLOB_TRY
    c = ctx_checked(ctx);
    if (!out) throw Error(MMFHE_ERR_BAD_ARG, "null output");
    BlobView v = parse_blob(blob, size);
    if (v.hash != params_hash(c->params)) throw Error(MMFHE_ERR_PARAM_MISMATCH, "key blob made for another parameter set");
    KeysBody kb = parse_keys(c->params, v);
    std::unique_ptr<mmfhe_keys> k(new mmfhe_keys());
    k->k.ctx = c;
    k->k.user = user_id;
    const size_t kw = key_words(c->params);
    k->k.rlk = load_key(*c, kb.words);
    for (size_t i = 1; i < kb.count; i++) {
        const int32_t r = norm_rot(*c, (int32_t)kb.ids[i]);
        if (k->k.gk.count(r)) throw Error(MMFHE_ERR_BAD_BLOB, "duplicate Galois key");
        k->k.gk[r] = load_key(*c, kb.words + i * kw);
    }
    *out = k.release();
    BLOB_CATCH(c)
}

mmfhe_status mmfhe_plan_load(mmfhe_ctx *ctx, const void *blob, size_t size, mmfhe_plan **out) {
    Context *c = nullptr;
    BLOB_TRY
    c = ctx_checked(ctx);
    if (!out) throw Error(MMFHE_ERR_BAD_ARG, "null output");
    BlobView v = parse_blob(blob, size);
    if (v.hash != params_hash(c->params)) throw Error(MMFHE_ERR_PARAM_MISMATCH, "plan blob made for another parameter set");
    PlanBody pb = parse_plan(c->params, v);
    std::unique_ptr<Plan> p;
    try {
        p.reset(create_plan(*c, pb.cfg));
    } catch (const Error &e) {
        if (e.code == MMFHE_ERR_BAD_ARG) throw Error(MMFHE_ERR_BAD_BLOB, std::string("plan blob configuration: ") + e.what());
        throw;
    }
    if (pb.count != p->keys.size()) throw Error(MMFHE_ERR_BAD_BLOB, "plan blob holds another number of constants");
    for (size_t i = 0; i < pb.count; i++)
        if (pb.levels[i] != p->keys[i].level) throw Error(MMFHE_ERR_BAD_BLOB, "plan blob constant at another level");
    size_t off = 0;
    for (size_t i = 0; i < pb.count; i++) {
        plan_set_const(*p, (uint32_t)i, pb.words + off, 0);
        off += (size_t)(pb.levels[i] + 1) * c->n;
    }
    CK(cudaStreamSynchronize(0));
    *out = new mmfhe_plan{p.release()};
    BLOB_CATCH(c)
}

mmfhe_status mmfhe_eval_checked(mmfhe_ctx *ctx, const mmfhe_plan *plan, mmfhe_keys *const *keys,
                                const mmfhe_ct_header *const *in_hdrs, const uint64_t *const *in_cts, size_t batch,
                                mmfhe_ct_header *const *out_hdrs, uint64_t *const *out_cts, void *stream) {
    Context *c = nullptr;
    BLOB_TRY
    c = ctx_checked(ctx);
    if (!plan || !plan->p) throw Error(MMFHE_ERR_BAD_ARG, "null plan");
    const Plan &p = *plan->p;
    if (p.ctx != c) throw Error(MMFHE_ERR_PARAM_MISMATCH, "plan belongs to another context");
    if (batch == 0) return MMFHE_OK;
    if (!keys || !in_hdrs || !in_cts || !out_hdrs || !out_cts) throw Error(MMFHE_ERR_BAD_ARG, "null window arrays");
    const uint64_t hash = params_hash(c->params);
    double log2_scale = 0.0;
    for (size_t w = 0; w < batch; w++) {
        if (!in_hdrs[w] || !out_hdrs[w]) throw Error(MMFHE_ERR_BAD_ARG, "null header array");
        for (int i = 0; i < p.n_in; i++) {
            const mmfhe_ct_header &h = in_hdrs[w][i];
            if (h.magic != MMFHE_CT_MAGIC || h.version != 1) throw Error(MMFHE_ERR_BAD_BLOB, "not an mmfhe ciphertext header");
            if (h.params_hash != hash) throw Error(MMFHE_ERR_PARAM_MISMATCH, "ciphertext made for another parameter set");
            if ((int)h.level != c->L)
                throw Error(MMFHE_ERR_LEVEL_MISMATCH, "window inputs must be at the top level " + std::to_string(c->L));
            if (!std::isfinite(h.log2_scale)) throw Error(MMFHE_ERR_BAD_BLOB, "ciphertext scale is not finite");
            if (w == 0 && i == 0) log2_scale = h.log2_scale;
            if (std::fabs(h.log2_scale - log2_scale) > 1e-9)
                throw Error(MMFHE_ERR_BAD_ARG, "inputs of one call must share one encryption scale");
        }
    }
    if (p.cfg.kind == MMFHE_CIRCUIT_GESTURE && p.cfg.input_scale > 0 &&
        std::fabs(std::log2(p.cfg.input_scale) - log2_scale) > 1e-9)
        throw Error(MMFHE_ERR_PARAM_MISMATCH, "inputs encrypted at another scale than the plan's input_scale");
    std::vector<const Keys *> ks(batch);
    for (size_t w = 0; w < batch; w++) {
        if (!keys[w]) throw Error(MMFHE_ERR_BAD_ARG, "null keys");
        if (keys[w]->k.ctx != c) throw Error(MMFHE_ERR_PARAM_MISMATCH, "keys belong to another context");
        ks[w] = &keys[w]->k;
    }
    std::vector<double> scales;
    eval_windows(*c, p, ks.data(), in_cts, batch, out_cts, (cudaStream_t)stream, false, std::exp2(log2_scale), &scales);
    for (size_t w = 0; w < batch; w++)
        for (size_t o = 0; o < p.out_levels.size(); o++) {
            mmfhe_ct_header &h = out_hdrs[w][o];
            memset(&h, 0, sizeof h);
            h.magic = MMFHE_CT_MAGIC;
            h.version = 1;
            h.level = (uint32_t)p.out_levels[o];
            h.log2_scale = o < scales.size() ? std::log2(scales[o]) : 0.0;
            h.params_hash = hash;
        }
    BLOB_CATCH(c)
}

}  // extern "C"
