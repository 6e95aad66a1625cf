// Context creation: parameter validation, prime selection, NTT twiddle
// tables and the per-level basis-conversion / rescale constants.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <set>

#include "hostmath.h"
#include "internal.h"
#include "kernels.h"

namespace mmfhe {

void cuda_check(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        if (e == cudaErrorMemoryAllocation) throw Error(MMFHE_ERR_OUT_OF_MEMORY, std::string(what) + ": out of device memory");
        throw Error(MMFHE_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

// ---------------------------------------------------------------------------
// pool
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// library-wide device memory accounting and the allocation-failure hook
// ---------------------------------------------------------------------------
namespace {
constexpr int kMaxTrackedDevices = 64;
std::atomic<uint64_t> g_dev_bytes[kMaxTrackedDevices];
std::atomic<uint64_t> g_dev_peak[kMaxTrackedDevices];
std::atomic<uint64_t> g_dev_allocs[kMaxTrackedDevices];
std::atomic<int64_t> g_fail_after{-1};

int tracked(int device) { return device >= 0 && device < kMaxTrackedDevices ? device : kMaxTrackedDevices - 1; }
}  // namespace

void *dev_alloc(int device, size_t bytes) {
    int64_t f = g_fail_after.load();
    while (f > 0 && !g_fail_after.compare_exchange_weak(f, f - 1)) {
    }
    if (f == 0) throw Error(MMFHE_ERR_OUT_OF_MEMORY, "injected allocation failure (" + std::to_string(bytes) + " bytes)");
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const int d = tracked(device);
    uint64_t now = g_dev_bytes[d].fetch_add(bytes) + bytes;
    uint64_t pk = g_dev_peak[d].load();
    while (now > pk && !g_dev_peak[d].compare_exchange_weak(pk, now)) {
    }
    g_dev_allocs[d].fetch_add(1);
    return p;
}

void dev_free(int device, void *p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    g_dev_bytes[tracked(device)].fetch_sub(bytes);
}

void mem_stats(int device, uint64_t *bytes, uint64_t *peak, uint64_t *allocs) {
    const int d = tracked(device);
    *bytes = g_dev_bytes[d].load();
    *peak = g_dev_peak[d].load();
    *allocs = g_dev_allocs[d].load();
}

void mem_peak_reset(int device) {
    const int d = tracked(device);
    g_dev_peak[d].store(g_dev_bytes[d].load());
}

void set_fail_after(int64_t n) { g_fail_after.store(n < 0 ? -1 : n); }

// ---------------------------------------------------------------------------
// pool
// ---------------------------------------------------------------------------
Pool::~Pool() { trim(); }

uint64_t *Pool::get(size_t words) {
    auto it = free_.find(words);
    if (it != free_.end()) {
        uint64_t *p = it->second;
        free_.erase(it);
        free_bytes_ -= words * 8;
        return p;
    }
    void *p = dev_alloc(device_, words * sizeof(uint64_t));
    if (!p) {
        cudaDeviceSynchronize();
        trim();   // release cached blocks and retry once
        p = dev_alloc(device_, words * sizeof(uint64_t));
        if (!p) throw Error(MMFHE_ERR_OUT_OF_MEMORY, "device allocation of " + std::to_string(words * 8) + " bytes failed");
    }
    held_ += words * 8;
    return (uint64_t *)p;
}

void Pool::put(uint64_t *p, size_t words) {
    free_.emplace(words, p);
    free_bytes_ += words * 8;
}

void Pool::trim() {
    for (auto &kv : free_) {
        dev_free(device_, kv.second, kv.first * 8);
        held_ -= kv.first * 8;
    }
    free_.clear();
    free_bytes_ = 0;
}

// ---------------------------------------------------------------------------
// parameters
// ---------------------------------------------------------------------------
static void select_primes(uint32_t log_n, uint32_t num_q, uint32_t q0_bits, uint32_t q_bits, uint32_t num_p,
                          uint32_t p_bits, std::vector<uint64_t> &qs, std::vector<uint64_t> &ps) {
    const uint64_t m = 2ull << log_n;
    std::set<uint64_t> used;
    auto below = [&](uint32_t bits) {
        uint64_t lim = 1ull << bits;
        uint64_t c = (lim - 1) / m * m + 1;
        if (c >= lim) c -= m;
        for (; c > m; c -= m)
            if (!used.count(c) && hm::is_prime(c)) return c;
        throw Error(MMFHE_ERR_BAD_ARG, "no prime below 2^bits");
    };
    auto above = [&](uint32_t bits) {
        uint64_t lim = 1ull << bits;
        uint64_t c = lim / m * m + 1;
        if (c <= lim) c += m;
        for (;; c += m)
            if (!used.count(c) && hm::is_prime(c)) return c;
    };
    qs.clear();
    ps.clear();
    uint64_t q0 = below(q0_bits);
    used.insert(q0);
    qs.push_back(q0);
    for (uint32_t i = 1; i < num_q; i++) {
        uint64_t p = (i % 2 == 1) ? below(q_bits) : above(q_bits);
        used.insert(p);
        qs.push_back(p);
    }
    for (uint32_t k = 0; k < num_p; k++) {
        uint64_t p = below(p_bits);
        used.insert(p);
        ps.push_back(p);
    }
}

mmfhe_status params_select(uint32_t log_n, uint32_t num_q, uint32_t q0_bits, uint32_t q_bits, uint32_t num_p,
                           uint32_t p_bits, uint32_t dnum, mmfhe_params *out) {
    if (!out || log_n < 10 || log_n > 16 || num_q < 1 || num_q > MMFHE_MAX_Q || num_p < 1 || num_p > MMFHE_MAX_P ||
        dnum < 1 || dnum > num_q || q0_bits < 21 || q0_bits > 61 || q_bits < 21 || q_bits > 60 || p_bits < 21 ||
        p_bits > 61)
        throw Error(MMFHE_ERR_BAD_ARG, "parameter out of range");
    std::vector<uint64_t> qs, ps;
    select_primes(log_n, num_q, q0_bits, q_bits, num_p, p_bits, qs, ps);
    memset(out, 0, sizeof *out);
    out->log_n = log_n;
    out->num_q = num_q;
    out->num_p = num_p;
    out->dnum = dnum;
    for (uint32_t i = 0; i < num_q; i++) out->q[i] = qs[i];
    for (uint32_t k = 0; k < num_p; k++) out->p[k] = ps[k];
    return MMFHE_OK;
}

static void validate(const mmfhe_params &p) {
    if (p.log_n < 10 || p.log_n > 16 || p.num_q < 1 || p.num_q > MMFHE_MAX_Q || p.num_p < 1 ||
        p.num_p > MMFHE_MAX_P || p.dnum < 1 || p.dnum > p.num_q || p.dnum > (uint32_t)MAX_DNUM)
        throw Error(MMFHE_ERR_BAD_BLOB, "parameter set out of range");
    uint32_t alpha = (p.num_q + p.dnum - 1) / p.dnum;
    if (alpha > p.num_p || alpha > (uint32_t)MAX_ALPHA) throw Error(MMFHE_ERR_BAD_BLOB, "digit size alpha exceeds K");
    if (p.num_q + p.num_p > (uint32_t)MAXPRIMES) throw Error(MMFHE_ERR_BAD_BLOB, "too many primes");
    std::set<uint64_t> seen;
    const uint64_t m = 2ull << p.log_n;
    auto chk = [&](uint64_t q) {
        if (q < (1ull << 20) || q >= (1ull << 61) || q % m != 1 || !hm::is_prime(q) || seen.count(q))
            throw Error(MMFHE_ERR_BAD_BLOB, "invalid prime " + std::to_string(q));
        seen.insert(q);
    };
    for (uint32_t i = 0; i < p.num_q; i++) chk(p.q[i]);
    for (uint32_t k = 0; k < p.num_p; k++) chk(p.p[k]);
}

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
static uint64_t *upload(Context &c, const std::vector<uint64_t> &h) {
    const size_t bytes = std::max<size_t>(8, h.size() * 8);
    void *p = dev_alloc(c.device, bytes);
    if (!p) throw Error(MMFHE_ERR_OUT_OF_MEMORY, "device allocation of context tables failed");
    c.owned.push_back({p, bytes});
    if (!h.empty()) CK(cudaMemcpy(p, h.data(), h.size() * 8, cudaMemcpyHostToDevice));
    return (uint64_t *)p;
}

static void build_level_consts(Context &c) {
    const int K = c.num_p;
    c.lv.assign(c.L + 1, LevelConsts{});
    for (int l = 0; l <= c.L; l++) {
        LevelConsts &lc = c.lv[l];
        lc.level = l;
        lc.digits.clear();
        for (int j = 0; j < c.dnum; j++) {
            std::vector<int> d;
            for (int i = j * c.alpha; i < std::min((j + 1) * c.alpha, l + 1); i++) d.push_back(i);
            if (!d.empty()) lc.digits.push_back(d);
        }
        lc.beta = (int)lc.digits.size();
        const int nre = l + 1 + K;
        std::vector<uint64_t> inv(MAX_DNUM * MAX_ALPHA, 0), inv_sh(MAX_DNUM * MAX_ALPHA, 0);
        std::vector<uint64_t> mm_(MAX_DNUM * MAX_ALPHA * MAXROWMAP, 0), mm_sh(MAX_DNUM * MAX_ALPHA * MAXROWMAP, 0);
        for (int j = 0; j < lc.beta; j++) {
            const auto &D = lc.digits[j];
            for (size_t u = 0; u < D.size(); u++) {
                uint64_t qi = c.primes[D[u]];
                uint64_t qhat_mod_qi = 1;
                for (size_t v = 0; v < D.size(); v++)
                    if (v != u) qhat_mod_qi = hm::mulmod(qhat_mod_qi, c.primes[D[v]] % qi, qi);
                uint64_t iv = hm::invmod(qhat_mod_qi, qi);
                inv[j * MAX_ALPHA + u] = iv;
                inv_sh[j * MAX_ALPHA + u] = hm::shoup(iv, qi);
                for (int t = 0; t < nre; t++) {
                    int pid = t <= l ? t : c.num_q + (t - l - 1);
                    uint64_t pt = c.primes[pid];
                    uint64_t v = 1;
                    for (size_t w = 0; w < D.size(); w++)
                        if (w != u) v = hm::mulmod(v, c.primes[D[w]] % pt, pt);
                    size_t ci = ((size_t)j * MAX_ALPHA + u) * MAXROWMAP + t;
                    mm_[ci] = v;
                    mm_sh[ci] = hm::shoup(v, pt);
                }
            }
        }
        // fused ModUp: Montgomery-form conversion factors; the inverse NTT's final
        // multiply by N^-1 (Qhat_{j,u})^-1 (q rows) or N^-1 Phat_k^-1 (p rows)
        std::vector<uint64_t> m_mont(mm_.size(), 0), ks(MAXPRIMES, 0), ks_sh(MAXPRIMES, 0);
        for (int j = 0; j < lc.beta; j++)
            for (size_t u = 0; u < lc.digits[j].size(); u++) {
                const int i = lc.digits[j][u];
                const uint64_t qi = c.primes[i];
                ks[i] = hm::mulmod(hm::invmod(c.n % qi, qi), inv[j * MAX_ALPHA + u], qi);
                ks_sh[i] = hm::shoup(ks[i], qi);
                for (int t = 0; t < nre; t++) {
                    const int pid = t <= l ? t : c.num_q + (t - l - 1);
                    const uint64_t pt = c.primes[pid];
                    const size_t ci = ((size_t)j * MAX_ALPHA + u) * MAXROWMAP + t;
                    m_mont[ci] = hm::mulmod(mm_[ci], c.mods.r64[pid], pt);
                }
            }
        for (int k = 0; k < K; k++) {
            const int pid = c.num_q + k;
            const uint64_t pk = c.primes[pid];
            uint64_t ph = 1;
            for (int m = 0; m < K; m++)
                if (m != k) ph = hm::mulmod(ph, c.primes[c.num_q + m] % pk, pk);
            ks[pid] = hm::mulmod(hm::invmod(c.n % pk, pk), hm::invmod(ph, pk), pk);
            ks_sh[pid] = hm::shoup(ks[pid], pk);
        }
        lc.d_up_mm = upload(c, m_mont);
        lc.d_ks_scale = upload(c, ks);
        lc.d_ks_scale_sh = upload(c, ks_sh);
        lc.d_up_inv = upload(c, inv);
        lc.d_up_inv_sh = upload(c, inv_sh);
        lc.d_up_m = upload(c, mm_);
        lc.d_up_m_sh = upload(c, mm_sh);
        std::vector<uint64_t> qinv(MMFHE_MAX_Q, 0), qinv_sh(MMFHE_MAX_Q, 0), qmod(MMFHE_MAX_Q, 0);
        if (l >= 1) {
            uint64_t ql = c.primes[l];
            for (int i = 0; i < l; i++) {
                uint64_t qi = c.primes[i];
                qmod[i] = ql % qi;
                qinv[i] = hm::invmod(ql % qi, qi);
                qinv_sh[i] = hm::shoup(qinv[i], qi);
            }
        }
        lc.d_rs_qinv = upload(c, qinv);
        lc.d_rs_qinv_sh = upload(c, qinv_sh);
        lc.d_rs_qmod = upload(c, qmod);
    }
    std::vector<uint64_t> pinv(MMFHE_MAX_P, 0), pinv_sh(MMFHE_MAX_P, 0);
    std::vector<uint64_t> phat(MMFHE_MAX_P * MMFHE_MAX_Q, 0), phat_sh(MMFHE_MAX_P * MMFHE_MAX_Q, 0);
    std::vector<uint64_t> pmod(MMFHE_MAX_Q, 0), pmod_sh(MMFHE_MAX_Q, 0), Pinv(MMFHE_MAX_Q, 0), Pinv_sh(MMFHE_MAX_Q, 0);
    for (int k = 0; k < K; k++) {
        uint64_t pk = c.primes[c.num_q + k];
        uint64_t ph = 1;
        for (int m = 0; m < K; m++)
            if (m != k) ph = hm::mulmod(ph, c.primes[c.num_q + m] % pk, pk);
        pinv[k] = hm::invmod(ph, pk);
        pinv_sh[k] = hm::shoup(pinv[k], pk);
        for (int i = 0; i < c.num_q; i++) {
            uint64_t qi = c.primes[i];
            uint64_t v = 1;
            for (int m = 0; m < K; m++)
                if (m != k) v = hm::mulmod(v, c.primes[c.num_q + m] % qi, qi);
            phat[k * MMFHE_MAX_Q + i] = v;
            phat_sh[k * MMFHE_MAX_Q + i] = hm::shoup(v, qi);
        }
    }
    for (int i = 0; i < c.num_q; i++) {
        uint64_t qi = c.primes[i];
        uint64_t P = 1;
        for (int m = 0; m < K; m++) P = hm::mulmod(P, c.primes[c.num_q + m] % qi, qi);
        pmod[i] = P;
        pmod_sh[i] = hm::shoup(P, qi);
        Pinv[i] = hm::invmod(P, qi);
        Pinv_sh[i] = hm::shoup(Pinv[i], qi);
    }
    std::vector<uint64_t> phat_mont(phat.size(), 0), negp_mont(MMFHE_MAX_Q, 0);
    for (int i = 0; i < c.num_q; i++) {
        const uint64_t qi = c.primes[i];
        for (int k = 0; k < K; k++)
            phat_mont[k * MMFHE_MAX_Q + i] = hm::mulmod(phat[k * MMFHE_MAX_Q + i], c.mods.r64[i], qi);
        negp_mont[i] = hm::mulmod((qi - pmod[i]) % qi, c.mods.r64[i], qi);
    }
    c.d_dn_phat_mont = upload(c, phat_mont);
    c.d_dn_negp_mont = upload(c, negp_mont);
    c.d_dn_pinv = upload(c, pinv);
    c.d_dn_pinv_sh = upload(c, pinv_sh);
    c.d_dn_phat = upload(c, phat);
    c.d_dn_phat_sh = upload(c, phat_sh);
    c.d_dn_pmod = upload(c, pmod);
    c.d_dn_pmod_sh = upload(c, pmod_sh);
    c.d_dn_Pinv = upload(c, Pinv);
    c.d_dn_Pinv_sh = upload(c, Pinv_sh);
}

void destroy_context(Context *c);

Context *create_context(const mmfhe_params &p, int device) {
    validate(p);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        throw Error(MMFHE_ERR_CUDA, "no CUDA device available");
    }
    if (device < 0 || device >= ndev) throw Error(MMFHE_ERR_BAD_ARG, "device index out of range");
    CK(cudaSetDevice(device));
    Context *c = new Context();
    try {
        c->device = device;
        CK(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
        c->params = p;
        c->logn = (int)p.log_n;
        c->n = 1u << p.log_n;
        c->num_q = (int)p.num_q;
        c->num_p = (int)p.num_p;
        c->dnum = (int)p.dnum;
        c->alpha = (c->num_q + c->dnum - 1) / c->dnum;
        c->L = c->num_q - 1;
        c->primes.assign(p.q, p.q + p.num_q);
        c->primes.insert(c->primes.end(), p.p, p.p + p.num_p);
        const int np = (int)c->primes.size();
        memset(&c->mods, 0, sizeof c->mods);
        for (int i = 0; i < np; i++) {
            c->mods.q[i] = c->primes[i];
            c->mods.mu[i] = hm::barrett_mu(c->primes[i]);
            c->mods.k[i] = hm::bitlen(c->primes[i]);
            uint64_t inv = 1;
            for (int it = 0; it < 7; it++) inv *= 2 - c->primes[i] * inv;   // Newton: q^-1 mod 2^64
            c->mods.qinv[i] = inv;
            c->mods.r64[i] = (uint64_t)(((hm::u128)1 << 64) % c->primes[i]);
        }
        uint64_t qmax = 0;
        for (int i = 0; i < c->num_q; i++) qmax = std::max(qmax, c->primes[i]);
        c->sum_terms_max = (int)std::min<uint64_t>(16, (~0ull) / qmax);
        for (int i = c->num_q; i < np; i++) qmax = std::max(qmax, c->primes[i]);
        c->sum_terms_max_qp = (int)std::min<uint64_t>(16, (~0ull) / qmax);
        // twiddles: fw[i] = psi^brv(i), iw[i] = psi^-brv(i)
        const uint32_t n = c->n;
        std::vector<uint64_t> tw(4ull * np * n), ninv(2ull * np);
        for (int id = 0; id < np; id++) {
            uint64_t q = c->primes[id];
            uint64_t psi = hm::primitive_root_2n(q, n);
            uint64_t ipsi = hm::invmod(psi, q);
            std::vector<uint64_t> pw(n), ipw(n);
            pw[0] = ipw[0] = 1;
            for (uint32_t i = 1; i < n; i++) {
                pw[i] = hm::mulmod(pw[i - 1], psi, q);
                ipw[i] = hm::mulmod(ipw[i - 1], ipsi, q);
            }
            uint64_t *fw = &tw[(0ull * np + id) * n], *fws = &tw[(1ull * np + id) * n];
            uint64_t *iw = &tw[(2ull * np + id) * n], *iws = &tw[(3ull * np + id) * n];
            for (uint32_t i = 0; i < n; i++) {
                uint32_t r = hm::bitrev(i, c->logn);
                fw[i] = pw[r];
                fws[i] = hm::shoup(fw[i], q);
                iw[i] = ipw[r];
                iws[i] = hm::shoup(iw[i], q);
            }
            ninv[id] = hm::invmod(n % q, q);
            ninv[np + id] = hm::shoup(ninv[id], q);
        }
        c->d_tw = upload(*c, tw);
        c->d_ninv = upload(*c, ninv);
        c->tw.fw = c->d_tw;
        c->tw.fw_sh = c->d_tw + 1ull * np * n;
        c->tw.iw = c->d_tw + 2ull * np * n;
        c->tw.iw_sh = c->d_tw + 3ull * np * n;
        c->tw.ninv = c->d_ninv;
        c->tw.ninv_sh = c->d_ninv + np;
        build_level_consts(*c);
        c->pool.reset(new Pool(device));
        CK(cudaDeviceSynchronize());
    } catch (...) {
        destroy_context(c);
        throw;
    }
    return c;
}

void destroy_context(Context *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    c->pool.reset();
    for (auto &o : c->owned) dev_free(c->device, o.first, o.second);
    for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
    delete c;
}

ModUpConsts modup_consts(const Context &c, int level) {
    const LevelConsts &lc = c.lv[level];
    return ModUpConsts{lc.d_up_inv, lc.d_up_inv_sh, lc.d_up_m, lc.d_up_m_sh, c.num_q};
}

ModDownConsts moddown_consts(const Context &c) {
    return ModDownConsts{c.d_dn_pinv, c.d_dn_pinv_sh, c.d_dn_phat, c.d_dn_phat_sh,
                         c.d_dn_pmod, c.d_dn_pmod_sh, c.d_dn_Pinv, c.d_dn_Pinv_sh, c.num_q};
}

RescaleConsts rescale_consts(const Context &c, int level) {
    const LevelConsts &lc = c.lv[level];
    return RescaleConsts{lc.d_rs_qinv, lc.d_rs_qinv_sh, lc.d_rs_qmod};
}

}  // namespace mmfhe
