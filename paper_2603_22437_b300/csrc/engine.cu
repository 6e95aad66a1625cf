// Homomorphic operations on device ciphertext batches (evaluation domain).
//
// Key switching is hybrid (dnum digits of alpha primes): ModUp of the digit
// (iNTT, FastBConv to the other Q_l * P primes, NTT), inner product with the
// switching key, ModDown (iNTT of the P rows, centered FastBConv P -> Q, NTT,
// subtract and multiply by P^-1).  A rotation is the hoisted schedule of a
// one-element set: the Galois automorphism is applied to the ModUp digits
// inside the key inner product and to c0 inside the ModDown combine.
#include <algorithm>
#include <cmath>
#include <map>
#include <set>

#include "engine.h"
#include "hostmath.h"

namespace mmfhe {

PidList pids_q(int nl) {
    PidList p{};
    for (int i = 0; i < nl && i < MAXROWMAP; i++) p.pid[i] = (uint8_t)i;
    return p;
}

int32_t norm_rot(const Context &c, int32_t k) {
    if (k == MMFHE_ROT_CONJ) return k;
    int32_t n2 = (int32_t)(c.n / 2);
    int32_t r = k % n2;
    return r < 0 ? r + n2 : r;
}

uint32_t galois_elt(const Context &c, int32_t k) {
    if (k == MMFHE_ROT_CONJ) return (uint32_t)(2 * c.n - 1);   // slot-wise complex conjugation
    return (uint32_t)hm::powmod(5, (uint64_t)norm_rot(c, k), 2ull * c.n);
}

CtB ct_new(Context &c, int B, int level, double scale) {
    CtB r;
    r.B = B;
    r.level = level;
    r.scale = scale;
    r.buf = Buf(c.pool.get(), (size_t)B * c.ct_words(level));
    return r;
}

PtDev pt_new(Context &c, int level, double scale) {
    PtDev p;
    p.level = level;
    p.scale = scale;
    p.buf = Buf(c.pool.get(), (size_t)(level + 1) * c.n);
    return p;
}

static std::vector<int> iota_pids(int nl) {
    std::vector<int> v(nl);
    for (int i = 0; i < nl; i++) v[i] = i;
    return v;
}

void ntt_q_blocks(Context &c, uint64_t *base, size_t blocks, int nl, bool inverse, cudaStream_t st) {
    RowsView v{base, make_map(nl, nl, iota_pids(nl)), blocks * nl};
    launch_ntt(c, v, v, inverse, st);
}

void ct_addsub(Context &c, CtB &out, const CtB &a, const CtB &b, bool sub, cudaStream_t st) {
    if (a.level != b.level || a.B != b.B) throw Error(MMFHE_ERR_LEVEL_MISMATCH, "add: operand levels differ");
    k_launch_addsub(c, out.ptr(), a.ptr(), b.ptr(), (size_t)a.B * 2 * (a.level + 1), pids_q(a.level + 1),
                    a.level + 1, sub, st);
}

void ct_mul_plain(Context &c, CtB &out, const CtB &a, const PtDev &pt, bool acc, cudaStream_t st) {
    if (a.level != pt.level) throw Error(MMFHE_ERR_LEVEL_MISMATCH, "mul_plain: level mismatch");
    k_launch_mul_plain(c, out.ptr(), a.ptr(), pt.buf.get(), (size_t)a.B * 2 * (a.level + 1), pids_q(a.level + 1),
                       a.level + 1, acc, st, pt.mont);
}

PtDev pt_qp_from_coeffs(Context &c, const uint64_t *words, int level, double scale, cudaStream_t st) {
    const int nl = level + 1, nre = nl + c.num_p;
    PtDev pt;
    pt.level = level;
    pt.scale = scale;
    pt.qp = true;
    pt.buf = Buf(c.pool.get(), (size_t)nre * c.n);
    CK(cudaMemcpyAsync(pt.buf.get(), words, (size_t)nl * c.n * 8, cudaMemcpyDefault, st));
    Buf flag(c.pool.get(), 1);
    CK(cudaMemsetAsync(flag.get(), 0, 8, st));
    k_launch_qp_extend(c, pt.buf.get(), level, (int *)flag.get(), st);
    uint64_t bad = 0;
    CK(cudaMemcpyAsync(&bad, flag.get(), 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (bad) throw Error(MMFHE_ERR_BAD_ARG, "plaintext coefficients of magnitude q_0 / 2 or more: no extension to the special primes");
    std::vector<int> pids(nre);
    for (int t = 0; t < nre; t++) pids[t] = t < nl ? t : c.num_q + (t - nl);
    RowsView v{pt.buf.get(), make_map(nre, nre, pids), (size_t)nre};
    launch_ntt(c, v, v, false, st);
    k_launch_mont_convert(c, v, true, st);
    pt.mont = true;
    return pt;
}

void pt_to_mont(Context &c, PtDev &pt, cudaStream_t st) {
    if (pt.mont) return;
    const int nl = pt.level + 1;
    RowsView v{pt.buf.get(), make_map(nl, nl, iota_pids(nl)), (size_t)nl};
    k_launch_mont_convert(c, v, true, st);
    pt.mont = true;
}

void ct_mul_int(Context &c, CtB &out, const CtB &a, long long k, cudaStream_t st) {
    k_launch_mul_int(c, out.ptr(), a.ptr(), (size_t)a.B * 2 * (a.level + 1), pids_q(a.level + 1), a.level + 1, k, st);
}

CtB ct_copy(Context &c, const CtB &a, cudaStream_t st) {
    CtB r = ct_new(c, a.B, a.level, a.scale);
    CK(cudaMemcpyAsync(r.ptr(), a.ptr(), (size_t)a.B * c.ct_words(a.level) * 8, cudaMemcpyDeviceToDevice, st));
    return r;
}

CtB ct_slice(Context &c, const CtB &a, int b0, int nb, cudaStream_t st) {
    if (b0 < 0 || nb < 0 || b0 + nb > a.B) throw Error(MMFHE_ERR_BAD_ARG, "slice outside the batch");
    CtB r = ct_new(c, nb, a.level, a.scale);
    const size_t w = c.ct_words(a.level);
    CK(cudaMemcpyAsync(r.ptr(), a.ptr() + (size_t)b0 * w, (size_t)nb * w * 8, cudaMemcpyDeviceToDevice, st));
    return r;
}

void ct_place(Context &c, CtB &dst, int b0, const CtB &src, cudaStream_t st) {
    if (src.level != dst.level || b0 < 0 || b0 + src.B > dst.B) throw Error(MMFHE_ERR_BAD_ARG, "place outside the batch");
    const size_t w = c.ct_words(src.level);
    CK(cudaMemcpyAsync(dst.ptr() + (size_t)b0 * w, src.ptr(), (size_t)src.B * w * 8, cudaMemcpyDeviceToDevice, st));
}

CtB ct_drop(Context &c, const CtB &a, int level, cudaStream_t st) {
    if (level > a.level || level < 0) throw Error(MMFHE_ERR_LEVEL_MISMATCH, "drop: bad level");
    if (level == a.level) return ct_copy(c, a, st);
    CtB r = ct_new(c, a.B, level, a.scale);
    int nl = level + 1;
    RowsView src{a.ptr(), make_map(nl, a.level + 1, iota_pids(nl)), (size_t)a.B * 2 * nl};
    RowsView dst{r.ptr(), make_map(nl, nl, iota_pids(nl)), (size_t)a.B * 2 * nl};
    launch_copy_rows(c, src, dst, st);
    return r;
}

TensorB tensor_new(Context &c, int B, int level) {
    TensorB t;
    t.B = B;
    t.level = level;
    t.buf = Buf(c.pool.get(), (size_t)B * 3 * (level + 1) * c.n);
    return t;
}

void tensor_acc(Context &c, TensorB &t, const CtB &a, const CtB &b, long long coef, bool init, cudaStream_t st) {
    if (a.level != b.level || a.level != t.level || a.B != t.B || b.B != t.B)
        throw Error(MMFHE_ERR_LEVEL_MISMATCH, "tensor: level mismatch");
    if (init) t.scale = a.scale * b.scale;
    k_launch_tensor(c, t.buf.get(), a.ptr(), b.ptr(), t.B, t.level, coef, !init, st);
}

DigitsB modup(Context &c, const uint64_t *d_eval, size_t block_stride_rows, int B, int level, cudaStream_t st) {
    const int nl = level + 1, nre = level + 1 + c.num_p;
    const LevelConsts &lc = c.lv[level];
    DigitsB dg;
    dg.B = B;
    dg.level = level;
    dg.beta = lc.beta;
    dg.own = d_eval;
    dg.own_stride = block_stride_rows * c.n;
    dg.buf = Buf(c.pool.get(), (size_t)B * lc.beta * nre * c.n);
    // y = [x (Qhat_{j,u})^-1]_{q_i} in coefficient form: the inverse NTT's last multiply
    Buf y(c.pool.get(), (size_t)B * nl * c.n);
    RowsView src{const_cast<uint64_t *>(d_eval), make_map(nl, (uint32_t)block_stride_rows, iota_pids(nl)), (size_t)B * nl};
    RowsView dst{y.get(), make_map(nl, nl, iota_pids(nl)), (size_t)B * nl};
    launch_ntt(c, src, dst, true, st, lc.d_ks_scale, lc.d_ks_scale_sh);
    // FastBConv to every other prime inside the forward NTT of each digit row
    launch_modup_ntt(c, dg.buf.get(), y.get(), B, level, st);
    return dg;
}

void digits_fill_own(Context &c, DigitsB &dg, cudaStream_t st) {
    const int nl = dg.level + 1, nre = nl + c.num_p;
    const LevelConsts &lc = c.lv[dg.level];
    for (int j = 0; j < dg.beta; j++) {
        std::vector<int> pids(nre, -1);
        for (int t : lc.digits[j]) pids[t] = t;
        RowsView src{const_cast<uint64_t *>(dg.own), make_map(nre, (uint32_t)(dg.own_stride / c.n), pids),
                     (size_t)dg.B * nre};
        RowsView dst{dg.buf.get() + (size_t)j * nre * c.n, make_map(nre, dg.beta * nre, pids), (size_t)dg.B * nre};
        launch_copy_rows(c, src, dst, st);
    }
}

CtB keyswitch_moddown(Context &c, const DigitsB &dg, const KeyPtrs &key, uint32_t galois, const uint64_t *add0,
                      const uint64_t *add1, size_t add_stride_words, double scale, cudaStream_t st, const CtB *plus) {
    const int level = dg.level, B = dg.B, nl = level + 1, nre = level + 1 + c.num_p, K = c.num_p;
    if (key.n != 1 && key.n != B) throw Error(MMFHE_ERR_BAD_ARG, "one switching key per window or one for all");
    if (plus && (plus->level != level || plus->B != B)) throw Error(MMFHE_ERR_LEVEL_MISMATCH, "add: operand levels differ");
    if (c.tune.keyip_fused) {
        // the inner product's words are formed where they are consumed: its P rows in the
        // load of z's inverse NTT, its Q rows in the combine (never stored)
        KeyipArgs ka{};
        ka.digits = dg.buf.get();
        ka.own = dg.own;
        ka.own_stride = dg.own_stride;
        ka.key = key;
        ka.beta = dg.beta;
        ka.alpha = c.alpha;
        ka.nre = nre;
        ka.level = level;
        ka.key_rows = c.num_q + c.num_p;
        ka.L1 = c.num_q;
        ka.w0 = 0;
        ka.galois = galois;
        Buf z(c.pool.get(), (size_t)B * 2 * K * c.n);
        launch_keyip_p_inv(c, z.get(), ka, B, level, st);
        Buf v(c.pool.get(), (size_t)B * 2 * nl * c.n);
        CtB out = ct_new(c, B, level, scale);
        CombineArgs a{out.ptr(), nullptr, add0, add1, add_stride_words, galois, plus ? plus->ptr() : nullptr};
        launch_moddown_ntt(c, v.get(), z.get(), a, B, level, st, &ka);
        return out;
    }
    Buf u(c.pool.get(), (size_t)B * 2 * nre * c.n);
    k_launch_keyip(c, u.get(), dg.buf.get(), dg.own, dg.own_stride, 0, key, B, level, dg.beta, galois, st);
    // z = [u_P Phat^-1]_P in coefficient form, [B*2][K][N]
    Buf z(c.pool.get(), (size_t)B * 2 * K * c.n);
    std::vector<int> pids(nre, -1);
    for (int k = 0; k < K; k++) pids[nl + k] = c.num_q + k;
    RowsView pv{u.get(), make_map(nre, nre, pids), (size_t)B * 2 * nre};
    RowMap zm = make_map(nre, K, pids);
    zm.row0 = nl;
    RowsView zv{z.get(), zm, (size_t)B * 2 * nre};
    launch_ntt(c, pv, zv, true, st, c.lv[level].d_ks_scale, c.lv[level].d_ks_scale_sh);
    // centered FastBConv P -> Q inside v's forward NTT; the combine inside its last pass
    Buf v(c.pool.get(), (size_t)B * 2 * nl * c.n);
    CtB out = ct_new(c, B, level, scale);
    CombineArgs a{out.ptr(), u.get(), add0, add1, add_stride_words, galois, plus ? plus->ptr() : nullptr};
    launch_moddown_ntt(c, v.get(), z.get(), a, B, level, st);
    return out;
}

CtB relin(Context &c, const Keys &k, const TensorB &t, cudaStream_t st) {
    const KeyPtrs key = relin_key(k);
    const int nl = t.level + 1;
    const uint64_t *base = t.buf.get();
    DigitsB dg = modup(c, base + (size_t)2 * nl * c.n, (size_t)3 * nl, t.B, t.level, st);
    return keyswitch_moddown(c, dg, key, 1, base, base + (size_t)nl * c.n, (size_t)3 * nl * c.n, t.scale, st);
}

CtB rescale(Context &c, const CtB &a, cudaStream_t st) {
    const int l = a.level;
    if (l < 1) throw Error(MMFHE_ERR_LEVEL_MISMATCH, "rescale at level 0");
    const int B = a.B;
    Buf last(c.pool.get(), (size_t)B * 2 * c.n);
    RowsView src{a.ptr() + (size_t)l * c.n, make_map(1, l + 1, {l}), (size_t)B * 2};
    RowsView dst{last.get(), make_map(1, 1, {l}), (size_t)B * 2};
    launch_ntt(c, src, dst, true, st);
    Buf tmp(c.pool.get(), (size_t)B * 2 * l * c.n);
    RescaleConsts rc = rescale_consts(c, l);
    k_launch_rescale_spread(c, tmp.get(), last.get(), B, l, rc, st);
    ntt_q_blocks(c, tmp.get(), (size_t)B * 2, l, false, st);
    CtB out = ct_new(c, B, l - 1, a.scale / (double)c.primes[l]);
    k_launch_rescale_combine(c, out.ptr(), a.ptr(), tmp.get(), B, l, rc, st);
    return out;
}

static const uint64_t *one_galois_key(const Keys &k, int32_t rot) {
    auto it = k.gk.find(rot);
    if (it == k.gk.end()) throw Error(MMFHE_ERR_NOT_FOUND, "Galois key for rotation " + std::to_string(rot) + " not loaded");
    return it->second.get();
}

KeyPtrs galois_key(const Keys &k, int32_t rot) {
    KeyPtrs p;
    if (k.windows.empty()) {
        p.k[0] = one_galois_key(k, rot);
        p.n = 1;
        return p;
    }
    if (k.windows.size() > (size_t)MAX_KEY_WINDOWS) throw Error(MMFHE_ERR_BAD_ARG, "too many key sets in one batch");
    for (size_t w = 0; w < k.windows.size(); w++) p.k[w] = one_galois_key(*k.windows[w], rot);
    p.n = (int)k.windows.size();
    return p;
}

KeyPtrs relin_key(const Keys &k) {
    KeyPtrs p;
    auto one = [](const Keys &x) {
        if (!x.rlk.get()) throw Error(MMFHE_ERR_NOT_FOUND, "relinearization key not loaded");
        return (const uint64_t *)x.rlk.get();
    };
    if (k.windows.empty()) {
        p.k[0] = one(k);
        p.n = 1;
        return p;
    }
    if (k.windows.size() > (size_t)MAX_KEY_WINDOWS) throw Error(MMFHE_ERR_BAD_ARG, "too many key sets in one batch");
    for (size_t w = 0; w < k.windows.size(); w++) p.k[w] = one(*k.windows[w]);
    p.n = (int)k.windows.size();
    return p;
}

std::vector<CtB> rotate_hoisted(Context &c, const Keys &k, const CtB &a, const std::vector<int32_t> &rots,
                                cudaStream_t st) {
    std::vector<CtB> out;
    out.reserve(rots.size());
    bool any = false;
    for (int32_t r : rots) {
        int32_t nr = norm_rot(c, r);
        if (nr) {
            galois_key(k, nr);   // fail before any work if a key is missing
            any = true;
        }
    }
    DigitsB dg;
    const int nl = a.level + 1;
    if (any) dg = modup(c, a.ptr() + (size_t)nl * c.n, (size_t)2 * nl, a.B, a.level, st);
    for (int32_t r : rots) {
        int32_t nr = norm_rot(c, r);
        if (nr == 0) {
            out.push_back(ct_copy(c, a, st));
            continue;
        }
        out.push_back(keyswitch_moddown(c, dg, galois_key(k, nr), galois_elt(c, nr), a.ptr(), nullptr,
                                        (size_t)2 * nl * c.n, a.scale, st));
    }
    return out;
}

CtB rotate(Context &c, const Keys &k, const CtB &a, int32_t rot, cudaStream_t st) {
    std::vector<CtB> v = rotate_hoisted(c, k, a, {rot}, st);
    return std::move(v[0]);
}

CtB rotate_add(Context &c, const Keys &k, const CtB &a, int32_t rot, const CtB &plus, cudaStream_t st) {
    int32_t nr = norm_rot(c, rot);
    if (nr == 0) {
        CtB r = ct_new(c, a.B, a.level, a.scale);
        ct_addsub(c, r, a, plus, false, st);
        return r;
    }
    const int nl = a.level + 1;
    const KeyPtrs key = galois_key(k, nr);
    DigitsB dg = modup(c, a.ptr() + (size_t)nl * c.n, (size_t)2 * nl, a.B, a.level, st);
    return keyswitch_moddown(c, dg, key, galois_elt(c, nr), a.ptr(), nullptr, (size_t)2 * nl * c.n, a.scale, st,
                             &plus);
}

CtB lincomb(Context &c, const std::vector<std::pair<const CtB *, double>> &terms, double scale, cudaStream_t st) {
    if (terms.empty()) throw Error(MMFHE_ERR_BAD_ARG, "lincomb of no terms");
    const CtB &x0 = *terms[0].first;
    const int nl = x0.level + 1;
    CtB out = ct_new(c, x0.B, x0.level, x0.scale * scale);
    const size_t chunk = (size_t)std::min(MAX_SUM_TERMS, c.sum_terms_max);
    for (size_t t0 = 0; t0 < terms.size(); t0 += chunk) {
        LincombTerms lt{};
        lt.n = (int)std::min(chunk, terms.size() - t0);
        for (int j = 0; j < lt.n; j++) {
            const CtB &x = *terms[t0 + j].first;
            if (x.level != x0.level || x.B != x0.B) throw Error(MMFHE_ERR_LEVEL_MISMATCH, "lincomb: operands differ");
            lt.ct[j] = x.ptr();
            // round half away from zero, as the encoder does
            const double v = std::round(scale * terms[t0 + j].second);
            const long long m = (long long)v;
            for (int i = 0; i < nl; i++) {
                const uint64_t q = c.primes[i];
                const uint64_t r = m >= 0 ? (uint64_t)m % q : (q - ((uint64_t)(-m) % q)) % q;
                lt.s[j][i] = (uint64_t)(((unsigned __int128)r * c.mods.r64[i]) % q);   // Montgomery form
            }
        }
        k_launch_lincomb(c, out.ptr(), lt, x0.B, x0.level, t0 > 0, st);
    }
    return out;
}

CtB add_plain(Context &c, const CtB &a, const PtDev &pt, cudaStream_t st) {
    if (a.level != pt.level) throw Error(MMFHE_ERR_LEVEL_MISMATCH, "add_plain: level mismatch");
    if (!pt.mont) throw Error(MMFHE_ERR_BAD_ARG, "add_plain: plaintext must be in Montgomery form");
    CtB r = ct_copy(c, a, st);
    k_launch_add_plain(c, r.ptr(), pt.buf.get(), r.B, r.level, st);
    return r;
}

CtB group_sum(Context &c, const CtB &a, int G, cudaStream_t st) {
    if (G < 1 || a.B % G) throw Error(MMFHE_ERR_BAD_ARG, "group_sum: batch not a multiple of the group");
    CtB r = ct_new(c, a.B / G, a.level, a.scale);
    k_launch_group_sum(c, r.ptr(), a.ptr(), r.B, G, a.level, st);
    return r;
}

CtB rotsum(Context &c, const Keys &k, const CtB &a, int32_t stride, uint32_t span, cudaStream_t st) {
    if (span <= 1) return ct_copy(c, a, st);
    // x <- x + Rot(x, stride s): the addition happens inside the key switch's last kernel
    CtB x = rotate_add(c, k, a, stride, a, st);
    for (uint32_t s = 2; s < span; s <<= 1) x = rotate_add(c, k, x, stride * (int32_t)s, x, st);
    return x;
}

CtB bsgs(Context &c, const Keys &k, const std::vector<BsgsTerm> &terms, int n1, int32_t stride, cudaStream_t st) {
    struct Item { const CtB *baby; const PtDev *pt; };
    std::map<int, std::vector<Item>> groups;   // giant step g = delta / n1 -> products
    int level = -1, B = 0;
    double scale = 0;
    for (const BsgsTerm &t : terms) {
        std::map<int, int> pos;
        for (size_t i = 0; i < t.baby_idx.size(); i++) pos[t.baby_idx[i]] = (int)i;
        for (const auto &d : t.diags) {
            // delta = g n1 + b with 0 <= b < n1 (floor division: deltas may be negative)
            const int g = d.first >= 0 ? d.first / n1 : -((-d.first + n1 - 1) / n1);
            auto it = pos.find(d.first - g * n1);
            if (it == pos.end()) throw Error(MMFHE_ERR_BAD_ARG, "bsgs: missing baby step");
            const CtB *bb = &(*t.baby)[it->second];
            groups[g].push_back(Item{bb, d.second});
            level = bb->level;
            B = bb->B;
            scale = bb->scale * d.second->scale;
        }
    }
    if (groups.empty()) throw Error(MMFHE_ERR_BAD_ARG, "bsgs: no diagonals");
    // the distinct baby steps: when they fit one reduction, every giant step's
    // inner sum comes from one pass over them (MULTI_SUM_GROUPS at a time)
    std::vector<const CtB *> babies;
    std::map<const CtB *, int> bpos;
    for (auto &kv : groups)
        for (const Item &it : kv.second)
            if (bpos.emplace(it.baby, (int)babies.size()).second) babies.push_back(it.baby);
    const int tmax = std::min(MAX_SUM_TERMS, c.sum_terms_max);
    bool fused = groups.size() > 1;
    for (auto &kv : groups) {   // one diagonal per baby step and group
        std::set<const CtB *> seen;
        for (const Item &it : kv.second) fused &= seen.insert(it.baby).second;
    }
    std::map<int, CtB> inners;
    if (fused) {
        for (const CtB *bb : babies)
            if (bb->level != level || bb->B != B) throw Error(MMFHE_ERR_LEVEL_MISMATCH, "bsgs: operand levels differ");
        std::vector<int> gs;
        for (auto &kv : groups) gs.push_back(kv.first);
        for (size_t g0 = 0; g0 < gs.size(); g0 += MULTI_SUM_GROUPS) {
            const int ng = (int)std::min<size_t>(MULTI_SUM_GROUPS, gs.size() - g0);
            for (int j = 0; j < ng; j++) inners.emplace(gs[g0 + j], ct_new(c, B, level, scale));
            // the baby steps in chunks of one reduction each, accumulated
            for (size_t t0 = 0; t0 < babies.size(); t0 += (size_t)tmax) {
                MultiSumTerms mt{};
                mt.nt = (int)std::min<size_t>((size_t)tmax, babies.size() - t0);
                mt.ng = ng;
                for (int t = 0; t < mt.nt; t++) mt.ct[t] = babies[t0 + t]->ptr();
                for (int j = 0; j < ng; j++) {
                    const int g = gs[g0 + j];
                    mt.out[j] = inners.at(g).ptr();
                    for (const Item &it : groups[g]) {
                        if (it.pt->level != level) throw Error(MMFHE_ERR_LEVEL_MISMATCH, "bsgs: operand levels differ");
                        if (!it.pt->mont) throw Error(MMFHE_ERR_BAD_ARG, "bsgs: diagonals must be in Montgomery form");
                        const int pos = bpos[it.baby] - (int)t0;
                        if (pos >= 0 && pos < mt.nt) mt.pt[j][pos] = it.pt->buf.get();
                    }
                }
                k_launch_mul_plain_sum_multi(c, mt, B, level, t0 > 0, st);
            }
        }
    }
    CtB acc;
    bool have = false;
    for (auto &kv : groups) {
        if (!inners.empty()) {
            CtB &inner = inners.at(kv.first);
            if (!have) {
                acc = kv.first != 0 ? rotate(c, k, inner, kv.first * n1 * stride, st) : std::move(inner);
                have = true;
            } else if (kv.first != 0) {
                acc = rotate_add(c, k, inner, kv.first * n1 * stride, acc, st);   // acc + Rot(inner)
            } else {
                ct_addsub(c, acc, acc, inner, false, st);
            }
            inners.erase(kv.first);
            continue;
        }
        // one fused launch per MAX_SUM_TERMS products of the giant step
        CtB inner = ct_new(c, B, level, scale);
        const auto &items = kv.second;
        const size_t chunk = (size_t)std::min(MAX_SUM_TERMS, c.sum_terms_max);
        for (size_t k0 = 0; k0 < items.size(); k0 += chunk) {
            SumTerms terms{};
            terms.n = (int)std::min<size_t>(chunk, items.size() - k0);
            for (int t = 0; t < terms.n; t++) {
                const Item &it = items[k0 + t];
                if (it.baby->level != level || it.pt->level != level || it.baby->B != B)
                    throw Error(MMFHE_ERR_LEVEL_MISMATCH, "bsgs: operand levels differ");
                if (!it.pt->mont) throw Error(MMFHE_ERR_BAD_ARG, "bsgs: diagonals must be in Montgomery form");
                terms.ct[t] = it.baby->ptr();
                terms.pt[t] = it.pt->buf.get();
            }
            k_launch_mul_plain_sum(c, inner.ptr(), terms, B, level, k0 > 0, st);
        }
        if (!have) {
            acc = kv.first != 0 ? rotate(c, k, inner, kv.first * n1 * stride, st) : std::move(inner);
            have = true;
        } else if (kv.first != 0) {
            acc = rotate_add(c, k, inner, kv.first * n1 * stride, acc, st);   // acc + Rot(inner)
        } else {
            ct_addsub(c, acc, acc, inner, false, st);
        }
    }
    return acc;
}

// ModDown of `blocks` blocks over Q_l * P (block k at u + k * ustride rows)
// into out [blocks][l+1][N]: inverse NTT of the P rows with Phat^-1 folded,
// centered conversion inside v's forward NTT, (u - v) P^-1 in its last pass.
static void moddown_blocks(Context &c, uint64_t *out, const uint64_t *u, size_t ustride, size_t blocks, int level,
                           cudaStream_t st) {
    const int nl = level + 1, nre = nl + c.num_p, K = c.num_p;
    Buf z(c.pool.get(), blocks * K * c.n);
    std::vector<int> pids(nre, -1);
    for (int kk = 0; kk < K; kk++) pids[nl + kk] = c.num_q + kk;
    RowsView pv{const_cast<uint64_t *>(u), make_map(nre, (uint32_t)ustride, pids), blocks * nre};
    RowMap zm = make_map(nre, K, pids);
    zm.row0 = nl;
    RowsView zv{z.get(), zm, blocks * nre};
    launch_ntt(c, pv, zv, true, st, c.lv[level].d_ks_scale, c.lv[level].d_ks_scale_sh);
    Buf v(c.pool.get(), blocks * nl * c.n);
    CombineArgs a{out, u, nullptr, nullptr, 0, 1, nullptr};
    a.u_stride = ustride;
    launch_moddown_ntt_blocks(c, v.get(), z.get(), a, blocks, level, st);
}

CtB bsgs_dh(Context &c, const Keys &k, const std::vector<BsgsSet> &sets, int n1, int32_t stride, cudaStream_t st) {
    if (sets.empty() || !sets[0].x) throw Error(MMFHE_ERR_BAD_ARG, "bsgs: no input");
    const CtB &x0 = *sets[0].x;
    const int level = x0.level, B = x0.B, nl = level + 1, nre = nl + c.num_p;
    const size_t qp_words = (size_t)B * 2 * nre * c.n;
    const ModDownConsts dc = moddown_consts(c);
    auto floor_div = [&](int d) { return d >= 0 ? d / n1 : -((-d + n1 - 1) / n1); };
    // babies needed per set, giant groups of (set, baby, diagonal)
    struct Item { int set, b; const PtDev *pt; };
    std::map<int, std::vector<Item>> groups;
    std::vector<std::set<int>> need(sets.size());
    double scale = 0;
    for (size_t s = 0; s < sets.size(); s++) {
        const BsgsSet &bs = sets[s];
        if (!bs.x || bs.x->level != level || bs.x->B != B) throw Error(MMFHE_ERR_LEVEL_MISMATCH, "bsgs: operand levels differ");
        for (const auto &d : bs.diags) {
            const PtDev *pt = d.second;
            if (pt->level != level || !pt->qp || !pt->mont)
                throw Error(MMFHE_ERR_BAD_ARG, "bsgs: diagonals must be over the extended basis, in Montgomery form");
            const int g = floor_div(d.first), b = d.first - g * n1;
            groups[g].push_back(Item{(int)s, b, pt});
            need[s].insert(b);
            scale = bs.x->scale * pt->scale;
        }
    }
    if (groups.empty()) throw Error(MMFHE_ERR_BAD_ARG, "bsgs: no diagonals");
    // every key before any work
    for (size_t s = 0; s < sets.size(); s++)
        for (int b : need[s]) {
            const int32_t r = norm_rot(c, b * stride + sets[s].offset);
            if (r) galois_key(k, r);
        }
    for (auto &kv : groups) {
        const int32_t r = norm_rot(c, kv.first * n1 * stride);
        if (r) galois_key(k, r);
    }
    // babies over Q_l * P; one ModUp per distinct input
    std::map<const CtB *, DigitsB> digits;
    std::map<std::pair<int, int>, Buf> babies;
    for (size_t s = 0; s < sets.size(); s++) {
        const CtB &x = *sets[s].x;
        for (int b : need[s]) {
            Buf u(c.pool.get(), qp_words);
            const int32_t r = norm_rot(c, b * stride + sets[s].offset);
            if (r == 0) {
                k_launch_qp_times_p(c, u.get(), x.ptr(), B, level, dc, st);
            } else {
                auto it = digits.find(&x);
                if (it == digits.end())
                    it = digits.emplace(&x, modup(c, x.ptr() + (size_t)nl * c.n, (size_t)2 * nl, B, level, st)).first;
                const DigitsB &dg = it->second;
                const uint32_t gal = galois_elt(c, r);
                k_launch_keyip(c, u.get(), dg.buf.get(), dg.own, dg.own_stride, 0, galois_key(k, r), B, level, dg.beta,
                               gal, st);
                k_launch_qp_add_pc0(c, u.get(), x.ptr(), B, level, gal, dc, st);
            }
            babies.emplace(std::make_pair((int)s, b), std::move(u));
        }
    }
    digits.clear();
    // inner sums, MULTI_SUM_GROUPS giant steps per pass over the babies; each
    // giant-step term accumulated into acc over Q_l * P
    std::vector<std::pair<int, int>> order;
    for (auto &kv : babies) order.push_back(kv.first);
    std::map<std::pair<int, int>, int> bpos;
    for (size_t i = 0; i < order.size(); i++) bpos[order[i]] = (int)i;
    std::vector<int> gs;
    for (auto &kv : groups) gs.push_back(kv.first);
    const int tmax = std::min(MAX_SUM_TERMS, c.sum_terms_max_qp);
    Buf acc(c.pool.get(), qp_words);
    bool have = false;
    for (size_t g0 = 0; g0 < gs.size(); g0 += MULTI_SUM_GROUPS) {
        const int ng = (int)std::min<size_t>(MULTI_SUM_GROUPS, gs.size() - g0);
        std::vector<Buf> inner;
        for (int j = 0; j < ng; j++) inner.emplace_back(c.pool.get(), qp_words);
        for (size_t t0 = 0; t0 < order.size(); t0 += (size_t)tmax) {
            MultiSumTerms mt{};
            mt.nt = (int)std::min<size_t>((size_t)tmax, order.size() - t0);
            mt.ng = ng;
            for (int t = 0; t < mt.nt; t++) mt.ct[t] = babies.at(order[t0 + t]).get();
            for (int j = 0; j < ng; j++) {
                mt.out[j] = inner[j].get();
                for (const Item &it : groups[gs[g0 + j]]) {
                    const int pos = bpos.at({it.set, it.b}) - (int)t0;
                    if (pos >= 0 && pos < mt.nt) {
                        if (mt.pt[j][pos]) throw Error(MMFHE_ERR_BAD_ARG, "bsgs: two diagonals for one baby and giant step");
                        mt.pt[j][pos] = it.pt->buf.get();
                    }
                }
            }
            k_launch_mul_plain_sum_multi(c, mt, B, level, t0 > 0, st, true);
        }
        for (int j = 0; j < ng; j++) {
            const int g = gs[g0 + j];
            const int32_t r = norm_rot(c, g * n1 * stride);
            if (r == 0) {
                k_launch_qp_giant_acc(c, acc.get(), inner[j].get(), nullptr, B, level, 1, have, st);
            } else {
                // c1 of the inner sum down to Q, then its key switch over Q_l * P
                Buf d(c.pool.get(), (size_t)B * nl * c.n);
                moddown_blocks(c, d.get(), inner[j].get() + (size_t)nre * c.n, (size_t)2 * nre, (size_t)B, level, st);
                DigitsB dg = modup(c, d.get(), (size_t)nl, B, level, st);
                Buf w(c.pool.get(), qp_words);
                const uint32_t gal = galois_elt(c, r);
                k_launch_keyip(c, w.get(), dg.buf.get(), dg.own, dg.own_stride, 0, galois_key(k, r), B, level, dg.beta,
                               gal, st);
                k_launch_qp_giant_acc(c, acc.get(), inner[j].get(), w.get(), B, level, gal, have, st);
            }
            have = true;
            inner[j].release();
        }
    }
    babies.clear();
    CtB out = ct_new(c, B, level, scale);
    moddown_blocks(c, out.ptr(), acc.get(), (size_t)nre, (size_t)B * 2, level, st);
    return out;
}

}  // namespace mmfhe
