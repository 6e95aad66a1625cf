// Element-wise and key-switching kernels (evaluation domain unless stated).
//
// Layouts (N words per row, rows contiguous):
//   ciphertext batch   [B][2][l+1][N]
//   tensor batch       [B][3][l+1][N]            (d0, d1, d2)
//   ModUp digits       [B][beta][l+1+K][N]        rows q_0..q_l, p_0..p_{K-1}
//   key-switch output  [B][2][l+1+K][N]
//   key                [dnum][2][L+1+K][N]        (device, evaluation domain)
#include <cuda_runtime.h>

#include <type_traits>

#include <algorithm>

#include "internal.h"
#include "kernels.h"
#include "modarith.cuh"

namespace mmfhe {

namespace {

constexpr int EW_THREADS = 256;

inline dim3 grid_for(size_t work) {
    size_t b = (work + EW_THREADS - 1) / EW_THREADS;
    return dim3((unsigned)std::min<size_t>(b, 148 * 64));
}

// 128-bit multiply-accumulate, the small-operand form for primes below
// SMALL_PRIME_LIMIT (S is uniform over a row, so over a warp).
template <bool S>
__device__ __forceinline__ void macq(uint64_t &hi, uint64_t &lo, uint64_t a, uint64_t b) {
    if (S) mm::mac128_small(hi, lo, a, b);
    else mm::mac128(hi, lo, a, b);
}
using SmallT = std::true_type;
using WideT = std::false_type;

__device__ __forceinline__ uint64_t mulq(uint64_t a, uint64_t b, const ModTab &mt, int pid) {
    return mm::mul_barrett(a, b, mt.q[pid], mt.mu[pid], mt.k[pid]);
}

// out[r] = a[r] (op) b[r]; rows have prime pid[r % period].
__global__ void k_addsub(uint64_t *out, const uint64_t *a, const uint64_t *b, size_t words, int logn, uint32_t period,
                         ModTab mt, PidList pl, int sub) {
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < words; w += (size_t)gridDim.x * blockDim.x) {
        int pid = pl.pid[(w >> logn) % period];
        uint64_t q = mt.q[pid];
        out[w] = sub ? mm::sub_mod(a[w], b[w], q) : mm::add_mod(a[w], b[w], q);
    }
}

// out[r] = c * a[r] mod q (c a small signed integer).
__global__ void k_mul_int(uint64_t *out, const uint64_t *a, size_t words, int logn, uint32_t period, ModTab mt,
                          PidList pl, long long c) {
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < words; w += (size_t)gridDim.x * blockDim.x) {
        int pid = pl.pid[(w >> logn) % period];
        uint64_t q = mt.q[pid];
        uint64_t cm = c >= 0 ? (uint64_t)c % q : (q - ((uint64_t)(-c) % q)) % q;
        out[w] = mulq(a[w], cm, mt, pid);
    }
}

// out[r] (+)= a[r] * pt[r % period]   (pt rows = one plaintext, shared by all
// blocks; mont: pt is in Montgomery form)
__global__ void k_mul_plain(uint64_t *out, const uint64_t *a, const uint64_t *pt, size_t words, int logn,
                            uint32_t period, ModTab mt, PidList pl, int accumulate, int mont) {
    const uint32_t n = 1u << logn;
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < words; w += (size_t)gridDim.x * blockDim.x) {
        uint32_t row = (uint32_t)(w >> logn) % period;
        int pid = pl.pid[row];
        const uint64_t av = a[w], pv = pt[(size_t)row * n + (w & (n - 1))];
        uint64_t v = mont ? mm::redc(mm::mulhi64(av, pv), av * pv, mt.q[pid], mt.qinv[pid]) : mulq(av, pv, mt, pid);
        out[w] = accumulate ? mm::add_mod(out[w], v, mt.q[pid]) : v;
    }
}

// c0 of every window (+)= pt (pt in Montgomery form: redc brings it back);
// c1 is untouched.  Ciphertext layout [B][2][nl][N].
__global__ void k_add_plain(uint64_t *ct, const uint64_t *pt, size_t words, int logn, int nl, ModTab mt) {
    const uint32_t n = 1u << logn;
    const size_t per = (size_t)nl << logn;
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < words; w += (size_t)gridDim.x * blockDim.x) {
        const size_t b = w / per, r = w - b * per;
        const int i = (int)(r >> logn);
        const uint64_t q = mt.q[i];
        uint64_t *dst = ct + b * 2 * per + r;
        *dst = mm::add_mod(*dst, mm::redc(0, pt[((size_t)i << logn) + (r & (n - 1))], q, mt.qinv[i]), q);
    }
}

// out[b] = sum_{g < G} in[b G + g] (ciphertexts of `wpc` words, rows of nl Q primes).
__global__ void k_group_sum(uint64_t *out, const uint64_t *in, size_t words, size_t wpc, int G, int logn, int nl,
                            ModTab mt) {
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < words; w += (size_t)gridDim.x * blockDim.x) {
        const size_t b = w / wpc, r = w - b * wpc;
        const uint64_t q = mt.q[(r >> logn) % nl];
        const uint64_t *src = in + b * G * wpc + r;
        uint64_t acc = src[0];
        for (int g = 1; g < G; g++) acc = mm::add_mod(acc, src[(size_t)g * wpc], q);
        out[w] = acc;
    }
}

// All giant steps of a BSGS product from one read of the baby steps.  A CTA
// owns MULTI_X consecutive slots x of one row (h, i) and walks every window:
// its threads keep the ng x T constant words of their own x in shared memory
// (read once per launch; each thread touches only its own column, so no
// barrier is needed), load the T baby words of a window once, and write the
// ng giant-step sums.
constexpr int MULTI_X = 64;
template <int T>
__global__ void __launch_bounds__(MULTI_X)
    k_mul_plain_sum_multi(MultiSumTerms a, int B, int logn, int nl, int nrows, int pid_p0, ModTab mt,
                          int accumulate) {
    extern __shared__ uint64_t sp[];   // [ng][T][MULTI_X]
    const uint32_t n = 1u << logn;
    const uint32_t tiles = n / MULTI_X;
    const uint32_t row = blockIdx.x / tiles;          // h * nrows + i
    const int i = (int)(row % (uint32_t)nrows);       // rows q_0..q_l, then p_0..p_{K-1} (extended basis)
    const int pid = i < nl ? i : pid_p0 + (i - nl);
    const uint32_t x = (blockIdx.x % tiles) * MULTI_X + threadIdx.x;
    const size_t poff = ((size_t)i << logn) + x;
    const int ng = a.ng, nt = a.nt;
    for (int g = 0; g < ng; g++)
#pragma unroll
        for (int t = 0; t < T; t++)
            sp[(g * T + t) * MULTI_X + threadIdx.x] = (t < nt && a.pt[g][t]) ? __ldg(a.pt[g][t] + poff) : 0;
    const uint64_t q = mt.q[pid], qinv = mt.qinv[pid];
    const size_t wstride = (size_t)2 * nrows << logn;
    const size_t off = ((size_t)row << logn) + x;
    uint64_t v[T], vn[T];
#pragma unroll
    for (int t = 0; t < T; t++) v[t] = t < nt ? __ldg(a.ct[t] + off) : 0;
    auto walk = [&](auto small) {
        constexpr bool S = decltype(small)::value;
        for (int b = 0; b < B; b++) {
            const size_t wo = (size_t)b * wstride + off;
            // the next window's baby words load under this window's arithmetic
#pragma unroll
            for (int t = 0; t < T; t++) vn[t] = (t < nt && b + 1 < B) ? __ldg(a.ct[t] + wo + wstride) : 0;
            for (int g = 0; g < ng; g++) {
                uint64_t hi = 0, lo = 0;
#pragma unroll
                for (int t = 0; t < T; t++) macq<S>(hi, lo, v[t], sp[(g * T + t) * MULTI_X + threadIdx.x]);
                const uint64_t r = mm::redc(hi, lo, q, qinv);
                uint64_t *o = a.out[g] + wo;
                *o = accumulate ? mm::add_mod(*o, r, q) : r;
            }
#pragma unroll
            for (int t = 0; t < T; t++) v[t] = vn[t];
        }
    };
    if (q < mm::SMALL_PRIME_LIMIT) walk(SmallT{});
    else walk(WideT{});
}

// ---------------------------------------------------------------------------
// Extended-basis (Q_l * P) helpers of the double-hoisted BSGS product.
// An extended ciphertext batch is [B][2][l+1+K][N]: rows q_0..q_l, then
// p_0..p_{K-1}, evaluation domain.
// ---------------------------------------------------------------------------

// (P c0, P c1) over Q_l * P from a ciphertext over Q_l: rows mod q_i times
// P mod q_i, rows mod p_k zero (P = 0 there).
__global__ void k_qp_times_p(uint64_t *out, const uint64_t *in, int B, int nl, int K, int logn, ModTab mt,
                             ModDownConsts dc) {
    const int nre = nl + K;
    const size_t total = ((size_t)B * 2 * nre) << logn;
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
        const size_t r = w >> logn, x = w & ((1u << logn) - 1);
        const int t = (int)(r % nre);
        const size_t bh = r / nre;
        if (t >= nl) {
            out[w] = 0;
            continue;
        }
        const uint64_t v = in[((bh * nl + t) << logn) + x];
        out[w] = mm::mul_shoup(v, dc.pmod[t], dc.pmod_sh[t], mt.q[t]);
    }
}

// u0 rows mod q_i += P * c0[perm(x)] mod q_i: the baby's c0 term (u = the key
// inner product of its rotation, [B][2][nre]; c0 of the input, [B][2][nl]).
__global__ void k_qp_add_pc0(uint64_t *u, const uint64_t *ct, int B, int nl, int K, int logn, uint32_t galois,
                             ModTab mt, ModDownConsts dc) {
    const int nre = nl + K;
    const uint32_t n = 1u << logn;
    const size_t total = ((size_t)B * nl) << logn;
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(w & (n - 1));
        const size_t r = w >> logn;
        const int i = (int)(r % nl);
        const size_t b = r / nl;
        const uint32_t px = galois == 1 ? x : mm::galois_perm(x, galois, logn);
        const uint64_t q = mt.q[i];
        const uint64_t pc = mm::mul_shoup(ct[((b * 2 * nl + i) << logn) + px], dc.pmod[i], dc.pmod_sh[i], q);
        uint64_t *U = u + ((b * 2 * nre + i) << logn) + x;
        *U = mm::add_mod(*U, pc, q);
    }
}

// Giant-step term of the double-hoisted product, accumulated over Q_l * P:
// w != null: acc_0 (+)= in_0[perm(x)] + w_0, acc_1 (+)= w_1 (in = the inner
// sum, w = the key inner product of its ModDown'd c1); w == null (no
// rotation): acc (+)= in.  All [B][2][nre][N].
__global__ void k_qp_giant_acc(uint64_t *acc, const uint64_t *in, const uint64_t *w, int B, int nl, int K, int logn,
                               uint32_t galois, ModTab mt, int pid_p0, int accumulate) {
    const int nre = nl + K;
    const uint32_t n = 1u << logn;
    const size_t total = ((size_t)B * 2 * nre) << logn;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(e & (n - 1));
        const size_t r = e >> logn;
        const int t = (int)(r % nre);
        const int h = (int)((r / nre) & 1);
        const int pid = t < nl ? t : pid_p0 + (t - nl);
        const uint64_t q = mt.q[pid];
        uint64_t v;
        if (!w) {
            v = in[e];
        } else {
            v = w[e];
            if (h == 0) {
                const uint32_t px = galois == 1 ? x : mm::galois_perm(x, galois, logn);
                v = mm::add_mod(v, in[((r << logn)) + px], q);
            }
        }
        acc[e] = accumulate ? mm::add_mod(acc[e], v, q) : v;
    }
}

// Rows of the special primes of a plan constant from its coefficient-form Q
// rows ([nl + K][N], rows 0..nl-1 given): the integer coefficient c is the
// centered residue of row 0, exact while |c| < q_0 / 2 (checked against row
// 1 when there is one: a mismatch sets *err), reduced mod every p_k.
__global__ void k_qp_extend(uint64_t *pt, int nl, int K, int logn, ModTab mt, int pid_p0, int *err) {
    const uint32_t n = 1u << logn;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const uint64_t q0 = mt.q[0], r0 = pt[x];
        const bool neg = r0 > (q0 >> 1);
        const uint64_t mag = neg ? q0 - r0 : r0;
        if (nl > 1) {
            const uint64_t q1 = mt.q[1], m1 = mag % q1;
            if ((neg ? (m1 ? q1 - m1 : 0) : m1) != pt[n + x]) atomicOr(err, 1);
        }
        for (int k = 0; k < K; k++) {
            const uint64_t pk = mt.q[pid_p0 + k], m = mag % pk;
            pt[((size_t)(nl + k) << logn) + x] = neg ? (m ? pk - m : 0) : m;
        }
    }
}

// Rows into (to = 1) or out of (to = 0) Montgomery form, in place.
__global__ void k_mont_convert(uint64_t *base, RowMap map, size_t rows, int logn, ModTab mt, int to) {
    const uint32_t n = 1u << logn;
    const size_t total = rows << logn;
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)(w >> logn);
        const uint8_t pid = map.pid[r % map.period];
        if (pid == SKIP) continue;
        uint64_t *p = base + (((size_t)(r / map.period) * map.block_stride + (r % map.period)) << logn) + (w & (n - 1));
        *p = to ? mulq(*p, mt.r64[pid], mt, pid) : mm::redc(0, *p, mt.q[pid], mt.qinv[pid]);
    }
}

// Tensor product accumulated with a small integer coefficient:
// d (+)= coef * (a0 b0, a0 b1 + a1 b0, a1 b1), per window b, limb i, word x.
__global__ void k_tensor(uint64_t *d, const uint64_t *a, const uint64_t *b, int B, int nl, int logn, ModTab mt,
                         long long coef, int accumulate) {
    const size_t per = (size_t)nl << logn;
    const size_t total = (size_t)B * per;
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
        size_t bb = w / per, rem = w - bb * per;
        int i = (int)(rem >> logn);
        uint64_t q = mt.q[i];
        const uint64_t *A = a + bb * 2 * per;
        const uint64_t *Bq = b + bb * 2 * per;
        uint64_t a0 = A[rem], a1 = A[per + rem], b0 = Bq[rem], b1 = Bq[per + rem];
        uint64_t t0 = mulq(a0, b0, mt, i);
        uint64_t t1 = mm::add_mod(mulq(a0, b1, mt, i), mulq(a1, b0, mt, i), q);
        uint64_t t2 = mulq(a1, b1, mt, i);
        if (coef != 1) {
            uint64_t cm = coef >= 0 ? (uint64_t)coef % q : (q - ((uint64_t)(-coef) % q)) % q;
            t0 = mulq(t0, cm, mt, i);
            t1 = mulq(t1, cm, mt, i);
            t2 = mulq(t2, cm, mt, i);
        }
        uint64_t *D = d + bb * 3 * per;
        if (accumulate) {
            D[rem] = mm::add_mod(D[rem], t0, q);
            D[per + rem] = mm::add_mod(D[per + rem], t1, q);
            D[2 * per + rem] = mm::add_mod(D[2 * per + rem], t2, q);
        } else {
            D[rem] = t0;
            D[per + rem] = t1;
            D[2 * per + rem] = t2;
        }
    }
}

// ModUp FastBConv of one level: for window b, digit j, word x:
//   y_u = [x_u * inv_{j,u}]_{q_u} (u over the digit's primes, coefficient form)
//   out[b][j][t][x] = sum_u y_u * M_{j,u,t} mod prime(t)      (t not in the digit)
//   out[b][j][t][x] = d_eval[b][t][x]                         (t in the digit)
// coef: [B][l+1][N] coefficient form of d; deval: d in the evaluation domain,
// window stride deval_stride words.
__global__ void k_modup_bconv(uint64_t *out, const uint64_t *coef, const uint64_t *deval, size_t deval_stride, int B,
                              int level, int beta, int alpha, int nrows_ext, int logn, ModTab mt, ModUpConsts mc) {
    const uint32_t n = 1u << logn;
    const size_t total = (size_t)B * beta * n;
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)(w & (n - 1));
        size_t bj = w >> logn;
        int j = (int)(bj % beta);
        size_t bb = bj / beta;
        int i0 = j * alpha;
        int cnt = min(alpha, level + 1 - i0);
        uint64_t y[MAX_ALPHA];
        const uint64_t *C = coef + (bb * (level + 1)) * n;
        for (int u = 0; u < cnt; u++) {
            int pi = i0 + u;
            y[u] = mm::mul_shoup(C[(size_t)pi * n + x], mc.inv[j * MAX_ALPHA + u], mc.inv_sh[j * MAX_ALPHA + u], mt.q[pi]);
        }
        uint64_t *O = out + ((bb * beta + j) * (size_t)nrows_ext) * n;
        const uint64_t *De = deval + bb * deval_stride;
        for (int t = 0; t < nrows_ext; t++) {
            if (t >= i0 && t < i0 + cnt) {
                O[(size_t)t * n + x] = De[(size_t)t * n + x];
                continue;
            }
            int pid = t <= level ? t : mc.pid_p0 + (t - level - 1);
            uint64_t qt = mt.q[pid];
            uint64_t acc = 0;
            for (int u = 0; u < cnt; u++) {
                size_t ci = ((size_t)j * MAX_ALPHA + u) * MAXROWMAP + t;
                acc += mm::mul_shoup_lazy(y[u], mc.m[ci], mc.m_sh[ci], qt);   // < 2q each
                acc = acc >= 2 * qt ? acc - 2 * qt : acc;
            }
            O[(size_t)t * n + x] = acc >= qt ? acc - qt : acc;
        }
    }
}

// Key inner product fused with the Galois permutation of the digits:
//   u_h[b][t][x] = sum_j digits[b][j][t][pi(x)] * key[j][h][krow(t)][x]
// A thread owns (t, x); the digit words of WG windows are loaded together.
// One key for every window: the thread holds the beta key words and walks all
// windows, so the key is read once per launch.  PW (a batch mixing users,
// key.k[b] for window b): a thread owns (t, x) for one group of WG windows.
// WG is picked by the autotuner (1, 2, 4 or 8).
template <int WG, bool PW, int KB>
__global__ void __launch_bounds__(EW_THREADS, WG <= 2 ? 4 : (WG == 4 ? 3 : 2))
    k_keyip(uint64_t *u, const uint64_t *digits, const uint64_t *own, size_t own_stride, size_t own_jstride,
            KeyPtrs key, int B, int level, int beta, int alpha, int nrows_ext, int key_rows, int L1, int logn,
            uint32_t galois, ModTab mt, int pid_p0) {
    const uint32_t n = 1u << logn;
    const size_t per_group = (size_t)nrows_ext * n;
    if (!PW) {
        // one key for every window: a thread keeps the beta key word pairs of
        // its (t, x) in registers and walks all windows, WG at a time, so the
        // key is read from memory once per launch
        for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < per_group;
             w += (size_t)gridDim.x * blockDim.x) {
            const uint32_t x = (uint32_t)(w & (n - 1));
            const int t = (int)(w >> logn);
            const int pid = t <= level ? t : pid_p0 + (t - level - 1);
            const int krow = t <= level ? t : L1 + (t - level - 1);
            const uint32_t px = galois == 1 ? x : mm::galois_perm(x, galois, logn);
            const uint64_t q = mt.q[pid], qinv = mt.qinv[pid];
            const int jown = t <= level ? t / alpha : -1;
            uint64_t kb[KB], ka[KB];   // beta <= KB
#pragma unroll
            for (int j = 0; j < KB; j++) {
                kb[j] = j < beta ? key.k[0][(((size_t)j * 2 + 0) * key_rows + krow) * n + x] : 0;
                ka[j] = j < beta ? key.k[0][(((size_t)j * 2 + 1) * key_rows + krow) * n + x] : 0;
            }
            auto walk = [&](auto small) {
                constexpr bool S = decltype(small)::value;
                for (int b0 = 0; b0 < B; b0 += WG) {
                    uint64_t h0[WG] = {}, l0[WG] = {}, h1[WG] = {}, l1[WG] = {};
#pragma unroll
                    for (int j = 0; j < KB; j++) {
                        if (j >= beta) break;
                        const uint64_t *src = j == jown ? own + j * own_jstride + (size_t)t * n + px
                                                        : digits + ((size_t)j * nrows_ext + t) * n + px;
                        const size_t wstride = j == jown ? own_stride : (size_t)beta * nrows_ext * n;
                        uint64_t dv[WG];
#pragma unroll
                        for (int k = 0; k < WG; k++) dv[k] = b0 + k < B ? src[(size_t)(b0 + k) * wstride] : 0;
#pragma unroll
                        for (int k = 0; k < WG; k++) {
                            macq<S>(h0[k], l0[k], dv[k], kb[j]);
                            macq<S>(h1[k], l1[k], dv[k], ka[j]);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < WG; k++) {
                        if (b0 + k >= B) break;
                        uint64_t *U = u + ((size_t)(b0 + k) * 2 * nrows_ext) * n;
                        U[(size_t)t * n + x] = mm::redc(h0[k], l0[k], q, qinv);
                        U[((size_t)nrows_ext + t) * n + x] = mm::redc(h1[k], l1[k], q, qinv);
                    }
                }
            };
            if (q < mm::SMALL_PRIME_LIMIT) walk(SmallT{});
            else walk(WideT{});
        }
        return;
    }
    const size_t total = per_group * (size_t)((B + WG - 1) / WG);
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
        const int b0 = (int)(w / per_group) * WG;
        const size_t tw = w % per_group;
        const uint32_t x = (uint32_t)(tw & (n - 1));
        const int t = (int)(tw >> logn);
        const int pid = t <= level ? t : pid_p0 + (t - level - 1);
        const int krow = t <= level ? t : L1 + (t - level - 1);
        const uint32_t px = galois == 1 ? x : mm::galois_perm(x, galois, logn);
        const uint64_t q = mt.q[pid], qinv = mt.qinv[pid];
        const int jown = t <= level ? t / alpha : -1;   // the digit whose own primes hold row t
        // keys are in Montgomery form: sum the 128-bit products of the digits
        // (beta q^2 < q 2^64 because beta <= 8 and q < 2^61), reduce once
        uint64_t h0[WG] = {}, l0[WG] = {}, h1[WG] = {}, l1[WG] = {};
        for (int j = 0; j < beta; j++) {
            const size_t kb_off = (((size_t)j * 2 + 0) * key_rows + krow) * n + x;
            const size_t ka_off = (((size_t)j * 2 + 1) * key_rows + krow) * n + x;
            uint64_t kb[PW ? WG : 1], ka[PW ? WG : 1];
            if (PW) {
#pragma unroll
                for (int k = 0; k < (PW ? WG : 1); k++) {
                    const uint64_t *K = key.k[b0 + k < B ? b0 + k : b0];
                    kb[k] = K[kb_off];
                    ka[k] = K[ka_off];
                }
            } else {
                kb[0] = key.k[0][kb_off];
                ka[0] = key.k[0][ka_off];
            }
            const uint64_t *src;
            size_t wstride;
            if (j == jown) {
                src = own + j * own_jstride + (size_t)t * n + px;
                wstride = own_stride;
            } else {
                src = digits + ((size_t)j * nrows_ext + t) * n + px;
                wstride = (size_t)beta * nrows_ext * n;
            }
            uint64_t dv[WG];
#pragma unroll
            for (int k = 0; k < WG; k++) dv[k] = b0 + k < B ? src[(size_t)(b0 + k) * wstride] : 0;
#pragma unroll
            for (int k = 0; k < WG; k++) {
                mm::mac128(h0[k], l0[k], dv[k], kb[PW ? k : 0]);
                mm::mac128(h1[k], l1[k], dv[k], ka[PW ? k : 0]);
            }
        }
#pragma unroll
        for (int k = 0; k < WG; k++) {
            if (b0 + k >= B) break;
            uint64_t *U = u + ((size_t)(b0 + k) * 2 * nrows_ext) * n;
            U[(size_t)t * n + x] = mm::redc(h0[k], l0[k], q, qinv);
            U[((size_t)nrows_ext + t) * n + x] = mm::redc(h1[k], l1[k], q, qinv);
        }
    }
}

// Asynchronous 8-byte copy global -> shared (completion tracked per thread).
__device__ __forceinline__ void cpa8(uint64_t *smem_dst, const uint64_t *gsrc) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int KEYIP_PIPE_THREADS = 128;

// The shared-key inner product of k_keyip with its window walk pipelined:
// a thread copies the digit words of its next group of WG windows into its
// own column of shared memory (asynchronous copies; it reads back only what
// it copied, so no barrier) while the current group's products run, so the
// loads of one group hide under the arithmetic of the previous one.  Same
// words as k_keyip.  beta <= KB.
template <int WG, int KB>
__global__ void __launch_bounds__(KEYIP_PIPE_THREADS, WG <= 4 ? 4 : 3)
    k_keyip_pipe(uint64_t *u, const uint64_t *digits, const uint64_t *own, size_t own_stride, size_t own_jstride,
                 KeyPtrs key, int B, int level, int beta, int alpha, int nrows_ext, int key_rows, int L1, int logn,
                 uint32_t galois, ModTab mt, int pid_p0) {
    extern __shared__ uint64_t kbuf[];   // [2][KB][WG][KEYIP_PIPE_THREADS]
    const int tid = threadIdx.x;
    auto at = [&](int s, int j, int k) -> uint64_t & {
        return kbuf[((s * KB + j) * WG + k) * KEYIP_PIPE_THREADS + tid];
    };
    const uint32_t n = 1u << logn;
    const size_t per_group = (size_t)nrows_ext * n;
    for (size_t w = blockIdx.x * (size_t)blockDim.x + tid; w < per_group; w += (size_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(w & (n - 1));
        const int t = (int)(w >> logn);
        const int pid = t <= level ? t : pid_p0 + (t - level - 1);
        const int krow = t <= level ? t : L1 + (t - level - 1);
        const uint32_t px = galois == 1 ? x : mm::galois_perm(x, galois, logn);
        const uint64_t q = mt.q[pid], qinv = mt.qinv[pid];
        const int jown = t <= level ? t / alpha : -1;
        uint64_t kb[KB], ka[KB];
        const uint64_t *src[KB];
        size_t ws[KB];
#pragma unroll
        for (int j = 0; j < KB; j++) {
            kb[j] = j < beta ? key.k[0][(((size_t)j * 2 + 0) * key_rows + krow) * n + x] : 0;
            ka[j] = j < beta ? key.k[0][(((size_t)j * 2 + 1) * key_rows + krow) * n + x] : 0;
            src[j] = j == jown ? own + j * own_jstride + (size_t)t * n + px : digits + ((size_t)j * nrows_ext + t) * n + px;
            ws[j] = j == jown ? own_stride : (size_t)beta * nrows_ext * n;
        }
        auto issue = [&](int b0, int s) {
#pragma unroll
            for (int j = 0; j < KB; j++)
#pragma unroll
                for (int k = 0; k < WG; k++)
                    if (j < beta && b0 + k < B) cpa8(&at(s, j, k), src[j] + (size_t)(b0 + k) * ws[j]);
            cpa_commit();
        };
        auto walk = [&](auto small) {
            constexpr bool S = decltype(small)::value;
            issue(0, 0);
            int s = 0;
            for (int b0 = 0; b0 < B; b0 += WG, s ^= 1) {
                if (b0 + WG < B) issue(b0 + WG, s ^ 1);
                else cpa_commit();   // an empty group keeps one group in flight behind this one
                cpa_wait<1>();       // this group's words have landed
                uint64_t h0[WG] = {}, l0[WG] = {}, h1[WG] = {}, l1[WG] = {};
#pragma unroll
                for (int j = 0; j < KB; j++) {
                    if (j >= beta) break;
#pragma unroll
                    for (int k = 0; k < WG; k++) {
                        const uint64_t dv = at(s, j, k);
                        macq<S>(h0[k], l0[k], dv, kb[j]);
                        macq<S>(h1[k], l1[k], dv, ka[j]);
                    }
                }
#pragma unroll
                for (int k = 0; k < WG; k++) {
                    if (b0 + k >= B) break;
                    uint64_t *U = u + ((size_t)(b0 + k) * 2 * nrows_ext) * n;
                    U[(size_t)t * n + x] = mm::redc(h0[k], l0[k], q, qinv);
                    U[((size_t)nrows_ext + t) * n + x] = mm::redc(h1[k], l1[k], q, qinv);
                }
            }
            cpa_wait<0>();
        };
        if (q < mm::SMALL_PRIME_LIMIT) walk(SmallT{});
        else walk(WideT{});
    }
}

// ModDown FastBConv P -> Q with centered representatives (coefficient form):
//   z_k = [u_{p_k} * Phat_k^-1]_{p_k}, negative representative when z_k > p_k/2
//   v_i = sum_k z_k * (Phat_k mod q_i) - c * (P mod q_i),  c = #negative z_k
// u: [B][2][l+1+K][N] with its P rows in coefficient form; v: [B][2][l+1][N].
__global__ void k_moddown_bconv(uint64_t *v, const uint64_t *u, int B, int level, int K, int logn, ModTab mt,
                                ModDownConsts dc) {
    const uint32_t n = 1u << logn;
    const int nre = level + 1 + K;
    const size_t total = (size_t)B * 2 * n;
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)(w & (n - 1));
        size_t bh = w >> logn;
        const uint64_t *U = u + bh * nre * n;
        uint64_t z[MMFHE_MAX_P];
        uint32_t negc = 0;
        for (int k = 0; k < K; k++) {
            uint64_t pk = mt.q[dc.pid_p0 + k];
            z[k] = mm::mul_shoup(U[(size_t)(level + 1 + k) * n + x], dc.pinv[k], dc.pinv_sh[k], pk);
            negc += z[k] > (pk >> 1) ? 1u : 0u;
        }
        uint64_t *V = v + bh * (level + 1) * n;
        for (int i = 0; i <= level; i++) {
            uint64_t q = mt.q[i];
            uint64_t acc = 0;
            for (int k = 0; k < K; k++) {
                size_t ci = (size_t)k * MMFHE_MAX_Q + i;
                acc += mm::mul_shoup_lazy(z[k], dc.phat[ci], dc.phat_sh[ci], q);
                acc = acc >= 2 * q ? acc - 2 * q : acc;
            }
            acc = acc >= q ? acc - q : acc;
            uint64_t corr = mm::mul_shoup(negc, dc.pmod[i], dc.pmod_sh[i], q);
            V[(size_t)i * n + x] = mm::sub_mod(acc, corr, q);
        }
    }
}

// out[b][h][i][x] = (u[b][h][i][x] - v[b][h][i][x]) * P^-1 mod q_i
//                   + add_h[b][i][perm(x)]   (add_h optional; perm = galois map)
__global__ void k_moddown_combine(uint64_t *out, const uint64_t *u, const uint64_t *v, const uint64_t *add0,
                                  const uint64_t *add1, size_t add_stride, uint32_t add_galois, int B, int level,
                                  int K, int logn, ModTab mt, ModDownConsts dc, const uint64_t *plus) {
    const uint32_t n = 1u << logn;
    const int nl = level + 1, nre = level + 1 + K;
    const size_t total = (size_t)B * 2 * nl * n;
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)(w & (n - 1));
        size_t r = w >> logn;
        int i = (int)(r % nl);
        size_t bh = r / nl;
        int h = (int)(bh & 1);
        size_t bb = bh >> 1;
        uint64_t q = mt.q[i];
        uint64_t uv = u[(bh * nre + i) * n + x];
        uint64_t vv = v[(bh * nl + i) * n + x];
        uint64_t res = mm::mul_shoup(mm::sub_mod(uv, vv, q), dc.Pinv[i], dc.Pinv_sh[i], q);
        const uint64_t *A = h == 0 ? add0 : add1;
        if (A) {
            uint32_t px = add_galois == 1 ? x : mm::galois_perm(x, add_galois, logn);
            res = mm::add_mod(res, A[bb * add_stride + (size_t)i * n + px], q);
        }
        if (plus) res = mm::add_mod(res, plus[w], q);   // same [B][2][l+1][N] layout as out
        out[w] = res;
    }
}

// Rescale, spread step: r = last limb (coefficient form, [B][2][N]) taken
// centered mod q_l, written as residues mod q_i for i < l into tmp [B][2][l][N].
__global__ void k_rescale_spread(uint64_t *tmp, const uint64_t *last, int B, int level, int logn, ModTab mt,
                                 RescaleConsts rc) {
    const uint32_t n = 1u << logn;
    const size_t total = (size_t)B * 2 * n;
    const uint64_t ql = mt.q[level];
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)(w & (n - 1));
        size_t bh = w >> logn;
        uint64_t r = last[bh * n + x];
        bool neg = r > (ql >> 1);
        uint64_t *T = tmp + bh * (size_t)level * n;
        for (int i = 0; i < level; i++) {
            uint64_t q = mt.q[i];
            uint64_t ri = mm::reduce_barrett(r, q, mt.mu[i], mt.k[i]);
            if (neg) ri = mm::sub_mod(ri, rc.qmod[i], q);   // r - q_l
            T[(size_t)i * n + x] = ri;
        }
    }
}

// out[b][h][i][x] = (c[b][h][i][x] - tmp[b][h][i][x]) * q_l^-1 mod q_i, i < l.
__global__ void k_rescale_combine(uint64_t *out, const uint64_t *c, const uint64_t *tmp, int B, int level, int logn,
                                  ModTab mt, RescaleConsts rc) {
    const uint32_t n = 1u << logn;
    const size_t total = (size_t)B * 2 * level * n;
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)(w & (n - 1));
        size_t r = w >> logn;
        int i = (int)(r % level);
        size_t bh = r / level;
        uint64_t q = mt.q[i];
        uint64_t cv = c[(bh * (level + 1) + i) * n + x];
        out[w] = mm::mul_shoup(mm::sub_mod(cv, tmp[w], q), rc.qinv[i], rc.qinv_sh[i], q);
    }
}

// out[w] (+)= sum_k ct_k[w] * pt_k[row(w)][x]: one read of every term, one
// write of the output (the BSGS inner sum of a giant step).  The constants of
// a giant step stay in L2 across the batch.
__global__ void k_mul_plain_sum(uint64_t *out, SumTerms terms, size_t words, int logn, int nl, ModTab mt,
                                int accumulate) {
    const uint32_t n = 1u << logn;
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < words; w += (size_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(w & (n - 1));
        const int i = (int)((w >> logn) % nl);
        const size_t poff = ((size_t)i << logn) + x;
        const uint64_t q = mt.q[i], qinv = mt.qinv[i];
        // constants are in Montgomery form: 128-bit sum of products, one reduction
        // (the launcher keeps terms.n * q < 2^64)
        uint64_t hi = 0, lo = 0;
        for (int t = 0; t < terms.n; t++) mm::mac128(hi, lo, __ldg(terms.ct[t] + w), __ldg(terms.pt[t] + poff));
        uint64_t v = mm::redc(hi, lo, q, qinv);
        out[w] = accumulate ? mm::add_mod(out[w], v, q) : v;
    }
}

// out[w] (+)= sum_k ct_k[w] * s_k[row(w)]: a linear combination of ciphertext
// batches with scalar constants (constant polynomials: the same residue at
// every position of a limb), the scalars in Montgomery form, one reduction.
__global__ void k_lincomb(uint64_t *out, LincombTerms terms, size_t words, int logn, int nl, ModTab mt,
                          int accumulate) {
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < words; w += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)((w >> logn) % nl);
        const uint64_t q = mt.q[i], qinv = mt.qinv[i];
        uint64_t hi = 0, lo = 0;
        for (int t = 0; t < terms.n; t++) mm::mac128(hi, lo, __ldg(terms.ct[t] + w), terms.s[t][i]);
        const uint64_t v = mm::redc(hi, lo, q, qinv);
        out[w] = accumulate ? mm::add_mod(out[w], v, q) : v;
    }
}

// Automorphism of whole rows in the evaluation domain.
__global__ void k_permute(uint64_t *out, const uint64_t *in, size_t rows, int logn, uint32_t galois) {
    const uint32_t n = 1u << logn;
    const size_t total = rows * n;
    for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)(w & (n - 1));
        out[w] = in[(w - x) + mm::galois_perm(x, galois, logn)];
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
#define LAUNCH(c, name, bytes, g, kern, ...)                  \
    do {                                                      \
        kernel_begin(c, st);                                  \
        kern<<<g, EW_THREADS, 0, st>>>(__VA_ARGS__);          \
        kernel_end(c, name, g, dim3(EW_THREADS), bytes, st);  \
        CK(cudaGetLastError());                               \
    } while (0)

// Algorithmic bytes: every distinct word a launch must read or write once.
static inline double W8(size_t words) { return 8.0 * (double)words; }

void k_launch_addsub(Context &c, uint64_t *out, const uint64_t *a, const uint64_t *b, size_t rows, const PidList &pl,
                     uint32_t period, bool sub, cudaStream_t st) {
    size_t words = rows << c.logn;
    if (!words) return;
    dim3 g = grid_for(words);
    LAUNCH(c, sub ? "sub" : "add", W8(3 * words), g, k_addsub, out, a, b, words, c.logn, period, c.mods, pl,
           sub ? 1 : 0);
}

void k_launch_mul_int(Context &c, uint64_t *out, const uint64_t *a, size_t rows, const PidList &pl, uint32_t period,
                      long long k, cudaStream_t st) {
    size_t words = rows << c.logn;
    if (!words) return;
    dim3 g = grid_for(words);
    LAUNCH(c, "mul_int", W8(2 * words), g, k_mul_int, out, a, words, c.logn, period, c.mods, pl, k);
}

void k_launch_mul_plain(Context &c, uint64_t *out, const uint64_t *a, const uint64_t *pt, size_t rows,
                        const PidList &pl, uint32_t period, bool acc, cudaStream_t st, bool mont) {
    size_t words = rows << c.logn;
    if (!words) return;
    dim3 g = grid_for(words);
    double bytes = W8((acc ? 3 : 2) * words + ((size_t)period << c.logn));
    LAUNCH(c, acc ? "mul_plain_acc" : "mul_plain", bytes, g, k_mul_plain, out, a, pt, words, c.logn, period, c.mods,
           pl, acc ? 1 : 0, mont ? 1 : 0);
}

void k_launch_add_plain(Context &c, uint64_t *ct, const uint64_t *pt, int B, int level, cudaStream_t st) {
    const int nl = level + 1;
    const size_t words = ((size_t)B * nl) << c.logn;
    if (!words) return;
    dim3 g = grid_for(words);
    LAUNCH(c, "add_plain", W8(2 * words + ((size_t)nl << c.logn)), g, k_add_plain, ct, pt, words, c.logn, nl, c.mods);
}

void k_launch_group_sum(Context &c, uint64_t *out, const uint64_t *in, int B, int G, int level, cudaStream_t st) {
    const int nl = level + 1;
    const size_t wpc = ((size_t)2 * nl) << c.logn, words = (size_t)B * wpc;
    if (!words) return;
    dim3 g = grid_for(words);
    LAUNCH(c, "group_sum", W8(words * (size_t)(G + 1)), g, k_group_sum, out, in, words, wpc, G, c.logn, nl, c.mods);
}

void k_launch_mont_convert(Context &c, const RowsView &v, bool to, cudaStream_t st) {
    size_t words = v.rows << c.logn;
    if (!words) return;
    dim3 g = grid_for(words);
    LAUNCH(c, to ? "to_mont" : "from_mont", W8(2 * words), g, k_mont_convert, v.base, v.map, v.rows, c.logn, c.mods,
           to ? 1 : 0);
}

void k_launch_tensor(Context &c, uint64_t *d, const uint64_t *a, const uint64_t *b, int B, int level, long long coef,
                     bool acc, cudaStream_t st) {
    size_t work = (size_t)B * (level + 1) * c.n;
    if (!work) return;
    dim3 g = grid_for(work);
    LAUNCH(c, "tensor", W8(work * (4 + (acc ? 6 : 3))), g, k_tensor, d, a, b, B, level + 1, c.logn, c.mods, coef,
           acc ? 1 : 0);
}

void k_launch_modup_bconv(Context &c, uint64_t *out, const uint64_t *coef, const uint64_t *deval, size_t deval_stride,
                          int B, int level, const ModUpConsts &mc, cudaStream_t st) {
    const LevelConsts &lc = c.lv[level];
    size_t work = (size_t)B * lc.beta * c.n;
    if (!work) return;
    dim3 g = grid_for(work);
    const size_t nl = level + 1, nre = nl + c.num_p;
    // reads: coefficient rows + evaluation rows of d; writes: every digit row
    double bytes = W8((size_t)B * c.n * (2 * nl + lc.beta * nre));
    LAUNCH(c, "modup_bconv", bytes, g, k_modup_bconv, out, coef, deval, deval_stride, B, level, lc.beta, c.alpha,
           level + 1 + c.num_p, c.logn, c.mods, mc);
}

void k_launch_keyip(Context &c, uint64_t *u, const uint64_t *digits, const uint64_t *own, size_t own_stride,
                    size_t own_jstride, const KeyPtrs &key, int B, int level, int beta, uint32_t galois,
                    cudaStream_t st) {
    if (key.n != 1 && key.n != B) throw Error(MMFHE_ERR_BAD_ARG, "keyip: one key or one per window");
    const bool pw = key.n > 1;
    int nre = level + 1 + c.num_p;
    size_t work = (size_t)nre * c.n;
    const int wg = c.tune.keyip_wg;
    // shared key: one thread per (t, x) walks the windows; per-window keys: one per (t, x, window group)
    dim3 g = grid_for(pw ? work * (size_t)((B + wg - 1) / wg) : work);
    // reads: B*beta digit rows + beta*2 key rows (per window when mixing users); writes: B*2 output rows
    double bytes = W8(work * ((size_t)B * beta + 2 * beta * (size_t)key.n + 2 * B));
    auto go = [&](auto wg_c, auto pw_c) {
        constexpr int WG = decltype(wg_c)::value;
        constexpr bool PW = decltype(pw_c)::value;
        if (!PW && c.tune.keyip_pipe && beta <= 4) {
            const size_t smem = (size_t)2 * 4 * WG * KEYIP_PIPE_THREADS * 8;
            static bool opted = false;
            if (!opted) {
                if (smem > 48 * 1024)
                    CK(cudaFuncSetAttribute(k_keyip_pipe<WG, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem));
                opted = true;
            }
            dim3 gp((unsigned)std::min<size_t>((work + KEYIP_PIPE_THREADS - 1) / KEYIP_PIPE_THREADS, 148 * 64));
            kernel_begin(c, st);
            k_keyip_pipe<WG, 4><<<gp, KEYIP_PIPE_THREADS, smem, st>>>(u, digits, own, own_stride, own_jstride, key,
                                                                     B, level, beta, c.alpha, nre,
                                                                     c.num_q + c.num_p, c.num_q, c.logn, galois,
                                                                     c.mods, c.num_q);
            kernel_end(c, "keyip", gp, dim3(KEYIP_PIPE_THREADS), bytes, st);
            CK(cudaGetLastError());
            return;
        }
        kernel_begin(c, st);
        auto kern = beta <= 4 ? k_keyip<WG, PW, 4> : k_keyip<WG, PW, MAX_DNUM>;
        kern<<<g, EW_THREADS, 0, st>>>(u, digits, own, own_stride, own_jstride, key, B, level, beta, c.alpha,
                                                  nre, c.num_q + c.num_p, c.num_q, c.logn, galois, c.mods, c.num_q);
        kernel_end(c, "keyip", g, dim3(EW_THREADS), bytes, st);
        CK(cudaGetLastError());
    };
    using T = std::true_type;
    using F = std::false_type;
    switch (wg) {
    case 1: pw ? go(std::integral_constant<int, 1>{}, T{}) : go(std::integral_constant<int, 1>{}, F{}); break;
    case 2: pw ? go(std::integral_constant<int, 2>{}, T{}) : go(std::integral_constant<int, 2>{}, F{}); break;
    case 8: pw ? go(std::integral_constant<int, 8>{}, T{}) : go(std::integral_constant<int, 8>{}, F{}); break;
    default: pw ? go(std::integral_constant<int, 4>{}, T{}) : go(std::integral_constant<int, 4>{}, F{}); break;
    }
}

void k_launch_moddown_bconv(Context &c, uint64_t *v, const uint64_t *u, int B, int level, const ModDownConsts &dc,
                            cudaStream_t st) {
    size_t work = (size_t)B * 2 * c.n;
    dim3 g = grid_for(work);
    double bytes = W8(work * (c.num_p + level + 1));
    LAUNCH(c, "moddown_bconv", bytes, g, k_moddown_bconv, v, u, B, level, c.num_p, c.logn, c.mods, dc);
}

void k_launch_moddown_combine(Context &c, uint64_t *out, const uint64_t *u, const uint64_t *v, const uint64_t *add0,
                              const uint64_t *add1, size_t add_stride, uint32_t add_galois, int B, int level,
                              const ModDownConsts &dc, cudaStream_t st, const uint64_t *plus) {
    size_t work = (size_t)B * 2 * (level + 1) * c.n;
    dim3 g = grid_for(work);
    double bytes = W8(work * 3 + (add0 ? work / 2 : 0) + (add1 ? work / 2 : 0) + (plus ? work : 0));
    LAUNCH(c, "moddown_combine", bytes, g, k_moddown_combine, out, u, v, add0, add1, add_stride, add_galois, B, level,
           c.num_p, c.logn, c.mods, dc, plus);
}

void k_launch_rescale_spread(Context &c, uint64_t *tmp, const uint64_t *last, int B, int level,
                             const RescaleConsts &rc, cudaStream_t st) {
    size_t work = (size_t)B * 2 * c.n;
    dim3 g = grid_for(work);
    LAUNCH(c, "rescale_spread", W8(work * (1 + level)), g, k_rescale_spread, tmp, last, B, level, c.logn, c.mods, rc);
}

void k_launch_rescale_combine(Context &c, uint64_t *out, const uint64_t *cc, const uint64_t *tmp, int B, int level,
                              const RescaleConsts &rc, cudaStream_t st) {
    size_t work = (size_t)B * 2 * level * c.n;
    dim3 g = grid_for(work);
    LAUNCH(c, "rescale_combine", W8(3 * work), g, k_rescale_combine, out, cc, tmp, B, level, c.logn, c.mods, rc);
}

void k_launch_mul_plain_sum(Context &c, uint64_t *out, const SumTerms &terms, int B, int level, bool acc,
                            cudaStream_t st) {
    const int nl = level + 1;
    size_t words = (size_t)B * 2 * nl * c.n;
    if (!words || terms.n == 0) return;
    if (terms.n > c.sum_terms_max) throw Error(MMFHE_ERR_BAD_ARG, "mul_plain_sum: too many terms for one reduction");
    dim3 g = grid_for(words);
    // reads every term once, its constant once, writes (and reads, when accumulating) the output
    double bytes = W8(words * (terms.n + (acc ? 2 : 1)) + (size_t)terms.n * nl * c.n);
    LAUNCH(c, "mul_plain_sum", bytes, g, k_mul_plain_sum, out, terms, words, c.logn, nl, c.mods, acc ? 1 : 0);
}

void k_launch_mul_plain_sum_multi(Context &c, const MultiSumTerms &terms, int B, int level, bool acc,
                                  cudaStream_t st, bool qp) {
    const int nl = qp ? level + 1 + c.num_p : level + 1;   // rows per part (extended basis: + K)
    if (B <= 0 || terms.ng <= 0 || terms.nt <= 0) return;
    if (terms.ng > MULTI_SUM_GROUPS || terms.nt > MAX_SUM_TERMS || terms.nt > (qp ? c.sum_terms_max_qp : c.sum_terms_max))
        throw Error(MMFHE_ERR_BAD_ARG, "mul_plain_sum_multi: too many groups or terms");
    if (c.n % MULTI_X) throw Error(MMFHE_ERR_BAD_ARG, "mul_plain_sum_multi: ring too small");
    const int T = terms.nt <= 8 ? 8 : MAX_SUM_TERMS;
    const size_t smem = (size_t)terms.ng * T * MULTI_X * sizeof(uint64_t);
    const dim3 g((unsigned)((size_t)2 * nl * c.n / MULTI_X));
    const size_t words = (size_t)B * 2 * nl * c.n;
    // reads every baby step once and every constant once; writes (and reads, when accumulating) ng outputs
    const double bytes = W8(words * (size_t)(terms.nt + terms.ng * (acc ? 2 : 1)) +
                            (size_t)terms.ng * terms.nt * nl * c.n);
    auto go = [&](auto kern) {
        if (smem > 48 * 1024) CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kernel_begin(c, st);
        kern<<<g, MULTI_X, smem, st>>>(terms, B, c.logn, level + 1, nl, c.num_q, c.mods, acc ? 1 : 0);
        kernel_end(c, qp ? "mul_plain_sum_qp" : "mul_plain_sum", g, dim3(MULTI_X), bytes, st);
        CK(cudaGetLastError());
    };
    if (T == 8) go(k_mul_plain_sum_multi<8>);
    else go(k_mul_plain_sum_multi<MAX_SUM_TERMS>);
}

void k_launch_lincomb(Context &c, uint64_t *out, const LincombTerms &terms, int B, int level, bool acc,
                      cudaStream_t st) {
    const int nl = level + 1;
    const size_t words = (size_t)B * 2 * nl * c.n;
    if (!words || terms.n == 0) return;
    if (terms.n > c.sum_terms_max) throw Error(MMFHE_ERR_BAD_ARG, "lincomb: too many terms for one reduction");
    dim3 g = grid_for(words);
    LAUNCH(c, "lincomb", W8(words * (terms.n + (acc ? 2 : 1))), g, k_lincomb, out, terms, words, c.logn, nl, c.mods,
           acc ? 1 : 0);
}

void k_launch_qp_times_p(Context &c, uint64_t *out, const uint64_t *in, int B, int level, const ModDownConsts &dc,
                         cudaStream_t st) {
    const int nl = level + 1, K = c.num_p;
    const size_t work = (size_t)B * 2 * (nl + K) * c.n;
    if (!work) return;
    LAUNCH(c, "qp_times_p", W8(work + (size_t)B * 2 * nl * c.n), grid_for(work), k_qp_times_p, out, in, B, nl, K,
           c.logn, c.mods, dc);
}

void k_launch_qp_add_pc0(Context &c, uint64_t *u, const uint64_t *ct, int B, int level, uint32_t galois,
                         const ModDownConsts &dc, cudaStream_t st) {
    const int nl = level + 1;
    const size_t work = (size_t)B * nl * c.n;
    if (!work) return;
    LAUNCH(c, "qp_add_pc0", W8(3 * work), grid_for(work), k_qp_add_pc0, u, ct, B, nl, c.num_p, c.logn, galois,
           c.mods, dc);
}

void k_launch_qp_giant_acc(Context &c, uint64_t *acc, const uint64_t *in, const uint64_t *w, int B, int level,
                           uint32_t galois, bool accumulate, cudaStream_t st) {
    const int nl = level + 1;
    const size_t work = (size_t)B * 2 * (nl + c.num_p) * c.n;
    if (!work) return;
    // reads the term's operands (w and the c0 half of in, or all of in), writes acc (and reads it
    // when accumulating)
    const size_t operands = w ? work + work / 2 : work;
    const double bytes = W8(operands + work * (accumulate ? 2 : 1));
    LAUNCH(c, "qp_giant_acc", bytes, grid_for(work), k_qp_giant_acc, acc, in, w, B, nl, c.num_p, c.logn, galois,
           c.mods, c.num_q, accumulate ? 1 : 0);
}

void k_launch_qp_extend(Context &c, uint64_t *pt, int level, int *err, cudaStream_t st) {
    const int nl = level + 1;
    LAUNCH(c, "qp_extend", W8((size_t)(2 + c.num_p) * c.n), grid_for(c.n), k_qp_extend, pt, nl, c.num_p, c.logn,
           c.mods, c.num_q, err);
}

void k_launch_permute(Context &c, uint64_t *out, const uint64_t *in, size_t rows, uint32_t galois, cudaStream_t st) {
    size_t work = rows * c.n;
    if (!work) return;
    dim3 g = grid_for(work);
    LAUNCH(c, "permute", W8(2 * work), g, k_permute, out, in, rows, c.logn, galois);
}

}  // namespace mmfhe
