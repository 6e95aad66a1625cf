/*
 * Oracle arithmetic core -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, obviously-correct modular arithmetic for the CPU oracle of the
 * RNS-CKKS evaluator (CKKS primer, "Three Primitive Operations"; Table 7 fixes
 * the scheme).  Every modular product is a 128-bit product followed by the
 * C '%' operator, every sum is fully reduced; nothing is fused.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * this library.  It shares no code with the CUDA path.
 *
 * Conventions: a "row" is N = 2^logn unsigned 64-bit residues of one
 * polynomial modulo one prime q (q < 2^62), coefficient order a_0 .. a_{N-1}
 * of a(X) in Z_q[X]/(X^N + 1).
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef uint64_t u64;

static u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
/* a, b in [0, q), q < 2^62 */
static u64 addmod(u64 a, u64 b, u64 q) { u64 s = a + b; return s >= q ? s - q : s; }
static u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

static u64 powmod(u64 b, u64 e, u64 q) {
    u64 r = 1 % q;
    b %= q;
    while (e) {
        if (e & 1) r = mulmod(r, b, q);
        b = mulmod(b, b, q);
        e >>= 1;
    }
    return r;
}

/* ---- element-wise vector operations (out may alias inputs) ---- */
void or_vec_add(u64 *out, const u64 *a, const u64 *b, size_t n, u64 q) {
    for (size_t i = 0; i < n; i++) out[i] = addmod(a[i] % q, b[i] % q, q);
}
void or_vec_sub(u64 *out, const u64 *a, const u64 *b, size_t n, u64 q) {
    for (size_t i = 0; i < n; i++) out[i] = submod(a[i] % q, b[i] % q, q);
}
void or_vec_neg(u64 *out, const u64 *a, size_t n, u64 q) {
    for (size_t i = 0; i < n; i++) out[i] = submod(0, a[i] % q, q);
}
void or_vec_mul(u64 *out, const u64 *a, const u64 *b, size_t n, u64 q) {
    for (size_t i = 0; i < n; i++) out[i] = mulmod(a[i], b[i], q);
}
/* out = a * s mod q, a[i] any 64-bit value, s any 64-bit value */
void or_vec_mul_scalar(u64 *out, const u64 *a, u64 s, size_t n, u64 q) {
    for (size_t i = 0; i < n; i++) out[i] = mulmod(a[i], s, q);
}
/* out = (acc + a * s) mod q */
void or_vec_mac_scalar(u64 *acc, const u64 *a, u64 s, size_t n, u64 q) {
    for (size_t i = 0; i < n; i++) acc[i] = addmod(acc[i] % q, mulmod(a[i], s, q), q);
}
/* out = a mod q for arbitrary 64-bit a */
void or_vec_mod(u64 *out, const u64 *a, size_t n, u64 q) {
    for (size_t i = 0; i < n; i++) out[i] = a[i] % q;
}
/* out = a mod q for signed 64-bit a (result in [0, q)) */
void or_vec_mod_signed(u64 *out, const int64_t *a, size_t n, u64 q) {
    for (size_t i = 0; i < n; i++) {
        int64_t v = a[i];
        if (v >= 0) out[i] = ((u64)v) % q;
        else {
            u64 m = ((u64)(-(v + 1)) + 1) % q;   /* |v| mod q without overflow */
            out[i] = m ? q - m : 0;
        }
    }
}

/* ---- negacyclic number-theoretic transform ----
 * Forward: A_j = a(psi^(2j+1)) = sum_k a_k psi^((2j+1)k) mod q, j = 0..N-1, in
 * natural order, where psi is a primitive 2N-th root of unity mod q.  It is
 * computed as the twist a_k <- a_k psi^k followed by a textbook cyclic radix-2
 * decimation-in-time transform with omega = psi^2 (bit-reversal permutation,
 * then log2 N butterfly stages).  Inverse undoes both steps exactly.
 */
static void bit_reverse(u64 *a, size_t n) {
    for (size_t i = 1, j = 0; i < n; i++) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { u64 t = a[i]; a[i] = a[j]; a[j] = t; }
    }
}

static void cyclic_ntt(u64 *a, size_t n, u64 omega, u64 q) {
    bit_reverse(a, n);
    for (size_t len = 2; len <= n; len <<= 1) {
        u64 wlen = powmod(omega, n / len, q);
        for (size_t i = 0; i < n; i += len) {
            u64 w = 1;
            for (size_t j = 0; j < len / 2; j++) {
                u64 u = a[i + j];
                u64 v = mulmod(a[i + j + len / 2], w, q);
                a[i + j] = addmod(u, v, q);
                a[i + j + len / 2] = submod(u, v, q);
                w = mulmod(w, wlen, q);
            }
        }
    }
}

void or_ntt_fwd(u64 *a, int logn, u64 q, u64 psi) {
    size_t n = (size_t)1 << logn;
    u64 pk = 1;
    for (size_t k = 0; k < n; k++) { a[k] = mulmod(a[k], pk, q); pk = mulmod(pk, psi, q); }
    cyclic_ntt(a, n, mulmod(psi, psi, q), q);
}

void or_ntt_inv(u64 *a, int logn, u64 q, u64 psi) {
    size_t n = (size_t)1 << logn;
    u64 psi_inv = powmod(psi, q - 2, q);
    cyclic_ntt(a, n, mulmod(psi_inv, psi_inv, q), q);
    u64 n_inv = powmod((u64)(n % q), q - 2, q);
    u64 pk = n_inv;
    for (size_t k = 0; k < n; k++) { a[k] = mulmod(a[k], pk, q); pk = mulmod(pk, psi_inv, q); }
}

/* Negacyclic product out = a * b in Z_q[X]/(X^N+1) via forward NTT of both
 * operands, point-wise product and inverse NTT. */
void or_polymul(u64 *out, const u64 *a, const u64 *b, int logn, u64 q, u64 psi) {
    size_t n = (size_t)1 << logn;
    u64 *fa = (u64 *)malloc(n * sizeof(u64));
    u64 *fb = (u64 *)malloc(n * sizeof(u64));
    memcpy(fa, a, n * sizeof(u64));
    memcpy(fb, b, n * sizeof(u64));
    or_ntt_fwd(fa, logn, q, psi);
    or_ntt_fwd(fb, logn, q, psi);
    for (size_t i = 0; i < n; i++) fa[i] = mulmod(fa[i], fb[i], q);
    or_ntt_inv(fa, logn, q, psi);
    memcpy(out, fa, n * sizeof(u64));
    free(fa);
    free(fb);
}

/* Galois automorphism sigma_g : a(X) -> a(X^g) on a coefficient row, g odd.
 * Coefficient k moves to index k*g mod 2N; landing in [N, 2N) negates it
 * because X^N = -1.  out must not alias a. */
void or_automorphism(u64 *out, const u64 *a, int logn, u64 g, u64 q) {
    size_t n = (size_t)1 << logn;
    u64 two_n = 2 * (u64)n;
    for (size_t k = 0; k < n; k++) {
        u64 idx = (u64)(((u128)k * g) % two_n);
        if (idx < n) out[idx] = a[k] % q;
        else out[idx - n] = submod(0, a[k] % q, q);
    }
}
