// Word-level modular arithmetic for 64-bit RNS limbs (primes q < 2^61).
//
// Two reductions are used:
//  * Barrett (Handbook of Applied Cryptography, Alg. 14.42, radix 2): for a
//    product z = a*b of two residues, z < q^2 < 2^(2k) with k = bitlen(q),
//    mu = floor(2^(2k) / q); qhat = floor(floor(z / 2^(k-1)) * mu / 2^(k+1));
//    z - qhat*q lies in [0, 3q).
//  * Shoup: multiplication by a fixed w < q with w' = floor(w * 2^64 / q):
//    a*w - floor(a*w'/2^64)*q lies in [0, 2q) for any 64-bit a.
// Both are written as __host__ __device__ so the host test harness runs the
// exact same code.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define MM_HD __host__ __device__ __forceinline__
#else
#define MM_HD inline
#endif

namespace mm {

MM_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// a*b mod q for a, b in [0, q).
MM_HD uint64_t mul_barrett(uint64_t a, uint64_t b, uint64_t q, uint64_t mu, uint32_t k) {
    uint64_t lo = a * b;
    uint64_t hi = mulhi64(a, b);
    uint64_t x = (hi << (65 - k)) | (lo >> (k - 1));          // floor(z / 2^(k-1)) < 2^(k+1)
    uint64_t tl = x * mu;
    uint64_t th = mulhi64(x, mu);
    uint64_t qhat = (th << (63 - k)) | (tl >> (k + 1));      // floor(x mu / 2^(k+1))
    uint64_t r = lo - qhat * q;                               // in [0, 3q), exact mod 2^64
    r = r >= q ? r - q : r;
    r = r >= q ? r - q : r;
    return r;
}

// x mod q for any x < 2^(2k) given as one 64-bit word (x < 2^64).
MM_HD uint64_t reduce_barrett(uint64_t x, uint64_t q, uint64_t mu, uint32_t k) {
    uint64_t xs = x >> (k - 1);
    uint64_t qhat = (mulhi64(xs, mu) << (63 - k)) | ((xs * mu) >> (k + 1));
    uint64_t r = x - qhat * q;
    r = r >= q ? r - q : r;
    r = r >= q ? r - q : r;
    return r;
}

// Shoup product, lazy: result in [0, 2q) for any a < 2^64.
MM_HD uint64_t mul_shoup_lazy(uint64_t a, uint64_t w, uint64_t wp, uint64_t q) {
    uint64_t qh = mulhi64(a, wp);
    return a * w - qh * q;
}

MM_HD uint64_t mul_shoup(uint64_t a, uint64_t w, uint64_t wp, uint64_t q) {
    uint64_t r = mul_shoup_lazy(a, w, wp, q);
    return r >= q ? r - q : r;
}

MM_HD uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q) {
    uint64_t s = a + b;
    return s >= q ? s - q : s;
}

MM_HD uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q) {
    return a >= b ? a - b : a + q - b;
}

// Montgomery reduction (R = 2^64): for T = hi*2^64 + lo < q*2^64, q odd,
// qinv = q^-1 mod 2^64, returns T * 2^-64 mod q in [0, q).  With
// m = lo*qinv, T - m*q is divisible by 2^64 and (T - m*q)/2^64 = hi - mulhi(m, q)
// lies in (-q, q).
MM_HD uint64_t redc(uint64_t hi, uint64_t lo, uint64_t q, uint64_t qinv) {
    uint64_t m = lo * qinv;
    uint64_t mh = mulhi64(m, q);
    return hi >= mh ? hi - mh : hi - mh + q;
}

// 128-bit multiply-accumulate (hi:lo) += a*b.
MM_HD void mac128(uint64_t &hi, uint64_t &lo, uint64_t a, uint64_t b) {
    uint64_t pl = a * b, ph = mulhi64(a, b);
    lo += pl;
    hi += ph + (lo < pl ? 1 : 0);
}

// (hi:lo) += a*b for a, b < 2^48 (residues, lazy or not, of primes below
// 2^47): with a = a1 2^32 + a0 and b = b1 2^32 + b0, a*b = a0 b0 +
// (a0 b1 + a1 b0) 2^32 + a1 b1 2^64, where the middle sum stays below 2^49
// and a1 b1 below 2^32, so three 32 x 32 -> 64 products and one 32-bit
// product replace the two 64 x 64 halves of the general case.
MM_HD void mac128_small(uint64_t &hi, uint64_t &lo, uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), b0 = (uint32_t)b, b1 = (uint32_t)(b >> 32);
    const uint64_t p0 = (uint64_t)a0 * b0;
    const uint64_t m = (uint64_t)a0 * b1 + (uint64_t)a1 * b0;
    const uint64_t top = a1 * b1;
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(p0), "l"(top));
    asm("add.cc.u64 %0, %0, %2;\n\taddc.u64 %1, %1, %3;" : "+l"(lo), "+l"(hi) : "l"(m << 32), "l"(m >> 32));
#else
    const unsigned __int128 t = (((unsigned __int128)hi << 64) | lo) + (unsigned __int128)a * b;
    hi = (uint64_t)(t >> 64);
    lo = (uint64_t)t;
#endif
}

// Primes whose residues take mac128_small.
constexpr uint64_t SMALL_PRIME_LIMIT = 1ull << 47;

// Reduce x in [0, 4q) to [0, q).
MM_HD uint64_t reduce_4q(uint64_t x, uint64_t q) {
    uint64_t q2 = q << 1;
    x = x >= q2 ? x - q2 : x;
    return x >= q ? x - q : x;
}

// Harvey forward (Cooley-Tukey) butterfly: X, Y in [0, 4q) -> [0, 4q).
MM_HD void ct_butterfly(uint64_t &X, uint64_t &Y, uint64_t w, uint64_t wp, uint64_t q) {
    uint64_t q2 = q << 1;
    uint64_t x = X >= q2 ? X - q2 : X;
    uint64_t t = mul_shoup_lazy(Y, w, wp, q);
    X = x + t;
    Y = x - t + q2;
}

// Harvey inverse (Gentleman-Sande) butterfly: X, Y in [0, 2q) -> [0, 2q).
MM_HD void gs_butterfly(uint64_t &X, uint64_t &Y, uint64_t w, uint64_t wp, uint64_t q) {
    uint64_t q2 = q << 1;
    uint64_t s = X + Y;
    uint64_t d = X - Y + q2;
    X = s >= q2 ? s - q2 : s;
    Y = mul_shoup_lazy(d, w, wp, q);
}

// Bit reversal of the low `bits` bits.
MM_HD uint32_t bitrev(uint32_t x, int bits) {
#if defined(__CUDA_ARCH__)
    return __brev(x) >> (32 - bits);
#else
    uint32_t r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
#endif
}

// Evaluation-domain Galois permutation: with row j holding a(psi^(2 brv(j) + 1)),
// (a o X^g) at position j equals a at position pi(j) where
// 2 brv(pi(j)) + 1 = (2 brv(j) + 1) g mod 2N.
MM_HD uint32_t galois_perm(uint32_t j, uint32_t g, int logn) {
    uint32_t two_n_mask = (2u << logn) - 1u;
    uint32_t e = 2u * bitrev(j, logn) + 1u;
    uint32_t eg = (uint32_t)(((uint64_t)e * g) & two_n_mask);
    return bitrev((eg - 1u) >> 1, logn);
}

}  // namespace mm
