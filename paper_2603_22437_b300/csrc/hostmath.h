// Host-side integer helpers: 128-bit modular arithmetic, primality, roots.
#pragma once
#include <stdint.h>

#include <vector>

namespace mmfhe {
namespace hm {

typedef unsigned __int128 u128;

inline uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) { return (uint64_t)((u128)a * b % m); }

inline uint64_t powmod(uint64_t b, uint64_t e, uint64_t m) {
    uint64_t r = 1 % m;
    b %= m;
    while (e) {
        if (e & 1) r = mulmod(r, b, m);
        b = mulmod(b, b, m);
        e >>= 1;
    }
    return r;
}

// modular inverse for prime m
inline uint64_t invmod(uint64_t a, uint64_t m) { return powmod(a % m, m - 2, m); }

inline uint64_t shoup(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

inline uint32_t bitlen(uint64_t x) { return x ? 64 - __builtin_clzll(x) : 0; }

inline uint64_t barrett_mu(uint64_t q) {
    uint32_t k = bitlen(q);
    return (uint64_t)(((u128)1 << (2 * k)) / q);
}

// Deterministic Miller-Rabin for 64-bit integers (first 12 prime bases).
inline bool is_prime(uint64_t n) {
    if (n < 2) return false;
    static const uint64_t bases[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t p : bases) {
        if (n % p == 0) return n == p;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (uint64_t a : bases) {
        uint64_t x = powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s; r++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { comp = false; break; }
        }
        if (comp) return false;
    }
    return true;
}

// A primitive 2n-th root of unity mod q (q prime, q = 1 mod 2n): psi =
// x^((q-1)/2n) for the first odd x >= 3 with psi^n = -1.
inline uint64_t primitive_root_2n(uint64_t q, uint64_t n) {
    for (uint64_t x = 3;; x += 2) {
        uint64_t psi = powmod(x, (q - 1) / (2 * n), q);
        if (powmod(psi, n, q) == q - 1) return psi;
    }
}

inline uint32_t bitrev(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

}  // namespace hm
}  // namespace mmfhe
