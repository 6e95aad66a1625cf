"""CKKS parameter sets and their arithmetic (test infrastructure only).

The paper fixes the scheme (CKKS, ring dimension N = 32768, multiplicative
depth 11, 128-bit classical security per the HE Standard, FLEXIBLEAUTO
scaling; Table 7 and the HE primer) and the scale (Delta = 2^40 for vital
signs, 2^50 for gestures; Sec. "Defense Against CKKS-Specific Attacks").  It
does not print the primes, the number of special primes or dnum.  The reading
used here (Table 5's key and ciphertext sizes force dnum = 3 with four special
primes at N = 2^15):

* Q = q_0 * q_1 * ... * q_L with q_0 of ``q0_bits`` bits and q_1..q_L near
  2^``q_bits``; P = p_0 ... p_{K-1} of ``p_bits`` bits; every prime is
  congruent to 1 mod 2N so a negacyclic NTT exists.
* Deterministic selection rule (shared by the CUDA library's own selector,
  written independently):
    1. q_0 = largest prime < 2^q0_bits with q = 1 mod 2N;
    2. q_1.. q_L alternate between the largest unused prime below 2^q_bits and
       the smallest unused prime above 2^q_bits (below first), which keeps
       the running scale Delta^2/q_l close to Delta;
    3. p_0..p_{K-1} = the largest unused primes < 2^p_bits, descending.
* Digits: the Q primes are cut into dnum groups of alpha = ceil((L+1)/dnum)
  consecutive primes (hybrid key switching).
"""
import math
from dataclasses import dataclass, field

# HE Standard (homomorphicencryption.org, 2018), classical 128-bit security,
# ternary secret: maximum log2(QP) per ring dimension.
HE_STD_128_MAX_LOGQP = {1024: 27, 2048: 54, 4096: 109, 8192: 218, 16384: 438, 32768: 881, 65536: 1772}


def is_prime(n):
    """Deterministic Miller-Rabin, exact for n < 3.3e24 (first 12 prime bases)."""
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for p in small:
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in small:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def _below(bits, m, exclude):
    """Largest primes < 2^bits with p = 1 mod m, skipping ``exclude`` (generator)."""
    c = ((1 << bits) - 1) // m * m + 1
    if c >= (1 << bits):
        c -= m
    while c > m:
        if c not in exclude and is_prime(c):
            yield c
        c -= m


def _above(bits, m, exclude):
    c = (1 << bits) // m * m + 1
    if c <= (1 << bits):
        c += m
    while True:
        if c not in exclude and is_prime(c):
            yield c
        c += m


def select_primes(log_n, num_q, q0_bits, q_bits, num_p, p_bits):
    """Deterministic prime chain (rule in the module docstring)."""
    m = 2 << log_n
    used = set()
    q0 = next(_below(q0_bits, m, used))
    used.add(q0)
    qs = [q0]
    for i in range(1, num_q):
        gen = _below(q_bits, m, used) if i % 2 == 1 else _above(q_bits, m, used)
        p = next(gen)
        used.add(p)
        qs.append(p)
    ps = []
    for _ in range(num_p):
        p = next(_below(p_bits, m, used))
        used.add(p)
        ps.append(p)
    return qs, ps


def primitive_2n_root(q, n):
    """Smallest-base primitive 2n-th root of unity mod q: psi = x^((q-1)/2n)
    for the first x >= 2 with psi^n = -1 mod q."""
    assert (q - 1) % (2 * n) == 0
    for x in range(2, q):
        psi = pow(x, (q - 1) // (2 * n), q)
        if pow(psi, n, q) == q - 1:
            return psi
    raise ValueError("no root")


@dataclass
class Params:
    log_n: int
    q: list            # Q primes q_0..q_L
    p: list            # special primes p_0..p_{K-1}
    dnum: int
    scale: float       # Delta
    psi: dict = field(default_factory=dict)

    def __post_init__(self):
        n = self.n
        for prime in self.q + self.p:
            assert is_prime(prime) and prime % (2 * n) == 1 and prime < (1 << 62)
            self.psi[prime] = primitive_2n_root(prime, n)

    @property
    def n(self):
        return 1 << self.log_n

    @property
    def slots(self):
        return self.n // 2

    @property
    def L(self):
        """Top level (number of Q primes minus one)."""
        return len(self.q) - 1

    @property
    def alpha(self):
        return -(-len(self.q) // self.dnum)

    def digits(self, level):
        """Prime indices of each key-switching digit at ``level`` (the last
        digit may be partial or absent below the top level)."""
        a = self.alpha
        out = []
        for j in range(self.dnum):
            d = [i for i in range(j * a, min((j + 1) * a, level + 1))]
            if d:
                out.append(d)
        return out

    def log_qp(self):
        return sum(math.log2(x) for x in self.q + self.p)

    def ct_bytes(self, level):
        return 2 * (level + 1) * self.n * 8

    def key_bytes(self):
        """One switching key: dnum digits x 2 polynomials over Q_L * P."""
        return self.dnum * 2 * (len(self.q) + len(self.p)) * self.n * 8


def make_params(log_n, num_q, q0_bits, q_bits, num_p, p_bits, dnum, log_scale):
    qs, ps = select_primes(log_n, num_q, q0_bits, q_bits, num_p, p_bits)
    return Params(log_n=log_n, q=qs, p=ps, dnum=dnum, scale=float(2 ** log_scale))


# Parameter sets of the two workloads (reading in the module docstring).
def fir_dft_params():
    """Small instance: N = 2^13, q_0 ~ 2^44 and three ~2^40 primes, one 44-bit
    special prime, dnum = 4 (alpha = 1); log QP ~ 208 <= 218."""
    return make_params(13, 4, 44, 40, 1, 44, 4, 40)


def vital_params():
    """Vital-sign chain: N = 2^15, depth 11 (12 Q primes: 60 + 11 x 40 bits),
    four 60-bit special primes, dnum = 3 (alpha = 4); log QP ~ 740 <= 881."""
    return make_params(15, 12, 60, 40, 4, 60, 3, 40)


def fc_params():
    """Polynomial-network instance (encrypted FC network of depth 5: three
    dense layers and two squares): N = 2^14, q_0 ~ 2^60 and five ~2^40
    primes, two 60-bit special primes, dnum = 3 (alpha = 2);
    log QP ~ 380 <= 438 (HE Standard, N = 2^14, 128-bit classical)."""
    return make_params(14, 6, 60, 40, 2, 60, 3, 40)


def gesture_learned_params():
    """Gesture chain with the learned degree-2 feature map: depth 9 (10 Q
    primes: 60 + 9 x 50 bits, Delta = 2^50), four 60-bit special primes,
    dnum = 3; log QP ~ 750 <= 881."""
    return make_params(15, 10, 60, 50, 4, 60, 3, 50)


def gesture_params():
    """Gesture chain: N = 2^15, depth 11 (12 Q primes: 60 + 11 x 50 bits,
    Delta = 2^50), four 60-bit special primes, dnum = 3 (alpha = 4);
    log QP ~ 850 <= 881."""
    return make_params(15, 12, 60, 50, 4, 60, 3, 50)
