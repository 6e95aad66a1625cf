"""Pins of the oracle's arithmetic layer against mathematics that does not
depend on the oracle: schoolbook convolution, direct polynomial evaluation,
big-integer CRT and division, the HE-Standard bound and the paper's sizes."""
import json
import os

import numpy as np
import pytest
import sympy

from oracle import _native as nat
from oracle import ckks as ck
from oracle import params as pm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_prime(n, bits=30):
    return next(pm._below(bits, 2 * n, set()))


def schoolbook_negacyclic(a, b, q):
    n = len(a)
    c = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                c[k] += int(a[i]) * int(b[j])
            else:
                c[k - n] -= int(a[i]) * int(b[j])
    return [x % q for x in c]


@pytest.mark.parametrize("n", [8, 16, 64])
def test_polymul_equals_schoolbook(n):
    q = small_prime(n)
    psi = pm.primitive_2n_root(q, n)
    g = np.random.default_rng(n)
    a = g.integers(0, q, n, dtype=np.uint64)
    b = g.integers(0, q, n, dtype=np.uint64)
    assert [int(x) for x in nat.polymul(a, b, q, psi)] == schoolbook_negacyclic(a, b, q)


def test_polymul_60bit_prime_schoolbook():
    n = 16
    q = next(pm._below(60, 2 * n, set()))
    psi = pm.primitive_2n_root(q, n)
    g = np.random.default_rng(1)
    a = g.integers(0, q, n, dtype=np.uint64)
    b = g.integers(0, q, n, dtype=np.uint64)
    assert [int(x) for x in nat.polymul(a, b, q, psi)] == schoolbook_negacyclic(a, b, q)


def test_ntt_is_evaluation_at_odd_powers_and_inverts():
    n = 16
    q = small_prime(n)
    psi = pm.primitive_2n_root(q, n)
    a = np.arange(1, n + 1, dtype=np.uint64) * 7919 % q
    A = nat.ntt_fwd(a, q, psi)
    for j in range(n):
        x = pow(psi, 2 * j + 1, q)
        assert int(A[j]) == sum(int(a[k]) * pow(x, k, q) for k in range(n)) % q
    assert np.array_equal(nat.ntt_inv(A, q, psi), a)


def test_automorphism_is_substitution():
    n, g = 16, 5
    q = small_prime(n)
    a = np.arange(n, dtype=np.uint64) + 3
    out = nat.automorphism(a, g, q)
    # a(X^g) evaluated at a root of X^n + 1 equals out evaluated there
    psi = pm.primitive_2n_root(q, n)
    for e in (1, 3, 7):
        x = pow(psi, e, q)
        lhs = sum(int(a[k]) * pow(x, k * g, q) for k in range(n)) % q
        rhs = sum(int(out[k]) * pow(x, k, q) for k in range(n)) % q
        assert lhs == rhs


@pytest.mark.parametrize("maker,log_n", [(pm.fir_dft_params, 13), (pm.vital_params, 15)])
def test_prime_chain_rule_and_security(maker, log_n):
    P = maker()
    m = 2 << log_n
    allp = P.q + P.p
    assert len(set(allp)) == len(allp)
    for x in allp:
        assert sympy.isprime(x) and x % m == 1 and x < 2 ** 61
    # q_1.. alternate below / above 2^q_bits
    qb = 40
    for i, x in enumerate(P.q[1:], start=1):
        assert (x < 2 ** qb) if i % 2 == 1 else (x > 2 ** qb)
    # 128-bit classical security bound of the HE Standard for this N
    assert P.log_qp() <= pm.HE_STD_128_MAX_LOGQP[P.n]
    assert P.alpha <= len(P.p)


def test_largest_prime_below_is_largest():
    # q_0 is the largest prime = 1 mod 2N below 2^bits: no larger candidate is prime
    P = pm.vital_params()
    m = 2 * P.n
    c = P.q[0] + m
    while c < 2 ** 60:
        assert not sympy.isprime(c)
        c += m


def test_table5_size_arithmetic():
    gold = json.load(open(os.path.join(GOLDEN, "table5_sizes.json")))
    mib = 2 ** 20
    N, K, dnum = 32768, 4, 3
    for app, limbs in (("vital", 11), ("gesture", 12)):
        ct = 2 * N * limbs * 8 / mib
        key = dnum * 2 * (limbs + K) * N * 8 / mib
        assert ct == pytest.approx(gold["ciphertext_MB"][app])
        assert key == pytest.approx(gold["relin_key_MB"][app])
    P = pm.vital_params()   # 12 Q limbs keep Table 1's depth 11
    assert P.ct_bytes(P.L) / mib == 6.0 and P.key_bytes() / mib == 24.0


def test_crt_roundtrip_bignum():
    P = pm.fir_dft_params()
    Q = 1
    for q in P.q:
        Q *= q
    g = np.random.default_rng(5)
    vals = [int(g.integers(0, 2 ** 62)) * int(g.integers(0, 2 ** 62)) % Q - Q // 2 for _ in range(P.n)]
    poly = np.stack([np.array([v % q for v in vals], dtype=np.uint64) for q in P.q])
    back = ck.crt_centered(P, poly, P.L)
    assert [int(x) for x in back] == vals


def _bignum(poly, primes):
    Q = 1
    for q in primes:
        Q *= q
    out = []
    for k in range(poly.shape[1]):
        x = 0
        for i, q in enumerate(primes):
            Qi = Q // q
            x += int(poly[i, k]) * Qi * pow(Qi, -1, q)
        out.append(x % Q)
    return out, Q


def test_fastbconv_overflow_bound():
    P = pm.vital_params()
    src = P.q[0:4]
    g = np.random.default_rng(2)
    n = 64
    x = np.stack([g.integers(0, q, n, dtype=np.uint64) for q in src])
    xb, Q = _bignum(x, src)
    dst = P.p + P.q[4:7]
    y = ck.fast_bconv(x, src, dst)
    for r, t in enumerate(dst):
        for k in range(n):
            u = ((int(y[r, k]) - xb[k]) * pow(Q, -1, t)) % t
            assert 0 <= u < len(src)


def test_fastbconv_centered_overflow_bound():
    P = pm.vital_params()
    src = P.p
    g = np.random.default_rng(3)
    n = 64
    x = np.stack([g.integers(0, q, n, dtype=np.uint64) for q in src])
    xb, Q = _bignum(x, src)
    dst = P.q[:5]
    y = ck.fast_bconv_centered(x, src, dst)
    half = len(src) // 2
    for r, t in enumerate(dst):
        for k in range(n):
            rem = xb[k] - Q if xb[k] > Q // 2 else xb[k]
            u = ((int(y[r, k]) - rem) * pow(Q, -1, t)) % t
            u = u - t if u > t // 2 else u
            assert -half <= u <= half


def test_rescale_equals_bignum_rounding():
    P = pm.fir_dft_params()
    g = np.random.default_rng(7)
    l = P.L
    c0 = np.stack([g.integers(0, q, P.n, dtype=np.uint64) for q in P.q])
    c1 = np.stack([g.integers(0, q, P.n, dtype=np.uint64) for q in P.q])
    out = ck.rescale(P, ck.Ciphertext(c0, c1, l, 1.0))
    ql = P.q[l]
    for src, res in ((c0, out.c0), (c1, out.c1)):
        xb, Q = _bignum(src, P.q)
        Qd = Q // ql
        for k in range(0, P.n, 97):
            x = xb[k]
            r = x % ql
            r = r - ql if r > ql // 2 else r
            expect = ((x - r) // ql) % Qd
            got = _bignum(res[:, k : k + 1], P.q[:l])[0][0]
            assert got == expect


def test_moddown_is_division_by_P():
    P = pm.fir_dft_params()
    l = P.L
    g = np.random.default_rng(8)
    prim = ck.qp_primes(P, l)
    u = np.stack([g.integers(0, q, 32, dtype=np.uint64) for q in prim])
    Pn = 1
    for p in P.p:
        Pn *= p
    res = np.zeros((l + 1, 32), dtype=np.uint64)
    # moddown works on rows of any length
    Pl = pm.Params.__new__(pm.Params)
    Pl.q, Pl.p, Pl.log_n, Pl.dnum = P.q, P.p, 5, P.dnum
    res = ck.moddown(Pl, u, l)
    ub, QP = _bignum(u, prim)
    ub = [x - QP if x > QP // 2 else x for x in ub]
    got, Qd = _bignum(res, P.q[: l + 1])
    for k in range(32):
        v = got[k] - Qd if got[k] > Qd // 2 else got[k]
        assert abs(v - ub[k] / Pn) <= len(P.p) / 2 + 0.5 + 1e-9


def test_encoding_slot_order_direct_evaluation():
    """m(zeta^(5^j)) = scale * z_j: slot j sits at the root zeta^(5^j)."""
    P = pm.Params.__new__(pm.Params)
    P.log_n = 4
    N = 16
    z = np.linspace(-1, 1, N // 2)
    scale = 2.0 ** 30
    m = ck.encode_coeffs(P, z, scale)
    zeta = np.exp(1j * np.pi / N)
    for j in range(N // 2):
        x = zeta ** pow(5, j, 2 * N)
        val = sum(int(m[k]) * x ** k for k in range(N))
        assert abs(val.real / scale - z[j]) < 1e-6 and abs(val.imag / scale) < 1e-6


def test_encode_decode_roundtrip():
    P = pm.fir_dft_params()
    z = np.random.default_rng(4).uniform(-3, 3, P.slots)
    pt = ck.encode(P, z, P.scale, P.L)
    assert np.abs(ck.decode(P, pt) - z).max() < P.n / P.scale


def test_table1_golden_depths():
    from oracle.circuits import VitalCircuit, VitalConfig
    gold = json.load(open(os.path.join(GOLDEN, "table1_depth.json")))
    P = pm.vital_params()
    c3 = VitalCircuit(P, VitalConfig(taylor_order=3))
    c1 = VitalCircuit(P, VitalConfig(taylor_order=1))
    # main-chain output level: top level minus the depth consumed
    assert P.L - (c3.lv_final_const - 1) == gold["vital_third_order_total_depth"]
    assert P.L - (c1.lv_final_const - 1) == gold["vital_first_order_total_depth"]
    st = gold["stages_cumulative"]
    assert P.L - c3.lv_fir == st["phase_extraction"]
    assert P.L - c3.lv_dphi == st["taylor_arctan_third_order"]
    # the side branch packs its G groups into one ciphertext behind a block
    # mask (one of the levels it has to spare, the main chain sets the depth):
    # K1 at depth 1, the mask at 2, K2's w = E^2 at the paper's depth + 1
    assert P.L - c3.lv_side_mask == 1
    assert P.L - c3.lv_side_const == st["soft_attention"] + 1
