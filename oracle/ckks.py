"""RNS-CKKS reference evaluator (test infrastructure only).

Everything is kept in coefficient form: a polynomial at level l is a uint64
array of shape (l+1, N) whose row i holds the residues mod q_i.  Products are
negacyclic ring products computed row by row (forward NTT, point-wise product,
inverse NTT), which equals the schoolbook product exactly.  Each function
follows one step of the scheme as restated in the module docstrings below; the
choices the paper leaves open (representatives, rounding, hoisting, where
ModDown happens) are fixed as listed in ``SPEC``.

Paper anchors: CKKS primer (key generation: sk, pk, rlk, one Galois key per
rotation amount; encoding N/2 real slots; addition, multiplication consuming a
level, rotation needing a Galois key); "Approximate arithmetic" (one rounding
per rescale); Table 7 (scheme, N, depth, FLEXIBLEAUTO scaling).
"""
import numpy as np

from . import _native as nat

SPEC = {
    "encoding": "m = round_half_away(scale * tau^-1(z)); slot j <-> root zeta^(5^j), zeta = exp(i pi / N)",
    "rotation": "Rot(x, k)[j] = x[(j + k) mod N/2]; Galois element g = 5^(k mod N/2) mod 2N",
    "fastbconv": "y_t = sum_i [x_i * (Qhat_i)^-1]_{q_i} * (Qhat_i mod t) mod t, representatives in [0, q_i)",
    "moddown": "c_i = (u_i - FastBConv~_{P->Q}([u]_P)_i) * P^-1 mod q_i, FastBConv~ with centered representatives",
    "rescale": "c_i = (c_i - r) * q_l^-1 mod q_i with r = centered [c]_{q_l} in (-q_l/2, q_l/2]",
    "keyswitch": "hybrid: dnum digits of alpha primes, digit j unscaled, key b_j = -a_j s + e_j + P*Qtilde_j*s'",
    "hoisting": "one ModUp of c1 shared by all rotations of a hoisted set; automorphism applied to the digits; ModDown per rotation; a single rotation is a hoisted set of one",
}


# ----------------------------------------------------------------------------
# small helpers
# ----------------------------------------------------------------------------
def _inv(a, m):
    return pow(int(a) % m, -1, m)


def _prod(xs):
    r = 1
    for x in xs:
        r *= int(x)
    return r


def round_half_away(x):
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


class Ciphertext:
    """(c0, c1) at ``level`` with real scale ``scale``; decrypts as c0 + c1*s."""

    def __init__(self, c0, c1, level, scale):
        self.c0, self.c1, self.level, self.scale = c0, c1, level, float(scale)

    def copy(self):
        return Ciphertext(self.c0.copy(), self.c1.copy(), self.level, self.scale)

    def words(self):
        """Coefficient-form words, layout [2][level+1][N]."""
        return np.stack([self.c0, self.c1])


class Plaintext:
    def __init__(self, m, level, scale):
        self.m, self.level, self.scale = m, level, float(scale)


# ----------------------------------------------------------------------------
# ring arithmetic on (limbs, N) arrays
# ----------------------------------------------------------------------------
def ring_mul(P, a, b, primes):
    return np.stack([nat.polymul(a[i], b[i], q, P.psi[q]) for i, q in enumerate(primes)])


def ring_add(a, b, primes):
    return np.stack([nat.add(a[i], b[i], q) for i, q in enumerate(primes)])


def ring_sub(a, b, primes):
    return np.stack([nat.sub(a[i], b[i], q) for i, q in enumerate(primes)])


def ring_neg(a, primes):
    return np.stack([nat.neg(a[i], q) for i, q in enumerate(primes)])


def ring_from_signed(coeffs, primes):
    """Signed integer coefficients (|c| < 2^63) reduced into each prime."""
    c = np.asarray(coeffs, dtype=np.int64)
    return np.stack([nat.mod_signed(c, q) for q in primes])


def ring_automorphism(a, g, primes):
    return np.stack([nat.automorphism(a[i], g, q) for i, q in enumerate(primes)])


def q_primes(P, level):
    return P.q[: level + 1]


def qp_primes(P, level):
    return P.q[: level + 1] + P.p


# ----------------------------------------------------------------------------
# CRT reconstruction, encoding and decoding
# ----------------------------------------------------------------------------
def crt_centered(P, poly, level):
    """Exact centered integer coefficients of an RNS polynomial over Q_level
    (Python ints in (-Q/2, Q/2])."""
    primes = q_primes(P, level)
    Q = _prod(primes)
    acc = np.zeros(poly.shape[1], dtype=object)
    for i, q in enumerate(primes):
        Qi = Q // q
        c = _inv(Qi, q)
        t = nat.mul_scalar(poly[i], c, q).astype(object)
        acc = acc + t * Qi
    acc = acc % Q
    half = Q // 2
    return np.where(acc > half, acc - Q, acc)


def _slot_index(N):
    """o_j = (5^j mod 2N - 1)/2 for j < N/2: position of slot j among the odd
    exponents 1, 3, ..., 2N-1."""
    n = N // 2
    e = np.empty(n, dtype=np.int64)
    x = 1
    for j in range(n):
        e[j] = x
        x = (x * 5) % (2 * N)
    return (e - 1) // 2, (2 * N - e - 1) // 2


def encode_coeffs(P, z, scale):
    """Integer coefficients of round(scale * tau^-1(z)) for a real slot vector.

    tau(m)_j = m(zeta^(5^j)); its inverse on a conjugate-symmetric vector Z
    over all odd exponents e is m_k = (1/N) sum_e Z_e zeta^(-e k), computed
    with one length-N FFT (library primitive) after the twist by zeta^-k.
    """
    N = P.n
    z = np.asarray(z, dtype=np.complex128)
    assert z.shape == (N // 2,)
    pos, neg = _slot_index(N)
    Z = np.zeros(N, dtype=np.complex128)
    Z[pos] = z
    Z[neg] = np.conj(z)
    k = np.arange(N)
    m = (np.exp(-1j * np.pi * k / N) * np.fft.fft(Z)).real / N
    c = round_half_away(m * scale)
    assert np.all(np.abs(c) < 2.0 ** 62)
    return c.astype(np.int64)


def encode(P, z, scale, level):
    return Plaintext(ring_from_signed(encode_coeffs(P, z, scale), q_primes(P, level)), level, scale)


def decode_coeffs(P, coeffs, scale):
    """Real slot values z_j = m(zeta^(5^j)) / scale from integer coefficients."""
    N = P.n
    m = np.array([float(x) for x in coeffs], dtype=np.float64) / scale
    k = np.arange(N)
    E = N * np.fft.ifft(m * np.exp(1j * np.pi * k / N))
    pos, _ = _slot_index(N)
    return E[pos].real


def decode(P, pt):
    return decode_coeffs(P, crt_centered(P, pt.m, pt.level), pt.scale)


def decode_complex(P, pt):
    """Complex slot values z_j = m(zeta^(5^j)) / scale."""
    N = P.n
    m = np.array([float(x) for x in crt_centered(P, pt.m, pt.level)], dtype=np.float64) / pt.scale
    k = np.arange(N)
    E = N * np.fft.ifft(m * np.exp(1j * np.pi * k / N))
    pos, _ = _slot_index(N)
    return E[pos]


# ----------------------------------------------------------------------------
# keys
# ----------------------------------------------------------------------------
class SecretKey:
    def __init__(self, P, s_coeffs):
        self.coeffs = np.asarray(s_coeffs, dtype=np.int64)
        self.rns = ring_from_signed(self.coeffs, P.q + P.p)   # rows q_0..q_L, p_0..p_{K-1}


class SwitchKey:
    """dnum x (b_j, a_j) over Q_L * P in coefficient form, array
    [dnum][2][L+1+K][N].  Row order q_0..q_L then p_0..p_{K-1}."""

    def __init__(self, P, data):
        self.data = data
        self._ntt = {}

    def row(self, P, j, part, prime_row):
        return self.data[j, part, prime_row]


def gen_switch_key(P, sk, s_from_rns, a_draw, e_draw):
    """Switching key from s' (``s_from_rns``, rows over Q_L*P) to s.

    For digit j with prime set D_j: b_j = -a_j*s + e_j + P * Qtilde_j * s',
    where Qtilde_j = (Q/Q_j) * [(Q/Q_j)^-1]_{Q_j} is 1 mod q_i for i in D_j
    and 0 mod every other q_i, and P = 0 mod every p_k.  ``a_draw`` holds
    uniform residues [dnum][L+1+K][N]; ``e_draw`` small signed integers
    [dnum][N].
    """
    primes = P.q + P.p
    nq = len(P.q)
    Pprod = _prod(P.p)
    digits = P.digits(P.L)
    data = np.zeros((P.dnum, 2, len(primes), P.n), dtype=np.uint64)
    for j in range(P.dnum):
        a = np.asarray(a_draw[j], dtype=np.uint64)
        e = ring_from_signed(e_draw[j], primes)
        b = ring_add(ring_neg(ring_mul(P, a, sk.rns, primes), primes), e, primes)
        if j < len(digits):
            for i in digits[j]:
                b[i] = nat.add(b[i], nat.mul_scalar(s_from_rns[i], Pprod % primes[i], primes[i]), primes[i])
        data[j, 0] = b
        data[j, 1] = a
    return SwitchKey(P, data)


# Key id of the conjugation X -> X^(2N-1) (slot values z -> conj(z)).
ROT_CONJ = -(1 << 31)


def galois_element(P, k):
    """g = 5^(k mod N/2) mod 2N: left rotation of the slot vector by k;
    k = ROT_CONJ: g = 2N - 1, complex conjugation of every slot."""
    if k == ROT_CONJ:
        return 2 * P.n - 1
    return pow(5, k % P.slots, 2 * P.n)


def key_id(P, k):
    """Index of the switching key of rotation k (or ROT_CONJ)."""
    return k if k == ROT_CONJ else k % P.slots


def gen_relin_key(P, sk, a_draw, e_draw):
    primes = P.q + P.p
    s2 = ring_mul(P, sk.rns, sk.rns, primes)
    return gen_switch_key(P, sk, s2, a_draw, e_draw)


def gen_galois_key(P, sk, k, a_draw, e_draw):
    primes = P.q + P.p
    sg = ring_automorphism(sk.rns, galois_element(P, k), primes)
    return gen_switch_key(P, sk, sg, a_draw, e_draw)


class PublicKey:
    def __init__(self, b, a):
        self.b, self.a = b, a


def gen_public_key(P, sk, a_draw, e_draw):
    """pk = (-a*s + e, a) over Q_L."""
    primes = P.q
    a = np.asarray(a_draw, dtype=np.uint64)[: len(primes)]
    e = ring_from_signed(e_draw, primes)
    s = sk.rns[: len(primes)]
    b = ring_add(ring_neg(ring_mul(P, a, s, primes), primes), e, primes)
    return PublicKey(b, a)


def encrypt(P, pk, pt, v_draw, e0_draw, e1_draw):
    """Public-key encryption at the top level: (v*b + e0 + m, v*a + e1)."""
    assert pt.level == P.L
    primes = P.q
    v = ring_from_signed(v_draw, primes)
    e0 = ring_from_signed(e0_draw, primes)
    e1 = ring_from_signed(e1_draw, primes)
    c0 = ring_add(ring_add(ring_mul(P, v, pk.b, primes), e0, primes), pt.m, primes)
    c1 = ring_add(ring_mul(P, v, pk.a, primes), e1, primes)
    return Ciphertext(c0, c1, P.L, pt.scale)


def decrypt(P, sk, ct):
    primes = q_primes(P, ct.level)
    s = sk.rns[: ct.level + 1]
    m = ring_add(ct.c0, ring_mul(P, ct.c1, s, primes), primes)
    return Plaintext(m, ct.level, ct.scale)


def decrypt_decode(P, sk, ct):
    return decode(P, decrypt(P, sk, ct))


# ----------------------------------------------------------------------------
# evaluator: depth-free operations
# ----------------------------------------------------------------------------
def add(P, a, b):
    assert a.level == b.level
    pr = q_primes(P, a.level)
    return Ciphertext(ring_add(a.c0, b.c0, pr), ring_add(a.c1, b.c1, pr), a.level, a.scale)


def add_plain(P, a, pt):
    """ct + pt: the plaintext joins c0; pt must be encoded at the
    ciphertext's scale and level."""
    assert a.level == pt.level and abs(pt.scale / a.scale - 1.0) < 1e-9
    pr = q_primes(P, a.level)
    return Ciphertext(ring_add(a.c0, pt.m, pr), a.c1.copy(), a.level, a.scale)


def sub(P, a, b):
    assert a.level == b.level
    pr = q_primes(P, a.level)
    return Ciphertext(ring_sub(a.c0, b.c0, pr), ring_sub(a.c1, b.c1, pr), a.level, a.scale)


def mul_int(P, a, k):
    """Multiply by a small integer constant (exact, no level consumed)."""
    pr = q_primes(P, a.level)
    c0 = np.stack([nat.mul_scalar(a.c0[i], k % q, q) for i, q in enumerate(pr)])
    c1 = np.stack([nat.mul_scalar(a.c1[i], k % q, q) for i, q in enumerate(pr)])
    return Ciphertext(c0, c1, a.level, a.scale)


def mul_scalar(P, a, c, scale):
    """ct * c for a real constant c encoded at `scale`: the constant
    polynomial round(scale c) (the encoding of a vector equal to c in every
    slot), so an exact integer multiply; the scale multiplies by `scale`."""
    m = int(round_half_away(scale * c))
    r = mul_int(P, a, m)
    return Ciphertext(r.c0, r.c1, a.level, a.scale * scale)


def drop_level(P, a, level):
    """Discard the top limbs (no division, scale unchanged)."""
    assert level <= a.level
    return Ciphertext(a.c0[: level + 1].copy(), a.c1[: level + 1].copy(), level, a.scale)


def mul_plain(P, a, pt):
    """ct * pt without rescale: scale multiplies."""
    assert a.level == pt.level
    pr = q_primes(P, a.level)
    return Ciphertext(ring_mul(P, a.c0, pt.m, pr), ring_mul(P, a.c1, pt.m, pr), a.level, a.scale * pt.scale)


def mul_plain_sum(P, pairs):
    """sum_i ct_i * pt_i (no rescale), every product taken as a negacyclic
    ring product; the sum is accumulated in the NTT domain (one forward
    transform per distinct operand, one inverse per output row), which is the
    same ring element as summing mul_plain results."""
    level = pairs[0][0].level
    pr = q_primes(P, level)
    acc = np.zeros((2, level + 1, P.n), dtype=np.uint64)
    for i, q in enumerate(pr):
        psi = P.psi[q]
        for ct, pt in pairs:
            assert ct.level == level and pt.level == level
            fct = _ct_ntt(P, ct, i)
            fpt = _pt_ntt(P, pt, i)
            for h in range(2):
                acc[h, i] = nat.add(acc[h, i], nat.mul(fct[h], fpt, q), q)
        for h in range(2):
            acc[h, i] = nat.ntt_inv(acc[h, i], q, psi)
    return Ciphertext(acc[0], acc[1], level, pairs[0][0].scale * pairs[0][1].scale)


def _ct_ntt(P, ct, i):
    """Forward NTT of row i of both halves, cached on the (never mutated)
    ciphertext object."""
    cache = ct.__dict__.setdefault("_ntt", {})
    if i not in cache:
        q = P.q[i]
        cache[i] = (nat.ntt_fwd(ct.c0[i], q, P.psi[q]), nat.ntt_fwd(ct.c1[i], q, P.psi[q]))
    return cache[i]


def _pt_ntt(P, pt, i):
    cache = pt.__dict__.setdefault("_ntt", {})
    if i not in cache:
        q = P.q[i]
        cache[i] = nat.ntt_fwd(pt.m[i], q, P.psi[q])
    return cache[i]


# ----------------------------------------------------------------------------
# tensor product, key switching, relinearization, rotation, rescale
# ----------------------------------------------------------------------------
class Tensor:
    """Degree-2 ciphertext (d0, d1, d2), decrypting as d0 + d1 s + d2 s^2."""

    def __init__(self, d0, d1, d2, level, scale):
        self.d0, self.d1, self.d2, self.level, self.scale = d0, d1, d2, level, scale


def tensor(P, a, b):
    assert a.level == b.level
    pr = q_primes(P, a.level)
    d0 = ring_mul(P, a.c0, b.c0, pr)
    d1 = ring_add(ring_mul(P, a.c0, b.c1, pr), ring_mul(P, a.c1, b.c0, pr), pr)
    d2 = ring_mul(P, a.c1, b.c1, pr)
    return Tensor(d0, d1, d2, a.level, a.scale * b.scale)


def tensor_add(P, x, y):
    assert x.level == y.level
    pr = q_primes(P, x.level)
    return Tensor(ring_add(x.d0, y.d0, pr), ring_add(x.d1, y.d1, pr), ring_add(x.d2, y.d2, pr), x.level, x.scale)


def tensor_sub(P, x, y):
    assert x.level == y.level
    pr = q_primes(P, x.level)
    return Tensor(ring_sub(x.d0, y.d0, pr), ring_sub(x.d1, y.d1, pr), ring_sub(x.d2, y.d2, pr), x.level, x.scale)


def tensor_mul_int(P, x, k):
    pr = q_primes(P, x.level)

    def f(d):
        return np.stack([nat.mul_scalar(d[i], k % q, q) for i, q in enumerate(pr)])

    return Tensor(f(x.d0), f(x.d1), f(x.d2), x.level, x.scale)


def fast_bconv(x_rows, src, dst):
    """FastBConv from the basis ``src`` to each modulus in ``dst``.

    y_t = sum_i [x_i * (Qhat_i)^-1 mod q_i] * (Qhat_i mod t) mod t with
    Qhat_i = prod(src)/q_i and every [.] taken in [0, q_i).  The integer
    sum_i [..]_i * Qhat_i equals x + u*prod(src) for some 0 <= u < len(src).
    """
    Qs = _prod(src)
    tv = [nat.mul_scalar(x_rows[i], _inv(Qs // q, q), q) for i, q in enumerate(src)]
    out = []
    for t in dst:
        acc = np.zeros(x_rows.shape[1], dtype=np.uint64)
        for i, q in enumerate(src):
            nat.mac_scalar(acc, tv[i], (Qs // q) % t, t)
        out.append(acc)
    return np.stack(out) if out else np.zeros((0, x_rows.shape[1]), dtype=np.uint64)


def modup(P, d, level):
    """Digit decomposition + ModUp of d (rows over Q_level).

    Returns one array per digit j, rows over q_0..q_level, p_0..p_{K-1}: the
    digit's own rows are copied, every other row is FastBConv of the digit.
    """
    targets = qp_primes(P, level)
    out = []
    for D in P.digits(level):
        src = [P.q[i] for i in D]
        others = [r for r in range(len(targets)) if not (r <= level and r in D)]
        conv = fast_bconv(d[D[0] : D[-1] + 1], src, [targets[r] for r in others])
        y = np.zeros((len(targets), P.n), dtype=np.uint64)
        for i in D:
            y[i] = d[i]
        for k, r in enumerate(others):
            y[r] = conv[k]
        out.append(y)
    return out


def fast_bconv_centered(x_rows, src, dst):
    """FastBConv with centered representatives: x~_i = [x_i (Qhat_i)^-1]_{q_i}
    taken in (-q_i/2, q_i/2]; y_t = sum_i x~_i * Qhat_i mod t.  The integer
    sum_i x~_i Qhat_i equals the centered remainder of x mod prod(src) plus
    u*prod(src) with |u| <= len(src)/2, so its error has zero mean."""
    Qs = _prod(src)
    tv = [nat.mul_scalar(x_rows[i], _inv(Qs // q, q), q) for i, q in enumerate(src)]
    neg = [t > (q // 2) for t, q in zip(tv, src)]          # representative is t - q_i
    count = np.sum(np.stack(neg), axis=0).astype(np.uint64)
    out = []
    for t in dst:
        acc = np.zeros(x_rows.shape[1], dtype=np.uint64)
        for i, q in enumerate(src):
            nat.mac_scalar(acc, tv[i], (Qs // q) % t, t)
        # (t_i - q_i) Qhat_i = t_i Qhat_i - prod(src): subtract count * prod(src)
        acc = nat.sub(acc, nat.mul_scalar(count, Qs % t, t), t)
        out.append(acc)
    return np.stack(out)


def moddown(P, u, level):
    """(u_i - FastBConv_{P->Q}([u]_P)_i) * P^-1 mod q_i for i <= level, with the
    centered FastBConv (so the division by P rounds with zero-mean error)."""
    nq = level + 1
    qs = q_primes(P, level)
    v = fast_bconv_centered(u[nq:], P.p, qs)
    Pprod = _prod(P.p)
    return np.stack([nat.mul_scalar(nat.sub(u[i], v[i], q), _inv(Pprod, q), q) for i, q in enumerate(qs)])


def key_rows(P, level):
    """Row indices of a switching key used at ``level`` (q_0..q_level, p's)."""
    nq = len(P.q)
    return list(range(level + 1)) + [nq + k for k in range(len(P.p))]


def inner_product(P, digits, key, level):
    """(sum_j y_j * b_j, sum_j y_j * a_j) over Q_level * P."""
    targets = qp_primes(P, level)
    rows = key_rows(P, level)
    u0 = np.zeros((len(targets), P.n), dtype=np.uint64)
    u1 = np.zeros((len(targets), P.n), dtype=np.uint64)
    for r, t in enumerate(targets):
        psi = P.psi[t]
        acc0 = np.zeros(P.n, dtype=np.uint64)
        acc1 = np.zeros(P.n, dtype=np.uint64)
        for j, y in enumerate(digits):
            fy = nat.ntt_fwd(y[r], t, psi)
            acc0 = nat.add(acc0, nat.mul(fy, _key_ntt(P, key, j, 0, rows[r]), t), t)
            acc1 = nat.add(acc1, nat.mul(fy, _key_ntt(P, key, j, 1, rows[r]), t), t)
        u0[r] = nat.ntt_inv(acc0, t, psi)
        u1[r] = nat.ntt_inv(acc1, t, psi)
    return u0, u1


def _key_ntt(P, key, j, part, row):
    k = (j, part, row)
    if k not in key._ntt:
        t = (P.q + P.p)[row]
        key._ntt[k] = nat.ntt_fwd(key.data[j, part, row], t, P.psi[t])
    return key._ntt[k]


def key_switch(P, d, key, level):
    """Hybrid key switching of d (rows over Q_level): ModUp, inner product with
    the key, ModDown of both halves."""
    digits = modup(P, d, level)
    u0, u1 = inner_product(P, digits, key, level)
    return moddown(P, u0, level), moddown(P, u1, level)


def relinearize(P, t, rlk):
    pr = q_primes(P, t.level)
    k0, k1 = key_switch(P, t.d2, rlk, t.level)
    return Ciphertext(ring_add(t.d0, k0, pr), ring_add(t.d1, k1, pr), t.level, t.scale)


def mul_relin(P, a, b, rlk):
    return relinearize(P, tensor(P, a, b), rlk)


def rescale(P, a):
    """Divide by q_l with the centered remainder; level and scale drop."""
    l = a.level
    ql = P.q[l]
    qs = q_primes(P, l - 1)

    def one(c):
        r = c[l].astype(np.int64)                     # q_l < 2^62 fits
        r = np.where(r > ql // 2, r - ql, r)          # centered, q_l odd
        inv = [_inv(ql, q) for q in qs]
        return np.stack([nat.mul_scalar(nat.sub(c[i], nat.mod_signed(r, q), q), inv[i], q) for i, q in enumerate(qs)])

    return Ciphertext(one(a.c0), one(a.c1), l - 1, a.scale / ql)


def rotate(P, a, k, gks):
    """Rot(a, k) with the hoisted schedule of a one-element set: ModUp of c1,
    automorphism X -> X^g of the digits, inner product with the Galois key of
    k, ModDown, plus the automorphism of c0."""
    return rotate_hoisted(P, a, [k], gks)[0]


def conjugate(P, a, gks):
    """Slot-wise complex conjugate (the automorphism X -> X^(2N-1)), switched
    back to s with the key ROT_CONJ, on the rotation's schedule."""
    return rotate_hoisted(P, a, [ROT_CONJ], gks)[0]


def rotate_hoisted(P, a, ks, gks):
    """Rotations of one ciphertext by every k in ``ks`` sharing one ModUp of c1:
    the automorphism is applied to the ModUp digits, then inner product and
    ModDown per rotation.  k = 0 returns a copy."""
    digits = modup(P, a.c1, a.level)
    pr = q_primes(P, a.level)
    prqp = qp_primes(P, a.level)
    out = []
    for k in ks:
        if key_id(P, k) == 0:
            out.append(a.copy())
            continue
        g = galois_element(P, k)
        rd = [ring_automorphism(y, g, prqp) for y in digits]
        u0, u1 = inner_product(P, rd, gks[key_id(P, k)], a.level)
        c0 = ring_automorphism(a.c0, g, pr)
        out.append(Ciphertext(ring_add(c0, moddown(P, u0, a.level), pr), moddown(P, u1, a.level), a.level, a.scale))
    return out


# ----------------------------------------------------------------------------
# double-hoisted BSGS product (Bossuat, Mouchet, Troncoso-Pastoriza and
# Hubaux, Eurocrypt 2021, Sec. 4): the baby rotations, the inner sums and the
# giant-step sum stay in the extended basis Q_level * P, scaled by P, and are
# brought down to Q once
# ----------------------------------------------------------------------------
def encode_qp(P, z, scale, level):
    """``encode`` with rows over Q_level * P (the extended basis): the same
    integer coefficients, reduced mod every q_i and p_k."""
    return Plaintext(ring_from_signed(encode_coeffs(P, z, scale), qp_primes(P, level)), level, scale)


def times_p(P, c, level):
    """P * c over Q_level * P for c over Q_level: rows P c_i mod q_i, and zero
    rows mod every p_k (P is 0 there)."""
    Pprod = _prod(P.p)
    rows = [nat.mul_scalar(c[i], Pprod % q, q) for i, q in enumerate(q_primes(P, level))]
    rows += [np.zeros(P.n, dtype=np.uint64) for _ in P.p]
    return np.stack(rows)


def bsgs_double_hoisted(P, a, diags, n1, stride, gks):
    """sum_g Rot_{g n1 stride}( sum_b D'_{g,b} (.) Rot_{b stride}(a) ), not
    rescaled, with every intermediate over Q_level * P:

      baby b  = (P sigma_b(c0) + u0, u1), u = <sigma_b(ModUp(c1)), key of b stride>,
                one ModUp of c1 shared by all babies, no ModDown;
      inner g = sum_b D'_{g,b} (.) baby b, with D' encoded over Q_level * P;
      giant g = inner g for g = 0; otherwise the c1 of inner g is brought to
                Q by ModDown and switched with the key of g n1 stride (ModUp,
                automorphism of the digits, inner product w), and
                (sigma_g(c0 of inner g) + w0, w1) is the term;
      result  = ModDown of each part of the sum of the terms.

    ``diags``: {delta: Plaintext over Q_level * P (encode_qp)}, delta =
    g n1 + b with 0 <= b < n1 (floor division), each pre-rotated by
    -g n1 stride as in the single-hoisted product."""
    return bsgs_double_hoisted_sets(P, {"x": (a, 0)}, {("x", d): pt for d, pt in diags.items()}, n1, stride, gks)


def bsgs_double_hoisted_sets(P, sets, diags, n1, stride, gks):
    """The double-hoisted product over several baby sets sharing the giant
    steps: set `name` holds the baby rotations Rot(x_name, b stride + off_name)
    of its input ``sets[name] = (x_name, off_name)``, and

      result = sum_g Rot_{g n1 stride}( sum_{name, b} D'_{name,g,b} (.) baby_{name,b} ),

    every baby, inner sum and giant-step term over Q_level * P as in
    ``bsgs_double_hoisted`` (one ModUp of c1 per distinct input ciphertext,
    shared by all its babies; one ModDown of each part at the end).
    ``diags``: {(name, delta): Plaintext over Q_level * P}, delta = g n1 + b,
    0 <= b < n1, pre-rotated by -g n1 stride."""
    level = next(iter(sets.values()))[0].level
    prq, prqp = q_primes(P, level), qp_primes(P, level)
    groups = {}
    for key in sorted(diags):
        groups.setdefault(key[1] // n1, []).append(key)
    digits = {}
    babies = {}
    for name, d in sorted(diags):
        b = d - (d // n1) * n1
        if (name, b) in babies:
            continue
        x, off = sets[name]
        assert x.level == level
        k = b * stride + off
        if key_id(P, k) == 0:
            babies[(name, b)] = (times_p(P, x.c0, level), times_p(P, x.c1, level))
            continue
        if id(x) not in digits:
            digits[id(x)] = modup(P, x.c1, level)
        g = galois_element(P, k)
        u0, u1 = inner_product(P, [ring_automorphism(y, g, prqp) for y in digits[id(x)]], gks[key_id(P, k)], level)
        babies[(name, b)] = (ring_add(times_p(P, ring_automorphism(x.c0, g, prq), level), u0, prqp), u1)
    acc0 = acc1 = None
    scale = None
    for gi in sorted(groups):
        in0 = np.zeros((len(prqp), P.n), dtype=np.uint64)
        in1 = np.zeros((len(prqp), P.n), dtype=np.uint64)
        for name, d in groups[gi]:
            pt = diags[(name, d)]
            assert pt.level == level and pt.m.shape[0] == len(prqp)
            b0, b1 = babies[(name, d - gi * n1)]
            in0 = ring_add(in0, ring_mul(P, b0, pt.m, prqp), prqp)
            in1 = ring_add(in1, ring_mul(P, b1, pt.m, prqp), prqp)
            scale = sets[name][0].scale * pt.scale
        k = gi * n1 * stride
        if key_id(P, k) == 0:
            t0, t1 = in0, in1
        else:
            g = galois_element(P, k)
            dg = modup(P, moddown(P, in1, level), level)
            w0, w1 = inner_product(P, [ring_automorphism(y, g, prqp) for y in dg], gks[key_id(P, k)], level)
            t0, t1 = ring_add(ring_automorphism(in0, g, prqp), w0, prqp), w1
        acc0 = t0 if acc0 is None else ring_add(acc0, t0, prqp)
        acc1 = t1 if acc1 is None else ring_add(acc1, t1, prqp)
    return Ciphertext(moddown(P, acc0, level), moddown(P, acc1, level), level, scale)
