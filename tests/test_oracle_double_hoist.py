"""Pins of the oracle's double-hoisted BSGS product (baby rotations, inner
sums and the giant-step sum in the extended basis Q*P, one ModDown at the
end; Bossuat et al., Eurocrypt 2021, Sec. 4).

* On a trivial ciphertext (c1 = 0) every key switch is exactly zero and the
  ModDown of P*X is exactly X, so the product must equal, word for word, the
  same sum of automorphisms and ring products taken directly over Q.
* On a real encryption it must decrypt to the plain matrix-vector product,
  as the single-hoisted product does.
"""
import numpy as np

import synth
from oracle import ckks as ck
from oracle import circuits as cc


def test_trivial_ciphertext_equals_the_direct_sum_over_q(small_setup):
    P, s = small_setup["P"], small_setup
    level, n1, stride = P.L - 1, 4, 16
    g = np.random.default_rng(3)
    prq = ck.q_primes(P, level)
    c0 = np.stack([g.integers(0, q, P.n, dtype=np.uint64) for q in prq])
    a = ck.Ciphertext(c0, np.zeros_like(c0), level, 1.0)
    deltas = [0, 1, 3, 4, 6, 9, 11]          # babies 0..3, giants 0..2, some (g, b) absent
    diags = {d: ck.encode_qp(P, g.uniform(-1, 1, P.slots), 2.0 ** 20, level) for d in deltas}
    y = ck.bsgs_double_hoisted(P, a, diags, n1, stride, s["gks"])

    want = np.zeros_like(c0)
    for gi in sorted({d // n1 for d in deltas}):
        inner = np.zeros_like(c0)
        for d in deltas:
            if d // n1 != gi:
                continue
            b = d - gi * n1
            rb = ck.ring_automorphism(c0, ck.galois_element(P, b * stride), prq) if b else c0
            inner = ck.ring_add(inner, ck.ring_mul(P, rb, diags[d].m[: level + 1], prq), prq)
        if gi:
            inner = ck.ring_automorphism(inner, ck.galois_element(P, gi * n1 * stride), prq)
        want = ck.ring_add(want, inner, prq)
    assert np.array_equal(y.c0, want)
    assert not y.c1.any()


def test_double_hoisted_decrypts_to_the_matvec_like_the_single_hoisted(small_setup):
    P, s = small_setup["P"], small_setup
    lay = cc.Layout(P.slots, 16, 256)     # R_c = 16, time axis of 256 positions
    g = np.random.default_rng(7)
    D = 12
    M = np.zeros((lay.f_pad, lay.f_pad))
    sup = np.zeros_like(M, dtype=bool)
    for t in range(lay.f_pad):
        for dd in range(D):
            M[t, (t + dd) % lay.f_pad] = g.uniform(-1, 1)
            sup[t, (t + dd) % lay.f_pad] = True
    x = g.uniform(-1, 1, P.slots)
    n1 = 4
    diags = cc.matrix_diagonals_all_offsets({"support": sup, "values": M}, lay)
    pre = {d: cc.prerotate(v, d // n1, n1, lay.r_c) for d, v in diags.items()}
    ct = ck.encrypt(P, s["pk"], ck.encode(P, x, P.scale, P.L), *synth.encryption_draws(7, P.n))

    qp = {d: ck.encode_qp(P, v, P.q[P.L], P.L) for d, v in pre.items()}
    y2 = ck.rescale(P, ck.bsgs_double_hoisted(P, ct, qp, n1, lay.r_c, s["gks"]))
    q_only = {("x", d): ck.encode(P, v, P.q[P.L], P.L) for d, v in pre.items()}
    ev = cc.Evaluator(P, s["rlk"], s["gks"])
    babies = {"x": ev.hoisted(ct, [b * lay.r_c for b in range(n1)])}
    y1 = ck.rescale(P, ev.bsgs(babies, q_only, n1, lay.r_c, P.L))

    X = x.reshape(lay.f_pad, lay.r_c)
    z2 = ck.decrypt_decode(P, s["sk"], y2).reshape(lay.f_pad, lay.r_c)
    z1 = ck.decrypt_decode(P, s["sk"], y1).reshape(lay.f_pad, lay.r_c)
    assert np.abs(z2 - M @ X).max() < 1e-5
    assert np.abs(z2 - z1).max() < 1e-5
    # the two schedules round differently: the words differ
    assert not np.array_equal(y2.c0, y1.c0)


def test_baby_sets_with_offsets_equal_the_direct_sum_over_q(small_setup):
    """Two baby sets of one input (the vital FIR's layout: offsets 0 and -1
    slot) and a set of a second input, sharing the giant steps: on trivial
    ciphertexts the product equals the direct sum over Q of
    sigma_{g n1 stride}( sum D'_{name,g,b} sigma_{b stride + off}(c0_name) )."""
    P, s = small_setup["P"], small_setup
    level, n1, stride = P.L - 1, 4, -16
    g = np.random.default_rng(5)
    prq = ck.q_primes(P, level)
    c0a = np.stack([g.integers(0, q, P.n, dtype=np.uint64) for q in prq])
    c0b = np.stack([g.integers(0, q, P.n, dtype=np.uint64) for q in prq])
    a = ck.Ciphertext(c0a, np.zeros_like(c0a), level, 1.0)
    b = ck.Ciphertext(c0b, np.zeros_like(c0b), level, 1.0)
    sets = {"s0": (a, 0), "s1": (a, -1), "t": (b, 0)}
    keys = [("s0", 0), ("s0", 2), ("s1", 1), ("s1", 4), ("s1", 5), ("t", 3), ("t", 8), ("s0", 9)]
    diags = {k: ck.encode_qp(P, g.uniform(-1, 1, P.slots), 2.0 ** 20, level) for k in keys}
    # c1 = 0: every key switch is exactly zero whatever the key, so any key
    # stands in for the rotations the small fixture has no key for
    gks = dict(s["gks"])
    some = next(iter(gks.values()))
    for name, d in keys:
        for r in ((d % n1) * stride + sets[name][1], (d // n1) * n1 * stride):
            gks.setdefault(ck.key_id(P, r), some)
    y = ck.bsgs_double_hoisted_sets(P, sets, diags, n1, stride, gks)
    want = np.zeros_like(c0a)
    for gi in sorted({d // n1 for _, d in keys}):
        inner = np.zeros_like(c0a)
        for name, d in keys:
            if d // n1 != gi:
                continue
            x, off = sets[name]
            r = (d - gi * n1) * stride + off
            rb = ck.ring_automorphism(x.c0, ck.galois_element(P, r), prq) if ck.key_id(P, r) else x.c0
            inner = ck.ring_add(inner, ck.ring_mul(P, rb, diags[(name, d)].m[: level + 1], prq), prq)
        if gi:
            inner = ck.ring_automorphism(inner, ck.galois_element(P, gi * n1 * stride), prq)
        want = ck.ring_add(want, inner, prq)
    assert np.array_equal(y.c0, want)
    assert not y.c1.any()
