"""GPU parity: every hot-path step of the CUDA library against the CPU oracle,
word for word (all arithmetic is exact modular integer arithmetic, so the bar
is bit-exact output ciphertexts), through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import ckks as ck
from oracle import circuits as cc

pytestmark = pytest.mark.gpu


def lib_params(P):
    import paper_2603_22437_b300 as M
    return M.params_from_primes(P.log_n, P.q, P.p, P.dnum)


def load_keys(ctx, P, rlk, gks):
    k = ctx.keys(7)
    k.set_relin(np.ascontiguousarray(rlk.data))
    for r, key in gks.items():
        k.set_galois(r, np.ascontiguousarray(key.data))
    return k


@pytest.fixture(scope="module")
def gsmall(small_setup):
    import paper_2603_22437_b300 as M
    s = small_setup
    ctx = M.Context(lib_params(s["P"]))
    keys = load_keys(ctx, s["P"], s["rlk"], s["gks"])
    return dict(s, ctx=ctx, keys=keys)


def rand_ct(P, level, seed, B=None):
    g = np.random.default_rng(seed)
    shape = (2, level + 1, P.n) if B is None else (B, 2, level + 1, P.n)
    out = np.empty(shape, dtype=np.uint64)
    for i, q in enumerate(P.q[: level + 1]):
        out[..., i, :] = g.integers(0, q, out[..., i, :].shape, dtype=np.uint64)
    return out


def as_ct(P, words, level):
    return ck.Ciphertext(words[0].copy(), words[1].copy(), level, 1.0)


def test_ntt_polymul_all_primes(gsmall):
    P, ctx = gsmall["P"], gsmall["ctx"]
    primes = P.q + P.p
    g = np.random.default_rng(1)
    a = np.stack([g.integers(0, q, P.n, dtype=np.uint64) for q in primes])
    b = np.stack([g.integers(0, q, P.n, dtype=np.uint64) for q in primes])
    out = np.empty_like(a)
    ctx.poly_mul(out, a, b, list(range(len(primes))))
    for i, q in enumerate(primes):
        assert np.array_equal(out[i], ck.nat.polymul(a[i], b[i], q, P.psi[q])), "prime %d" % i
    x = a.copy()
    ctx.ntt(x, list(range(len(primes))))
    assert not np.array_equal(x, a)
    ctx.ntt(x, list(range(len(primes))), inverse=True)
    assert np.array_equal(x, a)


@pytest.mark.parametrize("level", [3, 1])
def test_add_mul_plain_rescale(gsmall, level):
    P, ctx = gsmall["P"], gsmall["ctx"]
    B = 3
    a, b = rand_ct(P, level, 2, B), rand_ct(P, level, 3, B)
    out = np.empty_like(a)
    ctx.ct_add(out, a, b, B, level)
    for w in range(B):
        r = ck.add(P, as_ct(P, a[w], level), as_ct(P, b[w], level))
        assert np.array_equal(out[w], r.words())
    pt = rand_ct(P, level, 4)[0]
    ctx.ct_mul_plain(out, a, pt, B, level)
    for w in range(B):
        r = ck.mul_plain(P, as_ct(P, a[w], level), ck.Plaintext(pt, level, 1.0))
        assert np.array_equal(out[w], r.words())
    res = np.empty((B, 2, level, P.n), dtype=np.uint64)
    ctx.ct_rescale(res, a, B, level)
    for w in range(B):
        assert np.array_equal(res[w], ck.rescale(P, as_ct(P, a[w], level)).words())


@pytest.mark.parametrize("level", [3, 2, 0])
def test_modup_keyswitch(gsmall, level):
    P, ctx, keys = gsmall["P"], gsmall["ctx"], gsmall["keys"]
    B = 2
    d = rand_ct(P, level, 5, B)[:, 0].copy()          # [B][l+1][N]
    beta = len(P.digits(level))
    nre = level + 1 + len(P.p)
    up = np.empty((B, beta, nre, P.n), dtype=np.uint64)
    ctx.modup(up, d, B, level)
    for w in range(B):
        ref = ck.modup(P, d[w], level)
        for j in range(beta):
            assert np.array_equal(up[w, j], ref[j]), "digit %d" % j
    out = np.empty((B, 2, level + 1, P.n), dtype=np.uint64)
    ctx.keyswitch(keys, out, d, B, level)
    for w in range(B):
        u0, u1 = ck.key_switch(P, d[w], gsmall["rlk"], level)
        assert np.array_equal(out[w, 0], u0) and np.array_equal(out[w, 1], u1)
    k = gsmall["rots"][0]
    ctx.keyswitch(keys, out, d, B, level, rotation=k)
    for w in range(B):
        u0, u1 = ck.key_switch(P, d[w], gsmall["gks"][k % P.slots], level)
        assert np.array_equal(out[w, 0], u0) and np.array_equal(out[w, 1], u1)


@pytest.mark.parametrize("level", [3, 1])
def test_mul_relin(gsmall, level):
    P, ctx, keys = gsmall["P"], gsmall["ctx"], gsmall["keys"]
    B = 2
    a, b = rand_ct(P, level, 6, B), rand_ct(P, level, 7, B)
    out = np.empty_like(a)
    ctx.ct_mul_relin(keys, out, a, b, B, level)
    for w in range(B):
        r = ck.mul_relin(P, as_ct(P, a[w], level), as_ct(P, b[w], level), gsmall["rlk"])
        assert np.array_equal(out[w], r.words())


@pytest.mark.parametrize("level", [3, 2])
def test_rotate_and_hoisted(gsmall, level):
    P, ctx, keys = gsmall["P"], gsmall["ctx"], gsmall["keys"]
    B = 2
    a = rand_ct(P, level, 8, B)
    ks = [0, 1, 3, 5, -16]
    outs = [np.empty_like(a) for _ in ks]
    ctx.ct_rotate_hoisted(keys, outs, a, B, level, ks)
    for w in range(B):
        ref = ck.rotate_hoisted(P, as_ct(P, a[w], level), ks, gsmall["gks"])
        for i, k in enumerate(ks):
            assert np.array_equal(outs[i][w], ref[i].words()), "k=%d" % k
    one = np.empty_like(a)
    ctx.ct_rotate(keys, one, a, B, level, 3)
    assert np.array_equal(one, outs[2])


def test_rotsum_bsgs(gsmall):
    P, ctx, keys = gsmall["P"], gsmall["ctx"], gsmall["keys"]
    level, B = 3, 2
    a = rand_ct(P, level, 9, B)
    out = np.empty_like(a)
    ctx.ct_rotsum(keys, out, a, B, level, 16, 8)
    ev = cc.Evaluator(P, gsmall["rlk"], gsmall["gks"])
    for w in range(B):
        assert np.array_equal(out[w], ev.rotsum(as_ct(P, a[w], level), 16, 8).words())
    g = np.random.default_rng(10)
    n1, stride = 4, 16
    deltas = list(range(12))
    diags = [np.stack([g.integers(0, q, P.n, dtype=np.uint64) for q in P.q[: level + 1]]) for _ in deltas]
    ctx.ct_bsgs(keys, out, a, B, level, stride, n1, deltas, diags)
    for w in range(B):
        x = as_ct(P, a[w], level)
        need = sorted({d % n1 for d in deltas})
        babies = {"x": dict(zip(need, ck.rotate_hoisted(P, x, [b * stride for b in need], gsmall["gks"])))}
        consts = {("x", d): ck.Plaintext(v, level, 1.0) for d, v in zip(deltas, diags)}
        assert np.array_equal(out[w], ev.bsgs(babies, consts, n1, stride, level).words())


def test_errors(gsmall):
    import paper_2603_22437_b300 as M
    P, ctx, keys = gsmall["P"], gsmall["ctx"], gsmall["keys"]
    a = rand_ct(P, 2, 1, 1)
    out = np.empty_like(a)
    with pytest.raises(M.MmfheError) as e:
        ctx.ct_rotate(keys, out, a, 1, 2, 7)           # no key for rotation 7
    assert e.value.name == "NOT_FOUND"
    with pytest.raises(M.MmfheError) as e:
        ctx.ct_rescale(out, a, 1, 0)
    assert e.value.name == "LEVEL_MISMATCH"
    bad = lib_params(P)
    bad.q[1] = bad.q[1] + 2
    with pytest.raises(M.MmfheError) as e:
        M.Context(bad)
    assert e.value.name == "BAD_BLOB"
    ctx.ct_add(out, a, a, 0, 2)                        # empty batch is a no-op


def test_sync_timeout_returns_status(gsmall):
    import torch
    import paper_2603_22437_b300 as M
    ctx = gsmall["ctx"]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        torch.cuda._sleep(200_000_000)                 # bounded busy wait (~0.1 s)
    with pytest.raises(M.MmfheError) as e:
        ctx.sync(s, timeout_ms=1)
    assert e.value.name == "TIMEOUT"
    ctx.sync(s, timeout_ms=30000)


# ---------------------------------------------------------------------------
# circuits
# ---------------------------------------------------------------------------
def oracle_const_words(plan, consts):
    """The oracle's encoded constants in the plan's constant order
    (coefficient-form words, one array per constant)."""
    out = []
    for tag, band, index, level in plan.const_keys():
        if tag in ("idx", "one", "pmask"):
            key = (tag,)
        elif tag in ("fw", "fone"):
            key = (tag, band)
        elif tag == "dre":
            key = ("dft", index)
        elif tag == "fir" and ("fir", band, index) in consts:
            key = ("fir", band, index)
        else:
            key = (tag, index)
        pt = consts[key]
        assert pt.level == level, key
        # constants encoded over Q_l * P cross the boundary as their Q rows;
        # the library extends them to the special primes itself
        out.append(np.ascontiguousarray(pt.m[: level + 1]))
    return out


def install_oracle_consts(plan, consts):
    for i, words in enumerate(oracle_const_words(plan, consts)):
        plan.set_const(i, words)


def encrypt_window(P, pk, lay, arrays, seed):
    """arrays: complex [F, R] streams -> ciphertexts (stream, group, re/im order)."""
    out = []
    for si, x in enumerate(arrays):
        re, im = lay.pack(x.real), lay.pack(x.imag)
        for c in range(lay.groups):
            for part, v in enumerate((re[c], im[c])):
                sd = seed + 1000 * si + 2 * c + part
                out.append(ck.encrypt(P, pk, ck.encode(P, v, P.scale, P.L), *synth.encryption_draws(sd, P.n)))
    return out


def read_values(P, sk, cts, readout):
    """The six values of a vital window (num_r, den_r, num_RR, den_RR,
    num_HR, den_HR) from its output ciphertexts (oracle Ciphertexts),
    decrypted and read at the plan's readout positions."""
    dec, vals = {}, []
    for o, slot in readout:
        if o not in dec:
            dec[o] = ck.decrypt_decode(P, sk, cts[o]).real
        vals.append(dec[o][slot])
    return vals


def window_words(cts):
    return np.ascontiguousarray(np.stack([c.words() for c in cts]))


def compare_plan_consts(plan_ref, plan_lib, P, max_frac=1e-3):
    """Every constant of plan_lib equals plan_ref's to +-1 per coefficient
    (last-bit differences of FP64 transcendental values may flip a rounding)."""
    nz = total = 0
    for i in range(plan_ref.num_consts()):
        a, b = plan_ref.get_const(i), plan_lib.get_const(i)
        for r in range(a.shape[0]):
            q = int(P.q[r])
            d = (a[r].astype(object) - b[r].astype(object)) % q
            d = np.where(d > q // 2, d - q, d).astype(np.int64)
            assert np.abs(d).max() <= 1, plan_ref.const_key(i)
            nz += int(np.count_nonzero(d))
            total += d.size
    assert nz <= max_frac * total


def test_fir_dft_circuit_batch_ragged(gsmall):
    """FIR + 200-point DFT on 40 range bins (3 groups, last one partial) for
    two windows in one batch, word-exact; library-designed constants agree
    with the oracle's encoding."""
    import paper_2603_22437_b300 as M
    from oracle import plain
    s = gsmall
    P, ctx, keys = s["P"], s["ctx"], s["keys"]
    circ = cc.FirDftCircuit(P, cc.FirDftConfig(bins=40))
    plan = ctx.plan(M.fir_dft_config(bins=40))
    assert plan.rotations() == circ.rotations()
    consts = circ.constants()
    install_oracle_consts(plan, consts)
    n_in, n_out, lv = plan.io()
    assert n_in == 2 * circ.lay.groups and lv == [P.L - 2] * n_out
    ins, refs = [], []
    for w, seed in enumerate((1000, 1001)):
        win = synth.vital_window(seed, frames=200, bins=40)
        s1, _ = plain.preprocess(win.z)
        cts = encrypt_window(P, s["pk"], circ.lay, [s1], 50 + 10 * w)
        ins.append(window_words(cts))
        pairs = [(cts[2 * c], cts[2 * c + 1]) for c in range(circ.lay.groups)]
        res = circ.run(cc.Evaluator(P, s["rlk"], s["gks"]), consts, pairs)
        refs.append(np.concatenate([x.words().reshape(-1) for pr in res for x in pr]))
    outs = [np.empty_like(r) for r in refs]
    ctx.eval(plan, keys, ins, outs)
    for w in range(2):
        assert np.array_equal(outs[w], refs[w]), "window %d" % w
    plan2 = ctx.plan(M.fir_dft_config(bins=40))
    plan2.encode_consts()
    compare_plan_consts(plan, plan2, P)


def test_launch_trace_is_data_oblivious(gsmall):
    """Theorem 2 on the GPU: the kernel launch sequence (names, grids, blocks)
    is identical for two different inputs."""
    import paper_2603_22437_b300 as M
    P, ctx, keys = gsmall["P"], gsmall["ctx"], gsmall["keys"]
    plan = ctx.plan(M.fir_dft_config(bins=16))
    plan.encode_consts()
    n_in, n_out, _ = plan.io()
    traces = []
    for seed in (1, 2):
        x = rand_ct(P, P.L, seed, n_in)
        out = np.empty(n_out * 2 * (P.L - 1) * P.n, dtype=np.uint64)
        ctx.trace(True)
        ctx.eval(plan, keys, [x], [out])
        traces.append(ctx.trace())
        ctx.trace(False)
    assert traces[0] == traces[1] and len(traces[0]) > 100


def test_bsgs_double_hoisted_two_baby_sets(gsmall):
    """The double-hoisted BSGS product (babies, inner sums and giant-step
    terms over Q*P, one ModDown at the end) with the vital FIR's shape: two
    baby sets of one input at offsets 0 and -1 slot, a negative stride,
    three giant steps, absent (giant, baby) pairs, a batch of two; word-exact
    against the oracle's bsgs_double_hoisted_sets."""
    P, ctx = gsmall["P"], gsmall["ctx"]
    level, n1, stride = P.L, 4, -16
    offsets = [0, -1]
    deltas = {0: [0, 1, 2, 5, 7, 9], 1: [0, 3, 4, 6, 10, 11]}
    rots = sorted(({(b * stride + o) % P.slots for o in offsets for b in range(n1)} |
                   {(g * n1 * stride) % P.slots for g in (1, 2)}) - {0})
    kd = synth.KeyDraws(91, P.n, P.q, P.p, P.dnum, rots)
    gks = {k: ck.gen_galois_key(P, gsmall["sk"], k, *kd.gk[k]) for k in rots}
    keys = load_keys(ctx, P, gsmall["rlk"], gks)
    g = np.random.default_rng(12)
    B = 2
    a = rand_ct(P, level, 13, B)
    diags, lib_diags = {}, []
    for s, ds in deltas.items():
        for d in ds:
            pt = ck.encode_qp(P, g.uniform(-1, 1, P.slots), 2.0 ** 30, level)
            diags[("s%d" % s, d)] = pt
            lib_diags.append((s, d, pt.m[: level + 1]))
    out = np.empty_like(a)
    ctx.ct_bsgs_dh(keys, out, a, B, level, stride, n1, offsets, lib_diags)
    for w in range(B):
        x = as_ct(P, a[w], level)
        ref = ck.bsgs_double_hoisted_sets(P, {"s0": (x, 0), "s1": (x, -1)}, diags, n1, stride, gks)
        assert np.array_equal(out[w], ref.words()), "window %d" % w
