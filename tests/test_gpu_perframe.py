"""The vital chain with per-frame packing (the paper's slow baseline) on the
GPU against the oracle, word for word, on a small window batch; the
library's own scalar and vector constants against the oracle's design; and
window 1 of the batch decrypted against the FP64 pipeline."""
import numpy as np
import pytest

import synth
from oracle import ckks as ck
from oracle import circuits as cc
from oracle import params as pm
from oracle import plain
from test_gpu_parity import lib_params, load_keys, window_words
from test_oracle_perframe import TINY

pytestmark = pytest.mark.gpu


def test_per_frame_chain_word_exact_and_decrypted():
    import paper_2603_22437_b300 as M
    P = pm.vital_params()
    cfg = cc.VitalConfig(**TINY)
    circ = cc.PerFrameVitalCircuit(P, cfg)
    rots = circ.rotations()
    kd = synth.KeyDraws(78, P.n, P.q, P.p, P.dnum, rots)
    sk = ck.SecretKey(P, kd.secret)
    pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
    rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
    gks = {k: ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
    F, R = cfg.frames, cfg.bins
    wins, cts = [], []
    for w in range(2):
        g = np.random.default_rng(50 + w)
        z = g.normal(size=(F, R)) + 1j * g.normal(size=(F, R))
        z[:, 1] += 3 * np.exp(1j * (0.8 + 0.3 * w) * np.arange(F))
        s1, s2 = plain.preprocess(z)
        wins.append((s1, s2))
        window = []
        for si, s in enumerate((s1, s2)):
            for t in range(F):
                for part, v in enumerate((s[t].real, s[t].imag)):
                    x = np.zeros(P.slots)
                    x[:R] = v
                    sd = 1000 * w + 200 * si + 2 * t + part
                    window.append(ck.encrypt(P, pk, ck.encode(P, x, P.scale, P.L), *synth.encryption_draws(sd, P.n)))
        cts.append(window)
    consts = circ.constants()
    ctx = M.Context(lib_params(P))
    keys = load_keys(ctx, P, rlk, gks)
    plan = ctx.plan(M.vital_config(bins=R, frames=F, fs_mhz=TINY["fs_mhz"], taps=TINY["taps"], per_frame=True))
    assert plan.rotations() == rots
    n_in, n_out, lv = plan.io()
    assert n_in == 4 * F and lv == [P.L - 3] * 2 + [P.L - 11] * 4
    # the library's own design agrees with the oracle's
    lib_scalars = plan.scalars()
    assert np.allclose(lib_scalars, circ.scalars(), rtol=1e-12, atol=1e-15)
    plan.encode_consts()
    for i, (tag, band, index, level) in enumerate(plan.const_keys()):
        a, b = plan.get_const(i), consts[tag].m
        d = np.array([[(int(x) - int(y)) % int(P.q[r]) for x, y in zip(a[r][:64], b[r][:64])] for r in range(level + 1)])
        assert np.all((d <= 1) | (d >= np.array([int(q) - 1 for q in P.q[: level + 1]])[:, None]))
    # word-exact run with the oracle's constants
    for i, (tag, band, index, level) in enumerate(plan.const_keys()):
        plan.set_const(i, np.ascontiguousarray(consts[tag].m))
    plan.set_scalars(circ.scalars())
    size = sum(2 * (l + 1) * P.n for l in lv)
    outs = [np.empty(size, dtype=np.uint64) for _ in range(2)]
    ctx.eval(plan, keys, [window_words(c) for c in cts], outs, vital=True)
    s1p = [(cts[0][2 * t], cts[0][2 * t + 1]) for t in range(F)]
    s2p = [(cts[0][2 * F + 2 * t], cts[0][2 * F + 2 * t + 1]) for t in range(F)]
    ref = circ.run(cc.Evaluator(P, rlk, gks), consts, s1p, s2p)
    assert np.array_equal(outs[0], np.concatenate([r.words().reshape(-1) for r in ref]))
    # window 1 decrypted against the FP64 pipeline
    s1, s2 = wins[1]
    sb, mc = plain.side_branch(s1), plain.main_chain(s2, cfg)
    off, dv = 0, []
    for l, r in zip(lv, ref):
        n = 2 * (l + 1) * P.n
        wds = outs[1][off: off + n].reshape(2, l + 1, P.n)
        dv.append(ck.decrypt_decode(P, sk, ck.Ciphertext(wds[0], wds[1], l, r.scale))[0])
        off += n
    assert abs(dv[0] / dv[1] - sb["num"] / sb["den"]) < 1e-6
    for b in range(2):
        bd = mc["bands"][b]
        assert abs(dv[2 + 2 * b] - bd["num"]) <= 1e-4 * abs(bd["num"])
        assert abs(60 * dv[2 + 2 * b] / dv[3 + 2 * b] - bd["bpm"]) < 1e-3
