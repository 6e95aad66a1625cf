"""Oracle pins of the per-frame packing (the paper's slow baseline): the
scalar multiply is the encoding of a constant vector, and the per-frame
chain decrypts to the FP64 plaintext pipeline of the same formulas."""
import numpy as np
import pytest

import synth
from oracle import ckks as ck
from oracle import circuits as cc
from oracle import params as pm
from oracle import plain

TINY = dict(bins=4, frames=6, fs_mhz=2000, taps=3)


def test_mul_scalar_is_the_constant_encoding():
    P = pm.fir_dft_params()
    g = np.random.default_rng(2)
    a = ck.Ciphertext(np.stack([g.integers(0, q, P.n, dtype=np.uint64) for q in P.q]),
                      np.stack([g.integers(0, q, P.n, dtype=np.uint64) for q in P.q]), P.L, 2.0 ** 40)
    for c in (0.7312, -2.5, 1e-3):
        got = ck.mul_scalar(P, a, c, float(P.q[P.L]))
        pt = ck.encode(P, np.full(P.slots, c), float(P.q[P.L]), P.L)
        ref = ck.mul_plain(P, a, pt)
        assert np.array_equal(got.words(), ref.words()) and got.scale == ref.scale


@pytest.mark.slow
def test_per_frame_chain_decrypts_to_fp64():
    P = pm.vital_params()
    cfg = cc.VitalConfig(**TINY)
    circ = cc.PerFrameVitalCircuit(P, cfg)
    assert circ.bands == [[1], [3]] and circ.rotations() == [1, 2]
    rots = circ.rotations()
    kd = synth.KeyDraws(77, P.n, P.q, P.p, P.dnum, rots)
    sk = ck.SecretKey(P, kd.secret)
    pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
    rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
    gks = {k: ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
    F, R = cfg.frames, cfg.bins
    g = np.random.default_rng(5)
    z = g.normal(size=(F, R)) + 1j * g.normal(size=(F, R))
    z[:, 1] += 3 * np.exp(1j * 0.8 * np.arange(F))
    s1, s2 = plain.preprocess(z)

    def enc(v, sd):
        x = np.zeros(P.slots)
        x[:R] = v
        return ck.encrypt(P, pk, ck.encode(P, x, P.scale, P.L), *synth.encryption_draws(sd, P.n))

    S1 = [(enc(s1[t].real, 10 + 4 * t), enc(s1[t].imag, 11 + 4 * t)) for t in range(F)]
    S2 = [(enc(s2[t].real, 12 + 4 * t), enc(s2[t].imag, 13 + 4 * t)) for t in range(F)]
    outs = circ.run(cc.Evaluator(P, rlk, gks), circ.constants(), S1, S2)
    assert [o.level for o in outs] == [P.L - 3] * 2 + [P.L - 11] * 4
    dv = [ck.decrypt_decode(P, sk, o)[0] for o in outs]
    sb, mc = plain.side_branch(s1), plain.main_chain(s2, cfg)
    assert abs(dv[0] / dv[1] - sb["num"] / sb["den"]) < 1e-6
    for b in range(2):
        bd = mc["bands"][b]
        assert abs(dv[2 + 2 * b] - bd["num"]) <= 1e-4 * abs(bd["num"])
        assert abs(dv[3 + 2 * b] - bd["den"]) <= 1e-4 * abs(bd["den"])
        assert abs(60 * dv[2 + 2 * b] / dv[3 + 2 * b] - bd["bpm"]) < 1e-3
