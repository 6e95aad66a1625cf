"""Pin of the vital chain's packed side branch (K1 energy, K2 soft power
attention, target-bin num / den) with several groups.

At 256 bins and 200 frames the window spans G = 4 groups of 64 bins.  The
oracle halves each group's frame sums twice, masks the first 64-frame block,
packs the four groups into one ciphertext, finishes the frame sums over a
block and then sums over bins and blocks, den's terms one frame after
num's in the same ciphertext.  A wrong block assignment, mask or
index vector moves energy between bins or groups; the check is against the
FP64 definition (E_r = sum_t |z[t, r]|^2, w = E^2, num = sum r w,
den = sum w), decrypted, on a window whose target bin lies in the third
group."""
import numpy as np

import synth
from oracle import ckks as ck
from oracle import circuits as cc
from oracle import params as pm
from oracle import plain


def test_packed_side_branch_decrypts_to_fp64():
    P = pm.vital_params()
    cfg = cc.VitalConfig(bins=256)
    circ = cc.VitalCircuit(P, cfg)
    lay = circ.lay
    assert lay.groups == 4 and circ.side_groups() == 4 and circ.side_block() == 64
    assert [circ.side_block_of(c) for c in range(4)] == [0, 3, 2, 1]
    rots = sorted({(lay.r_c << i) % P.slots for i in range(8)} | {1 << i for i in range(6)} | {(-lay.r_c) % P.slots})
    kd = synth.KeyDraws(11, P.n, P.q, P.p, P.dnum, rots)
    sk = ck.SecretKey(P, kd.secret)
    pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
    rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
    gks = {k: ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
    del kd
    seed = next(s for s in range(5000, 5100) if 128 <= synth.vital_window(s, bins=256).target_bin < 192)
    win = synth.vital_window(seed, frames=200, bins=256)
    s1, _ = plain.preprocess(win.z)
    re, im = lay.pack(s1.real), lay.pack(s1.imag)
    cts = [(ck.encrypt(P, pk, ck.encode(P, re[c], P.scale, P.L), *synth.encryption_draws(300 + 2 * c, P.n)),
            ck.encrypt(P, pk, ck.encode(P, im[c], P.scale, P.L), *synth.encryption_draws(301 + 2 * c, P.n)))
           for c in range(lay.groups)]
    consts = circ.constants()
    ev = cc.Evaluator(P, rlk, gks)
    ps = [ev.rescale(ev.square_sum([a, b])) for a, b in cts]
    side = circ.side_branch(ev, consts, ps)
    assert side.level == P.L - 4
    v = ck.decrypt_decode(P, sk, side).real
    got_num, got_den = v[0], v[lay.r_c]      # den one frame after num
    assert circ.readout()[:2] == [(0, 0), (0, lay.r_c)]
    sb = plain.side_branch(s1)
    assert abs(got_den / sb["den"] - 1) < 1e-5
    assert abs(got_num / sb["num"] - 1) < 1e-5
    assert abs(got_num / got_den - sb["num"] / sb["den"]) < 1e-6
    assert round(sb["num"] / sb["den"]) == win.target_bin
