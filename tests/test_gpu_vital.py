"""The vital-sign chain at its full size (N = 2^15, depth 11, 200 frames x 256
range bins, 16 input ciphertexts per window) on the GPU against the oracle:
word-exact output ciphertexts for a window of a batch, batch/alone
equality, and decrypted rates against the FP64 plaintext pipeline."""
import numpy as np
import pytest

import synth
from oracle import ckks as ck
from oracle import circuits as cc
from oracle import params as pm
from oracle import plain

from test_gpu_parity import (compare_plan_consts, encrypt_window, install_oracle_consts, lib_params, load_keys,
                             read_values, window_words)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vital():
    import paper_2603_22437_b300 as M
    P = pm.vital_params()
    cfg = cc.VitalConfig(bins=256, taylor_order=3)
    circ = cc.VitalCircuit(P, cfg)
    rots = circ.rotations()
    kd = synth.KeyDraws(21, P.n, P.q, P.p, P.dnum, rots)
    sk = ck.SecretKey(P, kd.secret)
    pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
    rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
    gks = {k: ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
    del kd
    consts = circ.constants()
    wins, cts = [], []
    for w, seed in enumerate((1001, 1003)):
        win = synth.vital_window(seed, frames=200, bins=256, randomize_rates=True)
        s1, s2 = plain.preprocess(win.z)
        wins.append((s1, s2))
        cts.append(encrypt_window(P, pk, circ.lay, [s1, s2], 300 + 100 * w))
    G = circ.lay.groups
    e = cts[0]
    s1p = [(e[2 * c], e[2 * c + 1]) for c in range(G)]
    s2p = [(e[2 * G + 2 * c], e[2 * G + 2 * c + 1]) for c in range(G)]
    ref0 = circ.run(cc.Evaluator(P, rlk, gks), consts, s1p, s2p)
    ctx = M.Context(lib_params(P))
    keys = load_keys(ctx, P, rlk, gks)
    plan = ctx.plan(M.vital_config(bins=256, taylor_order=3))
    install_oracle_consts(plan, consts)
    return dict(P=P, cfg=cfg, circ=circ, sk=sk, wins=wins, ins=[window_words(c) for c in cts], ref0=ref0,
                ctx=ctx, keys=keys, plan=plan, rots=rots, consts=consts)


def out_buffers(v, B):
    _, n_out, lv = v["plan"].io()
    P = v["P"]
    size = sum(2 * (l + 1) * P.n for l in lv)
    return [np.empty(size, dtype=np.uint64) for _ in range(B)], lv


def split(P, flat, lv):
    outs, off = [], 0
    for l in lv:
        w = 2 * (l + 1) * P.n
        outs.append(flat[off : off + w].reshape(2, l + 1, P.n))
        off += w
    return outs


def test_plan_matches_oracle_structure(vital):
    assert vital["plan"].rotations() == vital["rots"]
    n_in, n_out, lv = vital["plan"].io()
    assert n_in == 16 and n_out == 3
    assert lv == [o.level for o in vital["ref0"]] == [7, 0, 0]
    assert vital["plan"].readout() == vital["circ"].readout()


def test_vital_batch_word_exact_and_decrypted(vital):
    P, ctx = vital["P"], vital["ctx"]
    outs, lv = out_buffers(vital, 2)
    ctx.eval(vital["plan"], vital["keys"], vital["ins"], outs, vital=True)
    got0 = split(P, outs[0], lv)
    for o, (g, r) in enumerate(zip(got0, vital["ref0"])):
        assert np.array_equal(g, r.words()), "output %d" % o
    # window 1 of the batch: decrypt and compare with the FP64 pipeline
    s1, s2 = vital["wins"][1]
    sb, mc = plain.side_branch(s1), plain.main_chain(s2, vital["cfg"])
    scales = [r.scale for r in vital["ref0"]]
    dv = read_values(P, vital["sk"], [ck.Ciphertext(g[0], g[1], l, sc)
                                      for g, l, sc in zip(split(P, outs[1], lv), lv, scales)],
                     vital["circ"].readout())
    assert abs(dv[0] / dv[1] - sb["num"] / sb["den"]) < 1e-6
    for b in range(2):
        bd = mc["bands"][b]
        assert bd["den"] > 1e-4
        assert abs(60 * dv[2 + 2 * b] / dv[3 + 2 * b] - bd["bpm"]) < 1e-3
    # the same window evaluated alone gives the same words
    alone, _ = out_buffers(vital, 1)
    ctx.eval(vital["plan"], vital["keys"], [vital["ins"][1]], alone, vital=True)
    assert np.array_equal(alone[0], outs[1])


def test_library_encoded_plan_matches(vital):
    """The library's own FP64 design of every constant (taps, DFT rows,
    masks, weights) and its encoder agree with the oracle's encoding to
    +-1 per coefficient; decrypted outputs agree to CKKS precision."""
    import paper_2603_22437_b300 as M
    ctx, P = vital["ctx"], vital["P"]
    plan2 = ctx.plan(M.vital_config(bins=256, taylor_order=3))
    plan2.encode_consts()
    compare_plan_consts(vital["plan"], plan2, P)
    outs, lv = out_buffers(vital, 1)
    ctx.eval(plan2, vital["keys"], [vital["ins"][0]], outs, vital=True)
    got = split(P, outs[0], lv)
    ro = vital["circ"].readout()
    va = read_values(P, vital["sk"], [ck.Ciphertext(g[0], g[1], r.level, r.scale) for g, r in zip(got, vital["ref0"])],
                     ro)
    vb = read_values(P, vital["sk"], vital["ref0"], ro)
    for a, b in zip(va, vb):
        assert abs(a - b) <= 1e-6 * max(1.0, abs(b))
    plan2.destroy()


def test_vital_full_batch_in_bench_launch_configuration(vital):
    """The bench's launch configuration: B = 64 windows per launch (the
    bench default), tiles chosen by the autotuner for that batch,
    device-resident buffers.  Window 0 of every pair must equal the oracle's
    output words; window 1 the words it has in the B = 2 run (itself checked
    against the decrypted FP64 pipeline above)."""
    import torch

    P, ctx = vital["P"], vital["ctx"]
    saved = ctx.tuning()
    B = 64
    t = ctx.autotune(B)
    outs2, lv = out_buffers(vital, 2)
    ctx.eval(vital["plan"], vital["keys"], vital["ins"], outs2, vital=True)
    d_in = [torch.from_numpy(vital["ins"][w % 2].reshape(-1).view(np.int64)).cuda() for w in range(B)]
    d_out = [torch.zeros(outs2[0].size, dtype=torch.int64, device="cuda") for _ in range(B)]
    ctx.eval(vital["plan"], vital["keys"], d_in, d_out, vital=True)
    torch.cuda.synchronize()
    ref0 = np.concatenate([r.words().reshape(-1) for r in vital["ref0"]])
    for w in range(B):
        got = d_out[w].cpu().numpy().view(np.uint64)
        assert np.array_equal(got, ref0 if w % 2 == 0 else outs2[1]), "window %d (tiles %s)" % (w, t)
    ctx.set_tuning(saved["ntt_cols_width"], saved["ntt_rows_threads"], saved["keyip_windows"], saved["conv_rows"])


@pytest.fixture(scope="module")
def vital_complex():
    """The same window with complex-slot packing (stream 1 then stream 2, one
    Re + i Im ciphertext per group), its own keys (the conjugation key)."""
    import paper_2603_22437_b300 as M
    P = pm.vital_params()
    cfg = cc.VitalConfig(bins=256, taylor_order=3, complex_slots=True)
    circ = cc.VitalCircuit(P, cfg)
    rots = circ.rotations()
    kd = synth.KeyDraws(22, P.n, P.q, P.p, P.dnum, rots)
    sk = ck.SecretKey(P, kd.secret)
    pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
    rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
    gks = {ck.key_id(P, k): ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
    del kd
    consts = circ.constants()
    win = synth.vital_window(1001, frames=200, bins=256, randomize_rates=True)
    s1, s2 = plain.preprocess(win.z)
    lay = circ.lay

    def stream(x, seed):
        v = lay.pack(x.real) + 1j * lay.pack(x.imag)
        return [ck.encrypt(P, pk, ck.encode(P, v[c], P.scale, P.L), *synth.encryption_draws(seed + c, P.n))
                for c in range(lay.groups)]

    c1, c2 = stream(s1, 400), stream(s2, 500)
    ref = circ.run(cc.Evaluator(P, rlk, gks), consts, c1, c2)
    ctx = M.Context(lib_params(P))
    keys = load_keys(ctx, P, rlk, gks)
    plan = ctx.plan(M.vital_config(bins=256, taylor_order=3, complex_slots=True))
    install_oracle_consts(plan, consts)
    return dict(P=P, cfg=cfg, circ=circ, sk=sk, s=(s1, s2), ins=[window_words(c1 + c2)], ref=ref, ctx=ctx,
                keys=keys, plan=plan)


def test_complex_slot_vital_word_exact_and_decrypted(vital_complex):
    """Complex-slot packing (half the input ciphertexts, 148 key switches
    against 169): output words equal the oracle's; decrypted rates within
    1e-3 bpm of the FP64 pipeline; the library's own constants to +-1."""
    import paper_2603_22437_b300 as M
    v = vital_complex
    P, ctx, plan = v["P"], v["ctx"], v["plan"]
    assert plan.rotations() == v["circ"].rotations() and plan.rotations()[0] == M.ROT_CONJ
    n_in, n_out, lv = plan.io()
    assert n_in == 8 and n_out == 3 and lv == [o.level for o in v["ref"]]
    assert plan.readout() == v["circ"].readout()
    outs, lv = out_buffers(v, 1)
    ctx.eval(plan, v["keys"], v["ins"], outs, vital=True)
    got = split(P, outs[0], lv)
    for o, (g, r) in enumerate(zip(got, v["ref"])):
        assert np.array_equal(g, r.words()), "output %d" % o
    dv = read_values(P, v["sk"], v["ref"], v["circ"].readout())
    sb, mc = plain.side_branch(v["s"][0]), plain.main_chain(v["s"][1], cc.VitalConfig(bins=256, taylor_order=3))
    assert abs(dv[0] / dv[1] - sb["num"] / sb["den"]) < 1e-6
    for b in range(2):
        bd = mc["bands"][b]
        assert bd["den"] > 1e-4       # seed 1001 lies above the noise floor in both bands
        assert abs(60 * dv[2 + 2 * b] / dv[3 + 2 * b] - bd["bpm"]) < 1e-3
    lib = ctx.plan(M.vital_config(bins=256, taylor_order=3, complex_slots=True))
    lib.encode_consts()
    compare_plan_consts(plan, lib, P)
