"""Uneven vital-sign windows through the batcher at full size, against the
oracle word for word.

The batching workload draws window lengths of 5..20 s at 20 frames/s, so a
window of F frames runs on a padded frame axis F_pad of 128, 256 or 512
slots, each with its own plan: FIR mask, Hann window, band bins k fs / F,
DFT diagonals, frequency weights and rotation set.  Here one window of
F = 100 (F_pad = 128, 2 groups, 8 input ciphertexts) and one of F = 400
(F_pad = 512, 8 groups, 32 input ciphertexts) are encrypted by the oracle,
queued in one batcher together with a second copy of the F = 400 window
(so that frame count runs as a batch of two), and flushed through captured
graphs.  Every output word must equal the oracle's evaluation of
``VitalCircuit(VitalConfig(frames=F))`` with the oracle's keys and encoded
constants, and the decrypted rates must be within 1e-3 bpm of the FP64
pipeline.

The two oracle chains (about 1 and 2.5 minutes of CPU time) run in spawned
worker processes, one per frame count, started before this test touches
the GPU in its own process state."""
import multiprocessing as mp

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FRAMES = (100, 400)
KEY_SEED = 31
# window seeds whose band powers lie inside the CKKS precision window at the
# default public gains (both bands between 0.05 and 1e4)
WINDOW_SEED = {100: 2105, 400: 2402}


def _union_rotations():
    from oracle import circuits as cc
    from oracle import params as pm
    P = pm.vital_params()
    rots = set()
    for F in FRAMES:
        rots |= set(cc.VitalCircuit(P, cc.VitalConfig(bins=256, frames=F)).rotations())
    return sorted(rots)


def _oracle_window(F):
    """Worker: keys (the draws of the union rotation list, so every worker
    sees the same key words), one encrypted window of F frames, the oracle
    chain.  Returns input words, output words, output scales, FP64 rates and
    this frame count's Galois keys (the constants are rebuilt by the caller)."""
    import synth
    from oracle import ckks as ck
    from oracle import circuits as cc
    from oracle import params as pm
    from oracle import plain
    from test_gpu_parity import encrypt_window, window_words

    P = pm.vital_params()
    cfg = cc.VitalConfig(bins=256, frames=F, taylor_order=3)
    circ = cc.VitalCircuit(P, cfg)
    rots = circ.rotations()
    kd = synth.KeyDraws(KEY_SEED, P.n, P.q, P.p, P.dnum, _union_rotations())
    sk = ck.SecretKey(P, kd.secret)
    pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
    rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
    gks = {k: ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
    win = synth.vital_window(WINDOW_SEED[F], frames=F, bins=256, randomize_rates=True)
    s1, s2 = plain.preprocess(win.z)
    cts = encrypt_window(P, pk, circ.lay, [s1, s2], 700 + F)
    G = circ.lay.groups
    s1p = [(cts[2 * c], cts[2 * c + 1]) for c in range(G)]
    s2p = [(cts[2 * G + 2 * c], cts[2 * G + 2 * c + 1]) for c in range(G)]
    ref = circ.run(cc.Evaluator(P, rlk, gks), circ.constants(), s1p, s2p)
    sb, mc = plain.side_branch(s1), plain.main_chain(s2, cfg)
    fp64 = {"r": sb["num"] / sb["den"], "bpm": [b["bpm"] for b in mc["bands"]], "den": [b["den"] for b in mc["bands"]]}
    return {
        "F": F,
        "in": window_words(cts),
        "out": [r.words() for r in ref],
        "levels": [r.level for r in ref],
        "scales": [r.scale for r in ref],
        "readout": circ.readout(),
        "fp64": fp64,
        "rlk": rlk.data,
        "gks": {k: v.data for k, v in gks.items()},
        "secret": kd.secret,
    }


@pytest.fixture(scope="module")
def uneven():
    with mp.get_context("spawn").Pool(len(FRAMES)) as pool:
        res = pool.map(_oracle_window, FRAMES)
    return {r["F"]: r for r in res}


def test_uneven_vital_windows_through_batcher_match_oracle(uneven):
    import paper_2603_22437_b300 as M
    from oracle import ckks as ck
    from oracle import circuits as cc
    from oracle import params as pm
    from test_gpu_parity import install_oracle_consts, lib_params, read_values

    P = pm.vital_params()
    ctx = M.Context(lib_params(P))
    keys = ctx.keys(5)
    keys.set_relin(np.ascontiguousarray(uneven[FRAMES[0]]["rlk"]))
    gks = {}
    for r in uneven.values():
        gks.update(r["gks"])
    assert sorted(gks) == _union_rotations()
    for k, words in gks.items():
        keys.set_galois(k, np.ascontiguousarray(words))
    b = ctx.batcher(M.vital_config(bins=256), max_batch=4, use_graphs=True)
    for F, r in uneven.items():
        plan = b.plan(F)
        assert set(plan.rotations()) <= set(gks)
        n_in, n_out, lv = plan.io()
        assert n_in == r["in"].shape[0] and lv == r["levels"]
        install_oracle_consts(plan, cc.VitalCircuit(P, cc.VitalConfig(bins=256, frames=F)).constants())
    subs = []
    for F in (400, 100, 400):
        r = uneven[F]
        out = np.zeros(sum(2 * (l + 1) * P.n for l in r["levels"]), dtype=np.uint64)
        b.submit(keys, F, np.ascontiguousarray(r["in"].reshape(-1)), out)
        subs.append((F, out))
    b.flush()
    st = b.stats()
    assert st["windows"] == 3 and st["batches"] == 2 and st["graph_replays"] == 2
    sk = ck.SecretKey(P, uneven[FRAMES[0]]["secret"])
    for i, (F, out) in enumerate(subs):
        r = uneven[F]
        ref = np.concatenate([w.reshape(-1) for w in r["out"]])
        assert np.array_equal(out, ref), "window %d (F=%d) differs from the oracle" % (i, F)
        # decrypted rates against the FP64 pipeline
        cts, off = [], 0
        for l, sc in zip(r["levels"], r["scales"]):
            w = 2 * (l + 1) * P.n
            c = out[off : off + w].reshape(2, l + 1, P.n)
            cts.append(ck.Ciphertext(c[0], c[1], l, sc))
            off += w
        dv = read_values(P, sk, cts, r["readout"])
        assert abs(dv[0] / dv[1] - r["fp64"]["r"]) < 1e-6
        for band in range(2):
            assert r["fp64"]["den"][band] > 0.05
            assert abs(60 * dv[2 + 2 * band] / dv[3 + 2 * band] - r["fp64"]["bpm"][band]) < 1e-3, (F, band)
    b.close()
