"""Decrypted accuracy of the vital chain over many windows (the paper's HR/RR
fidelity against the plaintext pipeline, Table 3: below 1e-3 bpm).

64 seeded full-size windows (200 frames x 256 bins, rates drawn per seed;
seeds 4000..4063, none of them used to calibrate the client's normalizer)
are preprocessed by the client (clutter removal, stream 1 by the window
maximum, stream 2 frame by frame and by the client's normalization factor),
encrypted, evaluated on the GPU in one batch of 64 (the bench's batch),
decrypted, and compared with the FP64 pipeline on the same inputs.

A window is inside the scheme's precision window when both bands' powers
(den, FP64) lie in [5e-3, 1e5]: below, the outputs' absolute noise (~5e-8)
exceeds the 1e-3 bpm budget; above, num nears q_0 / (2 Delta).  Every
window inside must be within 1e-3 bpm in both bands; the count of windows
outside is reported (MMFHE_ACCURACY_OUT names a JSON file for the summary).
The two fixed public gains cannot hold every synthetic window: the chain
raises the band amplitude to the 24th power, and one factor per window
cannot level both bands."""
import json
import multiprocessing as mp
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SEEDS = list(range(4000, 4064))
KEY_SEED = 41
LO, HI = 5e-3, 1e5


def _keys(rot_chunk):
    """Worker: the Galois keys of `rot_chunk` (draws of the full rotation
    list, so every worker sees the same key words); chunk None: the secret,
    public and relinearization keys."""
    import synth
    from oracle import ckks as ck
    from oracle import circuits as cc
    from oracle import params as pm
    P = pm.vital_params()
    rots = cc.VitalCircuit(P, cc.VitalConfig(bins=256)).rotations()
    kd = synth.KeyDraws(KEY_SEED, P.n, P.q, P.p, P.dnum, rots)
    sk = ck.SecretKey(P, kd.secret)
    if rot_chunk is None:
        pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
        return {"secret": kd.secret, "pk": (pk.b, pk.a), "rlk": ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e).data}
    return {k: ck.gen_galois_key(P, sk, k, *kd.gk[k]).data for k in rot_chunk}


def _window(args):
    """Worker: one window preprocessed, normalized and encrypted, with its
    FP64 pipeline results."""
    seed, pk_words = args
    import synth
    from oracle import ckks as ck
    from oracle import circuits as cc
    from oracle import params as pm
    from oracle import plain
    from test_gpu_parity import encrypt_window, window_words
    P = pm.vital_params()
    cfg = cc.VitalConfig(bins=256, taylor_order=3)
    lay = cc.Layout(P.slots, 256, 200)
    win = synth.vital_window(seed, frames=200, bins=256, randomize_rates=True)
    s1, s2 = plain.preprocess(win.z)
    s = plain.stream2_scale(s2, cfg)
    s2 = s2 * s
    pk = ck.PublicKey(*pk_words)
    cts = encrypt_window(P, pk, lay, [s1, s2], 10 * seed)
    sb, mc = plain.side_branch(s1), plain.main_chain(s2, cfg)
    return {"seed": seed, "scale": s, "in": window_words(cts), "r": sb["num"] / sb["den"],
            "bpm": [b["bpm"] for b in mc["bands"]], "den": [b["den"] for b in mc["bands"]]}


def test_decrypted_rates_over_64_windows():
    import paper_2603_22437_b300 as M
    from oracle import ckks as ck
    from oracle import circuits as cc
    from oracle import params as pm
    from test_gpu_parity import install_oracle_consts, lib_params

    P = pm.vital_params()
    circ = cc.VitalCircuit(P, cc.VitalConfig(bins=256))
    rots = circ.rotations()
    workers = max(2, min(16, os.cpu_count() or 2))
    with mp.get_context("spawn").Pool(workers) as pool:
        chunks = [rots[i::workers - 1] for i in range(workers - 1)]
        parts = pool.map(_keys, [None] + chunks)
        base = parts[0]
        wins = pool.map(_window, [(s, base["pk"]) for s in SEEDS])
    gks = {}
    for p in parts[1:]:
        gks.update(p)
    ctx = M.Context(lib_params(P))
    keys = ctx.keys(9)
    keys.set_relin(np.ascontiguousarray(base["rlk"]))
    for k, w in gks.items():
        keys.set_galois(k, np.ascontiguousarray(w))
    plan = ctx.plan(M.vital_config(bins=256, taylor_order=3))
    install_oracle_consts(plan, circ.constants())
    _, _, lv = plan.io()
    out_words = sum(2 * (l + 1) * P.n for l in lv)
    outs = [np.empty(out_words, dtype=np.uint64) for _ in wins]
    ctx.eval(plan, keys, [w["in"] for w in wins], outs, vital=True)
    sk = ck.SecretKey(P, base["secret"])
    # output scales follow the oracle's scale arithmetic (a counting run)
    scales = [o.scale for o in circ.run(cc.CountingEvaluator(P), circ.constants(), *_shapes(circ, P))]
    rows = []
    for w, o in zip(wins, outs):
        dv, off = [], 0
        for l, sc in zip(lv, scales):
            n = 2 * (l + 1) * P.n
            c = o[off : off + n].reshape(2, l + 1, P.n)
            dv.append(ck.decrypt_decode(P, sk, ck.Ciphertext(c[0], c[1], l, sc))[0])
            off += n
        err = [abs(60 * dv[2 + 2 * b] / dv[3 + 2 * b] - w["bpm"][b]) for b in range(2)]
        inside = all(LO <= d <= HI for d in w["den"])
        rows.append({"seed": w["seed"], "scale": w["scale"], "den": w["den"], "bpm": w["bpm"], "err_bpm": err,
                     "err_r": abs(dv[0] / dv[1] - w["r"]), "inside": inside})
    ins = [r for r in rows if r["inside"]]
    summary = {
        "windows": len(rows),
        "inside_precision_window": len(ins),
        "below_floor": sum(1 for r in rows if min(r["den"]) < LO),
        "above_ceiling": sum(1 for r in rows if max(r["den"]) > HI),
        "mae_bpm_inside": {"RR": float(np.mean([r["err_bpm"][0] for r in ins])),
                           "HR": float(np.mean([r["err_bpm"][1] for r in ins]))},
        "max_bpm_inside": float(max(max(r["err_bpm"]) for r in ins)),
        "max_err_target_bin": float(max(r["err_r"] for r in rows)),
        "rows": rows,
    }
    path = os.environ.get("MMFHE_ACCURACY_OUT")
    if path:
        with open(path, "w") as f:
            json.dump(summary, f, indent=1, default=float)
    assert len(ins) >= 0.7 * len(rows)
    for r in ins:
        assert max(r["err_bpm"]) < 1e-3, r
    assert summary["max_err_target_bin"] < 1e-6


def _shapes(circ, P):
    """Top-level stand-ins of one window's inputs for a counting run."""
    from oracle import circuits as cc
    G = circ.lay.groups
    s = [(cc._Shape(P.L, P.scale), cc._Shape(P.L, P.scale)) for _ in range(G)]
    return s, list(s)
