"""Decrypted accuracy of the vital chain over many windows (the paper's HR/RR
fidelity against the plaintext pipeline, Table 3: below 1e-3 bpm).

64 seeded full-size windows (200 frames x 256 bins, rates drawn per seed;
seeds 4000..4063, none of them used by the normalizer's CPU pins) are
preprocessed by the client (clutter removal, stream 1 by the window
maximum, stream 2 frame by frame and by the client's normalization factor),
encrypted, evaluated on the GPU in one batch, decrypted, and compared with
the FP64 pipeline on the same inputs.

The client's factor puts both bands' powers (den) at the centre of the
scheme's precision window [5e-3, 1e5] (below, the outputs' absolute noise,
~5e-8, exceeds the 1e-3 bpm budget; above, num nears q_0 / (2 Delta)); a
window whose two bands cannot share one factor is encrypted twice, each
copy normalized for one band, and band b is read from its copy.  Checked:
every band of every window is inside the window in its copy and within
1e-3 bpm of the FP64 pipeline (MMFHE_ACCURACY_OUT names a JSON file for the
summary)."""
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
    """Worker: one window preprocessed, normalized and encrypted (one or two
    copies), with the FP64 pipeline results of each copy."""
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
    pk = ck.PublicKey(*pk_words)
    sb = plain.side_branch(s1)
    copies = []
    for k, (s, bands) in enumerate(plain.stream2_scales(s2, cfg)):
        cts = encrypt_window(P, pk, lay, [s1, s2 * s], 10 * seed + k)
        mc = plain.main_chain(s2 * s, cfg)
        copies.append({"scale": s, "bands": bands, "in": window_words(cts),
                       "bpm": [b["bpm"] for b in mc["bands"]], "den": [b["den"] for b in mc["bands"]]})
    return {"seed": seed, "r": sb["num"] / sb["den"], "copies": copies}


def test_decrypted_rates_over_64_windows():
    import paper_2603_22437_b300 as M
    from oracle import ckks as ck
    from oracle import circuits as cc
    from oracle import params as pm
    from test_gpu_parity import install_oracle_consts, lib_params, read_values

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
    inputs = [c["in"] for w in wins for c in w["copies"]]
    outs = [np.empty(out_words, dtype=np.uint64) for _ in inputs]
    ctx.eval(plan, keys, inputs, outs, vital=True)
    sk = ck.SecretKey(P, base["secret"])
    # output scales follow the oracle's scale arithmetic (a counting run)
    scales = [o.scale for o in circ.run(cc.CountingEvaluator(P), circ.constants(), *_shapes(circ, P))]

    readout = plan.readout()
    assert readout == circ.readout()

    def decrypt(o):
        cts, off = [], 0
        for l, sc in zip(lv, scales):
            n = 2 * (l + 1) * P.n
            c = o[off : off + n].reshape(2, l + 1, P.n)
            cts.append(ck.Ciphertext(c[0], c[1], l, sc))
            off += n
        return read_values(P, sk, cts, readout)

    rows, k = [], 0
    for w in wins:
        err, den, bpm, scl, err_r = [None, None], [None, None], [None, None], [None, None], 0.0
        for c in w["copies"]:
            dv = decrypt(outs[k])
            k += 1
            err_r = max(err_r, abs(dv[0] / dv[1] - w["r"]))
            for b in c["bands"]:
                err[b] = abs(60 * dv[2 + 2 * b] / dv[3 + 2 * b] - c["bpm"][b])
                den[b], bpm[b], scl[b] = c["den"][b], c["bpm"][b], c["scale"]
        rows.append({"seed": w["seed"], "copies": len(w["copies"]), "scale": scl, "den": den, "bpm": bpm,
                     "err_bpm": err, "err_r": err_r, "inside": all(LO <= d <= HI for d in den)})
    summary = {
        "windows": len(rows),
        "copies": len(inputs),
        "split_windows": sum(1 for r in rows if r["copies"] == 2),
        "inside_precision_window": sum(1 for r in rows if r["inside"]),
        "within_1e-3_bpm_both_bands": sum(1 for r in rows if max(r["err_bpm"]) < 1e-3),
        "below_floor": sum(1 for r in rows if min(r["den"]) < LO),
        "above_ceiling": sum(1 for r in rows if max(r["den"]) > HI),
        "mae_bpm": {"RR": float(np.mean([r["err_bpm"][0] for r in rows])),
                    "HR": float(np.mean([r["err_bpm"][1] for r in rows]))},
        "max_bpm": float(max(max(r["err_bpm"]) for r in rows)),
        "max_err_target_bin": float(max(r["err_r"] for r in rows)),
        "rows": rows,
    }
    path = os.environ.get("MMFHE_ACCURACY_OUT")
    if path:
        with open(path, "w") as f:
            json.dump(summary, f, indent=1, default=float)
    assert summary["below_floor"] == 0 and summary["above_ceiling"] == 0
    for r in rows:
        assert max(r["err_bpm"]) < 1e-3, r
    assert summary["max_err_target_bin"] < 1e-6


def _shapes(circ, P):
    """Top-level stand-ins of one window's inputs for a counting run."""
    from oracle import circuits as cc
    G = circ.lay.groups
    s = [(cc._Shape(P.L, P.scale), cc._Shape(P.L, P.scale)) for _ in range(G)]
    return s, list(s)
