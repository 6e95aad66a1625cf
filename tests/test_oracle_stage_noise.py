"""Per-kernel encryption noise of the vital chain (the paper's kernel
fidelity study, Table 2): the MSE and largest absolute error between each
kernel's decrypted output and the same kernel of the FP64 pipeline on the
same inputs, measured cumulatively (after all preceding kernels).  The
oracle's words are the GPU's word for word (the parity tests), so its
intermediates are the library's.

One full-size window at N = 2^15 (64 bins, 200 frames, third-order K7).  The
decoded slots are compared only where the layout holds data:
  K1 energy p[t, r] at slot (t, r); K1 integration E[r] and K2 w = E^2 at
  the block start of the packed side branch; K4 I[t], Q[t] at (t, 0); K5
  band b's filtered I, Q at (t, b); K7 3 dphi (the chain's y (3x^2 - y^2))
  at (t, b); K3 Re X_k at (k, b) and Im X_k at (k + F_pad/2, b); |X_k|^2
  and its square at (k, b).
Every kernel stays below the paper's bound of 1e-5 in MSE, and the decrypted
outputs give the FP64 target bin and rates (Table 3's 1e-3 bpm bound).  With
MMFHE_NOISE_OUT set the measured rows are written there as JSON."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import ckks as ck
from oracle import circuits as cc
from oracle import params as pm
from oracle import plain


@pytest.mark.slow
def test_per_kernel_encryption_noise_and_rates():
    P = pm.vital_params()
    cfg = cc.VitalConfig(bins=64)
    circ = cc.VitalCircuit(P, cfg)
    lay = circ.lay
    rots = circ.rotations()
    kd = synth.KeyDraws(3, P.n, P.q, P.p, P.dnum, rots)
    sk = ck.SecretKey(P, kd.secret)
    pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
    rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
    gks = {k: ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
    del kd
    win = synth.vital_window(1003, frames=200, bins=64, randomize_rates=True)
    s1, s2 = plain.preprocess(win.z)

    def stream(x, seed):
        re, im = lay.pack(x.real), lay.pack(x.imag)
        return [(ck.encrypt(P, pk, ck.encode(P, re[c], P.scale, P.L), *synth.encryption_draws(seed + 2 * c, P.n)),
                 ck.encrypt(P, pk, ck.encode(P, im[c], P.scale, P.L), *synth.encryption_draws(seed + 2 * c + 1, P.n)))
                for c in range(lay.groups)]

    circ.record = {}
    outs = circ.run(cc.Evaluator(P, rlk, gks), circ.constants(), stream(s1, 100), stream(s2, 200))
    taps = circ.record
    sb, mc = plain.side_branch(s1), plain.main_chain(s2, cfg)
    dec = lambda ct: ck.decrypt_decode(P, sk, ct).real
    F, R, H = cfg.frames, cfg.bins, lay.f_pad // 2
    at = lambda v, pos: np.array([v[lay.slot(t, r)] for t, r in pos])
    rows = {}

    def row(name, depth, got, want):
        err = np.asarray(got) - np.asarray(want)
        rows[name] = {"mse": float(np.mean(err ** 2)), "max_abs_err": float(np.abs(err).max()), "depth": depth,
                      "values": int(err.size), "max_abs_value": float(np.abs(want).max())}

    pos_tr = [(t, r) for t in range(F) for r in range(R)]
    row("K1 energy", P.L - taps["K1_energy"][0].level, at(dec(taps["K1_energy"][0]), pos_tr),
        [sb["p"][t, r] for t, r in pos_tr])
    pos_r = [(0, r) for r in range(R)]
    row("K1 integration", P.L - taps["K1_integration"].level, at(dec(taps["K1_integration"]), pos_r), sb["E"])
    row("K2 soft attention", P.L - taps["K2_soft_attention"].level, at(dec(taps["K2_soft_attention"]), pos_r),
        sb["w"])
    I, Q = taps["K4_phase_extraction"]
    pos_t0 = [(t, 0) for t in range(F)]
    row("K4 phase extraction", P.L - I.level, np.concatenate([at(dec(I), pos_t0), at(dec(Q), pos_t0)]),
        np.concatenate([mc["I"], mc["Q"]]))
    If, Qf = taps["K5_fir"]
    got, want = [], []
    for b in range(2):
        pos = [(t, b) for t in range(F)]
        got += [at(dec(If), pos), at(dec(Qf), pos)]
        want += [mc["bands"][b]["If"], mc["bands"][b]["Qf"]]
    row("K5 FIR filter", P.L - If.level, np.concatenate(got), np.concatenate(want))
    d = dec(taps["K7_taylor_arctan"])
    row("K7 Taylor arctan", P.L - taps["K7_taylor_arctan"].level,
        np.concatenate([at(d, [(t, b) for t in range(F)]) for b in range(2)]),
        np.concatenate([3 * mc["bands"][b]["dphi"] for b in range(2)]))
    x, pw, sh = dec(taps["K3_dft"]), dec(taps["power"]), dec(taps["sharpen"])
    g1, w1, g2, w2, g3, w3 = [], [], [], [], [], []
    for b, bd in enumerate(mc["bands"]):
        ks = bd["bins"]
        g1 += [at(x, [(k, b) for k in ks]), at(x, [(k + H, b) for k in ks])]
        w1 += [bd["X"].real, bd["X"].imag]
        g2.append(at(pw, [(k, b) for k in ks]))
        w2.append(bd["P"])
        g3.append(at(sh, [(k, b) for k in ks]))
        w3.append(bd["S"])
    row("K3 narrowband DFT", P.L - taps["K3_dft"].level, np.concatenate(g1), np.concatenate(w1))
    row("|X|^2", P.L - taps["power"].level, np.concatenate(g2), np.concatenate(w2))
    row("sharpen (|X|^2)^2", P.L - taps["sharpen"].level, np.concatenate(g3), np.concatenate(w3))
    path = os.environ.get("MMFHE_NOISE_OUT")
    if path:
        with open(path, "w") as f:
            json.dump({"window_seed": 1003, "bins": R, "frames": F, "rows": rows}, f, indent=1)
    for name, r in rows.items():
        assert r["mse"] < 1e-5, (name, r)
    assert len(outs) == 3
    full = [ck.decrypt_decode(P, sk, o).real for o in outs]
    dv = [full[o][slot] for o, slot in circ.readout()]
    assert abs(dv[0] / dv[1] - sb["num"] / sb["den"]) < 1e-6
    for b in range(2):
        bd = mc["bands"][b]
        assert bd["den"] > 5e-3
        assert abs(60 * dv[2 + 2 * b] / dv[3 + 2 * b] - bd["bpm"]) < 1e-3
