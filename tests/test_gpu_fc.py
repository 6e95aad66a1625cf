"""Polynomial network (the paper's FC network with square activations) on
the GPU: the circuit against the oracle word for word; the plaintext GPU
training on synthetic gesture features; encrypted inference whose decrypted
labels equal the FP64 labels of the same network."""
import numpy as np
import pytest

import synth
from oracle import ckks as ck
from oracle import circuits as cc
from oracle import params as pm
from test_fc_fold import quad_forward
from test_gpu_parity import lib_params, load_keys, window_words
from test_oracle_fc import random_net

pytestmark = pytest.mark.gpu

DIMS = (120, 32, 16, 6)


@pytest.fixture(scope="module")
def fc():
    import paper_2603_22437_b300 as M
    P = pm.fc_params()
    circ = cc.FcCircuit(P, cc.FcConfig(dims=DIMS))
    rots = circ.rotations()
    kd = synth.KeyDraws(41, P.n, P.q, P.p, P.dnum, rots)
    sk = ck.SecretKey(P, kd.secret)
    pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
    rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
    gks = {k: ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
    ctx = M.Context(lib_params(P))
    keys = load_keys(ctx, P, rlk, gks)
    return dict(P=P, circ=circ, sk=sk, pk=pk, rlk=rlk, gks=gks, ctx=ctx, keys=keys, rots=rots)


def encrypt_features(f, x, seed):
    P = f["P"]
    v = cc.fc_pack(x, f["circ"].D, P.slots)
    return ck.encrypt(P, f["pk"], ck.encode(P, v, P.scale, P.L), *synth.encryption_draws(seed, P.n))


def test_fc_circuit_word_exact(fc):
    import paper_2603_22437_b300 as M
    P, circ, ctx, keys = fc["P"], fc["circ"], fc["ctx"], fc["keys"]
    plan = ctx.plan(M.fc_config(DIMS))
    assert plan.rotations() == fc["rots"]
    n_in, n_out, lv = plan.io()
    assert (n_in, n_out, lv) == (1, 1, [P.L - 2 * circ.layers + 1])
    mats = random_net(circ.cfg, 9)
    consts = circ.constants(mats)
    for i, (tag, layer, k, level) in enumerate(plan.const_keys()):
        assert tag == "fcw" and consts[("fcw", layer, k)].level == level
        plan.set_const(i, np.ascontiguousarray(consts[("fcw", layer, k)].m))
    xs = [np.random.default_rng(10 + w).normal(size=DIMS[0]) for w in range(3)]
    cts = [encrypt_features(fc, x, 60 + w) for w, x in enumerate(xs)]
    ins = [window_words([c]) for c in cts]
    outs = [np.empty(2 * (lv[0] + 1) * P.n, dtype=np.uint64) for _ in xs]
    ctx.eval(plan, keys, ins, outs)
    ev = cc.Evaluator(P, fc["rlk"], fc["gks"])
    for w, c in enumerate(cts):
        ref = circ.run(ev, consts, c)
        assert np.array_equal(outs[w], ref.words().reshape(-1)), "window %d" % w
    # the library's own encoder of the same matrices agrees to +-1 per coefficient
    plan2 = ctx.plan(M.fc_config(DIMS))
    for l, W in enumerate(mats):
        plan2.set_fc_layer(l, W)
    nz = total = 0
    for i in range(plan.num_consts()):
        a, b = plan.get_const(i), plan2.get_const(i)
        for r in range(a.shape[0]):
            q = int(P.q[r])
            d = (a[r].astype(object) - b[r].astype(object)) % q
            d = np.where(d > q // 2, d - q, d).astype(np.int64)
            assert np.abs(d).max() <= 1
            nz += int(np.count_nonzero(d))
            total += d.size
    assert nz <= 1e-3 * total
    with pytest.raises(M.MmfheError):
        plan2.encode_consts()


def test_trained_network_encrypted_labels_equal_fp64(fc):
    import paper_2603_22437_b300 as M
    P, circ, ctx, keys = fc["P"], fc["circ"], fc["ctx"], fc["keys"]
    X, y = synth.gesture_dataset(0, 6000)
    alpha = float(np.float32(0.1))
    w, train_acc = ctx.train_poly_net(X[:5000], y[:5000], DIMS, alpha=alpha, epochs=20, batch=128, lr=0.05, seed=3)
    test_pred = np.array([quad_forward(w, DIMS, alpha, x).argmax() for x in X[5000:]])
    test_acc = float((test_pred == y[5000:]).mean())
    assert train_acc > 0.9 and test_acc > 0.9, (train_acc, test_acc)
    mats = M.fold_poly_net(DIMS, alpha, w, circ.D)
    plan = ctx.plan(M.fc_config(DIMS))
    for l, W in enumerate(mats):
        plan.set_fc_layer(l, W)
    _, _, lv = plan.io()
    sel = list(range(5000, 5008))
    cts = [encrypt_features(fc, X[i], 900 + i) for i in sel]
    outs = [np.empty(2 * (lv[0] + 1) * P.n, dtype=np.uint64) for _ in sel]
    ctx.eval(plan, keys, [window_words([c]) for c in cts], outs)
    C = DIMS[-1]
    # the output scale follows from the level schedule alone: take it from the oracle's run
    scale_out = circ.run(cc.Evaluator(P, fc["rlk"], fc["gks"]), circ.constants(mats), cts[0]).scale
    for j, i in enumerate(sel):
        ref = cc.fc_forward(mats, X[i], circ.D)[:C]
        words = outs[j].reshape(2, lv[0] + 1, P.n)
        dec = ck.decrypt_decode(P, fc["sk"], ck.Ciphertext(words[0], words[1], lv[0], scale_out))[:C]
        assert dec.argmax() == ref.argmax() == quad_forward(w, DIMS, alpha, X[i]).argmax()
        assert np.allclose(dec, ref, atol=1e-4 * max(1.0, np.abs(ref).max()))
