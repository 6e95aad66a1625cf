"""Oracle pins of the polynomial network (FC layers with square
activations): the diagonal decomposition equals the dense product, and the
homomorphic network decrypts to the FP64 forward pass."""
import numpy as np
import pytest

import synth
from oracle import ckks as ck
from oracle import circuits as cc
from oracle import params as pm


def random_net(cfg, seed, scale=0.3):
    """D x D layer matrices on the FC support, constant row kept."""
    g = np.random.default_rng(seed)
    D, mats = cfg.width, []
    for l in range(len(cfg.dims) - 1):
        W = np.zeros((D, D))
        a, b = cfg.dims[l], cfg.dims[l + 1]
        W[:b, :a] = g.normal(0, scale / np.sqrt(a), (b, a))
        W[:b, D - 1] = g.normal(0, 0.1, b)
        W[D - 1, D - 1] = 1.0
        mats.append(W)
    return mats


def test_fc_diagonals_reconstruct_the_dense_product():
    P = pm.fc_params()
    circ = cc.FcCircuit(P)
    D = circ.D
    mats = random_net(circ.cfg, 3)
    x = cc.fc_pack(np.random.default_rng(4).normal(size=120), D, P.slots)
    for l, W in enumerate(mats):
        y = sum(circ.diagonal(W, k) * cc.rotate_slots(x, k) for k in circ.present(l))
        assert np.allclose(y[:D], W @ x[:D], atol=1e-12)
        assert np.allclose(y, np.tile(W @ x[:D], P.slots // D), atol=1e-12)
    # absent diagonals are exactly zero
    for l, W in enumerate(mats):
        for k in set(range(D)) - set(circ.present(l)):
            assert not np.any(circ.diagonal(W, k))


def test_fc_circuit_decrypts_to_fp64():
    P = pm.fc_params()
    circ = cc.FcCircuit(P)
    D = circ.D
    rots = circ.rotations()
    kd = synth.KeyDraws(31, P.n, P.q, P.p, P.dnum, rots)
    sk = ck.SecretKey(P, kd.secret)
    pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
    rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
    gks = {k: ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
    mats = random_net(circ.cfg, 5)
    consts = circ.constants(mats)
    x = np.random.default_rng(6).normal(size=120)
    ct = ck.encrypt(P, pk, ck.encode(P, cc.fc_pack(x, D, P.slots), P.scale, P.L), *synth.encryption_draws(7, P.n))
    out = circ.run(cc.Evaluator(P, rlk, gks), consts, ct)
    assert out.level == P.L - 2 * (circ.layers - 1) - 1
    got = ck.decrypt_decode(P, sk, out)
    ref = cc.fc_forward(mats, x, D)
    C = circ.cfg.dims[-1]
    for period in (0, 7, P.slots // D - 1):
        assert np.allclose(got[period * D: period * D + C], ref[:C], atol=1e-6 * max(1.0, np.abs(ref[:C]).max()))
