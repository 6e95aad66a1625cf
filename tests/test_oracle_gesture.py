"""Oracle pins of the gesture chain (K3 Doppler DFT -> K1 -> K6 -> soft
power gamma = 4 -> weighting -> frame accumulation -> FC1^2 -> FC2^2 -> FC3):
the FP64 pipeline against numpy's FFT, the notch against its definition, the
slot-domain BSGS and hybrid FC1 decompositions against dense products, and
the homomorphic circuit decrypting to the FP64 pipeline."""
import numpy as np
import pytest

import synth
from oracle import ckks as ck
from oracle import circuits as cc
from oracle import params as pm
from oracle import plain

TINY = cc.GestureConfig(antennas=2, bins=4, chirps=8, frames=20, fc_dims=(7, 5, 3), width=16)


def tiny_params():
    """Test-only ring (N = 2^11, no security claim) with the gesture chain's
    modulus shape: q_0 60 bits + 11 x 50 bits, four 60-bit special primes,
    dnum = 3."""
    return pm.make_params(11, 12, 60, 50, 4, 60, 3, 50)


def random_gesture_net(cfg, seed):
    g = np.random.default_rng(seed)
    W, (d1, d2, c) = cfg.width, cfg.fc_dims
    W0 = np.zeros((W, cfg.ard + 1))
    W0[:d1, : cfg.ard] = g.normal(0, 1.0, (d1, cfg.ard))
    W0[:d1, cfg.ard] = g.normal(0, 0.3, d1)
    W1 = np.zeros((W, W))
    W1[:d2, :d1] = g.normal(0, 0.5 / np.sqrt(d1), (d2, d1))
    W1[:d2, W - 1] = g.normal(0, 0.1, d2)
    W1[W - 1, W - 1] = 1.0
    W2 = np.zeros((W, W))
    W2[:c, :d2] = g.normal(0, 0.5 / np.sqrt(d2), (c, d2))
    W2[:c, W - 1] = g.normal(0, 0.1, c)
    W2[W - 1, W - 1] = 1.0
    return [W0, W1, W2]


def tiny_window(seed, cfg=TINY):
    w = synth.gesture_window(seed, frames=cfg.frames, antennas=cfg.antennas, rbins=cfg.bins, chirps=cfg.chirps)
    return plain.gesture_preprocess(w.z)


def test_doppler_dft_equals_fftshifted_fft():
    zt = tiny_window(1, cc.GestureConfig())
    D = zt.shape[-1]
    ref = np.fft.fftshift(np.fft.fft(zt * cc.hann(D), axis=-1), axes=-1)
    d = plain.gesture_features(zt)["d"]
    assert np.allclose(d, ref, atol=1e-12)
    assert np.abs(d).max() <= 1.0


def test_notch_zeroes_exactly_the_zero_doppler_bin():
    assert list(np.nonzero(cc.notch_mask(32) == 0)[0]) == [16]
    assert list(np.nonzero(cc.notch_mask(33) == 0)[0]) == [16, 17]
    # a chirp-constant (zero-Doppler) signal peaks at the notched bin
    cfg = cc.GestureConfig(antennas=1, bins=1, chirps=32, frames=1)
    zt = np.ones((1, 1, 1, 32), dtype=complex) / cc.hann(32).sum()
    r = plain.gesture_features(zt, cfg)
    assert np.argmax(np.abs(r["d"][0, 0, 0])) == 16
    assert r["p"][0, 0, 0, 16] == 0.0 and r["p"][0, 0, 0, 15] > 0.0


def test_block_diagonal_bsgs_in_the_clear():
    """Slot-domain restatement of K3's BSGS (diagonals, pre-rotation, floor
    split of negative deltas) equals I (x) M applied block by block."""
    P = tiny_params()
    circ = cc.GestureCircuit(P, TINY)
    D, n1 = TINY.chirps, circ.n1
    M = cc.dft_kernel(D).imag
    v = np.random.default_rng(2).normal(size=P.slots) * circ.lay.active()
    babies = [cc.rotate_slots(v, b) for b in range(n1)]
    groups = {}
    for delta in circ.deltas:
        dg = cc.prerotate(circ.doppler_diagonal(M, delta), delta // n1, n1, 1)
        groups.setdefault(delta // n1, []).append(dg * babies[delta % n1])
    out = sum(cc.rotate_slots(sum(t), g * n1) for g, t in groups.items())
    ref = (v.reshape(-1, D) @ M.T).reshape(-1) * circ.lay.active()
    assert np.allclose(out, ref, atol=1e-12)


def test_hybrid_fc1_in_the_clear():
    """FC1's extended diagonals restated on slot vectors give W0 x in slots
    0..width-2 of every period and 0 in slot width-1, the slot of the
    constant 1 the later layers' biases read (its bias is added after FC1).
    Row width-1 of W0 is made nonzero, so a rule that let it into the
    product would leave (W0 x)[width-1] in the constant's slot and fail."""
    P = tiny_params()
    circ = cc.GestureCircuit(P, TINY)
    mats = random_gesture_net(TINY, 3)
    W0 = mats[0][:, : TINY.ard].copy()
    W0[TINY.width - 1] = np.random.default_rng(5).normal(size=TINY.ard)
    x = np.random.default_rng(4).normal(size=TINY.ard)
    xs = np.zeros(P.slots)
    for j in range(circ.lay.k):
        xs[j * circ.lay.ard_pad: j * circ.lay.ard_pad + TINY.ard] = x
    t = sum(circ.fc1_diagonal(W0, k) * cc.rotate_slots(xs, k) for k in range(TINY.width))
    y = t.copy()
    for i in range(int(np.log2(circ.lay.ard_pad // TINY.width))):
        y = y + cc.rotate_slots(y, TINY.width << i)
    want = W0 @ x
    assert abs(want[TINY.width - 1]) > 1e-3
    want[TINY.width - 1] = 0.0
    assert np.allclose(y, np.tile(want, P.slots // TINY.width), atol=1e-9)


def test_depth_and_rotations_full_size():
    P = pm.gesture_params()
    circ = cc.GestureCircuit(P)
    assert (circ.lay.k, circ.lay.pairs) == (2, 30)
    ev = cc.CountingEvaluator(P)

    class Any(dict):
        def __missing__(self, k):
            return None
    pairs = [(cc._Shape(P.L), cc._Shape(P.L)) for _ in range(circ.lay.pairs)]
    assert circ.run(ev, Any(), pairs).level == 0    # depth 11 (Table 1)
    assert len(circ.rotations()) == 23


@pytest.mark.parametrize("frames", [20, 13])
def test_gesture_circuit_decrypts_to_fp64(frames):
    """20 frames fill two ciphertext pairs of 16 frame positions; 13 leave
    the last positions of the only pair empty (ragged tail)."""
    cfg = cc.GestureConfig(antennas=2, bins=4, chirps=8, frames=frames, fc_dims=(7, 5, 3), width=16)
    P = tiny_params()
    circ = cc.GestureCircuit(P, cfg)
    rots = circ.rotations()
    kd = synth.KeyDraws(51, P.n, P.q, P.p, P.dnum, rots)
    sk = ck.SecretKey(P, kd.secret)
    pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
    rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
    gks = {k: ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
    mats = random_gesture_net(cfg, 5)
    consts = circ.constants(mats)
    zt = tiny_window(6, cfg)
    cts = [tuple(ck.encrypt(P, pk, ck.encode(P, v, P.scale, P.L), *synth.encryption_draws(70 + 2 * i + h, P.n))
                 for h, v in enumerate(pair)) for i, pair in enumerate(circ.lay.pack(zt))]
    ev = cc.Evaluator(P, rlk, gks)
    ref = plain.gesture_features(zt, cfg)["feat"]
    feat = circ.features(ev, consts, cts)
    assert feat.level == P.L - 6
    dec = ck.decrypt_decode(P, sk, feat)
    for j in range(circ.lay.k):
        got = dec[j * circ.lay.ard_pad: j * circ.lay.ard_pad + cfg.ard]
        assert np.allclose(got, ref.reshape(-1), atol=1e-9 * max(1.0, np.abs(ref).max()))
    out = circ.run(ev, consts, cts)
    assert out.level == 0
    logits = ck.decrypt_decode(P, sk, out)[: cfg.fc_dims[-1]]
    want = cc.gesture_forward(mats, ref, cfg)[: cfg.fc_dims[-1]]
    assert np.allclose(logits, want, rtol=1e-6, atol=1e-6 * np.abs(want).max())


def test_conjugation_is_slotwise_complex_conjugate():
    """The automorphism X -> X^(2N-1) with its switching key conjugates every
    slot (textbook CKKS property), within the encryption noise."""
    P = tiny_params()
    kd = synth.KeyDraws(81, P.n, P.q, P.p, P.dnum, [ck.ROT_CONJ])
    sk = ck.SecretKey(P, kd.secret)
    pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
    gks = {ck.ROT_CONJ: ck.gen_galois_key(P, sk, ck.ROT_CONJ, *kd.gk[ck.ROT_CONJ])}
    g = np.random.default_rng(82)
    z = g.normal(size=P.slots) + 1j * g.normal(size=P.slots)
    ct = ck.encrypt(P, pk, ck.encode(P, z, P.scale, P.L), *synth.encryption_draws(83, P.n))
    assert np.allclose(ck.decode_complex(P, ck.decrypt(P, sk, ct)), z, atol=1e-8)
    cz = ck.conjugate(P, ct, gks)
    assert np.allclose(ck.decode_complex(P, ck.decrypt(P, sk, cz)), np.conj(z), atol=1e-8)
    assert not np.allclose(np.conj(z), z, atol=1e-3)


def test_complex_block_diagonal_bsgs_in_the_clear():
    """With Re + i Im in one slot, one product by the complex W (its
    diagonals, pre-rotation, floor split) equals d_re + i d_im of Eq. K3."""
    P = tiny_params()
    cfg = cc.GestureConfig(antennas=2, bins=4, chirps=8, frames=20, fc_dims=(7, 5, 3), width=16, complex_slots=True)
    circ = cc.GestureCircuit(P, cfg)
    D, n1 = cfg.chirps, circ.n1
    W = cc.dft_kernel(D)
    g = np.random.default_rng(7)
    v = (g.normal(size=P.slots) + 1j * g.normal(size=P.slots)) * circ.lay.active()
    babies = [cc.rotate_slots(v, b) for b in range(n1)]
    groups = {}
    for delta in circ.deltas:
        dg = cc.prerotate(circ.doppler_diagonal(W, delta), delta // n1, n1, 1)
        groups.setdefault(delta // n1, []).append(dg * babies[delta % n1])
    out = sum(cc.rotate_slots(sum(t), gg * n1) for gg, t in groups.items())
    ref = (v.reshape(-1, D) @ W.T).reshape(-1) * circ.lay.active()
    assert np.allclose(out, ref, atol=1e-12)


@pytest.mark.parametrize("frames", [20, 13])
def test_complex_slot_gesture_circuit_decrypts_to_fp64(frames):
    cfg = cc.GestureConfig(antennas=2, bins=4, chirps=8, frames=frames, fc_dims=(7, 5, 3), width=16,
                           complex_slots=True)
    P = tiny_params()
    circ = cc.GestureCircuit(P, cfg)
    rots = circ.rotations()
    assert rots[0] == ck.ROT_CONJ
    kd = synth.KeyDraws(52, P.n, P.q, P.p, P.dnum, rots)
    sk = ck.SecretKey(P, kd.secret)
    pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
    rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
    gks = {ck.key_id(P, k): ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
    mats = random_gesture_net(cfg, 5)
    consts = circ.constants(mats)
    zt = tiny_window(6, cfg)
    cts = [ck.encrypt(P, pk, ck.encode(P, v, P.scale, P.L), *synth.encryption_draws(90 + i, P.n))
           for i, v in enumerate(circ.lay.pack_complex(zt))]
    ev = cc.Evaluator(P, rlk, gks)
    ref = plain.gesture_features(zt, cfg)["feat"]
    feat = circ.features(ev, consts, cts)
    assert feat.level == P.L - 6
    dec = ck.decrypt_decode(P, sk, feat)
    for j in range(circ.lay.k):
        got = dec[j * circ.lay.ard_pad: j * circ.lay.ard_pad + cfg.ard]
        assert np.allclose(got, ref.reshape(-1), atol=1e-9 * max(1.0, np.abs(ref).max()))
    out = circ.run(ev, consts, cts)
    assert out.level == 0
    logits = ck.decrypt_decode(P, sk, out)[: cfg.fc_dims[-1]]
    want = cc.gesture_forward(mats, ref, cfg)[: cfg.fc_dims[-1]]
    assert np.allclose(logits, want, rtol=1e-6, atol=1e-6 * np.abs(want).max())


def test_learned_feature_map_depth_9_full_size():
    """The learned map a p + b p^2 takes one level where p (p^2)^2 takes
    three: the chain ends at level 0 on the 10-prime parameter set."""
    P = pm.gesture_learned_params()
    circ = cc.GestureCircuit(P, cc.GestureConfig(feature_coef=(1.0, 2.0)))
    ev = cc.CountingEvaluator(P)

    class Any(dict):
        def __missing__(self, k):
            return cc._Shape(0)
    pairs = [(cc._Shape(P.L), cc._Shape(P.L)) for _ in range(circ.lay.pairs)]
    assert P.L == 9 and circ.run(ev, Any(), pairs).level == 0
    assert circ.rotations() == cc.GestureCircuit(pm.gesture_params()).rotations()


@pytest.mark.parametrize("cplx", [False, True])
def test_learned_feature_map_decrypts_to_fp64(cplx):
    """The learned feature map in the encrypted chain (test-only ring with the
    learned chain's 10-prime modulus shape) decrypts to the FP64 features
    a p + b p^2 summed over frames, and its logits to the FP64 network."""
    cfg = cc.GestureConfig(antennas=2, bins=4, chirps=8, frames=20, fc_dims=(7, 5, 3), width=16,
                           feature_coef=(0.7, 2.5), complex_slots=cplx)
    P = pm.make_params(11, 10, 60, 50, 4, 60, 3, 50)
    circ = cc.GestureCircuit(P, cfg)
    rots = circ.rotations()
    kd = synth.KeyDraws(53, P.n, P.q, P.p, P.dnum, rots)
    sk = ck.SecretKey(P, kd.secret)
    pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
    rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
    gks = {ck.key_id(P, k): ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
    mats = random_gesture_net(cfg, 7)
    consts = circ.constants(mats)
    zt = tiny_window(8, cfg)
    if cplx:
        cts = [ck.encrypt(P, pk, ck.encode(P, v, P.scale, P.L), *synth.encryption_draws(90 + 2 * i, P.n))
               for i, v in enumerate(circ.lay.pack_complex(zt))]
    else:
        cts = [tuple(ck.encrypt(P, pk, ck.encode(P, v, P.scale, P.L), *synth.encryption_draws(90 + 2 * i + h, P.n))
                     for h, v in enumerate(pair)) for i, pair in enumerate(circ.lay.pack(zt))]
    ev = cc.Evaluator(P, rlk, gks)
    r = plain.gesture_features(zt, cfg)
    a, b = cfg.feature_coef
    assert np.allclose(r["f"], a * r["p"] + b * r["p"] ** 2)
    feat = circ.features(ev, consts, cts)
    assert feat.level == P.L - 4
    dec = ck.decrypt_decode(P, sk, feat)
    ref = r["feat"]
    for j in range(circ.lay.k):
        got = dec[j * circ.lay.ard_pad: j * circ.lay.ard_pad + cfg.ard]
        assert np.allclose(got, ref.reshape(-1), atol=1e-9 * max(1.0, np.abs(ref).max()))
    out = circ.run(ev, consts, cts)
    assert out.level == 0
    logits = ck.decrypt_decode(P, sk, out)[: cfg.fc_dims[-1]]
    want = cc.gesture_forward(mats, ref, cfg)[: cfg.fc_dims[-1]]
    assert np.allclose(logits, want, rtol=1e-6, atol=1e-6 * np.abs(want).max())
