"""Gesture chain on the GPU (paper Sec. "Example Pipelines", Encrypted
Dynamic Radar Classification; Table 1 pipeline 2): output ciphertexts word
for word against the oracle for two windows in one batch; the library's own
constant encodings against the oracle's; and a network trained by the
library's plaintext trainer on pooled features of synthetic gesture windows,
whose decrypted encrypted-chain labels equal the FP64 labels."""
import multiprocessing as mp

import numpy as np
import pytest

import synth
from oracle import ckks as ck
from oracle import circuits as cc
from oracle import params as pm
from oracle import plain
from test_gpu_parity import compare_plan_consts, lib_params, load_keys, window_words

pytestmark = pytest.mark.gpu

KEY_SEED = 61
SMALL = cc.GestureConfig(frames=4)          # the full frame shape, 2 ciphertext pairs
SMALL_C = cc.GestureConfig(frames=4, complex_slots=True)   # complex-slot packing: 2 ciphertexts
POOL_R = 4                                  # training features: antennas summed, range pooled by 4


def oracle_setup(cfg):
    P = pm.gesture_params()
    circ = cc.GestureCircuit(P, cfg)
    rots = circ.rotations()
    kd = synth.KeyDraws(KEY_SEED, P.n, P.q, P.p, P.dnum, rots)
    sk = ck.SecretKey(P, kd.secret)
    pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
    rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
    gks = {ck.key_id(P, k): ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
    return P, circ, sk, pk, rlk, gks


def random_mats(cfg, seed):
    g = np.random.default_rng(seed)
    W, (d1, d2, c) = cfg.width, cfg.fc_dims
    W0 = np.zeros((W, cfg.ard + 1))
    W0[:d1, : cfg.ard] = g.normal(0, 1.0, (d1, cfg.ard))
    W0[:d1, cfg.ard] = g.normal(0, 0.3, d1)
    mats = [W0]
    for a, b in ((d1, d2), (d2, c)):
        M = np.zeros((W, W))
        M[:b, :a] = g.normal(0, 0.5 / np.sqrt(a), (b, a))
        M[:b, W - 1] = g.normal(0, 0.1, b)
        M[W - 1, W - 1] = 1.0
        mats.append(M)
    return mats


def encrypt_pairs(P, pk, circ, zt, seed):
    """The window's input ciphertexts: (re, im) per pair, or with complex
    slots one Re + i Im ciphertext per pair."""
    if circ.cfg.complex_slots:
        return [ck.encrypt(P, pk, ck.encode(P, v, P.scale, P.L), *synth.encryption_draws(seed + 2 * i, P.n))
                for i, v in enumerate(circ.lay.pack_complex(zt))]
    return [tuple(ck.encrypt(P, pk, ck.encode(P, v, P.scale, P.L), *synth.encryption_draws(seed + 2 * i + h, P.n))
                  for h, v in enumerate(pair)) for i, pair in enumerate(circ.lay.pack(zt))]


def flat(cts):
    return [c for x in cts for c in (x if isinstance(x, tuple) else (x,))]


def _oracle_window(job):
    """Worker (spawned process): the oracle's output words of window w."""
    w, cplx = job
    cfg = SMALL_C if cplx else SMALL
    P, circ, sk, pk, rlk, gks = oracle_setup(cfg)
    zt = plain.gesture_preprocess(synth.gesture_window(300 + w, frames=cfg.frames).z)
    cts = encrypt_pairs(P, pk, circ, zt, 5000 + 100 * w)
    out = circ.run(cc.Evaluator(P, rlk, gks), circ.constants(random_mats(cfg, 9)), cts)
    return window_words(flat(cts)), out.words(), out.scale


@pytest.fixture(scope="module")
def gest():
    # the oracle runs in spawned processes, started before this process touches the GPU
    pool = mp.get_context("spawn").Pool(4)
    pending = pool.map_async(_oracle_window, [(0, False), (1, False), (0, True), (1, True)])
    import paper_2603_22437_b300 as M
    P, circ, sk, pk, rlk, gks = oracle_setup(SMALL)
    ctx = M.Context(lib_params(P))
    keys = load_keys(ctx, P, rlk, gks)
    _, circ_c, sk_c, pk_c, rlk_c, gks_c = oracle_setup(SMALL_C)
    keys_c = load_keys(ctx, P, rlk_c, gks_c)
    yield dict(P=P, circ=circ, sk=sk, pk=pk, rlk=rlk, gks=gks, ctx=ctx, keys=keys, pending=pending,
               circ_c=circ_c, sk_c=sk_c, pk_c=pk_c, keys_c=keys_c)
    pool.close()
    pool.join()


def install(plan, consts, D):
    for i, (tag, band, index, level) in enumerate(plan.const_keys()):
        if tag in ("gdft_c", "gdft_s", "gdft_ms", "gdft_w"):
            key = (tag, index - D)
        elif tag == "fcw":
            key = ("fcw", band, index)
        else:
            key = (tag,)
        assert consts[key].level == level, key
        plan.set_const(i, np.ascontiguousarray(consts[key].m))


def gesture_config(M, cfg):
    return M.gesture_config(antennas=cfg.antennas, bins=cfg.bins, chirps=cfg.chirps, frames=cfg.frames,
                            fc_dims=cfg.fc_dims, fc_width=cfg.width, complex_slots=cfg.complex_slots,
                            feature_coef=cfg.feature_coef)


def test_gesture_word_exact_two_windows(gest):
    import paper_2603_22437_b300 as M
    P, circ, ctx, keys = gest["P"], gest["circ"], gest["ctx"], gest["keys"]
    plan = ctx.plan(gesture_config(M, SMALL))
    assert plan.rotations() == circ.rotations()
    assert plan.io() == (2 * circ.lay.pairs, 1, [0])
    consts = circ.constants(random_mats(SMALL, 9))
    install(plan, consts, SMALL.chirps)
    ref = gest["pending"].get(timeout=1800)[:2]
    ins = [r[0] for r in ref]
    outs = [np.empty(2 * P.n, dtype=np.uint64) for _ in ref]
    ctx.eval(plan, keys, ins, outs)
    for w, (_, want, scale) in enumerate(ref):
        assert np.array_equal(outs[w], want.reshape(-1)), "window %d" % w
        assert abs(gesture_out_scale(P, circ) / scale - 1) < 1e-12
    # the library's own encoding of the same constants agrees to +-1
    lib = ctx.plan(gesture_config(M, SMALL))
    lib.encode_consts()
    for l, W in enumerate(random_mats(SMALL, 9)):
        lib.set_fc_layer(l, W)
    compare_plan_consts(plan, lib, P)


def test_complex_slot_gesture_word_exact_two_windows(gest):
    """Complex-slot packing (Re + i Im in one slot, one input ciphertext per
    pair, the conjugation key): two windows in one batch word for word
    against the oracle; the library's complex encodings to +-1."""
    import paper_2603_22437_b300 as M
    P, circ, ctx, keys = gest["P"], gest["circ_c"], gest["ctx"], gest["keys_c"]
    plan = ctx.plan(gesture_config(M, SMALL_C))
    assert plan.rotations() == circ.rotations() and plan.rotations()[0] == M.ROT_CONJ
    assert plan.io() == (circ.lay.pairs, 1, [0])
    install(plan, circ.constants(random_mats(SMALL_C, 9)), SMALL_C.chirps)
    ref = gest["pending"].get(timeout=1800)[2:]
    outs = [np.empty(2 * P.n, dtype=np.uint64) for _ in ref]
    ctx.eval(plan, keys, [r[0] for r in ref], outs)
    for w, (_, want, scale) in enumerate(ref):
        assert np.array_equal(outs[w], want.reshape(-1)), "window %d" % w
    lib = ctx.plan(gesture_config(M, SMALL_C))
    lib.encode_consts()
    for l, W in enumerate(random_mats(SMALL_C, 9)):
        lib.set_fc_layer(l, W)
    compare_plan_consts(plan, lib, P)


def pooled(feat):
    """[A, R, D] -> antennas summed, range pooled by POOL_R: [R / POOL_R * D]."""
    A, R, D = feat.shape
    return feat.sum(0).reshape(R // POOL_R, POOL_R, D).sum(1).reshape(-1)


def _features(seed):
    w = synth.gesture_window(seed)
    return pooled(plain.gesture_features(plain.gesture_preprocess(w.z))["feat"]), w.label


def expand_first(first, cfg, kappa):
    """FC1 over the pooled features (scaled by kappa) -> FC1 over every
    feature slot a R D + r D + d (pooling and scale folded into W0)."""
    W0 = np.zeros((cfg.width, cfg.ard + 1))
    a, r, d = np.meshgrid(np.arange(cfg.antennas), np.arange(cfg.bins), np.arange(cfg.chirps), indexing="ij")
    slot = (a * cfg.bins * cfg.chirps + r * cfg.chirps + d).reshape(-1)
    pool_idx = ((r // POOL_R) * cfg.chirps + d).reshape(-1)
    W0[:, slot] = kappa * first[:, pool_idx]
    W0[:, cfg.ard] = first[:, -1]
    return W0


def test_trained_gesture_labels_equal_fp64(gest):
    import paper_2603_22437_b300 as M
    from test_fc_fold import quad_forward
    P, ctx, keys = gest["P"], gest["ctx"], gest["keys"]
    cfg = cc.GestureConfig()
    circ = cc.GestureCircuit(P, cfg)
    n_train, n_test = 2000, 400
    with mp.get_context("spawn").Pool(8) as pool:
        data = pool.map(_features, range(20000, 20000 + n_train + n_test), chunksize=25)
    X = np.array([d[0] for d in data])
    y = np.array([d[1] for d in data], dtype=np.int32)
    kappa = 1.0 / X[:n_train].std(axis=0).max()
    dims = (X.shape[1],) + tuple(cfg.fc_dims)
    alpha = float(np.float32(0.1))
    w, train_acc = ctx.train_poly_net(X[:n_train] * kappa, y[:n_train], dims, alpha=alpha, epochs=40, batch=64,
                                      lr=0.005, seed=5)
    test_pred = np.array([quad_forward(w, dims, alpha, x * kappa).argmax() for x in X[n_train:]])
    test_acc = float((test_pred == y[n_train:]).mean())
    print("gesture network: train %.3f test %.3f" % (train_acc, test_acc))
    assert train_acc > 0.7 and test_acc > 0.6, (train_acc, test_acc)
    first, tail = M.fold_poly_net_wide(dims, alpha, w, cfg.width)
    mats = [expand_first(first, cfg, kappa), tail[0], tail[1]]
    plan = ctx.plan(gesture_config(M, cfg))
    plan.encode_consts()
    for l, Wm in enumerate(mats):
        plan.set_fc_layer(l, Wm)
    sel = list(range(20000 + n_train, 20000 + n_train + 3))
    wins = [synth.gesture_window(s) for s in sel]
    zts = [plain.gesture_preprocess(wd.z) for wd in wins]
    cts = [encrypt_pairs(P, gest["pk"], circ, zt, 7000 + 200 * i) for i, zt in enumerate(zts)]
    ins = [window_words([c for pair in ct for c in pair]) for ct in cts]
    outs = [np.empty(2 * P.n, dtype=np.uint64) for _ in sel]
    ctx.eval(plan, keys, ins, outs)
    C = cfg.fc_dims[-1]
    for j, zt in enumerate(zts):
        feat = plain.gesture_features(zt)["feat"]
        want = cc.gesture_forward(mats, feat, cfg)[:C]
        quad = quad_forward(w, dims, alpha, pooled(feat) * kappa)
        ct = ck.Ciphertext(outs[j].reshape(2, 1, P.n)[0], outs[j].reshape(2, 1, P.n)[1], 0, gesture_out_scale(P, circ))
        got = ck.decrypt_decode(P, gest["sk"], ct)[:C]
        assert got.argmax() == want.argmax() == quad.argmax()
        assert np.allclose(got, want, atol=1e-4 * max(1.0, np.abs(want).max()))
    # the same network on complex-slot packing (one input ciphertext per pair)
    cfg_c = cc.GestureConfig(complex_slots=True)
    circ_c = cc.GestureCircuit(P, cfg_c)
    plan_c = ctx.plan(gesture_config(M, cfg_c))
    plan_c.encode_consts()
    for l, Wm in enumerate(mats):
        plan_c.set_fc_layer(l, Wm)
    cts_c = [encrypt_pairs(P, gest["pk_c"], circ_c, zt, 8000 + 200 * i) for i, zt in enumerate(zts)]
    outs_c = [np.empty(2 * P.n, dtype=np.uint64) for _ in sel]
    ctx.eval(plan_c, gest["keys_c"], [window_words(ct) for ct in cts_c], outs_c)
    for j, zt in enumerate(zts):
        want = cc.gesture_forward(mats, plain.gesture_features(zt)["feat"], cfg)[:C]
        o = outs_c[j].reshape(2, 1, P.n)
        got = ck.decrypt_decode(P, gest["sk_c"], ck.Ciphertext(o[0], o[1], 0, gesture_out_scale(P, circ_c)))[:C]
        assert got.argmax() == want.argmax()
        assert np.allclose(got, want, atol=1e-4 * max(1.0, np.abs(want).max()))


def gesture_out_scale(P, circ):
    """Scale of the logits ciphertext: the evaluator's scale arithmetic
    after FC1 (FC1's output scale from the circuit, then square, FC2,
    square, FC3 with constants at q_l)."""
    q, L = P.q, P.L
    s = circ.fc1_out_scale(P.scale)
    s = s * s / q[L - 7]
    s = s * q[L - 8] / q[L - 8]
    s = s * s / q[L - 9]
    return s * q[L - 10] / q[L - 10]


def test_gesture_bench_launch_configuration(gest):
    """The bench's launch configuration: B = 16 full windows (30 pairs
    each, 480 ciphertexts per Doppler launch), autotuned tiles, device
    buffers.  Every window equals, word for word, the same window in a batch
    of two (whose kernels the word-exact test above ties to the oracle)."""
    import torch

    import paper_2603_22437_b300 as M
    from test_gpu_parity import rand_ct
    P, ctx, keys = gest["P"], gest["ctx"], gest["keys"]
    cfg = cc.GestureConfig()
    plan = ctx.plan(gesture_config(M, cfg))
    plan.encode_consts()
    for l, W in enumerate(random_mats(cfg, 17)):
        plan.set_fc_layer(l, W)
    n_in, _, lv = plan.io()
    saved = ctx.tuning()
    B = 16
    t = ctx.autotune(B)
    wins = [np.ascontiguousarray(rand_ct(P, P.L, 900 + w, n_in).reshape(-1)) for w in range(3)]
    d_in = [torch.from_numpy(wins[w % 3].view(np.int64)).cuda() for w in range(B)]
    d_out = [torch.zeros(2 * P.n, dtype=torch.int64, device="cuda") for _ in range(B)]
    ctx.eval(plan, keys, d_in, d_out)
    torch.cuda.synchronize()
    ref = []
    for w0 in (0, 2):
        outs = [np.empty(2 * P.n, dtype=np.uint64) for _ in range(2)]
        ctx.eval(plan, keys, [wins[w0], wins[(w0 + 1) % 3]], outs)
        ref += outs
    ref = {0: ref[0], 1: ref[1], 2: ref[2]}
    for w in range(B):
        assert np.array_equal(d_out[w].cpu().numpy().view(np.uint64), ref[w % 3]), "window %d (tiles %s)" % (w, t)
    ctx.set_tuning(saved["ntt_cols_width"], saved["ntt_rows_threads"], saved["keyip_windows"], saved["conv_rows"])
