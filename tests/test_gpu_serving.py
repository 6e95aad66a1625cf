"""Serving loop on the GPU: windows of several users with their own keys and
uneven frame counts, submitted from two threads while earlier ones run,
under a key budget that holds two users' keys (so keys are evicted and
reloaded).  Every window's output equals, word for word, the same window
evaluated alone with mmfhe_eval; the server's plans carry the oracle's
encoded constants, and the first window of every user also equals the CPU
oracle's evaluation with that user's key words; a user whose keys lack a
rotation fails alone, without disturbing the others."""
import threading
import time

import numpy as np
import pytest

from oracle import ckks as ck
from test_gpu_batching import oracle_fir_dft, oracle_fir_dft_words
from test_gpu_parity import gsmall, install_oracle_consts, oracle_const_words, rand_ct  # noqa: F401  (module fixture)

pytestmark = pytest.mark.gpu


def user_keys(P, rots, seed):
    """Uniform switching-key words (valid residues; the comparison is
    word-exact, so keys need not come from a secret)."""
    g = np.random.default_rng(seed)
    rows = P.q + P.p

    def one():
        out = np.empty((P.dnum, 2, len(rows), P.n), dtype=np.uint64)
        for i, q in enumerate(rows):
            out[:, :, i, :] = g.integers(0, q, out[:, :, i, :].shape, dtype=np.uint64)
        return out

    return one(), {r: one() for r in rots}


@pytest.mark.parametrize("keyip_fused", [0, 1])
def test_serving_mix_equals_alone(gsmall, keyip_fused):
    """keyip_fused = 1: the batches mixing users form each window's key
    inner product (its own key) inside the ModDown passes; the windows
    evaluated alone use the stored inner product, so the two paths are
    compared word for word."""
    import paper_2603_22437_b300 as M
    P, ctx = gsmall["P"], gsmall["ctx"]
    saved = ctx.tuning()
    ctx.set_tuning(saved["ntt_cols_width"], saved["ntt_rows_threads"], saved["keyip_windows"], saved["conv_rows"],
                   keyip_fused)
    base = M.fir_dft_config(bins=40)
    plans = {}
    for F in (200, 150):
        plans[F] = ctx.plan(M.fir_dft_config(bins=40, frames=F))
        install_oracle_consts(plans[F], oracle_fir_dft(P, 40, F)[1])
    rots = sorted(set(plans[200].rotations()) | set(plans[150].rotations()))
    users = {u: user_keys(P, rots, 40 + u) for u in range(3)}
    n_in, _, lv = plans[200].io()
    out_words = sum(2 * (l + 1) * P.n for l in lv)
    key_set = (1 + len(rots)) * P.dnum * 2 * (len(P.q) + len(P.p)) * P.n * 8
    srv = ctx.server(base, max_batch=2, streams=2, key_budget_bytes=2 * key_set + key_set // 2)
    for u, (relin, gal) in users.items():
        srv.add_user(u, relin, gal)
    for F, plan in plans.items():
        for i, words in enumerate(oracle_const_words(plan, oracle_fir_dft(P, 40, F)[1])):
            srv.set_const(F, i, words)
    # user 9: no Galois keys at all -> its windows fail with NOT_FOUND
    bad_relin, _ = user_keys(P, [], 99)
    srv.add_user(9, bad_relin, {})
    with pytest.raises(M.MmfheError) as e:
        srv.submit(12345, 200, np.zeros(8, dtype=np.uint64), np.zeros(8, dtype=np.uint64))
    assert e.value.name == "NOT_FOUND"

    jobs = []
    for i in range(14):
        u = i % 3
        F = 200 if (i // 3) % 2 == 0 else 150
        x = np.ascontiguousarray(rand_ct(P, P.L, 300 + i, n_in).reshape(-1))
        jobs.append((u, F, x, np.zeros(out_words, dtype=np.uint64)))
    tickets = [None] * len(jobs)

    def producer(idx):
        for i in idx:
            u, F, x, out = jobs[i]
            tickets[i] = srv.submit(u, F, x, out)
            time.sleep(0.002 * (i % 3))

    th = [threading.Thread(target=producer, args=(list(range(k, len(jobs), 2)),)) for k in range(2)]
    for t in th:
        t.start()
    bad = srv.submit(9, 200, jobs[0][2], np.zeros(out_words, dtype=np.uint64))
    for t in th:
        t.join()
    lat = [srv.wait(t) for t in tickets]
    assert all(x > 0 for x in lat)
    with pytest.raises(M.MmfheError) as e:
        srv.wait(bad)
    assert e.value.name == "NOT_FOUND"
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(jobs) and st["failed"] == 1 and st["submitted"] == len(jobs) + 1
    assert st["key_loads"] >= 4 and st["key_evictions"] >= 1
    assert st["p99_ms"] >= st["p50_ms"] > 0 and 1 <= st["mean_batch"] <= 2

    # alone: each window by itself, with its own user's keys
    ctx.set_tuning(saved["ntt_cols_width"], saved["ntt_rows_threads"], saved["keyip_windows"], saved["conv_rows"], 0)
    for u in users:
        relin, gal = users[u]
        k = ctx.keys(100 + u)
        k.set_relin(relin)
        for r, w in gal.items():
            k.set_galois(r, w)
        for i, (uu, F, x, out) in enumerate(jobs):
            if uu != u:
                continue
            ref = np.empty(out_words, dtype=np.uint64)
            ctx.eval(plans[F], k, [x], [ref])
            assert np.array_equal(out, ref), "window %d (user %d, F=%d)" % (i, u, F)
        k.unload()
        # the user's first window against the CPU oracle with the user's key words
        i = next(i for i, j in enumerate(jobs) if j[0] == u)
        _, F, x, out = jobs[i]
        orlk = ck.SwitchKey(P, relin)
        ogks = {r: ck.SwitchKey(P, w) for r, w in gal.items()}
        assert np.array_equal(out, oracle_fir_dft_words(P, orlk, ogks, 40, F, x)), "window %d vs the oracle" % i
    ctx.set_tuning(saved["ntt_cols_width"], saved["ntt_rows_threads"], saved["keyip_windows"], saved["conv_rows"],
                   saved["keyip_fused"])


def test_serving_vital_and_gesture_windows_concurrently(gsmall):
    """Two parameter sets on one GPU (the small FIR+DFT instance and the
    gesture chain's N = 2^15, Delta = 2^50 ring), one server each, windows of
    both kinds and several users submitted interleaved from two threads:
    every output equals the window evaluated alone."""
    import paper_2603_22437_b300 as M
    from oracle import params as pm
    from test_gpu_parity import lib_params
    P1, ctx1 = gsmall["P"], gsmall["ctx"]
    P2 = pm.gesture_params()
    ctx2 = M.Context(lib_params(P2))
    gcfg = M.gesture_config(antennas=1, bins=8, chirps=32, frames=4, fc_dims=(7, 5, 3), fc_width=16)
    cfg1 = M.fir_dft_config(bins=40)
    plan1, plan2 = ctx1.plan(cfg1), ctx2.plan(gcfg)
    plan1.encode_consts()
    plan2.encode_consts()
    g = np.random.default_rng(5)
    ard = 1 * 8 * 32
    mats = [np.zeros((16, ard + 1)), np.zeros((16, 16)), np.zeros((16, 16))]
    mats[0][:7] = g.normal(0, 0.1, (7, ard + 1))
    mats[1][:5, :7] = g.normal(0, 0.3, (5, 7))
    mats[2][:3, :5] = g.normal(0, 0.3, (3, 5))
    for m in mats[1:]:
        m[15, 15] = 1.0
    for l, W in enumerate(mats):
        plan2.set_fc_layer(l, W)
    users1 = {u: user_keys(P1, plan1.rotations(), 60 + u) for u in range(2)}
    users2 = {u: user_keys(P2, plan2.rotations(), 70 + u) for u in range(2)}
    srv1 = ctx1.server(cfg1, max_batch=2, streams=2)
    srv2 = ctx2.server(gcfg, max_batch=2, streams=1)
    for l, W in enumerate(mats):
        srv2.set_fc_layer(l, W)
    with pytest.raises(M.MmfheError):
        srv1.set_fc_layer(0, mats[1])      # the FIR+DFT circuit has no learned layers
    for u, (r, gal) in users1.items():
        srv1.add_user(u, r, gal)
    for u, (r, gal) in users2.items():
        srv2.add_user(u, r, gal)
    jobs = []
    for i in range(8):
        kind = i % 2
        P, plan = (P1, plan1) if kind == 0 else (P2, plan2)
        n_in, _, lv = plan.io()
        x = np.ascontiguousarray(rand_ct(P, P.L, 500 + i, n_in).reshape(-1))
        out = np.zeros(sum(2 * (l + 1) * P.n for l in lv), dtype=np.uint64)
        jobs.append((kind, (i // 2) % 2, x, out))
    tickets = [None] * len(jobs)

    def producer(idx):
        for i in idx:
            kind, u, x, out = jobs[i]
            srv = srv1 if kind == 0 else srv2
            tickets[i] = (srv, srv.submit(u, 200 if kind == 0 else 4, x, out))

    th = [threading.Thread(target=producer, args=(list(range(k, len(jobs), 2)),)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    for srv, t in tickets:
        assert srv.wait(t) > 0
    assert srv1.stats()["completed"] == 4 and srv2.stats()["completed"] == 4
    srv1.close()
    srv2.close()
    for kind, ctx, plan, users in ((0, ctx1, plan1, users1), (1, ctx2, plan2, users2)):
        for u, (relin, gal) in users.items():
            k = ctx.keys(200 + u)
            k.set_relin(relin)
            for r, w in gal.items():
                k.set_galois(r, w)
            for i, (kk, uu, x, out) in enumerate(jobs):
                if kk != kind or uu != u:
                    continue
                ref = np.empty_like(out)
                ctx.eval(plan, k, [x], [ref])
                assert np.array_equal(out, ref), "window %d (kind %d, user %d)" % (i, kind, u)
            k.unload()


def test_cancelled_request_never_runs(gsmall):
    """A queued window is cancelled before its batch is dispatched (the
    server holds its first batch up to 3 s for more windows): its wait
    returns CANCELLED and its output buffer stays untouched, the windows
    around it complete with the words they have alone, and a complete
    window or an unknown ticket cannot be cancelled."""
    import paper_2603_22437_b300 as M
    P, ctx = gsmall["P"], gsmall["ctx"]
    base = M.fir_dft_config(bins=40)
    plan = ctx.plan(base)
    plan.encode_consts()
    relin, gal = user_keys(P, plan.rotations(), 77)
    n_in, _, lv = plan.io()
    out_words = sum(2 * (l + 1) * P.n for l in lv)
    srv = ctx.server(base, max_batch=8, streams=1, batch_wait_us=3_000_000)
    srv.add_user(5, relin, gal)
    xs = [np.ascontiguousarray(rand_ct(P, P.L, 700 + i, n_in).reshape(-1)) for i in range(3)]
    outs = [np.zeros(out_words, dtype=np.uint64) for _ in xs]
    tickets = [srv.submit(5, 200, x, o) for x, o in zip(xs, outs)]
    srv.cancel(tickets[1])
    with pytest.raises(M.MmfheError) as e:
        srv.wait(tickets[1])
    assert e.value.name == "CANCELLED"
    for i in (0, 2):
        assert srv.wait(tickets[i]) > 0
    srv.drain()
    st = srv.stats()
    assert st["cancelled"] == 1 and st["completed"] == 2 and st["failed"] == 0
    for name, fn in (("BUSY", lambda: srv.cancel(tickets[0])), ("NOT_FOUND", lambda: srv.cancel(987654))):
        with pytest.raises(M.MmfheError) as e:
            fn()
        assert e.value.name == name
    srv.close()
    assert not outs[1].any()
    k = ctx.keys(55)
    k.set_relin(relin)
    for r, w in gal.items():
        k.set_galois(r, w)
    for i in (0, 2):
        ref = np.empty(out_words, dtype=np.uint64)
        ctx.eval(plan, k, [xs[i]], [ref])
        assert np.array_equal(outs[i], ref), "window %d" % i
    k.unload()
