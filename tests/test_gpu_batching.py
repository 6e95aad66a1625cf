"""Batching runtime on the GPU: a captured CUDA graph replays the evaluation
word for word, and the batcher (windows of uneven frame counts from several
users, grouped, cut into batches, replayed from graphs or evaluated directly)
returns for every window exactly the words a lone mmfhe_eval returns.

The batcher's plans carry the oracle's encoded constants, and one window of
every frame count (F = 200 and the uneven F = 150) is compared word for
word with the CPU oracle's evaluation of the same input words; every window
is also compared with the library's own unbatched call on a plan built for
its frame count."""
import numpy as np
import pytest

from oracle import ckks as ck
from oracle import circuits as cc
from test_gpu_parity import gsmall, install_oracle_consts, load_keys, rand_ct  # noqa: F401  (module fixture)

pytestmark = pytest.mark.gpu


def io_words(ctx, plan):
    n_in, n_out, lv = plan.io()
    return n_in * 2 * (ctx.L + 1) * ctx.n, sum(2 * (l + 1) * ctx.n for l in lv)


def window_inputs(P, plan, seed):
    n_in, _, _ = plan.io()
    return np.ascontiguousarray(rand_ct(P, P.L, seed, n_in).reshape(-1))


_ORACLE_CIRCUITS = {}


def oracle_fir_dft(P, bins, frames):
    """The oracle's FIR + DFT circuit and its encoded constants (cached)."""
    key = (P.n, tuple(P.q), bins, frames)
    if key not in _ORACLE_CIRCUITS:
        circ = cc.FirDftCircuit(P, cc.FirDftConfig(bins=bins, frames=frames))
        _ORACLE_CIRCUITS[key] = (circ, circ.constants())
    return _ORACLE_CIRCUITS[key]


def oracle_fir_dft_words(P, rlk, gks, bins, frames, x):
    """The oracle's output words of the FIR + DFT circuit on the input words x
    ([n_in][2][L+1][N] flattened: group c's Re then Im ciphertext)."""
    circ, consts = oracle_fir_dft(P, bins, frames)
    w = x.reshape(-1, 2, P.L + 1, P.n)
    cts = [ck.Ciphertext(w[i][0].copy(), w[i][1].copy(), P.L, P.scale) for i in range(w.shape[0])]
    pairs = [(cts[2 * c], cts[2 * c + 1]) for c in range(circ.lay.groups)]
    res = circ.run(cc.Evaluator(P, rlk, gks), consts, pairs)
    return np.concatenate([ct.words().reshape(-1) for pr in res for ct in pr])


def alone(ctx, plan, keys, x):
    _, ow = io_words(ctx, plan)
    out = np.empty(ow, dtype=np.uint64)
    ctx.eval(plan, keys, [x], [out])
    return out


def test_graph_replay_matches_eval(gsmall):
    import torch

    import paper_2603_22437_b300 as M
    P, ctx, keys = gsmall["P"], gsmall["ctx"], gsmall["keys"]
    plan = ctx.plan(M.fir_dft_config(bins=40))
    plan.encode_consts()
    iw, ow = io_words(ctx, plan)
    B = 2
    d_in = [torch.zeros(iw, dtype=torch.int64, device="cuda") for _ in range(B)]
    d_out = [torch.zeros(ow, dtype=torch.int64, device="cuda") for _ in range(B)]
    g = ctx.graph(plan, keys, d_in, d_out)
    kernels, held = g.info()
    assert kernels > 100 and held > 0
    for trial in range(2):
        xs = [window_inputs(P, plan, 100 + 10 * trial + w) for w in range(B)]
        for w in range(B):
            d_in[w].copy_(torch.from_numpy(xs[w].view(np.int64)))
        l0 = ctx.launch_count()
        g.launch()
        torch.cuda.synchronize()
        assert ctx.launch_count() - l0 == kernels
        ref = [np.empty(ow, dtype=np.uint64) for _ in range(B)]
        ctx.eval(plan, keys, xs, ref)
        for w in range(B):
            assert np.array_equal(d_out[w].cpu().numpy().view(np.uint64), ref[w]), (trial, w)
    g.close()


def test_graph_rejects_host_buffers(gsmall):
    import paper_2603_22437_b300 as M
    P, ctx, keys = gsmall["P"], gsmall["ctx"], gsmall["keys"]
    plan = ctx.plan(M.fir_dft_config(bins=16))
    plan.encode_consts()
    iw, ow = io_words(ctx, plan)
    with pytest.raises(M.MmfheError) as e:
        ctx.graph(plan, keys, [np.zeros(iw, dtype=np.uint64)], [np.zeros(ow, dtype=np.uint64)])
    assert e.value.name == "BAD_ARG"


@pytest.mark.parametrize("use_graphs", [True, False])
def test_batcher_uneven_frames_two_users(gsmall, use_graphs):
    import paper_2603_22437_b300 as M
    P, ctx = gsmall["P"], gsmall["ctx"]
    users = [gsmall["keys"], load_keys(ctx, P, gsmall["rlk"], gsmall["gks"])]
    frames = [200, 150, 200, 150, 200, 200, 150]
    refplans = {}
    b = ctx.batcher(M.fir_dft_config(bins=40), max_batch=2, use_graphs=use_graphs)
    for F in sorted(set(frames)):
        _, consts = oracle_fir_dft(P, 40, F)
        refplans[F] = ctx.plan(M.fir_dft_config(bins=40, frames=F))
        install_oracle_consts(refplans[F], consts)
        install_oracle_consts(b.plan(F), consts)
        assert set(refplans[F].rotations()) <= set(gsmall["gks"])
    subs = []
    for i, F in enumerate(frames):
        x = window_inputs(P, refplans[F], 500 + i)
        out = np.zeros(io_words(ctx, refplans[F])[1], dtype=np.uint64)
        k = users[i % 2]
        b.submit(k, F, x, out)
        subs.append((k, F, x, out))
    b.flush()
    for i, (k, F, x, out) in enumerate(subs):
        assert np.array_equal(out, alone(ctx, refplans[F], k, x)), "window %d (F=%d)" % (i, F)
    if use_graphs:
        # the first window of each frame count against the CPU oracle
        for F in (200, 150):
            i = frames.index(F)
            ref = oracle_fir_dft_words(P, gsmall["rlk"], gsmall["gks"], 40, F, subs[i][2])
            assert np.array_equal(subs[i][3], ref), "window %d (F=%d) differs from the oracle" % (i, F)
    st = b.stats()
    assert st["windows"] == len(frames) and st["plans_created"] == 2
    # (F, user) groups: (200,u0) x3, (150,u1) x2, (200,u1) x1, (150,u0) x1 -> batches of <= 2
    assert st["batches"] == 2 + 1 + 1 + 1
    if use_graphs:
        assert st["graph_replays"] == st["batches"] and st["graphs_captured"] == 5
        # a second flush of the same shapes replays the cached graphs
        for k, F, x, out in subs:
            out[:] = 0
            b.submit(k, F, x, out)
        b.flush()
        assert b.stats()["graphs_captured"] == 5
        for i, (k, F, x, out) in enumerate(subs):
            assert np.array_equal(out, alone(ctx, refplans[F], k, x)), "replay window %d" % i
    b.forget_keys(users[1])
    b.close()


def test_batcher_plan_budget_evicts(gsmall):
    import paper_2603_22437_b300 as M
    P, ctx, keys = gsmall["P"], gsmall["ctx"], gsmall["keys"]
    b = ctx.batcher(M.fir_dft_config(bins=16), max_batch=4, use_graphs=True, plan_budget_bytes=1)
    for rnd in range(2):
        subs = []
        for i, F in enumerate((200, 180)):
            plan = b.plan(F)
            x = window_inputs(P, plan, 900 + 10 * rnd + i)
            out = np.zeros(io_words(ctx, plan)[1], dtype=np.uint64)
            b.submit(keys, F, x, out)
            subs.append((F, x, out))
        b.flush()
        for F, x, out in subs:
            ref = ctx.plan(M.fir_dft_config(bins=16, frames=F))
            ref.encode_consts()
            assert np.array_equal(out, alone(ctx, ref, keys, x)), (rnd, F)
            ref.destroy()
    st = b.stats()
    assert st["plans_evicted"] >= 2 and st["plans_created"] >= 3
    b.close()


def test_every_tile_variant_gives_the_same_words(gsmall):
    """The autotuner only picks among variants that compute identical words:
    the FIR + DFT circuit (NTTs, fused ModUp / ModDown, key inner products of
    relinearisations and rotations) under every tile shape and conversion
    row grouping, the combine on persistent pipelined CTAs or one tile per
    CTA, with the key
    inner product stored by its own kernel (its window walk plain or
    pipelined through shared memory) or formed inside the ModDown passes,
    equals the default-shape result, which
    the parity tests pin to the oracle."""
    import paper_2603_22437_b300 as M
    P, ctx, keys = gsmall["P"], gsmall["ctx"], gsmall["keys"]
    plan = ctx.plan(M.fir_dft_config(bins=40))
    plan.encode_consts()
    xs = [window_inputs(P, plan, 77 + w) for w in range(3)]
    saved = ctx.tuning()
    ctx.set_tuning(16, 256, 4)
    ref = [np.empty(io_words(ctx, plan)[1], dtype=np.uint64) for _ in xs]
    ctx.eval(plan, keys, xs, ref)
    for cw in (8, 16):
        for rt in (128, 256):
            for wg, rg, fu, pi, cp in ((1, 4, 0, 1, 1), (2, 2, 1, 0, 0), (8, 1, 0, 1, 0), (2, 1, 0, 1, 1),
                                       (4, 2, 0, 1, 1), (4, 4, 1, 0, 1)):
                ctx.set_tuning(cw, rt, wg, rg, fu, pi, cp)
                outs = [np.empty_like(r) for r in ref]
                ctx.eval(plan, keys, xs, outs)
                for w in range(3):
                    assert np.array_equal(outs[w], ref[w]), (cw, rt, wg, rg, fu, pi, cp, w)
    with pytest.raises(M.MmfheError):
        ctx.set_tuning(32, 256, 4)
    t = ctx.autotune(3)
    assert t["ntt_cols_width"] in (8, 16) and t["ntt_rows_threads"] in (128, 256)
    assert t["keyip_windows"] in (1, 2, 4, 8)
    assert min(t["ntt_ms"]) > 0 and min(t["keyip_ms"]) > 0 and min(t["keyip_pipe_ms"]) > 0
    assert t["keyip_pipe"] in (0, 1) and t["combine_pipe"] in (0, 1) and min(t["combine_pipe_ms"]) > 0
    assert t["conv_rows"] in (1, 2, 4) and min(t["conv_ms"]) > 0
    assert t["keyip_fused"] == 1   # the last variant's setting: the autotuner leaves it unchanged
    ctx.set_tuning(saved["ntt_cols_width"], saved["ntt_rows_threads"], saved["keyip_windows"], saved["conv_rows"],
                   saved["keyip_fused"])
