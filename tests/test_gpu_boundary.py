"""The boundary on the GPU, through the C ABI: evaluation keys and a plan
loaded from serialized blobs evaluate the small FIR + DFT circuit to the
oracle's words; the header-checked evaluation reports the outputs' levels
and scales as the oracle tracks them and refuses ciphertexts of another
parameter set or level; blobs of another parameter set or truncated blobs
are refused before anything is uploaded; an allocation failure injected on
the host returns OUT_OF_MEMORY and leaves the context usable."""
import math

import numpy as np
import pytest

from oracle import ckks as ck
from test_gpu_batching import oracle_fir_dft
from test_gpu_parity import gsmall, lib_params, oracle_const_words  # noqa: F401  (module fixture)

pytestmark = pytest.mark.gpu


def _blobs(s):
    import paper_2603_22437_b300 as M
    P = s["P"]
    params = lib_params(P)
    kb = M.keys_blob(params, s["rlk"].data, {k: v.data for k, v in s["gks"].items()})
    cfg = M.fir_dft_config(bins=40)
    ref_plan = s["ctx"].plan(cfg)
    circ, consts = oracle_fir_dft(P, 40, 200)
    words = oracle_const_words(ref_plan, consts)
    pb = M.plan_blob(params, cfg, [(ref_plan.const_key(i)[3], w) for i, w in enumerate(words)])
    return params, kb, pb, circ, consts


def _window(s, circ, seed):
    from oracle import plain
    import synth
    from test_gpu_parity import encrypt_window, window_words
    P = s["P"]
    win = synth.vital_window(seed, frames=200, bins=40)
    s1, _ = plain.preprocess(win.z)
    cts = encrypt_window(P, s["pk"], circ.lay, [s1], 90)
    return cts, window_words(cts)


def test_loaded_keys_and_plan_match_oracle_with_headers(gsmall):
    import paper_2603_22437_b300 as M
    s = gsmall
    P, ctx = s["P"], s["ctx"]
    params, kb, pb, circ, consts = _blobs(s)
    keys = ctx.keys_load(kb, user_id=12)
    plan = ctx.plan_load(pb)
    assert plan.rotations() == circ.rotations()
    cts, x = _window(s, circ, 1002)
    pairs = [(cts[2 * c], cts[2 * c + 1]) for c in range(circ.lay.groups)]
    from oracle import circuits as cc
    res = circ.run(cc.Evaluator(P, s["rlk"], s["gks"]), consts, pairs)
    ref = np.concatenate([ct.words().reshape(-1) for pr in res for ct in pr])
    n_in, n_out, lv = plan.io()
    hin = [[M.ct_header(params, P.L, P.scale)] * n_in]
    out = np.zeros_like(ref)
    hout = ctx.eval_checked(plan, keys, hin, [x], [out])
    assert np.array_equal(out, ref)
    flat = [ct for pr in res for ct in pr]
    assert len(hout[0]) == n_out == len(flat)
    for h, ct in zip(hout[0], flat):
        assert h.level == ct.level and h.params_hash == M.params_hash(params)
        assert abs(h.log2_scale - math.log2(ct.scale)) < 1e-9
    # the same evaluation without headers
    out2 = np.zeros_like(ref)
    ctx.eval(plan, keys, [x], [out2])
    assert np.array_equal(out2, ref)

    def refused(hdrs, **kw):
        with pytest.raises(M.MmfheError) as e:
            ctx.eval_checked(plan, keys, hdrs, [x], [np.zeros_like(ref)], **kw)
        return e.value.name

    other = M.vital_params()
    assert refused([[M.ct_header(other, P.L, P.scale)] * n_in]) == "PARAM_MISMATCH"
    assert refused([[M.ct_header(params, P.L - 1, P.scale)] * n_in]) == "LEVEL_MISMATCH"
    mixed = [M.ct_header(params, P.L, P.scale)] * (n_in - 1) + [M.ct_header(params, P.L, 2 * P.scale)]
    assert refused([mixed]) == "BAD_ARG"
    junk = M.ct_header(params, P.L, P.scale)
    junk.magic = 0
    assert refused([[junk] * n_in]) == "BAD_BLOB"
    keys.unload()
    plan.destroy()


def test_blobs_of_another_parameter_set_or_truncated_are_refused(gsmall):
    import paper_2603_22437_b300 as M
    s = gsmall
    ctx = s["ctx"]
    _, kb, pb, _, _ = _blobs(s)
    vctx = M.Context(M.vital_params())
    for fn, blob in ((vctx.keys_load, kb), (vctx.plan_load, pb)):
        with pytest.raises(M.MmfheError) as e:
            fn(blob)
        assert e.value.name == "PARAM_MISMATCH"
    for fn, blob in ((ctx.keys_load, kb), (ctx.plan_load, pb)):
        with pytest.raises(M.MmfheError) as e:
            fn(np.ascontiguousarray(blob[:-100]))
        assert e.value.name == "BAD_BLOB"


def test_injected_allocation_failure_returns_out_of_memory(gsmall):
    """A fresh context (empty scratch pool): with the hook armed, the first
    evaluation needs device scratch and fails with OUT_OF_MEMORY; disarmed,
    the same context evaluates the window to the oracle's words."""
    import paper_2603_22437_b300 as M
    s = gsmall
    P = s["P"]
    params, kb, pb, circ, consts = _blobs(s)
    ctx = M.Context(params)
    keys = ctx.keys_load(kb)
    plan = ctx.plan_load(pb)
    cts, x = _window(s, circ, 1004)
    _, n_out, lv = plan.io()
    out = np.zeros(n_out * 2 * (lv[0] + 1) * P.n, dtype=np.uint64)
    before = ctx.mem_stats()
    try:
        M.debug_fail_allocations(0)
        with pytest.raises(M.MmfheError) as e:
            ctx.eval(plan, keys, [x], [out])
        assert e.value.name == "OUT_OF_MEMORY" and "injected" in str(e.value)
    finally:
        M.debug_fail_allocations(-1)
    assert ctx.mem_stats()["allocations"] == before["allocations"]
    ctx.eval(plan, keys, [x], [out])
    from oracle import circuits as cc
    pairs = [(cts[2 * c], cts[2 * c + 1]) for c in range(circ.lay.groups)]
    res = circ.run(cc.Evaluator(P, s["rlk"], s["gks"]), consts, pairs)
    assert np.array_equal(out, np.concatenate([ct.words().reshape(-1) for pr in res for ct in pr]))
    st = ctx.mem_stats()
    assert st["allocations"] > before["allocations"] and st["peak_bytes"] >= st["device_bytes"] > 0
    assert st["pool_bytes"] > 0
