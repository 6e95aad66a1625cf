"""The allocation-free key switch (mmfhe_keyswitch_noalloc) against the
ordinary one (mmfhe_keyswitch), through the C ABI.

Callers that may not allocate device memory inside a call (host callbacks,
code that must not take the allocator's lock, runtimes owning all device
memory) use the no-allocation variant; its output must equal the ordinary
entry point's word for word -- the tolerance of every integer test here --
on two calls in a row (a relinearization-key switch, then a Galois-key
switch on different input, so stale scratch contents would show), the
first call must also equal the CPU oracle's key switch, the calls must
leave the library's device allocations untouched (no cudaMalloc, no growth
of the context's pool), and it must refuse sizes beyond its fixed scratch
and buffers that are not on the context's device with a clear error.  This
file is collected last so that a run stopping at the first failure has
already run every other test; it builds its own context and passes alone or
after them.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _uniform_rows(g, primes, rows_shape, n):
    out = np.empty(rows_shape + (len(primes), n), dtype=np.uint64)
    for i, q in enumerate(primes):
        out[..., i, :] = g.integers(0, q, out[..., i, :].shape, dtype=np.uint64)
    return out


def test_noalloc_keyswitch_matches_ordinary_twice():
    import torch

    import paper_2603_22437_b300 as M
    from oracle import ckks as ck
    from oracle import params as pm
    from paper_2603_22437_b300 import _lib

    params = M.vital_params()
    P = pm.vital_params()
    assert P.q == params.primes_q and P.p == params.primes_p
    ctx = M.Context(params)
    n = 1 << params.log_n
    q, p = params.primes_q, params.primes_p
    g = np.random.default_rng(77)
    keys = ctx.keys(3)
    relin = np.ascontiguousarray(_uniform_rows(g, q + p, (params.dnum, 2), n))
    keys.set_relin(relin)
    keys.set_galois(64, np.ascontiguousarray(_uniform_rows(g, q + p, (params.dnum, 2), n)))
    dev = torch.device("cuda", 0)
    for call, (level, batch, rotation) in enumerate(((11, 1, None), (7, 2, 64))):
        d = np.ascontiguousarray(_uniform_rows(g, q[: level + 1], (batch,), n))
        ref = np.empty((batch, 2, level + 1, n), dtype=np.uint64)
        ctx.keyswitch(keys, ref, d, batch, level, rotation=rotation)
        d_dev = torch.from_numpy(d.view(np.int64)).to(dev)
        out_dev = torch.zeros((batch, 2, level + 1, n), dtype=torch.int64, device=dev)
        torch.cuda.synchronize()
        before = ctx.mem_stats()
        ctx.keyswitch_noalloc(keys, out_dev, d_dev, batch, level, rotation=rotation)
        torch.cuda.synchronize()
        after = ctx.mem_stats()
        for f in ("device_bytes", "allocations", "pool_bytes", "pool_free_bytes"):
            assert after[f] == before[f], (call, f, before, after)
        got = out_dev.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, ref), "call %d differs from mmfhe_keyswitch" % call
        if call == 0:
            u0, u1 = ck.key_switch(P, d[0], ck.SwitchKey(P, relin), level)
            assert np.array_equal(got[0, 0], u0) and np.array_equal(got[0, 1], u1), "differs from the oracle"

    # sizes beyond the fixed scratch and host buffers are refused with a status
    big = torch.zeros((4, 12, n), dtype=torch.int64, device=dev)
    big_out = torch.zeros((4, 2, 12, n), dtype=torch.int64, device=dev)
    with pytest.raises(_lib.MmfheError) as e:
        ctx.keyswitch_noalloc(keys, big_out, big, 4, 11)
    assert e.value.name == "BAD_ARG" and "scratch" in str(e.value)
    host = np.zeros((1, 12, n), dtype=np.uint64)
    with pytest.raises(_lib.MmfheError) as e:
        ctx.keyswitch_noalloc(keys, np.zeros((1, 2, 12, n), dtype=np.uint64), host, 1, 11)
    assert e.value.name == "BAD_ARG"
