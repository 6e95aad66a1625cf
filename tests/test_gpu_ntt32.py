"""Word-size ablation on the GPU: the 32-bit-word NTT (primes below 2^30)
against the oracle's negacyclic products, word for word."""
import numpy as np
import pytest

from oracle import ckks as ck
from oracle import params as pm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("log_n", [12, 15])
def test_ntt32_polymul_and_round_trip(log_n):
    import torch

    import paper_2603_22437_b300 as M
    n = 1 << log_n
    primes = M.ntt32_primes(log_n, 30, 3) + M.ntt32_primes(log_n, 24, 1)
    nt = M.Ntt32(log_n, primes)
    g = np.random.default_rng(log_n)
    B = 2   # two batches of rows: row r uses primes[r mod 4]
    a = np.stack([g.integers(0, primes[r % 4], n, dtype=np.uint32) for r in range(4 * B)])
    b = np.stack([g.integers(0, primes[r % 4], n, dtype=np.uint32) for r in range(4 * B)])
    fa, fb = a.copy(), b.copy()
    nt.run(fa)                            # host buffers
    da = torch.from_numpy(b.view(np.int32)).cuda()
    nt.run(da)                            # device buffer
    torch.cuda.synchronize()
    fb = da.cpu().numpy().view(np.uint32)
    q = np.array([primes[r % 4] for r in range(4 * B)], dtype=np.uint64)[:, None]
    assert np.all(fa.astype(np.uint64) < q) and np.all(fb.astype(np.uint64) < q)
    c = ((fa.astype(np.uint64) * fb.astype(np.uint64)) % q).astype(np.uint32)
    nt.run(c, inverse=True)
    for r in range(4 * B):
        p = primes[r % 4]
        psi = pm.primitive_2n_root(p, n)
        want = ck.nat.polymul(a[r].astype(np.uint64), b[r].astype(np.uint64), p, psi)
        assert np.array_equal(c[r].astype(np.uint64), want), "row %d" % r
    back = fa.copy()
    nt.run(back, inverse=True)
    assert np.array_equal(back, a)
    nt.close()


def test_ntt32_rejects_bad_primes():
    import paper_2603_22437_b300 as M
    with pytest.raises(M.MmfheError) as e:
        M.Ntt32(12, [(1 << 30) + 8193 * 0 + 1])
    assert e.value.name in ("BAD_BLOB", "BAD_ARG")


def test_ntt_batch_matches_rowwise_transform():
    import torch

    import paper_2603_22437_b300 as M
    P = pm.fir_dft_params()
    ctx = M.Context(M.params_from_primes(P.log_n, P.q, P.p, P.dnum))
    g = np.random.default_rng(3)
    blocks, limbs = 3, len(P.q)
    x = np.stack([np.stack([g.integers(0, q, P.n, dtype=np.uint64) for q in P.q]) for _ in range(blocks)])
    ref = x.reshape(-1, P.n).copy()
    ctx.ntt(ref, [r % limbs for r in range(blocks * limbs)])
    d = torch.from_numpy(x.view(np.int64)).cuda()
    ctx.ntt_batch(d, blocks, limbs)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy().view(np.uint64).reshape(-1, P.n), ref)
    ctx.ntt_batch(d, blocks, limbs, inverse=True)
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy().view(np.uint64), x)
    with pytest.raises(M.MmfheError):
        ctx.ntt_batch(x, blocks, limbs)       # host memory
