"""Host side of the word-size ablation: the 32-bit prime rule (no GPU)."""
import pytest
import sympy


@pytest.mark.parametrize("log_n,bits,count", [(15, 30, 24), (13, 28, 6), (10, 20, 4)])
def test_ntt32_primes_are_the_largest_ntt_primes(log_n, bits, count):
    import paper_2603_22437_b300 as M
    ps = M.ntt32_primes(log_n, bits, count)
    m = 2 << log_n
    assert len(ps) == count and ps == sorted(ps, reverse=True)
    for p in ps:
        assert sympy.isprime(p) and p % m == 1 and p < 2 ** bits
    # nothing of the form k 2N + 1 between them (or above the first) is prime
    for x in range(ps[0] + m, 2 ** bits, m):
        assert not sympy.isprime(x)
    for hi, lo in zip(ps, ps[1:]):
        for x in range(lo + m, hi, m):
            assert not sympy.isprime(x)


def test_ntt32_primes_bad_args():
    import paper_2603_22437_b300 as M
    with pytest.raises(M.MmfheError):
        M.ntt32_primes(15, 31, 1)        # words must keep 4q below 2^32
    with pytest.raises(M.MmfheError):
        M.ntt32_primes(16, 30, 1)        # a 32-bit row of 2^16 words exceeds shared memory
