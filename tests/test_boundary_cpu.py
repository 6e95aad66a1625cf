"""Host-side checks of what crosses the trust boundary (no GPU): the
parameter fingerprint, the ciphertext header, and the validation of
serialized evaluation keys and plans -- truncated blobs, residues not below
their primes, corrupted words, another parameter set, inconsistent plan
levels -- each returns its status through the C ABI.

The fingerprint and the checksum are recomputed here from their documented
definition (word-wise FNV-1a over 64-bit words) so that the library's
implementation is checked against the format, not against itself."""
import ctypes

import numpy as np
import pytest

FNV_OFFSET, FNV_PRIME, MASK = 0xCBF29CE484222325, 0x100000001B3, (1 << 64) - 1


def fnv_words(words):
    h = FNV_OFFSET
    for w in words:
        h = ((h ^ int(w)) * FNV_PRIME) & MASK
    return h


def uniform_key(g, params):
    n = 1 << params.log_n
    primes = params.primes_q + params.primes_p
    out = np.empty((params.dnum, 2, len(primes), n), dtype=np.uint64)
    for i, q in enumerate(primes):
        out[:, :, i, :] = g.integers(0, q, out[:, :, i, :].shape, dtype=np.uint64)
    return out


def status_of(fn, *args):
    import paper_2603_22437_b300 as M
    with pytest.raises(M.MmfheError) as e:
        fn(*args)
    return e.value.name, str(e.value)


@pytest.fixture(scope="module")
def small():
    import paper_2603_22437_b300 as M
    params = M.fir_dft_params()
    g = np.random.default_rng(4)
    relin = uniform_key(g, params)
    galois = {1: uniform_key(g, params), 16: uniform_key(g, params), M.ROT_CONJ: uniform_key(g, params)}
    return params, relin, galois, M.keys_blob(params, relin, galois)


def test_params_hash_follows_its_definition():
    import paper_2603_22437_b300 as M
    for params in (M.fir_dft_params(), M.vital_params(), M.gesture_params()):
        words = [params.log_n, params.num_q, params.num_p, params.dnum] + params.primes_q + params.primes_p
        assert M.params_hash(params) == fnv_words(words)
    assert len({M.params_hash(p) for p in (M.fir_dft_params(), M.vital_params(), M.gesture_params())}) == 3


def test_ct_header_fields():
    import paper_2603_22437_b300 as M
    params = M.vital_params()
    h = M.ct_header(params, 11, 2.0 ** 40)
    assert ctypes.sizeof(h) == 32
    assert bytes(ctypes.string_at(ctypes.addressof(h), 4)) == b"MMCT"
    assert h.version == 1 and h.level == 11 and h.log2_scale == 40.0 and h.params_hash == M.params_hash(params)
    assert status_of(M.ct_header, params, 12, 2.0 ** 40)[0] == "LEVEL_MISMATCH"
    assert status_of(M.ct_header, params, 3, -1.0)[0] == "BAD_ARG"


def test_key_blob_layout_and_round_trip(small):
    import paper_2603_22437_b300 as M
    params, relin, galois, blob = small
    assert M.blob_check(params, blob) == M.BLOB_KEYS
    w = blob.view(np.uint64)
    assert bytes(w[:1].tobytes()) == b"MMFHEBLB"
    assert int(w[1]) & 0xFFFFFFFF == 1 and int(w[1]) >> 32 == M.BLOB_KEYS
    assert int(w[2]) == M.params_hash(params)
    body = int(w[3])
    assert w.size == 4 + body + 1 and int(w[-1]) == fnv_words(w[:-1])
    kw = params.dnum * 2 * (params.num_q + params.num_p) << params.log_n
    assert int(w[4]) == 4 and int(w[5]) == kw
    ids = w[6:10].view(np.int64).tolist()
    assert ids == [0, M.ROT_CONJ, 1, 16]          # relinearization key first, then rotations as given
    keys = w[10:-1].reshape(4, kw)
    assert np.array_equal(keys[0], relin.reshape(-1)) and np.array_equal(keys[3], galois[16].reshape(-1))


def test_truncated_and_corrupted_key_blobs(small):
    import paper_2603_22437_b300 as M
    params, _, _, blob = small
    # truncated: the header no longer matches the size
    cut = np.ascontiguousarray(blob[: blob.size - 1000])
    name, msg = status_of(M.blob_check, params, cut)
    assert name == "BAD_BLOB" and "size" in msg
    # a word changed without a matching checksum
    bad = blob.copy()
    bad[20] ^= 1
    name, msg = status_of(M.blob_check, params, bad)
    assert name == "BAD_BLOB" and "checksum" in msg
    # a residue equal to its prime, checksum made consistent: the range check catches it
    bad = blob.copy()
    bad[10] = params.primes_q[0]
    bad[-1] = fnv_words(bad[:-1])
    name, msg = status_of(M.blob_check, params, bad)
    assert name == "BAD_BLOB" and "residue" in msg
    # a foreign magic, and an unknown key id
    bad = blob.copy()
    bad[0] = 0
    assert status_of(M.blob_check, params, bad)[0] == "BAD_BLOB"
    bad = blob.copy()
    bad[7] = 0
    bad[-1] = fnv_words(bad[:-1])
    name, msg = status_of(M.blob_check, params, bad)
    assert name == "BAD_BLOB" and "id" in msg


def test_key_blob_of_another_parameter_set(small):
    import paper_2603_22437_b300 as M
    params, _, _, blob = small
    other = M.params_select(13, 4, 44, 40, 1, 44, 2)     # same ring, other digit count
    assert M.params_hash(other) != M.params_hash(params)
    assert status_of(M.blob_check, other, blob)[0] == "PARAM_MISMATCH"


def test_key_blob_writer_refuses_bad_keys(small):
    import paper_2603_22437_b300 as M
    params, relin, galois, _ = small
    bad = relin.copy()
    bad[0, 0, 2, 5] = params.primes_q[2]
    name, msg = status_of(M.keys_blob, params, bad, {})
    assert name == "BAD_BLOB" and "residue" in msg
    assert status_of(M.keys_blob, params, relin, {0: relin})[0] == "BAD_ARG"


def test_plan_blob_round_trip_and_errors():
    import paper_2603_22437_b300 as M
    params = M.fir_dft_params()
    cfg = M.fir_dft_config(bins=16)
    n = 1 << params.log_n
    g = np.random.default_rng(9)
    consts = []
    for lv in (3, 3, 2):
        w = np.stack([g.integers(0, q, n, dtype=np.uint64) for q in params.primes_q[: lv + 1]])
        consts.append((lv, w))
    blob = M.plan_blob(params, cfg, consts)
    assert M.blob_check(params, blob) == M.BLOB_PLAN
    w = blob.view(np.uint64)
    assert int(w[-1]) == fnv_words(w[:-1])
    cfg_words = (ctypes.sizeof(M.CircuitConfig) + 7) // 8
    assert int(w[4]) == ctypes.sizeof(M.CircuitConfig)
    assert int(w[5 + cfg_words]) == 3 and w[6 + cfg_words : 9 + cfg_words].tolist() == [3, 3, 2]
    # the last constant's top row ends the body
    assert np.array_equal(w[-1 - n : -1], consts[2][1][2])
    # a level above the top level, made consistent otherwise
    bad = blob.copy()
    bad[8 + cfg_words] = params.num_q
    bad[-1] = fnv_words(bad[:-1])
    assert status_of(M.blob_check, params, bad)[0] == "BAD_BLOB"
    # truncated
    assert status_of(M.blob_check, params, np.ascontiguousarray(blob[:-9]))[0] == "BAD_BLOB"
    # a residue out of range in a constant
    bad = blob.copy()
    bad[9 + cfg_words] = params.primes_q[0] + 1
    bad[-1] = fnv_words(bad[:-1])
    assert status_of(M.blob_check, params, bad)[0] == "BAD_BLOB"
    assert status_of(M.plan_blob, params, cfg, [(params.num_q, consts[0][1])])[0] == "LEVEL_MISMATCH"


def test_allocation_failure_hook_is_host_side():
    """Arming and disarming the allocation-failure hook needs no device."""
    import paper_2603_22437_b300 as M
    M.debug_fail_allocations(0)
    M.debug_fail_allocations(-1)
