"""CPU-side checks of the C ABI: the shared library loads and exports every
symbol include/mmfhe.h declares; host-only entry points (prime selection,
encoder, window packing) agree with the oracle; without a GPU the device
entry points fail with a status instead of crashing."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    src = open(os.path.join(ROOT, "include", "mmfhe.h")).read()
    return sorted(set(re.findall(r"\b(mmfhe_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_header_symbol():
    from paper_2603_22437_b300 import _lib
    L = _lib.lib()
    names = header_symbols()
    assert len(names) >= 35
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_params_select_matches_oracle():
    import paper_2603_22437_b300 as M
    from oracle import params as pm
    for mine, ref in ((M.fir_dft_params(), pm.fir_dft_params()), (M.vital_params(), pm.vital_params())):
        assert mine.primes_q == ref.q and mine.primes_p == ref.p


def test_params_select_rejects_bad_args():
    import paper_2603_22437_b300 as M
    with pytest.raises(M.MmfheError) as e:
        M.params_select(9, 4, 44, 40, 1, 44, 4)
    assert e.value.name == "BAD_ARG"


def test_encoder_matches_oracle():
    import paper_2603_22437_b300 as M
    from oracle import ckks as ck
    from oracle import params as pm
    P = pm.vital_params()
    p = M.vital_params()
    z = np.random.default_rng(3).uniform(-2, 2, P.slots)
    for scale, level in ((P.scale, P.L), (float(P.q[5]), 5)):
        a = M.encode(p, z, scale, level)
        b = ck.encode(P, z, scale, level).m
        assert np.array_equal(a, b)


def test_pack_window_matches_oracle_layout():
    import paper_2603_22437_b300 as M
    from oracle import circuits as cc
    vals = np.random.default_rng(1).normal(size=(200, 100))
    assert np.array_equal(M.pack_window(15, vals), cc.Layout(16384, 100, 200).pack(vals))


def test_no_device_is_a_status_not_a_crash():
    import torch
    import paper_2603_22437_b300 as M
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(M.MmfheError) as e:
        M.Context(M.fir_dft_params())
    assert e.value.name == "CUDA"
