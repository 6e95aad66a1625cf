import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300)")
    config.addinivalue_line("markers", "slow: takes more than ~30 s")


@pytest.fixture(scope="session")
def small_setup():
    """Oracle keys for the small FIR+DFT parameter set (N = 2^13)."""
    from oracle import ckks as ck, circuits as cc, params as pm
    import synth
    P = pm.fir_dft_params()
    circ = cc.FirDftCircuit(P)
    rots = sorted(set(circ.rotations()) | {1, 3, 5})
    kd = synth.KeyDraws(11, P.n, P.q, P.p, P.dnum, rots)
    sk = ck.SecretKey(P, kd.secret)
    pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
    rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
    gks = {k % P.slots: ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
    return {"P": P, "sk": sk, "pk": pk, "rlk": rlk, "gks": gks, "circ": circ, "rots": rots}
