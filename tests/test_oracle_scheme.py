"""Pins of the oracle's scheme and circuit layer: encryption round trips,
rotation as a slot permutation, relinearized products, key switching,
BSGS against a plain matrix-vector product, the DSP constants against library
routines, and the circuits against the FP64 plaintext pipeline."""
import numpy as np
import pytest
import scipy.signal

import synth
from oracle import ckks as ck
from oracle import circuits as cc
from oracle import plain
from oracle import params as pm


def enc(s, z, seed=7, level=None):
    P = s["P"]
    ct = ck.encrypt(P, s["pk"], ck.encode(P, z, P.scale, P.L), *synth.encryption_draws(seed, P.n))
    return ct if level is None else ck.drop_level(P, ct, level)


def dec(s, ct):
    return ck.decrypt_decode(s["P"], s["sk"], ct)


def test_encrypt_decrypt(small_setup):
    P = small_setup["P"]
    z = np.random.default_rng(1).uniform(-1, 1, P.slots)
    assert np.abs(dec(small_setup, enc(small_setup, z)) - z).max() < 1e-6


@pytest.mark.parametrize("k", [1, 3, 5, -16])
def test_rotation_is_slot_permutation(small_setup, k):
    P = small_setup["P"]
    z = np.random.default_rng(2).uniform(-1, 1, P.slots)
    r = ck.rotate(P, enc(small_setup, z), k, small_setup["gks"])
    assert np.abs(dec(small_setup, r) - np.roll(z, -k)).max() < 1e-6


def test_hoisted_rotations(small_setup):
    P = small_setup["P"]
    z = np.random.default_rng(3).uniform(-1, 1, P.slots)
    ct = enc(small_setup, z)
    ks = [0, 1, 3, 5]
    outs = ck.rotate_hoisted(P, ct, ks, small_setup["gks"])
    for k, o in zip(ks, outs):
        assert np.abs(dec(small_setup, o) - np.roll(z, -k)).max() < 1e-6
    # a single rotation is the hoisted schedule of a one-element set
    r = ck.rotate(P, ct, 3, small_setup["gks"])
    assert np.array_equal(r.c0, outs[2].c0) and np.array_equal(r.c1, outs[2].c1)


def test_mul_relin_rescale(small_setup):
    P = small_setup["P"]
    g = np.random.default_rng(4)
    a, b = g.uniform(-1, 1, P.slots), g.uniform(-1, 1, P.slots)
    m = ck.rescale(P, ck.mul_relin(P, enc(small_setup, a, 1), enc(small_setup, b, 2), small_setup["rlk"]))
    assert m.level == P.L - 1
    assert np.abs(dec(small_setup, m) - a * b).max() < 1e-6


def test_keyswitch_decrypts_to_d_times_s2(small_setup):
    """KS(d) with the relinearization key: u0 + u1 s = d s^2 + small (mod Q)."""
    P, sk = small_setup["P"], small_setup["sk"]
    l = P.L
    g = np.random.default_rng(5)
    pr = ck.q_primes(P, l)
    d = np.stack([g.integers(0, q, P.n, dtype=np.uint64) for q in pr])
    u0, u1 = ck.key_switch(P, d, small_setup["rlk"], l)
    s = sk.rns[: l + 1]
    lhs = ck.ring_add(u0, ck.ring_mul(P, u1, s, pr), pr)
    rhs = ck.ring_mul(P, d, ck.ring_mul(P, s, s, pr), pr)
    err = ck.crt_centered(P, ck.ring_sub(lhs, rhs, pr), l)
    assert max(abs(int(x)) for x in err) < 2 ** 20


def test_mul_plain_and_add(small_setup):
    P = small_setup["P"]
    g = np.random.default_rng(6)
    a, c = g.uniform(-1, 1, P.slots), g.uniform(-1, 1, P.slots)
    ct = enc(small_setup, a)
    pt = ck.encode(P, c, P.q[P.L], P.L)
    r = ck.rescale(P, ck.add(P, ck.mul_plain(P, ct, pt), ck.mul_plain(P, ct, pt)))
    assert np.abs(dec(small_setup, r) - 2 * a * c).max() < 1e-6


def test_bsgs_equals_plain_matvec(small_setup):
    P, s = small_setup["P"], small_setup
    lay = cc.Layout(P.slots, 16, 256)     # R_c = 16, time axis of 256 positions
    g = np.random.default_rng(7)
    D = 12
    M = np.zeros((lay.f_pad, lay.f_pad))
    sup = np.zeros_like(M, dtype=bool)
    for t in range(lay.f_pad):
        for dd in range(D):
            M[t, (t + dd) % lay.f_pad] = g.uniform(-1, 1)
            sup[t, (t + dd) % lay.f_pad] = True
    x = g.uniform(-1, 1, P.slots)
    n1 = 4
    diags = cc.matrix_diagonals_all_offsets({"support": sup, "values": M}, lay)
    consts = {("x", d): ck.encode(P, cc.prerotate(v, d // n1, n1, lay.r_c), P.q[P.L], P.L) for d, v in diags.items()}
    ks = [b * lay.r_c for b in range(n1)]
    ev = cc.Evaluator(P, s["rlk"], s["gks"])
    babies = {"x": ev.hoisted(enc(s, x), ks)}
    # keys for the giant steps 4*16, 8*16 are in the fixture's rotation set
    y = ck.rescale(P, ev.bsgs(babies, consts, n1, lay.r_c, P.L))
    X = x.reshape(lay.f_pad, lay.r_c)
    assert np.abs(dec(s, y).reshape(lay.f_pad, lay.r_c) - M @ X).max() < 1e-5


def test_rotsum(small_setup):
    P, s = small_setup["P"], small_setup
    x = np.random.default_rng(8).uniform(-1, 1, P.slots)
    ev = cc.Evaluator(P, s["rlk"], s["gks"])
    y = ev.rotsum(enc(s, x), 16, 16)
    expect = sum(np.roll(x, -16 * m) for m in range(16))
    assert np.abs(dec(s, y) - expect).max() < 1e-5


def test_dft_kernel_equals_numpy_fft():
    D = 200
    v = np.random.default_rng(9).normal(size=D) + 1j * np.random.default_rng(10).normal(size=D)
    W = cc.dft_kernel(D)
    expect = np.fft.fftshift(np.fft.fft(np.hanning(D) * v))
    assert np.abs(W @ v - expect).max() < 1e-9


def test_fir_taps_equal_scipy_firwin():
    for lo, hi in ((0.1, 0.6), (0.8, 2.5)):
        h = cc.fir_bandpass(64, lo, hi, 20.0)
        assert np.abs(h - scipy.signal.firwin(64, [lo, hi], pass_zero=False, fs=20.0)).max() < 1e-12


def test_fir_toeplitz_equals_convolution():
    h = cc.fir_bandpass(64, 0.8, 2.5, 20.0)
    x = np.random.default_rng(11).normal(size=200)
    M = cc.fir_toeplitz(h, 200, 256)["values"]
    xp = np.zeros(256)
    xp[:200] = x
    assert np.abs((M @ xp)[:200] - np.convolve(h, x)[:200]).max() < 1e-12


def test_band_bins():
    assert cc.band_bins(200, 20000, (100, 600)) == [1, 2, 3, 4, 5, 6]
    assert cc.band_bins(200, 20000, (800, 2500)) == list(range(8, 26))


def test_taylor_arctan_third_order():
    y = np.linspace(-0.3, 0.3, 61)
    approx = y * 1.0 ** 2 - y ** 3 / 3
    assert np.all(np.abs(approx - np.arctan(y)) <= np.abs(y) ** 5 / 5 + 1e-15)


def test_fir_dft_circuit_decrypts_to_fp64(small_setup):
    s = small_setup
    P, circ = s["P"], s["circ"]
    consts = circ.constants()
    win = synth.vital_window(1000, frames=200, bins=64)
    s1, _ = plain.preprocess(win.z)
    lay = circ.lay
    re, im = lay.pack(s1.real), lay.pack(s1.imag)
    ev = cc.Evaluator(P, s["rlk"], s["gks"])
    out = circ.run(ev, consts, [(enc(s, re[0], 21), enc(s, im[0], 22))])
    cfg = circ.cfg
    h = cc.fir_bandpass(cfg.taps, 0.8, 2.5, 20.0)
    x = s1[:, : lay.r_c]
    xf = np.stack([np.convolve(h, x[:, r])[:200] for r in range(lay.r_c)], axis=1)
    d = cc.dft_kernel(200) @ xf
    dre = dec(s, out[0][0]).reshape(lay.f_pad, lay.r_c)[:200]
    dim = dec(s, out[0][1]).reshape(lay.f_pad, lay.r_c)[:200]
    assert out[0][0].level == P.L - 2
    assert np.abs(dre - d.real).max() < 1e-5 and np.abs(dim - d.imag).max() < 1e-5


def test_circuit_trace_is_data_oblivious(small_setup):
    """Theorem 2: the operation trace depends only on public configuration."""
    s = small_setup
    P = s["P"]
    lay = cc.Layout(P.slots, 16, 200)
    traces = []
    for seed in (1, 2):
        x = np.random.default_rng(seed).uniform(-1, 1, P.slots)
        ev = cc.Evaluator(P, s["rlk"], s["gks"], trace=True)
        ct = enc(s, x, seed)
        y = ev.rotsum(ev.rescale(ev.square_sum([ct])), 16, 8)
        ev.hoisted(y, [16, 32])
        traces.append(ev.trace)
    assert traces[0] == traces[1] and len(traces[0]) > 5
