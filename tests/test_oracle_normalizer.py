"""Pins of the client-side normalization of stream 2 (the client's linear-time
normalization factor before encryption, Sec. "Discussion").

* Homogeneity: multiplying stream 2 by s multiplies num and den of both
  bands by exactly s^120 in the FP64 pipeline, so the rates are unchanged
  (the factor only moves a window into the scheme's precision window).
* The frequency-domain band powers the client computes equal the FP64
  pipeline's den (a direct-form FIR and direct DFT sums) to rounding.
* On 200 seeds every band lands inside [5e-3, 1e5] in the copy normalized
  for it; fewer than three windows in five are inside unnormalized, and
  fewer than one in six needs two copies.
"""
import numpy as np
import pytest

import synth
from oracle import circuits as cc
from oracle import plain

CFG = cc.VitalConfig(bins=256, taylor_order=3)
LO, HI = 5e-3, 1e5
LO_L, HI_L = plain.NORM_WINDOW_LOG10


@pytest.mark.parametrize("seed", [1000, 1017, 1101])
def test_scaling_stream2_scales_band_powers_by_s_to_the_120(seed):
    win = synth.vital_window(seed, frames=200, bins=256, randomize_rates=True)
    _, s2 = plain.preprocess(win.z)
    s = 1.07
    a, b = plain.main_chain(s2, CFG), plain.main_chain(s2 * s, CFG)
    for ba, bb in zip(a["bands"], b["bands"]):
        assert abs(np.log10(bb["den"]) - np.log10(ba["den"]) - 120 * np.log10(s)) < 1e-9
        assert abs(np.log10(bb["num"]) - np.log10(ba["num"]) - 120 * np.log10(s)) < 1e-9
        assert abs(bb["bpm"] - ba["bpm"]) < 1e-9 * ba["bpm"]


@pytest.mark.parametrize("seed", [1000, 1017, 1018, 1070, 1101, 1102, 1165, 1199])
def test_band_powers_equal_the_fp64_chain(seed):
    win = synth.vital_window(seed, frames=200, bins=256, randomize_rates=True)
    _, s2 = plain.preprocess(win.z)
    got = plain.stream2_band_powers(s2, CFG)
    want = [b["den"] for b in plain.main_chain(s2, CFG)["bands"]]
    for g, w in zip(got, want):
        assert abs(g / w - 1) < 1e-9, (g, w)


def test_every_band_lands_inside_its_copy():
    inside_raw, split = 0, 0
    for seed in range(1000, 1200):
        win = synth.vital_window(seed, frames=200, bins=256, randomize_rates=True)
        _, s2 = plain.preprocess(win.z)
        d = [bd["den"] for bd in plain.main_chain(s2, CFG)["bands"]]
        inside_raw += all(LO <= v <= HI for v in d)
        copies = plain.stream2_scales(s2, CFG)
        assert len(copies) in (1, 2)
        assert sorted(b for _, bands in copies for b in bands) == [0, 1]
        split += len(copies) == 2
        if len(copies) == 2:      # only when one factor cannot hold both bands with the margin
            assert abs(np.log10(d[0] / d[1])) > (HI_L - LO_L) - 2 * plain.NORM_MARGIN
        for s, bands in copies:
            ds = [bd["den"] for bd in plain.main_chain(s2 * s, CFG)["bands"]]
            for b in bands:
                assert LO <= ds[b] <= HI, (seed, b, ds[b])
    assert inside_raw < 0.6 * 200
    assert split < 200 / 6
