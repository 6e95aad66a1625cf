"""Pins of the client-side normalization of stream 2 (the client's linear-time
normalization factor before encryption, Sec. "Discussion").

* Homogeneity: multiplying stream 2 by s multiplies num and den of both
  bands by exactly s^120 in the FP64 pipeline, so the rates are unchanged
  (the factor only moves a window into the scheme's precision window).
* The stored calibration constants are what ``calibrate_stream2`` computes
  on the seeds they were fitted on.
* On those seeds, the factor puts both bands inside [5e-3, 1e5] for at least
  four windows in five, against fewer than three in five unnormalized.
"""
import numpy as np
import pytest

import synth
from oracle import circuits as cc
from oracle import plain

CFG = cc.VitalConfig(bins=256, taylor_order=3)
LO, HI = 5e-3, 1e5


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


def test_calibration_constants_recompute():
    c = plain.calibrate_stream2(range(1000, 1200), CFG)
    assert np.allclose(c, plain.STREAM2_CAL_LOG10, atol=0.005)


def test_normalization_brings_most_windows_into_the_precision_window():
    inside = [0, 0]
    for seed in range(1000, 1200):
        win = synth.vital_window(seed, frames=200, bins=256, randomize_rates=True)
        _, s2 = plain.preprocess(win.z)
        for k, x in enumerate((s2, s2 * plain.stream2_scale(s2, CFG))):
            d = [bd["den"] for bd in plain.main_chain(x, CFG)["bands"]]
            inside[k] += all(LO <= v <= HI for v in d)
    assert inside[0] < 0.6 * 200
    assert inside[1] >= 0.8 * 200
