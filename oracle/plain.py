"""FP64 plaintext pipeline of the same kernel formulas (test oracle).

This is the paper's baseline (2), "identical DSP kernels executed on
unencrypted data" (Sec. "Setup", Baselines), written directly on the
[frames x bins] arrays: K1 energy (Eq. energy), K2 soft power attention
(Eq. soft power weight, gamma = 2), K4 soft I/Q (Eqs. phase mask / phase
I/Q, P_phi = 2), K5 causal FIR (Eq. fir), K7 Taylor arctan (Eq. taylor),
K3 narrowband windowed DFT, |X|^2, merge + square, weighted frequency
average.  Client preprocessing (Sec. "Pre-Cloud Client-Side Algorithms"):
clutter removal by mean subtraction over frames, then normalisation --
stream 1 by the window maximum, stream 2 frame by frame.

The gesture chain (Sec. "Example Pipelines", pipeline 2 of Table 1) on
[frames x antennas x bins x chirps] arrays: K3 windowed fftshifted Doppler
DFT per (frame, antenna, bin), K1 power, K6 notch, w = p^4, feature p w,
summed over frames.  Its client preprocessing: mean subtraction over frames,
then one window-global scale so every Doppler value has |d| <= 1.
"""
import numpy as np

from .circuits import GestureConfig, VitalConfig, band_bins, dft_kernel, fir_bandpass, hann, notch_mask


def preprocess(z):
    """Returns (stream1, stream2) complex arrays [F, R]."""
    zt = z - z.mean(axis=0, keepdims=True)
    s1 = zt / np.abs(zt).max()
    s2 = zt / np.abs(zt).max(axis=1, keepdims=True)
    return s1, s2


# Client-side normalization of stream 2 (Sec. "Discussion", end-to-end
# implementation: the client estimates a stable normalization factor in
# linear time before encryption, from a calibrated Parseval-based energy
# estimate).  Every stage of the third-order main chain is homogeneous in the
# scale s of stream 2 (I, Q grow as s^5, y and x as s^10, dphi as s^30, the
# band powers S as s^120), so num_b and den_b of both bands grow by s^120 and
# the rates num_b / den_b are unchanged: s only moves the window into the
# precision window of the scheme.  The estimate: E_b = (1/F) sum over the
# FFT bins f of band b of |FFT(zc)_f|^2, the energy of band b of the soft I/Q
# phasor zc[t] = sum_r |z_r[t]|^4 z_r[t] that K4 forms (Parseval); the band
# powers scale as E_b^12 (E_b ~ A^2 for a band amplitude A, den_b ~ A^24), so
# log10 den_b is predicted as 12 log10 E_b + c_b, and s puts the larger
# prediction at 10^T.  c_b: ``calibrate_stream2`` over seeds 1000..1199 of
# the synthetic workload (200 frames x 256 bins, rates drawn per seed);
# T: the level that keeps the most of those windows with both bands in
# [5e-3, 1e5] (below: the absolute noise of the outputs, ~5e-8, exceeds the
# 1e-3 bpm budget; above: num nears q_0 / (2 Delta)).
STREAM2_CAL_LOG10 = (-16.66, -22.65)
STREAM2_TARGET_LOG10 = 2.25


def stream2_band_energy(s2, cfg=VitalConfig()):
    """E_b of the soft I/Q phasor of stream 2 for every band (O(F R + F log F))."""
    F = s2.shape[0]
    p = s2.real ** 2 + s2.imag ** 2
    zc = (p * p * s2).sum(axis=1)
    Z = np.fft.fft(zc)
    f = np.fft.fftfreq(F, d=1000.0 / cfg.fs_mhz)
    out = []
    for lo, hi in cfg.bands_mhz:
        band = (np.abs(f) >= lo / 1000) & (np.abs(f) <= hi / 1000)
        out.append(float((np.abs(Z[band]) ** 2).sum() / F))
    return out


def stream2_scale(s2, cfg=VitalConfig(), cal=STREAM2_CAL_LOG10, target=STREAM2_TARGET_LOG10):
    """The factor the client multiplies stream 2 by before encryption (third
    order; the first-order chain is left unscaled)."""
    if cfg.taylor_order != 3:
        return 1.0
    E = stream2_band_energy(s2, cfg)
    pred = max(12 * np.log10(max(e, 1e-300)) + c for e, c in zip(E, cal))
    return float(10.0 ** ((target - pred) / 120.0))


def calibrate_stream2(seeds, cfg=VitalConfig()):
    """c_b = mean over seeded synthetic windows of log10 den_b - 12 log10 E_b
    (FP64 pipeline of this module, unnormalized stream 2)."""
    from synth import vital_window
    acc = [[], []]
    for seed in seeds:
        win = vital_window(seed, frames=cfg.frames, bins=cfg.bins, randomize_rates=True)
        _, s2 = preprocess(win.z)
        E = stream2_band_energy(s2, cfg)
        mc = main_chain(s2, cfg)
        for b in range(2):
            acc[b].append(np.log10(mc["bands"][b]["den"]) - 12 * np.log10(E[b]))
    return tuple(float(np.mean(a)) for a in acc)


def side_branch(s1):
    p = s1.real ** 2 + s1.imag ** 2
    E = p.sum(axis=0)
    w = E ** 2
    r = np.arange(len(E))
    return {"p": p, "E": E, "w": w, "num": float((r * w).sum()), "den": float(w.sum())}


def main_chain(s2, cfg=VitalConfig()):
    F = s2.shape[0]
    p = s2.real ** 2 + s2.imag ** 2
    m = p ** 2
    I = (m * s2.real).sum(axis=1)
    Q = (m * s2.imag).sum(axis=1)
    out = {"p": p, "m": m, "I": I, "Q": Q, "bands": []}
    fs = cfg.fs_mhz / 1000
    w = hann(F)
    t = np.arange(F)
    powers = {}
    for b, band in enumerate(cfg.bands_mhz):
        h = fir_bandpass(cfg.taps, band[0] / 1000, band[1] / 1000, fs)
        If = np.array([sum(h[k] * I[tt - k] for k in range(len(h)) if tt - k >= 0) for tt in range(F)])
        Qf = np.array([sum(h[k] * Q[tt - k] for k in range(len(h)) if tt - k >= 0) for tt in range(F)])
        If1 = np.concatenate([[0.0], If[:-1]])
        Qf1 = np.concatenate([[0.0], Qf[:-1]])
        y = Qf * If1 - If * Qf1
        x = If * If1 + Qf * Qf1
        dphi = y * x ** 2 - y ** 3 / 3 if cfg.taylor_order == 3 else y
        ks = band_bins(F, cfg.fs_mhz, band)
        g = cfg.gains()[b]
        X = np.array([g * (w * dphi * np.exp(-2j * np.pi * k * t / F)).sum() for k in ks])
        P = np.abs(X) ** 2
        for k, v in zip(ks, P):
            powers[k] = v
        out["bands"].append({"If": If, "Qf": Qf, "y": y, "x": x, "dphi": dphi, "bins": ks, "X": X, "P": P})
    S = {k: v ** 2 for k, v in powers.items()}
    for b, bd in enumerate(out["bands"]):
        ks = bd["bins"]
        bd["S"] = np.array([S[k] for k in ks])
        bd["num"] = float(sum(k * fs / F * S[k] for k in ks))       # Hz-weighted
        bd["den"] = float(sum(S[k] for k in ks))
        bd["bpm"] = 60.0 * bd["num"] / bd["den"]
    return out


def gesture_preprocess(z):
    """z [F, A, R, D] complex -> clutter-removed, scaled frames: divided by
    max |z~| times sum_n w[n] (the DFT's window gain) so |d| <= 1."""
    zt = z - z.mean(axis=0, keepdims=True)
    D = z.shape[-1]
    return zt / (np.abs(zt).max() * hann(D).sum())


def gesture_features(zt, cfg=GestureConfig()):
    """Accumulated weighted features [A, R, D] and the intermediates."""
    W = dft_kernel(cfg.chirps)
    d = (zt.reshape(-1, cfg.chirps) @ W.T).reshape(zt.shape)   # K3 per (frame, antenna, bin)
    p = d.real ** 2 + d.imag ** 2                  # K1
    p = p * notch_mask(cfg.chirps)                 # K6
    if cfg.feature_coef is not None:               # the learned map a p + b p^2
        a, b = cfg.feature_coef
        f = a * p + b * p * p
        return {"d": d, "p": p, "f": f, "feat": f.sum(axis=0)}
    w = (p * p) ** 2                               # soft power, gamma = 4
    f = p * w                                      # feature weighting
    return {"d": d, "p": p, "w": w, "f": f, "feat": f.sum(axis=0)}
