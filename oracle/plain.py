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
    w = (p * p) ** 2                               # soft power, gamma = 4
    f = p * w                                      # feature weighting
    return {"d": d, "p": p, "w": w, "f": f, "feat": f.sum(axis=0)}
