"""Seeded synthetic inputs shared by the oracle tests and the CUDA path.

This module draws random numbers and builds synthetic radar windows; it holds
none of the homomorphic scheme's arithmetic.  The randomness a CKKS client
draws (ternary secret, discrete-Gaussian errors, uniform ring elements) is
produced here and passed into whichever implementation consumes it.

Radar windows follow the paper's vital-sign setup (Sec. "Processing
configuration": R range bins x F frames, 20 Hz frame rate, 10 s window;
Appendix A: a target bin whose phase follows 4 pi d(t) / lambda) with the
workload recipe:

* one target bin r* ~ U{8 .. R-9}; chest displacement
  d(t) = a_h sin(2 pi f_h t + phi_h) + a_r sin(2 pi f_r t + phi_r),
  a_h = 0.5 mm, a_r = 4 mm, carrier 77 GHz (lambda = c / 77 GHz);
* fixed-rate workload: f_h = 1.2 Hz, f_r = 0.25 Hz; randomized workload:
  f_h ~ U(0.8, 2.0) Hz, f_r ~ U(0.1, 0.5) Hz;
* target amplitude 1 with a random static phase, every bin (target included)
  gets N(0, sigma^2) noise per real component, sigma = 0.05.
"""
import numpy as np

C_LIGHT = 299_792_458.0
F_CARRIER = 77e9
LAMBDA_M = C_LIGHT / F_CARRIER

GAUSS_SIGMA = 3.19
GAUSS_TAIL = 6.0


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# randomness of the scheme's client (passed in as inputs)
# ---------------------------------------------------------------------------
def ternary(g, n):
    """Uniform ternary coefficients in {-1, 0, 1}."""
    return g.integers(-1, 2, size=n, dtype=np.int64)


def gaussian(g, n, sigma=GAUSS_SIGMA, tail=GAUSS_TAIL):
    """Rounded Gaussian integers, |x| <= tail*sigma (resampled outside)."""
    x = np.rint(g.normal(0.0, sigma, size=n))
    bound = np.floor(tail * sigma)
    bad = np.abs(x) > bound
    while bad.any():
        x[bad] = np.rint(g.normal(0.0, sigma, size=int(bad.sum())))
        bad = np.abs(x) > bound
    return x.astype(np.int64)


def uniform_residues(g, primes, n):
    """Rows of uniform residues, row i in [0, primes[i])."""
    out = np.empty((len(primes), n), dtype=np.uint64)
    for i, q in enumerate(primes):
        out[i] = g.integers(0, int(q), size=n, dtype=np.uint64)
    return out


class KeyDraws:
    """All randomness of one client key generation for a given rotation list.

    secret: ternary s; pk: (a over Q, e); rlk / gk[k]: (a [dnum][Q*P rows],
    e [dnum]) per switching key.  Draw order is fixed (s, pk, rlk, then the
    rotation keys in the order given) so every consumer sees the same values.
    """

    def __init__(self, seed, n, q_primes, p_primes, dnum, rotations):
        g = rng(seed)
        qp = list(q_primes) + list(p_primes)
        self.secret = ternary(g, n)
        self.pk_a = uniform_residues(g, q_primes, n)
        self.pk_e = gaussian(g, n)
        self.rlk_a = np.stack([uniform_residues(g, qp, n) for _ in range(dnum)])
        self.rlk_e = np.stack([gaussian(g, n) for _ in range(dnum)])
        self.gk = {}
        for k in rotations:
            a = np.stack([uniform_residues(g, qp, n) for _ in range(dnum)])
            e = np.stack([gaussian(g, n) for _ in range(dnum)])
            self.gk[k] = (a, e)


def encryption_draws(seed, n):
    """(v, e0, e1) for one public-key encryption."""
    g = rng(seed)
    return ternary(g, n), gaussian(g, n), gaussian(g, n)


def uniform_ciphertexts(seed, q_primes, n, count):
    """``count`` ciphertexts of uniform residues, layout [count][2][L+1][N].

    Under the RLWE assumption a ciphertext is indistinguishable from such a
    pair; the cloud's work is independent of the values (data-oblivious
    circuit), so this is the cloud's view of a batch of encrypted windows.
    """
    g = rng(seed)
    out = np.empty((count, 2, len(q_primes), n), dtype=np.uint64)
    for c in range(count):
        for h in range(2):
            out[c, h] = uniform_residues(g, q_primes, n)
    return out


# ---------------------------------------------------------------------------
# synthetic radar windows
# ---------------------------------------------------------------------------
class VitalWindow:
    """Complex range profiles z[t, r] (F frames x R bins) of one window."""

    def __init__(self, z, fs, target_bin, f_heart, f_resp):
        self.z = z
        self.fs = fs
        self.target_bin = target_bin
        self.f_heart = f_heart
        self.f_resp = f_resp


def vital_window(seed, frames=200, bins=64, fs=20.0, randomize_rates=False, sigma=0.05):
    g = rng(seed)
    t = np.arange(frames) / fs
    r_star = int(g.integers(8, bins - 8))
    if randomize_rates:
        f_h = float(g.uniform(0.8, 2.0))
        f_r = float(g.uniform(0.1, 0.5))
    else:
        f_h, f_r = 1.2, 0.25
    ph_h, ph_r, ph0 = g.uniform(0, 2 * np.pi, size=3)
    d = 0.5e-3 * np.sin(2 * np.pi * f_h * t + ph_h) + 4e-3 * np.sin(2 * np.pi * f_r * t + ph_r)
    z = sigma * (g.normal(size=(frames, bins)) + 1j * g.normal(size=(frames, bins)))
    z[:, r_star] += np.exp(1j * (ph0 + 4 * np.pi * d / LAMBDA_M))
    return VitalWindow(z, fs, r_star, f_h, f_r)


# ---------------------------------------------------------------------------
# Synthetic gesture windows (feature level)
# ---------------------------------------------------------------------------
GESTURE_CLASSES = 6
GESTURE_FEATURES = 120   # 4 time segments x (14 range + 16 Doppler) energy bins


def gesture_features(seed, frames=60, fs=20.0, rbins=56, dbins=32, segs=4):
    """One 3 s gesture window as range / Doppler energy features.

    1-3 point scatterers (a hand and fingers) follow a parametric radial
    trajectory of one of six classes (push, pull, push-pull, fast
    oscillation, double tap, hold), speed U(0.2, 1.5) m/s, SNR U(10, 25) dB,
    random start range and timing.  Per frame each scatterer puts its power
    into one range and one Doppler bin; exponential noise of unit mean fills
    every bin.  Features: log(1 + energy) of 4 time segments x (range bins
    pooled by 4, Doppler bins pooled by 2).  Returns (features[120], label).
    """
    g = rng(seed)
    cls = int(g.integers(GESTURE_CLASSES))
    t = np.arange(frames) / fs
    T = frames / fs
    speed = g.uniform(0.2, 1.5)
    amp = 10 ** (g.uniform(10, 25) / 20)
    ph = g.uniform(0, 2 * np.pi)
    t0 = g.uniform(0, 0.3 * T)
    tt = np.clip(t - t0, 0, None)
    if cls == 0:
        v = -speed * (tt > 0)
    elif cls == 1:
        v = speed * (tt > 0)
    elif cls == 2:
        v = speed * np.sin(2 * np.pi * tt / T + ph) * (tt > 0)
    elif cls == 3:
        v = speed * np.sin(6 * np.pi * tt / T + ph) * (tt > 0)
    elif cls == 4:
        s = np.sin(4 * np.pi * tt / T)
        v = speed * np.sign(s) * (np.abs(s) > 0.5)
    else:
        v = 0.05 * speed * g.normal(size=frames)
    r = np.clip(g.uniform(0.25, 0.6) + np.cumsum(v) / fs, 0.05, 0.95)
    rmap = g.exponential(1.0, size=(frames, rbins))
    dmap = g.exponential(1.0, size=(frames, dbins))
    for _ in range(int(g.integers(1, 4))):
        a2 = (amp * g.uniform(0.5, 1.0)) ** 2
        rb = np.clip(((r + g.uniform(-0.03, 0.03)) * rbins).astype(int), 0, rbins - 1)
        db = np.clip((v * g.uniform(0.9, 1.1) / 3.0 * (dbins / 2) + dbins / 2).astype(int), 0, dbins - 1)
        rmap[np.arange(frames), rb] += a2
        dmap[np.arange(frames), db] += a2
    seg = frames // segs
    f = []
    for k in range(segs):
        f.append(rmap[k * seg:(k + 1) * seg].sum(0).reshape(-1, 4).sum(1))
        f.append(dmap[k * seg:(k + 1) * seg].sum(0).reshape(-1, 2).sum(1))
    return np.log1p(np.concatenate(f)), cls


# ---------------------------------------------------------------------------
# Synthetic gesture windows (range-profile level: the cloud's encrypted input)
# ---------------------------------------------------------------------------
GESTURE_CARRIER_HZ = 60.5e9          # BGT60TR13C-class 60 GHz radar
GESTURE_LAMBDA_M = C_LIGHT / GESTURE_CARRIER_HZ
GESTURE_RANGE_RES_M = 0.0375         # 4 GHz chirp bandwidth
GESTURE_CHIRP_S = 0.5e-3             # chirp repetition: +-2.5 m/s unambiguous


class GestureWindow:
    """Complex range profiles z[t, a, r, c] (F frames x A antennas x R range
    bins x D chirps) of one gesture window, with its class label."""

    def __init__(self, z, label, fs):
        self.z = z
        self.label = label
        self.fs = fs


def _trajectory(g, cls, frames, fs):
    """Radial velocity v(t) (m/s) of one of the six gesture classes (push,
    pull, push-pull, fast oscillation, double tap, hold), speed U(0.2, 1.5)
    m/s, random start within the first 30 % of the window."""
    t = np.arange(frames) / fs
    T = frames / fs
    speed = g.uniform(0.2, 1.5)
    ph = g.uniform(0, 2 * np.pi)
    t0 = g.uniform(0, 0.3 * T)
    tt = np.clip(t - t0, 0, None)
    if cls == 0:
        v = -speed * (tt > 0)
    elif cls == 1:
        v = speed * (tt > 0)
    elif cls == 2:
        v = speed * np.sin(2 * np.pi * tt / T + ph) * (tt > 0)
    elif cls == 3:
        v = speed * np.sin(6 * np.pi * tt / T + ph) * (tt > 0)
    elif cls == 4:
        s = np.sin(4 * np.pi * tt / T)
        v = speed * np.sign(s) * (np.abs(s) > 0.5)
    else:
        v = 0.05 * speed * g.normal(size=frames)
    return v


def gesture_window(seed, frames=60, antennas=4, rbins=64, chirps=32, fs=20.0, sigma=1.0):
    """One 3 s gesture window at the range-FFT output (the paper's client
    input type (ii)).

    1-3 point scatterers (hand and fingers) follow the class trajectory:
    range r(t) = r_0 + integral of v, r_0 ~ U(0.25, 0.6) m, each scatterer
    offset by U(-3, 3) cm in range, its velocity scaled by U(0.9, 1.1) and
    seen at an angle theta ~ U(-30, 30) degrees.  A scatterer of amplitude a
    adds, in frame t, antenna k and chirp c, a range response split linearly
    between the two bins around r / dr with the phase
    4 pi (r + v T_c c) / lambda + pi k sin(theta).  SNR = a^2 / (2 sigma^2)
    ~ U(10, 25) dB per sample; every sample gets N(0, sigma^2) noise per real
    component; two static reflectors (clutter) sit at random bins."""
    g = rng(seed)
    cls = int(g.integers(GESTURE_CLASSES))
    v = _trajectory(g, cls, frames, fs)
    r = np.clip(g.uniform(0.25, 0.6) + np.cumsum(v) / fs, 0.05, (rbins - 2) * GESTURE_RANGE_RES_M)
    z = sigma * (g.normal(size=(frames, antennas, rbins, chirps)) + 1j * g.normal(size=(frames, antennas, rbins, chirps)))
    c = np.arange(chirps)[None, :]
    k = np.arange(antennas)[:, None]
    snr_db = g.uniform(10, 25)
    for _ in range(int(g.integers(1, 4))):
        a = np.sqrt(2 * sigma ** 2 * 10 ** (snr_db / 10)) * g.uniform(0.5, 1.0)
        rs = np.clip(r + g.uniform(-0.03, 0.03), 0.0, (rbins - 2) * GESTURE_RANGE_RES_M)
        vs = v * g.uniform(0.9, 1.1)
        th = np.deg2rad(g.uniform(-30, 30))
        pos = rs / GESTURE_RANGE_RES_M
        b0 = np.floor(pos).astype(int)
        frac = (pos - b0)[:, None, None]
        phase = (4 * np.pi * (rs[:, None, None] + vs[:, None, None] * GESTURE_CHIRP_S * c[None]) / GESTURE_LAMBDA_M
                 + np.pi * k[None] * np.sin(th))
        sig = a * np.exp(1j * phase)                         # [F, A, D]
        t = np.arange(frames)
        z[t, :, b0, :] += (1 - frac) * sig
        z[t, :, b0 + 1, :] += frac * sig
    for _ in range(2):                                       # static clutter
        z[:, :, int(g.integers(rbins)), :] += 30 * sigma * np.exp(1j * g.uniform(0, 2 * np.pi))
    return GestureWindow(z, cls, fs)


def gesture_dataset(first_seed, count):
    X = np.empty((count, GESTURE_FEATURES))
    y = np.empty(count, dtype=np.int32)
    for i in range(count):
        X[i], y[i] = gesture_features(first_seed + i)
    return X, y
