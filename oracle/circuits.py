"""Slot layout, public constants and the homomorphic circuits (test oracle).

Two circuits are restated here, step by step, on top of ``ckks``:

* ``fir_dft``: the small instance -- a 64-tap bandpass FIR (K5, Eq. for
  I_f = T I) followed by the windowed, fftshifted D-point DFT of Eq. (K3)
  (d_re = C v_re - S v_im, d_im = S v_re + C v_im), both as BSGS diagonal
  matrix-vector products, applied to every range bin of a window.
* ``vital``: the vital-sign chain of Sec. "Example Pipelines"
  (K1 -> K2 -> K4 -> K5 -> K7 -> K3 -> K1 -> K2) with the level schedule of
  Table 1 (depth 11 with the third-order Taylor arctan, 9 with first order).

Slot layout (batched packing, Sec. "Packing"): frames are packed frame-major,
slot(t, r) = t * R_c + r with F_pad = 2^ceil(log2 F) frame positions and
R_c = (N/2) / F_pad range bins per ciphertext; a window's R bins fill
G = ceil(R / R_c) ciphertexts per real/imaginary part; padding is zero.

Readings of passages the paper leaves open (each restated in the design
notes): constants are encoded at scale q_l of the level they multiply so the
rescale returns the ciphertext scale; BSGS baby steps are hoisted, giant steps
are ordinary rotations, one rescale follows each matrix product -- except the
vital chain's FIR and DFT products, which are double-hoisted (babies, inner
sums and giant-step terms in the extended basis Q*P, one ModDown at the end,
diagonals encoded over Q*P; Bossuat et al., Eurocrypt 2021, Sec. 4); products that
are summed share one relinearization (lazy relinearization); the 1/3 of the
third-order Taylor term is realised as 3 x^2 - y^2 (exact integer multiply)
with the 1/3 folded into the DFT constants; the DFT of the vital chain keeps
the band rows only (narrowband), placed at position k of frequency k fs / F,
scaled by 1/F; FIR taps are a Hamming-windowed-sinc bandpass normalised to
unit gain at the band centre.
"""
import math
from dataclasses import dataclass, field

import numpy as np

from . import ckks as ck


# ----------------------------------------------------------------------------
# configuration and slot layout (A0)
# ----------------------------------------------------------------------------
def next_pow2(x):
    return 1 << max(0, math.ceil(math.log2(x)))


@dataclass
class Layout:
    slots: int
    bins: int           # R
    frames: int         # F

    @property
    def f_pad(self):
        return next_pow2(self.frames)

    @property
    def r_c(self):
        return self.slots // self.f_pad

    @property
    def groups(self):
        return -(-self.bins // self.r_c)

    def slot(self, t, r):
        return t * self.r_c + r

    def pack(self, values):
        """values [F, R] real -> G slot vectors (frame-major, zero padded)."""
        F, R = values.shape
        assert F == self.frames and R == self.bins
        out = np.zeros((self.groups, self.slots))
        for c in range(self.groups):
            r0, r1 = c * self.r_c, min((c + 1) * self.r_c, R)
            blk = np.zeros((self.f_pad, self.r_c))
            blk[:F, : r1 - r0] = values[:, r0:r1]
            out[c] = blk.reshape(-1)
        return out


@dataclass
class FirDftConfig:
    bins: int = 64
    frames: int = 200
    fs_mhz: int = 20000
    taps: int = 64
    band_mhz: tuple = (800, 2500)


@dataclass
class VitalConfig:
    bins: int = 256
    frames: int = 200
    fs_mhz: int = 20000
    taps: int = 64
    bands_mhz: tuple = ((100, 600), (800, 2500))     # respiration, heart (Sec. "Example Pipelines")
    taylor_order: int = 3
    # complex-slot packing: each stream's Re + i Im in one ciphertext per group
    complex_slots: bool = False
    # public per-band spectral gains g_b of the narrowband DFT
    # X_b[k] = g_b * sum_t w[t] dphi[t] exp(-j 2 pi k t / F) (None = defaults)
    dft_gains: tuple = None

    def gains(self):
        """Default gains put the median DFT magnitude of the synthetic
        workload near 0.5 so that |X|^2 and its square stay inside the
        precision window of Delta = 2^40 and below q_0 / (2 Delta) at the
        last level."""
        if self.dft_gains is not None:
            return self.dft_gains
        return (30.0, 1.0) if self.taylor_order == 3 else (1.5, 0.2)


# ----------------------------------------------------------------------------
# public DSP constants (FP64)
# ----------------------------------------------------------------------------
def fir_bandpass(taps, f_lo_hz, f_hi_hz, fs_hz):
    """Hamming-windowed-sinc bandpass, unit gain at the band centre."""
    M = (taps - 1) / 2.0
    m = np.arange(taps) - M
    a, b = f_lo_hz / fs_hz, f_hi_hz / fs_hz                  # cycles / sample
    h = 2 * b * np.sinc(2 * b * m) - 2 * a * np.sinc(2 * a * m)
    h = h * (0.54 - 0.46 * np.cos(2 * np.pi * np.arange(taps) / (taps - 1)))
    fc = 0.5 * (a + b)
    return h / np.sum(h * np.cos(2 * np.pi * fc * m))


def hann(n):
    """Symmetric Hann ('Hanning') window w[k] = 0.5 - 0.5 cos(2 pi k / (n-1))."""
    return 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(n) / (n - 1))


def dft_kernel(D):
    """W[d, n] = w[n] exp(-j 2 pi sigma(d) n / D), sigma(d) = (d + D/2) mod D
    (Eq. K3)."""
    d = np.arange(D)[:, None]
    n = np.arange(D)[None, :]
    sig = (d + D // 2) % D
    return hann(D)[None, :] * np.exp(-2j * np.pi * sig * n / D)


def band_bins(frames, fs_mhz, band_mhz):
    """Frequency bins k with f_lo <= k fs / F <= f_hi (exact integer test)."""
    lo, hi = band_mhz
    return [k for k in range(frames // 2 + 1) if lo * frames <= k * fs_mhz <= hi * frames]


# ----------------------------------------------------------------------------
# BSGS diagonal matrix-vector product (A9) and rotate-and-sum (A10)
# ----------------------------------------------------------------------------
def bsgs_split(num_diag):
    """n1 = 2^ceil(log2(D)/2) baby steps, n2 = D / n1 giant steps."""
    D = next_pow2(num_diag)
    n1 = 1 << math.ceil(math.log2(D) / 2)
    return n1, D // n1


def rotate_slots(v, k):
    """Rot(v, k)[j] = v[(j + k) mod n]."""
    return np.roll(v, -k)


def matrix_diagonals(M_time, lay, row_offset=0, col_offset=0):
    """Diagonals of a time-axis matrix (rows = output positions, columns =
    input positions over F_pad) in the frame-major layout.

    Output slot(t, row_offset) receives sum_u M[t, u] x[slot(u, col_offset)],
    realised as sum_delta diag_delta (.) Rot(x, delta * R_c) with
    diag_delta[slot(t, row_offset)] = M[t, (t + delta) mod F_pad] (requires
    row_offset == col_offset since the rotation keeps the in-frame offset).
    Returns {delta: slot vector}; structurally absent diagonals are omitted.
    """
    assert row_offset == col_offset
    Fp = lay.f_pad
    out = {}
    present = np.zeros(Fp, dtype=bool)
    rows, cols = np.nonzero(M_time["support"])
    present[(cols - rows) % Fp] = True
    for delta in np.nonzero(present)[0]:
        v = np.zeros(lay.slots)
        t = np.arange(Fp)
        v[t * lay.r_c + row_offset] = M_time["values"][t, (t + delta) % Fp]
        out[int(delta)] = v
    return out


def prerotate(diag, g, n1, stride):
    """D'_{g,b} = Rot(D_delta, -g n1 stride)."""
    return rotate_slots(diag, -g * n1 * stride)


class Evaluator:
    """Evaluation context: parameters, keys and the op trace (for the
    data-obliviousness check of Theorem 2)."""

    def __init__(self, P, rlk, gks, trace=False):
        self.P, self.rlk, self.gks = P, rlk, gks
        self.trace = [] if trace else None

    def _t(self, *rec):
        if self.trace is not None:
            self.trace.append(rec)

    # thin wrappers that record the trace
    def tensor(self, a, b):
        self._t("tensor", a.level)
        return ck.tensor(self.P, a, b)

    def relin(self, t):
        self._t("relin", t.level)
        return ck.relinearize(self.P, t, self.rlk)

    def rescale(self, a):
        self._t("rescale", a.level)
        return ck.rescale(self.P, a)

    def rotate(self, a, k):
        self._t("rotate", a.level, k)
        return ck.rotate(self.P, a, k, self.gks)

    def conjugate(self, a):
        self._t("conjugate", a.level)
        return ck.conjugate(self.P, a, self.gks)

    def hoisted(self, a, ks):
        self._t("hoisted", a.level, tuple(ks))
        return ck.rotate_hoisted(self.P, a, ks, self.gks)

    def add(self, a, b):
        self._t("add", a.level)
        return ck.add(self.P, a, b)

    def add_plain(self, a, pt):
        self._t("add_plain", a.level)
        return ck.add_plain(self.P, a, pt)

    def sub(self, a, b):
        self._t("sub", a.level)
        return ck.sub(self.P, a, b)

    def mul_plain(self, a, pt):
        self._t("mul_plain", a.level)
        return ck.mul_plain(self.P, a, pt)

    def drop(self, a, level):
        return ck.drop_level(self.P, a, level)

    def tensor_add(self, x, y):
        return ck.tensor_add(self.P, x, y)

    def tensor_sub(self, x, y):
        return ck.tensor_sub(self.P, x, y)

    def tensor_mul_int(self, x, k):
        return ck.tensor_mul_int(self.P, x, k)

    def mul_plain_sum(self, pairs):
        return ck.mul_plain_sum(self.P, pairs)

    def lincomb(self, terms, scale):
        """sum_i c_i x_i for real constants c_i, each encoded at `scale`
        (constant polynomials), not rescaled."""
        self._t("lincomb", terms[0][0].level, len(terms))
        acc = None
        for x, c in terms:
            t = ck.mul_scalar(self.P, x, c, scale)
            acc = t if acc is None else ck.add(self.P, acc, t)
        return acc

    def rotsum(self, a, stride, span):
        """x <- x + Rot(x, stride 2^i), i < log2(span): slot j then holds
        sum_{m < span} x[j + m stride]."""
        for i in range(int(math.log2(span))):
            a = self.add(a, self.rotate(a, stride << i))
        return a

    def square_sum(self, xs):
        """relin(sum_i x_i (x) x_i), not rescaled (lazy relinearization)."""
        t = self.tensor(xs[0], xs[0])
        for x in xs[1:]:
            t = self.tensor_add(t, self.tensor(x, x))
        return self.relin(t)

    def bsgs(self, babies, consts, n1, stride, level):
        """Giant-step half of the BSGS product (A9).

        ``babies[name][b]`` = Rot(x_name, b stride) (b < n1, from a hoisted
        set); ``consts[(name, delta)]`` = encoded pre-rotated diagonal
        D'_{g,b} with delta = g n1 + b.  Returns
        sum_g Rot( sum_{name,b} D'_{g,b} (.) babies[name][b], g n1 stride ),
        not rescaled.  Absent diagonals / giant groups are skipped.
        """
        groups = {}
        for (name, delta) in consts:
            groups.setdefault(delta // n1, []).append((name, delta))
        acc = None
        for g in sorted(groups):
            pairs = []
            for (name, delta) in sorted(groups[g]):
                pairs.append((babies[name][delta % n1], consts[(name, delta)]))
                self._t("mul_plain", level, name, delta)
            inner = self.mul_plain_sum(pairs)
            if g:
                inner = self.rotate(inner, g * n1 * stride)
            acc = inner if acc is None else self.add(acc, inner)
        return acc


    def bsgs_dh(self, sets, consts, n1, stride):
        """The double-hoisted BSGS product (A9; Bossuat, Mouchet,
        Troncoso-Pastoriza and Hubaux, Eurocrypt 2021, Sec. 4): baby set
        `name` holds Rot(x_name, b stride + off_name) for
        ``sets[name] = (x_name, off_name)``; ``consts[(name, delta)]`` =
        pre-rotated diagonal D'_{g,b} encoded over Q*P (delta = g n1 + b).
        Babies, inner sums and giant-step terms stay in the extended basis;
        one ModDown ends the product.  Not rescaled."""
        level = next(iter(sets.values()))[0].level
        for (name, delta) in sorted(consts):
            self._t("mul_plain_qp", level, name, delta)
        self._t("bsgs_dh", level, tuple(sorted((n, o) for n, (_, o) in sets.items())), n1, stride)
        return ck.bsgs_double_hoisted_sets(self.P, sets, consts, n1, stride, self.gks)


class _Shape:
    """Level/scale stand-in for a ciphertext in a counting run."""

    def __init__(self, level, scale=1.0):
        self.level, self.scale = level, scale


def _scale_of(x):
    """Scale of a stand-in or constant; a constant left out of a counting run
    (None) counts as scale 1."""
    return 1.0 if x is None else x.scale


class CountingEvaluator(Evaluator):
    """Runs a circuit without computing it: every operation returns a
    level- and scale-tracking stand-in and key switches are tallied, each
    weighted by the number of limbs it touches (level + 1 + K).  Used to
    size a bounded sample of the oracle's work, and for the output scales
    of a circuit (the scale arithmetic of the real evaluator)."""

    def __init__(self, P):
        super().__init__(P, None, None)
        self.ks_weight = 0
        self.K = len(P.p)

    def _ks(self, level, n=1):
        self.ks_weight += n * (level + 1 + self.K)

    def tensor(self, a, b):
        return _Shape(a.level, a.scale * b.scale)

    def relin(self, t):
        self._ks(t.level)
        return _Shape(t.level, t.scale)

    def rescale(self, a):
        return _Shape(a.level - 1, a.scale / self.P.q[a.level])

    def rotate(self, a, k):
        if ck.key_id(self.P, k):
            self._ks(a.level)
        return _Shape(a.level, a.scale)

    def conjugate(self, a):
        self._ks(a.level)
        return _Shape(a.level, a.scale)

    def hoisted(self, a, ks):
        self._ks(a.level, sum(1 for k in ks if ck.key_id(self.P, k)))
        return [_Shape(a.level, a.scale) for _ in ks]

    def add(self, a, b):
        return _Shape(a.level, a.scale)

    def add_plain(self, a, pt):
        return _Shape(a.level, a.scale)

    sub = add

    def mul_plain(self, a, pt):
        return _Shape(a.level, a.scale * _scale_of(pt))

    def drop(self, a, level):
        return _Shape(level, a.scale)

    def tensor_add(self, x, y):
        return _Shape(x.level, x.scale)

    tensor_sub = tensor_add

    def tensor_mul_int(self, x, k):
        return _Shape(x.level, x.scale)

    def mul_plain_sum(self, pairs):
        return _Shape(pairs[0][0].level, pairs[0][0].scale * _scale_of(pairs[0][1]))

    def bsgs_dh(self, sets, consts, n1, stride):
        x = next(iter(sets.values()))[0]
        self._ks(x.level, dh_key_switches(self.P, sets, consts, n1, stride))
        return _Shape(x.level, x.scale * _scale_of(next(iter(consts.values()))))


def dh_key_switches(P, sets, consts, n1, stride):
    """Key switches of a double-hoisted BSGS product: one per distinct
    baby rotation and one per giant step with a nonzero rotation."""
    babies = {(name, d - (d // n1) * n1) for name, d in consts}
    n = sum(1 for name, b in babies if ck.key_id(P, b * stride + sets[name][1]))
    n += sum(1 for g in {d // n1 for _, d in consts} if ck.key_id(P, g * n1 * stride))
    return n


class SampleBudgetExceeded(Exception):
    pass


class BudgetEvaluator(Evaluator):
    """Real evaluation that tallies the same key-switch weight as
    CountingEvaluator and stops once `budget_s` seconds have elapsed."""

    def __init__(self, P, rlk, gks, budget_s):
        import time
        super().__init__(P, rlk, gks)
        self._time = time.perf_counter
        self.t0 = self._time()
        self.budget = budget_s
        self.ks_weight = 0
        self.K = len(P.p)

    def _check(self):
        if self._time() - self.t0 > self.budget:
            raise SampleBudgetExceeded()

    def relin(self, t):
        self._check()
        r = super().relin(t)
        self.ks_weight += t.level + 1 + self.K
        return r

    def rotate(self, a, k):
        self._check()
        r = super().rotate(a, k)
        if ck.key_id(self.P, k):
            self.ks_weight += a.level + 1 + self.K
        return r

    def hoisted(self, a, ks):
        self._check()
        r = super().hoisted(a, ks)
        self.ks_weight += (a.level + 1 + self.K) * sum(1 for k in ks if ck.key_id(self.P, k))
        return r

    def conjugate(self, a):
        self._check()
        r = super().conjugate(a)
        self.ks_weight += a.level + 1 + self.K
        return r

    def bsgs_dh(self, sets, consts, n1, stride):
        self._check()
        r = super().bsgs_dh(sets, consts, n1, stride)
        self.ks_weight += (r.level + 1 + self.K) * dh_key_switches(self.P, sets, consts, n1, stride)
        return r


# ----------------------------------------------------------------------------
# FIR + DFT circuit (small instance)
# ----------------------------------------------------------------------------
class FirDftCircuit:
    """Bandpass FIR along time for every range bin, then the D = F point
    windowed fftshifted DFT (Eq. K3), on G groups x (Re, Im) ciphertexts."""

    def __init__(self, P, cfg=FirDftConfig()):
        self.P, self.cfg = P, cfg
        self.lay = Layout(P.slots, cfg.bins, cfg.frames)
        self.n1_fir, self.n2_fir = bsgs_split(cfg.taps)
        self.n1_dft, self.n2_dft = bsgs_split(self.lay.f_pad)

    def fir_matrix(self):
        cfg, Fp = self.cfg, self.lay.f_pad
        h = fir_bandpass(cfg.taps, cfg.band_mhz[0] / 1000, cfg.band_mhz[1] / 1000, cfg.fs_mhz / 1000)
        return fir_toeplitz(h, cfg.frames, Fp)

    def dft_matrices(self):
        D, Fp = self.cfg.frames, self.lay.f_pad
        W = dft_kernel(D)
        sup = np.zeros((Fp, Fp), dtype=bool)
        sup[:D, :D] = True
        out = {}
        for name, vals in (("c", W.real), ("s", W.imag), ("ms", -W.imag)):
            M = np.zeros((Fp, Fp))
            M[:D, :D] = vals
            out[name] = {"support": sup, "values": M}
        return out

    def fir_diagonals(self):
        """FIR as diagonals over negative rotations: Rot(x, -k R_c), k < taps."""
        M = self.fir_matrix()
        lay, Fp = self.lay, self.lay.f_pad
        out = {}
        for k in range(self.cfg.taps):
            v = np.zeros(lay.slots)
            t = np.arange(Fp)
            for r in range(lay.r_c):
                v[t * lay.r_c + r] = M["values"][t, (t - k) % Fp] * M["support"][t, (t - k) % Fp]
            out[k] = v
        return out

    def rotations(self):
        lay = self.lay
        ks = set()
        ks |= {-b * lay.r_c for b in range(1, self.n1_fir)}
        ks |= {-g * self.n1_fir * lay.r_c for g in range(1, self.n2_fir)}
        ks |= {b * lay.r_c for b in range(1, self.n1_dft)}
        ks |= {g * self.n1_dft * lay.r_c for g in range(1, self.n2_dft)}
        return sorted({k % self.P.slots for k in ks})

    def constants(self):
        """Encoded constants keyed (name, delta) -> Plaintext."""
        P, lay = self.P, self.lay
        L = P.L
        out = {}
        n1 = self.n1_fir
        for k, v in self.fir_diagonals().items():
            out[("fir", k)] = ck.encode(P, prerotate(v, k // n1, n1, -lay.r_c), P.q[L], L)
        n1 = self.n1_dft
        for name, M in self.dft_matrices().items():
            for delta, v in matrix_diagonals_all_offsets(M, lay).items():
                out[("dft_" + name, delta)] = ck.encode(P, prerotate(v, delta // n1, n1, lay.r_c), P.q[L - 1], L - 1)
        return out

    def run(self, ev, consts, cts):
        """cts: list of G (re, im) ciphertext pairs at level L.  Returns the
        list of G (d_re, d_im) pairs at level L - 2."""
        lay = self.lay
        fir = {("x", k): consts[("fir", k)] for k in range(self.cfg.taps)}
        out = []
        for re, im in cts:
            vf = []
            for x in (re, im):
                babies = {"x": ev.hoisted(x, [-b * lay.r_c for b in range(self.n1_fir)])}
                vf.append(ev.rescale(ev.bsgs(babies, fir, self.n1_fir, -lay.r_c, x.level)))
            n1 = self.n1_dft
            babies = {
                "re": ev.hoisted(vf[0], [b * lay.r_c for b in range(n1)]),
                "im": ev.hoisted(vf[1], [b * lay.r_c for b in range(n1)]),
            }
            keys = [k for k in consts if k[0].startswith("dft_")]
            c_re = {("re", d): consts[(n, d)] for (n, d) in keys if n == "dft_c"}
            c_re.update({("im", d): consts[(n, d)] for (n, d) in keys if n == "dft_ms"})
            c_im = {("re", d): consts[(n, d)] for (n, d) in keys if n == "dft_s"}
            c_im.update({("im", d): consts[(n, d)] for (n, d) in keys if n == "dft_c"})
            lvl = vf[0].level
            d_re = ev.rescale(ev.bsgs(babies, c_re, n1, lay.r_c, lvl))
            d_im = ev.rescale(ev.bsgs(babies, c_im, n1, lay.r_c, lvl))
            out.append((d_re, d_im))
        return out


def fir_toeplitz(h, frames, f_pad):
    """Causal FIR with zero initial state as a time-axis matrix:
    y[t] = sum_k h[k] x[t - k], t < F, t - k >= 0."""
    M = np.zeros((f_pad, f_pad))
    sup = np.zeros((f_pad, f_pad), dtype=bool)
    for t in range(frames):
        for k in range(len(h)):
            if t - k >= 0:
                M[t, t - k] = h[k]
                sup[t, t - k] = True
    return {"support": sup, "values": M}


def matrix_diagonals_all_offsets(M_time, lay):
    """Like matrix_diagonals but the same time-axis matrix acts on every
    in-frame offset r (every range bin of the group)."""
    Fp = lay.f_pad
    present = np.zeros(Fp, dtype=bool)
    rows, cols = np.nonzero(M_time["support"])
    present[(cols - rows) % Fp] = True
    out = {}
    t = np.arange(Fp)
    for delta in np.nonzero(present)[0]:
        blk = np.repeat(M_time["values"][t, (t + delta) % Fp][:, None], lay.r_c, axis=1)
        out[int(delta)] = blk.reshape(-1)
    return out


# ----------------------------------------------------------------------------
# vital-sign chain (A11)
# ----------------------------------------------------------------------------
class VitalCircuit:
    """K1 -> K2 side branch (target bin num/den) and the HR/RR main chain
    K4 -> K5 -> K7 -> K3 -> |X|^2 -> merge + square -> weighted frequency
    average, on a window of 2 streams x G groups x (Re, Im) ciphertexts.

    Level schedule (Table 1), L0 = top level:
      side: K1 p (L0-1); each group's frame sums halved log2 G' times,
            the first block masked (L0-2), the groups packed into one
            ciphertext, rotate-sum over a block; K2 w = E^2 (L0-3); index /
            one vectors (L0-4), rotate-sum over bins, then over blocks ->
            num_r, den_r (``side_branch``).
      main: K4 p (L0-1), m = p^2 (L0-2), I, Q = sum m Re, m Im (L0-3),
            rotate-sum over bins (the sums sit in bin slot 0 of every
            frame); K5 FIR of both bands in one BSGS product per part
            (L0-4): band b's output lands in bin slot b of every frame (the
            HR taps read baby steps shifted by one slot); K7 y, x (L0-5),
            third order: u = 3x^2 - y^2 (L0-6), dphi3 = y u (L0-7), both
            bands at once slot by slot; K3 narrowband DFT (+1): real rows
            at position k, imaginary rows at k + F_pad/2, band b in slot b;
            |X|^2 (+2), the imaginary half added onto the real by one
            rotation; square (+3); x f_k and x 1 (+4) per band, den's
            products moved span_b frames on, one rotate-sum per band.
    Outputs: [side branch, band RR, band HR]; ``readout`` gives where
    num_r, den_r, num_RR, den_RR, num_HR, den_HR sit.
    """

    def __init__(self, P, cfg=VitalConfig()):
        self.P, self.cfg = P, cfg
        self.lay = Layout(P.slots, cfg.bins, cfg.frames)
        self.n1_fir, self.n2_fir = bsgs_split(cfg.taps)
        self.n1_dft, self.n2_dft = bsgs_split(self.lay.f_pad)
        self.bands = [band_bins(cfg.frames, cfg.fs_mhz, b) for b in cfg.bands_mhz]
        L0 = P.L
        self.lv_side_mask = L0 - 1
        self.lv_side_const = L0 - 3
        self.lv_fir = L0 - 3
        self.lv_dphi = L0 - 7 if cfg.taylor_order == 3 else L0 - 5
        self.lv_final_const = self.lv_dphi - 3
        assert self.lv_final_const >= 1, "not enough levels for the chain"
        self.record = None   # a dict: run() records each kernel's output ciphertexts in it

    def _record(self, name, value):
        if self.record is not None:
            self.record[name] = value

    # -- public constants ----------------------------------------------------
    def taps(self, b):
        lo, hi = self.cfg.bands_mhz[b]
        return fir_bandpass(self.cfg.taps, lo / 1000, hi / 1000, self.cfg.fs_mhz / 1000)

    def dft_gain(self, b):
        """g_b over the factor the chain's phase signal carries: 3 dphi for
        the third-order chain; with complex slots 2i Im(w^3) = 6i dphi (third
        order) or 2i Im(w) = 2i dphi (first order), whose square is negated
        by the i (and squared away by the sharpening)."""
        if self.cfg.complex_slots:
            return self.cfg.gains()[b] / (6.0 if self.cfg.taylor_order == 3 else 2.0)
        return self.cfg.gains()[b] * (1.0 / 3.0 if self.cfg.taylor_order == 3 else 1.0)

    def dft_time_matrix(self, b):
        """Band b's narrowband DFT rows over the frames: Re X_k in row k,
        Im X_k in row k + F_pad/2 (X_k = g_b sum_t w[t] dphi[t] e^{-j 2 pi k t / F});
        applied in bin slot b."""
        F, Fp = self.cfg.frames, self.lay.f_pad
        H = Fp // 2
        assert max(self.bands[b]) < H, "band beyond half the padded window"
        w = hann(F)
        t = np.arange(F)
        M = np.zeros((Fp, Fp))
        sup = np.zeros((Fp, Fp), dtype=bool)
        for k in self.bands[b]:
            ang = 2 * np.pi * k * t / F
            M[k, :F] = self.dft_gain(b) * w * np.cos(ang)
            M[k + H, :F] = -self.dft_gain(b) * w * np.sin(ang)
            sup[k, :F] = sup[k + H, :F] = True
        return {"support": sup, "values": M}

    def span(self, b):
        return next_pow2(max(self.bands[b]) + 1)

    def span_all(self):
        return max(self.span(b) for b in range(len(self.bands)))

    def fir_diagonals(self, b):
        """Band b's causal FIR as diagonals over the frames, in bin slot b
        (its input baby steps are shifted by b slots)."""
        lay, F = self.lay, self.cfg.frames
        h = self.taps(b)
        out = {}
        for k in range(self.cfg.taps):
            v = np.zeros(lay.slots)
            for t in range(k, F):
                v[lay.slot(t, b)] = h[k]
            out[k] = v
        return out

    def rotations(self):
        lay, cfg = self.lay, self.cfg
        ks = set()
        ks |= {lay.r_c << i for i in range(int(math.log2(lay.f_pad)))}
        ks |= {1 << i for i in range(int(math.log2(lay.r_c)))}
        ks |= {-b * lay.r_c - s for b in range(self.n1_fir) for s in (0, 1)}
        ks |= {-g * self.n1_fir * lay.r_c for g in range(1, self.n2_fir)}
        ks.add(-lay.r_c)
        for b in range(len(self.bands)):
            for delta in matrix_diagonals(self.dft_time_matrix(b), lay):
                if delta % self.n1_dft:
                    ks.add((delta % self.n1_dft) * lay.r_c)
                if delta // self.n1_dft:
                    ks.add((delta // self.n1_dft) * self.n1_dft * lay.r_c)
        ks |= {lay.r_c << i for i in range(int(math.log2(self.span_all())))}
        ks |= {-self.span(b) * lay.r_c for b in range(len(self.bands))}     # den beside num in a band's sums
        ks.add((lay.f_pad // 2) * lay.r_c)
        ks.add(1)
        out = sorted({k % self.P.slots for k in ks} - {0})
        return ([ck.ROT_CONJ] if self.cfg.complex_slots else []) + out

    def side_groups(self):
        """G rounded up to a power of two: the number of frame blocks."""
        return next_pow2(self.lay.groups)

    def side_block(self):
        """Frames per block of the packed side branch: F_pad / G'."""
        return self.lay.f_pad // self.side_groups()

    def side_block_of(self, c):
        """Block that group c lands in: packing adds group c + 2^j, rotated
        by 2^j blocks, onto group c at tree level j, so c moves by -c."""
        return (-c) % self.side_groups()

    def side_branch(self, ev, consts, ps):
        """K1 -> K2 on the G groups' energies p_c (frame-major, stride r_c):
        E_c[r] = sum_t p_c[t, r], w = E^2, num_r = sum gbin w, den_r = sum w.

        Each group's frame sum is halved log2 G' times (G' = G rounded up to
        a power of two), which leaves the sums over F_pad / G' frame blocks
        periodic in the block; the mask keeps block 0; the groups are packed
        into one ciphertext by a rotation tree (group c lands in block -c mod
        G'); one rotate-and-sum over a block finishes every group's E at its
        block start.  w = E^2 is squared once, the index / one vectors keep
        the valid bins, den's products move one frame on, and a rotate-and-
        sum over the bins and then over the blocks leaves num_r in slot 0 and
        den_r in slot r_c of one ciphertext."""
        lay = self.lay
        Gp, blk = self.side_groups(), self.side_block()
        self._record("K1_energy", ps)
        parts = []
        for p in ps:
            x = ev.rotsum(p, blk * lay.r_c, Gp)      # sum over the frames t + j F_pad / G'
            parts.append(ev.rescale(ev.mul_plain(x, consts[("pmask",)])))
        parts += [None] * (Gp - len(parts))
        j = 0
        while len(parts) > 1:
            nxt = []
            for a in range(0, len(parts), 2):
                x, y = parts[a], parts[a + 1]
                if y is not None:
                    y = ev.rotate(y, (blk << j) * lay.r_c)
                    x = y if x is None else ev.add(x, y)
                nxt.append(x)
            parts, j = nxt, j + 1
        E = ev.rotsum(parts[0], lay.r_c, blk)
        w = ev.rescale(ev.square_sum([E]))
        self._record("K1_integration", E)
        self._record("K2_soft_attention", w)
        # num and den share one ciphertext: den's terms moved one frame on
        # (block starts + 1 frame, never reached by the other's sums)
        tn = ev.rescale(ev.mul_plain(w, consts[("idx",)]))
        td = ev.rescale(ev.mul_plain(w, consts[("one",)]))
        t = ev.add(tn, ev.rotate(td, -lay.r_c))
        t = ev.rotsum(t, 1, lay.r_c)
        return ev.rotsum(t, blk * lay.r_c, Gp)

    def constant_keys(self):
        """Keys of every constant ``constants()`` encodes, without encoding."""
        keys = [("pmask",), ("idx",), ("one",)]
        for b in range(len(self.bands)):
            keys += [("fir", b, k) for k in range(self.cfg.taps)]
        present = set()
        for b in range(len(self.bands)):
            rows, cols = np.nonzero(self.dft_time_matrix(b)["support"])
            present |= set(((cols - rows) % self.lay.f_pad).tolist())
        keys += [("dft", int(d)) for d in sorted(present)]
        keys += [(t, b) for b in range(len(self.bands)) for t in ("fw", "fone")]
        return keys

    def constants(self):
        P, lay, cfg = self.P, self.lay, self.cfg
        out = {}
        # side branch: the mask of a group's first frame block, and the
        # target-bin index / one vectors at the packed block starts
        lv = self.lv_side_mask
        blk = self.side_block()
        mask = np.zeros(lay.slots)
        for t in range(blk):
            for r in range(lay.r_c):
                mask[lay.slot(t, r)] = 1.0
        out[("pmask",)] = ck.encode(P, mask, P.q[lv], lv)
        lv = self.lv_side_const
        idx, one = np.zeros(lay.slots), np.zeros(lay.slots)
        for c in range(lay.groups):
            t0 = self.side_block_of(c) * blk
            for r in range(lay.r_c):
                gbin = c * lay.r_c + r
                if gbin < cfg.bins:
                    idx[lay.slot(t0, r)] = gbin
                    one[lay.slot(t0, r)] = 1.0
        out[("idx",)] = ck.encode(P, idx, P.q[lv], lv)
        out[("one",)] = ck.encode(P, one, P.q[lv], lv)
        # the FIR and DFT diagonals multiply double-hoisted baby steps, which
        # live in the extended basis: encoded over Q_l * P
        lv = self.lv_fir
        for b in range(len(self.bands)):
            for k, v in self.fir_diagonals(b).items():
                v = prerotate(v, k // self.n1_fir, self.n1_fir, -lay.r_c)
                out[("fir", b, k)] = ck.encode_qp(P, v, P.q[lv], lv)
        lv = self.lv_dphi
        diags = {}
        for b in range(len(self.bands)):
            for delta, v in matrix_diagonals(self.dft_time_matrix(b), lay).items():
                # band b's rows act on bin slot b
                diags[delta] = diags.get(delta, 0.0) + np.roll(v, b)
        for delta, v in diags.items():
            v = prerotate(v, delta // self.n1_dft, self.n1_dft, lay.r_c)
            out[("dft", delta)] = ck.encode_qp(P, v, P.q[lv], lv)
        # one weight pair per band: each band's sums leave in ciphertexts of
        # their own, so a band far above the other cannot overflow the other's
        # sums at the last level
        lv = self.lv_final_const
        fs_hz = cfg.fs_mhz / 1000
        for b, ks in enumerate(self.bands):
            fw, fo = np.zeros(lay.slots), np.zeros(lay.slots)
            for k in ks:
                fw[lay.slot(k, b)] = k * fs_hz / cfg.frames          # Hz; the client multiplies by 60
                fo[lay.slot(k, b)] = 1.0
            out[("fw", b)] = ck.encode(P, fw, P.q[lv], lv)
            out[("fone", b)] = ck.encode(P, fo, P.q[lv], lv)
        return out

    def band_sums(self, ev, consts, S):
        """Weighted frequency average of both bands from the sharpened powers
        S (band b in bin slot b): num_b = sum_k (k fs / F) S_k and den_b =
        sum_k S_k over band b's bins, each band by its own masks in a
        ciphertext of its own: den's products moved span_b frames on, one
        rotate-and-sum over band b's span leaves num_b in slot b and den_b in
        slot span_b r_c + b.  Returns [band RR, band HR]."""
        out = []
        for b in range(len(self.bands)):
            tn = ev.rescale(ev.mul_plain(S, consts[("fw", b)]))
            td = ev.rescale(ev.mul_plain(S, consts[("fone", b)]))
            t = ev.add(tn, ev.rotate(td, -self.span(b) * self.lay.r_c))
            out.append(ev.rotsum(t, self.lay.r_c, self.span(b)))
        return out

    def readout(self):
        """(output, slot) of num_r, den_r, num_RR, den_RR, num_HR, den_HR."""
        rc = self.lay.r_c
        return [(0, 0), (0, rc), (1, 0), (1, self.span(0) * rc), (2, 1), (2, self.span(1) * rc + 1)]

    # -- the chain -----------------------------------------------------------
    def run(self, ev, consts, s1, s2):
        """s1, s2: lists of G (re, im) ciphertext pairs (stream 1 feeds K1,
        stream 2 feeds K4), all at the top level; with complex slots lists
        of G ciphertexts of Re + i Im.  Returns three ciphertexts (``readout``)."""
        P, lay, cfg = self.P, self.lay, self.cfg
        G = lay.groups
        if cfg.complex_slots:
            return self._run_complex(ev, consts, s1, s2)
        # side branch: K1 energy, K2 soft power attention (gamma = 2)
        side = self.side_branch(ev, consts, [ev.rescale(ev.square_sum([re, im])) for re, im in s1])

        # K4 soft I/Q extraction (P_phi = 2)
        m = []
        for re, im in s2:
            p = ev.rescale(ev.square_sum([re, im]))
            m.append(ev.rescale(ev.square_sum([p])))
        lv = m[0].level
        iq = []
        for part in (0, 1):
            t = None
            for c in range(G):
                x = ev.drop(s2[c][part], lv)
                tc = ev.tensor(m[c], x)
                t = tc if t is None else ev.tensor_add(t, tc)
            iq.append(ev.rotsum(ev.rescale(ev.relin(t)), 1, lay.r_c))
        I, Q = iq
        self._record("K4_phase_extraction", (I, Q))

        # K5 FIR of both bands in one double-hoisted BSGS product per part:
        # the baby steps of I (and Q) share one ModUp, unshifted for RR
        # (output in bin slot 0) and shifted by one slot for HR (slot 1)
        n1 = self.n1_fir
        fir = {}
        for b in range(len(self.bands)):
            for k in range(cfg.taps):
                fir[("s%d" % b, k)] = consts[("fir", b, k)]
        filtered = []
        for x in (I, Q):
            sets = {"s0": (x, 0), "s1": (x, -1)}
            filtered.append(ev.rescale(ev.bsgs_dh(sets, fir, n1, -lay.r_c)))
        If, Qf = filtered
        self._record("K5_fir", (If, Qf))
        # K7 differential phase, both bands slot by slot
        If1 = ev.rotate(If, -lay.r_c)
        Qf1 = ev.rotate(Qf, -lay.r_c)
        y = ev.rescale(ev.relin(ev.tensor_sub(ev.tensor(Qf, If1), ev.tensor(If, Qf1))))
        x = ev.rescale(ev.relin(ev.tensor_add(ev.tensor(If, If1), ev.tensor(Qf, Qf1))))
        if cfg.taylor_order == 3:
            u = ev.tensor_sub(ev.tensor_mul_int(ev.tensor(x, x), 3), ev.tensor(y, y))
            u = ev.rescale(ev.relin(u))
            yd = ev.drop(y, u.level)
            dphi = ev.rescale(ev.relin(ev.tensor(yd, u)))
        else:
            dphi = y
        self._record("K7_taylor_arctan", dphi)

        # K3 narrowband DFT (both bands, each in its bin slot), |X|^2
        n1 = self.n1_dft
        cl = {("x", key[1]): pt for key, pt in consts.items() if key[0] == "dft"}
        X = ev.rescale(ev.bsgs_dh({"x": (dphi, 0)}, cl, n1, lay.r_c))
        pw = ev.rescale(ev.square_sum([X]))
        # Re^2 at k, Im^2 at k + F_pad/2: one rotation adds them
        Mg = ev.add(pw, ev.rotate(pw, (lay.f_pad // 2) * lay.r_c))
        self._record("K3_dft", X)
        self._record("power", Mg)

        # sharpen (gamma = 2), weighted frequency average (RR in slot 0, HR in slot 1)
        S = ev.rescale(ev.square_sum([Mg]))
        self._record("sharpen", S)
        return [side] + self.band_sums(ev, consts, S)

    def _run_complex(self, ev, consts, s1, s2):
        """The same chain on complex slots z = Re + i Im: |z|^2 = z conj(z);
        K4 gives Z = I + i Q in one ciphertext; the FIR is real-linear, so one
        product per band filters both parts; K7 forms w = Z conj(Z') = x + i y,
        third order Im(w^3) = 3 x^2 y - y^3 = 3 dphi, taken as
        w^3 - conj(w^3) = 2i Im(w^3) (the DFT gains absorb 2i, reading in
        dft_gain); first order w - conj(w) = 2i y."""
        lay, cfg = self.lay, self.cfg
        G = lay.groups

        def abs2(z):
            return ev.rescale(ev.relin(ev.tensor(z, ev.conjugate(z))))

        side = self.side_branch(ev, consts, [abs2(z) for z in s1])

        # K4: Z = sum_r m z (I + i Q), P_phi = 2
        m = [ev.rescale(ev.square_sum([abs2(z)])) for z in s2]
        lv = m[0].level
        t = None
        for c in range(G):
            tc = ev.tensor(m[c], ev.drop(s2[c], lv))
            t = tc if t is None else ev.tensor_add(t, tc)
        Z = ev.rotsum(ev.rescale(ev.relin(t)), 1, lay.r_c)

        # K5: both bands in one product (RR in bin slot 0, HR in slot 1)
        n1 = self.n1_fir
        fir = {}
        for b in range(len(self.bands)):
            for k in range(cfg.taps):
                fir[("s%d" % b, k)] = consts[("fir", b, k)]
        Zf = ev.rescale(ev.bsgs_dh({"s0": (Z, 0), "s1": (Z, -1)}, fir, n1, -lay.r_c))

        # K7: w = Zf conj(Zf at t-1) = x + i y
        wc = ev.rescale(ev.relin(ev.tensor(Zf, ev.conjugate(ev.rotate(Zf, -lay.r_c)))))
        if cfg.taylor_order == 3:
            w2 = ev.rescale(ev.square_sum([wc]))
            w3 = ev.rescale(ev.relin(ev.tensor(ev.drop(wc, w2.level), w2)))
            dphi = ev.sub(w3, ev.conjugate(w3))
        else:
            dphi = ev.sub(wc, ev.conjugate(wc))

        # K3, |X|^2 (negated by the i), sharpen, weighted frequency average
        n1 = self.n1_dft
        cl = {("x", key[1]): pt for key, pt in consts.items() if key[0] == "dft"}
        X = ev.rescale(ev.bsgs_dh({"x": (dphi, 0)}, cl, n1, lay.r_c))
        pw = ev.rescale(ev.square_sum([X]))
        Mg = ev.add(pw, ev.rotate(pw, (lay.f_pad // 2) * lay.r_c))
        S = ev.rescale(ev.square_sum([Mg]))
        return [side] + self.band_sums(ev, consts, S)


# ---------------------------------------------------------------------------
# Polynomial network: the paper's FC network with square activations
# (Sec. "Cloud-Side Algorithms", fully connected layers with a square
# activation; the weights are learned).  Every layer is a dense map on a slot
# period of D = width slots; slot D - 1 of every period holds the constant 1,
# so the biases are the last column of each D x D matrix and row D - 1 keeps
# the constant (W[D-1][D-1] = 1).  A square follows every layer but the last.
# ---------------------------------------------------------------------------
@dataclass
class FcConfig:
    dims: tuple = (120, 32, 16, 6)   # d_0 (inputs), d_1, ..., d_L (outputs)
    width: int = 128                 # D, a power of two above every d_l


class FcCircuit:
    def __init__(self, P, cfg=FcConfig()):
        D = cfg.width
        assert D & (D - 1) == 0 and max(cfg.dims) < D <= P.slots
        self.P, self.cfg, self.D = P, cfg, D
        self.layers = len(cfg.dims) - 1
        self.n1, self.n2 = bsgs_split(D)
        # input level of layer l: a dense layer and a square take one level each
        self.levels = [P.L - 2 * l for l in range(self.layers)]
        assert self.levels[-1] >= 1, "not enough levels for the network"

    def present(self, l):
        """Structurally non-zero diagonals of layer l: rows d_{l+1} and the
        constant row, columns d_l and the constant column."""
        D = self.D
        rows = list(range(self.cfg.dims[l + 1])) + [D - 1]
        cols = list(range(self.cfg.dims[l])) + [D - 1]
        return sorted({(j - i) % D for i in rows for j in cols})

    def diagonal(self, W, k):
        """diag_k[j] = W[j mod D][(j mod D + k) mod D] over all slots."""
        D = self.D
        i = np.arange(self.P.slots) % D
        return np.asarray(W, dtype=np.float64)[i, (i + k) % D]

    def constants(self, mats):
        P, out = self.P, {}
        for l in range(self.layers):
            lv = self.levels[l]
            for k in self.present(l):
                v = prerotate(self.diagonal(mats[l], k), k // self.n1, self.n1, 1)
                out[("fcw", l, k)] = ck.encode(P, v, P.q[lv], lv)
        return out

    def rotations(self):
        ks = set(range(1, self.n1)) | {g * self.n1 for g in range(1, self.n2)}
        return sorted(ks)

    def run(self, ev, consts, x):
        for l in range(self.layers):
            babies = {"x": ev.hoisted(x, list(range(self.n1)))}
            cl = {("x", k): consts[("fcw", l, k)] for k in self.present(l)}
            y = ev.rescale(ev.bsgs(babies, cl, self.n1, 1, x.level))
            if l < self.layers - 1:
                y = ev.rescale(ev.square_sum([y]))
            x = y
        return x


def fc_pack(x, D, slots):
    """Input slot vector: features in slots 0..d_0-1, the constant 1 in slot
    D - 1, repeated with period D."""
    v = np.zeros(D)
    v[: len(x)] = x
    v[D - 1] = 1.0
    return np.tile(v, slots // D)


def fc_forward(mats, x, D):
    """FP64 forward pass of the same network on one period."""
    v = np.zeros(D)
    v[: len(x)] = x
    v[D - 1] = 1.0
    for l, W in enumerate(mats):
        v = np.asarray(W, dtype=np.float64) @ v
        if l < len(mats) - 1:
            v = v * v
    return v


# ---------------------------------------------------------------------------
# Per-frame packing (the paper's slow baseline, Sec. "Packing"): one
# ciphertext per frame and stream part, range bin r in slot r.  Sums over bins
# become rotate-and-sums (the result lands in slot 0); everything across
# frames -- the FIR, the t-1 pairs of K7, the DFT -- is ciphertext-level
# arithmetic with scalar constants.  Same formulas and level schedule as
# VitalCircuit, so the decrypted outputs agree with the FP64 pipeline alike.
# ---------------------------------------------------------------------------
class PerFrameVitalCircuit:
    def __init__(self, P, cfg=VitalConfig()):
        assert cfg.taylor_order == 3 and cfg.bins <= P.slots
        self.P, self.cfg = P, cfg
        self.base = VitalCircuit.__new__(VitalCircuit)   # shares the public DSP design
        self.base.P, self.base.cfg = P, cfg
        self.bands = [band_bins(cfg.frames, cfg.fs_mhz, b) for b in cfg.bands_mhz]
        self.span = next_pow2(cfg.bins)
        assert P.L - 11 >= 0, "not enough levels for the chain"

    def constants(self):
        """Slot vectors of the side branch (bin index, ones) at level L0 - 2."""
        P, R = self.P, self.cfg.bins
        lv = P.L - 2
        idx, one = np.zeros(P.slots), np.zeros(P.slots)
        idx[:R] = np.arange(R)
        one[:R] = 1.0
        return {"idx": ck.encode(P, idx, P.q[lv], lv), "one": ck.encode(P, one, P.q[lv], lv)}

    def rotations(self):
        return sorted({1 << i for i in range(int(math.log2(self.span)))})

    def scalars(self):
        """The public scalar constants, in the order the library's plan keeps
        them: per band the FIR taps h[0..taps); per band, per bin k, the DFT
        coefficients g w[t] cos(2 pi k t / F) for t = 1..F-1, then
        -g w[t] sin(2 pi k t / F) (g includes the 1/3); per band, per bin k,
        the frequency k fs / F in Hz."""
        cfg, F = self.cfg, self.cfg.frames
        out = []
        for b in range(len(self.bands)):
            out.extend(self.base.taps(b))
        wn, t = hann(F), np.arange(1, F)
        for b, ks in enumerate(self.bands):
            g = self.base.dft_gain(b)
            for k in ks:
                ang = 2 * np.pi * k * t / F
                out.extend(g * wn[t] * np.cos(ang))
                out.extend(-g * wn[t] * np.sin(ang))
        for ks in self.bands:
            out.extend(k * (cfg.fs_mhz / 1000) / F for k in ks)
        return np.array(out, dtype=np.float64)

    def run(self, ev, consts, s1, s2, scalars=None):
        """s1, s2: lists of F (re, im) ciphertext pairs (one pair per frame),
        top level.  Returns [num_r, den_r, num_RR, den_RR, num_HR, den_HR]
        with the values in slot 0."""
        P, cfg = self.P, self.cfg
        F = cfg.frames
        q = P.q
        sc = iter(self.scalars() if scalars is None else scalars)
        taps = [[next(sc) for _ in range(cfg.taps)] for _ in self.bands]
        dft = [{k: ([next(sc) for _ in range(1, F)], [next(sc) for _ in range(1, F)]) for k in ks} for ks in self.bands]
        fhz = [[next(sc) for _ in ks] for ks in self.bands]
        # side branch: K1 energy, summed over frames; K2 w = E^2
        E = None
        for re, im in s1:
            p = ev.rescale(ev.square_sum([re, im]))
            E = p if E is None else ev.add(E, p)
        w = ev.rescale(ev.square_sum([E]))
        num_r = ev.rotsum(ev.rescale(ev.mul_plain(w, consts["idx"])), 1, self.span)
        den_r = ev.rotsum(ev.rescale(ev.mul_plain(w, consts["one"])), 1, self.span)
        # K4 soft I/Q: per frame p, m = p^2, I = sum_r m Re, Q = sum_r m Im
        I, Q = [], []
        for re, im in s2:
            p = ev.rescale(ev.square_sum([re, im]))
            m = ev.rescale(ev.square_sum([p]))
            for part, out in ((re, I), (im, Q)):
                x = ev.drop(part, m.level)
                out.append(ev.rotsum(ev.rescale(ev.relin(ev.tensor(m, x))), 1, self.span))
        outs = [num_r, den_r]
        S = {}
        for b, ks in enumerate(self.bands):
            # K5 causal FIR over frames
            h = taps[b]
            lv = I[0].level
            If = [ev.rescale(ev.lincomb([(I[t - k], h[k]) for k in range(cfg.taps) if t - k >= 0], q[lv]))
                  for t in range(F)]
            Qf = [ev.rescale(ev.lincomb([(Q[t - k], h[k]) for k in range(cfg.taps) if t - k >= 0], q[lv]))
                  for t in range(F)]
            # K7 third order, frames t >= 1 (dphi[0] = 0)
            dphi = [None]
            for t in range(1, F):
                y = ev.rescale(ev.relin(ev.tensor_sub(ev.tensor(Qf[t], If[t - 1]), ev.tensor(If[t], Qf[t - 1]))))
                x = ev.rescale(ev.relin(ev.tensor_add(ev.tensor(If[t], If[t - 1]), ev.tensor(Qf[t], Qf[t - 1]))))
                u = ev.rescale(ev.relin(ev.tensor_sub(ev.tensor_mul_int(ev.tensor(x, x), 3), ev.tensor(y, y))))
                dphi.append(ev.rescale(ev.relin(ev.tensor(ev.drop(y, u.level), u))))
            # K3 narrowband DFT (gain carries the 1/3), |X|^2
            lv = dphi[1].level
            for k in ks:
                cre, cim = dft[b][k]
                re_k = ev.rescale(ev.lincomb([(dphi[t], cre[t - 1]) for t in range(1, F)], q[lv]))
                im_k = ev.rescale(ev.lincomb([(dphi[t], cim[t - 1]) for t in range(1, F)], q[lv]))
                Pk = ev.rescale(ev.square_sum([re_k, im_k]))
                S[k] = ev.rescale(ev.square_sum([Pk]))    # merge + sharpen: bands are disjoint in k
        for b, ks in enumerate(self.bands):
            lv = S[ks[0]].level
            outs.append(ev.rescale(ev.lincomb([(S[k], f) for k, f in zip(ks, fhz[b])], q[lv])))
            outs.append(ev.rescale(ev.lincomb([(S[k], 1.0) for k in ks], q[lv])))
        return outs



# ---------------------------------------------------------------------------
# Gesture chain (Sec. "Example Pipelines", Encrypted Dynamic Radar
# Classification; depth accounting of Table 1, pipeline 2): per frame K3
# Doppler DFT -> K1 power map -> K6 notch -> K2 soft power (gamma = 4) ->
# feature weighting p x w; frame accumulation; FC1^2 -> FC2^2 -> FC3.
#
# Slot layout (Sec. "Packing"): within a frame, antenna a, range bin r and
# chirp c sit in slot a R D + r D + c; the A R D slots are padded to
# ARD_pad = 2^ceil(log2(A R D)) and k = (N/2) / ARD_pad frames share one
# ciphertext pair (frame f in pair f // k at offset (f mod k) ARD_pad).
#
# Readings (restated in the design notes): the notch of Eq. (notch mask)
# zeroes d in the closed range [floor(D/2), ceil(D/2)] (the half-open range
# printed is empty for even D; the closed one is the zero-Doppler bin D/2
# after the fftshift); the weighted feature is p (.) w with p the notched
# power map and w = p^4 (both ciphertexts); FC1 reads every feature slot
# (hybrid diagonal method: width extended diagonals, then a rotate-and-sum
# over the ARD_pad / width blocks of a period); its bias and the constant 1
# of slot width-1 (biases of later layers) are one plaintext added after
# FC1's rescale, encoded at the ciphertext's scale.
# ---------------------------------------------------------------------------
@dataclass
class GestureConfig:
    antennas: int = 4           # A (virtual antennas)
    bins: int = 64              # R range bins
    chirps: int = 32            # D chirps = Doppler bins
    frames: int = 60            # F
    fc_dims: tuple = (31, 16, 6)  # d_1, d_2, classes (d_0 = A R D feature slots)
    width: int = 32             # slot period of the FC layers after FC1
    complex_slots: bool = False # Re + i Im in one complex slot: one ciphertext per frame group
    # feature map between the notch and the frame accumulation: None = the
    # paper's soft power gamma = 4 and weighting f = p (p^2)^2 (three levels);
    # (a, b) = the learned f = a p + b p^2 (one level)
    feature_coef: tuple = None

    @property
    def feature_depth(self):
        return 3 if self.feature_coef is None else 1

    @property
    def ard(self):
        return self.antennas * self.bins * self.chirps


def notch_mask(D):
    """m[d] of Eq. (notch mask), read as zero on [floor(D/2), ceil(D/2)]."""
    m = np.ones(D)
    m[D // 2: -(-D // 2) + 1] = 0.0
    return m


class GestureLayout:
    def __init__(self, slots, cfg):
        self.cfg = cfg
        self.ard_pad = next_pow2(cfg.ard)
        assert self.ard_pad <= slots
        self.k = slots // self.ard_pad           # frames per ciphertext pair
        self.pairs = -(-cfg.frames // self.k)
        self.slots = slots

    def pack_complex(self, zt):
        """zt [F, A, R, D] complex -> list of complex slot vectors (Re + i Im)."""
        return [re + 1j * im for re, im in self.pack(zt)]

    def pack(self, zt):
        """zt [F, A, R, D] complex -> list of (re, im) slot vectors."""
        cfg = self.cfg
        out = []
        for p in range(self.pairs):
            re, im = np.zeros(self.slots), np.zeros(self.slots)
            for j in range(self.k):
                f = p * self.k + j
                if f < cfg.frames:
                    v = zt[f].reshape(-1)
                    re[j * self.ard_pad: j * self.ard_pad + cfg.ard] = v.real
                    im[j * self.ard_pad: j * self.ard_pad + cfg.ard] = v.imag
            out.append((re, im))
        return out

    def active(self):
        """1 on the A R D feature slots of every frame position."""
        v = np.zeros(self.slots)
        for j in range(self.k):
            v[j * self.ard_pad: j * self.ard_pad + self.cfg.ard] = 1.0
        return v


class GestureCircuit:
    def __init__(self, P, cfg=GestureConfig()):
        self.P, self.cfg = P, cfg
        self.lay = GestureLayout(P.slots, cfg)
        D, W = cfg.chirps, cfg.width
        assert W & (W - 1) == 0 and max(cfg.fc_dims) < W and W <= self.lay.ard_pad
        assert len(cfg.fc_dims) == 3
        self.n1, _ = bsgs_split(2 * D)           # K3: deltas -(D-1) .. D-1
        self.deltas = list(range(-(D - 1), D))
        self.nf1, _ = bsgs_split(W)              # FC layers
        self.fc_tail = FcCircuit.__new__(FcCircuit)   # layers 2 and 3 on period W
        self.fc_tail.P, self.fc_tail.D = P, W
        self.fc_tail.cfg = FcConfig(dims=tuple(cfg.fc_dims), width=W)
        self.fc_tail.layers = 2
        self.fc_tail.n1, self.fc_tail.n2 = bsgs_split(W)
        L = P.L
        # levels (Table 1): K3 L->L-1, |z|^2 ->L-2, notch ->L-3, two squares
        # ->L-5, weighting ->L-6, FC1 ->L-7, square ->L-8, FC2 ->L-9, square
        # ->L-10, FC3 ->L-11; the learned feature map a p + b p^2 takes one
        # level instead of three (features at L-4, logits at L-9)
        lf = L - 3 - cfg.feature_depth
        assert lf - 5 >= 0, "not enough levels for the gesture chain"
        self.lv_dft, self.lv_notch, self.lv_fc1 = L, L - 2, lf
        self.lv_fc = [lf, lf - 2, lf - 4]

    # -- public constants --------------------------------------------------
    def doppler_diagonal(self, M, delta):
        """diag_delta[s] = M[i][i + delta], i = s mod D, on active slots whose
        block holds column i + delta (block-diagonal I (x) M of Eq. K3)."""
        D = self.cfg.chirps
        i = np.arange(self.P.slots) % D
        j = i + delta
        ok = (j >= 0) & (j < D)
        v = np.zeros(self.P.slots, dtype=M.dtype)
        v[ok] = M[i[ok], j[ok]]
        return v * self.lay.active()

    def fc1_diagonal(self, W0, k):
        """Extended diagonal k of FC1 (W0: width x (A R D), no bias column):
        diag_k[s] = W0[s mod width][(s + k) mod ARD_pad], zero on padding
        columns and on row width-1.  Slot width-1 of every period carries the
        constant 1 that the later layers read as their bias input (the FC
        layers of Sec. "Encrypted ML Inference" fold the bias into the
        matrix); FC1's own bias vector, with that 1 in slot width-1, is added
        after the rescale, so FC1's product must leave the slot empty."""
        P, cfg, n = self.P, self.cfg, self.lay.ard_pad
        s = np.arange(P.slots)
        col = (s + k) % n
        v = np.zeros(P.slots)
        ok = (col < cfg.ard) & (s % cfg.width != cfg.width - 1)   # slot width-1 carries the constant
        v[ok] = W0[s[ok] % cfg.width, col[ok]]
        return v

    def notch_scale(self, scale_in):
        """Scale of the notched power, following the evaluator's scale
        arithmetic (products multiply scales, a rescale at level l divides
        by q_l, constants carry scale q_l)."""
        q, L = self.P.q, self.P.L
        s = scale_in * q[L] / q[L]                 # K3
        s = s * s / q[L - 1]                       # |z|^2
        return s * q[L - 2] / q[L - 2]             # notch

    def fc1_out_scale(self, scale_in):
        """Scale of FC1's rescaled output (the same arithmetic)."""
        q, L = self.P.q, self.P.L
        p = self.notch_scale(scale_in)
        if self.cfg.feature_coef is not None:
            f = p * p / q[L - 3]                   # (notched p) x (b p + a)
            return f * q[L - 4] / q[L - 4]         # FC1
        w = p * p / q[L - 3]
        w = w * w / q[L - 4]                       # gamma = 4
        f = p * w / q[L - 5]                       # weighting
        return f * q[L - 6] / q[L - 6]             # FC1

    def constants(self, mats, scale_in=None):
        """mats[0]: width x (A R D + 1) (bias last); mats[1], mats[2]:
        width x width in the FC layout (bias column width-1)."""
        P, cfg, q = self.P, self.cfg, self.P.q
        L = P.L
        Wd = dft_kernel(cfg.chirps)
        C, S = Wd.real, Wd.imag
        out = {}
        for delta in self.deltas:
            g = delta // self.n1
            if cfg.complex_slots:
                v = prerotate(self.doppler_diagonal(Wd, delta), g, self.n1, 1)
                out[("gdft_w", delta)] = ck.encode(P, v, q[L], L)
                continue
            for tag, M in (("gdft_c", C), ("gdft_s", S), ("gdft_ms", -S)):
                v = prerotate(self.doppler_diagonal(M, delta), g, self.n1, 1)
                out[(tag, delta)] = ck.encode(P, v, q[L], L)
        m = np.tile(notch_mask(cfg.chirps), P.slots // cfg.chirps) * self.lay.active()
        out[("notch",)] = ck.encode(P, m, q[L - 2], L - 2)
        if cfg.feature_coef is not None:
            a, b = cfg.feature_coef
            out[("notch_b",)] = ck.encode(P, b * m, q[L - 2], L - 2)
            # a joins the product b p by addition: encoded at that ciphertext's scale
            scale_in = P.scale if scale_in is None else scale_in
            out[("feat_a",)] = ck.encode(P, a * self.lay.active(), self.notch_scale(scale_in), L - 3)
        W0 = np.asarray(mats[0], dtype=np.float64)
        assert W0.shape == (cfg.width, cfg.ard + 1)
        lv = self.lv_fc[0]
        for k in range(cfg.width):
            v = prerotate(self.fc1_diagonal(W0[:, :cfg.ard], k), k // self.nf1, self.nf1, 1)
            out[("fcw", 0, k)] = ck.encode(P, v, q[lv], lv)
        b = W0[:, cfg.ard].copy()
        b[cfg.width - 1] = 1.0
        s_out = self.fc1_out_scale(P.scale if scale_in is None else scale_in)
        out[("fcb",)] = ck.encode(P, np.tile(b, P.slots // cfg.width), s_out, lv - 1)
        for l in (1, 2):
            lv = self.lv_fc[l]
            for k in self.fc_tail.present(l - 1):
                v = prerotate(self.fc_tail.diagonal(mats[l], k), k // self.nf1, self.nf1, 1)
                out[("fcw", l, k)] = ck.encode(P, v, q[lv], lv)
        return out

    def rotations(self):
        P, cfg, lay = self.P, self.cfg, self.lay
        ks = set(range(1, self.n1))
        ks |= {(d // self.n1) * self.n1 for d in self.deltas}
        ks |= {lay.ard_pad << i for i in range(int(math.log2(lay.k)))}
        ks |= set(range(1, self.nf1)) | {g * self.nf1 for g in range(1, cfg.width // self.nf1)}
        ks |= {cfg.width << i for i in range(int(math.log2(lay.ard_pad // cfg.width)))}
        out = sorted({k % P.slots for k in ks} - {0})
        return ([ck.ROT_CONJ] if cfg.complex_slots else []) + out

    # -- the circuit ---------------------------------------------------------
    def features(self, ev, consts, pairs):
        """K3 -> K1 -> K6 -> soft power -> weighting (or the learned feature
        map) per pair, then the accumulation over every frame; returns the
        feature ciphertext (every frame position of it holds the sum) at
        level L - 6 (learned: L - 4).  pairs:
        (re, im) ciphertexts, or with complex slots one ciphertext each."""
        acc = None
        for pair in pairs:
            if self.cfg.complex_slots:
                # K3 on Re + i Im: one product with the complex W (Eq. K3 in one
                # step); K1 |d|^2 = d conj(d)
                z = pair
                babies = {"z": ev.hoisted(z, list(range(self.n1)))}
                cw = {("z", delta): consts[("gdft_w", delta)] for delta in self.deltas}
                d = ev.rescale(ev.bsgs(babies, cw, self.n1, 1, z.level))
                p = ev.rescale(ev.relin(ev.tensor(d, ev.conjugate(d))))   # K1
            else:
                re, im = pair
                babies = {"re": ev.hoisted(re, list(range(self.n1))), "im": ev.hoisted(im, list(range(self.n1)))}
                c_re = {}
                c_im = {}
                for delta in self.deltas:
                    c_re[("re", delta)] = consts[("gdft_c", delta)]
                    c_re[("im", delta)] = consts[("gdft_ms", delta)]
                    c_im[("re", delta)] = consts[("gdft_s", delta)]
                    c_im[("im", delta)] = consts[("gdft_c", delta)]
                d_re = ev.rescale(ev.bsgs(babies, c_re, self.n1, 1, re.level))
                d_im = ev.rescale(ev.bsgs(babies, c_im, self.n1, 1, re.level))
                p = ev.rescale(ev.square_sum([d_re, d_im]))            # K1
            if self.cfg.feature_coef is not None:
                # learned map a p + b p^2 = (notched p) x (b notched p + a), one level
                pb = ev.add_plain(ev.rescale(ev.mul_plain(p, consts[("notch_b",)])), consts[("feat_a",)])
                pn = ev.rescale(ev.mul_plain(p, consts[("notch",)]))   # K6
                f = ev.rescale(ev.relin(ev.tensor(pn, pb)))
                acc = f if acc is None else ev.add(acc, f)
                continue
            p = ev.rescale(ev.mul_plain(p, consts[("notch",)]))    # K6
            w = ev.rescale(ev.square_sum([p]))                     # K2, gamma = 4
            w = ev.rescale(ev.square_sum([w]))
            f = ev.rescale(ev.relin(ev.tensor(ev.drop(p, w.level), w)))   # p x w
            acc = f if acc is None else ev.add(acc, f)
        return ev.rotsum(acc, self.lay.ard_pad, self.lay.k)

    def run(self, ev, consts, pairs):
        """pairs: the window's (re, im) ciphertexts at the top level.
        Returns the logits ciphertext (level L - 11, logits in slots
        0..classes-1 of every width-slot period)."""
        cfg = self.cfg
        x = self.features(ev, consts, pairs)
        babies = {"x": ev.hoisted(x, list(range(self.nf1)))}
        cl = {("x", k): consts[("fcw", 0, k)] for k in range(cfg.width)}
        y = ev.rescale(ev.bsgs(babies, cl, self.nf1, 1, x.level))
        y = ev.rotsum(y, cfg.width, self.lay.ard_pad // cfg.width)
        y = ev.add_plain(y, consts[("fcb",)])
        x = ev.rescale(ev.square_sum([y]))
        for l in (1, 2):
            babies = {"x": ev.hoisted(x, list(range(self.nf1)))}
            cl = {("x", k): consts[("fcw", l, k)] for k in self.fc_tail.present(l - 1)}
            y = ev.rescale(ev.bsgs(babies, cl, self.nf1, 1, x.level))
            x = ev.rescale(ev.square_sum([y])) if l == 1 else y
        return x


def gesture_forward(mats, feat, cfg):
    """FP64 forward pass of the same network on the accumulated features
    feat [A, R, D] (slot order a R D + r D + d)."""
    W0 = np.asarray(mats[0], dtype=np.float64)
    v = W0[:, : cfg.ard] @ feat.reshape(-1) + W0[:, cfg.ard]
    v[cfg.width - 1] = 1.0
    v = v * v
    v = np.asarray(mats[1], dtype=np.float64) @ v
    v = v * v
    return np.asarray(mats[2], dtype=np.float64) @ v
