"""B300 (sm_103a) homomorphic evaluation of the mmFHE cloud-side kernel chain.

Python binding of libmmfhe (include/mmfhe.h): RNS-CKKS key switching
(batched NTT, ModUp/ModDown basis conversion, Galois automorphisms, the dnum
key inner product, rescale, hoisted BSGS rotations) and the paper's
vital-sign circuit, evaluated on batches of ciphertext windows on one GPU.
The binding only marshals arguments; every operation runs in the library.
"""
import ctypes

import numpy as np

from . import _lib
from ._lib import (CIRCUIT_FC, CIRCUIT_FIR_DFT, CIRCUIT_GESTURE, CIRCUIT_VITAL, CIRCUIT_VITAL_PER_FRAME, CONST_TAGS, ROT_CONJ, BatcherConfig, BatcherStats, CircuitConfig, ConstKey,
                   BLOB_KEYS, BLOB_PLAN, CtHeader, MmfheError, Params, ServerConfig, ServerStats, Tuning, check, ptr,
                   ptr_array, stream_ptr)

__all__ = ["Context", "Keys", "Plan", "Graph", "Batcher", "Server", "params_select", "params_from_primes", "encode", "pack_window", "MmfheError",
           "Params", "CIRCUIT_FIR_DFT", "CIRCUIT_VITAL", "CIRCUIT_FC", "vital_config", "fir_dft_config",
           "fc_config", "fir_dft_params", "vital_params", "fc_params", "fold_poly_net", "CIRCUIT_GESTURE",
           "gesture_params", "gesture_config", "fold_poly_net_wide", "Ntt32", "ntt32_primes", "ROT_CONJ"]


def params_select(log_n, num_q, q0_bits, q_bits, num_p, p_bits, dnum):
    """Deterministic prime chain (host only)."""
    p = Params()
    check(_lib.lib().mmfhe_params_select(log_n, num_q, q0_bits, q_bits, num_p, p_bits, dnum, ctypes.byref(p)))
    return p


def params_from_primes(log_n, q, p, dnum):
    out = Params()
    out.log_n, out.num_q, out.num_p, out.dnum = log_n, len(q), len(p), dnum
    for i, x in enumerate(q):
        out.q[i] = int(x)
    for i, x in enumerate(p):
        out.p[i] = int(x)
    return out


def fir_dft_params():
    """N = 2^13, q_0 ~ 2^44 + 3 x 2^40, one 44-bit special prime, dnum = 4."""
    return params_select(13, 4, 44, 40, 1, 44, 4)


def vital_params():
    """N = 2^15, depth 11 (q_0 60 bits + 11 x 40 bits), K = 4 x 60 bits, dnum = 3."""
    return params_select(15, 12, 60, 40, 4, 60, 3)


def encode(params, slots, scale, level):
    """Encode N/2 real slots at `scale` into uint64[level+1][N] (host)."""
    slots = np.ascontiguousarray(slots, dtype=np.float64)
    out = np.empty((level + 1, 1 << params.log_n), dtype=np.uint64)
    check(_lib.lib().mmfhe_encode(ctypes.byref(params), ptr(slots), float(scale), level, ptr(out)))
    return out


def params_hash(params):
    """The parameter-set fingerprint carried by headers and blobs."""
    v = ctypes.c_uint64()
    _lib.check(_lib.lib().mmfhe_params_hash(ctypes.byref(params), ctypes.byref(v)))
    return v.value


def ct_header(params, level, scale):
    """The 32-byte header of a ciphertext at `level` and `scale`."""
    h = _lib.CtHeader()
    _lib.check(_lib.lib().mmfhe_ct_header_make(ctypes.byref(params), level, float(scale), ctypes.byref(h)))
    return h


def _blob_buffer(nbytes):
    return np.zeros((nbytes + 7) // 8, dtype=np.uint64)


def keys_blob(params, relin, galois):
    """Serialize evaluation keys: relin words and {rotation: words}."""
    rots = sorted(galois, key=lambda r: (r != ROT_CONJ, r))
    relin = np.ascontiguousarray(relin, dtype=np.uint64)
    gal = [np.ascontiguousarray(galois[r], dtype=np.uint64) for r in rots]
    rarr = (ctypes.c_int32 * max(1, len(rots)))(*rots)
    garr = ptr_array(gal) if gal else None
    size = ctypes.c_size_t()
    L = _lib.lib()
    _lib.check(L.mmfhe_keys_blob_write(ctypes.byref(params), ptr(relin), len(rots), rarr, garr, None, 0,
                                       ctypes.byref(size)))
    out = _blob_buffer(size.value)
    _lib.check(L.mmfhe_keys_blob_write(ctypes.byref(params), ptr(relin), len(rots), rarr, garr, ptr(out),
                                       out.nbytes, ctypes.byref(size)))
    return out


def plan_blob(params, cfg, consts):
    """Serialize a plan: its configuration and [(level, words)] constants in
    the plan's order."""
    levels = (ctypes.c_uint32 * max(1, len(consts)))(*[lv for lv, _ in consts])
    words = [np.ascontiguousarray(w, dtype=np.uint64) for _, w in consts]
    warr = ptr_array(words) if words else None
    size = ctypes.c_size_t()
    L = _lib.lib()
    args = (ctypes.byref(params), ctypes.byref(cfg), ctypes.sizeof(CircuitConfig), len(consts), levels, warr)
    _lib.check(L.mmfhe_plan_blob_write(*args, None, 0, ctypes.byref(size)))
    out = _blob_buffer(size.value)
    _lib.check(L.mmfhe_plan_blob_write(*args, ptr(out), out.nbytes, ctypes.byref(size)))
    return out


def blob_check(params, blob):
    """Validate a blob without a GPU; returns its kind (BLOB_KEYS or BLOB_PLAN)."""
    kind = ctypes.c_uint32()
    _lib.check(_lib.lib().mmfhe_blob_check(ctypes.byref(params), ptr(blob), blob.nbytes, ctypes.byref(kind)))
    return kind.value


def debug_fail_allocations(after):
    """Host-side failure injection for tests: after `after` more successful
    device allocations every library allocation fails with OUT_OF_MEMORY
    (without calling cudaMalloc); after < 0 disarms."""
    _lib.check(_lib.lib().mmfhe_debug_fail_allocations(int(after)))


def pack_window(log_n, values):
    """Batched-packing layout of a [F, R] real array into G slot vectors."""
    values = np.ascontiguousarray(values, dtype=np.float64)
    F, R = values.shape
    n = 1 << (log_n - 1)
    fp = 1
    while fp < F:
        fp <<= 1
    G = -(-R // (n // fp))
    out = np.empty((G, n), dtype=np.float64)
    check(_lib.lib().mmfhe_pack_window(log_n, F, R, ptr(values), ptr(out)))
    return out


def vital_config(bins=256, frames=200, fs_mhz=20000, taps=64, taylor_order=3,
                 bands_mhz=((100, 600), (800, 2500)), dft_gains=(0.0, 0.0), per_frame=False, complex_slots=False):
    """The vital chain; per_frame=True: the per-frame packing (one ciphertext
    per frame and part, the paper's slow baseline); complex_slots=True: each
    stream's Re + i Im in one ciphertext per group (needs the key ROT_CONJ)."""
    c = CircuitConfig()
    c.complex_slots = int(bool(complex_slots))
    kind = CIRCUIT_VITAL_PER_FRAME if per_frame else CIRCUIT_VITAL
    c.kind, c.bins, c.frames, c.fs_mhz, c.taps, c.taylor_order = kind, bins, frames, fs_mhz, taps, taylor_order
    c.num_bands = 2
    for b in range(2):
        c.band_lo_mhz[b], c.band_hi_mhz[b] = bands_mhz[b]
        c.dft_gain[b] = dft_gains[b]
    return c


def fc_params():
    """N = 2^14, q_0 ~ 2^60 + 5 x 2^40, two 60-bit special primes, dnum = 3:
    depth 5, enough for three dense layers and two squares."""
    return params_select(14, 6, 60, 40, 2, 60, 3)


def fc_config(dims=(120, 32, 16, 6), width=128):
    """Polynomial network: dense layers d_0 -> ... -> d_L on a slot period of
    `width` (slot width-1 holds the constant 1), square after each but the last."""
    c = CircuitConfig()
    c.kind, c.bins, c.taps = CIRCUIT_FC, width, len(dims) - 1
    for i, d in enumerate(dims):
        c.fc_dims[i] = d
    return c


def fold_poly_net(dims, alpha, weights, width=128):
    """Trained quadratic-activation weights -> the pure-square D x D layer
    matrices of an FC plan (host only)."""
    d = (ctypes.c_uint32 * len(dims))(*dims)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    mats = np.empty((len(dims) - 1, width, width), dtype=np.float64)
    check(_lib.lib().mmfhe_fold_poly_net(d, len(dims) - 1, float(alpha), ptr(w), width, ptr(mats)))
    return mats


def fold_poly_net_wide(dims, alpha, weights, width=32):
    """As fold_poly_net for a network whose input width d_0 may exceed
    `width` (a gesture plan's FC1): returns (first, mats), first = width x
    (d_0 + 1), mats = (layers-1) x width x width."""
    d = (ctypes.c_uint32 * len(dims))(*dims)
    w = np.ascontiguousarray(weights, dtype=np.float32)
    first = np.empty((width, dims[0] + 1), dtype=np.float64)
    mats = np.empty((max(1, len(dims) - 2), width, width), dtype=np.float64)
    check(_lib.lib().mmfhe_fold_poly_net_wide(d, len(dims) - 1, float(alpha), ptr(w), width, ptr(first), ptr(mats)))
    return first, mats[: len(dims) - 2]


def gesture_params(learned=False):
    """N = 2^15, Delta = 2^50: q_0 60 bits + 11 x 50 bits for the paper's
    depth-11 chain, or + 9 x 50 bits for the chain with the learned degree-2
    feature map (depth 9); K = 4 x 60 bits, dnum = 3."""
    return params_select(15, 10 if learned else 12, 60, 50, 4, 60, 3)


FEATURE_POWER, FEATURE_LEARNED = 0, 1


def gesture_config(antennas=4, bins=64, chirps=32, frames=60, fc_dims=(31, 16, 6), fc_width=32,
                   input_scale=2.0 ** 50, complex_slots=False, feature_coef=None):
    """The gesture chain: K3 Doppler DFT -> K1 -> K6 -> feature map, summed
    over frames, then FC1^2 -> FC2^2 -> FC3 (fc_dims = d_1, d_2, classes on a
    slot period of fc_width).  Feature map: the paper's w = p^4 and p w, or
    with feature_coef = (a, b) the learned a p + b p^2.  complex_slots:
    Re + i Im of a frame group in one ciphertext (needs the key ROT_CONJ)."""
    c = CircuitConfig()
    c.kind, c.bins, c.frames = CIRCUIT_GESTURE, bins, frames
    c.complex_slots = int(bool(complex_slots))
    c.antennas, c.chirps, c.fc_width, c.input_scale = antennas, chirps, fc_width, float(input_scale)
    c.fc_dims[0] = antennas * bins * chirps
    for i, d in enumerate(fc_dims):
        c.fc_dims[i + 1] = d
    if feature_coef is not None:
        c.feature_map = FEATURE_LEARNED
        c.feature_coef[0], c.feature_coef[1] = float(feature_coef[0]), float(feature_coef[1])
    return c


def ntt32_primes(log_n, bits, count):
    """The `count` largest primes below 2^bits that are 1 mod 2N (host only)."""
    out = (ctypes.c_uint32 * count)()
    check(_lib.lib().mmfhe_ntt32_select_primes(log_n, bits, count, out))
    return [out[i] for i in range(count)]


class Ntt32:
    """Word-size ablation: the negacyclic NTT on 32-bit RNS words (primes
    below 2^30), one shared-memory pass per row."""

    def __init__(self, log_n, primes, device=0):
        arr = (ctypes.c_uint32 * len(primes))(*primes)
        h = ctypes.c_void_p()
        check(_lib.lib().mmfhe_ntt32_create(log_n, arr, len(primes), device, ctypes.byref(h)))
        self.h, self.log_n, self.primes = h, log_n, list(primes)

    def run(self, rows, inverse=False, stream=None):
        """In place on uint32 rows [..., N] (numpy or a CUDA tensor), row r
        under primes[r mod len(primes)]."""
        n_rows = (rows.numel() if hasattr(rows, "numel") else rows.size) >> self.log_n
        check(_lib.lib().mmfhe_ntt32_run(self.h, ptr(rows), n_rows, int(inverse), stream_ptr(stream)))

    def close(self):
        if getattr(self, "h", None):
            _lib.lib().mmfhe_ntt32_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fir_dft_config(bins=64, frames=200, fs_mhz=20000, taps=64, band_mhz=(800, 2500)):
    c = CircuitConfig()
    c.kind, c.bins, c.frames, c.fs_mhz, c.taps = CIRCUIT_FIR_DFT, bins, frames, fs_mhz, taps
    c.num_bands = 1
    c.band_lo_mhz[0], c.band_hi_mhz[0] = band_mhz
    return c


class Context:
    """One parameter set on one CUDA device."""

    def __init__(self, params, device=0):
        self.params = params
        self.n = 1 << params.log_n
        self.L = params.num_q - 1
        h = ctypes.c_void_p()
        check(_lib.lib().mmfhe_ctx_create(ctypes.byref(params), ctypes.sizeof(Params), device, ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _lib.lib().mmfhe_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, status):
        check(status, self.h)

    def sync(self, stream=None, timeout_ms=60000):
        self._c(_lib.lib().mmfhe_sync(self.h, stream_ptr(stream), timeout_ms))

    def launch_count(self):
        v = ctypes.c_uint64()
        self._c(_lib.lib().mmfhe_launch_count(self.h, ctypes.byref(v)))
        return v.value

    def mem_stats(self):
        """Device bytes the library holds on this context's device (now and
        at the high-water mark), its cudaMalloc count, and this context's pool."""
        m = _lib.MemStats()
        self._c(_lib.lib().mmfhe_mem_stats_get(self.h, ctypes.byref(m)))
        return {n: int(getattr(m, n)) for n, _ in _lib.MemStats._fields_}

    def mem_peak_reset(self):
        self._c(_lib.lib().mmfhe_mem_peak_reset(self.h))

    def trace(self, enable=None):
        """Enable/disable the launch trace, or (enable=None) return it."""
        if enable is not None:
            self._c(_lib.lib().mmfhe_trace_enable(self.h, int(enable)))
            return None
        n = ctypes.c_size_t()
        self._c(_lib.lib().mmfhe_trace_get(self.h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value + 1)
        self._c(_lib.lib().mmfhe_trace_get(self.h, buf, n.value + 1, ctypes.byref(n)))
        return buf.value.decode().splitlines()

    def profile(self, enable=None):
        """Enable/disable per-kernel event profiling, or (enable=None) return
        {kernel: (launches, total_ms, algorithmic_bytes, butterflies, conversion_macs)}."""
        if enable is not None:
            self._c(_lib.lib().mmfhe_profile_enable(self.h, int(enable)))
            return None
        n = ctypes.c_uint32()
        self._c(_lib.lib().mmfhe_profile_get(self.h, None, 0, ctypes.byref(n)))
        arr = (_lib.KernelStat * max(1, n.value))()
        self._c(_lib.lib().mmfhe_profile_get(self.h, arr, n.value, ctypes.byref(n)))
        return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms, arr[i].bytes, arr[i].butterflies,
                                       arr[i].macs) for i in range(n.value)}

    def butterfly_peak(self):
        """(64-bit, 32-bit) forward butterflies per second of a register-resident
        loop on this device: the integer-pipe ceiling of the NTT arithmetic."""
        a, b = ctypes.c_double(), ctypes.c_double()
        self._c(_lib.lib().mmfhe_measure_butterfly_peak(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def mac_peak(self):
        """Products per second of a register-resident loop of the base
        conversion's Montgomery multiply-accumulate on this device."""
        a = ctypes.c_double()
        self._c(_lib.lib().mmfhe_measure_mac_peak(self.h, ctypes.byref(a)))
        return a.value

    def keys(self, user_id=0):
        return Keys(self, user_id)

    def train_poly_net(self, X, labels, dims, alpha=0.1, epochs=30, batch=128, lr=0.05, seed=1):
        """Plaintext GPU training of the quadratic-activation network.
        Returns (flat float32 weights, training accuracy)."""
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.ascontiguousarray(labels, dtype=np.int32)
        d = (ctypes.c_uint32 * len(dims))(*dims)
        nw = sum(dims[l + 1] * (dims[l] + 1) for l in range(len(dims) - 1))
        w = np.empty(nw, dtype=np.float32)
        acc = ctypes.c_float()
        self._c(_lib.lib().mmfhe_train_poly_net(self.h, ptr(X), ptr(y), len(y), d, len(dims) - 1, float(alpha), epochs,
                                                 batch, float(lr), seed, ptr(w), ctypes.byref(acc)))
        return w, acc.value

    def autotune(self, batch, level=None):
        """Time the NTT / key-inner-product tile variants on `batch`
        ciphertexts at `level` (default: top) and keep the fastest."""
        t = Tuning()
        self._c(_lib.lib().mmfhe_autotune(self.h, batch, self.L if level is None else level, ctypes.byref(t)))
        return _tuning_dict(t)

    def tuning(self):
        t = Tuning()
        self._c(_lib.lib().mmfhe_tuning_get(self.h, ctypes.byref(t)))
        return _tuning_dict(t)

    def set_tuning(self, cols_width, rows_threads, keyip_windows, conv_rows=1, keyip_fused=0, keyip_pipe=0,
                   combine_pipe=0):
        t = Tuning(cols_width, rows_threads, keyip_windows, conv_rows)
        t.keyip_fused = keyip_fused
        t.keyip_pipe = keyip_pipe
        t.combine_pipe = combine_pipe
        self._c(_lib.lib().mmfhe_tuning_set(self.h, ctypes.byref(t)))

    def graph(self, plan, keys, ins, outs):
        """Capture one evaluation of `plan` on device buffers as a CUDA graph."""
        return Graph(self, plan, keys, ins, outs)

    def batcher(self, base_cfg, **kw):
        return Batcher(self, base_cfg, **kw)

    def server(self, base_cfg, **kw):
        return Server(self, base_cfg, **kw)

    def plan(self, cfg):
        return Plan(self, cfg)

    def keys_load(self, blob, user_id=0):
        """Resident keys from a serialized key blob (validated first)."""
        h = ctypes.c_void_p()
        self._c(_lib.lib().mmfhe_keys_load(self.h, user_id, ptr(blob), blob.nbytes, ctypes.byref(h)))
        return Keys._from_handle(self, h)

    def plan_load(self, blob):
        """A plan from a serialized plan blob (validated first)."""
        h = ctypes.c_void_p()
        self._c(_lib.lib().mmfhe_plan_load(self.h, ptr(blob), blob.nbytes, ctypes.byref(h)))
        p = Plan._borrowed(self, h)
        p.owned = True
        return p

    # --- primitives (coefficient-form buffers) -----------------------------
    def ntt(self, rows, prime_idx, inverse=False, stream=None):
        pid = np.ascontiguousarray(prime_idx, dtype=np.uint32)
        self._c(_lib.lib().mmfhe_ntt(self.h, ptr(rows), ptr(pid), len(pid), int(inverse), stream_ptr(stream)))

    def ntt_batch(self, rows, blocks, limbs, inverse=False, stream=None):
        """The evaluator's batched transform on device rows [blocks][limbs][N] (asynchronous)."""
        self._c(_lib.lib().mmfhe_ntt_batch(self.h, ptr(rows), blocks, limbs, int(inverse), stream_ptr(stream)))

    def poly_mul(self, out, a, b, prime_idx, stream=None):
        pid = np.ascontiguousarray(prime_idx, dtype=np.uint32)
        self._c(_lib.lib().mmfhe_poly_mul(self.h, ptr(out), ptr(a), ptr(b), ptr(pid), len(pid), stream_ptr(stream)))

    def ct_add(self, out, a, b, batch, level, stream=None):
        self._c(_lib.lib().mmfhe_ct_add(self.h, ptr(out), ptr(a), ptr(b), batch, level, stream_ptr(stream)))

    def ct_mul_plain(self, out, ct, pt, batch, level, stream=None):
        self._c(_lib.lib().mmfhe_ct_mul_plain(self.h, ptr(out), ptr(ct), ptr(pt), batch, level, stream_ptr(stream)))

    def ct_mul_relin(self, keys, out, a, b, batch, level, stream=None):
        self._c(_lib.lib().mmfhe_ct_mul_relin(self.h, keys.h, ptr(out), ptr(a), ptr(b), batch, level,
                                              stream_ptr(stream)))

    def ct_rescale(self, out, a, batch, level, stream=None):
        self._c(_lib.lib().mmfhe_ct_rescale(self.h, ptr(out), ptr(a), batch, level, stream_ptr(stream)))

    def ct_rotate(self, keys, out, a, batch, level, k, stream=None):
        self._c(_lib.lib().mmfhe_ct_rotate(self.h, keys.h, ptr(out), ptr(a), batch, level, k, stream_ptr(stream)))

    def ct_rotate_hoisted(self, keys, outs, a, batch, level, ks, stream=None):
        ka = (ctypes.c_int32 * len(ks))(*ks)
        self._c(_lib.lib().mmfhe_ct_rotate_hoisted(self.h, keys.h, ptr_array(outs), ptr(a), batch, level, ka, len(ks),
                                                   stream_ptr(stream)))

    def modup(self, out, d, batch, level, stream=None):
        self._c(_lib.lib().mmfhe_modup(self.h, ptr(out), ptr(d), batch, level, stream_ptr(stream)))

    def keyswitch(self, keys, out, d, batch, level, rotation=None, stream=None):
        which, rot = (0, 0) if rotation is None else (1, rotation)
        self._c(_lib.lib().mmfhe_keyswitch(self.h, keys.h, which, rot, ptr(out), ptr(d), batch, level,
                                           stream_ptr(stream)))

    def keyswitch_noalloc(self, keys, out, d, batch, level, rotation=None, stream=None):
        """Key switch using only the library's fixed device scratch array (no
        device allocation in the call); out and d must be device buffers."""
        which, rot = (0, 0) if rotation is None else (1, rotation)
        self._c(_lib.lib().mmfhe_keyswitch_noalloc(self.h, keys.h, which, rot, ptr(out), ptr(d), batch, level,
                                                   stream_ptr(stream)))

    def ct_rotsum(self, keys, out, a, batch, level, stride, span, stream=None):
        self._c(_lib.lib().mmfhe_ct_rotsum(self.h, keys.h, ptr(out), ptr(a), batch, level, stride, span,
                                           stream_ptr(stream)))

    def ct_bsgs(self, keys, out, a, batch, level, stride, n1, deltas, diags, stream=None):
        da = np.ascontiguousarray(deltas, dtype=np.uint32)
        self._c(_lib.lib().mmfhe_ct_bsgs(self.h, keys.h, ptr(out), ptr(a), batch, level, stride, n1, ptr(da),
                                         ptr_array(diags), len(diags), stream_ptr(stream)))

    def ct_bsgs_dh(self, keys, out, a, batch, level, stride, n1, offsets, diags, stream=None):
        """Double-hoisted BSGS product; diags = [(set, delta, words over Q_level)]."""
        offs = np.ascontiguousarray(offsets, dtype=np.int32)
        so = np.ascontiguousarray([d[0] for d in diags], dtype=np.uint32)
        da = np.ascontiguousarray([d[1] for d in diags], dtype=np.uint32)
        words = [np.ascontiguousarray(d[2]) for d in diags]
        self._c(_lib.lib().mmfhe_ct_bsgs_dh(self.h, keys.h, ptr(out), ptr(a), batch, level, stride, n1, len(offs),
                                            ptr(offs), ptr(so), ptr(da), ptr_array(words), len(words),
                                            stream_ptr(stream)))

    # --- circuits -------------------------------------------------------------
    def eval(self, plan, keys, ins, outs, stream=None, vital=False):
        """Evaluate `plan` on len(ins) windows; keys is one Keys or a list."""
        B = len(ins)
        kl = keys if isinstance(keys, (list, tuple)) else [keys] * B
        karr = (ctypes.c_void_p * B)(*[k.h.value for k in kl])
        f = _lib.lib().mmfhe_eval_vital if vital else _lib.lib().mmfhe_eval
        self._c(f(self.h, plan.h, karr, ptr_array(ins), B, ptr_array(outs), stream_ptr(stream)))

    def eval_checked(self, plan, keys, in_hdrs, ins, outs, stream=None):
        """mmfhe_eval with ciphertext headers: in_hdrs[w] = list of n_in
        CtHeader; returns the output headers per window."""
        B = len(ins)
        n_in, n_out, _ = plan.io()
        kl = keys if isinstance(keys, (list, tuple)) else [keys] * B
        karr = (ctypes.c_void_p * B)(*[k.h.value for k in kl])
        hin = [(_lib.CtHeader * n_in)(*h) for h in in_hdrs]
        hout = [(_lib.CtHeader * n_out)() for _ in range(B)]
        hin_arr = (ctypes.c_void_p * B)(*[ctypes.addressof(h) for h in hin])
        hout_arr = (ctypes.c_void_p * B)(*[ctypes.addressof(h) for h in hout])
        self._c(_lib.lib().mmfhe_eval_checked(self.h, plan.h, karr, hin_arr, ptr_array(ins), B, hout_arr,
                                              ptr_array(outs), stream_ptr(stream)))
        return [list(h) for h in hout]


def _tuning_dict(t):
    return {"ntt_cols_width": t.ntt_cols_width, "ntt_rows_threads": t.ntt_rows_threads,
            "keyip_windows": t.keyip_windows, "conv_rows": t.conv_rows, "ntt_ms": list(t.ntt_ms),
            "keyip_ms": list(t.keyip_ms), "conv_ms": list(t.conv_ms), "keyip_fused": t.keyip_fused,
            "keyip_pipe": t.keyip_pipe, "keyip_pipe_ms": list(t.keyip_pipe_ms),
            "combine_pipe": t.combine_pipe, "combine_pipe_ms": list(t.combine_pipe_ms)}


class Graph:
    """A captured CUDA graph of one evaluation on fixed device buffers."""

    def __init__(self, ctx, plan, keys, ins, outs):
        self.ctx = ctx
        B = len(ins)
        kl = keys if isinstance(keys, (list, tuple)) else [keys] * B
        karr = (ctypes.c_void_p * B)(*[k.h.value for k in kl])
        h = ctypes.c_void_p()
        ctx._c(_lib.lib().mmfhe_graph_capture(ctx.h, plan.h, karr, ptr_array(ins), B, ptr_array(outs),
                                               ctypes.byref(h)))
        self.h = h

    def launch(self, stream=None):
        self.ctx._c(_lib.lib().mmfhe_graph_launch(self.h, stream_ptr(stream)))

    def info(self):
        """(kernels per replay, device bytes held)."""
        k, b = ctypes.c_uint64(), ctypes.c_uint64()
        self.ctx._c(_lib.lib().mmfhe_graph_info(self.h, ctypes.byref(k), ctypes.byref(b)))
        return k.value, b.value

    def close(self):
        if getattr(self, "h", None):
            _lib.lib().mmfhe_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batcher:
    """Queues windows of any frame count and user; flush() evaluates them in
    batches (one plan per frame count, one graph per (frames, keys, size))."""

    def __init__(self, ctx, base_cfg, max_batch=16, use_graphs=True, plan_budget_bytes=0, graph_budget_bytes=0):
        self.ctx = ctx
        self.base = base_cfg
        cfg = BatcherConfig(max_batch, int(bool(use_graphs)), plan_budget_bytes, graph_budget_bytes)
        h = ctypes.c_void_p()
        ctx._c(_lib.lib().mmfhe_batcher_create(ctx.h, ctypes.byref(base_cfg), ctypes.sizeof(CircuitConfig),
                                                ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h
        self._held = []   # buffers of queued windows stay alive until flush

    def plan(self, frames):
        """The batcher's plan for `frames` (borrowed: valid until evicted)."""
        h = ctypes.c_void_p()
        self.ctx._c(_lib.lib().mmfhe_batcher_plan(self.h, frames, ctypes.byref(h)))
        return Plan._borrowed(self.ctx, h)

    def submit(self, keys, frames, inp, out):
        self.ctx._c(_lib.lib().mmfhe_batcher_submit(self.h, keys.h, frames, ptr(inp), ptr(out)))
        self._held.append((inp, out))

    def flush(self, stream=None):
        try:
            self.ctx._c(_lib.lib().mmfhe_batcher_flush(self.h, stream_ptr(stream)))
        finally:
            self._held = []

    def forget_keys(self, keys):
        self.ctx._c(_lib.lib().mmfhe_batcher_forget_keys(self.h, keys.h))

    def stats(self):
        st = BatcherStats()
        self.ctx._c(_lib.lib().mmfhe_batcher_stats_get(self.h, ctypes.byref(st)))
        return {n: getattr(st, n) for n, _ in BatcherStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            _lib.lib().mmfhe_batcher_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop: submit windows of registered users from any thread; a
    native worker batches and runs them (see mmfhe_server_* in mmfhe.h)."""

    def __init__(self, ctx, base_cfg, max_batch=16, streams=2, key_budget_bytes=0, batch_wait_us=0):
        self.ctx = ctx
        cfg = ServerConfig(max_batch, streams, key_budget_bytes, batch_wait_us)
        h = ctypes.c_void_p()
        ctx._c(_lib.lib().mmfhe_server_create(ctx.h, ctypes.byref(base_cfg), ctypes.sizeof(CircuitConfig),
                                               ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h
        self._users = {}     # registered key words stay referenced until close
        self._live = {}      # ticket -> (input, output) kept alive until waited

    def add_user(self, user_id, relin, galois):
        """galois: {rotation: words}; the arrays must stay unchanged."""
        rots = sorted(galois)
        rarr = (ctypes.c_int32 * max(1, len(rots)))(*rots)
        garr = ptr_array([galois[r] for r in rots]) if rots else None
        self.ctx._c(_lib.lib().mmfhe_server_add_user(self.h, user_id, ptr(relin), rarr, garr, len(rots)))
        self._users[user_id] = (relin, galois, rarr, garr)

    def set_fc_layer(self, layer, W):
        """FC / gesture servers: a learned layer for every plan (before the first submit)."""
        W = np.ascontiguousarray(W, dtype=np.float64)
        self.ctx._c(_lib.lib().mmfhe_server_set_fc_layer(self.h, layer, ptr(W), W.size))

    def set_const(self, frames, index, words):
        """Install a caller-encoded constant (coefficient form) in the plan the
        server creates for `frames` (before the first submit)."""
        w = np.ascontiguousarray(words, dtype=np.uint64)
        self.ctx._c(_lib.lib().mmfhe_server_set_const(self.h, frames, index, ptr(w), w.size))

    def submit(self, user_id, frames, inp, out):
        t = ctypes.c_uint64()
        self.ctx._c(_lib.lib().mmfhe_server_submit(self.h, user_id, frames, ptr(inp), ptr(out), ctypes.byref(t)))
        self._live[t.value] = (inp, out)
        return t.value

    def cancel(self, ticket):
        """Cancel a window that is still queued (BUSY once it runs)."""
        self.ctx._c(_lib.lib().mmfhe_server_cancel(self.h, ticket))

    def wait(self, ticket, timeout_ms=600000):
        """Latency (ms) of a completed window; raises on timeout or failure."""
        lat = ctypes.c_double()
        self.ctx._c(_lib.lib().mmfhe_server_wait(self.h, ticket, timeout_ms, ctypes.byref(lat)))
        self._live.pop(ticket, None)
        return lat.value

    def drain(self, timeout_ms=600000):
        self.ctx._c(_lib.lib().mmfhe_server_drain(self.h, timeout_ms))
        self._live.clear()

    def stats(self):
        st = ServerStats()
        self.ctx._c(_lib.lib().mmfhe_server_stats_get(self.h, ctypes.byref(st)))
        return {n: getattr(st, n) for n, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None):
            _lib.lib().mmfhe_server_destroy(self.h)
            self.h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Keys:
    """Evaluation keys of one user, resident in device memory."""

    def __init__(self, ctx, user_id=0):
        self.ctx = ctx
        h = ctypes.c_void_p()
        ctx._c(_lib.lib().mmfhe_keys_create(ctx.h, user_id, ctypes.byref(h)))
        self.h = h

    @classmethod
    def _from_handle(cls, ctx, h):
        k = cls.__new__(cls)
        k.ctx, k.h = ctx, h
        return k

    def set_relin(self, words):
        self.ctx._c(_lib.lib().mmfhe_keys_set_relin(self.h, ptr(words)))

    def set_galois(self, k, words):
        self.ctx._c(_lib.lib().mmfhe_keys_set_galois(self.h, int(k), ptr(words)))

    def unload(self):
        if getattr(self, "h", None):
            _lib.lib().mmfhe_keys_unload(self.h)
            self.h = None


class Plan:
    """A circuit's public configuration and encoded constants."""

    def __init__(self, ctx, cfg):
        self.ctx = ctx
        self.cfg = cfg
        self.owned = True
        h = ctypes.c_void_p()
        ctx._c(_lib.lib().mmfhe_plan_create(ctx.h, ctypes.byref(cfg), ctypes.sizeof(CircuitConfig), ctypes.byref(h)))
        self.h = h

    @classmethod
    def _borrowed(cls, ctx, h):
        p = cls.__new__(cls)
        p.ctx, p.cfg, p.h, p.owned = ctx, None, h, False
        return p

    def num_consts(self):
        v = ctypes.c_uint32()
        self.ctx._c(_lib.lib().mmfhe_plan_num_consts(self.h, ctypes.byref(v)))
        return v.value

    def const_key(self, i):
        k = ConstKey()
        self.ctx._c(_lib.lib().mmfhe_plan_const_key(self.h, i, ctypes.byref(k)))
        return (CONST_TAGS[k.tag], k.band, k.index, k.level)

    def const_keys(self):
        return [self.const_key(i) for i in range(self.num_consts())]

    def set_const(self, i, words):
        self.ctx._c(_lib.lib().mmfhe_plan_set_const(self.h, i, ptr(words)))

    def get_const(self, i):
        level = self.const_key(i)[3]
        out = np.empty((level + 1, self.ctx.n), dtype=np.uint64)
        self.ctx._c(_lib.lib().mmfhe_plan_get_const(self.h, i, ptr(out)))
        return out

    def encode_consts(self):
        self.ctx._c(_lib.lib().mmfhe_plan_encode_consts(self.h))

    def scalars(self):
        n = ctypes.c_uint32()
        self.ctx._c(_lib.lib().mmfhe_plan_num_scalars(self.h, ctypes.byref(n)))
        out = np.empty(n.value, dtype=np.float64)
        if n.value:
            self.ctx._c(_lib.lib().mmfhe_plan_get_scalars(self.h, ptr(out), n.value))
        return out

    def set_scalars(self, values):
        v = np.ascontiguousarray(values, dtype=np.float64)
        self.ctx._c(_lib.lib().mmfhe_plan_set_scalars(self.h, ptr(v), len(v)))

    def set_fc_layer(self, layer, W):
        """FC plans: encode a layer from its D x D matrix."""
        W = np.ascontiguousarray(W, dtype=np.float64)
        self.ctx._c(_lib.lib().mmfhe_plan_set_fc_layer(self.h, layer, ptr(W)))

    def rotations(self):
        n = ctypes.c_uint32()
        self.ctx._c(_lib.lib().mmfhe_plan_rotations(self.h, None, 0, ctypes.byref(n)))
        arr = (ctypes.c_int32 * max(1, n.value))()
        self.ctx._c(_lib.lib().mmfhe_plan_rotations(self.h, arr, n.value, ctypes.byref(n)))
        return [arr[i] for i in range(n.value)]

    def io(self):
        ni, no = ctypes.c_uint32(), ctypes.c_uint32()
        lv = (ctypes.c_uint32 * 16)()
        self.ctx._c(_lib.lib().mmfhe_plan_io(self.h, ctypes.byref(ni), ctypes.byref(no), lv))
        return ni.value, no.value, [lv[i] for i in range(no.value)]

    def readout(self):
        """(output index, slot) of num_r, den_r, num_RR, den_RR, num_HR,
        den_HR for a vital plan; [] for other circuits."""
        oi, sl, n = (ctypes.c_uint32 * 6)(), (ctypes.c_uint32 * 6)(), ctypes.c_uint32()
        self.ctx._c(_lib.lib().mmfhe_plan_readout(self.h, oi, sl, 6, ctypes.byref(n)))
        return [(oi[i], sl[i]) for i in range(n.value)]

    def destroy(self):
        if getattr(self, "h", None) and self.owned:
            _lib.lib().mmfhe_plan_destroy(self.h)
        self.h = None
