"""ctypes binding of libmmfhe (argument marshalling only).

Every function here forwards to the C ABI declared in include/mmfhe.h; all
arithmetic runs in the library's CUDA kernels.  Buffers may be numpy arrays
(host memory) or torch tensors (host or CUDA memory).  A missing shared
object raises immediately: there is no fallback path.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "libmmfhe.so")

MAX_Q, MAX_P = 32, 8

OK = 0
ERRORS = {
    -1: "BAD_ARG", -2: "BAD_BLOB", -3: "PARAM_MISMATCH", -4: "LEVEL_MISMATCH", -5: "OUT_OF_MEMORY",
    -6: "CUDA", -7: "TIMEOUT", -8: "NOT_FOUND", -9: "BUSY", -10: "CANCELLED",
}
CIRCUIT_FIR_DFT, CIRCUIT_VITAL, CIRCUIT_FC, CIRCUIT_VITAL_PER_FRAME, CIRCUIT_GESTURE = 1, 2, 3, 4, 5
CONST_TAGS = {1: "idx", 2: "one", 3: "fir", 4: "dre", 5: "dim", 6: "fw", 7: "fone", 8: "dft_c", 9: "dft_s",
              10: "dft_ms", 11: "fcw", 12: "gdft_c", 13: "gdft_s", 14: "gdft_ms", 15: "notch", 16: "fcb",
              17: "gdft_w", 18: "notch_b", 19: "feat_a", 20: "pmask"}
ROT_CONJ = -(1 << 31)   # key id of the slot-wise complex conjugation


class MmfheError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code
        self.name = ERRORS.get(code, "?")


class Params(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_uint32), ("num_q", ctypes.c_uint32), ("num_p", ctypes.c_uint32),
                ("dnum", ctypes.c_uint32), ("q", ctypes.c_uint64 * MAX_Q), ("p", ctypes.c_uint64 * MAX_P)]

    @property
    def primes_q(self):
        return [int(self.q[i]) for i in range(self.num_q)]

    @property
    def primes_p(self):
        return [int(self.p[i]) for i in range(self.num_p)]


class CircuitConfig(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_uint32), ("bins", ctypes.c_uint32), ("frames", ctypes.c_uint32),
                ("fs_mhz", ctypes.c_uint32), ("taps", ctypes.c_uint32), ("taylor_order", ctypes.c_uint32),
                ("num_bands", ctypes.c_uint32), ("band_lo_mhz", ctypes.c_uint32 * 2),
                ("band_hi_mhz", ctypes.c_uint32 * 2), ("dft_gain", ctypes.c_double * 2), ("fc_dims", ctypes.c_uint32 * 9),
                ("antennas", ctypes.c_uint32), ("chirps", ctypes.c_uint32), ("fc_width", ctypes.c_uint32),
                ("complex_slots", ctypes.c_uint32), ("input_scale", ctypes.c_double),
                ("feature_map", ctypes.c_uint32), ("feature_coef", ctypes.c_double * 2)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("butterflies", ctypes.c_double), ("macs", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("ntt_cols_width", ctypes.c_uint32), ("ntt_rows_threads", ctypes.c_uint32),
                ("keyip_windows", ctypes.c_uint32), ("conv_rows", ctypes.c_uint32), ("ntt_ms", ctypes.c_float * 4),
                ("keyip_ms", ctypes.c_float * 4), ("conv_ms", ctypes.c_float * 3), ("keyip_fused", ctypes.c_uint32),
                ("keyip_pipe", ctypes.c_uint32), ("keyip_pipe_ms", ctypes.c_float * 4),
                ("combine_pipe", ctypes.c_uint32), ("combine_pipe_ms", ctypes.c_float * 3)]


class BatcherConfig(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_uint32), ("use_graphs", ctypes.c_uint32),
                ("plan_budget_bytes", ctypes.c_uint64), ("graph_budget_bytes", ctypes.c_uint64)]


class BatcherStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("windows", "batches", "graph_replays", "graphs_captured",
                                                "graphs_evicted", "plans_created", "plans_evicted", "plan_bytes",
                                                "graph_bytes")]


class ServerConfig(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_uint32), ("streams", ctypes.c_uint32), ("key_budget_bytes", ctypes.c_uint64),
                ("batch_wait_us", ctypes.c_uint32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "failed", "batches", "key_loads",
                                                "key_evictions", "keys_resident", "key_bytes")] + \
               [(n, ctypes.c_double) for n in ("mean_batch", "p50_ms", "p99_ms", "windows_per_s")] + \
               [("cancelled", ctypes.c_uint64)]


class MemStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("device_bytes", "peak_bytes", "allocations", "pool_bytes",
                                                "pool_free_bytes")]


class CtHeader(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_uint32), ("version", ctypes.c_uint16), ("reserved0", ctypes.c_uint16),
                ("level", ctypes.c_uint32), ("reserved1", ctypes.c_uint32), ("log2_scale", ctypes.c_double),
                ("params_hash", ctypes.c_uint64)]


BLOB_KEYS, BLOB_PLAN = 1, 2


class ConstKey(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint32), ("band", ctypes.c_uint32), ("index", ctypes.c_uint32),
                ("level", ctypes.c_uint32)]


_VP = ctypes.c_void_p
_U32, _U64, _I32, _SZ, _INT = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_size_t, ctypes.c_int
_PP = ctypes.POINTER(ctypes.c_void_p)

_SIGS = {
    "mmfhe_params_select": [_U32, _U32, _U32, _U32, _U32, _U32, _U32, ctypes.POINTER(Params)],
    "mmfhe_ctx_create": [ctypes.POINTER(Params), _SZ, _INT, _PP],
    "mmfhe_ctx_destroy": [_VP],
    "mmfhe_sync": [_VP, _VP, _U32],
    "mmfhe_launch_count": [_VP, ctypes.POINTER(_U64)],
    "mmfhe_mem_stats_get": [_VP, ctypes.POINTER(MemStats)],
    "mmfhe_mem_peak_reset": [_VP],
    "mmfhe_debug_fail_allocations": [ctypes.c_int64],
    "mmfhe_trace_enable": [_VP, _INT],
    "mmfhe_trace_get": [_VP, ctypes.c_char_p, _SZ, ctypes.POINTER(_SZ)],
    "mmfhe_profile_enable": [_VP, _INT],
    "mmfhe_profile_get": [_VP, _VP, _U32, ctypes.POINTER(_U32)],
    "mmfhe_measure_butterfly_peak": [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "mmfhe_measure_mac_peak": [_VP, _VP],
    "mmfhe_plan_set_fc_layer": [_VP, _U32, _VP],
    "mmfhe_plan_num_scalars": [_VP, ctypes.POINTER(_U32)],
    "mmfhe_plan_get_scalars": [_VP, _VP, _U32],
    "mmfhe_plan_set_scalars": [_VP, _VP, _U32],
    "mmfhe_train_poly_net": [_VP, _VP, _VP, _U64, _VP, _U32, ctypes.c_float, _U32, _U32, ctypes.c_float, _U64, _VP,
                             ctypes.POINTER(ctypes.c_float)],
    "mmfhe_fold_poly_net": [_VP, _U32, ctypes.c_float, _VP, _U32, _VP],
    "mmfhe_fold_poly_net_wide": [_VP, _U32, ctypes.c_float, _VP, _U32, _VP, _VP],
    "mmfhe_autotune": [_VP, _U32, _U32, _VP],
    "mmfhe_tuning_get": [_VP, _VP],
    "mmfhe_tuning_set": [_VP, _VP],
    "mmfhe_graph_capture": [_VP, _VP, _VP, _VP, _SZ, _VP, _PP],
    "mmfhe_graph_launch": [_VP, _VP],
    "mmfhe_graph_info": [_VP, ctypes.POINTER(_U64), ctypes.POINTER(_U64)],
    "mmfhe_graph_destroy": [_VP],
    "mmfhe_server_create": [_VP, _VP, _SZ, _VP, _PP],
    "mmfhe_server_add_user": [_VP, _U64, _VP, _VP, _VP, _U32],
    "mmfhe_server_set_fc_layer": [_VP, _U32, _VP, _SZ],
    "mmfhe_server_set_const": [_VP, _U32, _U32, _VP, _SZ],
    "mmfhe_ntt32_select_primes": [_U32, _U32, _U32, _VP],
    "mmfhe_ntt_batch": [_VP, _VP, _SZ, _U32, ctypes.c_int, _VP],
    "mmfhe_ntt32_create": [_U32, _VP, _U32, ctypes.c_int, _PP],
    "mmfhe_ntt32_run": [_VP, _VP, _SZ, ctypes.c_int, _VP],
    "mmfhe_ntt32_destroy": [_VP],
    "mmfhe_server_submit": [_VP, _U64, _U32, _VP, _VP, ctypes.POINTER(_U64)],
    "mmfhe_server_wait": [_VP, _U64, _U32, ctypes.POINTER(ctypes.c_double)],
    "mmfhe_server_cancel": [_VP, _U64],
    "mmfhe_server_drain": [_VP, _U32],
    "mmfhe_server_stats_get": [_VP, _VP],
    "mmfhe_server_destroy": [_VP],
    "mmfhe_batcher_create": [_VP, _VP, _SZ, _VP, _PP],
    "mmfhe_batcher_plan": [_VP, _U32, _PP],
    "mmfhe_batcher_submit": [_VP, _VP, _U32, _VP, _VP],
    "mmfhe_batcher_flush": [_VP, _VP],
    "mmfhe_batcher_forget_keys": [_VP, _VP],
    "mmfhe_batcher_stats_get": [_VP, _VP],
    "mmfhe_batcher_destroy": [_VP],
    "mmfhe_keys_create": [_VP, _U64, _PP],
    "mmfhe_keys_set_relin": [_VP, _VP],
    "mmfhe_keys_set_galois": [_VP, _I32, _VP],
    "mmfhe_keys_unload": [_VP],
    "mmfhe_ntt": [_VP, _VP, _VP, _SZ, _INT, _VP],
    "mmfhe_poly_mul": [_VP, _VP, _VP, _VP, _VP, _SZ, _VP],
    "mmfhe_ct_add": [_VP, _VP, _VP, _VP, _SZ, _U32, _VP],
    "mmfhe_ct_mul_plain": [_VP, _VP, _VP, _VP, _SZ, _U32, _VP],
    "mmfhe_ct_mul_relin": [_VP, _VP, _VP, _VP, _VP, _SZ, _U32, _VP],
    "mmfhe_ct_rescale": [_VP, _VP, _VP, _SZ, _U32, _VP],
    "mmfhe_ct_rotate": [_VP, _VP, _VP, _VP, _SZ, _U32, _I32, _VP],
    "mmfhe_ct_rotate_hoisted": [_VP, _VP, _VP, _VP, _SZ, _U32, _VP, _SZ, _VP],
    "mmfhe_modup": [_VP, _VP, _VP, _SZ, _U32, _VP],
    "mmfhe_keyswitch": [_VP, _VP, _INT, _I32, _VP, _VP, _SZ, _U32, _VP],
    "mmfhe_keyswitch_noalloc": [_VP, _VP, _INT, _I32, _VP, _VP, _SZ, _U32, _VP],
    "mmfhe_ct_rotsum": [_VP, _VP, _VP, _VP, _SZ, _U32, _I32, _U32, _VP],
    "mmfhe_ct_bsgs": [_VP, _VP, _VP, _VP, _SZ, _U32, _I32, _U32, _VP, _VP, _SZ, _VP],
    "mmfhe_ct_bsgs_dh": [_VP, _VP, _VP, _VP, _SZ, _U32, _I32, _U32, _U32, _VP, _VP, _VP, _VP, _SZ, _VP],
    "mmfhe_plan_create": [_VP, ctypes.POINTER(CircuitConfig), _SZ, _PP],
    "mmfhe_plan_destroy": [_VP],
    "mmfhe_plan_num_consts": [_VP, ctypes.POINTER(_U32)],
    "mmfhe_plan_const_key": [_VP, _U32, ctypes.POINTER(ConstKey)],
    "mmfhe_plan_set_const": [_VP, _U32, _VP],
    "mmfhe_plan_get_const": [_VP, _U32, _VP],
    "mmfhe_plan_encode_consts": [_VP],
    "mmfhe_plan_rotations": [_VP, _VP, _U32, ctypes.POINTER(_U32)],
    "mmfhe_plan_io": [_VP, ctypes.POINTER(_U32), ctypes.POINTER(_U32), _VP],
    "mmfhe_plan_readout": [_VP, _VP, _VP, _U32, ctypes.POINTER(_U32)],
    "mmfhe_eval": [_VP, _VP, _VP, _VP, _SZ, _VP, _VP],
    "mmfhe_eval_vital": [_VP, _VP, _VP, _VP, _SZ, _VP, _VP],
    "mmfhe_pack_window": [_U32, _U32, _U32, _VP, _VP],
    "mmfhe_params_hash": [ctypes.POINTER(Params), ctypes.POINTER(_U64)],
    "mmfhe_ct_header_make": [ctypes.POINTER(Params), _U32, ctypes.c_double, ctypes.POINTER(CtHeader)],
    "mmfhe_eval_checked": [_VP, _VP, _VP, _VP, _VP, _SZ, _VP, _VP, _VP],
    "mmfhe_keys_blob_write": [ctypes.POINTER(Params), _VP, _U32, _VP, _VP, _VP, _SZ, ctypes.POINTER(_SZ)],
    "mmfhe_plan_blob_write": [ctypes.POINTER(Params), ctypes.POINTER(CircuitConfig), _SZ, _U32, _VP, _VP, _VP, _SZ,
                              ctypes.POINTER(_SZ)],
    "mmfhe_blob_check": [ctypes.POINTER(Params), _VP, _SZ, ctypes.POINTER(_U32)],
    "mmfhe_keys_load": [_VP, _U64, _VP, _SZ, _PP],
    "mmfhe_plan_load": [_VP, _VP, _SZ, _PP],
    "mmfhe_encode": [ctypes.POINTER(Params), _VP, ctypes.c_double, _U32, _VP],
}

_lib = None


def lib():
    """Load libmmfhe.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(SO_PATH):
            raise ImportError("libmmfhe.so not built: run paper_2603_22437_b300/build.py")
        L = ctypes.CDLL(SO_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int32
        L.mmfhe_last_error.argtypes = [_VP]
        L.mmfhe_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def check(status, ctx=None):
    if status != OK:
        msg = lib().mmfhe_last_error(ctx)
        raise MmfheError(status, msg.decode() if msg else "")


def ptr(x):
    """Data pointer of a numpy array or torch tensor (contiguous)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "array must be C-contiguous"
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "tensor must be contiguous"
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError("unsupported buffer type %r" % type(x))


def ptr_array(xs):
    arr = (ctypes.c_void_p * len(xs))()
    for i, x in enumerate(xs):
        arr[i] = ptr(x)
    return arr


def stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)
