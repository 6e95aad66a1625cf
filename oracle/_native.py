"""ctypes loader for the oracle's C core (test infrastructure only).

The shared object is compiled from ``core.c`` with gcc on first use (or by
``__graft_entry__.build()``) into ``oracle/_build``.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "core.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle_core.so")

_lib = None


def build(force=False):
    """Compile core.c into a shared object (gcc, -O2)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        u64p = ctypes.POINTER(ctypes.c_uint64)
        i64p = ctypes.POINTER(ctypes.c_int64)
        sz, u64, ci = ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int
        sig = {
            "or_vec_add": [u64p, u64p, u64p, sz, u64],
            "or_vec_sub": [u64p, u64p, u64p, sz, u64],
            "or_vec_neg": [u64p, u64p, sz, u64],
            "or_vec_mul": [u64p, u64p, u64p, sz, u64],
            "or_vec_mul_scalar": [u64p, u64p, u64, sz, u64],
            "or_vec_mac_scalar": [u64p, u64p, u64, sz, u64],
            "or_vec_mod": [u64p, u64p, sz, u64],
            "or_vec_mod_signed": [u64p, i64p, sz, u64],
            "or_ntt_fwd": [u64p, ci, u64, u64],
            "or_ntt_inv": [u64p, ci, u64, u64],
            "or_polymul": [u64p, u64p, u64p, ci, u64, u64],
            "or_automorphism": [u64p, u64p, ci, u64, u64],
        }
        for name, args in sig.items():
            f = getattr(_lib, name)
            f.argtypes = args
            f.restype = None
    return _lib


def _p(a):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _u(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def add(a, b, q):
    a, b = _u(a), _u(b)
    out = np.empty_like(a)
    lib().or_vec_add(_p(out), _p(a), _p(b), a.size, int(q))
    return out


def sub(a, b, q):
    a, b = _u(a), _u(b)
    out = np.empty_like(a)
    lib().or_vec_sub(_p(out), _p(a), _p(b), a.size, int(q))
    return out


def neg(a, q):
    a = _u(a)
    out = np.empty_like(a)
    lib().or_vec_neg(_p(out), _p(a), a.size, int(q))
    return out


def mul(a, b, q):
    a, b = _u(a), _u(b)
    out = np.empty_like(a)
    lib().or_vec_mul(_p(out), _p(a), _p(b), a.size, int(q))
    return out


def mul_scalar(a, s, q):
    a = _u(a)
    out = np.empty_like(a)
    lib().or_vec_mul_scalar(_p(out), _p(a), int(s) % (1 << 64), a.size, int(q))
    return out


def mac_scalar(acc, a, s, q):
    """acc <- (acc + a*s) mod q, in place; returns acc."""
    a = _u(a)
    assert acc.dtype == np.uint64 and acc.flags["C_CONTIGUOUS"]
    lib().or_vec_mac_scalar(_p(acc), _p(a), int(s) % (1 << 64), a.size, int(q))
    return acc


def mod(a, q):
    a = _u(a)
    out = np.empty_like(a)
    lib().or_vec_mod(_p(out), _p(a), a.size, int(q))
    return out


def mod_signed(a, q):
    a = np.ascontiguousarray(a, dtype=np.int64)
    out = np.empty(a.shape, dtype=np.uint64)
    lib().or_vec_mod_signed(_p(out), a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), a.size, int(q))
    return out


def ntt_fwd(a, q, psi):
    out = _u(a).copy()
    lib().or_ntt_fwd(_p(out), int(out.size).bit_length() - 1, int(q), int(psi))
    return out


def ntt_inv(a, q, psi):
    out = _u(a).copy()
    lib().or_ntt_inv(_p(out), int(out.size).bit_length() - 1, int(q), int(psi))
    return out


def polymul(a, b, q, psi):
    a, b = _u(a), _u(b)
    out = np.empty_like(a)
    lib().or_polymul(_p(out), _p(a), _p(b), int(a.size).bit_length() - 1, int(q), int(psi))
    return out


def automorphism(a, g, q):
    a = _u(a)
    out = np.empty_like(a)
    lib().or_automorphism(_p(out), _p(a), int(a.size).bit_length() - 1, int(g), int(q))
    return out
