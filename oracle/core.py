"""ctypes wrapper of the C oracle (test infrastructure only).

See ``oracle.c`` for what is computed and which passages it follows.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile oracle.c with the host C compiler (plain -O2, no ISA flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            lib.oracle_join.restype = P
            lib.oracle_join.argtypes = [P, P, I64, P, P, I64, P, I64]
            lib.oracle_result_size.restype = I64
            lib.oracle_result_size.argtypes = [P]
            lib.oracle_result_out_j.restype = I64
            lib.oracle_result_out_j.argtypes = [P]
            lib.oracle_result_copy.restype = None
            lib.oracle_result_copy.argtypes = [P, P, P, P]
            lib.oracle_result_free.restype = None
            lib.oracle_result_free.argtypes = [P]
            lib.oracle_rank_map.restype = I64
            lib.oracle_rank_map.argtypes = [P, I64, P, P]
            _lib = lib
    return _lib


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _join(r_key, r_val, s_key, s_val, x_filter=None):
    lib = _load()
    rk, rv, sk, sv = _i32(r_key), _i32(r_val), _i32(s_key), _i32(s_val)
    if rk.size != rv.size or sk.size != sv.size:
        raise ValueError("column lengths differ")
    xf = None if x_filter is None else _i32(x_filter)
    res = lib.oracle_join(_ptr(rk), _ptr(rv), rk.size, _ptr(sk), _ptr(sv), sk.size,
                          None if xf is None else _ptr(xf), 0 if xf is None else xf.size)
    if not res:
        raise MemoryError("oracle_join failed to allocate")
    try:
        n = lib.oracle_result_size(res)
        out_j = lib.oracle_result_out_j(res)
        x = np.empty(n, np.int32)
        z = np.empty(n, np.int32)
        c = np.empty(n, np.int64)
        lib.oracle_result_copy(res, _ptr(x), _ptr(z), _ptr(c))
    finally:
        lib.oracle_result_free(res)
    return x, z, c, int(out_j)


def join_project(r_key, r_val, s_key, s_val, x_filter=None):
    """Pi_{x,z}(R(x,y) join_y S(z,y)) as (out_x, out_z, out_j).

    Pairs are distinct and in canonical order (x, then z, signed int32).
    ``x_filter`` restricts the result to those x values (their rows of the
    full result). ``out_j`` is |OUT_J| of the (restricted) join."""
    x, z, _, out_j = _join(r_key, r_val, s_key, s_val, x_filter)
    return x, z, out_j


def join_count(r_key, r_val, s_key, s_val, x_filter=None):
    """Join-Aggregate COUNT per (x, z): (out_x, out_z, out_cnt, out_j)."""
    return _join(r_key, r_val, s_key, s_val, x_filter)


def rank_map(vals):
    """Order-preserving dense ids: (ids, dict) with dict ascending and
    ids[i] = number of distinct values smaller than vals[i]."""
    lib = _load()
    v = _i32(vals)
    ids = np.empty(v.size, np.int32)
    d = np.empty(v.size, np.int32)
    n = lib.oracle_rank_map(_ptr(v), v.size, _ptr(ids), _ptr(d))
    if n < 0:
        raise MemoryError("oracle_rank_map failed to allocate")
    return ids, d[:n].copy()
