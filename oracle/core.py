"""ctypes binding of the plain C oracle decoder (test infrastructure only)."""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fp_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_CORRUPT, ERR_CAPACITY, ERR_OVERFLOW = 0, 1, 4, 5, 6
BIT_CORRUPT, BIT_CAPACITY, BIT_OVERFLOW = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no vendor code involved)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P, U8, U32, U64, I = (ctypes.c_void_p, ctypes.c_uint8, ctypes.c_uint32,
                                  ctypes.c_uint64, ctypes.c_int)
            lib.fpo_decode.argtypes = [I, P, P, U32, P, U64, P, U32, P, U64, P, P, P]
            lib.fpo_decode.restype = I
            lib.fpo_decode_mt.argtypes = [I, P, P, U32, P, U64, P, U32, P, U64, P, P, P, I]
            lib.fpo_decode_mt.restype = I
            lib.fpo_unpack12.argtypes = [P, U64, P]
            lib.fpo_unpack12.restype = None
            lib.fpo_sidecar.argtypes = [I, P, P, U32, P, U64, P, U32, U32, P, U64]
            lib.fpo_sidecar.restype = U64
            lib.fpo_decode_rows.argtypes = [I, P, P, U32, P, U64, P, U32, P, U32, P, U64, P, P, P]
            lib.fpo_decode_rows.restype = I
            lib.fpo_decode_packed.argtypes = [I, I, P, P, U32, P, U64, P, U32, P, U64, P, P, P]
            lib.fpo_decode_packed.restype = I
            _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclasses.dataclass
class OracleResult:
    status: int
    err_bits: int
    total: int
    data: np.ndarray | None
    offsets: np.ndarray | None


def _args(codec, dict_data, dict_offsets, stream, code_offsets):
    dd = np.ascontiguousarray(dict_data, np.uint8)
    do = np.ascontiguousarray(dict_offsets, np.uint32)
    st = np.ascontiguousarray(stream, np.uint8)
    co = np.ascontiguousarray(code_offsets, np.uint32)
    if dd.size == 0:
        dd = np.zeros(1, np.uint8)
    if st.size == 0:
        st = np.zeros(1, np.uint8)
        st_bytes = 0
    else:
        st_bytes = int(np.asarray(stream).size)
    return dd, do, st, st_bytes, co


def decode(codec: int, dict_data, dict_offsets, stream, code_offsets,
           capacity: int | None = None, threads: int = 1) -> OracleResult:
    """Decode a column.  ``capacity=None`` sizes the output exactly."""
    lib = _load()
    dd, do, st, st_bytes, co = _args(codec, dict_data, dict_offsets, stream, code_offsets)
    n_strings = co.size - 1
    total = ctypes.c_uint64(0)
    err = ctypes.c_uint(0)
    if capacity is None:
        r = lib.fpo_decode(codec, _ptr(dd), _ptr(do), do.size - 1, _ptr(st), st_bytes,
                           _ptr(co), n_strings, None, 0, None, ctypes.byref(total), ctypes.byref(err))
        if r not in (OK, ERR_OVERFLOW):
            return OracleResult(r, err.value, total.value, None, None)
        capacity = total.value
    out = np.zeros(max(capacity, 1), np.uint8)
    offs = np.zeros(n_strings + 1, np.uint32)
    if threads > 1:
        r = lib.fpo_decode_mt(codec, _ptr(dd), _ptr(do), do.size - 1, _ptr(st), st_bytes,
                              _ptr(co), n_strings, _ptr(out), capacity, _ptr(offs),
                              ctypes.byref(total), ctypes.byref(err), threads)
    else:
        r = lib.fpo_decode(codec, _ptr(dd), _ptr(do), do.size - 1, _ptr(st), st_bytes,
                           _ptr(co), n_strings, _ptr(out), capacity, _ptr(offs),
                           ctypes.byref(total), ctypes.byref(err))
    return OracleResult(r, err.value, total.value, out[:min(total.value, capacity)], offs)


def decode_mt(codec, dict_data, dict_offsets, stream, code_offsets, threads: int,
              capacity: int | None = None) -> OracleResult:
    return decode(codec, dict_data, dict_offsets, stream, code_offsets, capacity, threads=max(2, threads))


def decoded_size(codec, dict_data, dict_offsets, stream, code_offsets) -> tuple[int, int]:
    lib = _load()
    dd, do, st, st_bytes, co = _args(codec, dict_data, dict_offsets, stream, code_offsets)
    total = ctypes.c_uint64(0)
    err = ctypes.c_uint(0)
    r = lib.fpo_decode(codec, _ptr(dd), _ptr(do), do.size - 1, _ptr(st), st_bytes,
                       _ptr(co), co.size - 1, None, 0, None, ctypes.byref(total), ctypes.byref(err))
    return r, int(total.value)


def sidecar(codec: int, dict_data, dict_offsets, stream, code_offsets, tile: int) -> np.ndarray | None:
    """The column's stored sidecar for tiles of ``tile`` slots (entry 0 the
    decoded size, then one entry per tile); None for an invalid column."""
    lib = _load()
    dd, do, st, st_bytes, co = _args(codec, dict_data, dict_offsets, stream, code_offsets)
    n_slots = st_bytes * 8 // {1: 16, 2: 12, 3: 8, 4: 12}[codec]
    cap = n_slots // tile + 3
    out = np.zeros(cap, np.uint64)
    t = lib.fpo_sidecar(codec, _ptr(dd), _ptr(do), do.size - 1, _ptr(st), st_bytes, _ptr(co), co.size - 1,
                        tile, _ptr(out), cap)
    return None if t == 0 else out[:1 + t]


def decode_rows(codec: int, dict_data, dict_offsets, stream, code_offsets, row_ids,
                capacity: int | None = None) -> OracleResult:
    """Decode the strings row_ids (in that order) of a column."""
    lib = _load()
    dd, do, st, st_bytes, co = _args(codec, dict_data, dict_offsets, stream, code_offsets)
    rows = np.ascontiguousarray(row_ids, np.uint32)
    m = int(rows.size)
    rp = _ptr(rows if m else np.zeros(1, np.uint32))
    total = ctypes.c_uint64(0)
    err = ctypes.c_uint(0)
    if capacity is None:
        r = lib.fpo_decode_rows(codec, _ptr(dd), _ptr(do), do.size - 1, _ptr(st), st_bytes, _ptr(co), co.size - 1,
                                rp, m, None, 0, None, ctypes.byref(total), ctypes.byref(err))
        if r not in (OK, ERR_OVERFLOW):
            return OracleResult(r, err.value, total.value, None, None)
        capacity = total.value
    out = np.zeros(max(capacity, 1), np.uint8)
    offs = np.zeros(m + 1, np.uint32)
    r = lib.fpo_decode_rows(codec, _ptr(dd), _ptr(do), do.size - 1, _ptr(st), st_bytes, _ptr(co), co.size - 1,
                            rp, m, _ptr(out), capacity, _ptr(offs), ctypes.byref(total), ctypes.byref(err))
    return OracleResult(r, err.value, total.value, out[:min(total.value, capacity)], offs)


def decode_packed(codec: int, bits: int, dict_data, dict_offsets, stream, code_offsets,
                  capacity: int | None = None) -> OracleResult:
    """Decode a column whose codes are bit-packed at ``bits`` bits per code
    (LSB-first), for the escape-free codecs."""
    lib = _load()
    dd, do, st, st_bytes, co = _args(codec, dict_data, dict_offsets, stream, code_offsets)
    n_strings = co.size - 1
    total = ctypes.c_uint64(0)
    err = ctypes.c_uint(0)
    if capacity is None:
        r = lib.fpo_decode_packed(codec, bits, _ptr(dd), _ptr(do), do.size - 1, _ptr(st), st_bytes, _ptr(co),
                                  n_strings, None, 0, None, ctypes.byref(total), ctypes.byref(err))
        if r not in (OK, ERR_OVERFLOW):
            return OracleResult(r, err.value, total.value, None, None)
        capacity = total.value
    out = np.zeros(max(capacity, 1), np.uint8)
    offs = np.zeros(n_strings + 1, np.uint32)
    r = lib.fpo_decode_packed(codec, bits, _ptr(dd), _ptr(do), do.size - 1, _ptr(st), st_bytes, _ptr(co), n_strings,
                              _ptr(out), capacity, _ptr(offs), ctypes.byref(total), ctypes.byref(err))
    return OracleResult(r, err.value, total.value, out[:min(total.value, capacity)], offs)


def unpack12(stream, n: int) -> np.ndarray:
    lib = _load()
    st = np.ascontiguousarray(stream, np.uint8)
    out = np.zeros(max(n, 1), np.uint16)
    lib.fpo_unpack12(_ptr(st), n, _ptr(out))
    return out[:n]


def decode_column(col, capacity=None, threads: int = 1) -> OracleResult:
    """Convenience: decode a :class:`synth.Column`."""
    return decode(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream,
                  col.code_offsets, capacity, threads)
