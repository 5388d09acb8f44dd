"""Python binding of libfastpair.so (C ABI in include/fastpair.h).

Argument marshalling only: every step of decoding runs in the library's
CUDA kernels.  The library is compiled in-tree for sm_103a by
:mod:`paper_2609_15034_gb300._build`; if it cannot be built or loaded,
every call raises -- there is no CPU fallback.

Functions keep the C names without the ``fp_`` prefix.  Device buffers are
passed as integer addresses (``tensor.data_ptr()``) or as torch tensors via
the ``*_tensors`` helpers; streams as ``cudaStream_t`` integers
(``torch.cuda.current_stream().cuda_stream``) or ``None`` for the default
stream.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

ONPAIR16, ONPAIR12, FSST8, FSST12 = 1, 2, 3, 4
CODEC_IDS = {"onpair16": ONPAIR16, "onpair12": ONPAIR12, "fsst8": FSST8, "fsst12": FSST12}
CODE_BITS = {ONPAIR16: 16, ONPAIR12: 12, FSST8: 8, FSST12: 12}

OK, ERR_ARG, ERR_CUDA, ERR_NOMEM, ERR_CORRUPT, ERR_CAPACITY, ERR_OVERFLOW, ERR_TIMEOUT, ERR_BUSY, \
    ERR_NOT_READY, ERR_INTERNAL = range(11)
STATUS_NAMES = {0: "FP_OK", 1: "FP_ERR_ARG", 2: "FP_ERR_CUDA", 3: "FP_ERR_NOMEM", 4: "FP_ERR_CORRUPT",
                5: "FP_ERR_CAPACITY", 6: "FP_ERR_OVERFLOW", 7: "FP_ERR_TIMEOUT", 8: "FP_ERR_BUSY",
                9: "FP_ERR_NOT_READY", 10: "FP_ERR_INTERNAL"}

_lock = threading.Lock()
_lib = None


class FastPairError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    from . import _build
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libfastpair.so (building it first if its sources changed)."""
    global _lib
    with _lock:
        if _lib is None:
            from . import _build
            path = _build.build()
            L = ctypes.CDLL(path)
            P, U32, U64, I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
            L.fp_dict_upload.argtypes = [I, P, P, U32, P, ctypes.POINTER(P)]
            L.fp_dict_free.argtypes = [P]
            L.fp_decode.argtypes = [I, P, P, U64, P, U32, P, U64, P, P]
            L.fp_decode_plain.argtypes = [I, P, P, U64, P, U32, P, U64, P, P]
            L.fp_decoded_size.argtypes = [I, P, P, U64, P, U32, P, ctypes.POINTER(U64)]
            L.fp_decode_noalloc.argtypes = [I, P, P, U64, P, U32, P, U64, P, P, P]
            L.fp_sync_status.argtypes = [P]
            L.fp_debug_stall_next.argtypes = [P, U32]
            L.fp_rows_size.argtypes = [I, P, P, U64, P, U32, P, U32, P, ctypes.POINTER(U64), ctypes.POINTER(U64)]
            L.fp_decode_rows.argtypes = [I, P, P, U64, P, U32, P, U32, U64, P, U64, P, P]
            L.fp_decode_packed.argtypes = [I, P, U32, P, U64, P, U32, P, U64, P, P]
            L.fp_tune_column.argtypes = [I, P, P, U64, P, U32, P, U64, P, ctypes.c_char_p, P,
                                         ctypes.POINTER(I), ctypes.POINTER(ctypes.c_float)]
            L.fp_tune_load.argtypes = [ctypes.c_char_p]
            L.fp_decoded_size_packed.argtypes = [I, P, U32, P, U64, P, U32, P, ctypes.POINTER(U64)]
            L.fp_last_error.restype = ctypes.c_char_p
            L.fp_variant_count.argtypes = [I]
            L.fp_variant_info.argtypes = [I, I, ctypes.POINTER(U32), ctypes.POINTER(U32), ctypes.POINTER(U32),
                                          ctypes.POINTER(U32)]
            L.fp_variant_select.argtypes = [I, I]
            L.fp_variant_selected.argtypes = [I]
            L.fp_variant_for.argtypes = [I, U64]
            L.fp_variant_for_dict.argtypes = [P, U64]
            L.fp_variant_width.argtypes = [I, I]
            L.fp_width_for_histogram.argtypes = [P]
            L.fp_dict_set_width.argtypes = [P, I]
            L.fp_dict_width.argtypes = [P]
            L.fp_plan_create.argtypes = [ctypes.POINTER(Chunk), U32, ctypes.c_char_p, P, ctypes.POINTER(P)]
            L.fp_plan_create_config.argtypes = [ctypes.POINTER(Chunk), U32, I, P, ctypes.POINTER(P)]
            L.fp_decode_batch.argtypes = [P, P]
            L.fp_plan_sync_status.argtypes = [P, P, P, P]
            L.fp_plan_info.argtypes = [P, ctypes.POINTER(PlanInfo)]
            L.fp_plan_destroy.argtypes = [P]
            L.fp_batch_config_info.argtypes = [I, P, ctypes.POINTER(U32), ctypes.POINTER(U32)]
            L.fp_serve_create.argtypes = [ctypes.POINTER(ServeConfig), ctypes.POINTER(P)]
            L.fp_serve_dict_put.argtypes = [P, U64, I, P, P, U32]
            L.fp_serve_submit.argtypes = [P, ctypes.POINTER(Request), ctypes.POINTER(U64)]
            L.fp_serve_poll.argtypes = [P, ctypes.POINTER(Result), U32, ctypes.POINTER(U32), ctypes.c_int64]
            L.fp_serve_release.argtypes = [P, U64]
            L.fp_serve_stats.argtypes = [P, ctypes.POINTER(ServeStats)]
            L.fp_serve_destroy.argtypes = [P]
            L.fp_sidecar_tile_slots.argtypes = [I]
            L.fp_sidecar_tile_slots.restype = U32
            L.fp_sidecar_entries.argtypes = [I, U64]
            L.fp_sidecar_entries.restype = U64
            L.fp_sidecar_scratch_bytes.argtypes = [I, U64]
            L.fp_sidecar_scratch_bytes.restype = U64
            L.fp_sidecar_build.argtypes = [I, P, P, U64, P, U32, P, U64, P, U64, P, P]
            L.fp_decode_sidecar.argtypes = [I, P, P, U64, P, U32, P, U64, P, U64, P, P, U64, P, P]
            for name in ("fp_dict_upload", "fp_dict_free", "fp_decode", "fp_decode_plain", "fp_decoded_size",
                         "fp_decode_noalloc",
                         "fp_sync_status", "fp_debug_stall_next", "fp_variant_info", "fp_variant_select",
                         "fp_dict_set_width", "fp_rows_size", "fp_decode_rows", "fp_decode_packed",
                         "fp_decoded_size_packed", "fp_tune_column", "fp_tune_load", "fp_tune_clear",
                         "fp_plan_create", "fp_plan_create_config", "fp_decode_batch", "fp_plan_sync_status",
                         "fp_plan_info", "fp_plan_destroy", "fp_batch_config_info", "fp_serve_create",
                         "fp_serve_dict_put", "fp_serve_submit", "fp_serve_poll", "fp_serve_release",
                         "fp_serve_stats", "fp_serve_destroy", "fp_sidecar_build", "fp_decode_sidecar"):
                getattr(L, name).restype = I
            _lib = L
            # the committed tuning table of this library's shapes (defaults per
            # GPU model and column size; unused on another SM count)
            import os
            table = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning", "gb300.txt")
            if os.path.exists(table):
                L.fp_tune_load(table.encode())
    return _lib


def last_error() -> str:
    return lib().fp_last_error().decode()


def _check(st: int, where: str) -> int:
    if st != OK:
        raise FastPairError(st, where, last_error())
    return st


def _stream(s) -> ctypes.c_void_p:
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        s = s.cuda_stream
    return ctypes.c_void_p(int(s))


class Chunk(ctypes.Structure):
    """fp_chunk: one column of a batch (device addresses as integers)."""
    _fields_ = [("codec", ctypes.c_int), ("dict", ctypes.c_void_p), ("d_codes", ctypes.c_void_p),
                ("codes_bytes", ctypes.c_uint64), ("d_code_offsets", ctypes.c_void_p),
                ("n_strings", ctypes.c_uint32), ("d_out_bytes", ctypes.c_void_p),
                ("out_capacity", ctypes.c_uint64), ("d_out_offsets", ctypes.c_void_p)]


class PlanInfo(ctypes.Structure):
    """fp_plan_info_t."""
    _fields_ = [("config", ctypes.c_uint32), ("n_configs", ctypes.c_uint32),
                ("slots_per_thread", ctypes.c_uint32 * 3), ("threads", ctypes.c_uint32),
                ("grid", ctypes.c_uint32), ("index_blocks", ctypes.c_uint32), ("from_cache", ctypes.c_uint32),
                ("slots_per_thread_fsst12", ctypes.c_uint32), ("total_tiles", ctypes.c_uint64),
                ("layout_bytes", ctypes.c_uint64),
                ("tune_ms", ctypes.c_float * 8)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("dict_cache_slots", ctypes.c_uint32),
                ("max_inflight", ctypes.c_uint32), ("n_streams", ctypes.c_uint32), ("max_wave", ctypes.c_uint32),
                ("batch_config", ctypes.c_int32), ("reserved", ctypes.c_uint32)]


class Request(ctypes.Structure):
    _fields_ = [("dict_key", ctypes.c_uint64), ("d_codes", ctypes.c_void_p), ("codes_bytes", ctypes.c_uint64),
                ("d_code_offsets", ctypes.c_void_p), ("n_strings", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("decoded_size", ctypes.c_uint64), ("user_tag", ctypes.c_uint64)]


class Result(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("d_out_bytes", ctypes.c_void_p), ("d_out_offsets", ctypes.c_void_p), ("bytes", ctypes.c_uint64),
                ("n_strings", ctypes.c_uint64), ("t_submit_ns", ctypes.c_int64), ("t_admit_ns", ctypes.c_int64),
                ("t_done_ns", ctypes.c_int64), ("user_tag", ctypes.c_uint64)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("released", ctypes.c_uint64), ("waves", ctypes.c_uint64),
                ("max_wave_seen", ctypes.c_uint32), ("queued", ctypes.c_uint32), ("bytes_decoded", ctypes.c_uint64),
                ("dict_hits", ctypes.c_uint64), ("dict_misses", ctypes.c_uint64), ("dict_evictions", ctypes.c_uint64),
                ("dicts_registered", ctypes.c_uint64), ("inflight_bytes", ctypes.c_uint64),
                ("peak_inflight_bytes", ctypes.c_uint64), ("inflight_requests", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class Dict:
    """A device-resident dictionary (fp_dict*)."""

    def __init__(self, codec: int, data: np.ndarray, offsets: np.ndarray, stream=None):
        data = np.ascontiguousarray(data, np.uint8)
        offsets = np.ascontiguousarray(offsets, np.uint32)
        if data.size == 0:
            data = np.zeros(1, np.uint8)
        h = ctypes.c_void_p()
        _check(lib().fp_dict_upload(codec, data.ctypes.data, offsets.ctypes.data, offsets.size - 1,
                                    _stream(stream), ctypes.byref(h)), "fp_dict_upload")
        self.codec = codec
        self.n_entries = offsets.size - 1
        self._h = h

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise ValueError("dictionary was freed")
        return self._h

    @property
    def width(self) -> int:
        """Dictionary read width fp_decode uses (8: split read, 16: whole entries)."""
        return lib().fp_dict_width(self.handle)

    def set_width(self, width: int, check: bool = True) -> int:
        st = lib().fp_dict_set_width(self.handle, int(width))
        return _check(st, "fp_dict_set_width") if check else st

    def free(self):
        if self._h is not None and _lib is not None:
            _lib.fp_dict_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def dict_upload(codec: int, data, offsets, stream=None) -> Dict:
    return Dict(codec, data, offsets, stream)


def decode(codec, d: Dict, codes_ptr: int, codes_bytes: int, code_offsets_ptr: int, n_strings: int,
           out_ptr: int, capacity: int, out_offsets_ptr: int, stream=None, check: bool = True) -> int:
    st = lib().fp_decode(codec, d.handle, codes_ptr, codes_bytes, code_offsets_ptr, n_strings, out_ptr,
                         capacity, out_offsets_ptr, _stream(stream))
    return _check(st, "fp_decode") if check else st


def decode_plain(codec, d: Dict, codes_ptr: int, codes_bytes: int, code_offsets_ptr: int, n_strings: int,
                 out_ptr: int, capacity: int, out_offsets_ptr: int, stream=None, check: bool = True) -> int:
    st = lib().fp_decode_plain(codec, d.handle, codes_ptr, codes_bytes, code_offsets_ptr, n_strings, out_ptr,
                               capacity, out_offsets_ptr, _stream(stream))
    return _check(st, "fp_decode_plain") if check else st


def decode_noalloc(codec, d: Dict, codes_ptr: int, codes_bytes: int, code_offsets_ptr: int, n_strings: int,
                   out_ptr: int, capacity: int, out_offsets_ptr: int, status_ptr: int, stream=None,
                   check: bool = True) -> int:
    """fp_decode_noalloc: decode with the library's fixed scratch (no device
    allocation); the call's data-error bits land in the uint32 at status_ptr."""
    st = lib().fp_decode_noalloc(codec, d.handle, codes_ptr, codes_bytes, code_offsets_ptr, n_strings, out_ptr,
                                 capacity, out_offsets_ptr, status_ptr, _stream(stream))
    return _check(st, "fp_decode_noalloc") if check else st


# ---- stored sidecar (fastpair_sidecar.h) -----------------------------------

def sidecar_tile_slots(codec: int) -> int:
    return lib().fp_sidecar_tile_slots(codec)


def sidecar_entries(codec: int, codes_bytes: int) -> int:
    return lib().fp_sidecar_entries(codec, codes_bytes)


def sidecar_scratch_bytes(codec: int, codes_bytes: int) -> int:
    return lib().fp_sidecar_scratch_bytes(codec, codes_bytes)


def sidecar_build(codec, d: Dict, codes_ptr: int, codes_bytes: int, code_offsets_ptr: int, n_strings: int,
                  sidecar_ptr: int, sidecar_entries: int, scratch_ptr: int, scratch_bytes: int, status_ptr: int,
                  stream=None, check: bool = True) -> int:
    """fp_sidecar_build: the column's stored table of tile output offsets."""
    st = lib().fp_sidecar_build(codec, d.handle, codes_ptr, codes_bytes, code_offsets_ptr, n_strings, sidecar_ptr,
                                sidecar_entries, scratch_ptr, scratch_bytes, status_ptr, _stream(stream))
    return _check(st, "fp_sidecar_build") if check else st


def decode_sidecar(codec, d: Dict, codes_ptr: int, codes_bytes: int, code_offsets_ptr: int, n_strings: int,
                   sidecar_ptr: int, sidecar_entries: int, out_ptr: int, capacity: int, out_offsets_ptr: int,
                   scratch_ptr: int, scratch_bytes: int, status_ptr: int, stream=None, check: bool = True) -> int:
    """fp_decode_sidecar: decode from a stored sidecar (no reduce, no tile scan)."""
    st = lib().fp_decode_sidecar(codec, d.handle, codes_ptr, codes_bytes, code_offsets_ptr, n_strings, sidecar_ptr,
                                 sidecar_entries, out_ptr, capacity, out_offsets_ptr, scratch_ptr, scratch_bytes,
                                 status_ptr, _stream(stream))
    return _check(st, "fp_decode_sidecar") if check else st


class SidecarColumn:
    """Device buffers for the stored-sidecar calls of one code buffer: the
    sidecar (uint64 entries), the scratch and the status word, allocated
    with torch.  `codes` is a uint8 CUDA tensor, `code_offsets` an int32 one."""

    def __init__(self, codec: int, d: Dict, codes, code_offsets, n_strings: int, codes_bytes: int | None = None):
        import torch
        self.codec, self.d, self.codes, self.code_offsets, self.n_strings = codec, d, codes, code_offsets, n_strings
        self.codes_bytes = codes.numel() * codes.element_size() if codes_bytes is None else codes_bytes
        self.entries = sidecar_entries(codec, self.codes_bytes)
        self.sidecar = torch.zeros(self.entries, dtype=torch.int64, device=codes.device)
        self.scratch_bytes = sidecar_scratch_bytes(codec, self.codes_bytes)
        self.scratch = torch.empty(self.scratch_bytes, dtype=torch.uint8, device=codes.device)
        self.status = torch.zeros(1, dtype=torch.int32, device=codes.device)

    def build(self, stream=None, check: bool = True) -> int:
        return sidecar_build(self.codec, self.d, self.codes.data_ptr(), self.codes_bytes,
                             self.code_offsets.data_ptr(), self.n_strings, self.sidecar.data_ptr(), self.entries,
                             self.scratch.data_ptr(), self.scratch_bytes, self.status.data_ptr(), stream, check)

    def decode(self, out, out_offsets, stream=None, check: bool = True, sidecar=None) -> int:
        """Decode into torch tensors from this column's sidecar (or another
        uint64 table of at least `entries` entries)."""
        sc = self.sidecar if sidecar is None else sidecar
        if sc.numel() < self.entries:
            raise ValueError("sidecar table too short")
        return decode_sidecar(self.codec, self.d, self.codes.data_ptr(), self.codes_bytes,
                              self.code_offsets.data_ptr(), self.n_strings, sc.data_ptr(), self.entries,
                              out.data_ptr() if out.numel() else 0, out.numel() * out.element_size(),
                              out_offsets.data_ptr(), self.scratch.data_ptr(), self.scratch_bytes,
                              self.status.data_ptr(), stream, check)

    def status_bits(self) -> int:
        """The last call's data-error bits (synchronises with the device)."""
        return int(self.status.cpu().numpy().view(np.uint32)[0])


def decoded_size(codec, d: Dict, codes_ptr: int, codes_bytes: int, code_offsets_ptr: int, n_strings: int,
                 stream=None) -> tuple[int, int]:
    """Returns (status, total bytes)."""
    tot = ctypes.c_uint64(0)
    st = lib().fp_decoded_size(codec, d.handle, codes_ptr, codes_bytes, code_offsets_ptr, n_strings,
                               _stream(stream), ctypes.byref(tot))
    return st, int(tot.value)


def sync_status(stream=None) -> int:
    return lib().fp_sync_status(_stream(stream))


def rows_size(codec, d: Dict, codes_ptr: int, codes_bytes: int, code_offsets_ptr: int, n_strings: int,
              row_ids_ptr: int, n_rows: int, stream=None):
    """fp_rows_size: (status, selected code slots, decoded bytes) of the
    rows row_ids[0 .. n_rows).  Synchronous."""
    slots, nbytes = ctypes.c_uint64(0), ctypes.c_uint64(0)
    st = lib().fp_rows_size(codec, d.handle, codes_ptr, codes_bytes, code_offsets_ptr, n_strings, row_ids_ptr,
                            n_rows, _stream(stream), ctypes.byref(slots), ctypes.byref(nbytes))
    return st, int(slots.value), int(nbytes.value)


def decode_rows(codec, d: Dict, codes_ptr: int, codes_bytes: int, code_offsets_ptr: int, n_strings: int,
                row_ids_ptr: int, n_rows: int, selected_slots: int, out_ptr: int, capacity: int, out_offsets_ptr: int,
                stream=None, check: bool = True) -> int:
    """fp_decode_rows: decode the strings row_ids[0 .. n_rows) in that order."""
    st = lib().fp_decode_rows(codec, d.handle, codes_ptr, codes_bytes, code_offsets_ptr, n_strings, row_ids_ptr,
                              n_rows, selected_slots, out_ptr, capacity, out_offsets_ptr, _stream(stream))
    return _check(st, "fp_decode_rows") if check else st


def decode_packed(codec, d: Dict, code_bits: int, codes_ptr: int, codes_bytes: int, code_offsets_ptr: int,
                  n_strings: int, out_ptr: int, capacity: int, out_offsets_ptr: int, stream=None,
                  check: bool = True) -> int:
    """fp_decode_packed: decode a column whose codes are bit-packed at code_bits bits."""
    st = lib().fp_decode_packed(codec, d.handle, code_bits, codes_ptr, codes_bytes, code_offsets_ptr, n_strings,
                                out_ptr, capacity, out_offsets_ptr, _stream(stream))
    return _check(st, "fp_decode_packed") if check else st


def decoded_size_packed(codec, d: Dict, code_bits: int, codes_ptr: int, codes_bytes: int, code_offsets_ptr: int,
                        n_strings: int, stream=None):
    """fp_decoded_size_packed: (status, decoded bytes).  Synchronous."""
    tot = ctypes.c_uint64(0)
    st = lib().fp_decoded_size_packed(codec, d.handle, code_bits, codes_ptr, codes_bytes, code_offsets_ptr,
                                      n_strings, _stream(stream), ctypes.byref(tot))
    return st, int(tot.value)


def debug_stall_next(spin_limit: int, stream=None) -> int:
    """fp_debug_stall_next: the next decode on ``stream`` gives up a
    look-back after ``spin_limit`` polls (failure-detection test hook)."""
    return lib().fp_debug_stall_next(_stream(stream), int(spin_limit))


def variant_count(codec: int) -> int:
    return lib().fp_variant_count(codec)


def variant_info(codec: int, v: int) -> dict:
    t, k, s, n = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().fp_variant_info(codec, v, ctypes.byref(t), ctypes.byref(k), ctypes.byref(s), ctypes.byref(n)),
           "fp_variant_info")
    return {"threads": t.value, "slots_per_thread": k.value, "dict_in_smem": bool(s.value),
            "warp_tiles": n.value == 3, "launches_per_call": n.value}


def variant_select(codec: int, v: int) -> None:
    _check(lib().fp_variant_select(codec, v), "fp_variant_select")


def variant_selected(codec: int) -> int:
    return lib().fp_variant_selected(codec)


def variant_for(codec: int, codes_bytes: int) -> int:
    """The variant fp_decode uses for a code buffer of codes_bytes bytes
    (with a dictionary of read width 8)."""
    return lib().fp_variant_for(codec, codes_bytes)


def variant_for_dict(d: Dict, codes_bytes: int) -> int:
    """The variant fp_decode uses with dictionary ``d`` for a code buffer of
    codes_bytes bytes."""
    return lib().fp_variant_for_dict(d.handle, codes_bytes)


def tune_column(codec, d: Dict, codes_ptr: int, codes_bytes: int, code_offsets_ptr: int, n_strings: int,
                out_ptr: int, capacity: int, out_offsets_ptr: int, table_path: str | None = None, stream=None):
    """fp_tune_column: (status, chosen variant, its ms)."""
    v, ms = ctypes.c_int(-1), ctypes.c_float(0.0)
    st = lib().fp_tune_column(codec, d.handle, codes_ptr, codes_bytes, code_offsets_ptr, n_strings, out_ptr, capacity,
                              out_offsets_ptr, table_path.encode() if table_path else None, _stream(stream),
                              ctypes.byref(v), ctypes.byref(ms))
    return st, v.value, ms.value


def tune_load(table_path: str) -> int:
    return _check(lib().fp_tune_load(table_path.encode()), "fp_tune_load")


def tune_clear() -> int:
    return lib().fp_tune_clear()


def variant_width(codec: int, v: int) -> int:
    return lib().fp_variant_width(codec, v)


def width_for_histogram(hist) -> int:
    """The paper's split-read rule on a token-length histogram (17 counts,
    lengths 0..16): 16 when more than 60 % of the tokens exceed 8 bytes."""
    h = np.zeros(17, np.uint64)
    a = np.asarray(hist, np.uint64)
    h[:min(17, a.size)] = a[:17]
    return lib().fp_width_for_histogram(h.ctypes.data)


# ---- torch conveniences (tensors are only carriers of device memory) -------

def decode_tensors(codec, d: Dict, codes, code_offsets, n_strings: int, out, out_offsets, stream=None,
                   plain: bool = False, check: bool = True) -> int:
    """Decode with torch tensors as buffers (uint8 codes/out, int32 offsets)."""
    fn = decode_plain if plain else decode
    return fn(codec, d, codes.data_ptr(), codes.numel() * codes.element_size(), code_offsets.data_ptr(),
              n_strings, out.data_ptr() if out.numel() else 0, out.numel() * out.element_size(),
              out_offsets.data_ptr(), stream, check)


def decoded_size_tensors(codec, d: Dict, codes, code_offsets, n_strings: int, stream=None) -> tuple[int, int]:
    return decoded_size(codec, d, codes.data_ptr(), codes.numel() * codes.element_size(),
                        code_offsets.data_ptr(), n_strings, stream)


# ---- batched decode (fp_plan_*) ----------------------------------------------

def chunk(codec, d: Dict, codes_ptr: int, codes_bytes: int, code_offsets_ptr: int, n_strings: int,
          out_ptr: int, capacity: int, out_offsets_ptr: int) -> Chunk:
    return Chunk(codec, d.handle.value, codes_ptr, codes_bytes, code_offsets_ptr, n_strings, out_ptr or None,
                 capacity, out_offsets_ptr)


def chunk_tensors(codec, d: Dict, codes, code_offsets, n_strings: int, out, out_offsets) -> Chunk:
    """fp_chunk from torch tensors (uint8 codes/out, int32 offsets)."""
    return chunk(codec, d, codes.data_ptr(), codes.numel() * codes.element_size(), code_offsets.data_ptr(),
                 n_strings, out.data_ptr() if out.numel() else 0, out.numel() * out.element_size(),
                 out_offsets.data_ptr())


class Plan:
    """fp_plan: a batch of chunks decoded by one graph launch.

    ``config=None`` tunes (optionally remembering the choice in
    ``tune_cache``); an integer fixes the configuration."""

    def __init__(self, chunks, tune_cache: str | None = None, config: int | None = None, stream=None):
        arr = (Chunk * len(chunks))(*chunks)
        self._keep = (arr, list(chunks))
        self.n_chunks = len(chunks)
        h = ctypes.c_void_p()
        if config is None:
            path = tune_cache.encode() if tune_cache else None
            _check(lib().fp_plan_create(arr, len(chunks), path, _stream(stream), ctypes.byref(h)), "fp_plan_create")
        else:
            _check(lib().fp_plan_create_config(arr, len(chunks), int(config), _stream(stream), ctypes.byref(h)),
                   "fp_plan_create_config")
        self._h = h

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise ValueError("plan was destroyed")
        return self._h

    def decode(self, stream=None, check: bool = True) -> int:
        st = lib().fp_decode_batch(self.handle, _stream(stream))
        return _check(st, "fp_decode_batch") if check else st

    def sync_status(self, stream=None):
        """Returns (status, per-chunk status array, per-chunk decoded sizes)."""
        sts = np.zeros(self.n_chunks, np.uint32)
        tot = np.zeros(self.n_chunks, np.uint64)
        st = lib().fp_plan_sync_status(self.handle, _stream(stream), sts.ctypes.data, tot.ctypes.data)
        return st, sts, tot

    def info(self) -> dict:
        pi = PlanInfo()
        _check(lib().fp_plan_info(self.handle, ctypes.byref(pi)), "fp_plan_info")
        return {"config": pi.config, "n_configs": pi.n_configs, "slots_per_thread": list(pi.slots_per_thread),
                "slots_per_thread_fsst12": pi.slots_per_thread_fsst12,
                "threads": pi.threads, "grid": pi.grid, "index_blocks": pi.index_blocks,
                "from_cache": bool(pi.from_cache), "total_tiles": pi.total_tiles, "layout_bytes": pi.layout_bytes,
                "tune_ms": [round(float(x), 4) for x in list(pi.tune_ms)[:pi.n_configs]]}

    def destroy(self):
        if self._h is not None and _lib is not None:
            _lib.fp_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def batch_config_count() -> int:
    return lib().fp_batch_config_count()


def batch_config_info(config: int) -> dict:
    k = (ctypes.c_uint32 * 3)()
    b, w = ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().fp_batch_config_info(config, ctypes.cast(k, ctypes.c_void_p), ctypes.byref(b), ctypes.byref(w)),
           "fp_batch_config_info")
    return {"slots_per_thread": list(k), "blocks_per_sm": b.value, "warp_tiles": bool(w.value)}


# ---- served decode (fp_serve_*) ----------------------------------------------

class Server:
    """fp_server: continuous-batching decode loop run by a library thread."""

    def __init__(self, hbm_budget: int, dict_cache_slots: int = 512, max_inflight: int = 4096, n_streams: int = 4,
                 max_wave: int = 256, batch_config: int = -1):
        cfg = ServeConfig(hbm_budget, dict_cache_slots, max_inflight, n_streams, max_wave, batch_config, 0)
        h = ctypes.c_void_p()
        _check(lib().fp_serve_create(ctypes.byref(cfg), ctypes.byref(h)), "fp_serve_create")
        self._h = h
        self._res = (Result * 1024)()

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise ValueError("server was destroyed")
        return self._h

    def dict_put(self, key: int, codec: int, data: np.ndarray, offsets: np.ndarray) -> None:
        data = np.ascontiguousarray(data, np.uint8)
        offsets = np.ascontiguousarray(offsets, np.uint32)
        if data.size == 0:
            data = np.zeros(1, np.uint8)
        _check(lib().fp_serve_dict_put(self.handle, key, codec, data.ctypes.data, offsets.ctypes.data,
                                       offsets.size - 1), "fp_serve_dict_put")

    def submit(self, dict_key: int, codes_ptr: int, codes_bytes: int, code_offsets_ptr: int, n_strings: int,
               decoded_size: int, user_tag: int = 0, check: bool = True):
        r = Request(dict_key, codes_ptr or None, codes_bytes, code_offsets_ptr, n_strings, 0, decoded_size, user_tag)
        t = ctypes.c_uint64()
        st = lib().fp_serve_submit(self.handle, ctypes.byref(r), ctypes.byref(t))
        if check:
            _check(st, "fp_serve_submit")
            return int(t.value)
        return st, int(t.value)

    def poll(self, max_results: int = 1024, timeout_s: float = 0.0) -> list:
        n = ctypes.c_uint32()
        m = min(max_results, len(self._res))
        _check(lib().fp_serve_poll(self.handle, self._res, m, ctypes.byref(n), int(timeout_s * 1e9)), "fp_serve_poll")
        out = []
        for i in range(n.value):
            r = self._res[i]
            out.append({"ticket": r.ticket, "status": r.status, "d_out_bytes": r.d_out_bytes or 0,
                        "d_out_offsets": r.d_out_offsets or 0, "bytes": r.bytes, "n_strings": r.n_strings,
                        "t_submit_ns": r.t_submit_ns, "t_admit_ns": r.t_admit_ns, "t_done_ns": r.t_done_ns,
                        "user_tag": r.user_tag})
        return out

    def release(self, ticket: int, check: bool = True) -> int:
        st = lib().fp_serve_release(self.handle, ticket)
        return _check(st, "fp_serve_release") if check else st

    def stats(self) -> dict:
        s = ServeStats()
        _check(lib().fp_serve_stats(self.handle, ctypes.byref(s)), "fp_serve_stats")
        return {name: getattr(s, name) for name, _ in ServeStats._fields_ if name != "reserved"}

    def destroy(self):
        if self._h is not None and _lib is not None:
            _lib.fp_serve_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def device_bytes(ptr: int, n: int):
    """A torch uint8 view of n bytes of device memory the library owns (for
    copying a served result out).  Only valid until the result is released."""
    import torch
    if n == 0:
        return torch.empty(0, dtype=torch.uint8, device="cuda")
    return _DeviceView(ptr, n).tensor()


class _DeviceView:
    def __init__(self, ptr: int, n: int):
        self.ptr, self.n = ptr, n

    def tensor(self):
        import torch
        self.__cuda_array_interface__ = {"shape": (self.n,), "typestr": "|u1", "data": (self.ptr, False),
                                         "version": 3, "strides": None}
        return torch.as_tensor(self, device="cuda")
