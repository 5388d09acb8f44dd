"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
the CPU oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle
import synth

GUARD = 0xA5
GUARD_BYTES = 64


def store_slots(codec: int, slots) -> np.ndarray:
    slots = np.asarray(slots, np.uint16)
    if codec == synth.ONPAIR16:
        return synth.pack16(slots)
    if codec in (synth.ONPAIR12, synth.FSST12):
        return synth.pack12(slots)
    return slots.astype(np.uint8)


def make_column(codec: int, tokens, slots, code_offsets, name="") -> synth.Column:
    d = synth.Dictionary.from_tokens(codec, tokens)
    stream = store_slots(codec, slots)
    return synth.Column(codec, d, stream, np.asarray(code_offsets, np.uint32), len(slots), name=name)


class DeviceColumn:
    """A column's inputs resident on the GPU (torch used as an allocator)."""

    def __init__(self, col: synth.Column, stream=None):
        import torch
        import paper_2609_15034_gb300 as fp
        self.col = col
        self.codec = col.codec
        self.dict = fp.Dict(col.codec, col.dictionary.data, col.dictionary.offsets, stream)
        s = np.ascontiguousarray(col.stream, np.uint8)
        self.codes_bytes = int(s.size)
        self.codes = torch.from_numpy(s if s.size else np.zeros(16, np.uint8)).cuda()
        self.code_offsets = torch.from_numpy(np.ascontiguousarray(col.code_offsets, np.uint32).view(np.int32)).cuda()
        self.n_strings = col.n_strings

    def decode(self, capacity: int | None = None, plain: bool = False, stream=None, code_offsets=None,
               n_strings=None):
        """Returns (status, bytes[:total], offsets, guard_ok, launch_status)."""
        import torch
        import paper_2609_15034_gb300 as fp
        co = self.code_offsets if code_offsets is None else code_offsets
        n = self.n_strings if n_strings is None else n_strings
        if capacity is None:
            st, total = fp.decoded_size(self.codec, self.dict, self.codes.data_ptr(), self.codes_bytes,
                                        co.data_ptr(), n, stream)
            assert st in (fp.OK, fp.ERR_OVERFLOW), (st, fp.last_error())
            capacity = total
        out = torch.full((capacity + GUARD_BYTES,), GUARD, dtype=torch.uint8, device="cuda")
        offs = torch.full((n + 1 + 16,), -1, dtype=torch.int32, device="cuda")
        fn = fp.decode_plain if plain else fp.decode
        launch = fn(self.codec, self.dict, self.codes.data_ptr(), self.codes_bytes, co.data_ptr(), n,
                    out.data_ptr(), capacity, offs.data_ptr(), stream, check=False)
        st = fp.sync_status(stream) if launch == fp.OK else launch
        out_h = out.cpu().numpy()
        offs_h = offs.cpu().numpy().view(np.uint32)
        guard_ok = bool(np.all(out_h[capacity:] == GUARD)) and bool(np.all(offs_h[n + 1:] == 0xFFFFFFFF))
        total = int(offs_h[n]) if st == fp.OK else None
        data = out_h[:total] if total is not None else out_h[:capacity]
        return st, data, offs_h[:n + 1], guard_ok, launch


def oracle_decode(col: synth.Column, capacity=None, threads: int = 1):
    return oracle.decode(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets,
                         capacity, threads)


def assert_same(col: synth.Column, dc: DeviceColumn | None = None, **kw):
    import paper_2609_15034_gb300 as fp
    dc = dc or DeviceColumn(col)
    st, data, offs, guard_ok, _ = dc.decode(**kw)
    ref = oracle_decode(col)
    assert ref.status == oracle.OK
    assert st == fp.OK, (st, fp.last_error())
    assert guard_ok
    np.testing.assert_array_equal(offs, ref.offsets)
    assert data.size == ref.data.size
    if not np.array_equal(data, ref.data):
        bad = int(np.nonzero(data != ref.data)[0][0])
        raise AssertionError(f"first differing byte at {bad} of {data.size}")
    return dc
