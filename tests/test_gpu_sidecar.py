"""GPU parity of the stored-sidecar calls (fastpair_sidecar.h): the table
fp_sidecar_build computes equals the oracle's definition entry for entry,
and fp_decode_sidecar, given either that table or the oracle's, decodes
every column exactly as the oracle does; a too-small output is reported
and a table from elsewhere never makes the decode write out of bounds."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import GUARD, GUARD_BYTES, DeviceColumn

pytestmark = pytest.mark.gpu

ONPAIR16, ONPAIR12, FSST8, FSST12 = synth.ONPAIR16, synth.ONPAIR12, synth.FSST8, synth.FSST12
CODECS = [ONPAIR16, ONPAIR12, FSST8, FSST12]


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_15034_gb300 as m
    return m


def cases():
    out = []
    for codec in CODECS:
        for k, n in enumerate((1, 5, 300, 5000, 40000)):
            out.append((codec, 1000 + 10 * codec + k, n, None))
        out.append((codec, 1100 + codec, 20000, (1234, 17001)))   # a slice: code_offsets start mid-buffer
        out.append((codec, 1200 + codec, 50, (7, 7)))             # no strings
    return out


def ident(c):
    codec, seed, n, sl = c
    return f"codec{codec}-n{n}" + (f"-slice{sl[0]}:{sl[1]}" if sl else "")


class Case:
    def __init__(self, fp, spec):
        import torch
        codec, seed, n, sl = spec
        self.col = synth.column(codec, seed, n)
        self.dc = DeviceColumn(self.col)
        co = np.asarray(self.col.code_offsets, np.uint32)
        if sl is not None:
            co = co[sl[0]:sl[1] + 1]
        self.co_h = co
        self.n = int(co.size - 1)
        self.co = torch.from_numpy(np.ascontiguousarray(co).view(np.int32)).cuda()
        self.ref = oracle.decode(codec, self.col.dictionary.data, self.col.dictionary.offsets, self.col.stream, co)
        assert self.ref.status == oracle.OK
        self.tile = fp.sidecar_tile_slots(codec)
        self.table = oracle.sidecar(codec, self.col.dictionary.data, self.col.dictionary.offsets, self.col.stream,
                                    co, self.tile)
        self.sc = fp.SidecarColumn(codec, self.dc.dict, self.dc.codes, self.co, self.n, self.dc.codes_bytes)

    def decode(self, fp, capacity=None, table=None):
        import torch
        cap = self.ref.total if capacity is None else capacity
        out = torch.full((cap + GUARD_BYTES,), GUARD, dtype=torch.uint8, device="cuda")
        offs = torch.full((self.n + 1 + 16,), -1, dtype=torch.int32, device="cuda")
        self.sc.decode(out[:cap], offs, sidecar=table)
        bits = self.sc.status_bits()
        out_h = out.cpu().numpy()
        offs_h = offs.cpu().numpy().view(np.uint32)
        guard_ok = bool(np.all(out_h[cap:] == GUARD)) and bool(np.all(offs_h[self.n + 1:] == 0xFFFFFFFF))
        return bits, out_h[:cap], offs_h[:self.n + 1], guard_ok


@pytest.mark.parametrize("spec", cases(), ids=ident)
def test_build_matches_oracle_table(fp, spec):
    c = Case(fp, spec)
    c.sc.build()
    assert c.sc.status_bits() == 0
    got = c.sc.sidecar.cpu().numpy().view(np.uint64)
    t = c.table.size
    np.testing.assert_array_equal(got[:t], c.table)


@pytest.mark.parametrize("spec", cases(), ids=ident)
def test_decode_from_built_and_from_oracle_tables(fp, spec):
    import torch
    c = Case(fp, spec)
    c.sc.build()
    for table in (None, torch.from_numpy(np.concatenate(
            [c.table, np.zeros(c.sc.entries - c.table.size, np.uint64)]).view(np.int64)).cuda()):
        bits, data, offs, guard_ok = c.decode(fp, table=table)
        assert bits == 0
        assert guard_ok
        np.testing.assert_array_equal(offs, c.ref.offsets)
        np.testing.assert_array_equal(data, c.ref.data)


@pytest.mark.parametrize("codec", CODECS)
def test_capacity_is_reported_and_respected(fp, codec):
    c = Case(fp, (codec, 1300 + codec, 3000, None))
    c.sc.build()
    bits, data, offs, guard_ok = c.decode(fp, capacity=c.ref.total // 2)
    assert bits & 2
    assert guard_ok


@pytest.mark.parametrize("codec", CODECS)
def test_foreign_table_stays_in_bounds(fp, codec):
    """A table from elsewhere: every write stays in bounds, and the decode's
    self-check (each tile's recomputed byte total against the next entry)
    reports the mismatch (bit 16)."""
    import torch
    c = Case(fp, (codec, 1400 + codec, 3000, None))
    rng = np.random.default_rng(codec)
    for hi in (1 << 12, 1 << 20, 1 << 62):
        t = rng.integers(0, hi, c.sc.entries, dtype=np.uint64)
        t[1::3] |= np.uint64(1 << 63)
        t[0] = c.ref.total   # size entry consistent, positions not
        bits, data, offs, guard_ok = c.decode(fp, table=torch.from_numpy(t.view(np.int64)).cuda())
        assert guard_ok
        assert bits & 16, bits


def test_arguments_are_checked(fp):
    import torch
    c = Case(fp, (ONPAIR12, 1500, 100, None))
    out = torch.empty(c.ref.total + 16, dtype=torch.uint8, device="cuda")
    offs = torch.empty(c.n + 1, dtype=torch.int32, device="cuda")
    common = (ONPAIR12, c.dc.dict, c.dc.codes.data_ptr(), c.dc.codes_bytes, c.co.data_ptr(), c.n)
    sc = c.sc
    with pytest.raises(fp.FastPairError):   # table shorter than the code buffer needs
        fp.sidecar_build(*common, sc.sidecar.data_ptr(), sc.entries - 1, sc.scratch.data_ptr(), sc.scratch_bytes,
                         sc.status.data_ptr())
    with pytest.raises(fp.FastPairError):   # scratch too small
        fp.decode_sidecar(*common, sc.sidecar.data_ptr(), sc.entries, out.data_ptr(), c.ref.total, offs.data_ptr(),
                          sc.scratch.data_ptr(), sc.scratch_bytes - 1, sc.status.data_ptr())
    with pytest.raises(fp.FastPairError):   # misaligned table
        fp.decode_sidecar(*common, sc.sidecar.data_ptr() + 4, sc.entries, out.data_ptr(), c.ref.total,
                          offs.data_ptr(), sc.scratch.data_ptr(), sc.scratch_bytes, sc.status.data_ptr())
    with pytest.raises(fp.FastPairError):   # dictionary of another codec
        fp.sidecar_build(FSST8, *common[1:], sc.sidecar.data_ptr(), sc.entries, sc.scratch.data_ptr(),
                         sc.scratch_bytes, sc.status.data_ptr())
