"""GPU parity at the full workload sizes, in the launch configuration the
bench times (the default decoder of each codec): the whole column is decoded
on the GPU and compared with the oracle's decode of the whole column (run on
all host cores) byte for byte and offset for offset.  At these sizes the
tile scan's look-back crosses dozens to hundreds of its 2,048-tile blocks.

The cascaded workload (16M strings, codes bit-packed at 10 bits) and the
selective-decode workload (1M random rows of the 10M-string column) are
compared whole in the same way.  A further test decodes mid-size columns
(several tile-scan blocks, hundreds of block-pipeline tiles) with every
compiled variant, element by element."""
import os

import numpy as np
import pytest

import bench
import oracle
import synth
from gpu_util import DeviceColumn, oracle_decode

pytestmark = pytest.mark.gpu

FULL = [("onpair16_100k", synth.ONPAIR16, 100_000), ("onpair12_10m", synth.ONPAIR12, 10_000_000),
        ("fsst8_16m", synth.FSST8, 16_000_000), ("fsst12_16m", synth.FSST12, 16_000_000)]


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_15034_gb300 as m
    yield m
    for c in (synth.ONPAIR16, synth.ONPAIR12, synth.FSST8, synth.FSST12):
        m.variant_select(c, -1)


def first_difference(a: np.ndarray, b: np.ndarray) -> int:
    return int(np.nonzero(a != b)[0][0])


@pytest.mark.parametrize("name,codec,n", FULL)
def test_full_size_every_element(fp, name, codec, n):
    import torch
    col = synth.column(codec, 0, n)
    d = fp.Dict(codec, col.dictionary.data, col.dictionary.offsets)
    codes = torch.from_numpy(col.stream).cuda()
    co = torch.from_numpy(col.code_offsets.view(np.int32)).cuda()
    st, total = fp.decoded_size_tensors(codec, d, codes, co, n)
    assert st == fp.OK
    ref = oracle.decode(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets,
                        threads=max(2, os.cpu_count() or 2))
    assert ref.status == oracle.OK and total == ref.total
    out = torch.empty(total + 64, dtype=torch.uint8, device="cuda")
    out[total:].fill_(0xA5)
    offs = torch.empty(n + 1 + 16, dtype=torch.int32, device="cuda")
    offs[n + 1:].fill_(-1)
    fp.decode(codec, d, codes.data_ptr(), codes.numel(), co.data_ptr(), n, out.data_ptr(), total, offs.data_ptr())
    assert fp.sync_status() == fp.OK, fp.last_error()
    out_h = out.cpu().numpy()
    offs_h = offs.cpu().numpy().view(np.uint32)
    assert np.all(out_h[total:] == 0xA5) and np.all(offs_h[n + 1:] == 0xFFFFFFFF), "write outside the buffers"
    if not np.array_equal(offs_h[:n + 1], ref.offsets):
        raise AssertionError(f"{name}: first differing offset at {first_difference(offs_h[:n + 1], ref.offsets)}")
    if not np.array_equal(out_h[:total], ref.data):
        raise AssertionError(f"{name}: first differing byte at {first_difference(out_h[:total], ref.data)}")
    d.free()


def compare(fp, name, out, offs, total, n, ref):
    out_h = out.cpu().numpy()
    offs_h = offs.cpu().numpy().view(np.uint32)
    assert np.all(out_h[total:] == 0xA5) and np.all(offs_h[n + 1:] == 0xFFFFFFFF), "write outside the buffers"
    if not np.array_equal(offs_h[:n + 1], ref.offsets):
        raise AssertionError(f"{name}: first differing offset at {first_difference(offs_h[:n + 1], ref.offsets)}")
    if not np.array_equal(out_h[:total], ref.data):
        raise AssertionError(f"{name}: first differing byte at {first_difference(out_h[:total], ref.data)}")


def guarded(total, n):
    import torch
    out = torch.empty(total + 64, dtype=torch.uint8, device="cuda")
    out[total:].fill_(0xA5)
    offs = torch.empty(n + 1 + 16, dtype=torch.int32, device="cuda")
    offs[n + 1:].fill_(-1)
    return out, offs


def test_full_size_cascaded_every_element(fp):
    import torch
    col, bits = bench.workload_column("fsst12_packed10_16m", 0)
    n, codec = col.n_strings, col.codec
    d = fp.Dict(codec, col.dictionary.data, col.dictionary.offsets)
    codes = torch.from_numpy(col.stream).cuda()
    co = torch.from_numpy(col.code_offsets.view(np.int32)).cuda()
    st, total = fp.decoded_size_packed(codec, d, bits, codes.data_ptr(), codes.numel(), co.data_ptr(), n)
    assert st == fp.OK
    ref = oracle.decode_packed(codec, bits, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets)
    assert ref.status == oracle.OK and total == ref.total
    out, offs = guarded(total, n)
    fp.decode_packed(codec, d, bits, codes.data_ptr(), codes.numel(), co.data_ptr(), n, out.data_ptr(), total,
                     offs.data_ptr())
    assert fp.sync_status() == fp.OK, fp.last_error()
    compare(fp, "fsst12_packed10_16m", out, offs, total, n, ref)
    d.free()


def test_full_size_selected_rows_every_element(fp):
    import torch
    col = synth.column(synth.ONPAIR12, 0, 10_000_000)
    rows_h = bench.rows_selection(col.n_strings, 1_000_000, 0)
    d = fp.Dict(col.codec, col.dictionary.data, col.dictionary.offsets)
    codes = torch.from_numpy(col.stream).cuda()
    co = torch.from_numpy(col.code_offsets.view(np.int32)).cuda()
    rows = torch.from_numpy(rows_h.view(np.int32)).cuda()
    m = rows_h.size
    st, slots, total = fp.rows_size(col.codec, d, codes.data_ptr(), codes.numel(), co.data_ptr(), col.n_strings,
                                    rows.data_ptr(), m)
    assert st == fp.OK
    ref = oracle.decode_rows(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets,
                             rows_h)
    assert ref.status == oracle.OK and total == ref.total
    out, offs = guarded(total, m)
    fp.decode_rows(col.codec, d, codes.data_ptr(), codes.numel(), co.data_ptr(), col.n_strings, rows.data_ptr(), m,
                   slots, out.data_ptr(), total, offs.data_ptr())
    assert fp.sync_status() == fp.OK, fp.last_error()
    compare(fp, "onpair12_10m_rows1m", out, offs, total, m, ref)
    d.free()


MID = [(synth.ONPAIR12, 600_000), (synth.FSST8, 1_000_000), (synth.ONPAIR16, 500_000)]


@pytest.mark.parametrize("codec,n", MID)
def test_every_variant_across_scan_blocks(fp, codec, n):
    col = synth.column(codec, 31, n)
    ref = oracle_decode(col)
    assert ref.status == oracle.OK
    # tiles of 512 or 1,024 slots: several blocks of 2,048 tiles in the tile scan
    assert col.n_slots > 4 * 2048 * 1024
    dc = DeviceColumn(col)
    try:
        for v in range(fp.variant_count(codec)):
            fp.variant_select(codec, v)
            st, data, offs, guard_ok, _ = dc.decode(capacity=ref.total)
            assert st == fp.OK, (v, fp.last_error())
            assert guard_ok, v
            if not np.array_equal(offs, ref.offsets):
                raise AssertionError(f"variant {v}: first differing offset at {first_difference(offs, ref.offsets)}")
            if not np.array_equal(data, ref.data):
                raise AssertionError(f"variant {v}: first differing byte at {first_difference(data, ref.data)}")
    finally:
        fp.variant_select(codec, -1)
