"""GPU parity at the full workload sizes, in the launch configuration the
bench times (the default decoder of each codec): the whole column is decoded
on the GPU and compared with the oracle's decode of the whole column (run on
all host cores) byte for byte and offset for offset.  At these sizes the
tile scan's look-back crosses dozens to hundreds of its 2,048-tile blocks.

A second test decodes mid-size columns (several tile-scan blocks, hundreds
of block-pipeline tiles) with every compiled variant, element by element."""
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import DeviceColumn, oracle_decode

pytestmark = pytest.mark.gpu

FULL = [("onpair16_100k", synth.ONPAIR16, 100_000), ("onpair12_10m", synth.ONPAIR12, 10_000_000),
        ("fsst8_16m", synth.FSST8, 16_000_000)]


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_15034_gb300 as m
    yield m
    for c in (synth.ONPAIR16, synth.ONPAIR12, synth.FSST8):
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
