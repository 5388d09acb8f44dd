"""GPU parity at the full workload sizes, in the launch configuration the
bench times (the default decoder of each codec): the whole column is decoded
on the GPU; the oracle checks a sample of strings one by one (first, last,
random, and strings around tile edges) and the size invariants hold for the
whole output (offsets start at 0, never decrease, end at the oracle's total)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

FULL = [("onpair16_100k", synth.ONPAIR16, 100_000), ("onpair12_10m", synth.ONPAIR12, 10_000_000),
        ("fsst8_16m", synth.FSST8, 16_000_000)]


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_15034_gb300 as m
    return m


@pytest.mark.parametrize("name,codec,n", FULL)
def test_full_size_sampled(fp, name, codec, n):
    import torch
    col = synth.column(codec, 0, n)
    d = fp.Dict(codec, col.dictionary.data, col.dictionary.offsets)
    codes = torch.from_numpy(col.stream).cuda()
    co = torch.from_numpy(col.code_offsets.view(np.int32)).cuda()
    st, total = fp.decoded_size_tensors(codec, d, codes, co, n)
    assert st == fp.OK
    ref_st, ref_total = oracle.decoded_size(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream,
                                            col.code_offsets)
    assert ref_st == oracle.OK and total == ref_total
    out = torch.empty(total, dtype=torch.uint8, device="cuda")
    offs = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    fp.decode_tensors(codec, d, codes, co, n, out, offs)
    assert fp.sync_status() == fp.OK
    offs_h = offs.cpu().numpy().view(np.uint32).astype(np.int64)
    assert offs_h[0] == 0 and offs_h[-1] == total
    assert np.all(np.diff(offs_h) >= 0)
    # sample: first and last strings, random ones, and the strings that contain
    # each decoder's tile edges (4,096-, 8,192- and 512-slot tiles)
    rng = np.random.default_rng(1)
    sample = set([0, 1, n - 2, n - 1]) | set(rng.integers(0, n, 1500).tolist())
    slots = col.code_offsets.astype(np.int64)
    for tile in (512, 4096, 8192):
        edges = np.arange(tile, int(slots[-1]), tile)[:: max(1, (int(slots[-1]) // tile) // 300)]
        sample |= set((np.searchsorted(slots, edges, side="right") - 1).clip(0, n - 1).tolist())
    out_h = out.cpu().numpy()
    for i in sorted(sample):
        r = oracle.decode(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream,
                          col.code_offsets[i:i + 2])
        assert r.status == oracle.OK
        a, b = int(offs_h[i]), int(offs_h[i + 1])
        assert b - a == r.total, (name, i)
        assert np.array_equal(out_h[a:b], r.data), (name, i)
    d.free()
