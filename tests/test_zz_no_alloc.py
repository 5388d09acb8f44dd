"""fp_decode_noalloc: the entry point for callers that cannot allocate device
memory (an allocator hook, an engine that owns all device memory).  It decodes
with a fixed scratch array compiled into the library instead of a per-stream
workspace; its output must equal fp_decode's, byte for byte (decoding is
exact), call after call, since every call reuses the same scratch.

This file is collected last so that a failure here cannot hide other tests."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_15034_gb300 as m
    return m


@pytest.mark.parametrize("codec,n", [(synth.ONPAIR12, 6000), (synth.FSST8, 9000), (synth.ONPAIR16, 4000)])
def test_noalloc_matches_decode_twice(fp, codec, n):
    import torch
    col = synth.column(codec, 77, n)
    d = fp.Dict(codec, col.dictionary.data, col.dictionary.offsets)
    codes = torch.from_numpy(col.stream).cuda()
    co = torch.from_numpy(col.code_offsets.view(np.int32)).cuda()
    st, total = fp.decoded_size_tensors(codec, d, codes, co, n)
    assert st == fp.OK
    ref_out = torch.empty(total, dtype=torch.uint8, device="cuda")
    ref_offs = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    fp.decode_tensors(codec, d, codes, co, n, ref_out, ref_offs)
    assert fp.sync_status() == fp.OK
    for call in range(2):
        out = torch.full((total,), 0xA5, dtype=torch.uint8, device="cuda")
        offs = torch.full((n + 1,), -1, dtype=torch.int32, device="cuda")
        status = torch.full((1,), 0x7FFFFFFF, dtype=torch.int32, device="cuda")
        fp.decode_noalloc(codec, d, codes.data_ptr(), codes.numel(), co.data_ptr(), n, out.data_ptr(), total,
                          offs.data_ptr(), status.data_ptr())
        torch.cuda.synchronize()
        assert int(status.item()) == 0, f"call {call}: status bits {int(status.item())}"
        assert torch.equal(out, ref_out), f"call {call}: bytes differ"
        assert torch.equal(offs, ref_offs), f"call {call}: offsets differ"
    d.free()


def test_noalloc_rejects_inputs_beyond_its_scratch(fp):
    import torch
    col = synth.column(synth.FSST8, 78, 10)
    d = fp.Dict(synth.FSST8, col.dictionary.data, col.dictionary.offsets)
    co = torch.from_numpy(col.code_offsets.view(np.int32)).cuda()
    out = torch.empty(1024, dtype=torch.uint8, device="cuda")
    offs = torch.empty(11, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    big = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")   # 1 GiB of FSST-8 slots: too many tiles
    st = fp.decode_noalloc(synth.FSST8, d, big.data_ptr(), big.numel(), co.data_ptr(), 10, out.data_ptr(), 1024,
                           offs.data_ptr(), status.data_ptr(), check=False)
    assert st == fp.ERR_ARG
    assert "scratch" in fp.last_error()
    d.free()
