"""fp_decode_noalloc: the entry point for callers that cannot allocate device
memory (an allocator hook, an engine that owns all device memory).  It decodes
with a fixed scratch array compiled into the library instead of a per-stream
workspace; its output must equal fp_decode's, byte for byte (decoding is
exact), call after call, since every call reuses the same scratch -- and the
oracle's.  Calls with the default block pipeline and with a selected
warp-tile variant (another scratch layout in the same array) alternate.

This file is collected last so that a failure here cannot hide other tests."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

CASES = [(synth.ONPAIR12, 6000), (synth.FSST8, 9000), (synth.ONPAIR16, 4000)]


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_15034_gb300 as m
    yield m
    for c in (synth.ONPAIR16, synth.ONPAIR12, synth.FSST8):
        m.variant_select(c, -1)


class Column:
    def __init__(self, fp, codec, n, seed):
        import torch
        self.codec, self.n = codec, n
        self.col = synth.column(codec, seed, n)
        self.d = fp.Dict(codec, self.col.dictionary.data, self.col.dictionary.offsets)
        self.codes = torch.from_numpy(self.col.stream).cuda()
        self.co = torch.from_numpy(self.col.code_offsets.view(np.int32)).cuda()
        self.ref = oracle.decode(codec, self.col.dictionary.data, self.col.dictionary.offsets, self.col.stream,
                                 self.col.code_offsets)
        assert self.ref.status == oracle.OK
        self.total = self.ref.total

    def noalloc(self, fp):
        import torch
        out = torch.full((self.total,), 0xA5, dtype=torch.uint8, device="cuda")
        offs = torch.full((self.n + 1,), -1, dtype=torch.int32, device="cuda")
        status = torch.full((1,), 0x7FFFFFFF, dtype=torch.int32, device="cuda")
        fp.decode_noalloc(self.codec, self.d, self.codes.data_ptr(), self.codes.numel(), self.co.data_ptr(),
                          self.n, out.data_ptr(), self.total, offs.data_ptr(), status.data_ptr())
        torch.cuda.synchronize()
        return out, offs, int(status.item())

    def check_oracle(self, out, offs, what):
        np.testing.assert_array_equal(offs.cpu().numpy().view(np.uint32), self.ref.offsets, err_msg=what)
        assert np.array_equal(out.cpu().numpy(), self.ref.data), f"{what}: bytes differ from the oracle"


@pytest.mark.parametrize("codec,n", CASES)
def test_noalloc_matches_decode_twice(fp, codec, n):
    import torch
    c = Column(fp, codec, n, 77)
    ref_out = torch.empty(c.total, dtype=torch.uint8, device="cuda")
    ref_offs = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    fp.decode_tensors(codec, c.d, c.codes, c.co, n, ref_out, ref_offs)
    assert fp.sync_status() == fp.OK
    for call in range(2):
        out, offs, bits = c.noalloc(fp)
        assert bits == 0, f"call {call}: status bits {bits}"
        assert torch.equal(out, ref_out), f"call {call}: bytes differ"
        assert torch.equal(offs, ref_offs), f"call {call}: offsets differ"
        c.check_oracle(out, offs, f"call {call}")
    c.d.free()


@pytest.mark.parametrize("codec,n", CASES)
def test_noalloc_warp_tiles_alternating_with_default(fp, codec, n):
    """A selected warp-tile variant and the default block pipeline use the
    same array with different layouts; calls that alternate between them
    must each start clean."""
    c = Column(fp, codec, n, 79)
    warp = [v for v in range(fp.variant_count(codec)) if fp.variant_info(codec, v)["launches_per_call"] == 3]
    assert warp
    try:
        for call, v in enumerate([-1, warp[-1], -1, warp[0], warp[-1]]):
            fp.variant_select(codec, v)
            out, offs, bits = c.noalloc(fp)
            assert bits == 0, f"call {call} (variant {v}): status bits {bits}"
            c.check_oracle(out, offs, f"call {call} (variant {v})")
    finally:
        fp.variant_select(codec, -1)
    c.d.free()


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
