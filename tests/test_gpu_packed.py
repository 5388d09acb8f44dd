"""GPU parity of the fused de-cascade (fp_decode_packed): columns whose codes
are bit-packed at any width from the dictionary's minimum to the codec's own
are decoded inside the kernels and must equal the oracle's
fpo_decode_packed byte for byte and offset for offset -- and the decode of
the same column in the codec's stored layout.  Slices, empty strings, tile
edges, corrupt codes and argument errors included."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import GUARD, GUARD_BYTES

pytestmark = pytest.mark.gpu

ONPAIR16, ONPAIR12, FSST8, FSST12 = synth.ONPAIR16, synth.ONPAIR12, synth.FSST8, synth.FSST12


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_15034_gb300 as m
    return m


def pack_bits(codes, b):
    codes = np.asarray(codes, np.uint32)
    bits = ((codes[:, None] >> np.arange(b, dtype=np.uint32)) & 1).astype(np.uint8).reshape(-1)
    return np.packbits(bits, bitorder="little")


def small_dict(codec, n_entries, rng):
    toks = [bytes(rng.integers(0, 256, int(rng.integers(1, synth.MAX_TOKEN[codec] + 1))).tolist())
            for _ in range(n_entries)]
    return synth.Dictionary.from_tokens(codec, toks)


def run(fp, codec, d_host, b, stream, co_h, capacity=None):
    import torch
    d = fp.Dict(codec, d_host.data, d_host.offsets)
    s = np.ascontiguousarray(stream, np.uint8)
    codes = torch.from_numpy(s if s.size else np.zeros(16, np.uint8)).cuda()
    co = torch.from_numpy(np.ascontiguousarray(co_h, np.uint32).view(np.int32)).cuda()
    n = int(co_h.size - 1)
    ref = oracle.decode_packed(codec, b, d_host.data, d_host.offsets, s, co_h)
    st, total = fp.decoded_size_packed(codec, d, b, codes.data_ptr(), int(s.size), co.data_ptr(), n)
    if ref.status == oracle.OK:
        assert st == fp.OK and total == ref.total, (st, total, ref.total)
    cap = ref.total if capacity is None else capacity
    out = torch.full((cap + GUARD_BYTES,), GUARD, dtype=torch.uint8, device="cuda")
    offs = torch.full((n + 1 + 16,), -1, dtype=torch.int32, device="cuda")
    fp.decode_packed(codec, d, b, codes.data_ptr(), int(s.size), co.data_ptr(), n, out.data_ptr(), cap,
                     offs.data_ptr())
    st = fp.sync_status()
    out_h = out.cpu().numpy()
    offs_h = offs.cpu().numpy().view(np.uint32)
    guard_ok = bool(np.all(out_h[cap:] == GUARD)) and bool(np.all(offs_h[n + 1:] == 0xFFFFFFFF))
    d.free()
    return st, ref, out_h[:cap], offs_h[:n + 1], guard_ok


@pytest.mark.parametrize("codec", [ONPAIR16, ONPAIR12, FSST12])
def test_every_width_matches_oracle(fp, codec):
    rng = np.random.default_rng(200 + codec)
    n_entries = {ONPAIR16: 3000, ONPAIR12: 1500, FSST12: 700}[codec]
    d = small_dict(codec, n_entries, rng)
    codes = rng.integers(0, n_entries, 150_000).astype(np.uint32)
    cuts = np.sort(rng.integers(0, codes.size, 9000))
    co = np.concatenate([[0], cuts, [codes.size]]).astype(np.uint32)
    native = synth.pack16(codes.astype(np.uint16)) if codec == ONPAIR16 else synth.pack12(codes.astype(np.uint16))
    plain = oracle.decode(codec, d.data, d.offsets, native, co)
    lo = int(np.ceil(np.log2(n_entries)))
    for b in range(lo, synth.CODE_BITS[codec] + 1):
        st, ref, out, offs, guard_ok = run(fp, codec, d, b, pack_bits(codes, b), co)
        assert ref.status == oracle.OK
        assert st == fp.OK, (b, fp.last_error())
        assert guard_ok, b
        np.testing.assert_array_equal(offs, ref.offsets, err_msg=f"width {b}")
        assert np.array_equal(out[:ref.total], ref.data), b
        np.testing.assert_array_equal(offs, plain.offsets)   # the cascade changes nothing in the output


@pytest.mark.parametrize("b", [1, 3, 7, 11])
def test_narrow_widths_slices_and_tile_edges(fp, b):
    codec = ONPAIR12
    rng = np.random.default_rng(300 + b)
    d = small_dict(codec, 1 << b, rng)
    codes = rng.integers(0, 1 << b, 3 * 8192 + 77).astype(np.uint32)
    stream = pack_bits(codes, b)
    edges = np.arange(0, codes.size, 256)
    co = np.sort(np.concatenate([[0], edges, edges, rng.integers(0, codes.size, 400), [codes.size] * 3]))
    co = co.astype(np.uint32)
    st, ref, out, offs, guard_ok = run(fp, codec, d, b, stream, co)
    assert st == fp.OK and guard_ok
    np.testing.assert_array_equal(offs, ref.offsets)
    assert np.array_equal(out[:ref.total], ref.data)
    # a slice starting at an odd slot
    sub = np.array([777, 778, 5000, 9001], np.uint32)
    st, ref, out, offs, guard_ok = run(fp, codec, d, b, stream, sub)
    assert st == fp.OK and guard_ok
    np.testing.assert_array_equal(offs, ref.offsets)
    assert np.array_equal(out[:ref.total], ref.data)


def test_corrupt_codes_and_arguments(fp):
    import torch
    rng = np.random.default_rng(7)
    d = small_dict(FSST12, 300, rng)
    codes = rng.integers(0, 512, 40000).astype(np.uint32)   # codes 300..511 have no token
    st, ref, out, offs, guard_ok = run(fp, FSST12, d, 9, pack_bits(codes, 9),
                                       np.array([0, 20000, 40000], np.uint32), capacity=100000)
    assert ref.status == oracle.ERR_CORRUPT
    assert st == fp.ERR_CORRUPT and guard_ok
    dd = fp.Dict(FSST8, *[np.frombuffer(b"abc", np.uint8), np.array([0, 1, 3], np.uint32)])
    buf = torch.zeros(64, dtype=torch.uint8, device="cuda")
    co = torch.zeros(2, dtype=torch.int32, device="cuda")
    o = torch.zeros(2, dtype=torch.int32, device="cuda")
    assert fp.decode_packed(FSST8, dd, 8, buf.data_ptr(), 64, co.data_ptr(), 1, buf.data_ptr(), 0, o.data_ptr(),
                            check=False) == fp.ERR_ARG
    d12 = fp.Dict(ONPAIR12, d.data, d.offsets)
    for b in (0, 13):
        assert fp.decode_packed(ONPAIR12, d12, b, buf.data_ptr(), 64, co.data_ptr(), 1, buf.data_ptr(), 0,
                                o.data_ptr(), check=False) == fp.ERR_ARG
    dd.free()
    d12.free()
