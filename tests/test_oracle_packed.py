"""The oracle's decode of cascaded (bit-packed) codes, fpo_decode_packed:
codes stored at b bits per code, LSB-first -- the layer the paper removes on
the host before decoding (Sec. 5: the stored, bit-packed codes are widened).
Pinned to hand-packed bytes at several widths, to the codec layouts it must
reduce to (b = 12 is the OnPair-12 / FSST-12 stream, b = 16 the OnPair-16
one), to round trips of generated columns repacked at every width their
dictionary allows by an independent numpy writer, and to its errors."""
import numpy as np
import pytest

import oracle
import synth
from golden_io import packed_cases

ONPAIR16, ONPAIR12, FSST8, FSST12 = synth.ONPAIR16, synth.ONPAIR12, synth.FSST8, synth.FSST12


def pack_bits(codes, b):
    """LSB-first writer (test side, numpy): code i at bits [b i, b i + b)."""
    codes = np.asarray(codes, np.uint32)
    bits = ((codes[:, None] >> np.arange(b, dtype=np.uint32)) & 1).astype(np.uint8).reshape(-1)
    return np.packbits(bits, bitorder="little")


def code_dictionary(n):
    """Token c = the two bytes of c (little-endian), so the decode spells the codes."""
    toks = [bytes([c & 0xFF, c >> 8]) for c in range(n)]
    data = np.frombuffer(b"".join(toks), np.uint8)
    offs = np.arange(0, 2 * n + 1, 2, dtype=np.uint32)
    return data, offs


def test_hand_packed_examples():
    for b, codes, stream in packed_cases():
        assert bytes(pack_bits(codes, b))[:len(stream)] == stream, b   # the writer agrees with the hand work
        codec = ONPAIR16 if b > 12 else ONPAIR12
        data, offs = code_dictionary(1 << (16 if codec == ONPAIR16 else 12))
        r = oracle.decode_packed(codec, b, data, offs, np.frombuffer(stream, np.uint8),
                                 np.array([0, len(codes)], np.uint32))
        assert r.status == oracle.OK, b
        got = np.frombuffer(bytes(r.data), np.uint16)
        assert got.tolist() == codes, b


@pytest.mark.parametrize("codec,b", [(ONPAIR12, 12), (FSST12, 12), (ONPAIR16, 16)])
def test_native_width_is_the_codec_layout(codec, b):
    col = synth.column(codec, 5, 3000)
    ref = oracle.decode(codec, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets)
    r = oracle.decode_packed(codec, b, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets)
    assert r.status == oracle.OK and ref.status == oracle.OK
    np.testing.assert_array_equal(r.offsets, ref.offsets)
    np.testing.assert_array_equal(r.data, ref.data)


@pytest.mark.parametrize("codec", [ONPAIR16, ONPAIR12, FSST12])
def test_round_trip_at_every_width(codec):
    rng = np.random.default_rng(codec)
    n_entries = {ONPAIR16: 700, ONPAIR12: 300, FSST12: 90}[codec]
    toks = [bytes(rng.integers(0, 256, int(rng.integers(1, synth.MAX_TOKEN[codec] + 1))).tolist())
            for _ in range(n_entries)]
    d = synth.Dictionary.from_tokens(codec, toks)
    codes = rng.integers(0, n_entries, 20000).astype(np.uint32)
    cuts = np.sort(rng.integers(0, codes.size, 1500))
    co = np.concatenate([[0], cuts, [codes.size]]).astype(np.uint32)
    stored = synth.pack16(codes.astype(np.uint16)) if codec == ONPAIR16 else synth.pack12(codes.astype(np.uint16))
    ref = oracle.decode(codec, d.data, d.offsets, stored, co)
    assert ref.status == oracle.OK
    min_bits = int(np.ceil(np.log2(n_entries)))
    for b in range(min_bits, synth.CODE_BITS[codec] + 1):
        r = oracle.decode_packed(codec, b, d.data, d.offsets, pack_bits(codes, b), co)
        assert r.status == oracle.OK, b
        np.testing.assert_array_equal(r.offsets, ref.offsets, err_msg=str(b))
        np.testing.assert_array_equal(r.data, ref.data, err_msg=str(b))


def test_errors():
    data, offs = code_dictionary(300)
    stream = pack_bits([1, 2, 299, 300, 5], 9)   # 300 is past the dictionary
    r = oracle.decode_packed(ONPAIR12, 9, data, offs, stream, np.array([0, 3, 5], np.uint32))
    assert r.status == oracle.ERR_CORRUPT
    # widths outside 1 .. the codec's own, and the escape codec, are argument errors
    for codec, b in ((ONPAIR12, 13), (ONPAIR12, 0), (ONPAIR16, 17), (FSST8, 8)):
        r = oracle.decode_packed(codec, b, data, offs, stream, np.array([0, 1], np.uint32))
        assert r.status == oracle.ERR_ARG, (codec, b)
    # code_offsets past the whole codes of the stream
    r = oracle.decode_packed(ONPAIR12, 9, data, offs, stream, np.array([0, stream.size * 8 // 9 + 1], np.uint32))
    assert r.status == oracle.ERR_CORRUPT
