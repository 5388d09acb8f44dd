"""Pins for the CPU oracle (no GPU).

Each test ties the oracle to something other than itself: hand-worked
fixtures written from the format definitions (paper Sec. 2.1, Sec. 5), a
closed-form special case that reduces to a numpy routine, brute force over
every 12-bit code pair against an independent bit writer, round trips
through an independent greedy encoder, and the size invariant.
"""
import numpy as np
import pytest

import oracle
import synth
from golden_io import concat_cases, pack12_cases, fsst8_escape_cases

ONPAIR16, ONPAIR12, FSST8 = synth.ONPAIR16, synth.ONPAIR12, synth.FSST8


def _store(codec, slots):
    slots = np.asarray(slots, np.uint16)
    if codec == ONPAIR16:
        return synth.pack16(slots)
    if codec == ONPAIR12:
        return synth.pack12(slots)
    return slots.astype(np.uint8)


def _dict(codec, tokens):
    return synth.Dictionary.from_tokens(codec, tokens)


# --------------------------------------------------------------------------
# hand-worked fixtures
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", concat_cases(), ids=lambda c: str(c["codec"]))
def test_concat_fixture(case):
    d = _dict(case["codec"], case["tokens"])
    stream = np.frombuffer(case["stream"], np.uint8)
    r = oracle.decode(case["codec"], d.data, d.offsets, stream, case["code_offsets"])
    assert r.status == oracle.OK
    assert r.data.tobytes() == case["expect_data"]
    np.testing.assert_array_equal(r.offsets, case["expect_offsets"])


@pytest.mark.parametrize("codes,stream", pack12_cases())
def test_pack12_fixture(codes, stream):
    # the hand-worked bytes pin both the generator's writer and the oracle's reader
    assert synth.pack12(np.array(codes, np.uint16)).tobytes() == stream
    np.testing.assert_array_equal(oracle.unpack12(np.frombuffer(stream, np.uint8), len(codes)), codes)


@pytest.mark.parametrize("slots,expect", fsst8_escape_cases())
def test_fsst8_escape_fixture(slots, expect):
    d = _dict(FSST8, [b"ab", b"c"])
    s = np.frombuffer(slots, np.uint8)
    r = oracle.decode(FSST8, d.data, d.offsets, s, np.array([0, s.size], np.uint32))
    if expect is None:
        assert r.status == oracle.ERR_CORRUPT
    else:
        assert r.status == oracle.OK
        assert r.data.tobytes() == expect
        np.testing.assert_array_equal(r.offsets, [0, len(expect)])


# --------------------------------------------------------------------------
# closed forms and special cases
# --------------------------------------------------------------------------

def test_unpack12_all_code_pairs():
    """Every ordered pair of 12-bit codes, at both nibble phases."""
    a = np.repeat(np.arange(4096, dtype=np.uint16), 4096)
    b = np.tile(np.arange(4096, dtype=np.uint16), 4096)
    seq = np.empty(2 * a.size + 1, np.uint16)
    seq[0] = 0x5A5   # shift by one code so pairs straddle both byte phases
    seq[1::2] = a
    seq[2::2] = b
    got = oracle.unpack12(synth.pack12(seq), seq.size)
    np.testing.assert_array_equal(got, seq)


@pytest.mark.parametrize("codec", [ONPAIR16, ONPAIR12])
def test_identity_dictionary_is_memcpy(codec):
    """With the 256 one-byte literals as codes 0..255 (Sec. 2.1), decoding is
    the identity on bytes: the output equals the code bytes and the offsets
    are the cumulative string lengths."""
    rng = np.random.default_rng(7)
    d = _dict(codec, [bytes([i]) for i in range(256)])
    lens = rng.integers(0, 50, 300)
    text = rng.integers(0, 256, int(lens.sum())).astype(np.uint8)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint32)
    r = oracle.decode(codec, d.data, d.offsets, _store(codec, text), offs)
    assert r.status == oracle.OK
    np.testing.assert_array_equal(r.data, text)
    np.testing.assert_array_equal(r.offsets, offs)


@pytest.mark.parametrize("codec", [ONPAIR16, ONPAIR12, FSST8])
def test_repetition(codec):
    toks = [b"x", b"hello", b"0123456789abcdef"[:synth.MAX_TOKEN[codec]], b"zz"]
    d = _dict(codec, toks)
    for c in range(len(toks)):
        slots = np.full(37, c, np.uint16)
        r = oracle.decode(codec, d.data, d.offsets, _store(codec, slots), np.array([0, 37], np.uint32))
        assert r.status == oracle.OK
        assert r.data.tobytes() == toks[c] * 37


# --------------------------------------------------------------------------
# round trips through the independent greedy encoder
# --------------------------------------------------------------------------

def _random_dict(rng, codec, n, alphabet):
    L = synth.MAX_TOKEN[codec]
    toks, seen = [], set()
    if codec != FSST8:
        for b in alphabet:   # OnPair dictionaries hold the one-byte literals
            toks.append(bytes([b]))
            seen.add(bytes([b]))
    while len(toks) < n:
        t = bytes(rng.choice(alphabet, int(rng.integers(1, L + 1))).tolist())
        if t not in seen:
            seen.add(t)
            toks.append(t)
    return toks


@pytest.mark.parametrize("codec", [ONPAIR16, ONPAIR12, FSST8])
@pytest.mark.parametrize("seed", range(40))
def test_round_trip(codec, seed):
    rng = np.random.default_rng(1000 * codec + seed)
    alphabet = np.frombuffer(b"abcdeXYZ-._/0\xff\x00", np.uint8)
    n = int(rng.integers(20, 120)) if codec != FSST8 else int(rng.integers(5, 60))
    toks = _random_dict(rng, codec, n, alphabet if codec != FSST8 else alphabet[:9])
    strings = []
    for _ in range(int(rng.integers(0, 30))):
        k = int(rng.integers(0, 60))
        src = alphabet if codec == FSST8 else alphabet
        strings.append(bytes(rng.choice(src, k).tolist()))
    slots, offs = oracle.encode_column(toks, strings, codec)
    d = _dict(codec, toks)
    r = oracle.decode(codec, d.data, d.offsets, _store(codec, slots), offs)
    assert r.status == oracle.OK
    assert r.data.tobytes() == b"".join(strings)
    np.testing.assert_array_equal(r.offsets, np.concatenate([[0], np.cumsum([len(s) for s in strings])]))


# --------------------------------------------------------------------------
# invariants on generated columns
# --------------------------------------------------------------------------

def _invariant_size(col):
    """Sum of the token lengths of non-escape codes plus one byte per escaped
    literal, from what the generator emitted."""
    tl = col.dictionary.token_lengths()
    codes = col.slot_codes.astype(np.int64)
    if col.codec == FSST8:
        lit = col.slot_is_literal
        normal = ~lit & (codes != 255)
        return int(tl[codes[normal]].sum() + lit.sum())
    return int(tl[codes].sum())


@pytest.mark.parametrize("codec", [ONPAIR16, ONPAIR12, FSST8])
def test_size_invariant_and_threads(codec):
    col = synth.column(codec, 3, 20000)
    r1 = oracle.decode_column(col)
    assert r1.status == oracle.OK
    assert r1.total == _invariant_size(col)
    assert r1.offsets[-1] == r1.total
    assert np.all(np.diff(r1.offsets.astype(np.int64)) >= 0)
    r4 = oracle.decode_column(col, threads=4)
    assert r4.status == oracle.OK
    np.testing.assert_array_equal(r1.data, r4.data)
    np.testing.assert_array_equal(r1.offsets, r4.offsets)


def test_generated_onpair12_strings_hit_targets():
    col = synth.column(ONPAIR12, 5, 5000)
    r = oracle.decode_column(col)
    lens = np.diff(r.offsets.astype(np.int64))
    assert lens.min() >= 20 and lens.max() <= 200


def test_slice_with_nonzero_first_offset():
    """code_offsets[0] != 0: the output is rebased to start at 0."""
    col = synth.column(ONPAIR12, 4, 3000)
    full = oracle.decode_column(col)
    sub = col.code_offsets[1000:2001]
    r = oracle.decode(ONPAIR12, col.dictionary.data, col.dictionary.offsets, col.stream, sub)
    base = full.offsets[1000]
    np.testing.assert_array_equal(r.offsets, full.offsets[1000:2001] - base)
    np.testing.assert_array_equal(r.data, full.data[base:full.offsets[2000]])


# --------------------------------------------------------------------------
# errors
# --------------------------------------------------------------------------

def test_code_beyond_dictionary_is_corrupt():
    d = _dict(ONPAIR16, [b"a", b"b"])
    r = oracle.decode(ONPAIR16, d.data, d.offsets, synth.pack16(np.array([0, 1, 2])),
                      np.array([0, 3], np.uint32))
    assert r.status == oracle.ERR_CORRUPT


def test_offsets_errors():
    d = _dict(ONPAIR16, [b"a", b"b"])
    s = synth.pack16(np.array([0, 1, 1]))
    assert oracle.decode(ONPAIR16, d.data, d.offsets, s, np.array([0, 2, 1, 3], np.uint32)).status == oracle.ERR_CORRUPT
    assert oracle.decode(ONPAIR16, d.data, d.offsets, s, np.array([0, 4], np.uint32)).status == oracle.ERR_CORRUPT


def test_capacity_error():
    d = _dict(ONPAIR16, [b"abc"])
    s = synth.pack16(np.zeros(10))
    r = oracle.decode(ONPAIR16, d.data, d.offsets, s, np.array([0, 10], np.uint32), capacity=29)
    assert r.status == oracle.ERR_CAPACITY and r.total == 30


def test_empty_column_and_empty_strings():
    d = _dict(ONPAIR12, [b"a"])
    r = oracle.decode(ONPAIR12, d.data, d.offsets, np.zeros(0, np.uint8), np.array([0], np.uint32))
    assert r.status == oracle.OK and r.total == 0 and list(r.offsets) == [0]
    r = oracle.decode(ONPAIR12, d.data, d.offsets, np.zeros(0, np.uint8), np.zeros(5, np.uint32))
    assert r.status == oracle.OK and list(r.offsets) == [0] * 5


def test_bad_dictionary_is_arg_error():
    d = _dict(FSST8, [b"123456789"])   # 9 bytes > FSST's 8-byte cap
    r = oracle.decode(FSST8, d.data, d.offsets, np.zeros(1, np.uint8), np.array([0, 1], np.uint32))
    assert r.status == oracle.ERR_ARG
