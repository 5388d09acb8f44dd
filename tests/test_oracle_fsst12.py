"""The oracle's FSST-12 codec (paper Sec. 2.1: 12-bit codes into a table of
symbols of at most 8 bytes, no escape), groundwork for that codec's decoder:
pinned to hand-worked bytes, to its limits, and to round trips through the
brute-force greedy encoder with codes packed by the generator's packer."""
import numpy as np
import pytest

import oracle
import synth
from golden_io import concat_cases

FSST12 = 4


def dict_arrays(tokens):
    data = np.frombuffer(b"".join(tokens), np.uint8)
    offs = np.zeros(len(tokens) + 1, np.uint32)
    offs[1:] = np.cumsum([len(t) for t in tokens])
    return data, offs


def test_hand_worked_fixture():
    for case in concat_cases("fsst12_small.txt"):
        data, offs = dict_arrays(case["tokens"])
        r = oracle.decode(FSST12, data, offs, np.frombuffer(case["stream"], np.uint8), case["code_offsets"])
        assert r.status == oracle.OK
        assert bytes(r.data) == case["expect_data"]
        np.testing.assert_array_equal(r.offsets, case["expect_offsets"])


def test_codes_above_255_and_255_is_not_an_escape():
    # 0x101 -> "xyz", 0xFF -> "q"; the string [0x101 0xFF 0x101] packed by hand
    # LSB-first: 01 F1 0F 01 01
    tokens = [bytes([65 + i % 26]) for i in range(0x102)]
    tokens[0xFF] = b"q"
    tokens[0x101] = b"xyz"
    data, offs = dict_arrays(tokens)
    stream = np.array([0x01, 0xF1, 0x0F, 0x01, 0x01], np.uint8)
    r = oracle.decode(FSST12, data, offs, stream, np.array([0, 3], np.uint32))
    assert r.status == oracle.OK and bytes(r.data) == b"xyzqxyz"


def test_limits():
    stream = np.zeros(3, np.uint8)
    co = np.array([0, 2], np.uint32)
    data, offs = dict_arrays([b"abcdefghi"])   # 9 bytes: fine for OnPair-12, too long for FSST-12
    assert oracle.decode(synth.ONPAIR12, data, offs, stream, co).status == oracle.OK
    assert oracle.decode(FSST12, data, offs, stream, co).status == oracle.ERR_ARG
    data, offs = dict_arrays([b"a"] * 4097)
    assert oracle.decode(FSST12, data, offs, stream, co).status == oracle.ERR_ARG
    data, offs = dict_arrays([b"a"] * 4096)
    assert oracle.decode(FSST12, data, offs, stream, co).status == oracle.OK
    # a code past the dictionary is corrupt input
    data, offs = dict_arrays([b"a", b"b"])
    stream = np.array([0x02, 0x00, 0x00], np.uint8)   # code 2
    assert oracle.decode(FSST12, data, offs, stream, np.array([0, 1], np.uint32)).status == oracle.ERR_CORRUPT


@pytest.mark.parametrize("seed", range(6))
def test_round_trip(seed):
    rng = np.random.default_rng(seed)
    alphabet = b"abcdefgh/._-0123456789"
    tokens = [bytes([b]) for b in range(256)]
    seen = set(tokens)
    while len(tokens) < 256 + int(rng.integers(50, 3000)):
        t = bytes(int(x) for x in rng.choice(list(alphabet), int(rng.integers(2, 9))))
        if t not in seen:
            seen.add(t)
            tokens.append(t)
    strings = [bytes(int(x) for x in rng.choice(list(alphabet), int(rng.integers(0, 60)))) for _ in range(80)]
    slots, co = oracle.encode_column(tokens, strings, FSST12)
    stream = synth.pack12(np.array(slots, np.uint16)) if slots else np.zeros(0, np.uint8)
    data, offs = dict_arrays(tokens)
    r = oracle.decode(FSST12, data, offs, stream, co)
    assert r.status == oracle.OK
    assert bytes(r.data) == b"".join(strings)
    np.testing.assert_array_equal(r.offsets, np.concatenate([[0], np.cumsum([len(s) for s in strings])]))
