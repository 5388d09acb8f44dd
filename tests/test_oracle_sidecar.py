"""The oracle's stored-sidecar definition (paper Sec. 3.1: output positions
stored beside the column) pinned to things other than itself: hand-worked
tables, the oracle decode's string offsets, per-slot byte counts computed
here from the dictionary and the generator's own bookkeeping, and the
relation between tile sizes."""
import numpy as np
import pytest

import oracle
import synth
from golden_io import sidecar_cases

ONPAIR16, ONPAIR12, FSST8 = synth.ONPAIR16, synth.ONPAIR12, synth.FSST8
FLAG = np.uint64(1 << 63)


def dict_arrays(tokens):
    data = np.frombuffer(b"".join(tokens), np.uint8)
    offs = np.zeros(len(tokens) + 1, np.uint32)
    offs[1:] = np.cumsum([len(t) for t in tokens])
    return data, offs


@pytest.mark.parametrize("case", sidecar_cases(), ids=lambda c: f"codec{c['codec']}-tile{c['tile']}")
def test_hand_worked_tables(case):
    data, offs = dict_arrays(case["tokens"])
    stream = np.frombuffer(case["stream"], np.uint8)
    got = oracle.sidecar(case["codec"], data, offs, stream, case["code_offsets"], case["tile"])
    np.testing.assert_array_equal(got, case["expect_sidecar"])


def slot_codes(col):
    """Codes of every slot, unpacked here with numpy (not by the oracle)."""
    s = np.ascontiguousarray(col.stream, np.uint8)
    if col.codec == ONPAIR16:
        return s[: s.size // 2 * 2].view("<u2").astype(np.int64)
    if col.codec == FSST8:
        return s.astype(np.int64)
    bits = np.unpackbits(s, bitorder="little")
    n = bits.size // 12
    return (bits[: 12 * n].reshape(n, 12).astype(np.int64) << np.arange(12)).sum(axis=1)


def slot_bytes(col):
    """Bytes each slot of the column produces, and which slots are literals,
    from the dictionary's token lengths and the generator's bookkeeping."""
    codes = slot_codes(col)
    lens = np.diff(np.asarray(col.dictionary.offsets, np.int64))
    c0, c1 = int(col.code_offsets[0]), int(col.code_offsets[-1])
    q = np.arange(c0, c1)
    if col.codec != FSST8:
        return lens[codes[q]], np.zeros(q.size, bool)
    lit = np.asarray(col.slot_is_literal, bool)[q]
    esc = (codes[q] == 255) & ~lit
    b = np.where(lit, 1, np.where(esc, 0, lens[np.minimum(codes[q], lens.size - 1)]))
    return b, lit


def columns():
    cols = []
    for codec in (ONPAIR16, ONPAIR12, FSST8):
        for seed, n in ((11, 1), (12, 57), (13, 3000)):
            cols.append(synth.column(codec, seed * 10 + codec, n))
    return cols


@pytest.mark.parametrize("col", columns(), ids=lambda c: c.name)
def test_one_slot_tiles_match_slot_bytes_and_string_offsets(col):
    sc = oracle.sidecar(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets, 1)
    dec = oracle.decode_column(col)
    assert dec.status == oracle.OK
    b, lit = slot_bytes(col)
    c0, c1 = int(col.code_offsets[0]), int(col.code_offsets[-1])
    assert sc.size == 1 + max(1, c1 - c0)
    assert int(sc[0]) == dec.total == int(b.sum())
    if c1 > c0:
        flags = (sc[1:] & FLAG) != 0
        np.testing.assert_array_equal(flags, lit)
        prefix = np.concatenate([[0], np.cumsum(b)[:-1]])
        np.testing.assert_array_equal((sc[1:] & ~FLAG).astype(np.int64), prefix)
        # where a string starts, the table holds its output offset
        starts = np.asarray(col.code_offsets[:-1], np.int64)
        inside = starts < c1
        np.testing.assert_array_equal((sc[1 + starts[inside] - c0] & ~FLAG).astype(np.int64),
                                      dec.offsets[:-1][inside].astype(np.int64))


@pytest.mark.parametrize("codec", [ONPAIR16, ONPAIR12, FSST8])
def test_larger_tiles_sample_the_one_slot_table(codec):
    col = synth.column(codec, 77 + codec, 2500)
    co = np.asarray(col.code_offsets, np.uint32)
    # a slice whose first slot is not tile-aligned, and the whole column
    for a, b in ((0, co.size - 1), (317, 2011)):
        sub = co[a:b + 1]
        one = oracle.sidecar(codec, col.dictionary.data, col.dictionary.offsets, col.stream, sub, 1)
        c0, c1 = int(sub[0]), int(sub[-1])
        for log2 in (1, 3, 5, 9, 10):
            tile = 1 << log2
            sc = oracle.sidecar(codec, col.dictionary.data, col.dictionary.offsets, col.stream, sub, tile)
            first, end = c0 // tile, -(-c1 // tile)
            assert sc.size == 1 + max(1, end - first)
            assert sc[0] == one[0]
            assert sc[1] == 0
            for u in range(1, sc.size - 1):
                s = (first + u) * tile
                assert sc[1 + u] == one[1 + s - c0], (tile, u)


def test_invalid_columns_have_no_table():
    data, offs = dict_arrays([b"a", b"bc"])
    stream = np.array([0, 1, 5], np.uint8)   # code 5 is past the dictionary
    assert oracle.sidecar(FSST8, data, offs, stream, np.array([0, 3], np.uint32), 2) is None
    stream = np.array([0, 255], np.uint8)    # escape in a string's last slot
    assert oracle.sidecar(FSST8, data, offs, stream, np.array([0, 2], np.uint32), 2) is None
    assert oracle.sidecar(FSST8, data, offs, np.array([0, 1], np.uint8), np.array([0, 3], np.uint32), 2) is None
