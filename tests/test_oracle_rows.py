"""The oracle's selective decode (a row subset of a column, random access to
single strings; paper Sec. 1 and Sec. 2.1) pinned to a hand-worked case, to
the identity selection, and to strings assembled here from the generator's
own text of every row."""
import numpy as np
import pytest

import oracle
import synth

ONPAIR16, ONPAIR12, FSST8 = synth.ONPAIR16, synth.ONPAIR12, synth.FSST8


def test_hand_worked_rows():
    # dictionary 0 -> "a", 1 -> "bc", 2 -> "def"; strings [1 0 2], [], [0 0]
    data = np.frombuffer(b"abcdef", np.uint8)
    offs = np.array([0, 1, 3, 6], np.uint32)
    stream = np.array([1, 0, 2, 0, 0], np.uint8)   # FSST-8 slots: one byte per code
    co = np.array([0, 3, 3, 5], np.uint32)
    r = oracle.decode_rows(FSST8, data, offs, stream, co, [2, 0, 2, 1])
    assert r.status == oracle.OK
    assert bytes(r.data) == b"aa" + b"bcadef" + b"aa"
    np.testing.assert_array_equal(r.offsets, [0, 2, 8, 10, 10])


def strings_of(col):
    """Every row's text from the generator's slot bookkeeping and the
    dictionary's tokens (not from the oracle)."""
    toks = col.dictionary.tokens()
    co = np.asarray(col.code_offsets, np.int64)
    codes = np.asarray(col.slot_codes, np.int64)
    lit = np.asarray(col.slot_is_literal, bool)
    out = []
    for i in range(co.size - 1):
        parts = []
        for q in range(co[i], co[i + 1]):
            if lit[q]:
                parts.append(bytes([codes[q]]))
            elif col.codec == FSST8 and codes[q] == 255:
                continue
            else:
                parts.append(toks[codes[q]])
        out.append(b"".join(parts))
    return out


@pytest.mark.parametrize("codec", [ONPAIR16, ONPAIR12, FSST8])
def test_rows_match_the_generators_strings(codec):
    col = synth.column(codec, 500 + codec, 400)
    text = strings_of(col)
    rng = np.random.default_rng(codec)
    for rows in (np.arange(col.n_strings), rng.integers(0, col.n_strings, 700), np.array([], np.int64),
                 np.full(5, col.n_strings - 1)):
        r = oracle.decode_rows(codec, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets,
                               rows)
        assert r.status == oracle.OK
        want = [text[k] for k in rows]
        assert bytes(r.data) == b"".join(want)
        np.testing.assert_array_equal(r.offsets, np.concatenate([[0], np.cumsum([len(w) for w in want])]))


def test_all_rows_in_order_is_the_column_decode():
    col = synth.column(ONPAIR12, 611, 2000)
    full = oracle.decode_column(col)
    r = oracle.decode_rows(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets,
                           np.arange(col.n_strings))
    np.testing.assert_array_equal(r.data, full.data)
    np.testing.assert_array_equal(r.offsets, full.offsets)


def test_row_out_of_range_and_capacity():
    col = synth.column(ONPAIR16, 612, 10)
    args = (col.codec, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets)
    assert oracle.decode_rows(*args, [0, 10]).status == oracle.ERR_ARG
    full = oracle.decode_rows(*args, [3, 4])
    r = oracle.decode_rows(*args, [3, 4], capacity=max(full.total - 1, 0))
    assert r.status == oracle.ERR_CAPACITY and r.total == full.total
