"""Host logic of bench.py: the selective-decode workload's row selection is
distinct, in range and in a seeded random order, its algorithmic bytes
count the selected rows' code slots exactly, and the bench line's tuned
shape comes from the committed tuning table's line for the GPU."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402


def test_rows_selection_is_distinct_seeded_and_unsorted():
    a = bench.rows_selection(10_000, 2_000, 0)
    assert a.dtype == np.uint32 and a.size == 2_000
    assert np.unique(a).size == 2_000 and a.max() < 10_000
    assert np.array_equal(a, bench.rows_selection(10_000, 2_000, 0))
    assert not np.array_equal(a, bench.rows_selection(10_000, 2_000, 1))
    assert not np.all(np.diff(a.astype(np.int64)) > 0)


def test_rows_algorithmic_bytes_counts_the_selected_slots():
    col = synth.column(synth.ONPAIR12, 3, 500)
    rows = np.array([4, 0, 17, 499], np.uint32)
    co = col.code_offsets.astype(np.int64)
    slots = sum(int(co[r + 1] - co[r]) for r in rows)
    total = 1234
    want = 4 * 4 + 8 * 4 + (slots * 12 + 7) // 8 + total + 4 * 5 + col.dictionary.n_entries * 17
    assert bench.rows_algorithmic_bytes(col, rows, total) == want


def test_tuned_entry_reads_the_committed_table():
    path = os.path.join(ROOT, "paper_2609_15034_gb300", "tuning", "gb300.txt")
    line = next(ln.split() for ln in open(path) if not ln.startswith("#"))
    sms, codec, width, cls = (int(x) for x in line[:4])
    codes_bytes = (1 << cls) * synth.CODE_BITS[codec] // 8
    e = bench.tuned_entry(codec, width, codes_bytes, sms)
    assert e is not None and e["size_class"] == cls
    assert bench.tuned_entry(codec, width, codes_bytes, sms + 1) is None
