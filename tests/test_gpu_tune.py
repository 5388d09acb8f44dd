"""The single-column autotuner (fp_tune_column / fp_tune_load /
fp_tune_clear): it picks a compiled shape of the dictionary's read width,
makes it the default for the column's size class (and nothing else), writes
it to a table that fp_tune_load reads back, and decoding with the tuned
default still equals the oracle."""
import os

import numpy as np
import pytest

import synth
from gpu_util import DeviceColumn, assert_same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_15034_gb300 as m
    yield m
    m.tune_clear()
    table = os.path.join(os.path.dirname(m.__file__), "tuning", "gb300.txt")
    if os.path.exists(table):
        m.tune_load(table)


@pytest.mark.parametrize("codec", [synth.ONPAIR16, synth.ONPAIR12, synth.FSST8, synth.FSST12])
def test_tune_sets_the_default_for_the_size_class(fp, codec, tmp_path):
    import torch
    fp.tune_clear()
    col = synth.column(codec, 33, 20000)
    dc = DeviceColumn(col)
    st, total = fp.decoded_size(codec, dc.dict, dc.codes.data_ptr(), dc.codes_bytes, dc.code_offsets.data_ptr(),
                                dc.n_strings)
    out = torch.empty(total, dtype=torch.uint8, device="cuda")
    offs = torch.empty(dc.n_strings + 1, dtype=torch.int32, device="cuda")
    table = str(tmp_path / "tune.txt")
    builtin = fp.variant_for_dict(dc.dict, dc.codes_bytes)
    st, v, ms = fp.tune_column(codec, dc.dict, dc.codes.data_ptr(), dc.codes_bytes, dc.code_offsets.data_ptr(),
                               dc.n_strings, out.data_ptr(), total, offs.data_ptr(), table)
    assert st == fp.OK, fp.last_error()
    assert 0 <= v < fp.variant_count(codec) and ms > 0
    assert fp.variant_width(codec, v) == dc.dict.width
    assert fp.variant_for_dict(dc.dict, dc.codes_bytes) == v
    assert_same(col, dc)
    # the table holds the choice; clearing restores the built-in default, loading restores the choice
    with open(table) as f:
        fields = f.read().split()
    assert int(fields[1]) == codec and int(fields[2]) == dc.dict.width and int(fields[4]) == v
    fp.tune_clear()
    assert fp.variant_for_dict(dc.dict, dc.codes_bytes) == builtin
    fp.tune_load(table)
    assert fp.variant_for_dict(dc.dict, dc.codes_bytes) == v
    # a selection still overrides
    fp.variant_select(codec, 0)
    assert fp.variant_for_dict(dc.dict, dc.codes_bytes) == 0
    fp.variant_select(codec, -1)
    fp.tune_clear()


def test_tune_load_ignores_foreign_entries(fp, tmp_path):
    fp.tune_clear()
    table = tmp_path / "foreign.txt"
    table.write_text("# another GPU and an unknown variant\n9999 2 16 20 3 1.0\n0 2 16 20 999 1.0\nnot a line\n")
    fp.tune_load(str(table))
    col = synth.column(synth.ONPAIR12, 34, 100)
    dc = DeviceColumn(col)
    fp.tune_clear()
    builtin = fp.variant_for_dict(dc.dict, 1 << 22)
    fp.tune_load(str(table))
    assert fp.variant_for_dict(dc.dict, 1 << 22) == builtin
    fp.tune_clear()
    with pytest.raises(fp.FastPairError):
        fp.tune_load(str(tmp_path / "missing.txt"))
