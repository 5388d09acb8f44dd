"""GPU parity of the selective decode (fp_rows_size / fp_decode_rows): the
strings of a row-id list, in that order, must equal the oracle's
fpo_decode_rows byte for byte and offset for offset, for every codec and
decoder variant, for selections that are empty, complete, random with
repeats, reversed, or single rows; and the slot count and decoded size
fp_rows_size reports must be the selection's.  Errors: an out-of-range row
id, and a selected_slots bound below the selection, keep every write in
bounds and are reported."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import GUARD, GUARD_BYTES, DeviceColumn

pytestmark = pytest.mark.gpu

CODECS = [synth.ONPAIR16, synth.ONPAIR12, synth.FSST8, synth.FSST12]
N = {synth.ONPAIR16: 6000, synth.ONPAIR12: 5000, synth.FSST8: 9000, synth.FSST12: 8000}


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_15034_gb300 as m
    yield m
    for c in CODECS:
        m.variant_select(c, -1)


def selections(n, rng):
    return {
        "empty": np.zeros(0, np.uint32),
        "all": np.arange(n, dtype=np.uint32),
        "reversed": np.arange(n, dtype=np.uint32)[::-1].copy(),
        "random_repeats": rng.integers(0, n, 3 * n // 2).astype(np.uint32),
        "sparse": np.sort(rng.choice(n, n // 50, replace=False)).astype(np.uint32),
        "one_first": np.array([0], np.uint32),
        "one_last": np.array([n - 1], np.uint32),
        "same_row": np.full(777, n // 3, np.uint32),
    }


class Rows:
    def __init__(self, fp, col: synth.Column):
        self.fp, self.col = fp, col
        self.dc = DeviceColumn(col)

    def run(self, rows, capacity=None, slots=None, check_size=True):
        import torch
        fp, col, dc = self.fp, self.col, self.dc
        m = int(rows.size)
        ids = torch.from_numpy(np.ascontiguousarray(rows if m else np.zeros(1, np.uint32)).view(np.int32)).cuda()
        ref = oracle.decode_rows(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets,
                                 rows)
        if check_size:
            st, got_slots, got_bytes = fp.rows_size(col.codec, dc.dict, dc.codes.data_ptr(), dc.codes_bytes,
                                                   dc.code_offsets.data_ptr(), dc.n_strings, ids.data_ptr(), m)
            assert st == fp.OK, fp.last_error()
            co = col.code_offsets.astype(np.int64)
            assert got_slots == int((co[rows.astype(np.int64) + 1] - co[rows.astype(np.int64)]).sum())
            assert got_bytes == ref.total
            slots = got_slots if slots is None else slots
        cap = ref.total if capacity is None else capacity
        out = torch.full((cap + GUARD_BYTES,), GUARD, dtype=torch.uint8, device="cuda")
        offs = torch.full((m + 1 + 16,), -1, dtype=torch.int32, device="cuda")
        launch = fp.decode_rows(col.codec, dc.dict, dc.codes.data_ptr(), dc.codes_bytes, dc.code_offsets.data_ptr(),
                                dc.n_strings, ids.data_ptr(), m, slots, out.data_ptr(), cap, offs.data_ptr(),
                                check=False)
        assert launch == fp.OK, fp.last_error()
        st = fp.sync_status()
        out_h = out.cpu().numpy()
        offs_h = offs.cpu().numpy().view(np.uint32)
        guard_ok = bool(np.all(out_h[cap:] == GUARD)) and bool(np.all(offs_h[m + 1:] == 0xFFFFFFFF))
        return st, ref, out_h[:cap], offs_h[:m + 1], guard_ok


@pytest.mark.parametrize("codec", CODECS)
def test_selections_match_oracle(fp, codec):
    rng = np.random.default_rng(70 + codec)
    r = Rows(fp, synth.column(codec, 70 + codec, N[codec]))
    for name, rows in selections(N[codec], rng).items():
        st, ref, out, offs, guard_ok = r.run(rows)
        assert ref.status == oracle.OK
        assert st == fp.OK, (name, fp.last_error())
        assert guard_ok, name
        np.testing.assert_array_equal(offs, ref.offsets, err_msg=name)
        assert np.array_equal(out[:ref.total], ref.data), name


@pytest.mark.parametrize("codec", CODECS)
def test_every_variant_on_a_random_selection(fp, codec):
    rng = np.random.default_rng(80 + codec)
    r = Rows(fp, synth.column(codec, 80 + codec, N[codec]))
    rows = rng.integers(0, N[codec], N[codec]).astype(np.uint32)
    try:
        for v in range(fp.variant_count(codec)):
            fp.variant_select(codec, v)
            st, ref, out, offs, guard_ok = r.run(rows)
            assert st == fp.OK and guard_ok, (v, fp.last_error())
            np.testing.assert_array_equal(offs, ref.offsets, err_msg=f"variant {v}")
            assert np.array_equal(out[:ref.total], ref.data), v
    finally:
        fp.variant_select(codec, -1)


@pytest.mark.parametrize("codec", [synth.ONPAIR12, synth.FSST8])
def test_large_selection_across_many_tiles(fp, codec):
    """A selection of 400k rows (several tile-scan blocks of the gathered
    stream), rows drawn with repeats."""
    rng = np.random.default_rng(90 + codec)
    n = 200_000
    r = Rows(fp, synth.column(codec, 90 + codec, n))
    rows = rng.integers(0, n, 2 * n).astype(np.uint32)
    st, ref, out, offs, guard_ok = r.run(rows)
    assert st == fp.OK and guard_ok, fp.last_error()
    np.testing.assert_array_equal(offs, ref.offsets)
    assert np.array_equal(out[:ref.total], ref.data)


def test_bad_row_id_and_small_bound(fp):
    import torch
    codec = synth.ONPAIR12
    col = synth.column(codec, 99, 3000)
    r = Rows(fp, col)
    rows = np.array([5, 17, 3000, 2], np.uint32)   # 3000 is past the last row
    ids = torch.from_numpy(rows.view(np.int32)).cuda()
    dc = r.dc
    st, slots, nbytes = fp.rows_size(codec, dc.dict, dc.codes.data_ptr(), dc.codes_bytes, dc.code_offsets.data_ptr(),
                                     dc.n_strings, ids.data_ptr(), rows.size)
    assert st == fp.ERR_CORRUPT
    assert fp.sync_status() == fp.OK   # the status was read and cleared
    out = torch.full((4096 + GUARD_BYTES,), GUARD, dtype=torch.uint8, device="cuda")
    offs = torch.full((rows.size + 1 + 16,), -1, dtype=torch.int32, device="cuda")
    fp.decode_rows(codec, dc.dict, dc.codes.data_ptr(), dc.codes_bytes, dc.code_offsets.data_ptr(), dc.n_strings,
                   ids.data_ptr(), rows.size, 4096, out.data_ptr(), 4096, offs.data_ptr())
    assert fp.sync_status() == fp.ERR_CORRUPT
    assert np.all(out.cpu().numpy()[4096:] == GUARD)
    assert np.all(offs.cpu().numpy()[rows.size + 1:] == -1)
    # a bound below the selection's slots: reported, writes stay in bounds
    good = np.arange(0, 3000, 7, dtype=np.uint32)
    _, _, _, _, _ = r.run(good)   # sizes it
    co = col.code_offsets.astype(np.int64)
    need = int((co[good + 1] - co[good]).sum())
    st, ref, out_h, offs_h, guard_ok = r.run(good, slots=need // 2, check_size=False)
    assert st in (fp.ERR_CAPACITY, fp.ERR_CORRUPT)
    assert guard_ok
    # and the stream works normally afterwards
    st, ref, out_h, offs_h, guard_ok = r.run(good)
    assert st == fp.OK and guard_ok
    np.testing.assert_array_equal(offs_h, ref.offsets)
