"""GPU parity: the CUDA path, called through the C ABI, against the CPU
oracle, byte for byte and offset for offset (decoding is exact; there is no
tolerance).  Sizes span several tiles with ragged tails; adversarial cases
cover empty inputs, tile-edge alignments, FSST-8 escape runs and errors.
Every codec: OnPair-16, OnPair-12, FSST-8 and FSST-12 (the paper's
escape-free 12-bit codec, Sec. 2.1)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import DeviceColumn, assert_same, make_column, oracle_decode

pytestmark = pytest.mark.gpu

ONPAIR16, ONPAIR12, FSST8, FSST12 = synth.ONPAIR16, synth.ONPAIR12, synth.FSST8, synth.FSST12
CODECS = [ONPAIR16, ONPAIR12, FSST8, FSST12]


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_15034_gb300 as m
    yield m
    for c in CODECS:
        m.variant_select(c, -1)


def variants(fp, codec):
    return list(range(fp.variant_count(codec)))


def each_variant(fp, codec):
    """Select every compiled variant of the codec in turn (block pipeline and
    warp tiles, every tile shape), then restore the defaults."""
    try:
        for v in variants(fp, codec):
            fp.variant_select(codec, v)
            yield v
    finally:
        fp.variant_select(codec, -1)


@pytest.mark.parametrize("codec", CODECS)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_generated_columns_all_variants(fp, codec, seed):
    n = {ONPAIR16: 7001, ONPAIR12: 3001, FSST8: 9001, FSST12: 8001}[codec]
    col = synth.column(codec, seed, n)
    dc = DeviceColumn(col)
    for v in variants(fp, codec):
        fp.variant_select(codec, v)
        assert_same(col, dc)
    fp.variant_select(codec, -1)


@pytest.mark.parametrize("codec", CODECS)
def test_plain_baseline_matches_oracle(fp, codec):
    col = synth.column(codec, 11, 5000)
    assert_same(col, plain=True)


@pytest.mark.parametrize("codec", CODECS)
def test_decoded_size(fp, codec):
    col = synth.column(codec, 12, 4000)
    dc = DeviceColumn(col)
    st, total = fp.decoded_size(codec, dc.dict, dc.codes.data_ptr(), dc.codes_bytes, dc.code_offsets.data_ptr(),
                                dc.n_strings)
    assert st == fp.OK
    assert total == oracle_decode(col).total


@pytest.mark.parametrize("codec", CODECS)
def test_deterministic(fp, codec):
    col = synth.column(codec, 13, 6000)
    dc = DeviceColumn(col)
    a = dc.decode()
    b = dc.decode()
    assert a[0] == b[0] == fp.OK
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(a[2], b[2])


# --------------------------------------------------------------------------
# adversarial shapes
# --------------------------------------------------------------------------

def _tokens(codec, rng, n, lo=1, hi=None):
    hi = hi or synth.MAX_TOKEN[codec]
    return [bytes(rng.integers(0, 256, int(rng.integers(lo, hi + 1))).tolist()) for _ in range(n)]


@pytest.mark.parametrize("codec", CODECS)
def test_empty_column(fp, codec):
    for _ in each_variant(fp, codec):
        col = make_column(codec, [b"ab"], [], [0])
        assert_same(col)
        col = make_column(codec, [b"ab"], [], [0, 0, 0, 0])
        assert_same(col)


@pytest.mark.parametrize("codec", CODECS)
def test_single_long_string_spans_many_tiles(fp, codec):
    rng = np.random.default_rng(5)
    toks = _tokens(codec, rng, 200 if codec != FSST8 else 200)
    slots = rng.integers(0, len(toks), 70001)
    col = make_column(codec, toks, slots, [0, slots.size])
    dc = DeviceColumn(col)
    for v in variants(fp, codec):
        fp.variant_select(codec, v)
        assert_same(col, dc)
    fp.variant_select(codec, -1)


@pytest.mark.parametrize("codec", CODECS)
@pytest.mark.parametrize("tok_len", ["one", "max"])
def test_uniform_token_lengths(fp, codec, tok_len):
    rng = np.random.default_rng(6)
    L = 1 if tok_len == "one" else synth.MAX_TOKEN[codec]
    toks = _tokens(codec, rng, 100, L, L)
    slots = rng.integers(0, 100, 40000)
    cuts = np.sort(rng.integers(0, slots.size, 3000))
    offs = np.concatenate([[0], cuts, [slots.size]])
    col = make_column(codec, toks, slots, offs)
    dc = DeviceColumn(col)
    for v in variants(fp, codec):
        fp.variant_select(codec, v)
        assert_same(col, dc)
    fp.variant_select(codec, -1)


@pytest.mark.parametrize("codec", CODECS)
def test_many_empty_strings_and_tile_edges(fp, codec):
    rng = np.random.default_rng(7)
    toks = _tokens(codec, rng, 50)
    n_slots = 3 * 8192 + 5
    slots = rng.integers(0, 50, n_slots)
    # boundaries at every multiple of 256 (tile edges of every variant), repeated
    edges = np.arange(0, n_slots, 256)
    cuts = np.sort(np.concatenate([edges, edges, rng.integers(0, n_slots, 500), [n_slots] * 3]))
    offs = np.concatenate([[0], cuts])
    col = make_column(codec, toks, slots, offs)
    dc = DeviceColumn(col)
    for v in variants(fp, codec):
        fp.variant_select(codec, v)
        assert_same(col, dc)
    fp.variant_select(codec, -1)


@pytest.mark.parametrize("codec", CODECS)
def test_output_size_residues_mod_16(fp, codec):
    rng = np.random.default_rng(8)
    toks = _tokens(codec, rng, 30)
    for r in range(16):
        for n_slots in (1, 7, 300, 5000):
            slots = rng.integers(0, 30, n_slots)
            col = make_column(codec, toks, slots, [0, n_slots])
            D = oracle_decode(col).total
            # trim or pad with a 1-byte token to land on residue r
            lens = [len(t) for t in toks]
            one = next((i for i, L in enumerate(lens) if L == 1), None)
            if one is None:
                toks2 = toks + [b"z"]
                one = len(toks2) - 1
            else:
                toks2 = toks
            extra = (r - D) % 16
            slots2 = np.concatenate([slots, np.full(extra, one)])
            col2 = make_column(codec, toks2, slots2, [0, slots2.size])
            assert oracle_decode(col2).total % 16 == r
            dc = DeviceColumn(col2)
            for _ in each_variant(fp, codec):
                assert_same(col2, dc)


@pytest.mark.parametrize("codec", CODECS)
@pytest.mark.parametrize("start", [1, 3, 255, 256, 2047, 2048, 2049, 4095, 4096, 8191])
def test_slices_with_nonzero_first_offset(fp, codec, start):
    col = synth.column(codec, 21, 4000)
    # cut the column at the first string boundary >= start, plus a raw start
    dc = DeviceColumn(col)
    import torch
    full = oracle_decode(col)
    co = col.code_offsets
    i0 = int(np.searchsorted(co, start))
    i1 = min(co.size - 1, i0 + 1500)
    sub = co[i0:i1 + 1].copy()
    t = torch.from_numpy(sub.view(np.int32)).cuda()
    for _ in each_variant(fp, codec):
        st, data, offs, guard_ok, _ = dc.decode(code_offsets=t, n_strings=sub.size - 1)
        assert st == fp.OK and guard_ok
        base = full.offsets[i0]
        np.testing.assert_array_equal(offs, full.offsets[i0:i1 + 1] - base)
        np.testing.assert_array_equal(data, full.data[base:full.offsets[i1]])
        # a slice that starts at an arbitrary (odd) slot inside a string
        if codec != FSST8:
            sub2 = np.array([start, start + 17, start + 900], np.uint32)
            col2 = synth.Column(codec, col.dictionary, col.stream, sub2, col.n_slots)
            assert_same(col2, dc, code_offsets=torch.from_numpy(sub2.view(np.int32)).cuda(), n_strings=2)


def test_fsst8_escape_runs_across_tiles(fp):
    rng = np.random.default_rng(9)
    toks = [b"ab", b"c", b"defgh", b"\xff\xfe"]
    units = []
    # long runs of escaped 0xFF (255 255 pairs) and escaped other bytes
    for _ in range(4000):
        k = int(rng.integers(0, 10))
        if k < 3:
            units += [255, 255] * int(rng.integers(1, 40))
        elif k < 5:
            units += [255, int(rng.integers(0, 256))]
        else:
            units.append(int(rng.integers(0, len(toks))))
    # string boundaries only at unit starts
    starts = [0]
    i = 0
    unit_starts = []
    while i < len(units):
        unit_starts.append(i)
        i += 2 if units[i] == 255 else 1
    cuts = sorted(rng.choice(unit_starts, 600, replace=False).tolist())
    offs = np.array(sorted(set([0] + cuts + [len(units)])), np.uint32)
    col = make_column(FSST8, toks, units, offs)
    dc = DeviceColumn(col)
    for v in variants(fp, FSST8):
        fp.variant_select(FSST8, v)
        assert_same(col, dc)
    fp.variant_select(FSST8, -1)
    # shift the whole stream so escape runs straddle every tile offset
    for shift in (1, 2, 15, 16, 17, 255):
        pad = [0] * shift
        col2 = make_column(FSST8, toks, pad + units, np.concatenate([[0], offs + shift]))
        dc2 = DeviceColumn(col2)
        for _ in each_variant(fp, FSST8):
            assert_same(col2, dc2)


# --------------------------------------------------------------------------
# errors: reported through fp_sync_status, writes stay in bounds
# --------------------------------------------------------------------------

@pytest.mark.parametrize("codec", [ONPAIR16, ONPAIR12, FSST12])
def test_corrupt_code(fp, codec):
    col = make_column(codec, [b"a", b"bc"], [0, 1, 5, 1] * 3000, [0, 6000, 12000])
    dc = DeviceColumn(col)
    for _ in each_variant(fp, codec):
        st, _, _, guard_ok, _ = dc.decode(capacity=40000)
        assert st == fp.ERR_CORRUPT and guard_ok


def test_dangling_escape(fp):
    col = make_column(FSST8, [b"a", b"bc"], [0, 1, 255, 1, 0], [0, 3, 5])
    dc = DeviceColumn(col)
    for _ in each_variant(fp, FSST8):
        st, _, _, guard_ok, _ = dc.decode(capacity=100)
        assert st == fp.ERR_CORRUPT and guard_ok


@pytest.mark.parametrize("codec", CODECS)
def test_bad_code_offsets(fp, codec):
    toks = [b"a", b"bc"]
    col = make_column(codec, toks, [0, 1] * 5000, [0, 4000, 3000, 10000])
    col2 = make_column(codec, toks, [0, 1] * 50, [0, 60, 150])
    dc, dc2 = DeviceColumn(col), DeviceColumn(col2)
    for _ in each_variant(fp, codec):
        st, _, _, guard_ok, _ = dc.decode(capacity=30000)
        assert st == fp.ERR_CORRUPT and guard_ok
        st, _, _, guard_ok, _ = dc2.decode(capacity=30000)
        assert st == fp.ERR_CORRUPT and guard_ok


@pytest.mark.parametrize("codec", CODECS)
def test_capacity(fp, codec):
    col = synth.column(codec, 31, 3000)
    total = oracle_decode(col).total
    dc = DeviceColumn(col)
    for _ in each_variant(fp, codec):
        for cap in (0, 1, total // 2, total - 1):
            st, _, _, guard_ok, _ = dc.decode(capacity=cap)
            assert st == fp.ERR_CAPACITY and guard_ok, cap
        assert_same(col, dc, capacity=total)


def test_argument_errors(fp):
    import torch
    col = synth.column(ONPAIR12, 1, 100)
    dc = DeviceColumn(col)
    out = torch.zeros(100000, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(101, dtype=torch.int32, device="cuda")
    # misaligned code buffer
    st = fp.decode(ONPAIR12, dc.dict, dc.codes.data_ptr() + 1, dc.codes_bytes - 1, dc.code_offsets.data_ptr(), 100,
                   out.data_ptr(), 100000, offs.data_ptr(), check=False)
    assert st == fp.ERR_ARG
    # codec / dictionary mismatch
    st = fp.decode(ONPAIR16, dc.dict, dc.codes.data_ptr(), dc.codes_bytes, dc.code_offsets.data_ptr(), 100,
                   out.data_ptr(), 100000, offs.data_ptr(), check=False)
    assert st == fp.ERR_ARG
    # bad dictionary
    with pytest.raises(fp.FastPairError):
        fp.Dict(FSST8, np.frombuffer(b"123456789", np.uint8), np.array([0, 9], np.uint32))
    assert fp.sync_status() == fp.OK


def test_two_streams_concurrently(fp):
    import torch
    a = synth.column(ONPAIR12, 41, 20000)
    b = synth.column(FSST8, 42, 20000)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    da, db = DeviceColumn(a), DeviceColumn(b)
    ra = oracle_decode(a)
    rb = oracle_decode(b)
    outs = []
    for dc, ref, s in ((da, ra, s1), (db, rb, s2)):
        out = torch.zeros(ref.total, dtype=torch.uint8, device="cuda")
        offs = torch.zeros(dc.n_strings + 1, dtype=torch.int32, device="cuda")
        fp.decode(dc.codec, dc.dict, dc.codes.data_ptr(), dc.codes_bytes, dc.code_offsets.data_ptr(), dc.n_strings,
                  out.data_ptr(), ref.total, offs.data_ptr(), s.cuda_stream)
        outs.append((out, offs, ref, s))
    for out, offs, ref, s in outs:
        assert fp.sync_status(s.cuda_stream) == fp.OK
        np.testing.assert_array_equal(out.cpu().numpy(), ref.data)
        np.testing.assert_array_equal(offs.cpu().numpy().view(np.uint32), ref.offsets)


# --------------------------------------------------------------------------
# dictionary read width W (paper Sec. 3.2 split planes, Sec. 4.3 rule)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("codec", [ONPAIR16, ONPAIR12])
def test_read_width_from_the_dictionary_and_both_widths_decode_alike(fp, codec):
    rng = np.random.default_rng(40 + codec)
    short = _tokens(codec, rng, 300, 1, 8)
    long_ = _tokens(codec, rng, 300, 9, 16)
    # the upload reads whole entries (W = 16, the faster width measured on
    # GB300); the paper's rule, applied to the dictionary's token lengths,
    # can set either width
    for toks, w in ((short, 8), (long_, 16), (short[:150] + long_[:150], 8),
                    (short[:119] + long_[:181], 16), (short[:120] + long_[:180], 8)):
        d = fp.Dict(codec, np.frombuffer(b"".join(toks), np.uint8),
                    np.concatenate([[0], np.cumsum([len(t) for t in toks])]).astype(np.uint32))
        assert d.width == 16
        assert fp.width_for_histogram(np.bincount([len(t) for t in toks], minlength=17)) == w, (len(toks), w)
        d.free()
    toks = short[:100] + long_[:200]
    slots = rng.integers(0, len(toks), 60000)
    cuts = np.sort(rng.integers(0, slots.size, 4000))
    col = make_column(codec, toks, slots, np.concatenate([[0], cuts, [slots.size]]))
    dc = DeviceColumn(col)
    assert dc.dict.width == 16
    for w in (16, 8, 16):
        dc.dict.set_width(w)
        assert dc.dict.width == w
        v = fp.variant_for_dict(dc.dict, dc.codes_bytes)
        assert fp.variant_width(codec, v) == w
        assert_same(col, dc)
    with pytest.raises(fp.FastPairError):
        dc.dict.set_width(12)


def test_fsst_dictionaries_read_8_bytes(fp):
    for codec in (FSST8, FSST12):
        col = synth.column(codec, 3, 10)
        d = fp.Dict(codec, col.dictionary.data, col.dictionary.offsets)
        assert d.width == 8
        with pytest.raises(fp.FastPairError):
            d.set_width(16)
        for v in range(fp.variant_count(codec)):
            assert fp.variant_width(codec, v) == 8
        d.free()
