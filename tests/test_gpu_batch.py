"""GPU parity of the batched decode (fp_plan_* / fp_decode_batch): every
chunk of a mixed-codec batch, each with its own dictionary, must equal the
oracle's decode of that chunk byte for byte and offset for offset, for every
compiled configuration and for the tuned one.  Errors stay with their chunk."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import GUARD, GUARD_BYTES, DeviceColumn, make_column, oracle_decode

pytestmark = pytest.mark.gpu

ONPAIR16, ONPAIR12, FSST8 = synth.ONPAIR16, synth.ONPAIR12, synth.FSST8


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_15034_gb300 as m
    return m


class BatchItem:
    """A chunk on the device with guarded output buffers sized by the oracle."""

    def __init__(self, fp, col, code_offsets=None, capacity=None, dc=None):
        import torch
        self.col = col
        self.dc = dc or DeviceColumn(col)
        co_h = col.code_offsets if code_offsets is None else np.asarray(code_offsets, np.uint32)
        self.co_h = co_h
        self.n = int(co_h.size - 1)
        self.co = torch.from_numpy(np.ascontiguousarray(co_h).view(np.int32)).cuda()
        self.ref = oracle.decode(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream, co_h)
        self.capacity = self.ref.total if capacity is None else capacity
        self.out = torch.full((self.capacity + GUARD_BYTES,), GUARD, dtype=torch.uint8, device="cuda")
        self.offs = torch.full((self.n + 1 + 16,), -1, dtype=torch.int32, device="cuda")

    def chunk(self, fp):
        return fp.chunk(self.col.codec, self.dc.dict, self.dc.codes.data_ptr(), self.dc.codes_bytes,
                        self.co.data_ptr(), self.n, self.out.data_ptr(), self.capacity, self.offs.data_ptr())

    def reset(self):
        self.out.fill_(GUARD)
        self.offs.fill_(-1)

    def check_data(self):
        """Output equals the oracle's; nothing written past the offsets array."""
        out_h = self.out.cpu().numpy()
        offs_h = self.offs.cpu().numpy().view(np.uint32)
        assert np.all(out_h[self.capacity:] == GUARD)
        assert np.all(offs_h[self.n + 1:] == 0xFFFFFFFF)
        np.testing.assert_array_equal(offs_h[:self.n + 1], self.ref.offsets)
        np.testing.assert_array_equal(out_h[:self.ref.total], self.ref.data)

    def check(self, ctx=""):
        out_h = self.out.cpu().numpy()
        offs_h = self.offs.cpu().numpy().view(np.uint32)
        name = f"{self.col.name} {ctx}"
        assert np.all(out_h[self.capacity:] == GUARD), f"{name}: write past capacity"
        assert np.all(offs_h[self.n + 1:] == 0xFFFFFFFF), f"{name}: write past offsets"
        data = out_h[:self.ref.total]
        bad_data = np.nonzero(data != self.ref.data)[0]
        np.testing.assert_array_equal(offs_h[:self.n + 1], self.ref.offsets,
                                      err_msg=f"{name} ({bad_data.size} bytes differ too)")
        if bad_data.size:
            raise AssertionError(f"{name}: first differing byte at {int(bad_data[0])} of {data.size}")


def mixed_items(fp, seed=0):
    """Chunks of all three codecs (2:1:1) and very different sizes, each with
    its own dictionary; includes empty chunks, one-string chunks and slices
    whose code_offsets start inside the code buffer."""
    rng = np.random.default_rng(seed)
    items = []
    sizes = [0, 1, 2, 3, 17, 300, 1000, 4097, 20000, 60000]
    codecs = [ONPAIR16, ONPAIR16, ONPAIR12, FSST8]
    k = 0
    for n in sizes:
        for codec in codecs:
            col = synth.column(codec, 100 + seed * 97 + k, max(n, 1))
            k += 1
            if n == 0:
                # no strings: code_offsets = [c] for some slot c
                items.append(BatchItem(fp, col, code_offsets=col.code_offsets[:1]))
            else:
                items.append(BatchItem(fp, col))
    # slices: a window of strings of a larger column, code buffer passed whole
    for codec in (ONPAIR16, ONPAIR12, FSST8):
        col = synth.column(codec, 300 + seed + codec, 12000)
        dc = DeviceColumn(col)
        a = int(rng.integers(1, 4000))
        b = int(rng.integers(a + 1, 11000))
        items.append(BatchItem(fp, col, code_offsets=col.code_offsets[a:b + 1], dc=dc))
    return items


def run_plan(fp, items, **kw):
    plan = fp.Plan([it.chunk(fp) for it in items], **kw)
    for it in items:
        it.reset()
    plan.decode()
    st, sts, tot = plan.sync_status()
    return plan, st, sts, tot


@pytest.mark.parametrize("seed", [0, 1])
def test_batch_every_config_matches_oracle(fp, seed):
    items = mixed_items(fp, seed)
    for cfg in range(fp.batch_config_count()):
        plan, st, sts, tot = run_plan(fp, items, config=cfg)
        assert st == fp.OK, (cfg, fp.last_error())
        assert np.all(sts == 0)
        for it, t in zip(items, tot):
            assert int(t) == it.ref.total
            it.check(f"config {cfg}")
        plan.destroy()


def test_batch_tuned_and_cache(fp, tmp_path):
    items = mixed_items(fp, 2)
    cache = str(tmp_path / "tune.txt")
    plan, st, sts, _ = run_plan(fp, items, tune_cache=cache)
    assert st == fp.OK, fp.last_error()
    info = plan.info()
    assert not info["from_cache"]
    assert all(ms > 0 for ms in info["tune_ms"]), info
    for it in items:
        it.check()
    plan.destroy()
    with open(cache) as f:
        lines = f.read().split()
    assert len(lines) == 2 and int(lines[1]) == info["config"]
    plan2, st, _, _ = run_plan(fp, items, tune_cache=cache)
    assert st == fp.OK
    assert plan2.info()["from_cache"] and plan2.info()["config"] == info["config"]
    for it in items:
        it.check()


def test_batch_graph_replay_follows_inputs(fp):
    """A plan binds buffers, not contents: refilling the code buffers between
    replays decodes the new contents."""
    import torch
    items = []
    for c in (ONPAIR16, ONPAIR12, FSST8):
        col = synth.column(c, 500 + c, 5000)
        ref_total = oracle_decode(col).total
        items.append(BatchItem(fp, col, capacity=2 * ref_total + 4096))
    plan = fp.Plan([it.chunk(fp) for it in items], config=0)
    for _ in range(3):
        for it in items:
            it.reset()
        plan.decode()
        st, _, tot = plan.sync_status()
        assert st == fp.OK
        for it, t in zip(items, tot):
            assert int(t) == it.ref.total
            it.check_data()
    # same dictionaries and string boundaries, new codes
    rng = np.random.default_rng(7)
    for it in items:
        col = it.col
        if col.codec == FSST8:
            slots = col.stream.copy()
            plain = (slots != 255) & ~col.slot_is_literal   # symbol codes only: escapes stay valid
            slots[plain] = rng.integers(0, 255, int(plain.sum()))
            new_stream = slots
        else:
            codes = rng.integers(0, col.dictionary.n_entries, col.n_slots).astype(np.uint16)
            new_stream = synth.pack16(codes) if col.codec == ONPAIR16 else synth.pack12(codes)
        assert new_stream.size == it.dc.codes_bytes
        it.dc.codes[:new_stream.size].copy_(torch.from_numpy(np.ascontiguousarray(new_stream)).cuda())
        it.ref = oracle.decode(col.codec, col.dictionary.data, col.dictionary.offsets, new_stream, it.co_h)
        assert it.ref.status == oracle.OK and it.ref.total <= it.capacity
    for it in items:
        it.reset()
    plan.decode()
    st, _, tot = plan.sync_status()
    assert st == fp.OK
    for it, t in zip(items, tot):
        assert int(t) == it.ref.total
        it.check_data()


def test_batch_errors_stay_with_their_chunk(fp):
    good = [BatchItem(fp, synth.column(c, 600 + c, 3000)) for c in (ONPAIR16, ONPAIR12, FSST8)]
    # corrupt: an OnPair-12 code beyond a 300-entry dictionary
    toks = [bytes([65 + i % 26]) * (1 + i % 5) for i in range(300)]
    slots = [1, 2, 299, 3000, 4, 5]
    bad_col = make_column(ONPAIR12, toks, slots, [0, 3, 6], name="corrupt")
    import torch
    dc_bad = DeviceColumn(bad_col)
    co = torch.from_numpy(bad_col.code_offsets.view(np.int32)).cuda()
    out_bad = torch.zeros(256, dtype=torch.uint8, device="cuda")
    offs_bad = torch.zeros(8, dtype=torch.int32, device="cuda")
    corrupt = fp.chunk(ONPAIR12, dc_bad.dict, dc_bad.codes.data_ptr(), dc_bad.codes_bytes, co.data_ptr(), 2,
                       out_bad.data_ptr(), 128, offs_bad.data_ptr())
    # capacity: a good column with too small an output buffer
    cap_item = BatchItem(fp, synth.column(FSST8, 610, 2000))
    cap_chunk = fp.chunk(FSST8, cap_item.dc.dict, cap_item.dc.codes.data_ptr(), cap_item.dc.codes_bytes,
                         cap_item.co.data_ptr(), cap_item.n, cap_item.out.data_ptr(), cap_item.ref.total // 2,
                         cap_item.offs.data_ptr())
    chunks = [good[0].chunk(fp), corrupt, good[1].chunk(fp), cap_chunk, good[2].chunk(fp)]
    for cfg in range(fp.batch_config_count()):
        plan = fp.Plan(chunks, config=cfg)
        for it in good:
            it.reset()
        cap_item.reset()
        plan.decode()
        st, sts, _ = plan.sync_status()
        assert st == fp.ERR_CORRUPT
        assert list(sts) == [fp.OK, fp.ERR_CORRUPT, fp.OK, fp.ERR_CAPACITY, fp.OK]
        for it in good:
            it.check()
        # capacity: nothing written past the declared capacity
        out_h = cap_item.out.cpu().numpy()
        assert np.all(out_h[cap_item.ref.total // 2:] == GUARD)
        # the status was cleared by the read
        plan.decode()
        st2, sts2, _ = plan.sync_status()
        assert list(sts2) == list(sts)
        plan.destroy()


def test_batch_rejects_bad_arguments(fp):
    import torch
    col = synth.column(ONPAIR16, 700, 100)
    it = BatchItem(fp, col)
    with pytest.raises(fp.FastPairError):
        fp.Plan([], config=0)
    c = it.chunk(fp)
    c.codec = ONPAIR12   # dictionary codec mismatch
    with pytest.raises(fp.FastPairError):
        fp.Plan([c], config=0)
    c = it.chunk(fp)
    c.d_out_bytes = it.out.data_ptr() + 1   # misaligned output
    with pytest.raises(fp.FastPairError):
        fp.Plan([c], config=0)
    with pytest.raises(fp.FastPairError):
        fp.Plan([it.chunk(fp)], config=fp.batch_config_count())


def test_batch_large_chunks(fp):
    """Chunks spanning hundreds of tiles next to tiny ones."""
    items = [BatchItem(fp, synth.column(ONPAIR12, 800, 150000)),
             BatchItem(fp, synth.column(FSST8, 801, 7)),
             BatchItem(fp, synth.column(ONPAIR16, 802, 120000)),
             BatchItem(fp, synth.column(FSST8, 803, 200000)),
             BatchItem(fp, synth.column(ONPAIR16, 804, 1))]
    for cfg in range(fp.batch_config_count()):
        plan, st, sts, tot = run_plan(fp, items, config=cfg)
        assert st == fp.OK, fp.last_error()
        for it in items:
            it.check()
        plan.destroy()


def test_batch_with_fsst12_chunks(fp):
    """FSST-12 chunks (the paper's escape-free 12-bit codec) in a mixed batch:
    decoded by every warp-tile configuration like the other codecs; the
    block-pipeline configurations, which have no FSST-12 queue, reject the
    plan, and the tuner skips them."""
    FSST12 = synth.FSST12
    items = mixed_items(fp, 3)
    for k, n in enumerate((1, 2, 700, 20000, 90000)):
        items.append(BatchItem(fp, synth.column(FSST12, 950 + k, n)))
    col = synth.column(FSST12, 960, 12000)
    items.append(BatchItem(fp, col, code_offsets=col.code_offsets[777:9001 + 1]))
    items.append(BatchItem(fp, col, code_offsets=col.code_offsets[5:6]))   # no strings
    chunks = [it.chunk(fp) for it in items]
    for cfg in range(fp.batch_config_count()):
        if not fp.batch_config_info(cfg)["warp_tiles"]:
            with pytest.raises(fp.FastPairError):
                fp.Plan(chunks, config=cfg)
            continue
        plan, st, sts, tot = run_plan(fp, items, config=cfg)
        assert st == fp.OK, (cfg, fp.last_error())
        assert plan.info()["slots_per_thread_fsst12"] > 0
        for it, t in zip(items, tot):
            assert int(t) == it.ref.total
            it.check(f"config {cfg}")
        plan.destroy()
    plan, st, _, _ = run_plan(fp, items)
    assert st == fp.OK
    info = plan.info()
    assert fp.batch_config_info(info["config"])["warp_tiles"]
    for c, ms in enumerate(info["tune_ms"]):
        assert (ms > 0) == fp.batch_config_info(c)["warp_tiles"], (c, ms)
    for it in items:
        it.check("tuned")
    plan.destroy()
