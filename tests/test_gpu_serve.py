"""GPU tests of the served decode (fp_serve_*): every request's result equals
the oracle's decode, alone and in a mix of concurrent requests; admission
respects the HBM budget; the dictionary cache evicts and reloads; errors stay
with their request."""
import threading
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

ONPAIR16, ONPAIR12, FSST8 = synth.ONPAIR16, synth.ONPAIR12, synth.FSST8


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_15034_gb300 as m
    return m


class Page:
    """A column on the device and the oracle's decode of it."""

    def __init__(self, col, key):
        import torch
        self.col = col
        self.key = key
        s = np.ascontiguousarray(col.stream, np.uint8)
        self.codes_bytes = int(s.size)
        self.codes = torch.from_numpy(s if s.size else np.zeros(16, np.uint8)).cuda()
        self.co = torch.from_numpy(np.ascontiguousarray(col.code_offsets, np.uint32).view(np.int32)).cuda()
        self.n = col.n_strings
        self.ref = oracle.decode(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets)
        assert self.ref.status == oracle.OK

    def submit(self, srv, tag=0, decoded_size=None, check=True):
        return srv.submit(self.key, self.codes.data_ptr(), self.codes_bytes, self.co.data_ptr(), self.n,
                          self.ref.total if decoded_size is None else decoded_size, tag, check=check)


def fetch(fp, res):
    data = fp.device_bytes(res["d_out_bytes"], res["bytes"]).cpu().numpy()
    offs = fp.device_bytes(res["d_out_offsets"], (res["n_strings"] + 1) * 4).cpu().numpy().view(np.uint32)
    return data, offs


def make_pages(seed=0, count=24):
    rng = np.random.default_rng(seed)
    pages = []
    for i in range(count):
        codec = [ONPAIR16, ONPAIR16, ONPAIR12, FSST8][i % 4]
        n = int(np.exp(rng.uniform(np.log(1), np.log(40000))))
        col = synth.column(codec, 900 + seed * 131 + i, n)
        pages.append(Page(col, key=1000 * seed + i))
    return pages


def register(srv, pages):
    for p in pages:
        d = p.col.dictionary
        srv.dict_put(p.key, p.col.codec, d.data, d.offsets)


def collect(fp, srv, n_expected, timeout=60.0):
    got = {}
    t_end = time.time() + timeout
    while len(got) < n_expected and time.time() < t_end:
        for r in srv.poll(timeout_s=0.05):
            got[r["ticket"]] = r
    assert len(got) == n_expected, f"{len(got)} of {n_expected} requests completed"
    return got


def test_serve_results_match_oracle(fp):
    pages = make_pages(0)
    srv = fp.Server(hbm_budget=1 << 30, dict_cache_slots=64, n_streams=4, max_wave=8)
    register(srv, pages)
    tickets = {p.submit(srv, tag=i): i for i, p in enumerate(pages)}
    got = collect(fp, srv, len(pages))
    for t, r in got.items():
        p = pages[tickets[t]]
        assert r["status"] == fp.OK and r["user_tag"] == tickets[t]
        assert r["bytes"] == p.ref.total
        data, offs = fetch(fp, r)
        np.testing.assert_array_equal(offs, p.ref.offsets)
        np.testing.assert_array_equal(data, p.ref.data)
        assert r["t_submit_ns"] <= r["t_admit_ns"] <= r["t_done_ns"]
        srv.release(t)
    st = srv.stats()
    assert st["completed"] == st["submitted"] == st["released"] == len(pages)
    assert st["failed"] == 0 and st["inflight_bytes"] == 0 and st["inflight_requests"] == 0
    assert st["bytes_decoded"] == sum(p.ref.total for p in pages)
    srv.destroy()


def test_serve_alone_equals_in_the_mix(fp):
    """Each request decoded alone (one stream, waves of one, submitted one at a
    time) and in a concurrent mix (four streams, waves of up to 16, all
    submitted at once from several threads) gives the same bytes."""
    pages = make_pages(1, count=32)
    alone = {}
    srv = fp.Server(hbm_budget=1 << 30, dict_cache_slots=64, n_streams=1, max_wave=1)
    register(srv, pages)
    for i, p in enumerate(pages):
        t = p.submit(srv, tag=i)
        r = collect(fp, srv, 1)[t]
        assert r["status"] == fp.OK
        alone[i] = fetch(fp, r)
        srv.release(t)
    srv.destroy()

    srv = fp.Server(hbm_budget=1 << 30, dict_cache_slots=64, n_streams=4, max_wave=16)
    register(srv, pages)
    tickets = {}
    lock = threading.Lock()

    def client(idx):
        for i in idx:
            t = pages[i].submit(srv, tag=i)
            with lock:
                tickets[t] = i

    ths = [threading.Thread(target=client, args=(list(range(k, len(pages), 4)),)) for k in range(4)]
    for th in ths:
        th.start()
    for th in ths:
        th.join()
    got = collect(fp, srv, len(pages))
    waves = srv.stats()["waves"]
    for t, r in got.items():
        i = tickets[t]
        assert r["status"] == fp.OK
        data, offs = fetch(fp, r)
        np.testing.assert_array_equal(data, alone[i][0])
        np.testing.assert_array_equal(offs, alone[i][1])
        np.testing.assert_array_equal(data, pages[i].ref.data)
        srv.release(t)
    assert waves < len(pages)   # requests were batched
    srv.destroy()


def test_serve_budget_backpressure(fp):
    pages = make_pages(2, count=16)
    biggest = max(p.ref.total + 4 * (p.n + 1) + p.codes_bytes + p.n * 4 for p in pages)
    budget = 2 * biggest + (1 << 16)
    srv = fp.Server(hbm_budget=budget, dict_cache_slots=64, n_streams=3, max_wave=4)
    register(srv, pages)
    tickets = {}
    for rep in range(3):
        for i, p in enumerate(pages):
            tickets[p.submit(srv, tag=i)] = i
    done = 0
    t_end = time.time() + 60
    while done < len(tickets) and time.time() < t_end:
        for r in srv.poll(timeout_s=0.05):
            assert r["status"] == fp.OK
            i = tickets[r["ticket"]]
            data, _ = fetch(fp, r)
            np.testing.assert_array_equal(data, pages[i].ref.data)
            srv.release(r["ticket"])
            done += 1
    assert done == len(tickets)
    st = srv.stats()
    assert st["peak_inflight_bytes"] <= budget
    srv.destroy()


def test_serve_dictionary_cache_evicts_and_reloads(fp):
    pages = make_pages(3, count=12)
    srv = fp.Server(hbm_budget=1 << 30, dict_cache_slots=2, n_streams=2, max_wave=2)
    register(srv, pages)
    order = [i % len(pages) for i in range(3 * len(pages))]
    tickets = {pages[i].submit(srv, tag=i): i for i in order}
    got = collect(fp, srv, len(tickets))
    for t, r in got.items():
        assert r["status"] == fp.OK
        data, offs = fetch(fp, r)
        np.testing.assert_array_equal(data, pages[tickets[t]].ref.data)
        srv.release(t)
    st = srv.stats()
    assert st["dict_evictions"] > 0 and st["dict_misses"] >= len(pages)
    assert st["dict_hits"] + st["dict_misses"] == len(tickets)
    srv.destroy()


def test_serve_errors_stay_with_their_request(fp):
    pages = make_pages(4, count=6)
    srv = fp.Server(hbm_budget=64 << 20, dict_cache_slots=16, n_streams=2, max_wave=8)
    register(srv, pages)
    # a corrupt column: OnPair-12 codes beyond a 300-entry dictionary
    toks = [bytes([65 + i % 26]) * (1 + i % 5) for i in range(300)]
    from gpu_util import make_column
    bad = Page.__new__(Page)
    col = make_column(ONPAIR12, toks, [1, 2, 299, 3000, 4, 5], [0, 3, 6], name="corrupt")
    import torch
    bad.col, bad.key, bad.n = col, 77777, 2
    bad.codes_bytes = int(col.stream.size)
    bad.codes = torch.from_numpy(np.ascontiguousarray(col.stream)).cuda()
    bad.co = torch.from_numpy(col.code_offsets.view(np.int32)).cuda()
    srv.dict_put(bad.key, ONPAIR12, col.dictionary.data, col.dictionary.offsets)
    t_bad = srv.submit(bad.key, bad.codes.data_ptr(), bad.codes_bytes, bad.co.data_ptr(), 2, 64)
    t_cap = pages[0].submit(srv, decoded_size=max(pages[0].ref.total // 2, 1))
    good = {p.submit(srv): p for p in pages}
    # unknown key, too large for the budget
    st, _ = srv.submit(123456789, pages[0].codes.data_ptr(), pages[0].codes_bytes, pages[0].co.data_ptr(),
                       pages[0].n, pages[0].ref.total, check=False)
    assert st == fp.ERR_ARG
    st, _ = pages[1].submit(srv, decoded_size=1 << 30, check=False)
    assert st == fp.ERR_BUSY
    with pytest.raises(fp.FastPairError):
        srv.dict_put(pages[0].key, pages[0].col.codec, pages[0].col.dictionary.data, pages[0].col.dictionary.offsets)
    got = collect(fp, srv, 2 + len(good))
    assert got[t_bad]["status"] == fp.ERR_CORRUPT
    assert got[t_cap]["status"] == fp.ERR_CAPACITY
    for t, p in good.items():
        assert got[t]["status"] == fp.OK
        data, _ = fetch(fp, got[t])
        np.testing.assert_array_equal(data, p.ref.data)
    for t in got:
        srv.release(t)
    assert srv.release(t_bad, check=False) == fp.ERR_ARG   # already released
    srv.destroy()


def test_serve_release_before_poll_is_refused(fp):
    pages = make_pages(5, count=2)
    srv = fp.Server(hbm_budget=1 << 28, dict_cache_slots=8, n_streams=1, max_wave=1)
    register(srv, pages)
    t = pages[0].submit(srv)
    time.sleep(0.5)   # completed by now, but not polled
    assert srv.release(t, check=False) == fp.ERR_NOT_READY
    got = collect(fp, srv, 1)
    assert got[t]["status"] == fp.OK
    srv.release(t)
    srv.destroy()
