"""Replay stress of the batched decode: both mixed-codec batches of the
batch parity test, every compiled configuration, one plan each replayed 200
times.  The first replay is compared with the oracle byte for byte and
offset for offset; every later replay (outputs cleared to a guard pattern
before each) must reproduce it exactly on the device, with status OK and
the right per-chunk totals.  A failure names the configuration, the replay
and the chunk."""
import numpy as np
import pytest

from test_gpu_batch import GUARD, mixed_items, run_plan

pytestmark = pytest.mark.gpu

REPLAYS = 200


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_15034_gb300 as m
    return m


@pytest.mark.parametrize("seed", [0, 1])
def test_batch_replays_are_stable(fp, seed):
    import torch
    items = mixed_items(fp, seed)
    for cfg in range(fp.batch_config_count()):
        plan, st, sts, tot = run_plan(fp, items, config=cfg)
        assert st == fp.OK, (cfg, fp.last_error())
        for it, t in zip(items, tot):
            assert int(t) == it.ref.total, (cfg, it.col.name)
            it.check(f"config {cfg} replay 0")
        ref_out = [it.out.clone() for it in items]
        ref_offs = [it.offs.clone() for it in items]
        for r in range(1, REPLAYS):
            for it in items:
                it.out.fill_(GUARD)
                it.offs.fill_(-1)
            plan.decode()
            st, sts, tot = plan.sync_status()
            assert st == fp.OK, (cfg, r, fp.STATUS_NAMES.get(st), fp.last_error())
            for k, it in enumerate(items):
                ok = torch.equal(it.out, ref_out[k]) and torch.equal(it.offs, ref_offs[k])
                if not ok:
                    offs_h = it.offs.cpu().numpy().view(np.uint32)
                    bad = np.nonzero(offs_h[:it.n + 1] != it.ref.offsets)[0]
                    raise AssertionError(f"config {cfg} replay {r} chunk {k} ({it.col.name}, {it.n} strings): "
                                         f"{bad.size} offsets differ, first at {bad[:5].tolist()}")
                assert int(tot[k]) == it.ref.total
        plan.destroy()
