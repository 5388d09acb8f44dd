"""Failure detection without a fault: the bounded look-back waits really run
out.  fp_debug_stall_next makes the next decode skip the first ticket of its
ticketed pass, so the first look-back word is never published (a flag that
nothing sets); the look-back that needs it must give up after the short
poll limit the hook sets, the call must report FP_ERR_TIMEOUT through
fp_sync_status with every write inside the caller's buffers, and the next
decode on the same stream must be normal and equal the oracle's.

Columns span several tickets: more than 2,048 warp tiles (two tile-scan
blocks) for the warp-tile decoder, and several 4,096-slot tiles for the
block pipeline.  The one-launch decode's first grid barrier is made to
wait for an arrival count no grid reaches."""
import numpy as np
import pytest

import synth
from gpu_util import DeviceColumn, oracle_decode

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fp():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2609_15034_gb300 as m
    yield m
    for c in (synth.ONPAIR16, synth.ONPAIR12, synth.FSST8, synth.FSST12):
        m.variant_select(c, -1)


def variant_with_launches(fp, codec, launches):
    for v in range(fp.variant_count(codec)):
        if fp.variant_info(codec, v)["launches_per_call"] == launches:
            return v
    raise AssertionError(f"no variant with {launches} launches per call")


@pytest.mark.parametrize("codec,n,launches", [
    (synth.ONPAIR16, 60_000, 3),    # warp tiles: ~1.2M slots, 2,300 warp tiles of 512
    (synth.FSST8, 200_000, 3),      # ~2.4M slots: 2,400 warp tiles of 1,024
    (synth.ONPAIR12, 30_000, 2),    # block pipeline: ~0.5M slots, 130 block tiles of 4,096
    (synth.ONPAIR16, 20_000, 1),    # one cooperative launch: its first grid barrier
    (synth.FSST12, 20_000, 1),
])
def test_lookback_gives_up_then_recovers(fp, codec, n, launches):
    import torch
    col = synth.column(codec, 900 + codec, n)
    fp.variant_select(codec, variant_with_launches(fp, codec, launches))
    try:
        dc = DeviceColumn(col)
        ref = oracle_decode(col)
        assert ref.total > 0
        # a normal call first: it creates the stream's workspace
        st, data, offs, guard_ok, _ = dc.decode(capacity=ref.total)
        assert st == fp.OK and guard_ok
        # stalled call: the look-back must give up after 64 polls
        assert fp.debug_stall_next(64) == fp.OK
        st, _, _, guard_ok, launch = dc.decode(capacity=ref.total)
        assert launch == fp.OK
        assert st == fp.ERR_TIMEOUT, (fp.STATUS_NAMES.get(st), fp.last_error())
        assert guard_ok, "a write left the caller's buffers"
        # the status was read and cleared; the next call is normal
        st, data, offs, guard_ok, _ = dc.decode(capacity=ref.total)
        assert st == fp.OK, fp.last_error()
        assert guard_ok
        np.testing.assert_array_equal(offs, ref.offsets)
        assert np.array_equal(data, ref.data)
        torch.cuda.synchronize()
    finally:
        fp.variant_select(codec, -1)


def test_stall_hook_arguments(fp):
    import torch
    s = torch.cuda.Stream()
    # no workspace on a fresh stream yet
    assert fp.debug_stall_next(64, s) == fp.ERR_ARG
    assert fp.debug_stall_next(0) == fp.ERR_ARG
    assert fp.debug_stall_next((1 << 20) + 1) == fp.ERR_ARG
