"""The multi-GPU bench path on CPU: world_size-2 gloo ranks (the GPU runs use
NCCL with the same calls).  Replicas are independent; the only collective is
the timing contract's max-over-ranks time and sum of decoded bytes, and the
reference arm prints from rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "decoded" (r + 1) GB in 10 * (r + 1) ms
    ms, nbytes = bench.combine_ranks(dist, 10.0 * (rank + 1), float((rank + 1) * 10**9), torch.device("cpu"))
    out_q.put((rank, ms, nbytes))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_gloo_world_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, nbytes in res:
        assert ms == 20.0            # the slowest rank's time
        assert nbytes == 3.0e9       # all ranks' bytes


def test_combine_ranks_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(None, 5.0, 7.0, None) == (5.0, 7.0)


def test_reference_arm_under_torchrun_prints_from_rank_0_only():
    """Two ranks through torchrun (gloo rendezvous on 127.0.0.1); rank 1 exits
    without work, rank 0 prints one reference line."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--workload", "onpair16_100k",
           "--ref-seconds", "0.2"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["cpu_baseline"]["kind"] == "oracle"
