"""Benchmark: decode throughput of a dictionary-compressed string column on
GB300, through the C ABI (libfastpair.so).

One step = one decode of the whole column (code unpack, length scan with
look-back, assembly, string offsets) with inputs resident in HBM.  Prints one
JSON line.  ``--impl reference`` times the CPU oracle instead (on the host
cores, bounded sample of the same workload).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOADS = {
    # name: (codec, n_strings, description)
    "onpair12_10m": (synth.ONPAIR12, 10_000_000,
                     "OnPair-12, 4,096-entry log-token dictionary, 10M strings of 20-200 B, Zipf(1.2)"),
    "fsst8_16m": (synth.FSST8, 16_000_000,
                  "FSST-8 with escapes, 255 URL/identifier symbols, 16M lognormal strings (median 40 B)"),
    "onpair16_100k": (synth.ONPAIR16, 100_000,
                      "OnPair-16, 65,536-entry dictionary, 100k strings of 1-40 codes, Zipf(1.1)"),
    "fsst12_16m": (synth.FSST12, 16_000_000,
                   "FSST-12 (escape-free 12-bit codes), 4,096 URL/identifier symbols of 1-8 B, 16M lognormal "
                   "strings (median 40 B), Zipf(1.0)"),
    "fsst12_packed10_16m": (synth.FSST12, 16_000_000,
                            "FSST-12 with a 1,024-symbol table, codes cascaded: bit-packed at 10 bits and "
                            "unpacked inside the decode (fp_decode_packed); 16M lognormal strings (median 40 B)"),
}
# selective decode: name -> (column workload, rows selected, description)
ROWS_WORKLOADS = {
    "onpair12_10m_rows1m": ("onpair12_10m", 1_000_000,
                            "1M distinct rows in random order out of the OnPair-12 10M-string column (fp_decode_rows: "
                            "row scan, gather of the selected codes, warp-tile decode); the column stays resident"),
}
ROWS_METRIC = "decoded GB/s of the selected rows (selective decode, column resident in HBM)"
# cascaded workloads: name -> (bits per stored code, dictionary entries)
PACKED_WORKLOADS = {"fsst12_packed10_16m": (10, 1024)}
# batched workloads: name -> (chunks, smallest and largest decoded chunk size, description)
BATCH_WORKLOADS = {
    "batched_4096": (4096, 4 << 10, 64 << 20,
                     "4,096 chunks, OnPair-16/OnPair-12/FSST-8 2:1:1, one dictionary each, decoded sizes "
                     "log-uniform 4 KB-64 MB, one persistent launch (CUDA graph)"),
    "batched_4096_16mb": (4096, 4 << 10, 16 << 20,
                          "4,096 chunks, OnPair-16/OnPair-12/FSST-8 2:1:1, one dictionary each, decoded sizes "
                          "log-uniform 4 KB-16 MB, one persistent launch (CUDA graph)"),
}
# served workloads: name -> (arrivals/s, seconds, smallest and largest decoded request, dictionary keys,
#                             HBM budget, description)
SERVE_WORKLOADS = {
    "served": (2000.0, 60.0, 64 << 10, 256 << 20, 512, 40 << 30,
               "Poisson arrivals at 2,000 requests/s, mixed-codec pages (2:1:1) of 64 KB-256 MB decoded "
               "(log-uniform), dictionaries Zipf(1.0) over 512 keys in a 512-slot device cache, 40 GB HBM budget"),
}
METRIC = "decoded GB/s (single-column decode, inputs resident in HBM)"
SERVE_METRIC = "served decode: aggregate decoded GB/s at the offered load, with p50/p99 latency"
SERVE_DEFAULT_CONFIG = 4   # the library's default batch configuration (warp tiles, one block of 16 warps per SM)
BATCH_METRIC = "decoded GB/s (batched decode of many chunks, inputs resident in HBM)"
L2_BYTES = 126 * 1024 * 1024


def combine_ranks(dist, total_ms: float, nbytes: float, device):
    """Whole-job timing of replicas: the slowest rank's time and the bytes
    all ranks decoded (no data-path collective; replicas are independent)."""
    import torch
    if dist is None:
        return total_ms, nbytes
    tt = torch.tensor([total_ms], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    bt = torch.tensor([nbytes], device=device, dtype=torch.float64)
    dist.all_reduce(bt, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(bt.item())


def env_rank():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    return r, w, lr


def algorithmic_bytes(col, total: int, codec: int, bits: int = 0) -> int:
    """Bytes a decode must move at least: the code slots it reads (at `bits`
    bits per code when they are stored bit-packed), the string offsets it
    reads and writes, the output it writes, the dictionary once."""
    co = col.code_offsets
    used_slots = int(co[-1]) - int(co[0])
    code_bytes = (used_slots * (bits or synth.CODE_BITS[codec]) + 7) // 8
    n = col.n_strings
    dict_bytes = col.dictionary.n_entries * (synth.MAX_TOKEN[codec] + 1)
    return code_bytes + 4 * (n + 1) + total + 4 * (n + 1) + dict_bytes


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def tuned_entry(codec: int, width: int, codes_bytes: int, sms: int):
    """The committed tuning table's line for this GPU's SM count, codec, read
    width and size class (floor(log2) of the buffer's code slots), if any:
    the shape the default decode uses and its time when it was tuned."""
    path = os.path.join(ROOT, "paper_2609_15034_gb300", "tuning", "gb300.txt")
    slots = codes_bytes * 8 // synth.CODE_BITS[codec]
    cls = max(slots, 1).bit_length() - 1
    found = None
    try:
        with open(path) as f:
            for ln in f:
                if ln.startswith("#"):
                    continue
                v = ln.split()
                if len(v) == 6 and [int(x) for x in v[:4]] == [sms, codec, width, cls]:
                    found = {"variant": int(v[4]), "ms": float(v[5]), "size_class": cls,
                             "table": "paper_2609_15034_gb300/tuning/gb300.txt"}
    except OSError:
        return None
    return found


def load_traffic(workload: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    a build whose single-column decode sources and flags equal this one's."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        from paper_2609_15034_gb300 import _build
        digest = _build.decode_path_digest()
        with open(path) as f:
            d = json.load(f)
        e = d.get(workload)
        if e and e.get("source_digest") == digest:
            return int(e["dram_bytes_per_launch"])
    except Exception:
        return None
    return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", gpu_id], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.strip().splitlines():
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def workload_column(name: str, seed: int, n: int = 0):
    """The workload's column (n strings; 0: the workload's own count) and, for
    cascaded workloads, its bits per stored code."""
    codec, n_default, _ = WORKLOADS[name]
    n = n or n_default
    if name in PACKED_WORKLOADS:
        bits, n_entries = PACKED_WORKLOADS[name]
        col = synth.fsst12_column(seed, n, dictionary=synth.fsst12_dictionary(seed, n_entries))
        # the stored codes, cascaded: bit-packed at `bits` bits
        return synth.Column(codec, col.dictionary, synth.pack_bits(col.slot_codes, bits), col.code_offsets,
                            col.n_slots, name=col.name), bits
    return synth.column(codec, seed, n), 0


def cpu_oracle_rate(col, target_s: float, threads: int, packed_bits: int = 0):
    """Time the oracle (as it stands) on a bounded prefix of the column (the
    oracle's decode of bit-packed codes runs on one thread)."""
    import oracle
    n = col.n_strings
    # size the sample from a short probe
    probe_n = min(n, 20000)
    co = col.code_offsets

    def dec(m):
        if packed_bits:
            return oracle.decode_packed(col.codec, packed_bits, col.dictionary.data, col.dictionary.offsets,
                                        col.stream, co[:m + 1])
        return oracle.decode(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream, co[:m + 1],
                             threads=threads)

    t0 = time.perf_counter()
    r = dec(probe_n)
    dt = max(time.perf_counter() - t0, 1e-4)
    rate = r.total / dt
    want_bytes = rate * target_s
    per_string = max(r.total / max(probe_n, 1), 1.0)
    m = int(min(n, max(probe_n, want_bytes / per_string)))
    t0 = time.perf_counter()
    r = dec(m)
    dt = time.perf_counter() - t0
    return r.total / dt / 1e9, m, r.total, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    codec, n, desc = WORKLOADS[args.workload]
    if args.n_strings:
        n = args.n_strings
    col, packed_bits = workload_column(args.workload, 0, n)
    threads = 1 if packed_bits else (os.cpu_count() or 1)
    vals, samples = [], []
    per_step = min(args.ref_seconds, 150.0 / (args.warmup + args.steps))
    for i in range(args.warmup + args.steps):
        gbs, m, total, dt = cpu_oracle_rate(col, per_step, threads, packed_bits)
        if i >= args.warmup:
            vals.append(gbs)
            samples.append((m, total, dt))
    value = statistics.mean(vals)
    m, total, dt = samples[-1]
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded generators; stand-in for the paper's real columns)",
        "config": {"workload": args.workload, "description": desc, "n_strings": n},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "sample": f"first {m} of {n} strings ({total} decoded bytes) per step"},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2609_15034_gb300 as fp

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    codec, n, desc = WORKLOADS[args.workload]
    if args.n_strings:
        n = args.n_strings
    col, packed_bits = workload_column(args.workload, rank, n)   # one independent replica column per rank
    assert col.n_strings == n
    fp.variant_select(codec, args.variant)

    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    d = fp.Dict(codec, col.dictionary.data, col.dictionary.offsets, sh)
    if args.width:
        d.set_width(args.width)
    codes = torch.from_numpy(col.stream).to(dev)
    co = torch.from_numpy(col.code_offsets.view(np.int32)).to(dev)
    if packed_bits:
        st, total = fp.decoded_size_packed(codec, d, packed_bits, codes.data_ptr(), codes.numel(), co.data_ptr(), n,
                                           sh)
    else:
        st, total = fp.decoded_size_tensors(codec, d, codes, co, n, sh)
    if st != fp.OK:
        raise RuntimeError(f"decoded_size: {fp.STATUS_NAMES[st]} {fp.last_error()}")
    out = torch.empty(total, dtype=torch.uint8, device=dev)
    offs = torch.empty(n + 1, dtype=torch.int32, device=dev)
    codes_bytes = codes.numel()
    sidecar = None
    if args.sidecar:
        # the stored-sidecar decode: the table is computed once beforehand
        # (untimed), as a column would carry it from compression
        sidecar = fp.SidecarColumn(codec, d, codes, co, n)
        sidecar.build(sh)
        if sidecar.status_bits() != 0:
            raise RuntimeError(f"sidecar build: data-error bits {sidecar.status_bits()}")

    def decode_call(codes_ptr, co_ptr, out_ptr, offs_ptr, stream):
        if packed_bits:
            fp.decode_packed(codec, d, packed_bits, codes_ptr, codes_bytes, co_ptr, n, out_ptr, total, offs_ptr, stream)
        else:
            fp.decode(codec, d, codes_ptr, codes_bytes, co_ptr, n, out_ptr, total, offs_ptr, stream)

    def step():
        if sidecar is not None:
            sidecar.decode(out, offs, sh)
        else:
            decode_call(codes.data_ptr(), co.data_ptr(), out.data_ptr(), offs.data_ptr(), sh)

    def status_ok():
        if sidecar is not None:
            return sidecar.status_bits() == 0
        return fp.sync_status(sh) == fp.OK

    # correctness gate on a sample before timing (the full oracle check lives in the tests)
    step()
    if not status_ok():
        raise RuntimeError(fp.last_error())

    gpu_id = "0"
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        if not gpu_id.startswith("GPU-"):
            gpu_id = "GPU-" + gpu_id
    except Exception:
        gpu_id = str(local_rank)
    sampler = ClockSampler(gpu_id)
    # settle clocks (untimed), then the warm-up steps
    t_end = time.time() + args.settle
    while time.time() < t_end:
        for _ in range(20):
            step()
        torch.cuda.synchronize()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    # a workload that fits in L2 gets L2 flushed between timed steps (a write
    # of twice its size), and its time is the sum of the steps' own events
    l2_resident = total + codes_bytes <= L2_BYTES
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev) if l2_resident else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    for i in range(args.steps):
        if flush is not None:
            flush.fill_(i & 0xff)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(launch_ms) if flush is not None else t0.elapsed_time(t1)
    del flush
    if not status_ok():
        raise RuntimeError(fp.last_error())
    total_ms, all_bytes = combine_ranks(dist, total_ms, float(total), dev)

    value = all_bytes * args.steps / (total_ms * 1e-3) / 1e9
    avg_launch_s = statistics.mean(launch_ms) * 1e-3
    alg = algorithmic_bytes(col, total, codec, packed_bits)
    peak, peak_kind = load_peaks()
    achieved = alg / avg_launch_s / 1e9

    extra = {}
    if rank == 0 and not args.quick:
        # plain one-thread-per-string GPU decode, same column, same clock (it
        # reads the codec's own layout, so not for cascaded codes)
        if not packed_bits:
            plain_ms = []
            for i in range(3 + args.plain_steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fp.decode_plain(codec, d, codes.data_ptr(), codes_bytes, co.data_ptr(), n, out.data_ptr(), total,
                                offs.data_ptr(), sh)
                b.record(stream)
                torch.cuda.synchronize()
                if i >= 3:
                    plain_ms.append(a.elapsed_time(b))
            if fp.sync_status(sh) != fp.OK:
                raise RuntimeError(fp.last_error())
            plain_gbs = total / (statistics.mean(plain_ms) * 1e-3) / 1e9
            extra["plain_gpu"] = {"value": round(plain_gbs, 2), "unit": "GB/s", "kind": "one thread per string",
                                  "ms": round(statistics.mean(plain_ms), 3)}

        # End to end through the public API with host buffers (pinned): every
        # step copies the column's codes and code_offsets host -> device,
        # decodes, and copies the bytes and offsets device -> host.  Steps are
        # pipelined the way a stream of columns would be: three streams (in,
        # decode, out) and two buffer sets, so one step's input copy overlaps
        # the previous step's output copy (the host link runs both directions
        # at once).
        h_codes = torch.from_numpy(col.stream).pin_memory()
        h_co = torch.from_numpy(col.code_offsets.view(np.int32)).pin_memory()
        sets = []
        for _ in range(2):
            sets.append({"codes": torch.empty_like(codes), "co": torch.empty_like(co), "out": torch.empty_like(out),
                         "offs": torch.empty_like(offs),
                         "h_out": torch.empty(total, dtype=torch.uint8).pin_memory(),
                         "h_offs": torch.empty(n + 1, dtype=torch.int32).pin_memory()})
        s_in, s_dec, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_dec = [torch.cuda.Event() for _ in range(2)]
        ev_out = [torch.cuda.Event() for _ in range(2)]

        def e2e_steps(k):
            for i in range(k):
                b, j = sets[i % 2], i % 2
                if i >= 2:
                    s_in.wait_event(ev_dec[j])     # the set's inputs are no longer read
                with torch.cuda.stream(s_in):
                    b["codes"].copy_(h_codes, non_blocking=True)
                    b["co"].copy_(h_co, non_blocking=True)
                ev_in[j].record(s_in)
                s_dec.wait_event(ev_in[j])
                if i >= 2:
                    s_dec.wait_event(ev_out[j])    # the set's outputs have been copied out
                decode_call(b["codes"].data_ptr(), b["co"].data_ptr(), b["out"].data_ptr(), b["offs"].data_ptr(),
                            s_dec.cuda_stream)
                ev_dec[j].record(s_dec)
                s_out.wait_event(ev_dec[j])
                with torch.cuda.stream(s_out):
                    b["h_out"].copy_(b["out"], non_blocking=True)
                    b["h_offs"].copy_(b["offs"], non_blocking=True)
                ev_out[j].record(s_out)

        e2e_steps(2)
        torch.cuda.synchronize()
        a, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2e_n = max(4, min(args.steps, 20))
        a.record(s_in)
        e2e_steps(e2e_n)
        b_ev.record(s_out)
        torch.cuda.synchronize()
        if fp.sync_status(s_dec.cuda_stream) != fp.OK:
            raise RuntimeError(fp.last_error())
        e2e_s = a.elapsed_time(b_ev) * 1e-3 / e2e_n
        extra["e2e"] = {"value": round(total / e2e_s / 1e9, 3), "unit": "GB/s",
                        "h2d_bytes_per_step": int(h_codes.numel() + h_co.numel() * 4),
                        "d2h_bytes_per_step": int(total + (n + 1) * 4),
                        "kind": "pinned host column in, bytes and offsets out, every step; steps pipelined on "
                                "three streams with two buffer sets"}
        # spot-check the host copies against the device result
        for b in sets:
            if not torch.equal(b["h_out"][:4096], out[:4096].cpu()) or not torch.equal(b["h_offs"], offs.cpu()):
                raise RuntimeError("end-to-end output mismatch")

        # CPU oracle on the host cores (reported baseline, not a target)
        threads = 1 if packed_bits else (os.cpu_count() or 1)
        gbs, m, tb, dt = cpu_oracle_rate(col, args.cpu_seconds, threads, packed_bits)
        extra["cpu_baseline"] = {"value": round(gbs, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                                 "sample": f"first {m} of {n} strings ({tb} decoded bytes), {dt:.1f} s"}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    if packed_bits:
        vinfo = {"kind": "packed codes (fp_decode_packed)", "code_bits": packed_bits, "launches_per_call": 3}
    else:
        var = fp.variant_for_dict(d, codes_bytes)
        vinfo = dict(fp.variant_info(codec, var), index=var, read_width=fp.variant_width(codec, var))
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        vinfo["tuned"] = tuned_entry(codec, d.width, codes_bytes, sms)   # the table's line (None: built-in default)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded generators; stand-in for the paper's real columns)",
        "config": {"workload": args.workload, "description": desc, "n_strings": n, "decoded_bytes": int(total),
                   "code_bytes": int(codes_bytes), "mean_bytes_per_code": round(total / max(col.n_slots, 1), 3),
                   "l2": "inputs and output larger than L2 (no flush needed)" if not l2_resident
                   else "L2 flushed between timed steps (a write of twice L2); time = sum of the steps' events",
                   "variant": vinfo, "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                     "traffic": load_traffic(args.workload), "algorithmic_bytes_per_launch": alg,
                     "kernel_ms": round(avg_launch_s * 1e3, 4)},
        "clocks": clocks,
        "gpu_launches": vinfo["launches_per_call"] * args.steps,   # index pass (+ reduce in the same launch, tile scan) + decode
    }
    if sidecar is not None:
        line["metric"] = "decoded GB/s from a stored sidecar (tile output offsets computed beforehand, untimed)"
        line["config"]["sidecar"] = {"tile_slots": fp.sidecar_tile_slots(codec), "entries": sidecar.entries}
        line["config"].pop("variant")
        line["roofline"]["traffic"] = None
        line["gpu_launches"] = 3 * args.steps   # index pass, size check, decode
    line.update(extra)
    if "e2e" not in line:
        line["e2e"] = None
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# Batched decode
# ---------------------------------------------------------------------------

POOL_STRINGS = {synth.ONPAIR16: 1_000_000, synth.ONPAIR12: 1_000_000, synth.FSST8: 2_000_000}


class BatchInputs:
    """Host side of a batch: per-codec pools of code streams and, per chunk,
    its codec, its own dictionary and a window of its codec's pool."""

    def __init__(self, n_chunks: int, lo: int, hi: int, seed: int = 0):
        rng = synth.rng_for(4, seed, 0)
        self.codecs = synth.codec_mix(rng, n_chunks)
        targets = synth.log_uniform_sizes(rng, n_chunks, lo, hi)
        self.pools = {c: synth.column(c, 1000 + seed, POOL_STRINGS[c]) for c in (synth.ONPAIR16, synth.ONPAIR12,
                                                                                 synth.FSST8)}
        per_string = {}
        for c, pool in self.pools.items():
            lens = pool.dictionary.token_lengths()
            if c == synth.FSST8:
                dec = int(np.where(pool.slot_is_literal, 1, np.where(pool.slot_codes == 255, 0,
                                   lens[np.minimum(pool.slot_codes, lens.size - 1)])).sum())
            else:
                dec = int(lens[pool.slot_codes].sum())
            per_string[c] = dec / pool.n_strings
        bases = [synth.onpair12_dictionary(s) for s in range(8)]
        self.chunks = []
        for i in range(n_chunks):
            c = int(self.codecs[i])
            pool = self.pools[c]
            n = int(max(1, min(pool.n_strings, round(targets[i] / per_string[c]))))
            start = int(rng.integers(0, pool.n_strings - n + 1))
            b0, b1, co = synth.pool_window(pool, start, n)
            d = synth.chunk_dictionary(c, 10_000 + i, bases)
            self.chunks.append((c, d, b0, b1, co))

    def host_column(self, i):
        c, d, b0, b1, co = self.chunks[i]
        return synth.Column(c, d, self.pools[c].stream[b0:b1], co, (b1 - b0) * 8 // synth.CODE_BITS[c])


def _align(x: int, a: int = 256) -> int:
    return (x + a - 1) // a * a


def rows_selection(n_strings: int, n_rows: int, seed: int):
    """n_rows distinct row ids of a column of n_strings, in random order."""
    rng = np.random.default_rng((7, seed, n_rows))
    return rng.permutation(n_strings)[:n_rows].astype(np.uint32)


def rows_algorithmic_bytes(col, rows, total: int) -> int:
    """Bytes a selective decode must move at least: the row ids, each
    selected row's two code offsets and code bytes, the output and its
    offsets, the dictionary once."""
    co = col.code_offsets.astype(np.int64)
    slots = int((co[rows.astype(np.int64) + 1] - co[rows]).sum())
    code_bytes = (slots * synth.CODE_BITS[col.codec] + 7) // 8
    d = col.dictionary
    return 4 * rows.size + 8 * rows.size + code_bytes + total + 4 * (rows.size + 1) + \
        d.n_entries * (synth.MAX_TOKEN[col.codec] + 1)


def run_rows(args, rank, world, local_rank):
    import torch
    import paper_2609_15034_gb300 as fp

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    base, n_rows, desc = ROWS_WORKLOADS[args.workload]
    codec, n, _ = WORKLOADS[base]
    if args.n_strings:
        n = args.n_strings
    n_rows = min(n_rows, n)
    col, _ = workload_column(base, rank, n)   # one independent replica column per rank
    rows_h = rows_selection(n, n_rows, rank)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    d = fp.Dict(codec, col.dictionary.data, col.dictionary.offsets, sh)
    codes = torch.from_numpy(col.stream).to(dev)
    co = torch.from_numpy(col.code_offsets.view(np.int32)).to(dev)
    rows = torch.from_numpy(rows_h.view(np.int32)).to(dev)
    codes_bytes = codes.numel()
    st, slots, total = fp.rows_size(codec, d, codes.data_ptr(), codes_bytes, co.data_ptr(), n, rows.data_ptr(),
                                    n_rows, sh)
    if st != fp.OK:
        raise RuntimeError(f"rows_size: {fp.STATUS_NAMES[st]} {fp.last_error()}")
    out = torch.empty(total, dtype=torch.uint8, device=dev)
    offs = torch.empty(n_rows + 1, dtype=torch.int32, device=dev)

    def rows_call(rows_ptr, out_ptr, offs_ptr, stream_h):
        fp.decode_rows(codec, d, codes.data_ptr(), codes_bytes, co.data_ptr(), n, rows_ptr, n_rows, slots, out_ptr,
                       total, offs_ptr, stream_h)

    def step():
        rows_call(rows.data_ptr(), out.data_ptr(), offs.data_ptr(), sh)

    step()
    if fp.sync_status(sh) != fp.OK:
        raise RuntimeError(fp.last_error())
    gpu_id = str(local_rank)
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        if not gpu_id.startswith("GPU-"):
            gpu_id = "GPU-" + gpu_id
    except Exception:
        pass
    sampler = ClockSampler(gpu_id)
    t_end = time.time() + args.settle
    while time.time() < t_end:
        for _ in range(20):
            step()
        torch.cuda.synchronize()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = t0.elapsed_time(t1)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    if fp.sync_status(sh) != fp.OK:
        raise RuntimeError(fp.last_error())
    total_ms, all_bytes = combine_ranks(dist, total_ms, float(total), dev)
    value = all_bytes * args.steps / (total_ms * 1e-3) / 1e9
    avg_s = statistics.mean(launch_ms) * 1e-3
    alg = rows_algorithmic_bytes(col, rows_h, total)
    peak, peak_kind = load_peaks()
    extra = {}
    if rank == 0 and not args.quick:
        # end to end: the row ids in from pinned host memory, the selected
        # strings and their offsets back, every step (the column is resident,
        # as in a column store that keeps it on the device)
        h_rows = torch.from_numpy(rows_h.view(np.int32)).pin_memory()
        h_out = torch.empty(total, dtype=torch.uint8).pin_memory()
        h_offs = torch.empty(n_rows + 1, dtype=torch.int32).pin_memory()
        d_rows = torch.empty_like(rows)

        def e2e_step():
            d_rows.copy_(h_rows, non_blocking=True)
            rows_call(d_rows.data_ptr(), out.data_ptr(), offs.data_ptr(), sh)
            h_out.copy_(out, non_blocking=True)
            h_offs.copy_(offs, non_blocking=True)

        for _ in range(3):
            e2e_step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2e_n = max(4, min(args.steps, 20))
        a.record(stream)
        for _ in range(e2e_n):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        if fp.sync_status(sh) != fp.OK:
            raise RuntimeError(fp.last_error())
        if not torch.equal(h_out[:4096], out[:4096].cpu()) or not torch.equal(h_offs, offs.cpu()):
            raise RuntimeError("end-to-end output mismatch")
        e2e_s = a.elapsed_time(b) * 1e-3 / e2e_n
        extra["e2e"] = {"value": round(total / e2e_s / 1e9, 3), "unit": "GB/s",
                        "h2d_bytes_per_step": int(4 * n_rows), "d2h_bytes_per_step": int(total + 4 * (n_rows + 1)),
                        "kind": "pinned host row ids in, selected bytes and offsets out, every step, one stream; "
                                "the column stays resident"}
        gbs, m, tb, dt = rows_cpu_rate(col, rows_h, args.cpu_seconds)
        extra["cpu_baseline"] = {"value": round(gbs, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                                 "sample": f"first {m} of {n_rows} selected rows ({tb} decoded bytes), {dt:.1f} s"}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    var = fp.variant_for_dict(d, max(8, slots * synth.CODE_BITS[codec] // 8))
    line = {
        "metric": ROWS_METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded generators; stand-in for the paper's real columns)",
        "config": {"workload": args.workload, "description": desc, "n_strings": n, "n_rows": n_rows,
                   "selected_slots": int(slots), "decoded_bytes": int(total),
                   "l2": "column and output larger than L2 (no flush needed)",
                   "variant": dict(fp.variant_info(codec, var), index=var),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": round(alg / avg_s / 1e9, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(alg / avg_s / 1e9 / peak, 4), "peak_kind": peak_kind, "traffic": None,
                     "algorithmic_bytes_per_launch": int(alg), "kernel_ms": round(avg_s * 1e3, 4)},
        "clocks": clocks,
        "gpu_launches": 7 * args.steps,   # row sums, their scan, row offsets, gather; reduce, tile scan, decode
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def rows_cpu_rate(col, rows, target_s: float):
    """Time the oracle's selective decode (as it stands) on a bounded prefix
    of the selection."""
    import oracle
    probe = min(rows.size, 20000)
    args = (col.codec, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets)
    t0 = time.perf_counter()
    r = oracle.decode_rows(*args, rows[:probe])
    dt = max(time.perf_counter() - t0, 1e-4)
    m = int(min(rows.size, max(probe, probe * target_s / dt)))
    t0 = time.perf_counter()
    r = oracle.decode_rows(*args, rows[:m])
    dt = time.perf_counter() - t0
    return r.total / dt / 1e9, m, r.total, dt


def run_rows_reference(args, rank, world):
    if rank != 0:
        return
    base, n_rows, desc = ROWS_WORKLOADS[args.workload]
    codec, n, _ = WORKLOADS[base]
    if args.n_strings:
        n = args.n_strings
    n_rows = min(n_rows, n)
    col, _ = workload_column(base, 0, n)
    rows = rows_selection(n, n_rows, 0)
    per_step = min(args.ref_seconds, 150.0 / (args.warmup + args.steps))
    vals, last = [], None
    for i in range(args.warmup + args.steps):
        gbs, m, tb, dt = rows_cpu_rate(col, rows, per_step)
        if i >= args.warmup:
            vals.append(gbs)
            last = (m, tb, dt)
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": ROWS_METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(last[2] * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded generators; stand-in for the paper's real columns)",
        "config": {"workload": args.workload, "description": desc, "n_strings": n, "n_rows": n_rows},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {last[0]} of {n_rows} selected rows ({last[1]} decoded bytes) per step"},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batched(args, rank, world, local_rank):
    import torch
    import paper_2609_15034_gb300 as fp

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    n_chunks, lo, hi, desc = BATCH_WORKLOADS[args.workload]
    t_gen = time.time()
    B = BatchInputs(n_chunks, lo, hi, seed=rank)
    t_gen = time.time() - t_gen
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    # inputs: every chunk's code window and code_offsets in one device buffer each
    code_off, co_off = [], []
    cb = cob = 0
    for (c, d, b0, b1, co) in B.chunks:
        code_off.append(cb)
        cb = _align(cb + (b1 - b0))
        co_off.append(cob)
        cob = _align(cob + co.size * 4)
    h_codes = np.zeros(cb, np.uint8)
    h_co = np.zeros(cob, np.uint8)
    for i, (c, d, b0, b1, co) in enumerate(B.chunks):
        h_codes[code_off[i]:code_off[i] + (b1 - b0)] = B.pools[c].stream[b0:b1]
        h_co[co_off[i]:co_off[i] + co.size * 4] = co.view(np.uint8)
    codes = torch.from_numpy(h_codes).to(dev)
    cos = torch.from_numpy(h_co).to(dev)
    dicts = [fp.Dict(c, d.data, d.offsets, sh) for (c, d, b0, b1, co) in B.chunks]

    # exact decoded sizes (the library's length pass), then one output buffer
    totals, out_off, offs_off = [], [], []
    ob = oob = 0
    for i, (c, d, b0, b1, co) in enumerate(B.chunks):
        st, tot = fp.decoded_size(c, dicts[i], codes.data_ptr() + code_off[i], b1 - b0,
                                  cos.data_ptr() + co_off[i], co.size - 1, sh)
        if st != fp.OK:
            raise RuntimeError(f"chunk {i}: {fp.STATUS_NAMES[st]} {fp.last_error()}")
        totals.append(tot)
        out_off.append(ob)
        ob = _align(ob + tot)
        offs_off.append(oob)
        oob = _align(oob + co.size * 4)
    out = torch.empty(max(ob, 256), dtype=torch.uint8, device=dev)
    offs = torch.empty(max(oob, 256), dtype=torch.uint8, device=dev)
    chunks = [fp.chunk(c, dicts[i], codes.data_ptr() + code_off[i], b1 - b0, cos.data_ptr() + co_off[i],
                       co.size - 1, out.data_ptr() + out_off[i], totals[i], offs.data_ptr() + offs_off[i])
              for i, (c, d, b0, b1, co) in enumerate(B.chunks)]
    total = int(sum(totals))
    t_tune = time.time()
    plan = fp.Plan(chunks, tune_cache=None, stream=sh)
    t_tune = time.time() - t_tune
    pinfo = plan.info()

    def step():
        plan.decode(sh)

    step()
    st, sts, tot = plan.sync_status(sh)
    if st != fp.OK or not np.array_equal(tot, np.asarray(totals, np.uint64)):
        raise RuntimeError(f"batch: {fp.STATUS_NAMES.get(st, st)} {fp.last_error()}")

    gpu_id = str(local_rank)
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        if not gpu_id.startswith("GPU-"):
            gpu_id = "GPU-" + gpu_id
    except Exception:
        pass
    sampler = ClockSampler(gpu_id)
    t_end = time.time() + args.settle
    while time.time() < t_end:
        step()
        torch.cuda.synchronize()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    total_ms = t0.elapsed_time(t1)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    st, sts, tot = plan.sync_status(sh)
    if st != fp.OK:
        raise RuntimeError(fp.last_error())
    total_ms, all_bytes = combine_ranks(dist, total_ms, float(total), dev)
    value = all_bytes * args.steps / (total_ms * 1e-3) / 1e9
    avg_s = statistics.mean(launch_ms) * 1e-3
    alg = 0
    for i, (c, d, b0, b1, co) in enumerate(B.chunks):
        used = int(co[-1]) - int(co[0])
        alg += (used * synth.CODE_BITS[c] + 7) // 8 + 8 * co.size + totals[i] + d.n_entries * (synth.MAX_TOKEN[c] + 1)
    peak, peak_kind = load_peaks()
    achieved = alg / avg_s / 1e9

    extra = {}
    if rank == 0 and not args.quick:
        # one launch (sequence) per chunk: the plain one-thread-per-string decode, and fp_decode
        def per_chunk(fn):
            fn(*chunk_args(0))
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 2
            a.record(stream)
            for _ in range(reps):
                for i in range(n_chunks):
                    fn(*chunk_args(i))
            b.record(stream)
            torch.cuda.synchronize()
            if fp.sync_status(sh) != fp.OK:
                raise RuntimeError(fp.last_error())
            ms = a.elapsed_time(b) / reps
            return total / (ms * 1e-3) / 1e9, ms

        def chunk_args(i):
            c, d, b0, b1, co = B.chunks[i]
            return (c, dicts[i], codes.data_ptr() + code_off[i], b1 - b0, cos.data_ptr() + co_off[i], co.size - 1,
                    out.data_ptr() + out_off[i], totals[i], offs.data_ptr() + offs_off[i], sh)

        pg, pms = per_chunk(fp.decode_plain)
        extra["plain_gpu"] = {"value": round(pg, 2), "unit": "GB/s",
                              "kind": "one plain launch sequence per chunk (one thread per string)",
                              "ms": round(pms, 2), "batched_over_plain": round(value / pg, 2)}
        sg, sms = per_chunk(fp.decode)
        extra["per_chunk_fp_decode"] = {"value": round(sg, 2), "unit": "GB/s",
                                        "kind": "one fp_decode call per chunk (single-column default decoder)",
                                        "ms": round(sms, 2)}

        # end to end: pinned host inputs in, decoded bytes and offsets out, every step
        hp_codes = torch.from_numpy(h_codes).pin_memory()
        hp_co = torch.from_numpy(h_co).pin_memory()
        hp_out = torch.empty(out.numel(), dtype=torch.uint8).pin_memory()
        hp_offs = torch.empty(offs.numel(), dtype=torch.uint8).pin_memory()

        def e2e_step():
            codes.copy_(hp_codes, non_blocking=True)
            cos.copy_(hp_co, non_blocking=True)
            plan.decode(sh)
            hp_out.copy_(out, non_blocking=True)
            hp_offs.copy_(offs, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2e_n = 3
        a.record(stream)
        for _ in range(e2e_n):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        if plan.sync_status(sh)[0] != fp.OK:
            raise RuntimeError(fp.last_error())
        e2e_s = a.elapsed_time(b) * 1e-3 / e2e_n
        extra["e2e"] = {"value": round(total / e2e_s / 1e9, 3), "unit": "GB/s",
                        "h2d_bytes_per_step": int(h_codes.size + h_co.size),
                        "d2h_bytes_per_step": int(out.numel() + offs.numel())}
        del hp_codes, hp_co, hp_out, hp_offs

        # CPU oracle on the host cores: whole chunks in order, about cpu_seconds of work
        import oracle
        threads = os.cpu_count() or 1
        done_b, t_cpu, k = 0, 0.0, 0
        while k < n_chunks and t_cpu < args.cpu_seconds:
            col = B.host_column(k)
            t = time.perf_counter()
            r = oracle.decode(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets,
                              threads=threads)
            t_cpu += time.perf_counter() - t
            done_b += r.total
            k += 1
        extra["cpu_baseline"] = {"value": round(done_b / t_cpu / 1e9, 4), "unit": "GB/s", "cores": threads,
                                 "kind": "oracle", "sample": f"first {k} of {n_chunks} chunks "
                                                             f"({done_b} decoded bytes), {t_cpu:.1f} s"}
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    counts = {synth.CODEC_NAMES[c]: int((B.codecs == c).sum()) for c in (synth.ONPAIR16, synth.ONPAIR12, synth.FSST8)}
    line = {
        "metric": BATCH_METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded generators; stand-in for the paper's real columns)",
        "config": {"workload": args.workload, "description": desc, "n_chunks": n_chunks, "codec_chunks": counts,
                   "decoded_bytes": total, "code_bytes": int(sum(b1 - b0 for (_, _, b0, b1, _) in B.chunks)),
                   "n_strings": int(sum(co.size - 1 for (*_, co) in B.chunks)),
                   "largest_chunk_bytes": int(max(totals)), "smallest_chunk_bytes": int(min(totals)),
                   "l2": "inputs and output larger than L2 (no flush needed)",
                   "plan": pinfo, "generation_s": round(t_gen, 1), "plan_create_s": round(t_tune, 2),
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                     "traffic": load_traffic(args.workload), "algorithmic_bytes_per_launch": alg,
                     "kernel_ms": round(avg_s * 1e3, 4)},
        "clocks": clocks,
        # per step one graph: index pass [+ reduce + tile scan] + the persistent decode kernel
        "gpu_launches": (4 if fp.batch_config_info(pinfo["config"])["warp_tiles"] else 2) * args.steps,
    }
    line.update(extra)
    if "e2e" not in line:
        line["e2e"] = None
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_batched_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    n_chunks, lo, hi, desc = BATCH_WORKLOADS[args.workload]
    B = BatchInputs(n_chunks, lo, hi, seed=0)
    threads = os.cpu_count() or 1
    per_step = min(args.ref_seconds, 150.0 / (args.warmup + args.steps))
    vals = []
    k = 0
    last = (0, 0, 0.0)
    for i in range(args.warmup + args.steps):
        done_b, t_cpu, first = 0, 0.0, k
        while t_cpu < per_step:
            col = B.host_column(k % n_chunks)
            t = time.perf_counter()
            r = oracle.decode(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets,
                              threads=threads)
            t_cpu += time.perf_counter() - t
            done_b += r.total
            k += 1
        if i >= args.warmup:
            vals.append(done_b / t_cpu / 1e9)
            last = (k - first, done_b, t_cpu)
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": BATCH_METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(last[2] * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded generators; stand-in for the paper's real columns)",
        "config": {"workload": args.workload, "description": desc, "n_chunks": n_chunks},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "sample": f"{last[0]} whole chunks ({last[1]} decoded bytes) per step"},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Served decode
# ---------------------------------------------------------------------------

SERVE_POOL_STRINGS = {synth.ONPAIR16: 2_600_000, synth.ONPAIR12: 2_500_000, synth.FSST8: 5_800_000}
PAGES_PER_CODEC = 64


class ServeInputs:
    """Pages (columns cut from per-codec pools, decoded sizes log-uniform),
    dictionary keys (each a dictionary of its codec's length profile, so a
    page's decoded size is the same under every key of its codec) and a
    Poisson request stream."""

    def __init__(self, rate, seconds, lo, hi, n_keys, seed=0, n_requests=None):
        rng = synth.rng_for(6, seed, 0)
        codecs = (synth.ONPAIR16, synth.ONPAIR12, synth.FSST8)
        self.pools = {c: synth.column(c, 2000 + seed, SERVE_POOL_STRINGS[c]) for c in codecs}
        self.pages = {c: [] for c in codecs}   # (byte0, byte1, code_offsets, decoded bytes)
        for c in codecs:
            pool = self.pools[c]
            cum = np.zeros(pool.n_slots + 1, np.int64)
            np.cumsum(synth.slot_bytes(pool), out=cum[1:])
            per_string = cum[-1] / pool.n_strings
            for t in synth.log_uniform_sizes(rng, PAGES_PER_CODEC, lo, hi):
                n = int(max(1, min(pool.n_strings, round(t / per_string))))
                start = int(rng.integers(0, pool.n_strings - n + 1))
                b0, b1, co = synth.pool_window(pool, start, n)
                a, b = int(pool.code_offsets[start]), int(pool.code_offsets[start + n])
                self.pages[c].append((b0, b1, co, int(cum[b] - cum[a])))
        key_codecs = synth.codec_mix(synth.rng_for(6, seed, 1), n_keys)
        self.keys = [(k, int(key_codecs[k])) for k in range(n_keys)]
        self.key_dicts = {}
        rank_to_key = rng.permutation(n_keys)
        cdf = synth.zipf_cdf(n_keys, 1.0)
        if n_requests is None:
            n_requests = int(rate * seconds * 1.2) + 16
        gaps = rng.exponential(1.0 / rate, n_requests)
        self.arrivals = np.cumsum(gaps)
        if n_requests and seconds:
            self.arrivals = self.arrivals[self.arrivals < seconds]
        n_req = self.arrivals.size
        self.req_key = rank_to_key[synth.zipf_draw(rng, cdf, n_req)]
        self.req_page = rng.integers(0, PAGES_PER_CODEC, n_req)

    def dictionary(self, key):
        if key not in self.key_dicts:
            codec = self.keys[key][1]
            self.key_dicts[key] = synth.same_shape_dictionary(self.pools[codec].dictionary, 7000 + key)
        return self.key_dicts[key]

    def request(self, i):
        key = int(self.req_key[i])
        codec = self.keys[key][1]
        return key, codec, int(self.req_page[i])

    def host_column(self, key, codec, page):
        b0, b1, co, _ = self.pages[codec][page]
        return synth.Column(codec, self.dictionary(key), self.pools[codec].stream[b0:b1], co,
                            (b1 - b0) * 8 // synth.CODE_BITS[codec])


def _progress(msg):
    sys.stderr.write(f"[{time.strftime('%H:%M:%S')}] {msg}\n")
    sys.stderr.flush()


def run_served(args, rank, world, local_rank):
    import faulthandler
    import threading
    import torch
    import paper_2609_15034_gb300 as fp

    faulthandler.dump_traceback_later(args.serve_watchdog, repeat=True)   # thread stacks if a phase hangs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    rate, seconds, lo, hi, n_keys, budget, desc = SERVE_WORKLOADS[args.workload]
    if args.serve_seconds:
        seconds = args.serve_seconds
    t_gen = time.time()
    I = ServeInputs(rate, seconds, lo, hi, n_keys, seed=rank)
    for k in range(n_keys):
        I.dictionary(k)
    t_gen = time.time() - t_gen
    _progress(f"served: inputs generated in {t_gen:.1f} s, {I.arrivals.size} requests")
    codecs = (synth.ONPAIR16, synth.ONPAIR12, synth.FSST8)
    # pages on the device: one buffer for codes, one for code_offsets
    page_dev = {}
    for c in codecs:
        for j, (b0, b1, co, dec) in enumerate(I.pages[c]):
            codes = torch.from_numpy(np.ascontiguousarray(I.pools[c].stream[b0:b1])).to(dev)
            cot = torch.from_numpy(co.view(np.int32)).to(dev)
            page_dev[(c, j)] = (codes, cot, b1 - b0, co.size - 1, dec)
    serve_cfg = args.serve_config if args.serve_config >= 0 else SERVE_DEFAULT_CONFIG
    srv = fp.Server(hbm_budget=budget, dict_cache_slots=512, n_streams=args.serve_streams,
                    max_wave=args.serve_wave, batch_config=serve_cfg)
    for k, c in I.keys:
        d = I.dictionary(k)
        srv.dict_put(k, c, d.data, d.offsets)
    _progress("served: server up, dictionaries registered")

    def submit(i, tag):
        key, c, pg = I.request(i)
        codes, cot, nbytes, n, dec = page_dev[(c, pg)]
        return srv.submit(key, codes.data_ptr(), nbytes, cot.data_ptr(), n, dec, tag)

    lat, sizes, done_t = [], [], []
    errors = []

    def consume(n_expected, keep=None):
        got = 0
        last = time.time()
        while got < n_expected:
            if time.time() - last > args.serve_stall:
                _progress(f"served: no result for {args.serve_stall} s; {got} of {n_expected}; stats {srv.stats()}")
                raise RuntimeError("served decode stalled")
            res = srv.poll(timeout_s=0.05)
            if res:
                last = time.time()
            for r in res:
                if r["status"] != fp.OK:
                    errors.append((r["ticket"], r["status"]))
                if keep is not None and r["user_tag"] in keep:
                    keep[r["user_tag"]] = fp.device_bytes(r["d_out_bytes"], r["bytes"]).clone()
                    torch.cuda.current_stream().synchronize()   # copied before the memory is released
                lat.append((r["t_done_ns"] - r["t_submit_ns"]) * 1e-6)
                sizes.append(r["bytes"])
                done_t.append(r["t_done_ns"])
                srv.release(r["ticket"])
                got += 1

    # warm-up: every key once (fills the dictionary cache), untimed
    warm = min(len(I.req_key), 64)
    for i in range(warm):
        submit(i, 0)
    consume(warm)
    lat.clear(); sizes.clear(); done_t.clear()
    st0 = srv.stats()
    _progress(f"served: warm-up done, stats {st0}")

    # open loop: Poisson arrivals; a sample of results is kept to cross-check
    n_req = int(I.arrivals.size)
    rs = np.random.default_rng(5)
    sample = {int(i): None for i in rs.choice(n_req, size=min(12, n_req), replace=False)}
    cons = threading.Thread(target=consume, args=(n_req, sample))
    gpu_id = str(local_rank)
    try:
        gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
        if not gpu_id.startswith("GPU-"):
            gpu_id = "GPU-" + gpu_id
    except Exception:
        pass
    sampler = ClockSampler(gpu_id)
    cons.start()
    t_start = time.perf_counter()
    t0_ns = time.monotonic_ns()
    late = 0
    for i in range(n_req):
        now = time.perf_counter() - t_start
        wait = I.arrivals[i] - now
        if wait > 0:
            time.sleep(wait)
        elif wait < -0.001:
            late += 1
        submit(i, i)
    cons.join()
    clocks = sampler.stop()
    st1 = srv.stats()
    _progress(f"served: open loop done, stats {st1}")
    span_s = (max(done_t) - t0_ns) * 1e-9
    tot_bytes = int(sum(sizes))
    value = tot_bytes / span_s / 1e9
    la = np.asarray(lat)
    if errors:
        raise RuntimeError(f"served requests failed: {errors[:5]}")

    # cross-check the sampled results against fp_decode of the same page and dictionary
    dicts = {}
    for i, out in sample.items():
        key, c, pg = I.request(i)
        codes, cot, nbytes, n, dec = page_dev[(c, pg)]
        if key not in dicts:
            d = I.dictionary(key)
            dicts[key] = fp.Dict(c, d.data, d.offsets)
        ref = torch.empty(dec, dtype=torch.uint8, device=dev)
        offs = torch.empty(n + 1, dtype=torch.int32, device=dev)
        fp.decode_tensors(c, dicts[key], codes[:nbytes], cot, n, ref, offs)
        if fp.sync_status() != fp.OK or not torch.equal(ref, out):
            raise RuntimeError(f"served request {i} differs from fp_decode")

    extra = {}
    if not args.quick:
        # closed loop at saturation: the same request mix, all queued at once
        n_sat = min(n_req, args.serve_saturation)
        lat_keep = (list(lat), list(sizes), list(done_t))
        lat.clear(); sizes.clear(); done_t.clear()
        cons = threading.Thread(target=consume, args=(n_sat,))
        cons.start()
        t0 = time.monotonic_ns()
        for i in range(n_sat):
            submit(i, i)
        cons.join()
        sat_s = (max(done_t) - t0) * 1e-9
        _progress("served: saturation run done")
        # algorithmic bytes of the saturation run's requests: codes, code_offsets, output, out_offsets
        sat_alg = 0
        for i in range(n_sat):
            key, c, pg = I.request(i)
            codes, cot, nbytes, n, dec = page_dev[(c, pg)]
            co = I.pages[c][pg][2]
            sat_alg += ((int(co[-1]) - int(co[0])) * synth.CODE_BITS[c] + 7) // 8 + 8 * (n + 1) + dec
        peak, peak_kind = load_peaks()
        extra["roofline"] = {"bound": "hbm", "achieved": round(sat_alg / sat_s / 1e9, 1), "peak": peak, "unit": "GB/s",
                             "frac": round(sat_alg / sat_s / 1e9 / peak, 4), "peak_kind": peak_kind, "traffic": None,
                             "algorithmic_bytes": sat_alg,
                             "measured_over": "closed-loop saturation run (waves of the persistent batched decode)"}
        sat_bytes = int(sum(sizes))
        sat_gbs = sat_bytes / sat_s / 1e9
        lat[:], sizes[:], done_t[:] = lat_keep

        # the same requests, one plain decode (one thread per string) per request, then one fp_decode per request
        for k, c in I.keys:
            if k not in dicts:
                d = I.dictionary(k)
                dicts[k] = fp.Dict(c, d.data, d.offsets)
        big = max(v[4] for v in page_dev.values())
        nmax = max(v[3] for v in page_dev.values())
        out = torch.empty(big + 16, dtype=torch.uint8, device=dev)
        offs = torch.empty(nmax + 1, dtype=torch.int32, device=dev)
        sh = torch.cuda.current_stream().cuda_stream

        def per_request(fn, count):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            nb = 0
            torch.cuda.synchronize()
            t = time.perf_counter()
            a.record()
            for i in range(count):
                key, c, pg = I.request(i)
                codes, cot, nbytes, n, dec = page_dev[(c, pg)]
                fn(c, dicts[key], codes.data_ptr(), nbytes, cot.data_ptr(), n, out.data_ptr(), dec, offs.data_ptr(), sh)
                nb += dec
            b.record()
            torch.cuda.synchronize()
            wall = time.perf_counter() - t
            if fp.sync_status(sh) != fp.OK:
                raise RuntimeError(fp.last_error())
            return nb / max(a.elapsed_time(b) * 1e-3, wall) / 1e9

        n_plain = min(n_sat, args.serve_plain)
        plain_gbs = per_request(fp.decode_plain, n_plain)
        single_gbs = per_request(fp.decode, n_plain)
        _progress("served: per-request baselines done")
        extra["saturation"] = {"requests": n_sat, "served_gbs": round(sat_gbs, 2),
                               "plain_per_request_gbs": round(plain_gbs, 2),
                               "fp_decode_per_request_gbs": round(single_gbs, 2),
                               "served_over_plain": round(sat_gbs / plain_gbs, 2),
                               "plain_requests": n_plain}
        extra["plain_gpu"] = {"value": round(plain_gbs, 2), "unit": "GB/s",
                              "kind": "one plain decode (one thread per string) per request, back to back"}

        # end to end: host pages in, decoded bytes out, per request (closed loop)
        n_e2e = min(n_req, 200)
        host_in = {}
        for i in range(n_e2e):
            key, c, pg = I.request(i)
            if (c, pg) not in host_in:
                codes, cot, nbytes, n, dec = page_dev[(c, pg)]
                host_in[(c, pg)] = (codes.cpu().pin_memory(), cot.cpu().pin_memory())
        e2e_codes = {k: torch.empty_like(v[0], device=dev) for k, v in host_in.items()}
        e2e_co = {k: torch.empty_like(v[1], device=dev) for k, v in host_in.items()}
        h_out = torch.empty(big + 16, dtype=torch.uint8).pin_memory()
        h2d = d2h = 0
        t = time.perf_counter()
        tickets = []
        nb = 0
        for i in range(n_e2e):
            key, c, pg = I.request(i)
            codes, cot, nbytes, n, dec = page_dev[(c, pg)]
            hc, hco = host_in[(c, pg)]
            e2e_codes[(c, pg)].copy_(hc, non_blocking=True)
            e2e_co[(c, pg)].copy_(hco, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            h2d += hc.numel() + hco.numel() * 4
            tk = srv.submit(key, e2e_codes[(c, pg)].data_ptr(), nbytes, e2e_co[(c, pg)].data_ptr(), n, dec, i)
            r = None
            while r is None:
                for x in srv.poll(timeout_s=0.05):
                    r = x
            h_out[:r["bytes"]].copy_(fp.device_bytes(r["d_out_bytes"], r["bytes"]))
            d2h += r["bytes"]
            nb += r["bytes"]
            srv.release(r["ticket"])
        e2e_s = time.perf_counter() - t
        _progress("served: end-to-end leg done")
        extra["e2e"] = {"value": round(nb / e2e_s / 1e9, 3), "unit": "GB/s",
                        "h2d_bytes_per_step": int(h2d / n_e2e), "d2h_bytes_per_step": int(d2h / n_e2e),
                        "kind": f"{n_e2e} requests one at a time: pinned host page -> device, serve, result -> host"}

        # CPU oracle on the host cores, whole requests in arrival order
        import oracle
        threads = os.cpu_count() or 1
        done_b, t_cpu, k = 0, 0.0, 0
        while k < n_req and t_cpu < args.cpu_seconds:
            key, c, pg = I.request(k)
            col = I.host_column(key, c, pg)
            t = time.perf_counter()
            r = oracle.decode(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets,
                              threads=threads)
            t_cpu += time.perf_counter() - t
            done_b += r.total
            k += 1
        extra["cpu_baseline"] = {"value": round(done_b / t_cpu / 1e9, 4), "unit": "GB/s", "cores": threads,
                                 "kind": "oracle", "sample": f"first {k} requests ({done_b} decoded bytes), "
                                                             f"{t_cpu:.1f} s"}
    st2 = srv.stats()
    srv.destroy()
    faulthandler.cancel_dump_traceback_later()
    waves = st1["waves"] - st0["waves"]
    line = {
        "metric": SERVE_METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
        "steps": n_req, "warmup": warm, "ms_per_step": round(float(la.mean()), 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded generators; stand-in for the paper's real columns)",
        "latency_ms": {"p50": round(float(np.percentile(la, 50)), 3), "p99": round(float(np.percentile(la, 99)), 3),
                       "mean": round(float(la.mean()), 3), "max": round(float(la.max()), 3)},
        "config": {"workload": args.workload, "description": desc, "arrival_rate": rate, "seconds": seconds,
                   "requests": n_req, "decoded_bytes": tot_bytes, "offered_gbs": round(tot_bytes / seconds / 1e9, 2),
                   "late_submissions": late, "n_streams": args.serve_streams, "max_wave": args.serve_wave,
                   "batch_config": serve_cfg,
                   "waves": waves, "mean_wave": round((st1["admitted"] - st0["admitted"]) / max(waves, 1), 2),
                   "dict_hits": st1["dict_hits"] - st0["dict_hits"],
                   "dict_misses": st1["dict_misses"] - st0["dict_misses"],
                   "peak_inflight_bytes": st2["peak_inflight_bytes"], "hbm_budget": budget,
                   "generation_s": round(t_gen, 1), "parallelism": "single GPU",
                   "ms_per_step": "mean request latency"},
        "clocks": clocks,
        # per wave: index pass [+ reduce + tile scan] + the persistent decode kernel
        "gpu_launches": (4 if fp.batch_config_info(serve_cfg)["warp_tiles"] else 2) * waves,
    }
    line.update(extra)
    if "e2e" not in line:
        line["e2e"] = None
    print(json.dumps(line), flush=True)


def run_served_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    rate, seconds, lo, hi, n_keys, budget, desc = SERVE_WORKLOADS[args.workload]
    I = ServeInputs(rate, seconds, lo, hi, n_keys, seed=0)
    threads = os.cpu_count() or 1
    per_step = min(args.ref_seconds, 150.0 / (args.warmup + args.steps))
    vals, k, last = [], 0, (0, 0, 0.0)
    for s_i in range(args.warmup + args.steps):
        done_b, t_cpu, first = 0, 0.0, k
        while t_cpu < per_step:
            key, c, pg = I.request(k % I.arrivals.size)
            col = I.host_column(key, c, pg)
            t = time.perf_counter()
            r = oracle.decode(col.codec, col.dictionary.data, col.dictionary.offsets, col.stream, col.code_offsets,
                              threads=threads)
            t_cpu += time.perf_counter() - t
            done_b += r.total
            k += 1
        if s_i >= args.warmup:
            vals.append(done_b / t_cpu / 1e9)
            last = (k - first, done_b, t_cpu)
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": SERVE_METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(last[2] * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded generators; stand-in for the paper's real columns)",
        "config": {"workload": args.workload, "description": desc},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                         "sample": f"{last[0]} whole requests ({last[1]} decoded bytes) per step"},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="onpair12_10m",
                    choices=sorted(WORKLOADS) + sorted(ROWS_WORKLOADS) + sorted(BATCH_WORKLOADS) +
                    sorted(SERVE_WORKLOADS))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--settle", type=float, default=1.0, help="seconds of untimed decoding before warm-up")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-seconds", type=float, default=5.0)
    ap.add_argument("--plain-steps", type=int, default=5)
    ap.add_argument("--quick", action="store_true", help="skip the baselines and the e2e leg")
    ap.add_argument("--sidecar", action="store_true",
                    help="single-column workloads: time fp_decode_sidecar on a table built beforehand (implies --quick)")
    ap.add_argument("--variant", type=int, default=-1, help="decode variant (-1: built-in default)")
    ap.add_argument("--width", type=int, default=0, choices=[0, 8, 16],
                    help="OnPair dictionary read width (0: the dictionary's own, by the split-read rule)")
    ap.add_argument("--n-strings", type=int, default=0, help="override the workload's string count")
    ap.add_argument("--serve-seconds", type=float, default=0.0, help="served: length of the arrival process")
    ap.add_argument("--serve-streams", type=int, default=4, help="served: concurrent waves")
    ap.add_argument("--serve-wave", type=int, default=256, help="served: requests per wave")
    ap.add_argument("--serve-saturation", type=int, default=2000, help="served: requests of the closed-loop run")
    ap.add_argument("--serve-plain", type=int, default=500, help="served: requests of the per-request baselines")
    ap.add_argument("--serve-stall", type=float, default=60.0, help="served: give up after this long without a result")
    ap.add_argument("--serve-config", type=int, default=-1, help="served: batch configuration of the waves (-1: default)")
    ap.add_argument("--serve-watchdog", type=float, default=300.0, help="served: dump thread stacks every N s")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    rank, world, local_rank = env_rank()
    batched = args.workload in BATCH_WORKLOADS
    served = args.workload in SERVE_WORKLOADS
    rows = args.workload in ROWS_WORKLOADS
    if args.sidecar:
        if batched or served or rows:
            ap.error("--sidecar applies to the single-column workloads")
        args.quick = True
    if args.impl == "reference":
        (run_batched_reference if batched else run_served_reference if served else
         run_rows_reference if rows else run_reference)(args, rank, world)
    elif rows:
        run_rows(args, rank, world, local_rank)
    elif served:
        if world > 1 and rank != 0:
            return   # one server per GPU is the product's unit; the served bench runs on rank 0
        run_served(args, rank, world, local_rank)
    elif batched:
        run_batched(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
