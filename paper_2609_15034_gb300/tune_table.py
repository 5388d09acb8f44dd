"""Write the decoder's tuning table for the GPU this runs on.

For every codec and read width, and for seeded synthetic columns from ten
thousand to ten million strings (the workloads' recipes, `synth`), run
fp_tune_column -- every compiled shape of the codec and width timed on the
column -- and append the fastest per size class to the table.  The binding
loads `tuning/gb300.txt` beside this file at start-up; entries are keyed by
the SM count, so a table from another GPU model stays unused.

    python -m paper_2609_15034_gb300.tune_table [output path]
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SIZES = [10_000, 30_000, 100_000, 300_000, 1_000_000, 3_000_000, 10_000_000]


def main(out_path: str) -> None:
    import torch

    import synth
    import paper_2609_15034_gb300 as fp

    os.makedirs(os.path.dirname(out_path), exist_ok=True)
    if os.path.exists(out_path):
        os.remove(out_path)
    with open(out_path, "w") as f:
        f.write(f"# sms codec width size_class variant ms -- {torch.cuda.get_device_name(0)}\n")
    fp.tune_clear()
    for codec in (synth.ONPAIR16, synth.ONPAIR12, synth.FSST8, synth.FSST12):
        widths = (16, 8) if codec in (synth.ONPAIR16, synth.ONPAIR12) else (8,)
        for n in SIZES:
            col = synth.column(codec, 0, n)
            d = fp.Dict(codec, col.dictionary.data, col.dictionary.offsets)
            codes = torch.from_numpy(col.stream).cuda()
            co = torch.from_numpy(col.code_offsets.view(np.int32)).cuda()
            st, total = fp.decoded_size_tensors(codec, d, codes, co, n)
            assert st == fp.OK, fp.last_error()
            out = torch.empty(total, dtype=torch.uint8, device="cuda")
            offs = torch.empty(n + 1, dtype=torch.int32, device="cuda")
            for w in widths:
                d.set_width(w)
                st, v, ms = fp.tune_column(codec, d, codes.data_ptr(), codes.numel(), co.data_ptr(), n, out.data_ptr(),
                                           total, offs.data_ptr(), out_path)
                assert st == fp.OK, fp.last_error()
                print(f"codec {codec} width {w} strings {n}: variant {v} {ms:.4f} ms", flush=True)
            d.free()
            del codes, co, out, offs
            torch.cuda.empty_cache()


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(HERE, "tuning", "gb300.txt"))
