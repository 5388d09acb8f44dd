"""The tile scan packs an FSST-8 element's second byte count as a 5-bit
difference from the first (fp_decoder.cuh, agg_payload_wide): over any run
of slots, the parse entered on a code and the parse entered on a literal
produce byte counts that differ by at most 8.  Checked here by exhaustive
enumeration of short slot sequences (escape 255 or a code of length 1..8)
and by random long ones, with a direct two-state parse."""
import itertools

import numpy as np


def parse_bytes(slots, lens, literal_first):
    """Bytes produced by slots entered in the given state, and the exit state."""
    state, total = literal_first, 0
    for s in slots:
        if state:
            total += 1          # a literal byte
            state = 0
        elif s == 255:
            state = 1           # escape: the next slot is a literal
        else:
            total += lens[s]
    return total, state


def test_two_parses_differ_by_at_most_8_exhaustive():
    lens = {c: c for c in range(1, 9)}          # code c has length c
    alphabet = [255, 1, 8]                      # escape, shortest and longest token
    worst = 0
    for n in range(1, 11):
        for slots in itertools.product(alphabet, repeat=n):
            b0, _ = parse_bytes(slots, lens, 0)
            b1, _ = parse_bytes(slots, lens, 1)
            worst = max(worst, abs(b1 - b0))
    assert worst <= 8


def test_two_parses_differ_by_at_most_8_random():
    rng = np.random.default_rng(0)
    lens = {c: 1 + c % 8 for c in range(255)}
    for _ in range(2000):
        n = int(rng.integers(1, 200))
        p255 = rng.choice([0.0, 0.3, 0.7, 0.95])
        slots = np.where(rng.random(n) < p255, 255, rng.integers(0, 255, n))
        b0, _ = parse_bytes(slots.tolist(), lens, 0)
        b1, _ = parse_bytes(slots.tolist(), lens, 1)
        assert abs(b1 - b0) <= 8
