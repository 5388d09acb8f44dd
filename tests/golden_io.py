"""Readers for the hand-written fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CODECS = {"onpair16": 1, "onpair12": 2, "fsst8": 3, "fsst12": 4}


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.split("#", 1)[0].strip()
            if ln:
                yield ln


def _hex(s):
    return bytes(int(t, 16) for t in s.split())


def concat_cases(name="concat_small.txt"):
    cases, cur = [], {}
    for ln in _lines(name):
        key, _, rest = ln.partition(" ")
        if key == "end":
            cases.append(cur)
            cur = {}
        elif key == "codec":
            cur["codec"] = CODECS[rest.strip()]
        elif key == "tokens":
            cur["tokens"] = [bytes.fromhex(t) for t in rest.split()]
        elif key in ("code_offsets", "expect_offsets"):
            cur[key] = np.array([int(t) for t in rest.split()], np.uint32)
        elif key in ("stream", "expect_data"):
            cur[key] = _hex(rest)
    return cases


def pack12_cases(name="pack12_examples.txt"):
    out = []
    for ln in _lines(name):
        lhs, rhs = ln.split("->")
        out.append(([int(t, 16) for t in lhs.split()], _hex(rhs)))
    return out


def fsst8_escape_cases(name="fsst8_escapes.txt"):
    out = []
    for ln in _lines(name):
        lhs, rhs = ln.split("->")
        rhs = rhs.strip()
        out.append((_hex(lhs), None if rhs == "CORRUPT" else _hex(rhs)))
    return out


def sidecar_cases(name="sidecar_small.txt"):
    """Stored-sidecar fixtures: a column plus `tile` and the expected table."""
    cases, cur = [], {}
    for ln in _lines(name):
        key, _, rest = ln.partition(" ")
        if key == "end":
            cases.append(cur)
            cur = {}
        elif key == "codec":
            cur["codec"] = CODECS[rest.strip()]
        elif key == "tokens":
            cur["tokens"] = [bytes.fromhex(t) for t in rest.split()]
        elif key == "code_offsets":
            cur[key] = np.array([int(t) for t in rest.split()], np.uint32)
        elif key == "stream":
            cur[key] = _hex(rest)
        elif key == "tile":
            cur[key] = int(rest)
        elif key == "expect_sidecar":
            cur[key] = np.array([int(t) for t in rest.split()], np.uint64)
    return cases


def packed_cases(name="packed_examples.txt"):
    """(bits, codes, stream bytes) of the hand-packed examples."""
    out = []
    for ln in _lines(name):
        head, _, rest = ln.partition(":")
        codes_s, _, stream_s = rest.partition("->")
        out.append((int(head), [int(t, 16) for t in codes_s.split()], _hex(stream_s)))
    return out
