"""Brute-force greedy encoder (test infrastructure only).

Used for round trips: ``decode(encode(s)) == s``.  At every input position it
tries every dictionary token and takes the longest one that matches; among
equally long matches it takes the lowest code.  For FSST-8, a position that
no symbol matches is written as the escape code 255 followed by the literal
byte (paper Sec. 2.1).  For OnPair codecs an unmatched byte is an error: their
dictionaries hold every one-byte literal (Sec. 2.1), so this only happens for
dictionaries built without them.
"""
from __future__ import annotations

import numpy as np

FSST8 = 3
ESCAPE = 255


def greedy_encode(tokens: list[bytes], text: bytes, fsst8: bool) -> list[int]:
    """Return the slot sequence (codes, and literal bytes after escapes)."""
    out: list[int] = []
    i = 0
    while i < len(text):
        best, best_len = -1, 0
        for code, tok in enumerate(tokens):
            L = len(tok)
            if L > best_len and text.startswith(tok, i):
                best, best_len = code, L
        if best < 0:
            if not fsst8:
                raise ValueError(f"byte {text[i]!r} at {i} is not covered by the dictionary")
            out += [ESCAPE, text[i]]
            i += 1
        else:
            out.append(best)
            i += best_len
    return out


def encode_column(tokens: list[bytes], strings: list[bytes], codec: int):
    """Encode strings into (slot list, code_offsets)."""
    slots: list[int] = []
    offs = [0]
    for s in strings:
        slots += greedy_encode(tokens, s, codec == FSST8)
        offs.append(len(slots))
    return slots, np.array(offs, np.uint32)
