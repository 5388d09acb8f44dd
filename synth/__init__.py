"""Seeded synthetic inputs for dictionary-compressed string columns.

This module is shared by the tests, the benchmark and the smoke check. It
produces *inputs* only: dictionaries in their interchange form (concatenated
token bytes plus ``uint32`` offsets), stored code streams and ``code_offsets``.
It performs no decoding: nothing here maps a code back to bytes, so it holds
none of the decoder's arithmetic.  The one bit-level routine, :func:`pack12`,
is the *writer* side of the 12-bit layout and is built from ``np.packbits``.

Randomness comes from numpy's Philox generator (a counter-based generator,
Salmon et al., SC'11) keyed by ``(workload id, seed, part)`` so that every
column is reproducible from its key.

Codec formats follow the paper's Sec. 2.1: OnPair-16 and OnPair-12 use 16-
and 12-bit codes into dictionaries of up to 65,536 / 4,096 tokens of at most
16 bytes; FSST-8 uses byte codes into a 255-symbol table of tokens of at most
8 bytes, with code 255 reserved as an escape followed by one literal byte;
FSST-12 uses 12-bit codes (stored like OnPair-12) into a table of up to 4,096
symbols of at most 8 bytes, with no escape.
"""
from __future__ import annotations

import dataclasses
import numpy as np

ONPAIR16, ONPAIR12, FSST8, FSST12 = 1, 2, 3, 4
CODEC_NAMES = {ONPAIR16: "onpair16", ONPAIR12: "onpair12", FSST8: "fsst8", FSST12: "fsst12"}
CODE_BITS = {ONPAIR16: 16, ONPAIR12: 12, FSST8: 8, FSST12: 12}
MAX_TOKEN = {ONPAIR16: 16, ONPAIR12: 16, FSST8: 8, FSST12: 8}
MAX_ENTRIES = {ONPAIR16: 65536, ONPAIR12: 4096, FSST8: 255, FSST12: 4096}
FSST_ESCAPE = 255

ALPHABET64 = np.frombuffer(
    b"ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789-_", np.uint8)
_LOWER = np.frombuffer(b"abcdefghijklmnopqrstuvwxyz", np.uint8)
_DIGITS = np.frombuffer(b"0123456789", np.uint8)
_HEX = np.frombuffer(b"0123456789abcdef", np.uint8)


def rng_for(*key: int) -> np.random.Generator:
    """Philox generator keyed by a tuple of non-negative ints."""
    return np.random.Generator(np.random.Philox(np.random.SeedSequence(list(key))))


@dataclasses.dataclass
class Dictionary:
    """A trained dictionary in interchange form: token ``i`` is
    ``data[offsets[i]:offsets[i+1]]``."""
    codec: int
    data: np.ndarray      # uint8, concatenated token bytes
    offsets: np.ndarray   # uint32, n_entries + 1

    @property
    def n_entries(self) -> int:
        return int(self.offsets.size - 1)

    def token_lengths(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64))

    @staticmethod
    def from_tokens(codec: int, tokens) -> "Dictionary":
        lens = np.array([len(t) for t in tokens], np.int64)
        offs = np.zeros(len(tokens) + 1, np.uint32)
        offs[1:] = np.cumsum(lens)
        data = np.frombuffer(b"".join(bytes(t) for t in tokens), np.uint8).copy()
        return Dictionary(codec, data, offs)

    def tokens(self):
        d = self.data.tobytes()
        o = self.offsets
        return [d[o[i]:o[i + 1]] for i in range(self.n_entries)]


@dataclasses.dataclass
class Column:
    """A compressed string column as it is stored.

    ``stream`` is the stored code buffer: little-endian uint16 codes for
    OnPair-16, the 12-bit LSB-first bitstream for OnPair-12, code and literal
    bytes ("slots") for FSST-8.  ``code_offsets[i]`` is the index of string
    ``i``'s first code slot; string ``i`` owns slots
    ``[code_offsets[i], code_offsets[i+1])``.
    """
    codec: int
    dictionary: Dictionary
    stream: np.ndarray        # uint8 stored code buffer
    code_offsets: np.ndarray  # uint32, n_strings + 1
    n_slots: int              # code slots in the stream
    # Generator-side bookkeeping (what the encoder emitted), for invariants:
    slot_codes: np.ndarray | None = None   # per slot: code, or literal byte (FSST)
    slot_is_literal: np.ndarray | None = None
    name: str = ""

    @property
    def n_strings(self) -> int:
        return int(self.code_offsets.size - 1)


# ---------------------------------------------------------------------------
# Stored-layout writers (encoder side)
# ---------------------------------------------------------------------------

def pack12(codes: np.ndarray, chunk: int = 1 << 22) -> np.ndarray:
    """Write 12-bit codes as an LSB-first bitstream: code ``i`` occupies
    stream bits ``[12 i, 12 i + 12)`` and stream bit ``b`` is bit ``b % 8`` of
    byte ``b // 8``.  The last byte is zero-padded."""
    codes = np.asarray(codes, dtype=np.uint16)
    if codes.size and int(codes.max()) >= 4096:
        raise ValueError("12-bit code out of range")
    out = np.zeros((codes.size * 12 + 7) // 8, np.uint8)
    chunk -= chunk % 2  # even chunks start on a byte boundary (2 codes = 3 bytes)
    for s in range(0, codes.size, chunk):
        c = codes[s:s + chunk]
        bits = np.unpackbits(c.astype("<u2").view(np.uint8).reshape(-1, 2),
                             axis=1, bitorder="little")[:, :12]
        packed = np.packbits(bits.reshape(-1), bitorder="little")
        out[s * 12 // 8: s * 12 // 8 + packed.size] = packed
    return out


def pack16(codes: np.ndarray) -> np.ndarray:
    return np.asarray(codes, dtype="<u2").view(np.uint8).copy()


# ---------------------------------------------------------------------------
# Distributions
# ---------------------------------------------------------------------------

def zipf_cdf(n: int, s: float) -> np.ndarray:
    w = np.arange(1, n + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def zipf_draw(rng: np.random.Generator, cdf: np.ndarray, size: int) -> np.ndarray:
    """Ranks 0..n-1 with P(rank k) proportional to (k+1)^-s."""
    r = np.searchsorted(cdf, rng.random(size), side="right")
    return np.minimum(r, cdf.size - 1)


def _random_strings(rng, alphabet: np.ndarray, lengths: np.ndarray) -> list[bytes]:
    tot = int(lengths.sum())
    pool = alphabet[rng.integers(0, alphabet.size, tot)].tobytes()
    out, p = [], 0
    for L in lengths.tolist():
        out.append(pool[p:p + L])
        p += L
    return out


# ---------------------------------------------------------------------------
# Dictionaries
# ---------------------------------------------------------------------------

def onpair16_dictionary(seed: int, n_entries: int = 65536) -> Dictionary:
    """65,536 tokens of 1-16 random bytes over a 64-symbol printable alphabet.
    Lengths are geometric with mean 6 (p = 1/6), redrawn until <= 16."""
    rng = rng_for(1, seed, 0)
    lens = rng.geometric(1.0 / 6.0, n_entries)
    bad = lens > 16
    while bad.any():
        lens[bad] = rng.geometric(1.0 / 6.0, int(bad.sum()))
        bad = lens > 16
    offs = np.zeros(n_entries + 1, np.uint32)
    offs[1:] = np.cumsum(lens)
    data = ALPHABET64[rng.integers(0, 64, int(offs[-1]))]
    return Dictionary(ONPAIR16, data.astype(np.uint8), offs)


def _log_tokens(rng, count: int) -> list[bytes]:
    """Distinct log-line-like tokens of 2..16 bytes: timestamp pieces, hex ids,
    lowercase words, level/key words and punctuation runs."""
    seen: set[bytes] = set()
    out: list[bytes] = []
    punct = [b" ", b"-", b":", b"[", b"]", b"(", b")", b",", b"=", b"/", b".",
             b"|", b";", b"_", b"'", b'"', b"<", b">", b"#", b"@", b"\t"]
    levels = [b"INFO", b"WARN", b"ERROR", b"DEBUG", b"TRACE", b"FATAL", b"NOTICE"]
    while len(out) < count:
        kind = int(rng.integers(0, 100))
        if kind < 22:    # timestamp pieces
            f = int(rng.integers(0, 6))
            n = rng.integers(0, 10000)
            if f == 0:
                t = b"%04d-%02d-" % (1990 + n % 40, 1 + n % 12)
            elif f == 1:
                t = b"%02d:%02d:" % (n % 24, (n // 24) % 60)
            elif f == 2:
                t = b"%02d.%03d " % (n % 60, n % 1000)
            elif f == 3:
                t = b"T%02d:%02d:%02d" % (n % 24, (n // 24) % 60, (n // 7) % 60)
            elif f == 4:
                t = b" %02d:" % (n % 60)
            else:
                t = b"%02d " % (n % 100)
        elif kind < 42:  # hex ids
            L = int(rng.integers(4, 15))
            t = _random_strings(rng, _HEX, np.array([L]))[0]
            if rng.random() < 0.3:
                t = (b"0x" + t)[:16]
        elif kind < 74:  # lowercase words with optional spacing
            L = int(rng.integers(2, 11))
            t = _random_strings(rng, _LOWER, np.array([L]))[0]
            r = rng.random()
            if r < 0.35:
                t = t + b" "
            elif r < 0.5:
                t = b" " + t
            elif r < 0.6:
                t = t + b"="
        elif kind < 82:  # levels and keys
            if rng.random() < 0.4:
                t = levels[int(rng.integers(0, len(levels)))]
                t = (b" " + t + b" ") if rng.random() < 0.5 else (b"[" + t + b"]")
            else:
                L = int(rng.integers(2, 8))
                t = _random_strings(rng, _LOWER, np.array([L]))[0] + b"="
        elif kind < 92:  # numbers
            L = int(rng.integers(2, 9))
            t = _random_strings(rng, _DIGITS, np.array([L]))[0]
        else:            # punctuation runs
            L = int(rng.integers(2, 5))
            t = b"".join(punct[int(i)] for i in rng.integers(0, len(punct), L))
        t = t[:16]
        if len(t) < 2 or t in seen:
            continue
        seen.add(t)
        out.append(t)
    return out


def onpair12_dictionary(seed: int) -> Dictionary:
    """4,096 tokens: codes 0..255 are the one-byte literals (Sec. 2.1: OnPair
    places every one-byte literal in its dictionary); codes 256..4095 are
    distinct log-line-like tokens of 2..16 bytes."""
    rng = rng_for(2, seed, 0)
    toks = [bytes([b]) for b in range(256)] + _log_tokens(rng, 4096 - 256)
    return Dictionary.from_tokens(ONPAIR12, toks)


def _url_tokens(rng, count: int) -> list[bytes]:
    fixed = [b"http", b"https", b"://", b"www.", b".com", b".org", b".net", b".html",
             b"/", b"?", b"&", b"=", b"%20", b"id", b"_", b"-", b".", b"index",
             b"user", b"page", b"search", b"q=", b"ref=", b"utm_", b"/api/", b"v1",
             b"/img/", b".png", b".jpg", b"item", b"cat", b"sess", b"uid="]
    seen: set[bytes] = set()
    out: list[bytes] = []
    for t in fixed:
        if len(out) < count and t not in seen:
            seen.add(t)
            out.append(t)
    while len(out) < count:
        kind = int(rng.integers(0, 10))
        if kind < 5:
            L = int(rng.integers(1, 9))
            t = _random_strings(rng, _LOWER, np.array([L]))[0]
        elif kind < 7:
            L = int(rng.integers(1, 5))
            t = _random_strings(rng, _DIGITS, np.array([L]))[0]
        elif kind < 9:
            L = int(rng.integers(2, 8))
            t = _random_strings(rng, _LOWER, np.array([L]))[0]
            t = (t + (b"/" if rng.random() < 0.5 else b"_"))[:8]
        else:
            L = int(rng.integers(1, 9))
            t = _random_strings(rng, ALPHABET64, np.array([L]))[0]
        if t in seen:
            continue
        seen.add(t)
        out.append(t)
    return out


def fsst8_dictionary(seed: int) -> Dictionary:
    """255 URL/identifier-like symbols of 1..8 bytes (codes 0..254)."""
    rng = rng_for(3, seed, 0)
    return Dictionary.from_tokens(FSST8, _url_tokens(rng, 255))


def fsst12_dictionary(seed: int, n_entries: int = 4096) -> Dictionary:
    """n_entries symbols (257..4,096): codes 0..255 are the one-byte symbols
    (an escape-free table must cover every byte), the rest distinct
    URL/identifier-like symbols of 2..8 bytes."""
    rng = rng_for(4, seed, 0, n_entries)
    want = n_entries - 256
    multi = [t for t in _url_tokens(rng, 6000) if len(t) >= 2][:want]
    while len(multi) < want:
        extra = [t for t in _url_tokens(rng, 2000) if len(t) >= 2 and t not in set(multi)]
        multi += extra[:want - len(multi)]
    return Dictionary.from_tokens(FSST12, [bytes([b]) for b in range(256)] + multi)


def pack_bits(codes: np.ndarray, bits: int, chunk: int = 1 << 22) -> np.ndarray:
    """Codes bit-packed at ``bits`` bits per code, LSB-first (code i at stream
    bits [bits i, bits i + bits)): the cascaded storage of a code column,
    written with np.packbits."""
    codes = np.asarray(codes, np.uint32)
    out = []
    step = chunk - chunk % 8   # whole bytes per chunk
    for a in range(0, codes.size, step):
        c = codes[a:a + step]
        b = ((c[:, None] >> np.arange(bits, dtype=np.uint32)) & 1).astype(np.uint8).reshape(-1)
        out.append(np.packbits(b, bitorder="little"))
    return np.concatenate(out) if out else np.zeros(0, np.uint8)


# ---------------------------------------------------------------------------
# Columns
# ---------------------------------------------------------------------------

def _fill_rounds(rng, targets: np.ndarray, draw):
    """Grow every string by one unit per round until its byte target is met.

    ``draw(rng, remaining)`` returns ``(codes, nbytes, is_escape)`` for the
    active strings.  Returns the units in string order and per-string unit
    counts."""
    n = targets.size
    remaining = targets.astype(np.int64).copy()
    active = np.arange(n, dtype=np.int64)
    counts = np.zeros(n, np.int64)
    rounds = []
    while active.size:
        codes, nbytes, esc = draw(rng, remaining[active])
        remaining[active] -= nbytes
        rounds.append((active, codes, esc))
        counts[active] += 1
        active = active[remaining[active] > 0]
    starts = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=starts[1:])
    units = np.empty(int(starts[-1]), np.uint16)
    units_esc = np.zeros(int(starts[-1]), bool)
    for r, (act, codes, esc) in enumerate(rounds):
        pos = starts[act] + r
        units[pos] = codes
        if esc is not None:
            units_esc[pos] = esc
    return units, units_esc, starts


def onpair16_column(seed: int = 0, n_strings: int = 100_000, dictionary=None,
                    max_codes: int = 40, zipf_s: float = 1.1) -> Column:
    """Each string has 1..max_codes codes (uniform count); codes are drawn
    Zipf(zipf_s) over the dictionary, ranks mapped to codes by a seeded
    permutation."""
    d = dictionary if dictionary is not None else onpair16_dictionary(seed)
    rng = rng_for(1, seed, 1)
    counts = rng.integers(1, max_codes + 1, n_strings)
    offs = np.zeros(n_strings + 1, np.int64)
    np.cumsum(counts, out=offs[1:])
    perm = rng.permutation(d.n_entries).astype(np.uint16)
    ranks = zipf_draw(rng, zipf_cdf(d.n_entries, zipf_s), int(offs[-1]))
    codes = perm[ranks]
    return Column(ONPAIR16, d, pack16(codes), offs.astype(np.uint32), int(codes.size),
                  slot_codes=codes, slot_is_literal=np.zeros(codes.size, bool),
                  name=f"onpair16 seed={seed} n={n_strings}")


def onpair12_column(seed: int = 0, n_strings: int = 10_000_000, dictionary=None,
                    lo: int = 20, hi: int = 200, zipf_s: float = 1.2) -> Column:
    """Strings of lo..hi decoded bytes (uniform target).  Codes are drawn
    Zipf(zipf_s) over the multi-byte tokens; a token that would overshoot the
    target is replaced by a one-byte literal code (printable ASCII), so every
    string decodes to exactly its target length."""
    d = dictionary if dictionary is not None else onpair12_dictionary(seed)
    rng = rng_for(2, seed, 1)
    lens = d.token_lengths()
    multi = np.nonzero(lens >= 2)[0]
    perm = multi[rng.permutation(multi.size)].astype(np.uint16)
    cdf = zipf_cdf(perm.size, zipf_s)
    tok_len = lens.astype(np.int64)

    def draw(rng, remaining):
        c = perm[zipf_draw(rng, cdf, remaining.size)]
        L = tok_len[c]
        lit = rng.integers(32, 127, remaining.size).astype(np.uint16)
        fits = L <= remaining
        return np.where(fits, c, lit), np.where(fits, L, 1), None

    targets = rng.integers(lo, hi + 1, n_strings)
    codes, _, starts = _fill_rounds(rng, targets, draw)
    return Column(ONPAIR12, d, pack12(codes), starts.astype(np.uint32), int(codes.size),
                  slot_codes=codes, slot_is_literal=np.zeros(codes.size, bool),
                  name=f"onpair12 seed={seed} n={n_strings}")


def fsst8_column(seed: int = 0, n_strings: int = 16_000_000, dictionary=None,
                 median: float = 40.0, sigma: float = 0.6, p_escape: float = 0.01,
                 zipf_s: float = 1.0) -> Column:
    """Lognormal target lengths (median, sigma), at least 1 byte.  Each unit is
    an escape (code 255) plus a uniform literal byte 0..255 with probability
    p_escape, else a symbol drawn Zipf(zipf_s) over the 255 symbols.  The last
    unit may overshoot the target."""
    d = dictionary if dictionary is not None else fsst8_dictionary(seed)
    rng = rng_for(3, seed, 1)
    perm = rng.permutation(d.n_entries).astype(np.uint16)
    cdf = zipf_cdf(d.n_entries, zipf_s)
    tok_len = d.token_lengths().astype(np.int64)

    def draw(rng, remaining):
        k = remaining.size
        c = perm[zipf_draw(rng, cdf, k)]
        esc = rng.random(k) < p_escape
        lit = rng.integers(0, 256, k).astype(np.uint16)
        return np.where(esc, lit, c), np.where(esc, 1, tok_len[c]), esc

    targets = np.maximum(1, np.rint(median * np.exp(sigma * rng.standard_normal(n_strings)))).astype(np.int64)
    units, esc, ustarts = _fill_rounds(rng, targets, draw)
    # Expand units to slots: an escaped literal takes two slots (255, byte).
    width = 1 + esc.astype(np.int64)
    upos = np.zeros(units.size + 1, np.int64)
    np.cumsum(width, out=upos[1:])
    stream = np.empty(int(upos[-1]), np.uint8)
    lit_flag = np.zeros(int(upos[-1]), bool)
    stream[upos[:-1]] = np.where(esc, FSST_ESCAPE, units).astype(np.uint8)
    epos = upos[:-1][esc] + 1
    stream[epos] = units[esc].astype(np.uint8)
    lit_flag[epos] = True
    code_offsets = upos[ustarts]
    return Column(FSST8, d, stream, code_offsets.astype(np.uint32), int(stream.size),
                  slot_codes=stream.astype(np.uint16), slot_is_literal=lit_flag,
                  name=f"fsst8 seed={seed} n={n_strings}")


def fsst12_column(seed: int = 0, n_strings: int = 16_000_000, dictionary=None,
                  median: float = 40.0, sigma: float = 0.6, zipf_s: float = 1.0) -> Column:
    """Lognormal target lengths (median, sigma), at least 1 byte; every code
    is a symbol drawn Zipf(zipf_s) over the whole table through a seeded
    permutation (no escapes).  The last symbol may overshoot the target."""
    d = dictionary if dictionary is not None else fsst12_dictionary(seed)
    rng = rng_for(4, seed, 1)
    perm = rng.permutation(d.n_entries).astype(np.uint16)
    cdf = zipf_cdf(d.n_entries, zipf_s)
    tok_len = d.token_lengths().astype(np.int64)

    def draw(rng, remaining):
        c = perm[zipf_draw(rng, cdf, remaining.size)]
        return c, tok_len[c], None

    targets = np.maximum(1, np.rint(median * np.exp(sigma * rng.standard_normal(n_strings)))).astype(np.int64)
    codes, _, starts = _fill_rounds(rng, targets, draw)
    return Column(FSST12, d, pack12(codes), starts.astype(np.uint32), int(codes.size),
                  slot_codes=codes, slot_is_literal=np.zeros(codes.size, bool),
                  name=f"fsst12 seed={seed} n={n_strings}")


# Full-size workloads (seed 0) and the small parity cases built with the same
# recipe.
WORKLOADS = {
    "onpair16_100k": lambda seed=0: onpair16_column(seed, 100_000),
    "onpair12_10m": lambda seed=0: onpair12_column(seed, 10_000_000),
    "fsst8_16m": lambda seed=0: fsst8_column(seed, 16_000_000),
    "fsst12_16m": lambda seed=0: fsst12_column(seed, 16_000_000),
}


def column(codec: int, seed: int, n_strings: int, **kw) -> Column:
    if codec == ONPAIR16:
        return onpair16_column(seed, n_strings, **kw)
    if codec == ONPAIR12:
        return onpair12_column(seed, n_strings, **kw)
    if codec == FSST8:
        return fsst8_column(seed, n_strings, **kw)
    if codec == FSST12:
        return fsst12_column(seed, n_strings, **kw)
    raise ValueError(codec)


# ---------------------------------------------------------------------------
# Batches of chunks and served requests: many columns, each with its own
# dictionary, cut from per-codec pools of code streams.  Any code stream is
# valid under any full dictionary of its codec (every code has a token), so
# a chunk pairs a window of its codec's pool with its own dictionary.
# ---------------------------------------------------------------------------

def onpair12_dictionary_variant(base: Dictionary, seed: int) -> Dictionary:
    """A distinct OnPair-12 dictionary from a base one: the one-byte literals
    stay at codes 0..255, the multi-byte tokens are permuted over codes
    256..4095 (seeded)."""
    rng = rng_for(2, seed, 7)
    n = base.n_entries
    idx = np.concatenate([np.arange(256), 256 + rng.permutation(n - 256)])
    lens = base.token_lengths()[idx]
    offs = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    src = np.repeat(base.offsets[:-1].astype(np.int64)[idx] - offs[:-1], lens) + np.arange(int(offs[-1]))
    return Dictionary(ONPAIR12, base.data[src].copy(), offs.astype(np.uint32))


def chunk_dictionary(codec: int, seed: int, onpair12_bases=None) -> Dictionary:
    """The dictionary of chunk `seed`: generated as for the single-column
    workloads (OnPair-12: a permuted variant of one of a few base
    dictionaries, which are slow to draw)."""
    if codec == ONPAIR16:
        return onpair16_dictionary(seed)
    if codec == FSST8:
        return fsst8_dictionary(seed)
    bases = onpair12_bases if onpair12_bases is not None else [onpair12_dictionary(0)]
    return onpair12_dictionary_variant(bases[seed % len(bases)], seed)


def log_uniform_sizes(rng, n: int, lo: int, hi: int) -> np.ndarray:
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n)).astype(np.int64)


def codec_mix(rng, n: int, ratio=(2, 1, 1)) -> np.ndarray:
    """Codecs in ratio OnPair-16 : OnPair-12 : FSST-8, shuffled."""
    r = np.asarray(ratio, np.float64)
    counts = np.floor(n * r / r.sum()).astype(np.int64)
    counts[0] += n - counts.sum()
    codecs = np.repeat(np.array([ONPAIR16, ONPAIR12, FSST8]), counts)
    return codecs[rng.permutation(n)]


def pool_window(pool: Column, start: int, n_strings: int):
    """Strings [start, start + n) of a pool column as a chunk: the byte range of
    the pool's stored code buffer that holds them, starting on a 48-byte
    boundary (a whole number of slots for every codec and 16-byte aligned),
    and code_offsets rebased to that range.  Returns (byte0, byte1, code_offsets)."""
    w = CODE_BITS[pool.codec]
    co = pool.code_offsets[start:start + n_strings + 1].astype(np.int64)
    first_byte = int(co[0]) * w // 8
    byte0 = first_byte - first_byte % 48
    slot0 = byte0 * 8 // w
    end_byte = (int(co[-1]) * w + 7) // 8
    return byte0, end_byte, (co - slot0).astype(np.uint32)


def same_shape_dictionary(base: Dictionary, seed: int) -> Dictionary:
    """A distinct dictionary with the token lengths of `base` code by code:
    the tokens of each length are permuted among the codes of that length
    (seeded).  Every code stream then decodes to the same number of bytes
    under `base` and under the new dictionary."""
    rng = rng_for(5, seed, base.codec)
    lens = base.token_lengths()
    idx = np.arange(lens.size)
    for L in np.unique(lens):
        sel = np.nonzero(lens == L)[0]
        idx[sel] = sel[rng.permutation(sel.size)]
    offs = base.offsets.astype(np.int64)
    src = np.repeat(offs[:-1][idx] - offs[:-1], lens) + np.arange(int(offs[-1]))
    return Dictionary(base.codec, base.data[src].copy(), base.offsets.copy())


def slot_bytes(col: Column) -> np.ndarray:
    """Decoded bytes each slot of a generated column contributes (from the
    generator's bookkeeping and the token lengths): the column's length
    profile, for sizing outputs of windows of it."""
    lens = col.dictionary.token_lengths()
    if col.codec == FSST8:
        codes = np.minimum(col.slot_codes, lens.size - 1)
        return np.where(col.slot_is_literal, 1, np.where(col.slot_codes == FSST_ESCAPE, 0, lens[codes]))
    return lens[col.slot_codes]
