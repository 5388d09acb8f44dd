/*
 * Plain CPU oracle for decoding dictionary-compressed string columns.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load or call this code.  It shares no
 * source, header, table or helper with the CUDA decoder.
 *
 * What it computes (the plain definition the GPU decoder must reproduce):
 *   - Decoding concatenates the tokens that the codes index, with no padding
 *     between tokens (paper Sec. 1 and Sec. 2.1; Sec. 3 "tokens are
 *     concatenated without padding").
 *   - Codec formats (Sec. 2.1): OnPair-16 = 16-bit codes, OnPair-12 = 12-bit
 *     codes, both into dictionaries of tokens of at most 16 bytes; FSST-8 =
 *     byte codes into a 255-symbol table of tokens of at most 8 bytes, where
 *     the reserved escape code 255 is followed by one literal byte; FSST-12
 *     = 12-bit codes into a table of up to 4,096 symbols of at most 8 bytes,
 *     with no escape (the paper's escape-free variant, stored like
 *     OnPair-12).
 *   - Output (Sec. 5): a variable-length string array: byte-packed string
 *     data plus an array of fixed-width offsets (uint32 here).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - 12-bit codes are stored as an LSB-first bitstream: code i occupies
 *     stream bits [12i, 12i+12), stream bit b is bit (b mod 8) of byte b/8.
 *   - OnPair-16 codes are little-endian 16-bit words.
 *   - code_offsets index code *slots*; for FSST-8 a literal byte is a slot.
 *   - An escape in the last slot of a string (no literal follows) and a code
 *     >= n_entries are corrupt input.  A corrupt code contributes no bytes.
 *   - out_offsets[0] = 0 even when code_offsets[0] != 0.
 *
 * Every loop is the definition written out: the 12-bit reader goes bit by
 * bit, token copies go byte by byte, and nothing is over-copied.
 *
 * Cascaded codes (fpo_decode_packed): the paper prepares columns on the host
 * by widening their stored, bit-packed codes (Sec. 5).  That layer is read
 * here as codes bit-packed at a width of b bits, LSB-first: code i occupies
 * stream bits [b i, b i + b) (b = 12 is the OnPair-12 / FSST-12 layout, b =
 * 16 the OnPair-16 one); everything else is the codec's decode.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

enum { FPO_ONPAIR16 = 1, FPO_ONPAIR12 = 2, FPO_FSST8 = 3, FPO_FSST12 = 4 };
enum { FPO_OK = 0, FPO_ERR_ARG = 1, FPO_ERR_CORRUPT = 4, FPO_ERR_CAPACITY = 5,
       FPO_ERR_OVERFLOW = 6 };
/* error kinds reported as a bit set */
enum { FPO_BIT_CORRUPT = 1, FPO_BIT_CAPACITY = 2, FPO_BIT_OVERFLOW = 4 };

static int code_bits(int codec) {
    return codec == FPO_ONPAIR16 ? 16 : (codec == FPO_ONPAIR12 || codec == FPO_FSST12) ? 12
                                      : codec == FPO_FSST8 ? 8 : 0;
}

/* Read stream bit b (LSB-first within each byte). */
static unsigned read_bit(const uint8_t* stream, uint64_t b) {
    return (stream[b / 8] >> (b % 8)) & 1u;
}

/* Code in slot s of a stored stream. */
static uint32_t read_code(int codec, const uint8_t* stream, uint64_t s) {
    if (codec == FPO_ONPAIR16) {
        return (uint32_t)stream[2 * s] | ((uint32_t)stream[2 * s + 1] << 8);
    }
    if (codec == FPO_ONPAIR12 || codec == FPO_FSST12) {
        uint32_t c = 0;
        for (unsigned k = 0; k < 12; ++k) c |= read_bit(stream, 12 * s + k) << k;
        return c;
    }
    return stream[s];
}

/* Unpack n 12-bit codes, bit by bit. */
void fpo_unpack12(const uint8_t* stream, uint64_t n, uint16_t* out) {
    for (uint64_t i = 0; i < n; ++i) out[i] = (uint16_t)read_code(FPO_ONPAIR12, stream, i);
}

typedef struct {
    int codec;
    const uint8_t* dict_bytes;
    const uint32_t* dict_offsets;
    uint32_t n_entries;
    const uint8_t* stream;
    uint64_t n_slots;          /* whole code slots present in the stream */
    const uint32_t* code_offsets;
    int packed_bits;           /* 0: the codec's stored layout; else codes bit-packed at this width */
} column_t;

/* Code in slot s of a column: the codec's layout, or b-bit packing read
 * bit by bit. */
static uint32_t column_code(const column_t* c, uint64_t s) {
    if (!c->packed_bits) return read_code(c->codec, c->stream, s);
    uint32_t v = 0;
    for (int k = 0; k < c->packed_bits; ++k) v |= read_bit(c->stream, (uint64_t)c->packed_bits * s + k) << k;
    return v;
}

/*
 * Decode strings [s0, s1) into out (whose byte 0 corresponds to output
 * position base).  When out is NULL only the sizes are computed.  Writes
 * relative string ends into ends[i - s0] (may be NULL).  Returns the number
 * of bytes produced and ORs error bits into *err.  Bytes beyond `cap`
 * (absolute) are not written.
 */
static uint64_t decode_range(const column_t* c, uint32_t s0, uint32_t s1, uint8_t* out,
                             uint64_t base, uint64_t cap, uint64_t* ends, unsigned* err) {
    uint64_t pos = base;
    for (uint32_t i = s0; i < s1; ++i) {
        uint64_t j = c->code_offsets[i], end = c->code_offsets[i + 1];
        while (j < end) {
            uint32_t code = column_code(c, j);
            if (c->codec == FPO_FSST8 && code == 255) {
                if (j + 1 >= end) { *err |= FPO_BIT_CORRUPT; j += 1; continue; }
                uint8_t lit = (uint8_t)column_code(c, j + 1);
                if (out && pos < cap) out[pos - base] = lit;
                pos += 1;
                j += 2;
                continue;
            }
            if (code >= c->n_entries) { *err |= FPO_BIT_CORRUPT; j += 1; continue; }
            for (uint32_t b = c->dict_offsets[code]; b < c->dict_offsets[code + 1]; ++b) {
                if (out && pos < cap) out[pos - base] = c->dict_bytes[b];
                pos += 1;
            }
            j += 1;
        }
        if (ends) ends[i - s0] = pos;
    }
    return pos - base;
}

static int check_column(const column_t* c, uint32_t n_strings, unsigned* err) {
    int w = code_bits(c->codec);
    if (!w) return FPO_ERR_ARG;
    uint32_t max_len = (c->codec == FPO_FSST8 || c->codec == FPO_FSST12) ? 8 : 16;
    uint32_t max_entries = c->codec == FPO_ONPAIR16 ? 65536u
                           : (c->codec == FPO_ONPAIR12 || c->codec == FPO_FSST12) ? 4096u : 255u;
    if (c->n_entries == 0 || c->n_entries > max_entries) return FPO_ERR_ARG;
    for (uint32_t e = 0; e < c->n_entries; ++e) {
        uint32_t L = c->dict_offsets[e + 1] - c->dict_offsets[e];
        if (c->dict_offsets[e + 1] < c->dict_offsets[e] || L < 1 || L > max_len) return FPO_ERR_ARG;
    }
    for (uint32_t i = 0; i < n_strings; ++i)
        if (c->code_offsets[i] > c->code_offsets[i + 1]) { *err |= FPO_BIT_CORRUPT; return FPO_ERR_CORRUPT; }
    if (c->code_offsets[n_strings] > c->n_slots) { *err |= FPO_BIT_CORRUPT; return FPO_ERR_CORRUPT; }
    return FPO_OK;
}

static int status_of(unsigned err) {
    if (err & FPO_BIT_CORRUPT) return FPO_ERR_CORRUPT;
    if (err & FPO_BIT_CAPACITY) return FPO_ERR_CAPACITY;
    if (err & FPO_BIT_OVERFLOW) return FPO_ERR_OVERFLOW;
    return FPO_OK;
}

/*
 * Decode a whole column.  out_offsets has n_strings + 1 entries.  Returns a
 * status (FPO_*); *err_bits receives the set of error kinds seen and
 * *total the decoded size (also when it exceeds the capacity).
 */
int fpo_decode(int codec, const uint8_t* dict_bytes, const uint32_t* dict_offsets, uint32_t n_entries,
               const uint8_t* stream, uint64_t stream_bytes, const uint32_t* code_offsets,
               uint32_t n_strings, uint8_t* out, uint64_t out_capacity, uint32_t* out_offsets,
               uint64_t* total, unsigned* err_bits) {
    column_t c = {codec, dict_bytes, dict_offsets, n_entries, stream,
                  code_bits(codec) ? stream_bytes * 8 / (uint64_t)code_bits(codec) : 0, code_offsets};
    unsigned err = 0;
    int st = check_column(&c, n_strings, &err);
    if (err_bits) *err_bits = err;
    if (st != FPO_OK) return st;
    uint64_t* ends = (uint64_t*)malloc(sizeof(uint64_t) * (n_strings ? n_strings : 1));
    if (!ends) return FPO_ERR_ARG;
    uint64_t D = decode_range(&c, 0, n_strings, out, 0, out ? out_capacity : 0, ends, &err);
    if (out_offsets) {
        out_offsets[0] = 0;
        for (uint32_t i = 0; i < n_strings; ++i) out_offsets[i + 1] = (uint32_t)ends[i];
    }
    free(ends);
    if (out && D > out_capacity) err |= FPO_BIT_CAPACITY;
    if (D > 0x7fffffffull) err |= FPO_BIT_OVERFLOW;
    if (total) *total = D;
    if (err_bits) *err_bits = err;
    return status_of(err);
}

/* ---- the same decode spread over threads, for the CPU baseline timing ---- */

typedef struct {
    const column_t* c;
    uint32_t s0, s1;
    uint8_t* out;
    uint64_t base, cap;
    uint64_t* ends;
    uint64_t size;
    unsigned err;
    int sizes_only;
} job_t;

static void* run_job(void* p) {
    job_t* j = (job_t*)p;
    if (j->sizes_only) {
        j->size = decode_range(j->c, j->s0, j->s1, NULL, 0, 0, NULL, &j->err);
    } else {
        decode_range(j->c, j->s0, j->s1, j->out + j->base, j->base, j->cap, j->ends, &j->err);
    }
    return NULL;
}

/*
 * Thread-parallel decode: each thread takes a contiguous string range; a
 * first pass sizes each range, a serial prefix places them, a second pass
 * decodes in place.  Same result as fpo_decode.
 */
int fpo_decode_mt(int codec, const uint8_t* dict_bytes, const uint32_t* dict_offsets, uint32_t n_entries,
                  const uint8_t* stream, uint64_t stream_bytes, const uint32_t* code_offsets,
                  uint32_t n_strings, uint8_t* out, uint64_t out_capacity, uint32_t* out_offsets,
                  uint64_t* total, unsigned* err_bits, int n_threads) {
    column_t c = {codec, dict_bytes, dict_offsets, n_entries, stream,
                  code_bits(codec) ? stream_bytes * 8 / (uint64_t)code_bits(codec) : 0, code_offsets};
    unsigned err = 0;
    int st = check_column(&c, n_strings, &err);
    if (err_bits) *err_bits = err;
    if (st != FPO_OK) return st;
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    job_t jobs[256];
    pthread_t th[256];
    uint64_t* ends = (uint64_t*)malloc(sizeof(uint64_t) * (n_strings ? n_strings : 1));
    if (!ends) return FPO_ERR_ARG;
    for (int t = 0; t < n_threads; ++t) {
        uint32_t s0 = (uint32_t)((uint64_t)n_strings * t / n_threads);
        uint32_t s1 = (uint32_t)((uint64_t)n_strings * (t + 1) / n_threads);
        job_t jb = {&c, s0, s1, out, 0, 0, ends + s0, 0, 0, 1};
        jobs[t] = jb;
    }
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, run_job, &jobs[t]);
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    uint64_t base = 0;
    for (int t = 0; t < n_threads; ++t) {
        jobs[t].base = base;
        base += jobs[t].size;
        err |= jobs[t].err;
        jobs[t].err = 0;
        jobs[t].sizes_only = 0;
        jobs[t].cap = out_capacity;
    }
    uint64_t D = base;
    if (out && D <= out_capacity) {
        for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, run_job, &jobs[t]);
        for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
        if (out_offsets) {
            out_offsets[0] = 0;
            for (uint32_t i = 0; i < n_strings; ++i) out_offsets[i + 1] = (uint32_t)ends[i];
        }
    } else if (out) {
        err |= FPO_BIT_CAPACITY;
    }
    free(ends);
    if (D > 0x7fffffffull) err |= FPO_BIT_OVERFLOW;
    if (total) *total = D;
    if (err_bits) *err_bits = err;
    return status_of(err);
}


/*
 * Stored sidecar of a column (paper Sec. 3.1: output positions recorded when
 * the column was compressed, read by the decoder instead of computed).  The
 * column's slots [c0, c1) (c0 = code_offsets[0], c1 = code_offsets[n]) are
 * cut into tiles of `tile` slots aligned to multiples of `tile`: tile u
 * starts at slot s_u = (c0 / tile + u) * tile, u = 0 .. T-1,
 * T = max(1, ceil(c1 / tile) - c0 / tile).
 *   entries[0]     = decoded size of the column;
 *   entries[1 + u] = bytes produced by the column's slots before
 *                    max(s_u, c0), with bit 63 set when slot s_u is the
 *                    literal byte of an FSST-8 escape.
 * The walk below is the decode's parse, slot by slot, recording the running
 * byte count whenever a slot starts a tile.  Returns T, or 0 when the
 * column is invalid or corrupt or entries has fewer than 1 + T elements.
 */
uint64_t fpo_sidecar(int codec, const uint8_t* dict_bytes, const uint32_t* dict_offsets, uint32_t n_entries,
                     const uint8_t* stream, uint64_t stream_bytes, const uint32_t* code_offsets,
                     uint32_t n_strings, uint32_t tile, uint64_t* entries, uint64_t max_entries) {
    column_t c = {codec, dict_bytes, dict_offsets, n_entries, stream, 0, code_offsets};
    int w = code_bits(codec);
    if (!w || tile == 0) return 0;
    c.n_slots = stream_bytes * 8 / (uint64_t)w;
    unsigned err = 0;
    if (check_column(&c, n_strings, &err) != FPO_OK) return 0;
    const uint64_t c0 = code_offsets[0], c1 = code_offsets[n_strings];
    const uint64_t first = c0 / tile, end = (c1 + tile - 1) / tile;
    const uint64_t T = end > first ? end - first : 1;
    if (1 + T > max_entries) return 0;
    for (uint64_t u = 0; u < T; ++u) entries[1 + u] = 0;
    uint64_t produced = 0;
    for (uint32_t i = 0; i < n_strings; ++i) {
        uint64_t j = code_offsets[i];
        const uint64_t e = code_offsets[i + 1];
        while (j < e) {
            if (j % tile == 0 && j > c0) entries[1 + (j / tile - first)] = produced;
            const uint32_t code = read_code(codec, stream, j);
            if (codec == FPO_FSST8 && code == 255) {
                if (j + 1 >= e) return 0;   /* escape without its literal */
                /* the literal slot: it may start a tile too, flagged as a literal */
                if ((j + 1) % tile == 0) entries[1 + ((j + 1) / tile - first)] = produced | (1ull << 63);
                produced += 1;
                j += 2;
                continue;
            }
            if (code >= n_entries) return 0;
            produced += dict_offsets[code + 1] - dict_offsets[code];
            j += 1;
        }
    }
    entries[0] = produced;
    return T;
}


/*
 * Selective decode: the strings row_ids[0..m-1] of a column (any order,
 * repeats allowed) decoded one after another into out, with
 * out_offsets[0] = 0 and out_offsets[k+1] = bytes after row_ids[k].  This is
 * random access to single strings, which FSST-family codecs allow because a
 * string's codes decode on their own (paper Sec. 1 and Sec. 2.1).  Each row
 * is decoded by the same walk as fpo_decode.  A row id >= n_strings is an
 * argument error.  Returns a status as fpo_decode.
 */
int fpo_decode_rows(int codec, const uint8_t* dict_bytes, const uint32_t* dict_offsets, uint32_t n_entries,
                    const uint8_t* stream, uint64_t stream_bytes, const uint32_t* code_offsets,
                    uint32_t n_strings, const uint32_t* row_ids, uint32_t m, uint8_t* out, uint64_t out_capacity,
                    uint32_t* out_offsets, uint64_t* total, unsigned* err_bits) {
    column_t c = {codec, dict_bytes, dict_offsets, n_entries, stream,
                  code_bits(codec) ? stream_bytes * 8 / (uint64_t)code_bits(codec) : 0, code_offsets};
    unsigned err = 0;
    int st = check_column(&c, n_strings, &err);
    if (err_bits) *err_bits = err;
    if (st != FPO_OK) return st;
    for (uint32_t k = 0; k < m; ++k)
        if (row_ids[k] >= n_strings) return FPO_ERR_ARG;
    uint64_t pos = 0;
    if (out_offsets) out_offsets[0] = 0;
    for (uint32_t k = 0; k < m; ++k) {
        const uint32_t r = row_ids[k];
        pos += decode_range(&c, r, r + 1, out ? out + pos : NULL, pos, out ? out_capacity : 0, NULL, &err);
        if (out_offsets) out_offsets[k + 1] = (uint32_t)pos;
    }
    if (out && pos > out_capacity) err |= FPO_BIT_CAPACITY;
    if (pos > 0x7fffffffull) err |= FPO_BIT_OVERFLOW;
    if (total) *total = pos;
    if (err_bits) *err_bits = err;
    return status_of(err);
}


/*
 * Decode a column whose codes are bit-packed at `bits` bits per code (the
 * cascade layer above; codecs without escapes: OnPair-16, OnPair-12 and
 * FSST-12, 1 <= bits <= the codec's own width).  Arguments and result as
 * fpo_decode.
 */
int fpo_decode_packed(int codec, int bits, const uint8_t* dict_bytes, const uint32_t* dict_offsets,
                      uint32_t n_entries, const uint8_t* stream, uint64_t stream_bytes,
                      const uint32_t* code_offsets, uint32_t n_strings, uint8_t* out, uint64_t out_capacity,
                      uint32_t* out_offsets, uint64_t* total, unsigned* err_bits) {
    if (codec == FPO_FSST8 || bits < 1 || bits > code_bits(codec)) return FPO_ERR_ARG;
    column_t c = {codec, dict_bytes, dict_offsets, n_entries, stream, stream_bytes * 8 / (uint64_t)bits,
                  code_offsets, bits};
    unsigned err = 0;
    int st = check_column(&c, n_strings, &err);
    if (err_bits) *err_bits = err;
    if (st != FPO_OK) return st;
    uint64_t* ends = (uint64_t*)malloc(sizeof(uint64_t) * (n_strings ? n_strings : 1));
    if (!ends) return FPO_ERR_ARG;
    uint64_t D = decode_range(&c, 0, n_strings, out, 0, out ? out_capacity : 0, ends, &err);
    if (out_offsets) {
        out_offsets[0] = 0;
        for (uint32_t i = 0; i < n_strings; ++i) out_offsets[i + 1] = (uint32_t)ends[i];
    }
    free(ends);
    if (out && D > out_capacity) err |= FPO_BIT_CAPACITY;
    if (D > 0x7fffffffull) err |= FPO_BIT_OVERFLOW;
    if (total) *total = D;
    if (err_bits) *err_bits = err;
    return status_of(err);
}
