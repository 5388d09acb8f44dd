/*
 * fastpair.h -- C ABI of the GB300 decoder for dictionary-compressed string
 * columns (FSST-family codecs, FastPair, arXiv 2609.15034).
 *
 * The problem (paper Sec. 1, Sec. 2.1): a column of strings is stored as a
 * stream of fixed-width codes; each code indexes a token of a trained
 * dictionary, and a string decodes to the concatenation of its codes'
 * tokens, with no padding between tokens.  The output (paper Sec. 5) is a
 * variable-length string array: byte-packed string data plus an array of
 * fixed-width offsets.
 *
 * Codecs (paper Sec. 2.1):
 *   FP_ONPAIR16  16-bit codes, up to 65,536 tokens of 1..16 bytes.
 *   FP_ONPAIR12  12-bit codes, up to 4,096 tokens of 1..16 bytes.
 *   FP_FSST8     8-bit codes, up to 255 tokens of 1..8 bytes; code 255 is the
 *                escape: the slot after it holds one literal byte.
 *   FP_FSST12    12-bit codes, up to 4,096 tokens of 1..8 bytes, no escape
 *                (the escape-free variant the paper decodes).
 *
 * Stored layouts:
 *   - OnPair-16: little-endian uint16 per code.
 *   - OnPair-12 and FSST-12: LSB-first bitstream; code i occupies stream
 *     bits [12 i, 12 i + 12), stream bit b is bit (b mod 8) of byte b / 8.
 *   - FSST-8: one byte per slot (codes and the literal bytes after escapes).
 *   A "slot" is one code position (for FSST-8 a literal byte is a slot too).
 *
 * Conventions for every call:
 *   - Pointers named d_* are device pointers owned by the caller; the library
 *     never frees them.  Pointers named h_* are host pointers.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     are stream-ordered and asynchronous unless stated otherwise.
 *   - Host-detectable argument errors return at once and launch nothing.
 *     Errors found in the data on the device (see fp_sync_status) are
 *     recorded in a sticky per-stream status word and never trap; on a data
 *     error the output contents are unspecified, but every write stays
 *     inside [d_out_bytes, d_out_bytes + out_capacity) and d_out_offsets.
 *   - fp_last_error() returns a thread-local text for the last failure.
 *
 * This header declares only what libfastpair.so exports.
 */
#ifndef FASTPAIR_H
#define FASTPAIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* fp_stream_t; /* same type as cudaStream_t */

typedef enum fp_codec {
    FP_ONPAIR16 = 1,
    FP_ONPAIR12 = 2,
    FP_FSST8 = 3,
    FP_FSST12 = 4
} fp_codec;

typedef enum fp_status {
    FP_OK = 0,
    FP_ERR_ARG = 1,       /* invalid argument (host-detected)                */
    FP_ERR_CUDA = 2,      /* a CUDA runtime call failed                      */
    FP_ERR_NOMEM = 3,     /* device or host allocation failed                */
    FP_ERR_CORRUPT = 4,   /* code >= n_entries, escape in a string's last     */
                          /* slot, code_offsets not monotone or past the      */
                          /* end of the code buffer                           */
    FP_ERR_CAPACITY = 5,  /* decoded size exceeds out_capacity                */
    FP_ERR_OVERFLOW = 6,  /* decoded size exceeds 2^31 - 1 (int32 offsets)    */
    FP_ERR_TIMEOUT = 7,   /* a bounded device-side wait gave up               */
    FP_ERR_BUSY = 8,      /* resource busy / budget exhausted                 */
    FP_ERR_NOT_READY = 9, /* result not available yet                         */
    FP_ERR_INTERNAL = 10  /* a decoder self-check failed: a warp tile's byte  */
                          /* total, recomputed by the decode, disagrees with  */
                          /* the offsets its length pass scanned (the output  */
                          /* is then wrong; writes stay in bounds)            */
} fp_status;

/* Opaque, library-owned, device-resident dictionary. */
typedef struct fp_dict fp_dict;

/*
 * fp_dict_upload -- validate a dictionary and make it device-resident.
 *
 * Paper Sec. 1 and Sec. 3.2: the decoder reads fixed-size dictionary
 * entries addressed directly by the code, plus a separate table of token
 * lengths.  This call repacks the interchange form (token i is
 * h_bytes[h_offsets[i] .. h_offsets[i+1])) into that device layout.
 *
 *   codec       one of fp_codec.
 *   h_bytes     host, concatenated token bytes (may be NULL only if every
 *               token is empty, which is itself invalid).
 *   h_offsets   host, n_entries + 1 non-decreasing uint32 offsets.
 *   n_entries   1..65,536 (OnPair-16), 1..4,096 (OnPair-12, FSST-12),
 *               1..255 (FSST-8).
 *   stream      stream for the uploads; the call synchronises it before it
 *               returns (the host buffers may be reused at once).
 *   out         receives the dictionary handle.
 *
 * OnPair dictionaries are also stored as two planes (bytes 0-7 and 8-15 of
 * every entry, paper Sec. 3.2) and carry a read width W: 8 = split read
 * (the low plane for every token, the high plane only for tokens longer
 * than 8 bytes), 16 = whole entries.  The upload sets W = 16, the faster
 * width on GB300 for every share of long tokens measured; the paper's rule
 * (Sec. 4.3: W = 8 unless more than 60 % of the tokens exceed 8 bytes) is
 * fp_width_for_histogram, and fp_dict_set_width applies either choice.
 *
 * Errors: FP_ERR_ARG if a token length is outside 1..16 (OnPair) or 1..8
 * (FSST-8, FSST-12), n_entries is out of range or a pointer is NULL;
 * FP_ERR_NOMEM; FP_ERR_CUDA.  Duplicate tokens are allowed.
 */
fp_status fp_dict_upload(fp_codec codec, const uint8_t* h_bytes, const uint32_t* h_offsets,
                         uint32_t n_entries, fp_stream_t stream, fp_dict** out);

/* Release a dictionary (synchronises the device first).  NULL is a no-op. */
fp_status fp_dict_free(fp_dict* dict);

/*
 * fp_width_for_histogram -- the paper's split-read rule (Sec. 4.3): 16 when
 * more than 60 % of the counted tokens are longer than 8 bytes, else 8.
 * hist[L] is the number of tokens of L bytes (L = 0..16) -- typically a
 * column's token occurrences, which the encoder holds.  An all-zero
 * histogram gives 8.
 */
int fp_width_for_histogram(const uint64_t* hist17);

/*
 * fp_dict_set_width / fp_dict_width -- the dictionary read width fp_decode
 * uses for this dictionary when no variant is selected: 8 (split read) or
 * 16 (whole entries).  FSST codecs have 8-byte entries and accept only 8.
 * FP_ERR_ARG for other values.  Not synchronised with decodes in flight
 * (set it before enqueueing the decodes that should use it).
 */
fp_status fp_dict_set_width(fp_dict* dict, int width);
int fp_dict_width(const fp_dict* dict);

/*
 * fp_decode -- decode one column into Arrow-style bytes plus offsets.
 *
 * Paper Sec. 2.1 and Sec. 3 (Algorithm 1): for every string i, the output
 * bytes d_out_bytes[d_out_offsets[i] .. d_out_offsets[i+1]) are the
 * concatenation of the tokens of the codes in slots
 * [d_code_offsets[i], d_code_offsets[i+1]); for FSST-8 an escape (255)
 * contributes the literal byte in the slot after it.  Output positions come
 * from a prefix sum of token lengths computed on the device in the same
 * launch (the paper stores them as a precomputed sidecar, Sec. 3.1).
 *
 *   codec           must equal the dictionary's codec.
 *   dict            from fp_dict_upload, on the current device.
 *   d_codes         device, stored code buffer, 16-byte aligned.
 *   codes_bytes     size of the code buffer in bytes; only whole slots in it
 *                   are read.
 *   d_code_offsets  device, n_strings + 1 uint32 slot indices, non-decreasing;
 *                   d_code_offsets[0] may be non-zero (a slice of a larger
 *                   stream).  Slots before it and after d_code_offsets[n]
 *                   are never decoded.
 *   n_strings       number of strings (0 allowed).
 *   d_out_bytes     device, 16-byte aligned, out_capacity bytes.
 *   out_capacity    bytes available at d_out_bytes.
 *   d_out_offsets   device, n_strings + 1 uint32; d_out_offsets[0] = 0.
 *   stream          launch stream.
 *
 * Returns FP_OK once the launch is enqueued, or a host-detected error
 * (FP_ERR_ARG, FP_ERR_NOMEM, FP_ERR_CUDA).  Data errors are reported by
 * fp_sync_status.  Calls on one stream share a library-owned workspace and
 * must not overlap; calls on different streams may run concurrently.
 * The first call on a stream allocates its workspace (call it once before
 * capturing the stream into a CUDA graph).
 */
fp_status fp_decode(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                    const uint32_t* d_code_offsets, uint32_t n_strings, uint8_t* d_out_bytes,
                    uint64_t out_capacity, uint32_t* d_out_offsets, fp_stream_t stream);

/*
 * fp_decoded_size -- decoded size of a column, synchronously.
 *
 * Same inputs and meaning as fp_decode; runs the length pass only and
 * synchronises `stream`.  *h_total receives the decoded size in bytes.
 * Returns the column's data status (FP_ERR_CORRUPT, FP_ERR_OVERFLOW, ...)
 * as fp_sync_status would.
 */
fp_status fp_decoded_size(fp_codec codec, const fp_dict* dict, const void* d_codes,
                          uint64_t codes_bytes, const uint32_t* d_code_offsets, uint32_t n_strings,
                          fp_stream_t stream, uint64_t* h_total);

/*
 * Selective decode (paper Sec. 1 and Sec. 2.1: strings of FSST-family
 * columns decode independently, which allows random access): the strings
 * d_row_ids[0 .. n_rows) of a column, in that order, into Arrow-style
 * output -- d_out_bytes[d_out_offsets[k] .. d_out_offsets[k+1]) is string
 * d_row_ids[k].  Row ids may repeat and need not be sorted.
 *
 * The calls gather the selected rows' codes into one contiguous stream in
 * the stream's workspace (a row-length pass, a scan of the row lengths and
 * a compaction) and decode that stream with fp_decode's kernels.
 *
 * fp_rows_size -- synchronous: *h_slots receives the number of code slots
 *   the selected rows hold (the `selected_slots` fp_decode_rows needs) and
 *   *h_bytes their decoded size.  Returns the data status as
 *   fp_sync_status would.
 *
 * fp_decode_rows -- asynchronous.  selected_slots >= the rows' code slots
 *   (fp_rows_size); it sizes the workspace.  Inputs as fp_decode, plus
 *   d_row_ids (device, n_rows uint32, 4-byte aligned); d_out_offsets has
 *   n_rows + 1 entries.
 *
 * Data errors (fp_sync_status): a row id >= n_strings, a selected row
 * whose code_offsets decrease or pass the code buffer, and the errors of
 * fp_decode in a selected row -> FP_ERR_CORRUPT; more selected slots than
 * selected_slots -> FP_ERR_CAPACITY (or FP_ERR_CORRUPT); the output and
 * overflow checks as fp_decode.  Rows that are not selected are not read.
 */
fp_status fp_rows_size(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                       const uint32_t* d_code_offsets, uint32_t n_strings, const uint32_t* d_row_ids,
                       uint32_t n_rows, fp_stream_t stream, uint64_t* h_slots, uint64_t* h_bytes);
fp_status fp_decode_rows(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                         const uint32_t* d_code_offsets, uint32_t n_strings, const uint32_t* d_row_ids,
                         uint32_t n_rows, uint64_t selected_slots, uint8_t* d_out_bytes, uint64_t out_capacity,
                         uint32_t* d_out_offsets, fp_stream_t stream);

/*
 * Cascaded codes (paper Sec. 2.1 and Sec. 5: FSST-family codes are integers
 * that lightweight numeric encodings compress further, and the paper widens
 * the stored, bit-packed codes on the host before it decodes).  These calls
 * decode a column whose codes are bit-packed at code_bits bits per code
 * (LSB-first: code i occupies stream bits [code_bits i, code_bits i +
 * code_bits), stream bit k is bit (k mod 8) of byte k / 8), unpacking them
 * inside the decode's own kernels -- no widened copy is made.  Typically
 * code_bits = ceil(log2(n_entries)) of the dictionary.
 *
 *   codec       FP_ONPAIR16, FP_ONPAIR12 or FP_FSST12 (escape-free codecs).
 *   code_bits   1 .. the codec's own width (16, 12, 12); at the codec's own
 *               width the layout is the codec's stored layout.
 *   d_codes     16-byte aligned; slots are the whole codes in codes_bytes.
 * Everything else (arguments, output, errors, workspace) as fp_decode /
 * fp_decoded_size; FP_ERR_ARG for another codec or width.
 */
fp_status fp_decode_packed(fp_codec codec, const fp_dict* dict, uint32_t code_bits, const void* d_codes,
                           uint64_t codes_bytes, const uint32_t* d_code_offsets, uint32_t n_strings,
                           uint8_t* d_out_bytes, uint64_t out_capacity, uint32_t* d_out_offsets, fp_stream_t stream);
fp_status fp_decoded_size_packed(fp_codec codec, const fp_dict* dict, uint32_t code_bits, const void* d_codes,
                                 uint64_t codes_bytes, const uint32_t* d_code_offsets, uint32_t n_strings,
                                 fp_stream_t stream, uint64_t* h_total);

/*
 * fp_decode_plain -- baseline decoder with one thread per string.
 *
 * Same arguments, result and error behaviour as fp_decode.  Each thread
 * walks its string's codes serially and copies token bytes one at a time
 * from the dictionary in its interchange layout (offset table, then bytes),
 * after a separate per-string length pass and prefix sum.  It exists to be
 * timed beside fp_decode.
 */
fp_status fp_decode_plain(fp_codec codec, const fp_dict* dict, const void* d_codes,
                          uint64_t codes_bytes, const uint32_t* d_code_offsets, uint32_t n_strings,
                          uint8_t* d_out_bytes, uint64_t out_capacity, uint32_t* d_out_offsets,
                          fp_stream_t stream);

/*
 * fp_sync_status -- synchronise `stream`, then read and clear its sticky
 * data-error status.  Returns FP_OK or, by priority, FP_ERR_TIMEOUT,
 * FP_ERR_INTERNAL, FP_ERR_CORRUPT, FP_ERR_CAPACITY, FP_ERR_OVERFLOW;
 * FP_ERR_CUDA if the synchronisation itself failed.
 */
fp_status fp_sync_status(fp_stream_t stream);

/* Thread-local description of the last error returned on this thread. */
const char* fp_last_error(void);

/*
 * fp_debug_stall_next -- failure-detection test hook (no counterpart in the
 * paper): make the next fp_decode on `stream` give up a bounded wait on
 * purpose, without any fault.  That call skips the first ticket of its
 * ticketed pass (the tile scan of the warp-tile decoder, or the decode of
 * the block pipeline), so the first look-back word is never published and
 * the look-back that needs it polls it `spin_limit` times (1..2^20; the
 * built-in limit is 2^20 polls with back-off), then gives up; the
 * one-launch decode's first grid barrier starts with an arrival count no
 * grid reaches, so its blocks give up there in the same way.  The call
 * reports FP_ERR_TIMEOUT through fp_sync_status; its output is unspecified
 * but every write stays in bounds.  Both settings end with that call: the
 * next decode on the stream is normal.
 *
 * The stream must already have a workspace (one earlier fp_decode on it);
 * FP_ERR_ARG otherwise.  Stream-ordered, asynchronous.
 */
fp_status fp_debug_stall_next(fp_stream_t stream, uint32_t spin_limit);

/*
 * fp_decode_noalloc -- fp_decode for callers that cannot allocate.
 *
 * This entry point has no counterpart in the paper.  It exists for callers
 * that cannot call cudaMalloc -- an allocator hook, or an engine that owns
 * every byte of device memory and forbids allocations behind its back --
 * since fp_decode allocates its per-stream workspace on first use.  Its
 * scratch is a
 * fixed 1 MiB array compiled into the library; every GPU that loads the
 * library keeps that array until the process exits.  The call allocates
 * nothing (no cudaMalloc, cudaFree or allocating library routine).
 *
 * Arguments, layout and result are those of fp_decode, plus:
 *   d_status   device, one uint32 written (stream-ordered) with the call's
 *              data-error bits: 0 = OK; 1 = corrupt input, 2 = decoded size
 *              above out_capacity, 4 = above 2^31-1, 8 = a bounded device
 *              wait gave up, 16 = a decoder self-check failed (see
 *              FP_ERR_INTERNAL).  fp_sync_status does not report these calls.
 *
 * Limits and sharing:
 *   - unless a variant is selected (fp_variant_select), this call uses the
 *     block pipeline, whose scratch covers a code buffer of up to about
 *     357M slots (OnPair codecs; 715M for FSST-8); a selected warp-tile
 *     variant covers about 26.8M slots with 16 slots per lane (512-slot
 *     tiles) and about 53.7M with 32 slots per lane (FSST-8's 1,024-slot
 *     tiles).  Larger inputs return FP_ERR_ARG with the limit in
 *     fp_last_error() -- use fp_decode for them.
 *   - the first call on a device looks up and clears the array
 *     (synchronously); make that first call before any stream capture.
 *   - every call, on any stream, shares the one array per device: calls
 *     that overlap on the GPU race and corrupt each other's results.
 *     Serialise them (one stream, or events).
 */
fp_status fp_decode_noalloc(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                            const uint32_t* d_code_offsets, uint32_t n_strings, uint8_t* d_out_bytes,
                            uint64_t out_capacity, uint32_t* d_out_offsets, uint32_t* d_status,
                            fp_stream_t stream);

/*
 * ---------------------------------------------------------------------------
 * Batched decode (no counterpart API in the paper, which decodes one column
 * per launch): many chunks -- each a column as fp_decode takes it, with its
 * own codec and dictionary -- decoded by one persistent kernel launch that
 * takes (chunk, tile) work items from device-side queues, replayed from a
 * CUDA graph.  Each chunk's result is exactly fp_decode's.
 * ---------------------------------------------------------------------------
 */
typedef struct fp_chunk {
    fp_codec codec;
    const fp_dict* dict;
    const void* d_codes;              /* as fp_decode (16-byte aligned)            */
    uint64_t codes_bytes;
    const uint32_t* d_code_offsets;   /* n_strings + 1 slot indices                */
    uint32_t n_strings;
    uint8_t* d_out_bytes;             /* 16-byte aligned                           */
    uint64_t out_capacity;
    uint32_t* d_out_offsets;          /* n_strings + 1                             */
} fp_chunk;

typedef struct fp_plan fp_plan;   /* opaque, library-owned */

/*
 * fp_plan_create -- validate the chunks, pick a tile configuration and
 * capture the batch into a CUDA graph.  Synchronous.
 *
 *   chunks           host array of n_chunks descriptors (copied; the device
 *                    buffers they name must stay valid while the plan is used,
 *                    and the dictionaries must outlive the plan).
 *   n_chunks         >= 1.
 *   tune_cache_path  NULL, or a text file: if it holds a configuration for
 *                    this plan's signature (SM count and the multiset of
 *                    (codec, half-octave of code slots)), it is used;
 *                    otherwise every configuration is timed on the plan's
 *                    own chunks and the fastest is appended to the file.
 *                    Tuning runs decode the chunks, writing their outputs.
 *   stream           stream of the tuning runs.
 *
 * The chunks' code buffers are tiled whole, so pass code buffers that start
 * close to each chunk's first slot.  Errors: FP_ERR_ARG (a chunk fails the
 * checks of fp_decode, n_chunks == 0), FP_ERR_NOMEM, FP_ERR_CUDA.
 */
fp_status fp_plan_create(const fp_chunk* chunks, uint32_t n_chunks, const char* tune_cache_path,
                         fp_stream_t stream, fp_plan** out);

/* fp_plan_create with configuration `config` (0 .. fp_batch_config_count()-1), no tuning. */
fp_status fp_plan_create_config(const fp_chunk* chunks, uint32_t n_chunks, int config, fp_stream_t stream,
                                fp_plan** out);

/*
 * fp_decode_batch -- decode every chunk of the plan (one graph launch on
 * `stream`).  Asynchronous.  Launches of one plan must not overlap (they
 * share its device state); use one stream or events.  Data errors are
 * recorded per chunk; read them with fp_plan_sync_status.
 */
fp_status fp_decode_batch(fp_plan* plan, fp_stream_t stream);

/*
 * fp_plan_sync_status -- synchronise `stream`, then read and clear the
 * plan's per-chunk data status.  h_chunk_status (optional, n_chunks
 * entries) receives each chunk's fp_status; h_chunk_total (optional)
 * each chunk's decoded size from its last decode.  Returns the most severe
 * status over all chunks (priority as fp_sync_status).
 */
fp_status fp_plan_sync_status(fp_plan* plan, fp_stream_t stream, uint32_t* h_chunk_status,
                              uint64_t* h_chunk_total);

typedef struct fp_plan_info_t {
    uint32_t config;               /* chosen configuration                      */
    uint32_t n_configs;            /* configurations compiled in                */
    uint32_t slots_per_thread[3];  /* OnPair-16, OnPair-12, FSST-8              */
    uint32_t threads;              /* threads per block                         */
    uint32_t grid;                 /* blocks of the persistent launch           */
    uint32_t index_blocks;         /* blocks of the index pass                  */
    uint32_t from_cache;           /* 1 if the configuration came from the file */
    uint32_t slots_per_thread_fsst12;  /* FSST-12 (0: the configuration has no FSST-12 queue) */
    uint64_t total_tiles;
    uint64_t layout_bytes;         /* device bytes of the plan's tables         */
    float tune_ms[8];              /* tuning time per configuration, -1 = untimed */
} fp_plan_info_t;

fp_status fp_plan_info(const fp_plan* plan, fp_plan_info_t* info);

/* Release a plan (synchronises the device first).  NULL is a no-op. */
fp_status fp_plan_destroy(fp_plan* plan);

/* Batch configurations: slots per thread per codec (OnPair-16, OnPair-12,
 * FSST-8), blocks per SM, and 1 for the warp-tile decoder (index pass,
 * reduce, tile scan and a persistent decode: four launches) or 0 for the
 * block pipeline (index pass and the persistent decode).  Out pointers may be
 * NULL.  FSST-12 chunks are decoded only by the warp-tile configurations
 * (with the OnPair-12 slots per thread); fp_plan_create skips the others for
 * plans that hold FSST-12 chunks and fp_plan_create_config rejects them with
 * FP_ERR_ARG. */
int fp_batch_config_count(void);
fp_status fp_batch_config_info(int config, uint32_t* slots_per_thread3, uint32_t* blocks_per_sm,
                               uint32_t* warp_tiles);

/*
 * ---------------------------------------------------------------------------
 * Served decode (no counterpart API in the paper): a request loop with
 * continuous batching.  Requests (a column already on the device plus the
 * key of a registered dictionary) are submitted from any thread; a
 * scheduler thread inside the library admits them in arrival order while
 * the bytes in flight stay within an HBM budget, keeps dictionaries in a
 * device cache, and decodes the admitted requests in waves -- one
 * persistent batched launch each -- on several streams at once, so requests
 * arriving while others run start as soon as a stream and memory free up.
 * Outputs live in a device arena owned by the server until released.
 * ---------------------------------------------------------------------------
 */
typedef struct fp_server fp_server;   /* opaque */

typedef struct fp_serve_config {
    uint64_t hbm_budget;        /* bytes: outputs (until released) + inputs (until decoded) in flight;
                                   the output arena of this size is allocated at creation */
    uint32_t dict_cache_slots;  /* device-resident dictionaries (0 = 512); 1.06 MiB each */
    uint32_t max_inflight;      /* admitted requests not yet decoded (0 = 4096) */
    uint32_t n_streams;         /* waves in flight at once (0 = 4) */
    uint32_t max_wave;          /* requests per wave (0 = 256) */
    int32_t batch_config;       /* batch configuration of the waves (fp_batch_config_info); negative:
                                   the library's default */
    uint32_t reserved;
} fp_serve_config;

typedef struct fp_request {
    uint64_t dict_key;                /* a key registered with fp_serve_dict_put        */
    const void* d_codes;              /* device, 16-byte aligned, as fp_decode           */
    uint64_t codes_bytes;
    const uint32_t* d_code_offsets;   /* device, n_strings + 1                           */
    uint32_t n_strings;
    uint32_t reserved;
    uint64_t decoded_size;            /* exact decoded bytes (column metadata); a smaller
                                         value fails the request with FP_ERR_CAPACITY     */
    uint64_t user_tag;                /* returned with the result                        */
} fp_request;

typedef struct fp_result {
    uint64_t ticket;
    uint32_t status;                  /* fp_status of the request                        */
    uint32_t reserved;
    uint8_t* d_out_bytes;             /* device, valid until fp_serve_release            */
    uint32_t* d_out_offsets;          /* device, n_strings + 1                           */
    uint64_t bytes;                   /* decoded bytes                                   */
    uint64_t n_strings;
    int64_t t_submit_ns, t_admit_ns, t_done_ns;   /* host steady clock                   */
    uint64_t user_tag;
} fp_result;

typedef struct fp_serve_stats_t {
    uint64_t submitted, admitted, completed, failed, released;
    uint64_t waves;
    uint32_t max_wave_seen;
    uint32_t queued;                  /* submitted, not yet admitted                     */
    uint64_t bytes_decoded;
    uint64_t dict_hits, dict_misses, dict_evictions, dicts_registered;
    uint64_t inflight_bytes, peak_inflight_bytes;
    uint32_t inflight_requests;
    uint32_t reserved;
} fp_serve_stats_t;

/* Create a server on the current device (allocates the output arena and the
 * dictionary slots, starts the scheduler thread). */
fp_status fp_serve_create(const fp_serve_config* config, fp_server** out);

/* Register a dictionary under `key` (validated and repacked on the host at
 * once; uploaded into a device slot when a request needs it).  Keys are
 * unique: FP_ERR_ARG if `key` exists. */
fp_status fp_serve_dict_put(fp_server* server, uint64_t key, fp_codec codec, const uint8_t* h_bytes,
                            const uint32_t* h_offsets, uint32_t n_entries);

/* Queue a request.  Returns at once with a ticket.  The input buffers must
 * stay valid and unchanged until the request completes.  FP_ERR_BUSY if the
 * request alone exceeds the HBM budget or the server is shutting down. */
fp_status fp_serve_submit(fp_server* server, const fp_request* request, uint64_t* ticket);

/* Take up to `max` completed requests (waiting up to timeout_ns for the
 * first one).  Each result's outputs stay valid until fp_serve_release. */
fp_status fp_serve_poll(fp_server* server, fp_result* out, uint32_t max, uint32_t* n, int64_t timeout_ns);

/* Return a polled request's output memory to the server.
 * FP_ERR_NOT_READY if the request has not completed or not been polled. */
fp_status fp_serve_release(fp_server* server, uint64_t ticket);

fp_status fp_serve_stats(fp_server* server, fp_serve_stats_t* out);

/* Stop admitting, finish the waves on the GPU, free everything (requests
 * still queued are dropped). */
fp_status fp_serve_destroy(fp_server* server);

/*
 * Decode variants (tile shapes).  A variant fixes the threads per block, the
 * code slots each thread decodes and where the dictionary is read from
 * (shared memory staged once per block, or the L1/L2 cache path).
 *
 * fp_variant_count  number of compiled variants for a codec.
 * fp_variant_info   describe variant v: threads per block, slots per thread,
 *                   1 if the dictionary is staged in shared memory, and the
 *                   kernel launches of one fp_decode call (2: index pass and
 *                   block-pipeline decode; 3: index pass and reduce in one
 *                   launch, tile scan, warp-tile decode; 1: the warp-tile
 *                   passes as phases of one cooperative launch, for small
 *                   columns).  Any out pointer may be NULL.
 * fp_variant_select make variant v the one fp_decode uses for the codec in
 *                   this process (v = -1 restores the defaults: tuned ones
 *                   (fp_tune_*), else built-in ones, which depend on the
 *                   size of the code buffer and on the dictionary's read
 *                   width).
 * fp_variant_selected  the variant selected for the codec, or with none
 *                   selected the default for large code buffers.
 * fp_variant_for    the variant fp_decode uses for a code buffer of
 *                   codes_bytes bytes (-1 for an unknown codec).
 */
int fp_variant_count(fp_codec codec);
fp_status fp_variant_info(fp_codec codec, int v, uint32_t* threads, uint32_t* slots_per_thread,
                          uint32_t* dict_in_smem, uint32_t* launches_per_call);
fp_status fp_variant_select(fp_codec codec, int v);
int fp_variant_selected(fp_codec codec);
int fp_variant_for(fp_codec codec, uint64_t codes_bytes);

/*
 * Autotuning of the single-column decode (no counterpart API in the paper,
 * whose shapes are chosen per column by hand, Sec. 4.1-4.4).
 *
 * fp_tune_column -- time every compiled variant of the codec whose read
 *   width equals the dictionary's (one warm-up, best of three decodes of
 *   the caller's column; inputs and outputs as fp_decode, which the runs
 *   write) and make the fastest the default for this device, codec, width
 *   and size class (floor(log2) of the code buffer's slots).  table_path:
 *   NULL, or a text file the choice is appended to ("sms codec width class
 *   variant ms").  *chosen / *best_ms (may be NULL) receive the variant and
 *   its time.  Synchronous.  Returns the column's data status.
 * fp_tune_load -- read such a file: its lines for this library's variants
 *   become defaults (entries for another SM count stay unused).
 * fp_tune_clear -- forget the tuned defaults (the built-in ones apply).
 * A variant selected with fp_variant_select overrides tuned defaults.
 */
fp_status fp_tune_column(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                         const uint32_t* d_code_offsets, uint32_t n_strings, uint8_t* d_out_bytes,
                         uint64_t out_capacity, uint32_t* d_out_offsets, const char* table_path, fp_stream_t stream,
                         int* chosen, float* best_ms);
fp_status fp_tune_load(const char* table_path);
fp_status fp_tune_clear(void);

/* The variant fp_decode uses with this dictionary (its codec and read
 * width) for a code buffer of codes_bytes bytes; -1 for NULL.  fp_variant_for
 * answers for read width 8. */
int fp_variant_for_dict(const fp_dict* dict, uint64_t codes_bytes);

/* Dictionary read width of variant v (16: whole entries, 8: split read);
 * 0 for an unknown codec or variant. */
int fp_variant_width(fp_codec codec, int v);

#ifdef __cplusplus
}
#endif
#endif /* FASTPAIR_H */
