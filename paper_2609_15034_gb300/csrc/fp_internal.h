// Internal declarations shared by the library's host and device sources.
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "fastpair.h"

struct fp_dict;

namespace fp {

// Sticky data-error bits in the per-stream status word.
constexpr uint32_t ERRB_CORRUPT = 1u;
constexpr uint32_t ERRB_CAPACITY = 2u;
constexpr uint32_t ERRB_OVERFLOW = 4u;
constexpr uint32_t ERRB_TIMEOUT = 8u;
// A warp tile's byte total, recomputed by the decode, differs from the
// offsets the tile scan (or a stored sidecar) gave its neighbour.
constexpr uint32_t ERRB_MISMATCH = 16u;

// Device workspace header (one per stream).  It is followed by the tile
// status words of the single-pass prefix scan (one u64 per tile, at
// `kWsHeaderBytes`) and by the tile -> first string index (tiles + 1 u32).
struct WsHeader {
    unsigned int tile_counter;   // next tile ticket
    unsigned int exit_counter;   // blocks that have finished
    unsigned int epoch;          // launch generation tag of tile status words
    unsigned int status;         // sticky ERRB_* bits
    unsigned long long rows_slots;   // selective decode: code slots of the selected rows
    unsigned long long total;    // decoded size of the last launch
    unsigned int abort;          // set when a bounded wait gave up
    unsigned int queue_counter[3];   // batched decode: next tile ticket of each codec queue
    unsigned int spin_limit;     // polls before a look-back gives up (0 = the built-in limit); reset per launch
    unsigned int bar_count;      // one-launch decode: blocks arrived at the current grid barrier
    unsigned int bar_gen;        // one-launch decode: grid barriers passed
    unsigned int pad[17];
};
constexpr size_t kWsHeaderBytes = 128;
static_assert(sizeof(WsHeader) == kWsHeaderBytes, "workspace header size");

constexpr unsigned kEpochBits = 26;
constexpr unsigned kEpochMask = (1u << kEpochBits) - 1u;

// Device view of a dictionary (passed by value to kernels).
struct DictView {
    const void* table;        // 2^w entries, 16 B (OnPair) or 8 B (FSST-8, FSST-12) each, zero padded
    const uint8_t* lens;      // 2^w token lengths; 0 = no token (or the FSST-8 escape)
    const void* planes;       // OnPair only: low plane (bytes 0-7 of each entry, 8 B stride),
                              // then high plane (bytes 8-15), 2^w entries each; else null
    const uint8_t* bytes;     // interchange layout: concatenated token bytes
    const uint32_t* offsets;  // interchange layout: n_entries + 1 offsets (rebased to 0)
    uint32_t n_entries;
};

struct DecodeParams {
    DictView dict;
    const uint8_t* codes;
    uint64_t codes_bytes;
    uint64_t max_slots;           // whole slots in the code buffer
    const uint32_t* code_offsets;
    uint32_t n_strings;
    uint8_t* out;
    uint64_t capacity;
    uint32_t* out_offsets;
    WsHeader* ws;                     // launch-wide counters, launch tag, abort flag
    unsigned long long* tile_status;  // look-back words of this column's tiles (tile 0 first)
    int size_only;
    unsigned int* err_word;           // where this column's data-error bits go
    unsigned long long* total_out;    // where this column's decoded size goes
    const uint32_t* first;            // tile -> first string boundary it owns (index pass)
    uint32_t packed_bits;             // cascaded codes: bits per code (packed decode only; else 0)
    uint32_t pad_;
};

// Tiles of a column: a tile is `tile` consecutive code slots, tile u covers
// slots [(first_tile + u) * tile, ...); the column's slots are [c_begin, c_end).
struct Extent {
    unsigned long long c_begin, c_end, first_tile, n_tiles;
    unsigned int bad;   // code_offsets[0] / [n] inconsistent with the code buffer
    unsigned int pad;
};

// Batched decode: one record per chunk, copied into a decode block's shared
// memory for every tile it takes.  The host fills `p` and `x.first_tile` /
// `x.n_tiles` (the chunk's code buffer is tiled whole); the index pass fills
// x.c_begin, x.c_end and x.bad.
struct alignas(16) SlotSrc {
    DecodeParams p;
    Extent x;
    uint32_t tile_base;   // queue ticket of the chunk's first tile
    uint32_t chunk;       // index of the chunk in the plan
    // warp-tile batches only
    unsigned long long wt_base;   // index of the chunk's first warp tile in the batch's element arrays
    uint32_t sb_base;             // the chunk's first tile-scan block (its look-back words start there)
    uint32_t n_sb;                // the chunk's tile-scan blocks
};
static_assert(sizeof(SlotSrc) % 16 == 0, "chunk records are copied in 16-byte pieces");

// One codec's work queue: tickets 0..n_tiles-1 over its chunks' tiles.
struct BatchQueue {
    const SlotSrc* src;          // chunk records of this codec
    const uint32_t* tile_chunk;  // ticket -> index into src
    uint32_t n_tiles;
    uint32_t n_chunks;
};

// Codec queues of a batch: OnPair-16, OnPair-12, FSST-8, FSST-12 (queue =
// codec - 1).  The block pipeline serves the first three; FSST-12 chunks
// need a warp-tile configuration.
constexpr int kQueues = 4;
constexpr int kBlockQueues = 3;

struct BatchParams {
    WsHeader* ws;
    BatchQueue q[kQueues];
    uint32_t split[2];    // block pipeline: blocks [0, split[0]) start on queue 0, [split[0], split[1]) on 1,
                          // the rest on 2
    // warp-tile batches only
    unsigned long long* agg;        // scan element of every warp tile
    unsigned long long* ex;         // scanned offset | entering state of every warp tile
    const uint2* scan_blocks;       // (queue << 30 | chunk, block within the chunk) per tile-scan block
    uint32_t n_scan_blocks;
    uint32_t pad;
};

// A compiled decoder shape.
struct Variant {
    int threads;
    int slots_per_thread;
    int dict_smem;
    size_t smem_bytes;
    const void* kernel;   // the decode kernel
    int warp_tiles;       // 0: block pipeline (one launch after the index pass);
                          // 1: warp tiles (index pass + reduce, tile scan and warp decode launches);
                          // 2: warp tiles in one cooperative launch (small columns)
    int width;            // dictionary read width W: 16 = whole entry, 8 = split read (low plane,
                          // high plane only for tokens longer than 8 bytes; paper Sec. 3.2)
    const void* reduce;   // warp tiles: the reduce kernel (its first blocks run the index pass)
    const void* scan;     // warp tiles: the tile scan kernel
};

// Variant tables (fp_decode.cu).
int variant_count(int codec);
const Variant* variant_get(int codec, int v);
// Default for a code buffer of max_slots slots and a dictionary read width
// (8 or 16; only the OnPair codecs have both).
int variant_default(int codec, uint64_t max_slots, int width);
// The decoder of codes bit-packed at a run-time width (fp_decode_packed):
// one warp-tile variant per escape-free codec, null for FSST-8.
const Variant* variant_packed(int codec);
// The variant fp_decode_noalloc uses when none is selected: the block
// pipeline where the codec has one (its scratch covers the largest inputs).
int noalloc_default(int codec);

// Launch helpers (fp_decode.cu, fp_plain.cu).
uint64_t variant_tile(const Variant& v);   // code slots per tile (block tile or warp tile)
// Device scratch a decode of a buffer of `max_slots` slots needs after the
// 128-byte workspace header.
size_t variant_scratch_bytes(const Variant& v, uint64_t max_slots);
// Index pass + decode of one column.  p.ws is the workspace header, `scratch`
// the variant's scratch; `grid` the decode kernel's persistent width.
cudaError_t launch_decode(int codec, const Variant& var, const DecodeParams& p, void* scratch, uint64_t max_slots,
                          int grid, int sms, cudaStream_t stream);
cudaError_t launch_plain(int codec, const DecodeParams& p, uint32_t* d_scratch, size_t scratch_words,
                         cudaStream_t stream);

// Selective decode (fp_rows.cu): the selected rows of a column and where their
// codes are gathered.
struct RowsArgs {
    const uint8_t* codes;          // the column's stored code buffer
    uint64_t max_slots;            // whole slots in it
    const uint32_t* code_offsets;  // n_strings + 1
    uint32_t n_strings;
    const uint32_t* row_ids;       // n_rows
    uint32_t n_rows;
};
// Scratch of a selective decode (after the decode's own scratch): the
// virtual code offsets v[0 .. n_rows], the scan's block sums, the gathered
// stream (codes_bytes of it are handed to the decode).
struct RowsLayout {
    size_t o_v, o_sums, o_codes, bytes;
    uint64_t codes_bytes;
};
RowsLayout rows_layout(int codec, uint32_t n_rows, uint64_t selected_slots);
// Row lengths, their scan into v (ws->rows_slots gets the total; more than
// selected_slots sets ERRB_CAPACITY) and, with `gather`, the gather of at
// most selected_slots codes: three or four launches.
cudaError_t launch_rows_gather(int codec, const RowsArgs& a, uint64_t selected_slots, bool gather, void* scratch,
                               const RowsLayout& L, WsHeader* ws, int sms, cudaStream_t stream);
size_t plain_scratch_words(uint32_t n_strings);

// A launch slot for batches built on the fly (the server's waves): device
// header and tables that grow on demand and are otherwise reused, pinned
// staging for the tables and for the per-chunk results (fp_batch.cu).
struct WaveBuffers {
    int sms = 0;
    uint32_t cap_chunks = 0;
    void* d_hdr = nullptr;                   // WsHeader | status u32[cap] | total u64[cap]
    uint32_t* d_status = nullptr;
    unsigned long long* d_total = nullptr;
    void* d_layout = nullptr;
    size_t layout_cap = 0;
    void* h_stage = nullptr;                 // pinned copy of the tables of the wave in flight
    size_t stage_cap = 0;
    uint32_t* h_status = nullptr;            // pinned: the last wave's per-chunk data-error bits
    unsigned long long* h_total = nullptr;   // pinned: the last wave's per-chunk decoded sizes
    uint32_t* h_ws_status = nullptr;         // pinned: the last wave's launch-wide bits (timeouts)
    uint64_t launches = 0;
};
fp_status wave_init(WaveBuffers& W, uint32_t cap_chunks);
void wave_free(WaveBuffers& W);
// Enqueue the decode of `n` chunks on `stream`: upload the tables, clear
// the per-chunk words, run the configuration's launches, then copy the
// per-chunk results into W.h_status / W.h_total.  The previous wave of W
// must have completed (its staging is reused).
fp_status wave_launch(WaveBuffers& W, const fp_chunk* chunks, uint32_t n, int config, cudaStream_t stream);
int batch_config_default();

// Host helpers (fp_api.cu).
fp_status fail(fp_status st, const char* fmt, ...);          // sets fp_last_error()
fp_status cuda_fail(cudaError_t e, const char* what);
bool valid_codec(int c);
uint64_t max_slots_of(int codec, uint64_t codes_bytes);
fp_status check_common(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                       const uint32_t* d_code_offsets, uint8_t* d_out_bytes, uint64_t out_capacity,
                       uint32_t* d_out_offsets, bool need_out);
fp_status status_from_bits(uint32_t bits);                    // with an fp_last_error() text
fp_status status_code(uint32_t bits);                         // without
// Validate a dictionary (interchange form) and repack it into the device
// layout: fixed-stride table, per-code lengths, offsets rebased to 0.
fp_status repack_dictionary(fp_codec codec, const uint8_t* h_bytes, const uint32_t* h_offsets, uint32_t n_entries,
                            std::vector<uint8_t>& table, std::vector<uint8_t>& lens, std::vector<uint32_t>& offs);

inline uint32_t code_bits(int codec) {
    return codec == FP_ONPAIR16 ? 16u : (codec == FP_ONPAIR12 || codec == FP_FSST12) ? 12u : codec == FP_FSST8 ? 8u : 0u;
}
inline bool is_onpair(int codec) { return codec == FP_ONPAIR16 || codec == FP_ONPAIR12; }
inline uint32_t max_token(int codec) { return is_onpair(codec) ? 16u : 8u; }
inline uint32_t max_entries(int codec) {
    return codec == FP_ONPAIR16 ? 65536u : (codec == FP_ONPAIR12 || codec == FP_FSST12) ? 4096u
                                         : codec == FP_FSST8 ? 255u : 0u;
}
inline uint32_t table_entries(int codec) {
    return codec == FP_ONPAIR16 ? 65536u : (codec == FP_ONPAIR12 || codec == FP_FSST12) ? 4096u : 256u;
}
inline uint32_t table_stride(int codec) { return is_onpair(codec) ? 16u : 8u; }

// The split-read rule of the paper (Sec. 4.3, gather width): read 8 bytes per token (W = 8)
// unless more than 60 % of the tokens are longer than 8 bytes (W = 16).
// hist[L] counts tokens of L bytes, L = 0..16.
inline int width_for_histogram(const uint64_t* hist) {
    uint64_t all = 0, long_ = 0;
    for (int L = 0; L <= 16; ++L) {
        all += hist[L];
        if (L > 8) long_ += hist[L];
    }
    return (all > 0 && long_ * 5 > all * 3) ? 16 : 8;
}

}  // namespace fp

// Opaque dictionary handle of the C ABI.
struct fp_dict {
    int codec = 0;
    int device = 0;
    uint32_t n_entries = 0;
    int width = 8;                 // dictionary read width fp_decode uses (8 or 16; FSST codecs: 8)
    void* d_table = nullptr;
    uint8_t* d_lens = nullptr;
    void* d_planes = nullptr;      // OnPair: split planes (see DictView); else null
    uint8_t* d_bytes = nullptr;
    uint32_t* d_offsets = nullptr;
    size_t table_bytes = 0;
    fp::DictView view() const {
        return fp::DictView{d_table, d_lens, d_planes, d_bytes, d_offsets, n_entries};
    }
};
