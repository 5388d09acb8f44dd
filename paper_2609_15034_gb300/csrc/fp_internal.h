// Internal declarations shared by the library's host and device sources.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fastpair.h"

namespace fp {

// Sticky data-error bits in the per-stream status word.
constexpr uint32_t ERRB_CORRUPT = 1u;
constexpr uint32_t ERRB_CAPACITY = 2u;
constexpr uint32_t ERRB_OVERFLOW = 4u;
constexpr uint32_t ERRB_TIMEOUT = 8u;

// Device workspace header (one per stream).  It is followed by the tile
// status words of the single-pass prefix scan (one u64 per tile, at
// `kWsHeaderBytes`) and by the tile -> first string index (tiles + 1 u32).
struct WsHeader {
    unsigned int tile_counter;   // next tile ticket
    unsigned int exit_counter;   // blocks that have finished
    unsigned int epoch;          // launch generation tag of tile status words
    unsigned int status;         // sticky ERRB_* bits
    unsigned long long reserved;
    unsigned long long total;    // decoded size of the last launch
    unsigned int abort;          // set when a bounded wait gave up
    unsigned int pad[23];
};
constexpr size_t kWsHeaderBytes = 128;
static_assert(sizeof(WsHeader) == kWsHeaderBytes, "workspace header size");

constexpr unsigned kEpochBits = 26;
constexpr unsigned kEpochMask = (1u << kEpochBits) - 1u;

// Device view of a dictionary (passed by value to kernels).
struct DictView {
    const void* table;        // 2^w entries, 16 B (OnPair) or 8 B (FSST-8) each, zero padded
    const uint8_t* lens;      // 2^w token lengths; 0 = no token (or the FSST-8 escape)
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
    WsHeader* ws;
    unsigned long long* tile_status;
    int size_only;
};

// A compiled tile shape.
struct Variant {
    int threads;
    int slots_per_thread;
    int dict_smem;
    size_t smem_bytes;
    const void* kernel;   // __global__ function
    int work_threads;     // threads that assemble output (slots per tile = work_threads * slots_per_thread)
};

// Variant tables (fp_decode.cu).
int variant_count(int codec);
const Variant* variant_get(int codec, int v);
int variant_default(int codec);

// Launch helpers (fp_decode.cu, fp_plain.cu).
uint64_t variant_tile(const Variant& v);   // code slots per tile
cudaError_t launch_decode(int codec, const Variant& var, const DecodeParams& p, uint32_t* first, int grid,
                          cudaStream_t stream);
cudaError_t launch_plain(int codec, const DecodeParams& p, uint32_t* d_scratch, size_t scratch_words,
                         cudaStream_t stream);
size_t plain_scratch_words(uint32_t n_strings);

inline uint32_t code_bits(int codec) {
    return codec == FP_ONPAIR16 ? 16u : codec == FP_ONPAIR12 ? 12u : codec == FP_FSST8 ? 8u : 0u;
}
inline uint32_t max_token(int codec) { return codec == FP_FSST8 ? 8u : 16u; }
inline uint32_t max_entries(int codec) {
    return codec == FP_ONPAIR16 ? 65536u : codec == FP_ONPAIR12 ? 4096u : codec == FP_FSST8 ? 255u : 0u;
}
inline uint32_t table_entries(int codec) {
    return codec == FP_ONPAIR16 ? 65536u : codec == FP_ONPAIR12 ? 4096u : 256u;
}
inline uint32_t table_stride(int codec) { return codec == FP_FSST8 ? 8u : 16u; }

}  // namespace fp

// Opaque dictionary handle of the C ABI.
struct fp_dict {
    int codec;
    int device;
    uint32_t n_entries;
    void* d_table;
    uint8_t* d_lens;
    uint8_t* d_bytes;
    uint32_t* d_offsets;
    size_t table_bytes;
    fp::DictView view() const {
        return fp::DictView{d_table, d_lens, d_bytes, d_offsets, n_entries};
    }
};
