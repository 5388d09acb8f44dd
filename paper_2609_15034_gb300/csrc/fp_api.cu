// Host side of the C ABI (include/fastpair.h): argument validation,
// dictionary repacking and upload, per-stream workspaces, variant selection
// and kernel launches.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "fp_internal.h"

namespace fp {

namespace {
thread_local std::string g_last_error;
}  // namespace

fp_status fail(fp_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

fp_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? FP_ERR_NOMEM : FP_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

bool valid_codec(int c) { return c == FP_ONPAIR16 || c == FP_ONPAIR12 || c == FP_FSST8 || c == FP_FSST12; }

namespace {

// ---- per-stream workspace ----------------------------------------------------
struct Workspace {
    void* d_mem = nullptr;        // WsHeader + the decoder's scratch
    size_t scratch_cap = 0;       // bytes after the header
    uint64_t launches = 0;
    uint32_t* d_plain = nullptr;  // scratch of the plain baseline
    size_t plain_words = 0;
};

std::mutex g_mu;
std::map<std::pair<int, cudaStream_t>, Workspace*> g_ws;

// Get (or grow) the workspace of (current device, stream): the header plus
// `scratch` bytes.
fp_status get_workspace(cudaStream_t stream, size_t scratch, size_t plain_words, Workspace** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace*& w = g_ws[{dev, stream}];
    if (!w) w = new Workspace();
    if (w->d_mem == nullptr || w->scratch_cap < scratch) {
        size_t cap = w->scratch_cap ? w->scratch_cap : (64u << 10);
        while (cap < scratch) cap *= 2;
        if (w->d_mem) {
            e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
            cudaFree(w->d_mem);
            w->d_mem = nullptr;
            w->scratch_cap = 0;
        }
        const size_t bytes = kWsHeaderBytes + cap;
        e = cudaMalloc(&w->d_mem, bytes);
        if (e != cudaSuccess) { w->d_mem = nullptr; return cuda_fail(e, "cudaMalloc(workspace)"); }
        // initialise in `stream` order, ahead of the launches that use it
        static const unsigned one = 1;   // epoch 0 is reserved for "never written"
        e = cudaMemsetAsync(w->d_mem, 0, bytes, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(workspace)");
        e = cudaMemcpyAsync(reinterpret_cast<char*>(w->d_mem) + offsetof(WsHeader, epoch), &one, sizeof(one),
                            cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(epoch)");
        w->scratch_cap = cap;
        w->launches = 0;
    }
    if (plain_words && w->plain_words < plain_words) {
        if (w->d_plain) {
            e = cudaStreamSynchronize(stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
            cudaFree(w->d_plain);
            w->d_plain = nullptr;
            w->plain_words = 0;
        }
        e = cudaMalloc(&w->d_plain, plain_words * sizeof(uint32_t));
        if (e != cudaSuccess) { w->d_plain = nullptr; return cuda_fail(e, "cudaMalloc(plain scratch)"); }
        w->plain_words = plain_words;
    }
    *out = w;
    return FP_OK;
}

Workspace* find_workspace(cudaStream_t stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_ws.find({dev, stream});
    return it == g_ws.end() ? nullptr : it->second;
}

// ---- variants and occupancy ----------------------------------------------------
std::atomic<int> g_selected[5] = {{-1}, {-1}, {-1}, {-1}, {-1}};

// Tuned shapes: (SM count, codec, read width, size class = floor(log2 of the
// code slots)) -> variant, from fp_tune_column or a loaded tuning file.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tuned;
std::atomic<int> g_tuned_any{0};
int g_sms_cached = 0;   // SM count of the device the first tuned lookup ran on

int size_class(uint64_t max_slots) {
    int c = 0;
    while (c < 63 && (max_slots >> (c + 1)) != 0) ++c;
    return c;
}

int device_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

// The selected variant, else a tuned one for this device, codec, width and
// size class, else the built-in default.
int selected_variant(int codec, uint64_t max_slots, int width) {
    const int v = g_selected[codec].load();
    if (v >= 0) return v;
    if (g_tuned_any.load()) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (!g_sms_cached) g_sms_cached = device_sms();
        auto it = g_tuned.find(std::make_tuple(g_sms_cached, codec, width, size_class(max_slots)));
        if (it != g_tuned.end() && variant_get(codec, it->second)) return it->second;
    }
    return variant_default(codec, max_slots, width);
}

struct DevInfo {
    int sms = 0;
    std::map<const void*, int> blocks_per_sm;
};
std::map<int, DevInfo> g_dev;

fp_status grid_for(const Variant& var, int* grid_per_wave, int* sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_mu);
    DevInfo& di = g_dev[dev];
    if (di.sms == 0) {
        e = cudaDeviceGetAttribute(&di.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    }
    auto it = di.blocks_per_sm.find(var.kernel);
    if (it == di.blocks_per_sm.end()) {
        e = cudaFuncSetAttribute(var.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)var.smem_bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, var.kernel, var.threads, var.smem_bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        if (nb < 1) return fail(FP_ERR_CUDA, "decode variant does not fit on an SM");
        it = di.blocks_per_sm.emplace(var.kernel, nb).first;
    }
    *grid_per_wave = it->second * di.sms;
    *sms = di.sms;
    return FP_OK;
}

}  // namespace

uint64_t max_slots_of(int codec, uint64_t codes_bytes) { return codes_bytes * 8 / code_bits(codec); }

fp_status check_common(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                       const uint32_t* d_code_offsets, uint8_t* d_out_bytes, uint64_t out_capacity,
                       uint32_t* d_out_offsets, bool need_out) {
    if (!valid_codec(codec)) return fail(FP_ERR_ARG, "unknown codec %d", (int)codec);
    if (!dict) return fail(FP_ERR_ARG, "dict is NULL");
    if (dict->codec != codec) return fail(FP_ERR_ARG, "dictionary codec %d != codec %d", dict->codec, (int)codec);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != dict->device)
        return fail(FP_ERR_ARG, "dictionary lives on device %d, current device is %d", dict->device, dev);
    if (!d_code_offsets) return fail(FP_ERR_ARG, "d_code_offsets is NULL");
    if (reinterpret_cast<uintptr_t>(d_code_offsets) % 4) return fail(FP_ERR_ARG, "d_code_offsets not 4-byte aligned");
    if (codes_bytes && !d_codes) return fail(FP_ERR_ARG, "d_codes is NULL");
    if (reinterpret_cast<uintptr_t>(d_codes) % 16) return fail(FP_ERR_ARG, "d_codes not 16-byte aligned");
    if (need_out) {
        if (!d_out_offsets) return fail(FP_ERR_ARG, "d_out_offsets is NULL");
        if (reinterpret_cast<uintptr_t>(d_out_offsets) % 4) return fail(FP_ERR_ARG, "d_out_offsets not 4-byte aligned");
        if (out_capacity && !d_out_bytes) return fail(FP_ERR_ARG, "d_out_bytes is NULL");
        if (reinterpret_cast<uintptr_t>(d_out_bytes) % 16) return fail(FP_ERR_ARG, "d_out_bytes not 16-byte aligned");
    }
    return FP_OK;
}

fp_status status_from_bits(uint32_t bits) {
    if (bits & ERRB_TIMEOUT) return fail(FP_ERR_TIMEOUT, "a bounded device-side wait gave up");
    if (bits & ERRB_MISMATCH)
        return fail(FP_ERR_INTERNAL, "decoder self-check: a warp tile's byte total disagrees with the scanned offsets");
    if (bits & ERRB_CORRUPT) return fail(FP_ERR_CORRUPT, "corrupt input (code >= n_entries, dangling escape or bad code_offsets)");
    if (bits & ERRB_CAPACITY) return fail(FP_ERR_CAPACITY, "decoded size exceeds out_capacity");
    if (bits & ERRB_OVERFLOW) return fail(FP_ERR_OVERFLOW, "decoded size exceeds 2^31-1");
    return FP_OK;
}

fp_status status_code(uint32_t bits) {
    if (bits & ERRB_TIMEOUT) return FP_ERR_TIMEOUT;
    if (bits & ERRB_MISMATCH) return FP_ERR_INTERNAL;
    if (bits & ERRB_CORRUPT) return FP_ERR_CORRUPT;
    if (bits & ERRB_CAPACITY) return FP_ERR_CAPACITY;
    if (bits & ERRB_OVERFLOW) return FP_ERR_OVERFLOW;
    return FP_OK;
}

namespace {

// Read and clear the workspace status (stream already synchronised); the
// clear is ordered before the stream's next launch.
fp_status take_status(Workspace* w, uint64_t* total, cudaStream_t stream) {
    WsHeader h;
    cudaError_t e = cudaMemcpy(&h, w->d_mem, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(status)");
    if (h.status) {
        e = cudaMemsetAsync(reinterpret_cast<char*>(w->d_mem) + offsetof(WsHeader, status), 0, sizeof(unsigned),
                            stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(status)");
    }
    if (total) *total = h.total;
    return status_from_bits(h.status);
}

fp_status run_decode(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                     const uint32_t* d_code_offsets, uint32_t n_strings, uint8_t* d_out_bytes,
                     uint64_t out_capacity, uint32_t* d_out_offsets, cudaStream_t stream, bool size_only,
                     Workspace** ws_out, uint32_t packed_bits = 0, int force_variant = -1) {
    const uint64_t max_slots = packed_bits ? codes_bytes * 8 / packed_bits : max_slots_of(codec, codes_bytes);
    const Variant* var = packed_bits          ? variant_packed(codec)
                         : force_variant >= 0 ? variant_get(codec, force_variant)
                                              : variant_get(codec, selected_variant(codec, max_slots, dict->width));
    if (!var) return fail(FP_ERR_ARG, "no decode variant for codec %d", (int)codec);
    if (n_strings == 0xffffffffu) return fail(FP_ERR_ARG, "n_strings must be below 2^32-1");
    const uint64_t tile = variant_tile(*var);
    const uint64_t n_tiles = max_slots / tile + 2;
    int per_wave = 0, sms = 0;
    fp_status st = grid_for(*var, &per_wave, &sms);
    if (st != FP_OK) return st;
    Workspace* w = nullptr;
    st = get_workspace(stream, variant_scratch_bytes(*var, max_slots), 0, &w);
    if (st != FP_OK) return st;
    if ((++w->launches & ((1ull << 25) - 1)) == 0) {
        // Tile status words carry a 26-bit launch tag; clear them well before it wraps.
        cudaError_t e = cudaMemsetAsync(reinterpret_cast<char*>(w->d_mem) + kWsHeaderBytes, 0, w->scratch_cap,
                                        stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
    DecodeParams p{};
    p.dict = dict->view();
    p.codes = static_cast<const uint8_t*>(d_codes);
    p.codes_bytes = codes_bytes;
    p.max_slots = max_slots;
    p.code_offsets = d_code_offsets;
    p.n_strings = n_strings;
    p.out = d_out_bytes;
    p.capacity = size_only ? 0 : out_capacity;
    p.out_offsets = d_out_offsets;
    p.ws = static_cast<WsHeader*>(w->d_mem);
    p.size_only = size_only ? 1 : 0;
    p.packed_bits = packed_bits;
    const uint64_t grid = (n_tiles < (uint64_t)per_wave && !var->warp_tiles) ? n_tiles : (uint64_t)per_wave;
    cudaError_t e = launch_decode(codec, *var, p, static_cast<char*>(w->d_mem) + kWsHeaderBytes, max_slots,
                                  (int)grid, sms, stream);
    if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    if (ws_out) *ws_out = w;
    return FP_OK;
}

// ---- selective decode --------------------------------------------------------
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

fp_status check_rows(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                     const uint32_t* d_code_offsets, uint32_t n_strings, const uint32_t* d_row_ids, uint32_t n_rows,
                     uint8_t* d_out_bytes, uint64_t out_capacity, uint32_t* d_out_offsets, bool need_out) {
    fp_status st = check_common(codec, dict, d_codes, codes_bytes, d_code_offsets, d_out_bytes, out_capacity,
                                d_out_offsets, need_out);
    if (st != FP_OK) return st;
    if (n_strings == 0xffffffffu || n_rows == 0xffffffffu) return fail(FP_ERR_ARG, "n_strings/n_rows must be below 2^32-1");
    if (n_rows && !d_row_ids) return fail(FP_ERR_ARG, "d_row_ids is NULL");
    if (reinterpret_cast<uintptr_t>(d_row_ids) % 4) return fail(FP_ERR_ARG, "d_row_ids not 4-byte aligned");
    return FP_OK;
}

// Enqueue a selective decode of at most `slots` selected code slots: row
// scan, gather, then the decode's launches on the gathered stream.
fp_status run_rows(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                   const uint32_t* d_code_offsets, uint32_t n_strings, const uint32_t* d_row_ids, uint32_t n_rows,
                   uint64_t slots, uint8_t* d_out_bytes, uint64_t out_capacity, uint32_t* d_out_offsets,
                   cudaStream_t stream, bool size_only, Workspace** ws_out) {
    if (slots > 0xffffffffull) return fail(FP_ERR_ARG, "selected_slots %llu: at most 2^32-1", (unsigned long long)slots);
    const RowsLayout RL = rows_layout(codec, n_rows, slots);
    const uint64_t dec_slots = max_slots_of(codec, RL.codes_bytes);
    const Variant* var = variant_get(codec, selected_variant(codec, dec_slots, dict->width));
    if (!var) return fail(FP_ERR_ARG, "no decode variant for codec %d", (int)codec);
    int per_wave = 0, sms = 0;
    fp_status st = grid_for(*var, &per_wave, &sms);
    if (st != FP_OK) return st;
    const size_t dec_bytes = al256(variant_scratch_bytes(*var, dec_slots));
    Workspace* w = nullptr;
    st = get_workspace(stream, dec_bytes + RL.bytes, 0, &w);
    if (st != FP_OK) return st;
    if ((++w->launches & ((1ull << 25) - 1)) == 0) {
        cudaError_t e = cudaMemsetAsync(reinterpret_cast<char*>(w->d_mem) + kWsHeaderBytes, 0, w->scratch_cap,
                                        stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    }
    char* scratch = static_cast<char*>(w->d_mem) + kWsHeaderBytes;
    char* rows = scratch + dec_bytes;
    WsHeader* ws = static_cast<WsHeader*>(w->d_mem);
    const RowsArgs a{static_cast<const uint8_t*>(d_codes), max_slots_of(codec, codes_bytes), d_code_offsets,
                     n_strings, d_row_ids, n_rows};
    cudaError_t e = launch_rows_gather(codec, a, slots, true, rows, RL, ws, sms, stream);
    if (e != cudaSuccess) return cuda_fail(e, "row gather launch");
    DecodeParams p{};
    p.dict = dict->view();
    p.codes = reinterpret_cast<const uint8_t*>(rows + RL.o_codes);
    p.codes_bytes = RL.codes_bytes;
    p.max_slots = dec_slots;
    p.code_offsets = reinterpret_cast<const uint32_t*>(rows + RL.o_v);
    p.n_strings = n_rows;
    p.out = d_out_bytes;
    p.capacity = size_only ? 0 : out_capacity;
    p.out_offsets = d_out_offsets;
    p.ws = ws;
    p.size_only = size_only ? 1 : 0;
    const uint64_t n_tiles = dec_slots / variant_tile(*var) + 2;
    const uint64_t grid = (n_tiles < (uint64_t)per_wave && !var->warp_tiles) ? n_tiles : (uint64_t)per_wave;
    e = launch_decode(codec, *var, p, scratch, dec_slots, (int)grid, sms, stream);
    if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    if (ws_out) *ws_out = w;
    return FP_OK;
}

}  // namespace

fp_status repack_dictionary(fp_codec codec, const uint8_t* h_bytes, const uint32_t* h_offsets, uint32_t n_entries,
                            std::vector<uint8_t>& table, std::vector<uint8_t>& lens, std::vector<uint32_t>& offs) {
    if (!valid_codec(codec)) return fail(FP_ERR_ARG, "unknown codec %d", (int)codec);
    if (!h_offsets || !h_bytes) return fail(FP_ERR_ARG, "h_bytes/h_offsets is NULL");
    if (n_entries < 1 || n_entries > max_entries(codec))
        return fail(FP_ERR_ARG, "n_entries %u out of range 1..%u", n_entries, max_entries(codec));
    const uint32_t L = max_token(codec);
    for (uint32_t i = 0; i < n_entries; ++i) {
        if (h_offsets[i + 1] < h_offsets[i]) return fail(FP_ERR_ARG, "h_offsets decrease at %u", i);
        const uint32_t len = h_offsets[i + 1] - h_offsets[i];
        if (len < 1 || len > L) return fail(FP_ERR_ARG, "token %u has length %u (allowed 1..%u)", i, len, L);
    }
    const uint32_t n_tab = table_entries(codec), stride = table_stride(codec);
    table.assign((size_t)n_tab * stride, 0);
    lens.assign(n_tab, 0);
    for (uint32_t i = 0; i < n_entries; ++i) {
        const uint32_t a = h_offsets[i], len = h_offsets[i + 1] - a;
        memcpy(&table[(size_t)i * stride], h_bytes + a, len);
        lens[i] = (uint8_t)len;
    }
    offs.resize(n_entries + 1);
    for (uint32_t i = 0; i <= n_entries; ++i) offs[i] = h_offsets[i] - h_offsets[0];
    return FP_OK;
}

}  // namespace fp

using namespace fp;

extern "C" {

const char* fp_last_error(void) { return g_last_error.c_str(); }

fp_status fp_dict_upload(fp_codec codec, const uint8_t* h_bytes, const uint32_t* h_offsets,
                         uint32_t n_entries, fp_stream_t stream_, fp_dict** out) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (!out) return fail(FP_ERR_ARG, "out is NULL");
    *out = nullptr;
    std::vector<uint8_t> table, lens;
    std::vector<uint32_t> offs;
    fp_status st = repack_dictionary(codec, h_bytes, h_offsets, n_entries, table, lens, offs);
    if (st != FP_OK) return st;
    const uint32_t base = h_offsets[0], nbytes = offs[n_entries];

    fp_dict* d = new fp_dict();
    d->codec = codec;
    d->n_entries = n_entries;
    d->table_bytes = table.size();
    // OnPair: the two 8-byte planes of the entries (for split reads) and the
    // read width.  The default is 16: on GB300 this decoder read whole
    // entries faster than split reads for every share of long tokens from 0
    // to 100 % (1-3 % with the table in shared memory, 5-13 % through L1), so
    // the paper's rule (fp_width_for_histogram) is left to callers, through
    // fp_dict_set_width.
    std::vector<uint8_t> planes;
    d->width = is_onpair(codec) ? 16 : 8;
    if (is_onpair(codec)) {
        const size_t n_tab = table_entries(codec);
        planes.resize(n_tab * 16);
        for (size_t i = 0; i < n_tab; ++i) {
            memcpy(&planes[i * 8], &table[i * 16], 8);
            memcpy(&planes[(n_tab + i) * 8], &table[i * 16 + 8], 8);
        }
    }
    cudaError_t e = cudaGetDevice(&d->device);
    if (e == cudaSuccess) e = cudaMalloc(&d->d_table, table.size());
    if (e == cudaSuccess && !planes.empty()) e = cudaMalloc(&d->d_planes, planes.size());
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&d->d_lens), lens.size());
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&d->d_bytes), nbytes ? nbytes : 1);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&d->d_offsets), offs.size() * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpyAsync(d->d_table, table.data(), table.size(), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && !planes.empty())
        e = cudaMemcpyAsync(d->d_planes, planes.data(), planes.size(), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d->d_lens, lens.data(), lens.size(), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && nbytes)
        e = cudaMemcpyAsync(d->d_bytes, h_bytes + base, nbytes, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d->d_offsets, offs.data(), offs.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        fp_dict_free(d);
        return cuda_fail(e, "dictionary upload");
    }
    *out = d;
    return FP_OK;
}

fp_status fp_dict_free(fp_dict* d) {
    if (!d) return FP_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(d->device);
    cudaDeviceSynchronize();
    cudaFree(d->d_table);
    cudaFree(d->d_lens);
    if (d->d_planes) cudaFree(d->d_planes);
    cudaFree(d->d_bytes);
    cudaFree(d->d_offsets);
    cudaSetDevice(prev);
    delete d;
    return FP_OK;
}

fp_status fp_rows_size(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                       const uint32_t* d_code_offsets, uint32_t n_strings, const uint32_t* d_row_ids,
                       uint32_t n_rows, fp_stream_t stream_, uint64_t* h_slots, uint64_t* h_bytes) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (!h_slots || !h_bytes) return fail(FP_ERR_ARG, "h_slots/h_bytes is NULL");
    fp_status st = check_rows(codec, dict, d_codes, codes_bytes, d_code_offsets, n_strings, d_row_ids, n_rows,
                              nullptr, 0, nullptr, false);
    if (st != FP_OK) return st;
    // 1: the selected rows' slot count (row scan alone)
    const RowsLayout RL0 = rows_layout(codec, n_rows, 0);
    Workspace* w = nullptr;
    st = get_workspace(stream, RL0.bytes, 0, &w);
    if (st != FP_OK) return st;
    int dev_sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dict->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    const RowsArgs a{static_cast<const uint8_t*>(d_codes), max_slots_of(codec, codes_bytes), d_code_offsets,
                     n_strings, d_row_ids, n_rows};
    e = launch_rows_gather(codec, a, ~0ull, false, static_cast<char*>(w->d_mem) + kWsHeaderBytes, RL0,
                           static_cast<WsHeader*>(w->d_mem), dev_sms, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "row scan");
    WsHeader h;
    e = cudaMemcpy(&h, w->d_mem, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(row scan)");
    *h_slots = h.rows_slots;
    *h_bytes = 0;
    if (h.status) return take_status(w, nullptr, stream);
    // 2: gather and size the selected rows
    st = run_rows(codec, dict, d_codes, codes_bytes, d_code_offsets, n_strings, d_row_ids, n_rows, h.rows_slots,
                  nullptr, 0, nullptr, stream, true, &w);
    if (st != FP_OK) return st;
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return take_status(w, h_bytes, stream);
}

fp_status fp_decode_rows(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                         const uint32_t* d_code_offsets, uint32_t n_strings, const uint32_t* d_row_ids,
                         uint32_t n_rows, uint64_t selected_slots, uint8_t* d_out_bytes, uint64_t out_capacity,
                         uint32_t* d_out_offsets, fp_stream_t stream) {
    fp_status st = check_rows(codec, dict, d_codes, codes_bytes, d_code_offsets, n_strings, d_row_ids, n_rows,
                              d_out_bytes, out_capacity, d_out_offsets, true);
    if (st != FP_OK) return st;
    return run_rows(codec, dict, d_codes, codes_bytes, d_code_offsets, n_strings, d_row_ids, n_rows, selected_slots,
                    d_out_bytes, out_capacity, d_out_offsets, reinterpret_cast<cudaStream_t>(stream), false, nullptr);
}

namespace {
fp_status check_packed(fp_codec codec, uint32_t code_bits_) {
    if (codec != FP_ONPAIR16 && codec != FP_ONPAIR12 && codec != FP_FSST12)
        return fail(FP_ERR_ARG, "packed codes: codec %d has escapes or is unknown", (int)codec);
    if (code_bits_ < 1 || code_bits_ > code_bits(codec))
        return fail(FP_ERR_ARG, "packed codes: %u bits per code, the codec allows 1..%u", code_bits_, code_bits(codec));
    return FP_OK;
}
}  // namespace

fp_status fp_decode_packed(fp_codec codec, const fp_dict* dict, uint32_t code_bits_, const void* d_codes,
                           uint64_t codes_bytes, const uint32_t* d_code_offsets, uint32_t n_strings,
                           uint8_t* d_out_bytes, uint64_t out_capacity, uint32_t* d_out_offsets, fp_stream_t stream) {
    fp_status st = check_common(codec, dict, d_codes, codes_bytes, d_code_offsets, d_out_bytes, out_capacity,
                                d_out_offsets, true);
    if (st == FP_OK) st = check_packed(codec, code_bits_);
    if (st != FP_OK) return st;
    if (n_strings == 0xffffffffu) return fail(FP_ERR_ARG, "n_strings must be below 2^32-1");
    return run_decode(codec, dict, d_codes, codes_bytes, d_code_offsets, n_strings, d_out_bytes, out_capacity,
                      d_out_offsets, reinterpret_cast<cudaStream_t>(stream), false, nullptr, code_bits_);
}

fp_status fp_decoded_size_packed(fp_codec codec, const fp_dict* dict, uint32_t code_bits_, const void* d_codes,
                                 uint64_t codes_bytes, const uint32_t* d_code_offsets, uint32_t n_strings,
                                 fp_stream_t stream_, uint64_t* h_total) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (!h_total) return fail(FP_ERR_ARG, "h_total is NULL");
    fp_status st = check_common(codec, dict, d_codes, codes_bytes, d_code_offsets, nullptr, 0, nullptr, false);
    if (st == FP_OK) st = check_packed(codec, code_bits_);
    if (st != FP_OK) return st;
    if (n_strings == 0xffffffffu) return fail(FP_ERR_ARG, "n_strings must be below 2^32-1");
    Workspace* w = nullptr;
    st = run_decode(codec, dict, d_codes, codes_bytes, d_code_offsets, n_strings, nullptr, 0, nullptr, stream, true,
                    &w, code_bits_);
    if (st != FP_OK) return st;
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return take_status(w, h_total, stream);
}

fp_status fp_tune_column(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                         const uint32_t* d_code_offsets, uint32_t n_strings, uint8_t* d_out_bytes,
                         uint64_t out_capacity, uint32_t* d_out_offsets, const char* table_path, fp_stream_t stream_,
                         int* chosen, float* best_ms) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    fp_status st = check_common(codec, dict, d_codes, codes_bytes, d_code_offsets, d_out_bytes, out_capacity,
                                d_out_offsets, true);
    if (st != FP_OK) return st;
    if (n_strings == 0xffffffffu) return fail(FP_ERR_ARG, "n_strings must be below 2^32-1");
    const uint64_t max_slots = max_slots_of(codec, codes_bytes);
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    int best = -1;
    float best_t = 0.0f;
    const int nv = variant_count(codec);
    for (int v = 0; v < nv && st == FP_OK; ++v) {
        if (variant_get(codec, v)->width != dict->width) continue;   // the dictionary's read width only
        float t_best = -1.0f;
        for (int r = 0; r < 4 && st == FP_OK; ++r) {   // one warm-up, best of three
            e = cudaEventRecord(a, stream);
            if (e == cudaSuccess)
                st = run_decode(codec, dict, d_codes, codes_bytes, d_code_offsets, n_strings, d_out_bytes,
                                out_capacity, d_out_offsets, stream, false, nullptr, 0, v);
            if (e == cudaSuccess && st == FP_OK) e = cudaEventRecord(b, stream);
            if (e == cudaSuccess && st == FP_OK) e = cudaEventSynchronize(b);
            float ms = 0.0f;
            if (e == cudaSuccess && st == FP_OK) e = cudaEventElapsedTime(&ms, a, b);
            if (e != cudaSuccess && st == FP_OK) st = cuda_fail(e, "tuning run");
            if (st == FP_OK && r > 0 && (t_best < 0.0f || ms < t_best)) t_best = ms;
        }
        if (st == FP_OK && (best < 0 || t_best < best_t)) {
            best = v;
            best_t = t_best;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != FP_OK) return st;
    // a data error in the column makes its timings meaningless
    st = fp_sync_status(stream_);
    if (st != FP_OK) return st;
    const int sms = device_sms();
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[std::make_tuple(sms, (int)codec, dict->width, size_class(max_slots))] = best;
        g_tuned_any.store(1);
    }
    if (table_path) {
        FILE* f = fopen(table_path, "a");
        if (!f) return fail(FP_ERR_ARG, "cannot open tuning table %s", table_path);
        fprintf(f, "%d %d %d %d %d %.4f\n", sms, (int)codec, dict->width, size_class(max_slots), best, best_t);
        fclose(f);
    }
    if (chosen) *chosen = best;
    if (best_ms) *best_ms = best_t;
    return FP_OK;
}

fp_status fp_tune_load(const char* table_path) {
    if (!table_path) return fail(FP_ERR_ARG, "table_path is NULL");
    FILE* f = fopen(table_path, "r");
    if (!f) return fail(FP_ERR_ARG, "cannot open tuning table %s", table_path);
    int sms, codec, width, cls, v, n = 0;
    float ms;
    char line[256];
    std::lock_guard<std::mutex> lk(g_tune_mu);
    while (fgets(line, sizeof(line), f)) {
        if (line[0] == '#') continue;
        if (sscanf(line, "%d %d %d %d %d %f", &sms, &codec, &width, &cls, &v, &ms) != 6) continue;
        if (!valid_codec(codec) || !variant_get(codec, v)) continue;   // built for another library
        g_tuned[std::make_tuple(sms, codec, width, cls)] = v;   // later lines win
        ++n;
    }
    fclose(f);
    if (n) g_tuned_any.store(1);
    return FP_OK;
}

fp_status fp_tune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned.clear();
    g_tuned_any.store(0);
    return FP_OK;
}

int fp_width_for_histogram(const uint64_t* hist17) { return hist17 ? width_for_histogram(hist17) : 8; }

fp_status fp_dict_set_width(fp_dict* dict, int width) {
    if (!dict) return fail(FP_ERR_ARG, "dict is NULL");
    if (width != 8 && width != 16) return fail(FP_ERR_ARG, "width %d: must be 8 or 16", width);
    if (width == 16 && !is_onpair(dict->codec)) return fail(FP_ERR_ARG, "FSST dictionaries have 8-byte entries");
    dict->width = width;
    return FP_OK;
}

int fp_dict_width(const fp_dict* dict) { return dict ? dict->width : 0; }

fp_status fp_decode(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                    const uint32_t* d_code_offsets, uint32_t n_strings, uint8_t* d_out_bytes,
                    uint64_t out_capacity, uint32_t* d_out_offsets, fp_stream_t stream) {
    fp_status st = check_common(codec, dict, d_codes, codes_bytes, d_code_offsets, d_out_bytes, out_capacity,
                                d_out_offsets, true);
    if (st != FP_OK) return st;
    return run_decode(codec, dict, d_codes, codes_bytes, d_code_offsets, n_strings, d_out_bytes, out_capacity,
                      d_out_offsets, reinterpret_cast<cudaStream_t>(stream), false, nullptr);
}

fp_status fp_decoded_size(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                          const uint32_t* d_code_offsets, uint32_t n_strings, fp_stream_t stream_,
                          uint64_t* h_total) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (!h_total) return fail(FP_ERR_ARG, "h_total is NULL");
    fp_status st = check_common(codec, dict, d_codes, codes_bytes, d_code_offsets, nullptr, 0, nullptr, false);
    if (st != FP_OK) return st;
    Workspace* w = nullptr;
    st = run_decode(codec, dict, d_codes, codes_bytes, d_code_offsets, n_strings, nullptr, 0, nullptr, stream,
                    true, &w);
    if (st != FP_OK) return st;
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return take_status(w, h_total, stream);
}

fp_status fp_decode_plain(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                          const uint32_t* d_code_offsets, uint32_t n_strings, uint8_t* d_out_bytes,
                          uint64_t out_capacity, uint32_t* d_out_offsets, fp_stream_t stream_) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    fp_status st = check_common(codec, dict, d_codes, codes_bytes, d_code_offsets, d_out_bytes, out_capacity,
                                d_out_offsets, true);
    if (st != FP_OK) return st;
    Workspace* w = nullptr;
    const size_t words = plain_scratch_words(n_strings);
    st = get_workspace(stream, 256, words, &w);
    if (st != FP_OK) return st;
    DecodeParams p{};
    memset(&p, 0, sizeof(p));
    p.dict = dict->view();
    p.codes = static_cast<const uint8_t*>(d_codes);
    p.codes_bytes = codes_bytes;
    p.max_slots = max_slots_of(codec, codes_bytes);
    p.code_offsets = d_code_offsets;
    p.n_strings = n_strings;
    p.out = d_out_bytes;
    p.capacity = out_capacity;
    p.out_offsets = d_out_offsets;
    p.ws = static_cast<WsHeader*>(w->d_mem);
    p.size_only = 0;
    cudaError_t e = launch_plain(codec, p, w->d_plain, w->plain_words, stream);
    if (e != cudaSuccess) return cuda_fail(e, "plain decode launch");
    return FP_OK;
}

fp_status fp_sync_status(fp_stream_t stream_) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    Workspace* w = find_workspace(stream);
    if (!w || !w->d_mem) return FP_OK;
    return take_status(w, nullptr, stream);
}

fp_status fp_debug_stall_next(fp_stream_t stream_, uint32_t spin_limit) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    if (spin_limit < 1 || spin_limit > (1u << 20)) return fail(FP_ERR_ARG, "spin_limit %u outside 1..2^20", spin_limit);
    Workspace* w = find_workspace(stream);
    if (!w || !w->d_mem) return fail(FP_ERR_ARG, "no workspace on this stream yet (decode once first)");
    // ticket 0 is taken here, so no launch ever publishes the first look-back
    // word; the kernels reset both fields when the launch ends
    // (pageable sources: each copy is staged before cudaMemcpyAsync returns);
    // a phantom arrival count that no grid reaches stalls the one-launch
    // path's first grid barrier
    const unsigned skip_first = 1u, limit = spin_limit, phantom = 1u << 30;
    char* h = static_cast<char*>(w->d_mem);
    cudaError_t e = cudaMemcpyAsync(h + offsetof(WsHeader, tile_counter), &skip_first, sizeof(unsigned),
                                    cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h + offsetof(WsHeader, bar_count), &phantom, sizeof(unsigned), cudaMemcpyHostToDevice,
                            stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h + offsetof(WsHeader, spin_limit), &limit, sizeof(unsigned), cudaMemcpyHostToDevice,
                            stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(stall)");
    return FP_OK;
}

int fp_variant_count(fp_codec codec) { return valid_codec(codec) ? variant_count(codec) : 0; }

fp_status fp_variant_info(fp_codec codec, int v, uint32_t* threads, uint32_t* slots_per_thread,
                          uint32_t* dict_in_smem, uint32_t* launches_per_call) {
    if (!valid_codec(codec)) return fail(FP_ERR_ARG, "unknown codec %d", (int)codec);
    const Variant* var = variant_get(codec, v);
    if (!var) return fail(FP_ERR_ARG, "variant %d out of range", v);
    if (threads) *threads = (uint32_t)var->threads;
    if (slots_per_thread) *slots_per_thread = (uint32_t)var->slots_per_thread;
    if (dict_in_smem) *dict_in_smem = (uint32_t)var->dict_smem;
    if (launches_per_call) *launches_per_call = var->warp_tiles == 2 ? 1u : var->warp_tiles ? 3u : 2u;
    return FP_OK;
}

fp_status fp_variant_select(fp_codec codec, int v) {
    if (!valid_codec(codec)) return fail(FP_ERR_ARG, "unknown codec %d", (int)codec);
    if (v != -1 && !variant_get(codec, v)) return fail(FP_ERR_ARG, "variant %d out of range", v);
    g_selected[codec].store(v);
    return FP_OK;
}

int fp_variant_selected(fp_codec codec) { return valid_codec(codec) ? selected_variant(codec, 1ull << 32, 8) : -1; }

int fp_variant_for(fp_codec codec, uint64_t codes_bytes) {
    return valid_codec(codec) ? selected_variant(codec, max_slots_of(codec, codes_bytes), 8) : -1;
}

int fp_variant_for_dict(const fp_dict* dict, uint64_t codes_bytes) {
    return dict && valid_codec(dict->codec)
               ? selected_variant(dict->codec, max_slots_of(dict->codec, codes_bytes), dict->width)
               : -1;
}

int fp_variant_width(fp_codec codec, int v) {
    const Variant* var = valid_codec(codec) ? variant_get(codec, v) : nullptr;
    return var ? var->width : 0;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Decoding without allocation.
//
// Some callers cannot call cudaMalloc at all: an allocator hook, or an
// embedding engine that owns all device memory and forbids other
// allocations.  fp_decode_noalloc serves them: its
// scratch (the workspace header, one status word per tile and the tile ->
// first string index) lives in the fixed array below, which every GPU that
// loads this library holds until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocScratchBytes = 1u << 20;   // 1 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
    bool ready = false;
    void* ptr = nullptr;        // device address of g_noalloc_scratch on this device
    uint64_t launches = 0;
};
std::mutex g_noalloc_mu;
std::map<int, NoAllocDevice> g_noalloc;

// Once per device, with that device current: look up the array's device
// address (in host code its name only stands for it) and initialise it.
fp_status noalloc_setup(NoAllocDevice** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocDevice& d = g_noalloc[dev];
    if (!d.ready) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        e = cudaMemset(ptr, 0, kNoAllocScratchBytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(scratch)");
        const unsigned one = 1;   // launch tag 0 means "never written"
        e = cudaMemcpy(static_cast<char*>(ptr) + offsetof(WsHeader, epoch), &one, sizeof(one),
                       cudaMemcpyHostToDevice);
        // complete before any stream (blocking or not) launches on the array
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(scratch epoch)");
        d.ptr = ptr;
        d.ready = true;
    }
    *out = &d;
    return FP_OK;
}

}  // namespace

extern "C" fp_status fp_decode_noalloc(fp_codec codec, const fp_dict* dict, const void* d_codes,
                                       uint64_t codes_bytes, const uint32_t* d_code_offsets, uint32_t n_strings,
                                       uint8_t* d_out_bytes, uint64_t out_capacity, uint32_t* d_out_offsets,
                                       uint32_t* d_status, fp_stream_t stream_) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    fp_status st = check_common(codec, dict, d_codes, codes_bytes, d_code_offsets, d_out_bytes, out_capacity,
                                d_out_offsets, true);
    if (st != FP_OK) return st;
    if (!d_status || reinterpret_cast<uintptr_t>(d_status) % 4) return fail(FP_ERR_ARG, "d_status must be a 4-byte aligned device pointer");
    if (n_strings == 0xffffffffu) return fail(FP_ERR_ARG, "n_strings must be below 2^32-1");
    const uint64_t max_slots = max_slots_of(codec, codes_bytes);
    // Unless a variant was selected, the block pipeline: its scratch (12 bytes
    // per 4,096-slot tile) covers far larger inputs than warp tiles' (20 bytes
    // per 512-slot tile).
    const int sel = g_selected[codec].load();
    const Variant* var = variant_get(codec, sel >= 0 ? sel : noalloc_default(codec));
    if (!var) return fail(FP_ERR_ARG, "no decode variant for codec %d", (int)codec);
    const uint64_t tile = variant_tile(*var);
    const uint64_t n_tiles = max_slots / tile + 2;
    const size_t need = variant_scratch_bytes(*var, max_slots);
    const size_t room = kNoAllocScratchBytes - kWsHeaderBytes;
    if (need > room) {
        // the largest buffer that fits, for the message
        uint64_t lo = 0, hi = max_slots;
        while (lo < hi) {
            const uint64_t mid = lo + (hi - lo + 1) / 2;
            if (variant_scratch_bytes(*var, mid) <= room) lo = mid; else hi = mid - 1;
        }
        return fail(FP_ERR_ARG,
                    "fp_decode_noalloc: a code buffer of %llu slots needs %llu scratch bytes; the fixed scratch holds "
                    "%llu (at most %llu slots with this variant); use fp_decode",
                    (unsigned long long)max_slots, (unsigned long long)need, (unsigned long long)room,
                    (unsigned long long)lo);
    }
    int per_wave = 0, sms = 0;
    st = grid_for(*var, &per_wave, &sms);
    if (st != FP_OK) return st;
    NoAllocDevice* nd = nullptr;
    st = noalloc_setup(&nd);
    if (st != FP_OK) return st;
    char* base = static_cast<char*>(nd->ptr);
    cudaError_t e;
    uint64_t launch_no;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);   // callers on several host threads share the count
        launch_no = ++nd->launches;
    }
    if ((launch_no & ((1ull << 25) - 1)) == 0) {
        // tile status words carry a 26-bit launch tag; clear them well before it wraps
        e = cudaMemsetAsync(base + kWsHeaderBytes, 0, room, stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(scratch)");
    }
    DecodeParams p{};
    p.dict = dict->view();
    p.codes = static_cast<const uint8_t*>(d_codes);
    p.codes_bytes = codes_bytes;
    p.max_slots = max_slots;
    p.code_offsets = d_code_offsets;
    p.n_strings = n_strings;
    p.out = d_out_bytes;
    p.capacity = out_capacity;
    p.out_offsets = d_out_offsets;
    p.ws = reinterpret_cast<WsHeader*>(base);
    p.size_only = 0;
    const uint64_t grid = (n_tiles < (uint64_t)per_wave && !var->warp_tiles) ? n_tiles : (uint64_t)per_wave;
    e = launch_decode(codec, *var, p, base + kWsHeaderBytes, max_slots, (int)grid, sms, stream);
    if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    // hand the call's data-error bits to the caller and clear them for the next call
    e = cudaMemcpyAsync(d_status, base + offsetof(WsHeader, status), sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                        stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + offsetof(WsHeader, status), 0, sizeof(uint32_t), stream);
    if (e != cudaSuccess) return cuda_fail(e, "status copy");
    return FP_OK;
}
