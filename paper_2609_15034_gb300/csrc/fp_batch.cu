// Batched decode: many column chunks (mixed codecs, one dictionary each) in
// one persistent launch, replayed from a CUDA graph.
//
// Work queue.  Chunks are grouped by codec into three queues; a queue's
// tickets run over the tiles of all its chunks (chunk after chunk), and a
// table maps a ticket to its chunk.  Every block runs the decode pipeline of
// fp_decoder.cuh on one queue until it is exhausted, then moves on to the
// next queue, so a block never idles while any queue has tiles.  Blocks are
// spread over the queues in proportion to their code slots at the start.
//
// Per-chunk state.  A chunk's code buffer is tiled whole (tile u = slots
// [u*T, (u+1)*T)); each chunk has its own look-back words, tile -> string
// index, data-error word and decoded size.  The decode block copies the
// chunk's record (SlotSrc) into its ring slot with the tile's inputs, so
// consecutive tiles of one block may belong to different chunks and codecs.
// Dictionaries are read through the L1 cache (a per-chunk copy into shared
// memory would have to be repeated at every chunk change).
//
// Autotuning.  The tile shape (code slots per thread for each codec) and
// the blocks per SM are compiled or launch-time choices; fp_plan_create
// times each candidate on the plan's own chunks and keeps the fastest,
// optionally remembering the choice in a text file keyed by a signature of
// the plan's size mix.  The chosen index pass + decode kernel are then
// captured into a CUDA graph, which fp_decode_batch replays.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fp_decoder.cuh"

namespace fp {
namespace {

constexpr u32 kIdxPerBlock = 2048;   // string boundaries per index block (256 threads x 8)

struct IdxBlock {
    u32 q_ci;    // queue in bits 30..31, chunk index within the queue below
    u32 start;   // first boundary of the block
};

struct IdxParams {
    const IdxBlock* blocks;
    SlotSrc* src[3];
    u32 tile[3];
};

// Index pass of a batch: each block handles up to kIdxPerBlock boundaries of
// one chunk; the chunk's first block also stores its slot range.
__global__ void __launch_bounds__(256) batch_index_kernel(const IdxParams ip) {
    const IdxBlock b = ip.blocks[blockIdx.x];
    const u32 q = b.q_ci >> 30, ci = b.q_ci & 0x3fffffffu;
    SlotSrc* cs = ip.src[q] + ci;
    const DecodeParams p = cs->p;
    Extent x;
    x.first_tile = 0;
    x.n_tiles = cs->x.n_tiles;
    slot_range(p, x);
    if (b.start == 0 && threadIdx.x == 0) {
        cs->x.c_begin = x.c_begin;
        cs->x.c_end = x.c_end;
        cs->x.bad = x.bad;
    }
    index_strings(p, x, ip.tile[q], (u64)b.start + threadIdx.x, (u64)b.start + kIdxPerBlock, 256,
                  const_cast<u32*>(p.first));
}

template <int K16, int K12, int K8, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) batch_kernel(const BatchParams bp) {
    const u32 epoch = *(volatile u32*)&bp.ws->epoch;
    const int q0 = blockIdx.x < bp.split[0] ? 0 : (blockIdx.x < bp.split[1] ? 1 : 2);
    bool reinit = false;
    for (int i = 0; i < 3; ++i) {
        const int q = (q0 + i) % 3;
        if (bp.q[q].n_tiles == 0) continue;
        if (q == 0) Decoder<FP_ONPAIR16, K16, false, MINB, true>::run_queue(bp, 0, epoch, reinit);
        else if (q == 1) Decoder<FP_ONPAIR12, K12, false, MINB, true>::run_queue(bp, 1, epoch, reinit);
        else Decoder<FP_FSST8, K8, false, MINB, true>::run_queue(bp, 2, epoch, reinit);
        reinit = true;
    }
    finish_launch(bp.ws, epoch);
}

struct BatchKernel {
    int k[3];            // code slots per thread: OnPair-16, OnPair-12, FSST-8
    int minb;            // blocks per SM the registers are budgeted for
    size_t smem_bytes;   // max over the three pipelines
    const void* kernel;
};

template <int K16, int K12, int K8, int MINB>
BatchKernel make_batch_kernel() {
    const size_t a = sizeof(typename Decoder<FP_ONPAIR16, K16, false, MINB, true>::S);
    const size_t b = sizeof(typename Decoder<FP_ONPAIR12, K12, false, MINB, true>::S);
    const size_t c = sizeof(typename Decoder<FP_FSST8, K8, false, MINB, true>::S);
    return BatchKernel{{K16, K12, K8}, MINB, std::max(a, std::max(b, c)),
                       (const void*)&batch_kernel<K16, K12, K8, MINB>};
}

const std::vector<BatchKernel>& batch_kernels() {
    static const std::vector<BatchKernel> v = {
        make_batch_kernel<16, 16, 16, 2>(),
        make_batch_kernel<8, 8, 16, 2>(),
    };
    return v;
}

// A candidate configuration: a compiled kernel and a launch width.
struct Config {
    int kernel;   // index into batch_kernels()
    int bps;      // blocks per SM launched (<= what fits)
};
const std::vector<Config>& configs() {
    static const std::vector<Config> v = {{0, 2}, {0, 1}, {1, 2}};
    return v;
}

}  // namespace
}  // namespace fp

using namespace fp;

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct fp_plan {
    int device = 0;
    int sms = 0;
    std::vector<fp_chunk> chunks;
    // plan-wide device memory: WsHeader | chunk status (u32 x n) | chunk totals (u64 x n)
    void* d_hdr = nullptr;
    uint32_t* d_status = nullptr;
    unsigned long long* d_total = nullptr;
    // layout of the chosen configuration
    int config = -1;
    void* d_layout = nullptr;
    size_t layout_bytes = 0;
    uint64_t total_tiles = 0;
    uint32_t n_idx_blocks = 0;
    int grid = 0;
    BatchParams bp{};
    IdxParams ip{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t launches = 0;
    unsigned long long* d_tile_status = nullptr;
    std::vector<float> tune_ms;   // per configuration, -1 = not timed
    bool from_cache = false;
};

namespace {

// Lay out the device tables of configuration `cfg` and fill the launch
// parameters; replaces the plan's previous layout.
fp_status build_layout(fp_plan* P, int cfg) {
    const Config& C = configs()[cfg];
    const BatchKernel& BK = batch_kernels()[C.kernel];
    const uint32_t n = (uint32_t)P->chunks.size();
    std::vector<uint32_t> qlist[3];
    for (uint32_t i = 0; i < n; ++i) qlist[P->chunks[i].codec - 1].push_back(i);

    std::vector<SlotSrc> src[3];
    std::vector<uint32_t> tchunk[3];
    std::vector<IdxBlock> iblk;
    uint64_t tile_glob = 0, first_glob = 0;
    uint64_t slots_q[3] = {0, 0, 0};
    for (int q = 0; q < 3; ++q) {
        const int codec = q + 1;
        const uint64_t T = (uint64_t)kWork * (uint64_t)BK.k[q];
        uint32_t tile_q = 0;
        for (uint32_t ci = 0; ci < qlist[q].size(); ++ci) {
            const uint32_t i = qlist[q][ci];
            const fp_chunk& c = P->chunks[i];
            const uint64_t ms = max_slots_of(codec, c.codes_bytes);
            uint64_t nt = (ms + T - 1) / T;
            if (nt == 0) nt = 1;
            if ((uint64_t)tile_q + nt > 0x7fffffffull) return fail(FP_ERR_ARG, "batch has too many tiles for one codec");
            slots_q[q] += ms;
            SlotSrc s;
            memset(&s, 0, sizeof(s));
            s.p.dict = c.dict->view();
            s.p.codes = static_cast<const uint8_t*>(c.d_codes);
            s.p.codes_bytes = c.codes_bytes;
            s.p.max_slots = ms;
            s.p.code_offsets = c.d_code_offsets;
            s.p.n_strings = c.n_strings;
            s.p.out = c.d_out_bytes;
            s.p.capacity = c.out_capacity;
            s.p.out_offsets = c.d_out_offsets;
            s.p.size_only = 0;
            // device pointers are filled in below, relative to the layout base
            s.p.tile_status = reinterpret_cast<unsigned long long*>((uintptr_t)tile_glob);
            s.p.first = reinterpret_cast<const uint32_t*>((uintptr_t)first_glob);
            s.p.err_word = P->d_status + i;
            s.p.total_out = P->d_total + i;
            s.p.ws = static_cast<WsHeader*>(P->d_hdr);
            s.x.first_tile = 0;
            s.x.n_tiles = nt;
            s.tile_base = tile_q;
            s.chunk = i;
            src[q].push_back(s);
            for (uint64_t u = 0; u < nt; ++u) tchunk[q].push_back(ci);
            const uint64_t nb = (uint64_t)c.n_strings + 1;
            for (uint64_t st = 0; st < nb; st += kIdxPerBlock)
                iblk.push_back(IdxBlock{((uint32_t)q << 30) | ci, (uint32_t)st});
            tile_q += (uint32_t)nt;
            tile_glob += nt;
            first_glob += nt + 1;
        }
    }
    if (iblk.size() > 0x7fffffffull) return fail(FP_ERR_ARG, "batch has too many strings");

    // device layout: src[0..2] | tile_chunk[0..2] | idx blocks | first | tile status
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0, o_src[3], o_tc[3];
    for (int q = 0; q < 3; ++q) { o_src[q] = off; off = al(off + src[q].size() * sizeof(SlotSrc)); }
    for (int q = 0; q < 3; ++q) { o_tc[q] = off; off = al(off + tchunk[q].size() * sizeof(uint32_t)); }
    const size_t o_ib = off; off = al(off + iblk.size() * sizeof(IdxBlock));
    const size_t o_first = off; off = al(off + first_glob * sizeof(uint32_t));
    const size_t o_ts = off; off = al(off + tile_glob * sizeof(unsigned long long));
    const size_t bytes = off;

    if (P->d_layout) {
        cudaFree(P->d_layout);
        P->d_layout = nullptr;
    }
    cudaError_t e = cudaMalloc(&P->d_layout, bytes);
    if (e != cudaSuccess) { P->d_layout = nullptr; return cuda_fail(e, "cudaMalloc(batch layout)"); }
    char* base = static_cast<char*>(P->d_layout);
    for (int q = 0; q < 3; ++q)
        for (SlotSrc& s : src[q]) {
            s.p.tile_status = reinterpret_cast<unsigned long long*>(base + o_ts) + (uintptr_t)s.p.tile_status;
            s.p.first = reinterpret_cast<const uint32_t*>(base + o_first) + (uintptr_t)s.p.first;
        }
    std::vector<char> host(bytes, 0);
    for (int q = 0; q < 3; ++q) {
        if (!src[q].empty()) memcpy(&host[o_src[q]], src[q].data(), src[q].size() * sizeof(SlotSrc));
        if (!tchunk[q].empty()) memcpy(&host[o_tc[q]], tchunk[q].data(), tchunk[q].size() * sizeof(uint32_t));
    }
    memcpy(&host[o_ib], iblk.data(), iblk.size() * sizeof(IdxBlock));
    e = cudaMemcpy(base, host.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(batch layout)");

    // launch width: blocks that fit, at most the configuration's per-SM count
    e = cudaFuncSetAttribute(BK.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BK.smem_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(batch)");
    int fit = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, BK.kernel, kThreads, BK.smem_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(batch)");
    if (fit < 1) return fail(FP_ERR_CUDA, "batch kernel does not fit on an SM");
    const int bps = std::min(fit, C.bps);
    uint64_t grid = (uint64_t)bps * (uint64_t)P->sms;
    if (grid > tile_glob) grid = tile_glob;
    if (grid < 1) grid = 1;

    BatchParams bp;
    memset(&bp, 0, sizeof(bp));
    bp.ws = static_cast<WsHeader*>(P->d_hdr);
    for (int q = 0; q < 3; ++q) {
        bp.q[q].src = reinterpret_cast<const SlotSrc*>(base + o_src[q]);
        bp.q[q].tile_chunk = reinterpret_cast<const uint32_t*>(base + o_tc[q]);
        bp.q[q].n_tiles = (uint32_t)tchunk[q].size();
        bp.q[q].n_chunks = (uint32_t)src[q].size();
    }
    // starting queues in proportion to code slots (at least one block per non-empty queue)
    const double tot = (double)(slots_q[0] + slots_q[1] + slots_q[2]) + 1e-9;
    uint32_t g[3];
    uint32_t left = (uint32_t)grid;
    for (int q = 0; q < 3; ++q) {
        g[q] = bp.q[q].n_tiles ? (uint32_t)std::floor((double)grid * (double)slots_q[q] / tot) : 0u;
        if (bp.q[q].n_tiles && g[q] == 0) g[q] = 1;
    }
    while (g[0] + g[1] + g[2] > left) {
        int m = 0;
        for (int q = 1; q < 3; ++q) if (g[q] > g[m]) m = q;
        --g[m];
    }
    g[2] = left - g[0] - g[1];
    bp.split[0] = g[0];
    bp.split[1] = g[0] + g[1];

    IdxParams ip;
    memset(&ip, 0, sizeof(ip));
    ip.blocks = reinterpret_cast<const IdxBlock*>(base + o_ib);
    for (int q = 0; q < 3; ++q) {
        ip.src[q] = reinterpret_cast<SlotSrc*>(base + o_src[q]);
        ip.tile[q] = (u32)(kWork * BK.k[q]);
    }
    P->config = cfg;
    P->layout_bytes = bytes;
    P->total_tiles = tile_glob;
    P->n_idx_blocks = (uint32_t)iblk.size();
    P->grid = (int)grid;
    P->bp = bp;
    P->ip = ip;
    P->d_tile_status = reinterpret_cast<unsigned long long*>(base + o_ts);
    return FP_OK;
}

cudaError_t launch_batch(const fp_plan* P, cudaStream_t stream) {
    const BatchKernel& BK = batch_kernels()[configs()[P->config].kernel];
    void* iargs[] = {(void*)&P->ip};
    cudaError_t e = cudaLaunchKernel((const void*)&batch_index_kernel, dim3(P->n_idx_blocks), dim3(256), iargs, 0,
                                     stream);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&P->bp};
    return cudaLaunchKernel(BK.kernel, dim3(P->grid), dim3(kThreads), args, BK.smem_bytes, stream);
}

// Signature of a plan's size mix for the tuning cache: the number of SMs and
// the multiset of (codec, half-octave of code slots).
std::string plan_signature(const fp_plan* P) {
    std::vector<uint32_t> keys;
    keys.reserve(P->chunks.size());
    for (const fp_chunk& c : P->chunks) {
        const double ms = (double)max_slots_of(c.codec, c.codes_bytes);
        keys.push_back(((uint32_t)c.codec << 8) | (uint32_t)std::floor(2.0 * std::log2(ms + 1.0)));
    }
    std::sort(keys.begin(), keys.end());
    uint64_t h = 1469598103934665603ull;   // FNV-1a, 64-bit
    auto mix = [&](uint32_t v) {
        for (int b = 0; b < 4; ++b) {
            h ^= (v >> (8 * b)) & 0xffu;
            h *= 1099511628211ull;
        }
    };
    mix((uint32_t)P->sms);
    for (uint32_t k : keys) mix(k);
    char buf[64];
    snprintf(buf, sizeof(buf), "b1-%016llx-%zu", (unsigned long long)h, P->chunks.size());
    return buf;
}

int cache_lookup(const char* path, const std::string& sig) {
    if (!path) return -1;
    FILE* f = fopen(path, "r");
    if (!f) return -1;
    char key[128];
    int cfg = -1, found = -1;
    while (fscanf(f, "%127s %d", key, &cfg) == 2)
        if (sig == key && cfg >= 0 && cfg < (int)configs().size()) found = cfg;
    fclose(f);
    return found;
}

void cache_store(const char* path, const std::string& sig, int cfg) {
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d\n", sig.c_str(), cfg);
    fclose(f);
}

void plan_release(fp_plan* P) {
    if (!P) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(P->device);
    cudaDeviceSynchronize();
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    if (P->d_layout) cudaFree(P->d_layout);
    if (P->d_hdr) cudaFree(P->d_hdr);
    cudaSetDevice(prev);
    delete P;
}

fp_status plan_create(const fp_chunk* chunks, uint32_t n, int force_cfg, const char* cache_path,
                      cudaStream_t stream, fp_plan** out) {
    if (!out) return fail(FP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!chunks || n == 0) return fail(FP_ERR_ARG, "a plan needs at least one chunk");
    if (n > (1u << 30)) return fail(FP_ERR_ARG, "too many chunks");
    for (uint32_t i = 0; i < n; ++i) {
        const fp_chunk& c = chunks[i];
        fp_status st = check_common(c.codec, c.dict, c.d_codes, c.codes_bytes, c.d_code_offsets, c.d_out_bytes,
                                    c.out_capacity, c.d_out_offsets, true);
        if (st != FP_OK) return fail(st, "chunk %u: %s", i, fp_last_error());
        if (c.n_strings == 0xffffffffu) return fail(FP_ERR_ARG, "chunk %u: n_strings must be below 2^32-1", i);
    }
    fp_plan* P = new fp_plan();
    P->chunks.assign(chunks, chunks + n);
    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P->sms, cudaDevAttrMultiProcessorCount, P->device);
    const size_t o_status = kWsHeaderBytes;
    const size_t o_total = (o_status + n * sizeof(uint32_t) + 7) & ~(size_t)7;
    const size_t hdr_bytes = o_total + (size_t)n * sizeof(unsigned long long);
    if (e == cudaSuccess) e = cudaMalloc(&P->d_hdr, hdr_bytes);
    if (e == cudaSuccess) e = cudaMemset(P->d_hdr, 0, hdr_bytes);
    if (e == cudaSuccess) {
        const unsigned one = 1;   // launch tag 0 means "never written"
        e = cudaMemcpy(static_cast<char*>(P->d_hdr) + offsetof(WsHeader, epoch), &one, sizeof(one),
                       cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        plan_release(P);
        return cuda_fail(e, "plan header");
    }
    P->d_status = reinterpret_cast<uint32_t*>(static_cast<char*>(P->d_hdr) + o_status);
    P->d_total = reinterpret_cast<unsigned long long*>(static_cast<char*>(P->d_hdr) + o_total);
    P->tune_ms.assign(configs().size(), -1.0f);

    int cfg = force_cfg;
    const std::string sig = plan_signature(P);
    if (cfg < 0) {
        cfg = cache_lookup(cache_path, sig);
        P->from_cache = cfg >= 0;
    }
    fp_status st = FP_OK;
    if (cfg < 0) {
        // time every configuration on the plan's own chunks: one warm-up run, then the best of two
        cudaEvent_t a = nullptr, b = nullptr;
        e = cudaEventCreate(&a);
        if (e == cudaSuccess) e = cudaEventCreate(&b);
        float best = 0.0f;
        for (int c = 0; c < (int)configs().size() && e == cudaSuccess && st == FP_OK; ++c) {
            st = build_layout(P, c);
            if (st != FP_OK) break;
            e = launch_batch(P, stream);
            float ms_best = -1.0f;
            for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
                e = cudaEventRecord(a, stream);
                if (e == cudaSuccess) e = launch_batch(P, stream);
                if (e == cudaSuccess) e = cudaEventRecord(b, stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(b);
                float ms = 0.0f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
                if (e == cudaSuccess && (ms_best < 0.0f || ms < ms_best)) ms_best = ms;
            }
            P->tune_ms[c] = ms_best;
            if (e == cudaSuccess && (cfg < 0 || ms_best < best)) {
                best = ms_best;
                cfg = c;
            }
        }
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        if (e != cudaSuccess) st = cuda_fail(e, "batch tuning run");
        if (st == FP_OK) {
            // the tuning runs may have recorded data errors: start the plan clean
            e = cudaMemset(P->d_status, 0, n * sizeof(uint32_t));
            if (e == cudaSuccess)
                e = cudaMemset(static_cast<char*>(P->d_hdr) + offsetof(WsHeader, status), 0, sizeof(unsigned));
            if (e != cudaSuccess) st = cuda_fail(e, "plan reset");
        }
        if (st == FP_OK) cache_store(cache_path, sig, cfg);
    }
    if (st == FP_OK && (cfg < 0 || cfg >= (int)configs().size()))
        st = fail(FP_ERR_ARG, "batch configuration %d out of range", cfg);
    // a fresh layout starts with zeroed look-back words
    if (st == FP_OK && P->config != cfg) st = build_layout(P, cfg);
    if (st == FP_OK) {
        // capture the index pass and the decode kernel into a graph
        cudaStream_t cap = nullptr;
        e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t el = launch_batch(P, cap);
            e = cudaStreamEndCapture(cap, &P->graph);
            if (e == cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&P->exec, P->graph, 0);
        if (cap) cudaStreamDestroy(cap);
        if (e != cudaSuccess) st = cuda_fail(e, "batch graph capture");
    }
    if (st != FP_OK) {
        const std::string msg = fp_last_error();
        plan_release(P);
        return fail(st, "%s", msg.c_str());
    }
    *out = P;
    return FP_OK;
}

}  // namespace

extern "C" {

fp_status fp_plan_create(const fp_chunk* chunks, uint32_t n_chunks, const char* tune_cache_path,
                         fp_stream_t stream, fp_plan** out) {
    return plan_create(chunks, n_chunks, -1, tune_cache_path, reinterpret_cast<cudaStream_t>(stream), out);
}

fp_status fp_plan_create_config(const fp_chunk* chunks, uint32_t n_chunks, int config, fp_stream_t stream,
                                fp_plan** out) {
    if (config < 0 || config >= (int)configs().size())
        return fail(FP_ERR_ARG, "batch configuration %d out of range 0..%d", config, (int)configs().size() - 1);
    return plan_create(chunks, n_chunks, config, nullptr, reinterpret_cast<cudaStream_t>(stream), out);
}

fp_status fp_decode_batch(fp_plan* plan, fp_stream_t stream_) {
    if (!plan) return fail(FP_ERR_ARG, "plan is NULL");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device)
        return fail(FP_ERR_ARG, "plan lives on device %d, current device is %d", plan->device, dev);
    cudaError_t e;
    if ((++plan->launches & ((1ull << 25) - 1)) == 0) {
        // look-back words carry a 26-bit launch tag; clear them well before it wraps
        e = cudaMemsetAsync(plan->d_tile_status, 0, plan->total_tiles * sizeof(unsigned long long), stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(batch status)");
    }
    e = cudaGraphLaunch(plan->exec, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch(batch)");
    return FP_OK;
}

fp_status fp_plan_sync_status(fp_plan* plan, fp_stream_t stream_, uint32_t* h_chunk_status,
                              uint64_t* h_chunk_total) {
    if (!plan) return fail(FP_ERR_ARG, "plan is NULL");
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    const uint32_t n = (uint32_t)plan->chunks.size();
    std::vector<uint32_t> bits(n);
    WsHeader h;
    e = cudaMemcpy(&h, plan->d_hdr, sizeof(h), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(bits.data(), plan->d_status, n * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h_chunk_total)
        e = cudaMemcpy(h_chunk_total, plan->d_total, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(plan->d_status, 0, n * sizeof(uint32_t));
    if (e == cudaSuccess && h.status)
        e = cudaMemset(static_cast<char*>(plan->d_hdr) + offsetof(WsHeader, status), 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "plan status");
    uint32_t all = h.status;
    uint32_t first_bad = n;
    for (uint32_t i = 0; i < n; ++i) {
        const uint32_t b = bits[i] | (h.status & ERRB_TIMEOUT);
        if (h_chunk_status) h_chunk_status[i] = (uint32_t)status_code(b);
        if (b && first_bad == n) first_bad = i;
        all |= b;
    }
    fp_status st = status_from_bits(all);
    if (st != FP_OK && first_bad < n) return fail(st, "%s (first failing chunk: %u)", fp_last_error(), first_bad);
    return st;
}

fp_status fp_plan_info(const fp_plan* plan, fp_plan_info_t* info) {
    if (!plan || !info) return fail(FP_ERR_ARG, "plan/info is NULL");
    const Config& C = configs()[plan->config];
    const BatchKernel& BK = batch_kernels()[C.kernel];
    memset(info, 0, sizeof(*info));
    info->config = (uint32_t)plan->config;
    for (int q = 0; q < 3; ++q) info->slots_per_thread[q] = (uint32_t)BK.k[q];
    info->threads = (uint32_t)kThreads;
    info->grid = (uint32_t)plan->grid;
    info->total_tiles = plan->total_tiles;
    info->index_blocks = plan->n_idx_blocks;
    info->layout_bytes = plan->layout_bytes;
    info->from_cache = plan->from_cache ? 1u : 0u;
    const size_t nc = std::min(configs().size(), sizeof(info->tune_ms) / sizeof(info->tune_ms[0]));
    for (size_t c = 0; c < nc; ++c) info->tune_ms[c] = plan->tune_ms[c];
    info->n_configs = (uint32_t)configs().size();
    return FP_OK;
}

fp_status fp_plan_destroy(fp_plan* plan) {
    plan_release(plan);
    return FP_OK;
}

int fp_batch_config_count(void) { return (int)configs().size(); }

fp_status fp_batch_config_info(int config, uint32_t* slots_per_thread3, uint32_t* blocks_per_sm) {
    if (config < 0 || config >= (int)configs().size()) return fail(FP_ERR_ARG, "batch configuration %d out of range", config);
    const Config& C = configs()[config];
    const BatchKernel& BK = batch_kernels()[C.kernel];
    if (slots_per_thread3)
        for (int q = 0; q < 3; ++q) slots_per_thread3[q] = (uint32_t)BK.k[q];
    if (blocks_per_sm) *blocks_per_sm = (uint32_t)C.bps;
    return FP_OK;
}

}  // extern "C"
