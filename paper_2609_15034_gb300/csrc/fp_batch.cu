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

#include "fp_warp.cuh"

namespace fp {
namespace {

constexpr u32 kIdxPerBlock = 256 * kIdxGroup;   // string boundaries per index block

struct IdxBlock {
    u32 q_ci;    // queue in bits 30..31, chunk index within the queue below
    u32 start;   // first boundary of the block
};

struct IdxParams {
    const IdxBlock* blocks;
    SlotSrc* src[kQueues];
    u32 tile[kQueues];
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
    index_groups(p, x, (u32)(__ffs((int)ip.tile[q]) - 1), b.start, (u64)b.start + kIdxPerBlock, threadIdx.x, 256,
                 const_cast<u32*>(p.first));
}

template <int K16, int K12, int K8, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) batch_kernel(const BatchParams bp) {
    const u32 epoch = *(volatile u32*)&bp.ws->epoch;
    const int q0 = blockIdx.x < bp.split[0] ? 0 : (blockIdx.x < bp.split[1] ? 1 : 2);
    for (int i = 0; i < kBlockQueues; ++i) {
        const int q = (q0 + i) % kBlockQueues;
        if (bp.q[q].n_tiles == 0) continue;
        if (q == 0) Decoder<FP_ONPAIR16, K16, false, MINB, true>::run_queue(bp, 0, epoch);
        else if (q == 1) Decoder<FP_ONPAIR12, K12, false, MINB, true>::run_queue(bp, 1, epoch);
        else Decoder<FP_FSST8, K8, false, MINB, true>::run_queue(bp, 2, epoch);
    }
    finish_launch(bp.ws, epoch);
}

// ---------------------------------------------------------------------------
// Warp-tile batches: index pass, reduce, tile scan and a persistent decode,
// every chunk in warp tiles of 32*K slots (K per codec).  Dictionaries are
// read through L1; each warp copies its current chunk's record into its own
// shared-memory slot.
// ---------------------------------------------------------------------------
template <int CODEC, int K>
__device__ __forceinline__ void reduce_queue(const BatchParams& bp, int q, u64 t, u64 t_end, u64 W) {
    typedef WarpCore<CODEC, K, false> C;
    const BatchQueue& Q = bp.q[q];
    const u32 lane = threadIdx.x & 31u;
    if (t >= t_end) return;
    // Software pipeline: the code words of tile t + W (its chunk record
    // already known) and the record of tile t + 2W are in flight while tile t
    // computes, so the chain ticket -> record -> codes -> lengths does not
    // stall the warp once per tile.
    const SlotSrc* rc = Q.src + __ldg(Q.tile_chunk + t);
    u64 q0 = C::lane_q0(rc->x, t - rc->tile_base);
    u32 wv[C::LANE_WORDS];
    bool fast = C::load_fast(rc->p, q0, wv);
    const SlotSrc* rn = t + W < t_end ? Q.src + __ldg(Q.tile_chunk + t + W) : nullptr;
    for (; t < t_end; t += W) {
        u32 nv[C::LANE_WORDS];
        bool nfast = false;
        u64 nq0 = 0;
        if (rn) {
            nq0 = C::lane_q0(rn->x, t + W - rn->tile_base);
            nfast = C::load_fast(rn->p, nq0, nv);
        }
        const SlotSrc* r2 = t + 2 * W < t_end ? Q.src + __ldg(Q.tile_chunk + t + 2 * W) : nullptr;
        const DecodeParams& p = rc->p;
        const Extent x = rc->x;
        typename C::R r;
        C::finish_load(p, x, q0, wv, fast, p.dict.lens, r);
        u32 err = 0;
        // every codec's element in the two-state form (OnPair: both states alike)
        const TElem e = C::tile_element(r, lane, err);
        if (lane == 31) bp.agg[rc->wt_base + (t - rc->tile_base)] = wt_pack<true>(e);
        if (err) atomicOr(p.err_word, err);
        rc = rn;
        rn = r2;
        q0 = nq0;
        fast = nfast;
#pragma unroll
        for (int i = 0; i < C::LANE_WORDS; ++i) wv[i] = nv[i];
    }
}

template <int K16, int K12, int K8>
__global__ void __launch_bounds__(256, 3) wbatch_reduce_kernel(const BatchParams bp) {
    // FSST-12 chunks run with the OnPair-12 slots per lane (both 12-bit codes)
    // Every block takes a contiguous range of each queue's tiles (its warps
    // interleaved inside it), so a block's warps mostly work in one chunk and
    // that chunk's length table stays in the SM's L1 (12 % faster than tiles
    // interleaved over the whole grid on the mixed 4,096-chunk batch).
    const u64 b = blockIdx.x, B = gridDim.x, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kQueues; ++q) {
        const u64 n = bp.q[q].n_tiles;
        const u64 lo = n * b / B, hi = n * (b + 1) / B;
        if (q == 0) reduce_queue<FP_ONPAIR16, K16>(bp, 0, lo + w, hi, 8);
        else if (q == 1) reduce_queue<FP_ONPAIR12, K12>(bp, 1, lo + w, hi, 8);
        else if (q == 2) reduce_queue<FP_FSST8, K8>(bp, 2, lo + w, hi, 8);
        else reduce_queue<FP_FSST12, K12>(bp, 3, lo + w, hi, 8);
    }
}

// Tile scan of every chunk: a ticket names one scan block of one chunk
// (blocks listed chunk after chunk); the look-back stays inside the chunk.
__global__ void __launch_bounds__(256) wbatch_scan_kernel(const BatchParams bp) {
    __shared__ ScanShared sh;
    WsHeader* ws = bp.ws;
    const u32 epoch = *(volatile u32*)&ws->epoch;
    for (;;) {
        if (threadIdx.x == 0) sh.ticket = atomicAdd(&ws->tile_counter, 1u);
        __syncthreads();
        const u32 i = sh.ticket;
        if (i >= bp.n_scan_blocks) break;
        const uint2 sb = __ldg(bp.scan_blocks + i);
        const SlotSrc* rec = bp.q[sb.x >> 30].src + (sb.x & 0x3fffffffu);
        scan_block<true>(rec->p, bp.agg + rec->wt_base, bp.ex + rec->wt_base, rec->x.n_tiles, sb.y, rec->n_sb,
                         rec->p.tile_status, epoch, ws, sh);
    }
    finish_launch(ws, epoch);
}

template <int CODEC, int K>
__device__ __forceinline__ void decode_queue(const BatchParams& bp, int q, u64 t, u64 t_end, u64 W,
                                             unsigned char* area_raw, SlotSrc& rs) {
    typedef WarpCore<CODEC, K, false> C;
    const BatchQueue& Q = bp.q[q];
    WarpArea<K>& area = *reinterpret_cast<WarpArea<K>*>(area_raw);
    const u32 lane = threadIdx.x & 31u;
    if (t >= t_end) return;
    // software pipeline as in the single-column decode: while tile t decodes,
    // the inputs of t + W are in flight and the boundaries of t + 2W are read
    const SlotSrc* rc = Q.src + __ldg(Q.tile_chunk + t);
    u32 lo, hi, lo1 = 0, hi1 = 0;
    C::bounds(rc->p, t - rc->tile_base, lo, hi);
    typename C::Fetch cur;
    C::fetch(rc->p, rc->x, bp.ex + rc->wt_base, t - rc->tile_base, lo, hi, cur);
    const SlotSrc* rn = nullptr;
    if (t + W < t_end) {
        rn = Q.src + __ldg(Q.tile_chunk + t + W);
        C::bounds(rn->p, t + W - rn->tile_base, lo1, hi1);
    }
    const SlotSrc* held = nullptr;   // the record copied into rs
    for (; t < t_end; t += W) {
        typename C::Fetch nxt;
        const u64 tn = t + W, t2 = t + 2 * W;
        const SlotSrc* r2 = nullptr;
        u32 lo2 = 0, hi2 = 0;
        if (tn < t_end) C::fetch(rn->p, rn->x, bp.ex + rn->wt_base, tn - rn->tile_base, lo1, hi1, nxt);
        if (t2 < t_end) {
            r2 = Q.src + __ldg(Q.tile_chunk + t2);
            C::bounds(r2->p, t2 - r2->tile_base, lo2, hi2);
        }
        if (rc != held) {
            // the chunk's record into the warp's slot (the previous tile is done with it)
            const uint4* g = reinterpret_cast<const uint4*>(rc);
            if (lane < sizeof(SlotSrc) / 16) reinterpret_cast<uint4*>(&rs)[lane] = g[lane];
            __syncwarp();
            held = rc;
        }
        u32 err = 0;
        // the error word's address is read before the tile: once the tile's
        // last __syncwarp() has passed, other lanes may overwrite the record
        unsigned* const err_word = rs.p.err_word;
        C::decode_tile(rs.p, rs.x, t - rs.tile_base, cur, bp.ex + rs.wt_base, nullptr, rs.p.dict.lens, area, err);
        if (err) atomicOr(err_word, err);
        cur = nxt;
        rc = rn;
        rn = r2;
        lo1 = lo2;
        hi1 = hi2;
    }
    __syncwarp();   // the record slot is reused by the next queue
}

template <int K>
struct WarpSlotBytes {
    static constexpr size_t v = sizeof(WarpArea<K>);
};

template <int K16, int K12, int K8, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) wbatch_decode_kernel(const BatchParams bp) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr size_t A = (WarpSlotBytes<K16>::v > WarpSlotBytes<K12>::v
                              ? (WarpSlotBytes<K16>::v > WarpSlotBytes<K8>::v ? WarpSlotBytes<K16>::v : WarpSlotBytes<K8>::v)
                              : (WarpSlotBytes<K12>::v > WarpSlotBytes<K8>::v ? WarpSlotBytes<K12>::v : WarpSlotBytes<K8>::v));
    constexpr size_t SLOT = (A + sizeof(SlotSrc) + 15) / 16 * 16;
    static_assert(A % 16 == 0, "per-warp areas keep 16-byte alignment");
    const u32 warp = threadIdx.x >> 5;
    unsigned char* mine = smem_raw + warp * SLOT;
    SlotSrc& rs = *reinterpret_cast<SlotSrc*>(mine + A);   // after the warp's scratch area
    // Warps take the tiles of each queue in turn, interleaved over the whole
    // grid (contiguous ranges per block were tried: 14 % slower, the blocks'
    // ranges end unevenly).
    const u64 gw = (u64)blockIdx.x * NW + warp, W = (u64)gridDim.x * NW;
    decode_queue<FP_ONPAIR16, K16>(bp, 0, gw, bp.q[0].n_tiles, W, mine, rs);
    decode_queue<FP_ONPAIR12, K12>(bp, 1, gw, bp.q[1].n_tiles, W, mine, rs);
    decode_queue<FP_FSST8, K8>(bp, 2, gw, bp.q[2].n_tiles, W, mine, rs);
    decode_queue<FP_FSST12, K12>(bp, 3, gw, bp.q[3].n_tiles, W, mine, rs);
}

template <int K16, int K12, int K8, int NW>
constexpr size_t wbatch_smem() {
    return (size_t)NW * (((WarpSlotBytes<K16>::v > WarpSlotBytes<K12>::v
                               ? (WarpSlotBytes<K16>::v > WarpSlotBytes<K8>::v ? WarpSlotBytes<K16>::v
                                                                              : WarpSlotBytes<K8>::v)
                               : (WarpSlotBytes<K12>::v > WarpSlotBytes<K8>::v ? WarpSlotBytes<K12>::v
                                                                              : WarpSlotBytes<K8>::v)) +
                          sizeof(SlotSrc) + 15) / 16 * 16);
}

struct BatchKernel {
    int k[kQueues];      // code slots per thread: OnPair-16, OnPair-12, FSST-8, FSST-12 (0: not served)
    int minb;            // blocks per SM the registers are budgeted for
    size_t smem_bytes;   // max over the three pipelines
    const void* kernel;  // the decode kernel
    int warp_tiles;      // 0: block pipeline; 1: warp tiles (reduce, scan, decode)
    int threads;         // threads per block of the decode kernel
    const void* reduce;
    const void* scan;
};

template <int K16, int K12, int K8, int MINB>
BatchKernel make_batch_kernel() {
    const size_t a = sizeof(typename Decoder<FP_ONPAIR16, K16, false, MINB, true>::S);
    const size_t b = sizeof(typename Decoder<FP_ONPAIR12, K12, false, MINB, true>::S);
    const size_t c = sizeof(typename Decoder<FP_FSST8, K8, false, MINB, true>::S);
    BatchKernel k{};
    k.k[0] = K16; k.k[1] = K12; k.k[2] = K8; k.k[3] = 0;   // no FSST-12 block pipeline
    k.minb = MINB;
    k.smem_bytes = std::max(a, std::max(b, c));
    k.kernel = (const void*)&batch_kernel<K16, K12, K8, MINB>;
    k.warp_tiles = 0;
    k.threads = kThreads;
    return k;
}

template <int K16, int K12, int K8, int NW, int MINB>
BatchKernel make_wbatch_kernel() {
    BatchKernel k{};
    k.k[0] = K16; k.k[1] = K12; k.k[2] = K8; k.k[3] = K12;
    k.minb = MINB;
    k.smem_bytes = wbatch_smem<K16, K12, K8, NW>();
    k.kernel = (const void*)&wbatch_decode_kernel<K16, K12, K8, NW, MINB>;
    k.warp_tiles = 1;
    k.threads = NW * 32;
    k.reduce = (const void*)&wbatch_reduce_kernel<K16, K12, K8>;
    k.scan = (const void*)&wbatch_scan_kernel;
    return k;
}

const std::vector<BatchKernel>& batch_kernels() {
    static const std::vector<BatchKernel> v = {
        make_batch_kernel<16, 16, 16, 2>(),
        make_batch_kernel<8, 8, 16, 2>(),
        make_wbatch_kernel<16, 16, 32, 8, 2>(),
        make_wbatch_kernel<16, 16, 32, 16, 1>(),
    };
    return v;
}

// A candidate configuration: a compiled kernel and a launch width.
struct Config {
    int kernel;   // index into batch_kernels()
    int bps;      // blocks per SM launched (<= what fits)
};
const std::vector<Config>& configs() {
    static const std::vector<Config> v = {{0, 2}, {0, 1}, {1, 2}, {2, 2}, {3, 1}};
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
    uint64_t status_words = 0;
    std::vector<float> tune_ms;   // per configuration, -1 = not timed
    bool from_cache = false;
};

namespace {

// Host image of a batch's device tables.  The device layout is
//   chunk records (per queue) | ticket -> chunk (per queue) | index blocks |
//   tile -> first string (per chunk) | look-back words (per tile);
// the image holds the first three parts (`table_bytes`); the index pass
// writes the fourth and the look-back words are tagged per launch.
struct LayoutImage {
    std::vector<char> bytes;
    size_t o_src[kQueues], o_tc[kQueues], o_ib, o_sb, o_first, o_ts, o_agg, o_ex, table_bytes, total_bytes;
    uint64_t total_tiles = 0;
    uint64_t status_words = 0;   // look-back words (per tile, or per tile-scan block with warp tiles)
    uint32_t n_idx = 0;
    uint32_t n_sb = 0;           // tile-scan blocks (warp tiles)
    uint32_t n_tiles_q[kQueues], n_chunks_q[kQueues];
    uint64_t slots_q[kQueues];
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Tables of `n` chunks for batch kernel BK.  Chunk i reports into
// d_status[i] / d_total[i].  Device addresses inside the records are
// offsets until relocate() adds the layout's base.
fp_status make_layout(const fp_chunk* chunks, uint32_t n, const BatchKernel& BK, uint32_t* d_status,
                      unsigned long long* d_total, WsHeader* ws, LayoutImage& L) {
    std::vector<uint32_t> qlist[kQueues];
    for (uint32_t i = 0; i < n; ++i) qlist[chunks[i].codec - 1].push_back(i);
    if (!qlist[3].empty() && BK.k[3] == 0)
        return fail(FP_ERR_ARG, "FSST-12 chunks need a warp-tile batch configuration");
    std::vector<SlotSrc> src[kQueues];
    std::vector<uint32_t> tchunk[kQueues];
    std::vector<IdxBlock> iblk;
    std::vector<uint2> sblk;
    uint64_t tile_glob = 0, first_glob = 0, sb_glob = 0;
    for (int q = 0; q < kQueues; ++q) {
        const int codec = q + 1;
        const uint64_t T = (uint64_t)(BK.warp_tiles ? 32 : kWork) * (uint64_t)BK.k[q];
        uint32_t tile_q = 0;
        L.slots_q[q] = 0;
        for (uint32_t ci = 0; ci < qlist[q].size(); ++ci) {
            const uint32_t i = qlist[q][ci];
            const fp_chunk& c = chunks[i];
            const uint64_t ms = max_slots_of(codec, c.codes_bytes);
            uint64_t nt = (ms + T - 1) / T;
            if (nt == 0) nt = 1;
            if ((uint64_t)tile_q + nt > 0x7fffffffull) return fail(FP_ERR_ARG, "batch has too many tiles for one codec");
            L.slots_q[q] += ms;
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
            const uint64_t n_sb = BK.warp_tiles ? (nt + kScanTile - 1) / kScanTile : 0;
            // look-back words: one per tile (block pipeline) or per tile-scan block (warp tiles)
            s.p.tile_status = reinterpret_cast<unsigned long long*>((uintptr_t)(BK.warp_tiles ? sb_glob : tile_glob));
            s.p.first = reinterpret_cast<const uint32_t*>((uintptr_t)first_glob);
            s.p.err_word = d_status + i;
            s.p.total_out = d_total + i;
            s.p.ws = ws;
            s.x.first_tile = 0;
            s.x.n_tiles = nt;
            s.tile_base = tile_q;
            s.chunk = i;
            s.wt_base = tile_glob;
            s.sb_base = (uint32_t)sb_glob;
            s.n_sb = (uint32_t)n_sb;
            for (uint64_t b = 0; b < n_sb; ++b) sblk.push_back(make_uint2(((uint32_t)q << 30) | ci, (uint32_t)b));
            sb_glob += n_sb;
            src[q].push_back(s);
            tchunk[q].insert(tchunk[q].end(), nt, ci);
            const uint64_t nb = (uint64_t)c.n_strings + 1;
            for (uint64_t st = 0; st < nb; st += kIdxPerBlock)
                iblk.push_back(IdxBlock{((uint32_t)q << 30) | ci, (uint32_t)st});
            tile_q += (uint32_t)nt;
            tile_glob += nt;
            first_glob += nt + 1;
        }
        L.n_tiles_q[q] = tile_q;
        L.n_chunks_q[q] = (uint32_t)src[q].size();
    }
    if (iblk.size() > 0x7fffffffull) return fail(FP_ERR_ARG, "batch has too many strings");
    size_t off = 0;
    for (int q = 0; q < kQueues; ++q) { L.o_src[q] = off; off = align256(off + src[q].size() * sizeof(SlotSrc)); }
    for (int q = 0; q < kQueues; ++q) { L.o_tc[q] = off; off = align256(off + tchunk[q].size() * sizeof(uint32_t)); }
    L.o_ib = off; off = align256(off + iblk.size() * sizeof(IdxBlock));
    L.o_sb = off; off = align256(off + sblk.size() * sizeof(uint2));
    L.table_bytes = off;
    L.o_first = off; off = align256(off + first_glob * sizeof(uint32_t));
    L.status_words = BK.warp_tiles ? sb_glob : tile_glob;
    L.o_ts = off; off = align256(off + L.status_words * sizeof(unsigned long long));
    L.o_agg = off; off = align256(off + (BK.warp_tiles ? tile_glob : 0) * sizeof(unsigned long long));
    L.o_ex = off; off = align256(off + (BK.warp_tiles ? tile_glob : 0) * sizeof(unsigned long long));
    L.total_bytes = off;
    L.total_tiles = tile_glob;
    L.n_idx = (uint32_t)iblk.size();
    L.n_sb = (uint32_t)sblk.size();
    L.bytes.assign(L.table_bytes, 0);
    for (int q = 0; q < kQueues; ++q) {
        if (!src[q].empty()) memcpy(&L.bytes[L.o_src[q]], src[q].data(), src[q].size() * sizeof(SlotSrc));
        if (!tchunk[q].empty()) memcpy(&L.bytes[L.o_tc[q]], tchunk[q].data(), tchunk[q].size() * sizeof(uint32_t));
    }
    if (!iblk.empty()) memcpy(&L.bytes[L.o_ib], iblk.data(), iblk.size() * sizeof(IdxBlock));
    if (!sblk.empty()) memcpy(&L.bytes[L.o_sb], sblk.data(), sblk.size() * sizeof(uint2));
    return FP_OK;
}

// Turn the records' offsets into addresses of a layout placed at `base`.
void relocate(LayoutImage& L, char* base) {
    for (int q = 0; q < kQueues; ++q) {
        SlotSrc* s = reinterpret_cast<SlotSrc*>(&L.bytes[L.o_src[q]]);
        for (uint32_t c = 0; c < L.n_chunks_q[q]; ++c) {
            s[c].p.tile_status = reinterpret_cast<unsigned long long*>(base + L.o_ts) + (uintptr_t)s[c].p.tile_status;
            s[c].p.first = reinterpret_cast<const uint32_t*>(base + L.o_first) + (uintptr_t)s[c].p.first;
        }
    }
}

// Blocks of the persistent launch: those that fit, at most `bps` per SM,
// spread over the queues in proportion to their code slots.
fp_status launch_shape(const LayoutImage& L, const BatchKernel& BK, int bps_limit, int sms, int* grid_out,
                       uint32_t split[2]) {
    cudaError_t e = cudaFuncSetAttribute(BK.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BK.smem_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(batch)");
    int fit = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, BK.kernel, BK.threads, BK.smem_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor(batch)");
    if (fit < 1) return fail(FP_ERR_CUDA, "batch kernel does not fit on an SM");
    const int bps = std::min(fit, bps_limit);
    uint64_t grid = (uint64_t)bps * (uint64_t)sms;
    const uint64_t per_block = BK.warp_tiles ? (uint64_t)(BK.threads / 32) : 1;   // tiles a block takes at once
    if (grid > (L.total_tiles + per_block - 1) / per_block) grid = (L.total_tiles + per_block - 1) / per_block;
    if (grid < 1) grid = 1;
    const double tot = (double)(L.slots_q[0] + L.slots_q[1] + L.slots_q[2]) + 1e-9;   // block-pipeline queues
    uint32_t g[3];
    for (int q = 0; q < 3; ++q) {
        g[q] = L.n_tiles_q[q] ? (uint32_t)std::floor((double)grid * (double)L.slots_q[q] / tot) : 0u;
        if (L.n_tiles_q[q] && g[q] == 0) g[q] = 1;
    }
    while (g[0] + g[1] + g[2] > (uint32_t)grid) {
        int m = 0;
        for (int q = 1; q < 3; ++q) if (g[q] > g[m]) m = q;
        --g[m];
    }
    g[2] = (uint32_t)grid - g[0] - g[1];
    split[0] = g[0];
    split[1] = g[0] + g[1];
    *grid_out = (int)grid;
    return FP_OK;
}

void make_params(const LayoutImage& L, const BatchKernel& BK, char* base, WsHeader* ws, const uint32_t split[2],
                 BatchParams& bp, IdxParams& ip) {
    memset(&bp, 0, sizeof(bp));
    bp.ws = ws;
    for (int q = 0; q < kQueues; ++q) {
        bp.q[q].src = reinterpret_cast<const SlotSrc*>(base + L.o_src[q]);
        bp.q[q].tile_chunk = reinterpret_cast<const uint32_t*>(base + L.o_tc[q]);
        bp.q[q].n_tiles = L.n_tiles_q[q];
        bp.q[q].n_chunks = L.n_chunks_q[q];
    }
    bp.split[0] = split[0];
    bp.split[1] = split[1];
    if (BK.warp_tiles) {
        bp.agg = reinterpret_cast<unsigned long long*>(base + L.o_agg);
        bp.ex = reinterpret_cast<unsigned long long*>(base + L.o_ex);
        bp.scan_blocks = reinterpret_cast<const uint2*>(base + L.o_sb);
        bp.n_scan_blocks = L.n_sb;
    }
    memset(&ip, 0, sizeof(ip));
    ip.blocks = reinterpret_cast<const IdxBlock*>(base + L.o_ib);
    for (int q = 0; q < kQueues; ++q) {
        ip.src[q] = reinterpret_cast<SlotSrc*>(base + L.o_src[q]);
        ip.tile[q] = (u32)((BK.warp_tiles ? 32 : kWork) * (BK.k[q] ? BK.k[q] : 16));
    }
}

cudaError_t launch_kernels(const BatchKernel& BK, const BatchParams& bp, const IdxParams& ip, uint32_t n_idx, int grid,
                           int sms, cudaStream_t stream) {
    void* iargs[] = {(void*)&ip};
    cudaError_t e = cudaLaunchKernel((const void*)&batch_index_kernel, dim3(n_idx), dim3(256), iargs, 0, stream);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&bp};
    if (BK.warp_tiles) {
        e = cudaLaunchKernel(BK.reduce, dim3((unsigned)(sms * 3)), dim3(256), args, 0, stream);
        if (e != cudaSuccess) return e;
        uint32_t sg = bp.n_scan_blocks < (uint32_t)(sms * 2) ? bp.n_scan_blocks : (uint32_t)(sms * 2);
        if (sg < 1) sg = 1;
        e = cudaLaunchKernel(BK.scan, dim3(sg), dim3(256), args, 0, stream);
        if (e != cudaSuccess) return e;
    }
    return cudaLaunchKernel(BK.kernel, dim3(grid), dim3(BK.threads), args, BK.smem_bytes, stream);
}

// Lay out configuration `cfg` for a plan (fresh device memory, zeroed
// look-back words) and fill its launch parameters.
fp_status build_layout(fp_plan* P, int cfg) {
    const Config& C = configs()[cfg];
    const BatchKernel& BK = batch_kernels()[C.kernel];
    LayoutImage L;
    fp_status st = make_layout(P->chunks.data(), (uint32_t)P->chunks.size(), BK, P->d_status, P->d_total,
                               static_cast<WsHeader*>(P->d_hdr), L);
    if (st != FP_OK) return st;
    if (P->d_layout) {
        cudaFree(P->d_layout);
        P->d_layout = nullptr;
    }
    cudaError_t e = cudaMalloc(&P->d_layout, L.total_bytes);
    if (e != cudaSuccess) { P->d_layout = nullptr; return cuda_fail(e, "cudaMalloc(batch layout)"); }
    char* base = static_cast<char*>(P->d_layout);
    relocate(L, base);
    e = cudaMemcpy(base, L.bytes.data(), L.table_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(base + L.table_bytes, 0, L.total_bytes - L.table_bytes);
    // the legacy-stream memset must be complete before launches on any stream
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "batch layout upload");
    uint32_t split[2];
    int grid = 0;
    st = launch_shape(L, BK, C.bps, P->sms, &grid, split);
    if (st != FP_OK) return st;
    make_params(L, BK, base, static_cast<WsHeader*>(P->d_hdr), split, P->bp, P->ip);
    P->config = cfg;
    P->layout_bytes = L.total_bytes;
    P->total_tiles = L.total_tiles;
    P->n_idx_blocks = L.n_idx;
    P->grid = grid;
    P->d_tile_status = reinterpret_cast<unsigned long long*>(base + L.o_ts);
    P->status_words = L.status_words;
    return FP_OK;
}

cudaError_t launch_batch(const fp_plan* P, cudaStream_t stream) {
    const BatchKernel& BK = batch_kernels()[configs()[P->config].kernel];
    return launch_kernels(BK, P->bp, P->ip, P->n_idx_blocks, P->grid, P->sms, stream);
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
        bool has_fsst12 = false;
        for (const fp_chunk& c : P->chunks) has_fsst12 |= c.codec == FP_FSST12;
        for (int c = 0; c < (int)configs().size() && e == cudaSuccess && st == FP_OK; ++c) {
            if (has_fsst12 && batch_kernels()[configs()[c].kernel].k[3] == 0) continue;   // no FSST-12 queue
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
    // every initialisation above ran on the legacy stream or the tuning
    // stream: complete it before the plan is launched on any stream
    if (st == FP_OK) {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) st = cuda_fail(e, "plan creation");
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

namespace fp {

// Warp tiles (16/16/32 slots per lane, one block of 16 warps per SM): the
// fastest configuration on the mixed 4,096-chunk batch (41 ms, against 50 ms
// for two blocks of 8 warps and 55 ms for the block pipeline).
int batch_config_default() { return 4; }

fp_status wave_init(WaveBuffers& W, uint32_t cap_chunks) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&W.sms, cudaDevAttrMultiProcessorCount, dev);
    W.cap_chunks = cap_chunks;
    const size_t o_total = (kWsHeaderBytes + cap_chunks * sizeof(uint32_t) + 7) & ~(size_t)7;
    const size_t hdr = o_total + (size_t)cap_chunks * sizeof(unsigned long long);
    if (e == cudaSuccess) e = cudaMalloc(&W.d_hdr, hdr);
    if (e == cudaSuccess) e = cudaMemset(W.d_hdr, 0, hdr);
    if (e == cudaSuccess) {
        const unsigned one = 1;   // launch tag 0 means "never written"
        e = cudaMemcpy(static_cast<char*>(W.d_hdr) + offsetof(WsHeader, epoch), &one, sizeof(one),
                       cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&W.h_status), cap_chunks * sizeof(uint32_t) + 64, 0);
    if (e == cudaSuccess)
        e = cudaHostAlloc(reinterpret_cast<void**>(&W.h_total), cap_chunks * sizeof(unsigned long long), 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();   // initialised before any lane stream uses it
    if (e != cudaSuccess) {
        wave_free(W);
        return cuda_fail(e, "wave buffers");
    }
    W.h_ws_status = W.h_status + cap_chunks;
    W.d_status = reinterpret_cast<uint32_t*>(static_cast<char*>(W.d_hdr) + kWsHeaderBytes);
    W.d_total = reinterpret_cast<unsigned long long*>(static_cast<char*>(W.d_hdr) + o_total);
    return FP_OK;
}

void wave_free(WaveBuffers& W) {
    if (W.d_hdr) cudaFree(W.d_hdr);
    if (W.d_layout) cudaFree(W.d_layout);
    if (W.h_stage) cudaFreeHost(W.h_stage);
    if (W.h_status) cudaFreeHost(W.h_status);
    if (W.h_total) cudaFreeHost(W.h_total);
    W = WaveBuffers();
}

fp_status wave_launch(WaveBuffers& W, const fp_chunk* chunks, uint32_t n, int config, cudaStream_t stream) {
    if (n == 0 || n > W.cap_chunks) return fail(FP_ERR_ARG, "wave of %u chunks (capacity %u)", n, W.cap_chunks);
    const Config& C = configs()[config];
    const BatchKernel& BK = batch_kernels()[C.kernel];
    LayoutImage L;
    WsHeader* ws = static_cast<WsHeader*>(W.d_hdr);
    fp_status st = make_layout(chunks, n, BK, W.d_status, W.d_total, ws, L);
    if (st != FP_OK) return st;
    cudaError_t e;
    if (L.total_bytes > W.layout_cap) {
        // grow (the only allocation of a wave; stream-ordered frees would race the previous wave)
        e = cudaStreamSynchronize(stream);
        if (e == cudaSuccess && W.d_layout) e = cudaFree(W.d_layout);
        W.d_layout = nullptr;
        W.layout_cap = 0;
        size_t cap = 1u << 20;
        while (cap < L.total_bytes) cap *= 2;
        if (e == cudaSuccess) e = cudaMalloc(&W.d_layout, cap);
        if (e == cudaSuccess) e = cudaMemsetAsync(W.d_layout, 0, cap, stream);   // ordered before the upload
        if (e != cudaSuccess) { W.d_layout = nullptr; return cuda_fail(e, "wave layout"); }
        W.layout_cap = cap;
    }
    if (L.table_bytes > W.stage_cap) {
        if (W.h_stage) cudaFreeHost(W.h_stage);
        W.h_stage = nullptr;
        W.stage_cap = 0;
        size_t cap = 1u << 16;
        while (cap < L.table_bytes) cap *= 2;
        e = cudaHostAlloc(&W.h_stage, cap, 0);
        if (e != cudaSuccess) { W.h_stage = nullptr; return cuda_fail(e, "wave staging"); }
        W.stage_cap = cap;
    }
    char* base = static_cast<char*>(W.d_layout);
    relocate(L, base);
    memcpy(W.h_stage, L.bytes.data(), L.table_bytes);
    if ((++W.launches & ((1ull << 25) - 1)) == 0) {
        // look-back words carry a 26-bit launch tag; clear them well before it wraps
        e = cudaMemsetAsync(base, 0, W.layout_cap, stream);
        if (e != cudaSuccess) return cuda_fail(e, "wave status clear");
    }
    e = cudaMemcpyAsync(base, W.h_stage, L.table_bytes, cudaMemcpyHostToDevice, stream);
    // the look-back words move with the table sizes: clear them, so that no
    // earlier wave's table bytes can pass for a published word
    if (e == cudaSuccess) e = cudaMemsetAsync(base + L.o_ts, 0, L.status_words * sizeof(unsigned long long), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(W.d_status, 0, n * sizeof(uint32_t), stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(static_cast<char*>(W.d_hdr) + offsetof(WsHeader, status), 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return cuda_fail(e, "wave upload");
    uint32_t split[2];
    int grid = 0;
    st = launch_shape(L, BK, C.bps, W.sms, &grid, split);
    if (st != FP_OK) return st;
    BatchParams bp;
    IdxParams ip;
    make_params(L, BK, base, ws, split, bp, ip);
    e = launch_kernels(BK, bp, ip, L.n_idx, grid, W.sms, stream);
    if (e != cudaSuccess) return cuda_fail(e, "wave launch");
    e = cudaMemcpyAsync(W.h_status, W.d_status, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(W.h_total, W.d_total, n * sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(W.h_ws_status, static_cast<char*>(W.d_hdr) + offsetof(WsHeader, status), sizeof(uint32_t),
                            cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return cuda_fail(e, "wave results");
    return FP_OK;
}

}  // namespace fp

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
        e = cudaMemsetAsync(plan->d_tile_status, 0, plan->status_words * sizeof(unsigned long long), stream);
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
    // clears ordered before the stream's next launch
    if (e == cudaSuccess) e = cudaMemsetAsync(plan->d_status, 0, n * sizeof(uint32_t), stream);
    if (e == cudaSuccess && h.status)
        e = cudaMemsetAsync(static_cast<char*>(plan->d_hdr) + offsetof(WsHeader, status), 0, sizeof(unsigned),
                            stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
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
    info->slots_per_thread_fsst12 = (uint32_t)BK.k[3];
    info->threads = (uint32_t)BK.threads;
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

fp_status fp_batch_config_info(int config, uint32_t* slots_per_thread3, uint32_t* blocks_per_sm,
                               uint32_t* warp_tiles) {
    if (config < 0 || config >= (int)configs().size()) return fail(FP_ERR_ARG, "batch configuration %d out of range", config);
    const Config& C = configs()[config];
    const BatchKernel& BK = batch_kernels()[C.kernel];
    if (slots_per_thread3)
        for (int q = 0; q < 3; ++q) slots_per_thread3[q] = (uint32_t)BK.k[q];
    if (blocks_per_sm) *blocks_per_sm = (uint32_t)C.bps;
    if (warp_tiles) *warp_tiles = (uint32_t)BK.warp_tiles;
    return FP_OK;
}

}  // extern "C"
