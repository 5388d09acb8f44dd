// Single-column decoder for sm_103a: the variant tables (their kernel
// instantiations are in fp_var*.cu) with their size- and width-dependent
// defaults, and the launches of one decode call (index pass + block-pipeline
// decode, or index pass and reduce in one grid + tile scan + warp-tile
// decode).
#include "fp_decoder.cuh"
#include "fp_warp.cuh"

namespace fp {
namespace {

// Index pass of the block pipeline over one column (grid-stride over its
// string boundaries).
__global__ void __launch_bounds__(256) index_kernel(const DecodeParams p, u32 tile, u32* first) {
    const Extent x = column_extent(p, tile);
    index_groups(p, x, (u32)(__ffsll((long long)tile) - 1), 0, (u64)p.n_strings + 1,
                 (u64)blockIdx.x * blockDim.x + threadIdx.x, (u64)gridDim.x * blockDim.x, first);
}

}  // namespace

// Variant tables (one translation unit per codec).
const Variant* variants_onpair16(int* n);
const Variant* variants_onpair12(int* n);
const Variant* variants_fsst8(int* n);
const Variant* variants_fsst12(int* n);

static const Variant* table_for(int codec, int* n) {
    switch (codec) {
        case FP_ONPAIR16: return variants_onpair16(n);
        case FP_ONPAIR12: return variants_onpair12(n);
        case FP_FSST8: return variants_fsst8(n);
        case FP_FSST12: return variants_fsst12(n);
        default: *n = 0; return nullptr;
    }
}

int variant_count(int codec) {
    int n;
    table_for(codec, &n);
    return n;
}

const Variant* variant_get(int codec, int v) {
    int n;
    const Variant* t = table_for(codec, &n);
    return (t && v >= 0 && v < n) ? &t[v] : nullptr;
}

// Defaults chosen by measurement on GB300 (synthetic columns, every variant
// timed at 30k..10M strings): warp tiles for every codec, one block of 16
// warps per SM for large columns.  The one-block shapes run the same code
// with the same registers and warps per SM as two blocks of 8 warps, with one
// copy of the dictionary per SM instead of two; they were faster for every
// codec (10M strings: OnPair-12 1446 vs 1342 GB/s, FSST-8 963 vs 902,
// OnPair-16 1029 vs 990).  OnPair-12 below 2^23 slots reads the dictionary
// through L1 (20 warps; staging it per block does not pay: 637 vs 613 GB/s
// at 300k strings); FSST-8 below 2^22 slots uses 16-slot lanes.  The OnPair
// codecs come in both read widths (split read W = 8, whole entries W = 16);
// the dictionary's width picks between them.  FSST-12 stages its 32 KiB
// table in shared memory at every size (16M strings: 1,134 GB/s with 32-slot
// lanes, 1,113 with 16; 300k strings: 368 against 337 through L1).
int variant_default(int codec, uint64_t max_slots, int width) {
    const bool split = width != 16;
    switch (codec) {
        case FP_ONPAIR12:
            if (max_slots >= (1ull << 23)) return split ? 6 : 8;
            return split ? 9 : 7;
        case FP_ONPAIR16: return split ? 5 : 4;
        case FP_FSST8: return max_slots >= (1ull << 22) ? 4 : 2;
        case FP_FSST12: return max_slots >= (1ull << 23) ? 2 : 0;
        default: return 0;
    }
}

int noalloc_default(int codec) {
    switch (codec) {
        case FP_FSST8: return 1;    // block pipeline, 32 slots per thread
        case FP_FSST12: return 0;   // no block pipeline: warp tiles
        default: return 0;          // block pipeline
    }
}

uint64_t variant_tile(const Variant& v) {
    return (uint64_t)(v.warp_tiles ? 32 : kWork) * (uint64_t)v.slots_per_thread;
}

namespace {

// Launch with programmatic stream serialization: the kernel may begin while
// the previous kernel on the stream finishes; it calls grid_wait() before it
// reads that kernel's results.
cudaError_t launch_after(const void* func, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, func, args);
}

constexpr size_t kExtentBytes = 64;
size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch layout of a variant for a buffer of max_slots slots.
struct ScratchLayout {
    uint64_t n_tiles;        // tiles (block tiles or warp tiles) covering the buffer, plus slack
    size_t o_status, o_first, o_agg, o_ex, o_extent, bytes;
};

ScratchLayout scratch_layout(const Variant& v, uint64_t max_slots) {
    ScratchLayout L{};
    L.n_tiles = max_slots / variant_tile(v) + 2;
    if (!v.warp_tiles) {
        L.o_status = 0;
        L.o_first = al256(L.n_tiles * sizeof(unsigned long long));
        L.bytes = al256(L.o_first + (L.n_tiles + 1) * sizeof(uint32_t));
        return L;
    }
    const uint64_t n_scan = L.n_tiles / kScanTile + 2;
    L.o_status = 0;
    L.o_extent = al256(n_scan * sizeof(unsigned long long));
    L.o_agg = L.o_extent + al256(kExtentBytes);
    L.o_ex = L.o_agg + al256(L.n_tiles * sizeof(u64));
    L.o_first = L.o_ex + al256(L.n_tiles * sizeof(u64));
    L.bytes = al256(L.o_first + (L.n_tiles + 1) * sizeof(uint32_t));
    return L;
}

}  // namespace

size_t variant_scratch_bytes(const Variant& v, uint64_t max_slots) { return scratch_layout(v, max_slots).bytes; }

cudaError_t launch_decode(int codec, const Variant& var, const DecodeParams& p_in, void* scratch, uint64_t max_slots,
                          int grid, int sms, cudaStream_t stream) {
    (void)codec;
    const ScratchLayout L = scratch_layout(var, max_slots);
    char* base = static_cast<char*>(scratch);
    DecodeParams p = p_in;
    p.err_word = &p.ws->status;
    p.total_out = &p.ws->total;
    p.tile_status = reinterpret_cast<unsigned long long*>(base + L.o_status);
    uint32_t* first = reinterpret_cast<uint32_t*>(base + L.o_first);
    p.first = first;
    const uint64_t tile = variant_tile(var);
    const uint64_t nb = (uint64_t)p.n_strings + 1;
    uint64_t ib = (nb + 256 * kIdxGroup - 1) / (256 * kIdxGroup);
    if (ib > (uint64_t)sms * 2) ib = (uint64_t)sms * 2;   // two index blocks per SM (an A/B: 8 per SM was 0.4 % slower)
    cudaError_t e;
    void* args[] = {(void*)&p};
    if (!var.warp_tiles) {
        index_kernel<<<(unsigned)ib, 256, 0, stream>>>(p, (u32)tile, first);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return cudaLaunchKernel(var.kernel, dim3(grid), dim3(var.threads), args, var.smem_bytes, stream);
    }

    Extent* xp = reinterpret_cast<Extent*>(base + L.o_extent);
    u64* agg = reinterpret_cast<u64*>(base + L.o_agg);
    u64* ex = reinterpret_cast<u64*>(base + L.o_ex);
    if (var.warp_tiles == 2) {
        // one cooperative launch: every block resident, phases split by grid barriers
        const int nw = var.threads / 32;
        uint64_t dg = (L.n_tiles + nw - 1) / nw;
        if (dg > (uint64_t)grid) dg = (uint64_t)grid;
        void* fargs[] = {(void*)&p, (void*)&xp, (void*)&agg, (void*)&ex};
        return cudaLaunchCooperativeKernel(var.kernel, dim3((unsigned)dg), dim3(var.threads), fargs, var.smem_bytes,
                                           stream);
    }

    // warp tiles: index pass + reduce in one launch, tile scan, decode.  The
    // first launch waits for everything before it (the previous call's decode
    // still reads this workspace); the next two may start early and wait in
    // the kernel for their predecessor.
    const uint64_t n_wt_max = L.n_tiles;   // upper bound; the kernels read the true count from *xp
    uint64_t rg = (n_wt_max + 7) / 8;
    const uint64_t rg_cap = (uint64_t)sms * 8;
    if (rg > rg_cap) rg = rg_cap;
    const Extent* cxp = xp;
    u32 ib32 = (u32)ib;
    void* rargs[] = {(void*)&p, (void*)&xp, (void*)&agg, (void*)&ib32};
    e = cudaLaunchKernel(var.reduce, dim3((unsigned)(rg + ib)), dim3(256), rargs, 0, stream);
    if (e != cudaSuccess) return e;
    uint64_t sg = n_wt_max / kScanTile + 1;
    if (sg > (uint64_t)sms * 2) sg = (uint64_t)sms * 2;
    const u64* cagg = agg;
    unsigned long long* st = p.tile_status;
    void* sargs[] = {(void*)&p, (void*)&cxp, (void*)&cagg, (void*)&ex, (void*)&st};
    e = launch_after(var.scan, dim3((unsigned)sg), dim3(256), sargs, 0, stream);
    if (e != cudaSuccess) return e;
    const u64* cex = ex;
    void* dargs[] = {(void*)&p, (void*)&cxp, (void*)&cex};
    const int nw = var.threads / 32;
    uint64_t dg = (n_wt_max + nw - 1) / nw;
    if (dg > (uint64_t)grid) dg = (uint64_t)grid;
    return launch_after(var.kernel, dim3((unsigned)dg), dim3(var.threads), dargs, var.smem_bytes, stream);
}

}  // namespace fp
