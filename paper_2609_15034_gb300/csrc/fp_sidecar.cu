// Decoding with a stored sidecar of output positions (paper Sec. 3.1).
//
// fp_sidecar_build runs the passes that fp_decode runs before its decode --
// index pass and reduce in one grid, then the tile scan -- and keeps the
// scanned tile offsets in a caller buffer, the column's decoded size in
// front.  fp_decode_sidecar runs the index pass (it needs the first string
// of every tile), a size check and the warp-tile decode on such a table.
// One warp-tile shape per codec, the fp_decode default for large columns,
// so a table's tile size is fixed by its codec.  Scratch comes from the
// caller; nothing here allocates device memory.
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>

#include "fp_decoder.cuh"
#include "fp_warp.cuh"
#include "fastpair_sidecar.h"

namespace fp {
namespace {

constexpr int kSidecarWarps = 16;   // warps per decode block, one block per SM

template <int CODEC>
struct Shape;
template <>
struct Shape<FP_ONPAIR16> {
    static constexpr int K = 16;
    static constexpr bool DSMEM = false;   // 1 MiB table: read through L1/L2
};
template <>
struct Shape<FP_ONPAIR12> {
    static constexpr int K = 16;
    static constexpr bool DSMEM = true;
};
template <>
struct Shape<FP_FSST8> {
    static constexpr int K = 32;
    static constexpr bool DSMEM = true;
};
template <>
struct Shape<FP_FSST12> {
    static constexpr int K = 16;
    static constexpr bool DSMEM = true;   // 32 KiB of 8-byte entries
};

uint32_t tile_slots(int codec) { return codec == FP_FSST8 ? 32u * 32u : 32u * 16u; }

// Size check of a stored table: entry 0 is the column's decoded size.
__global__ void __launch_bounds__(32) sidecar_check_kernel(const u64* total, u64 capacity, unsigned* err) {
    if (threadIdx.x != 0) return;
    const u64 t = *total;
    u32 bits = 0;
    if (t > capacity) bits |= ERRB_CAPACITY;
    if (t > 0x7fffffffull) bits |= ERRB_OVERFLOW;
    if (bits) atomicOr(err, bits);
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch: workspace header | look-back words of the tile scan | extent |
// tile elements | tile -> first string.
struct Layout {
    uint64_t n_tiles;   // upper bound on the column's tiles
    uint64_t n_scan;
    size_t o_status, o_extent, o_agg, o_first, bytes;
};

Layout layout(int codec, uint64_t codes_bytes) {
    Layout L{};
    L.n_tiles = max_slots_of(codec, codes_bytes) / tile_slots(codec) + 2;
    L.n_scan = L.n_tiles / kScanTile + 2;
    L.o_status = al256(kWsHeaderBytes);
    L.o_extent = L.o_status + al256(L.n_scan * sizeof(u64));
    L.o_agg = L.o_extent + al256(sizeof(Extent));
    L.o_first = L.o_agg + al256(L.n_tiles * sizeof(u64));
    L.bytes = L.o_first + al256((L.n_tiles + 1) * sizeof(u32));
    return L;
}

std::mutex g_mu;
std::map<int, int> g_sms;                     // device -> SM count
std::map<std::pair<int, int>, bool> g_attr;   // (device, codec) -> decode smem attribute set

template <int CODEC>
struct Path {
    static constexpr int K = Shape<CODEC>::K;
    static constexpr bool DSMEM = Shape<CODEC>::DSMEM;
    typedef WarpCore<CODEC, K, DSMEM> C;

    static size_t decode_smem() {
        return (size_t)C::DICT_BYTES + (DSMEM ? (size_t)C::LENS_BYTES : 0) + kSidecarWarps * sizeof(WarpArea<K>);
    }
    // dictionary reads: whole 16-byte entries for the OnPair codecs (staged
    // for OnPair-12, through L1 for OnPair-16), 8-byte entries for FSST
    static constexpr int W = (CODEC == FP_ONPAIR16 || CODEC == FP_ONPAIR12) ? 16 : 8;
    static const void* decode_kernel() {
        return (const void*)&warp_decode_kernel<CODEC, K, DSMEM, kSidecarWarps, 1, W>;
    }
    // Index pass in blocks [0, ib), reduce in the next rg blocks (rg = 0: index only).
    static cudaError_t index_reduce(const DecodeParams& p, Extent* xp, u64* agg, uint64_t ib, uint64_t rg,
                                    cudaStream_t s) {
        u32 ib32 = (u32)ib;
        void* args[] = {(void*)&p, (void*)&xp, (void*)&agg, (void*)&ib32};
        return cudaLaunchKernel((const void*)&reduce_kernel<CODEC, K, DSMEM>, dim3((unsigned)(ib + rg)), dim3(256),
                                args, 0, s);
    }
    static cudaError_t scan(const DecodeParams& p, const Extent* xp, const u64* agg, u64* ex, uint64_t grid,
                            cudaStream_t s) {
        unsigned long long* st = p.tile_status;
        void* args[] = {(void*)&p, (void*)&xp, (void*)&agg, (void*)&ex, (void*)&st};
        return cudaLaunchKernel((const void*)&tiles_scan_kernel<CODEC == FP_FSST8>, dim3((unsigned)grid), dim3(256),
                                args, 0, s);
    }
    static cudaError_t decode(const DecodeParams& p, const Extent* xp, const u64* ex, uint64_t grid, cudaStream_t s) {
        void* args[] = {(void*)&p, (void*)&xp, (void*)&ex};
        return cudaLaunchKernel(decode_kernel(), dim3((unsigned)grid), dim3(kSidecarWarps * 32), args, decode_smem(),
                                s);
    }
};

fp_status device_setup(int codec, int* sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_sms.find(dev);
    if (it == g_sms.end()) {
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        it = g_sms.emplace(dev, n).first;
    }
    *sms = it->second;
    bool& done = g_attr[{dev, codec}];
    if (!done) {
        const void* k = codec == FP_ONPAIR16 ? Path<FP_ONPAIR16>::decode_kernel()
                        : codec == FP_ONPAIR12 ? Path<FP_ONPAIR12>::decode_kernel()
                        : codec == FP_FSST12   ? Path<FP_FSST12>::decode_kernel()
                                               : Path<FP_FSST8>::decode_kernel();
        const size_t smem = codec == FP_ONPAIR16 ? Path<FP_ONPAIR16>::decode_smem()
                            : codec == FP_ONPAIR12 ? Path<FP_ONPAIR12>::decode_smem()
                            : codec == FP_FSST12   ? Path<FP_FSST12>::decode_smem()
                                                   : Path<FP_FSST8>::decode_smem();
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(sidecar decode)");
        done = true;
    }
    return FP_OK;
}

// Checks of the arguments both calls add to fp_decode's; fills the layout.
fp_status check_sidecar_args(fp_codec codec, uint64_t codes_bytes, uint32_t n_strings, const void* d_sidecar,
                             uint64_t sidecar_entries, void* d_scratch, uint64_t scratch_bytes,
                             const uint32_t* d_status, Layout* L) {
    if (n_strings == 0xffffffffu) return fail(FP_ERR_ARG, "n_strings must be below 2^32-1");
    if (!d_sidecar) return fail(FP_ERR_ARG, "d_sidecar is NULL");
    if (reinterpret_cast<uintptr_t>(d_sidecar) % 8) return fail(FP_ERR_ARG, "d_sidecar not 8-byte aligned");
    const uint64_t need = fp_sidecar_entries(codec, codes_bytes);
    if (sidecar_entries < need)
        return fail(FP_ERR_ARG, "sidecar has %llu entries, the code buffer needs %llu",
                    (unsigned long long)sidecar_entries, (unsigned long long)need);
    *L = layout(codec, codes_bytes);
    if (!d_scratch) return fail(FP_ERR_ARG, "d_scratch is NULL");
    if (reinterpret_cast<uintptr_t>(d_scratch) % 16) return fail(FP_ERR_ARG, "d_scratch not 16-byte aligned");
    if (scratch_bytes < L->bytes)
        return fail(FP_ERR_ARG, "scratch has %llu bytes, the code buffer needs %llu",
                    (unsigned long long)scratch_bytes, (unsigned long long)L->bytes);
    if (!d_status) return fail(FP_ERR_ARG, "d_status is NULL");
    if (reinterpret_cast<uintptr_t>(d_status) % 4) return fail(FP_ERR_ARG, "d_status not 4-byte aligned");
    return FP_OK;
}

DecodeParams column_params(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                           const uint32_t* d_code_offsets, uint32_t n_strings, char* scratch, const Layout& L,
                           uint32_t* d_status) {
    DecodeParams p;
    memset(&p, 0, sizeof(p));
    p.dict = dict->view();
    p.codes = static_cast<const uint8_t*>(d_codes);
    p.codes_bytes = codes_bytes;
    p.max_slots = max_slots_of(codec, codes_bytes);
    p.code_offsets = d_code_offsets;
    p.n_strings = n_strings;
    p.ws = reinterpret_cast<WsHeader*>(scratch);
    p.tile_status = reinterpret_cast<unsigned long long*>(scratch + L.o_status);
    p.err_word = d_status;
    p.first = reinterpret_cast<const uint32_t*>(scratch + L.o_first);
    return p;
}

uint64_t index_blocks(uint32_t n_strings, int sms) {
    const uint64_t nb = (uint64_t)n_strings + 1;
    uint64_t ib = (nb + 256 * kIdxGroup - 1) / (256 * kIdxGroup);
    if (ib > (uint64_t)sms * 8) ib = (uint64_t)sms * 8;
    return ib;
}

template <int CODEC>
cudaError_t build_launches(const DecodeParams& p, char* scratch, const Layout& L, u64* ex, int sms, cudaStream_t s) {
    typedef Path<CODEC> P;
    Extent* xp = reinterpret_cast<Extent*>(scratch + L.o_extent);
    u64* agg = reinterpret_cast<u64*>(scratch + L.o_agg);
    uint64_t rg = (L.n_tiles + 7) / 8;
    if (rg > (uint64_t)sms * 8) rg = (uint64_t)sms * 8;
    cudaError_t e = P::index_reduce(p, xp, agg, index_blocks(p.n_strings, sms), rg, s);
    if (e != cudaSuccess) return e;
    uint64_t sg = L.n_tiles / kScanTile + 1;
    if (sg > (uint64_t)sms * 2) sg = (uint64_t)sms * 2;
    return P::scan(p, xp, agg, ex, sg, s);
}

template <int CODEC>
cudaError_t decode_launches(const DecodeParams& p, char* scratch, const Layout& L, const u64* sidecar, int sms,
                            cudaStream_t s) {
    typedef Path<CODEC> P;
    Extent* xp = reinterpret_cast<Extent*>(scratch + L.o_extent);
    cudaError_t e = P::index_reduce(p, xp, nullptr, index_blocks(p.n_strings, sms), 0, s);
    if (e != cudaSuccess) return e;
    sidecar_check_kernel<<<1, 32, 0, s>>>(sidecar, p.capacity, p.err_word);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uint64_t grid = (L.n_tiles + kSidecarWarps - 1) / kSidecarWarps;
    if (grid > (uint64_t)sms) grid = (uint64_t)sms;
    return P::decode(p, xp, sidecar + 1, grid, s);
}

}  // namespace
}  // namespace fp

using namespace fp;

extern "C" {

uint32_t fp_sidecar_tile_slots(fp_codec codec) { return valid_codec(codec) ? tile_slots(codec) : 0u; }

uint64_t fp_sidecar_entries(fp_codec codec, uint64_t codes_bytes) {
    return valid_codec(codec) ? max_slots_of(codec, codes_bytes) / tile_slots(codec) + 3 : 0u;
}

uint64_t fp_sidecar_scratch_bytes(fp_codec codec, uint64_t codes_bytes) {
    return valid_codec(codec) ? layout(codec, codes_bytes).bytes : 0u;
}

fp_status fp_sidecar_build(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                           const uint32_t* d_code_offsets, uint32_t n_strings, uint64_t* d_sidecar,
                           uint64_t sidecar_entries, void* d_scratch, uint64_t scratch_bytes,
                           uint32_t* d_status, fp_stream_t stream_) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    fp_status st = check_common(codec, dict, d_codes, codes_bytes, d_code_offsets, nullptr, 0, nullptr, false);
    if (st != FP_OK) return st;
    Layout L;
    st = check_sidecar_args(codec, codes_bytes, n_strings, d_sidecar, sidecar_entries, d_scratch, scratch_bytes,
                            d_status, &L);
    if (st != FP_OK) return st;
    int sms = 0;
    st = device_setup(codec, &sms);
    if (st != FP_OK) return st;
    char* scratch = static_cast<char*>(d_scratch);
    // fresh look-back state: counters and words zero, launch tag 1 (0 means "never written")
    cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(uint32_t), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, L.o_agg, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(scratch + offsetof(WsHeader, epoch), 1, 1, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(sidecar scratch)");
    DecodeParams p = column_params(codec, dict, d_codes, codes_bytes, d_code_offsets, n_strings, scratch, L, d_status);
    p.size_only = 1;   // no output buffer: no capacity check
    p.total_out = reinterpret_cast<unsigned long long*>(d_sidecar);
    u64* ex = reinterpret_cast<u64*>(d_sidecar) + 1;
    if (codec == FP_ONPAIR16) e = build_launches<FP_ONPAIR16>(p, scratch, L, ex, sms, stream);
    else if (codec == FP_ONPAIR12) e = build_launches<FP_ONPAIR12>(p, scratch, L, ex, sms, stream);
    else if (codec == FP_FSST12) e = build_launches<FP_FSST12>(p, scratch, L, ex, sms, stream);
    else e = build_launches<FP_FSST8>(p, scratch, L, ex, sms, stream);
    if (e != cudaSuccess) return cuda_fail(e, "sidecar build launch");
    return FP_OK;
}

fp_status fp_decode_sidecar(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                            const uint32_t* d_code_offsets, uint32_t n_strings, const uint64_t* d_sidecar,
                            uint64_t sidecar_entries, uint8_t* d_out_bytes, uint64_t out_capacity,
                            uint32_t* d_out_offsets, void* d_scratch, uint64_t scratch_bytes,
                            uint32_t* d_status, fp_stream_t stream_) {
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    fp_status st = check_common(codec, dict, d_codes, codes_bytes, d_code_offsets, d_out_bytes, out_capacity,
                                d_out_offsets, true);
    if (st != FP_OK) return st;
    Layout L;
    st = check_sidecar_args(codec, codes_bytes, n_strings, d_sidecar, sidecar_entries, d_scratch, scratch_bytes,
                            d_status, &L);
    if (st != FP_OK) return st;
    int sms = 0;
    st = device_setup(codec, &sms);
    if (st != FP_OK) return st;
    char* scratch = static_cast<char*>(d_scratch);
    cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(uint32_t), stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(status)");
    DecodeParams p = column_params(codec, dict, d_codes, codes_bytes, d_code_offsets, n_strings, scratch, L, d_status);
    p.out = d_out_bytes;
    p.capacity = out_capacity;
    p.out_offsets = d_out_offsets;
    const u64* sc = reinterpret_cast<const u64*>(d_sidecar);
    if (codec == FP_ONPAIR16) e = decode_launches<FP_ONPAIR16>(p, scratch, L, sc, sms, stream);
    else if (codec == FP_ONPAIR12) e = decode_launches<FP_ONPAIR12>(p, scratch, L, sc, sms, stream);
    else if (codec == FP_FSST12) e = decode_launches<FP_FSST12>(p, scratch, L, sc, sms, stream);
    else e = decode_launches<FP_FSST8>(p, scratch, L, sc, sms, stream);
    if (e != cudaSuccess) return cuda_fail(e, "sidecar decode launch");
    return FP_OK;
}

}  // extern "C"
