// Kernel instantiations behind the variant tables: each codec's table lives
// in its own translation unit (fp_var16.cu, fp_var12.cu, fp_var8.cu,
// fp_var12f.cu) so that they compile in parallel.
#pragma once
#include "fp_decoder.cuh"
#include "fp_warp.cuh"

namespace fp {
namespace {

template <int CODEC, int K, bool DSMEM, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) decode_kernel(const DecodeParams p) {
    Decoder<CODEC, K, DSMEM, MINB>::run(p);
}

// Block pipeline: whole 16-byte OnPair entries (W = 16), 8-byte FSST-8 ones.
template <int CODEC, int K, bool DSMEM, int MINB>
Variant make_variant() {
    typedef Decoder<CODEC, K, DSMEM, MINB> D;
    Variant v{};
    v.threads = kThreads;
    v.slots_per_thread = K;
    v.dict_smem = DSMEM ? 1 : 0;
    v.smem_bytes = sizeof(typename D::S);
    v.kernel = (const void*)&decode_kernel<CODEC, K, DSMEM, MINB>;
    v.warp_tiles = 0;
    v.width = CODEC == FP_FSST8 ? 8 : 16;
    return v;
}

template <int CODEC, int K, bool DSMEM, int NW, int MINB, int W>
Variant make_warp_variant() {
    typedef WarpCore<CODEC, K, DSMEM, W> C;
    Variant v{};
    v.threads = NW * 32;
    v.slots_per_thread = K;
    v.dict_smem = DSMEM ? 1 : 0;
    v.smem_bytes = (size_t)C::DICT_BYTES + (DSMEM ? (size_t)C::LENS_BYTES : 0) + NW * sizeof(WarpArea<K>);
    v.kernel = (const void*)&warp_decode_kernel<CODEC, K, DSMEM, NW, MINB, W>;
    v.warp_tiles = 1;
    v.reduce = (const void*)&reduce_kernel<CODEC, K, DSMEM>;
    v.scan = (const void*)&tiles_scan_kernel<CODEC == FP_FSST8>;
    v.width = W;
    return v;
}

// Warp tiles in one cooperative launch (small columns).
template <int CODEC, int K, bool DSMEM, int NW, int W>
Variant make_fused_variant() {
    typedef WarpCore<CODEC, K, DSMEM, W> C;
    Variant v{};
    v.threads = NW * 32;
    v.slots_per_thread = K;
    v.dict_smem = DSMEM ? 1 : 0;
    v.smem_bytes = (size_t)C::DICT_BYTES + (DSMEM ? (size_t)C::LENS_BYTES : 0) + NW * sizeof(WarpArea<K>);
    v.kernel = (const void*)&fused_decode_kernel<CODEC, K, DSMEM, NW, W>;
    v.warp_tiles = 2;
    v.width = W;
    return v;
}

// Packed codes (run-time width): the warp-tile decoder with a per-lane
// shared-memory scratch for the code words.
template <int CODEC, bool DSMEM, int NW>
Variant make_packed_variant() {
    constexpr int K = 16, W = (CODEC == FP_FSST12) ? 8 : 16;
    typedef WarpCore<CODEC, K, DSMEM, W, true> C;
    Variant v{};
    v.threads = NW * 32;
    v.slots_per_thread = K;
    v.dict_smem = DSMEM ? 1 : 0;
    v.smem_bytes = (size_t)C::DICT_BYTES + (DSMEM ? (size_t)C::LENS_BYTES : 0) + NW * sizeof(WarpArea<K>) +
                   (size_t)NW * 32 * C::PK_STRIDE * sizeof(u32);
    v.kernel = (const void*)&warp_decode_kernel<CODEC, K, DSMEM, NW, 1, W, true>;
    v.warp_tiles = 1;
    v.reduce = (const void*)&reduce_kernel<CODEC, K, DSMEM, true>;
    v.scan = (const void*)&tiles_scan_kernel<false>;
    v.width = W;
    return v;
}

}  // namespace
}  // namespace fp
