// FSST-12 decode variants (12-bit codes, 4,096 entries of 8 bytes: 32 KiB,
// small enough to stage in shared memory).
#include "fp_variants.cuh"

namespace fp {

const Variant* variants_fsst12(int* n) {
    static const Variant v[] = {
        make_warp_variant<FP_FSST12, 16, true, 16, 1, 8>(),
        make_warp_variant<FP_FSST12, 16, false, 20, 1, 8>(),
        make_warp_variant<FP_FSST12, 32, true, 16, 1, 8>(),
        make_fused_variant<FP_FSST12, 16, true, 16, 8>(),   // one launch (small columns)
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}

}  // namespace fp
