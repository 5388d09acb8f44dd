// FSST-8 decode variants.
#include "fp_variants.cuh"

namespace fp {

const Variant* variants_fsst8(int* n) {
    static const Variant v[] = {
        make_variant<FP_FSST8, 16, true, 2>(),
        make_variant<FP_FSST8, 32, true, 2>(),
        make_warp_variant<FP_FSST8, 16, true, 8, 3, 8>(),
        make_warp_variant<FP_FSST8, 32, true, 8, 2, 8>(),
        make_warp_variant<FP_FSST8, 32, true, 16, 1, 8>(),
        make_fused_variant<FP_FSST8, 16, true, 16, 8>(),   // one launch (small columns)
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}

}  // namespace fp
