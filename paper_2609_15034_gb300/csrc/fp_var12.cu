// OnPair-12 decode variants.
#include "fp_variants.cuh"

namespace fp {

const Variant* variants_onpair12(int* n) {
    static const Variant v[] = {
        make_variant<FP_ONPAIR12, 16, true, 2>(),
        make_variant<FP_ONPAIR12, 16, false, 2>(),
        make_variant<FP_ONPAIR12, 8, true, 2>(),
        make_warp_variant<FP_ONPAIR12, 16, true, 8, 2, 8>(),
        make_warp_variant<FP_ONPAIR12, 16, false, 8, 3, 16>(),
        make_warp_variant<FP_ONPAIR12, 16, true, 10, 2, 8>(),
        make_warp_variant<FP_ONPAIR12, 16, true, 16, 1, 8>(),
        make_warp_variant<FP_ONPAIR12, 16, false, 20, 1, 16>(),
        make_warp_variant<FP_ONPAIR12, 16, true, 16, 1, 16>(),    // both planes from shared memory
        make_warp_variant<FP_ONPAIR12, 16, false, 20, 1, 8>(),    // split read from the global planes
        make_fused_variant<FP_ONPAIR12, 16, false, 16, 16>(),   // one launch (small columns)
        make_fused_variant<FP_ONPAIR12, 16, true, 16, 16>(),
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}

}  // namespace fp
