// OnPair-16 decode variants (the 1 MiB table is read through L1/L2).
#include "fp_variants.cuh"

namespace fp {

const Variant* variants_onpair16(int* n) {
    static const Variant v[] = {
        make_variant<FP_ONPAIR16, 16, false, 2>(),
        make_variant<FP_ONPAIR16, 8, false, 2>(),
        make_warp_variant<FP_ONPAIR16, 16, false, 8, 3, 16>(),
        make_warp_variant<FP_ONPAIR16, 16, false, 8, 2, 16>(),
        make_warp_variant<FP_ONPAIR16, 16, false, 16, 1, 16>(),
        make_warp_variant<FP_ONPAIR16, 16, false, 16, 1, 8>(),   // split read from the global planes
        make_fused_variant<FP_ONPAIR16, 16, false, 16, 16>(),   // one launch (small columns)
    };
    *n = (int)(sizeof(v) / sizeof(v[0]));
    return v;
}

}  // namespace fp
