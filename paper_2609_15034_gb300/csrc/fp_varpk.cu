// Decoders of cascaded codes: codes bit-packed at a run-time width (1..16
// bits, LSB-first) and unpacked inside the reduce and decode kernels, one
// variant per escape-free codec (one block of 16 warps per SM; the 12-bit
// codecs stage their tables in shared memory, OnPair-16 reads through L1).
#include "fp_variants.cuh"

namespace fp {

const Variant* variant_packed(int codec) {
    static const Variant v16 = make_packed_variant<FP_ONPAIR16, false, 16>();
    static const Variant v12 = make_packed_variant<FP_ONPAIR12, true, 16>();
    static const Variant v12f = make_packed_variant<FP_FSST12, true, 16>();
    switch (codec) {
        case FP_ONPAIR16: return &v16;
        case FP_ONPAIR12: return &v12;
        case FP_FSST12: return &v12f;
        default: return nullptr;
    }
}

}  // namespace fp
