// Single-column decoder for sm_103a: the kernel instantiations of the
// decode pipeline (fp_decoder.cuh), its variant table and the launch of the
// index pass plus the decode kernel.
#include "fp_decoder.cuh"

namespace fp {
namespace {

// Index pass over one column (grid-stride over its string boundaries).
__global__ void __launch_bounds__(256) index_kernel(const DecodeParams p, u32 tile, u32* first) {
    const Extent x = column_extent(p, tile);
    index_strings(p, x, tile, (u64)blockIdx.x * blockDim.x + threadIdx.x, (u64)p.n_strings + 1,
                  (u64)gridDim.x * blockDim.x, first);
}

template <int CODEC, int K, bool DSMEM, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) decode_kernel(const DecodeParams p) {
    Decoder<CODEC, K, DSMEM, MINB>::run(p);
}

}  // namespace

// ---------------------------------------------------------------------------
// Variant tables
// ---------------------------------------------------------------------------
template <int CODEC, int K, bool DSMEM, int MINB>
static Variant make_variant() {
    typedef Decoder<CODEC, K, DSMEM, MINB> D;
    return Variant{kThreads, K, DSMEM ? 1 : 0, sizeof(typename D::S),
                   (const void*)&decode_kernel<CODEC, K, DSMEM, MINB>};
}

static const Variant* table_for(int codec, int* n) {
    static const Variant v16[] = {
        make_variant<FP_ONPAIR16, 16, false, 2>(),
        make_variant<FP_ONPAIR16, 8, false, 2>(),
    };
    static const Variant v12[] = {
        make_variant<FP_ONPAIR12, 16, true, 2>(),
        make_variant<FP_ONPAIR12, 16, false, 2>(),
        make_variant<FP_ONPAIR12, 8, true, 2>(),
    };
    static const Variant v8[] = {
        make_variant<FP_FSST8, 16, true, 2>(),
        make_variant<FP_FSST8, 32, true, 2>(),
    };
    switch (codec) {
        case FP_ONPAIR16: *n = (int)(sizeof(v16) / sizeof(v16[0])); return v16;
        case FP_ONPAIR12: *n = (int)(sizeof(v12) / sizeof(v12[0])); return v12;
        case FP_FSST8: *n = (int)(sizeof(v8) / sizeof(v8[0])); return v8;
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

int variant_default(int codec) { (void)codec; return 0; }

uint64_t variant_tile(const Variant& v) { return (uint64_t)kWork * (uint64_t)v.slots_per_thread; }

cudaError_t launch_decode(int codec, const Variant& var, const DecodeParams& p_in, uint32_t* first, int grid,
                          cudaStream_t stream) {
    (void)codec;
    DecodeParams p = p_in;
    p.err_word = &p.ws->status;
    p.total_out = &p.ws->total;
    p.first = first;
    const uint64_t tile = variant_tile(var);
    const uint64_t nb = (uint64_t)p.n_strings + 1;
    uint64_t ib = (nb + 255) / 256;
    if (ib > 4096) ib = 4096;
    index_kernel<<<(unsigned)ib, 256, 0, stream>>>(p, (u32)tile, first);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&p};
    return cudaLaunchKernel(var.kernel, dim3(grid), dim3(var.threads), args, var.smem_bytes, stream);
}

}  // namespace fp
