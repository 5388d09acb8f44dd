// Selective decode (paper Sec. 1 and Sec. 2.1: the strings of an FSST-family
// column decode independently, so a subset of rows can be decoded alone).
//
// The selected rows' code slots are laid out one after another in a virtual
// slot space: row k occupies virtual slots [v[k], v[k+1]), v being the
// exclusive scan of the rows' slot counts.  Three launches build v (the
// per-block sums of the row lengths, the scan of those sums, the per-block
// exclusive offsets), a fourth gathers the selected codes into one
// contiguous stored stream (each thread writes whole aligned words of it), and
// fp_decode's kernels then decode that stream with v as its code_offsets.
#include <cstddef>

#include "fp_decoder.cuh"

namespace fp {
namespace {

constexpr int kRowBlock = 256;
constexpr int kRowItems = 2048;   // rows per scan block (8 per thread)
constexpr int kRowPer = kRowItems / kRowBlock;

// Slot count of selected row k (0, with ERRB_CORRUPT, for a bad row).
__device__ __forceinline__ u32 row_len(const RowsArgs& a, u32 k, u32& err) {
    const u32 id = __ldg(a.row_ids + k);
    if (id >= a.n_strings) {
        err |= ERRB_CORRUPT;
        return 0u;
    }
    const u32 b = __ldg(a.code_offsets + id), e = __ldg(a.code_offsets + id + 1);
    if (e < b || (u64)e > a.max_slots) {
        err |= ERRB_CORRUPT;
        return 0u;
    }
    return e - b;
}

// Pass 1: each block sums the slot counts of its kRowItems rows and stores
// the counts in v[] (the next pass turns them into offsets in place).
__global__ void __launch_bounds__(kRowBlock) rows_sums_kernel(const RowsArgs a, u32* v, u64* block_sums,
                                                            unsigned* err_word) {
    __shared__ u64 red[kRowBlock / 32];
    const u64 base = (u64)blockIdx.x * kRowItems + (u64)threadIdx.x * kRowPer;
    u32 err = 0;
    u64 s = 0;
#pragma unroll
    for (int k = 0; k < kRowPer; ++k) {
        const u64 r = base + k;
        if (r < a.n_rows) {
            const u32 L = row_len(a, (u32)r, err);
            v[r] = L;
            s += L;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
    if ((threadIdx.x & 31u) == 0u) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 t = 0;
        for (int w = 0; w < kRowBlock / 32; ++w) t += red[w];
        block_sums[blockIdx.x] = t;
    }
    if (err) atomicOr(err_word, err);
}

// Pass 2 (one block): exclusive scan of the block sums; the total goes to
// ws->rows_slots and must fit the bound (and 32-bit offsets).
__global__ void __launch_bounds__(kRowBlock) rows_scan_sums_kernel(u64* block_sums, u32 nb, u64 bound, WsHeader* ws) {
    __shared__ u64 wsum[kRowBlock / 32];
    __shared__ u64 carry_s;
    const u32 lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (u32 base = 0; base < nb; base += kRowBlock) {
        const u32 i = base + threadIdx.x;
        const u64 x = i < nb ? block_sums[i] : 0;
        u64 inc = x;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const u64 y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= (u32)d) inc += y;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        u64 before = 0, tot = 0;
        for (u32 w = 0; w < kRowBlock / 32; ++w) {
            if (w < warp) before += wsum[w];
            tot += wsum[w];
        }
        const u64 carry = carry_s;
        if (i < nb) block_sums[i] = carry + before + inc - x;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const u64 total = carry_s;
        ws->rows_slots = total;
        if (total > bound || total > 0xffffffffull) atomicOr(&ws->status, ERRB_CAPACITY);
    }
}

// Pass 3: v[k] = slots of the rows before k (in place), v[n_rows] = total.
__global__ void __launch_bounds__(kRowBlock) rows_offsets_kernel(const RowsArgs a, u32* v, const u64* block_sums) {
    __shared__ u64 wsum[kRowBlock / 32];
    const u32 lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const u64 base = (u64)blockIdx.x * kRowItems + (u64)threadIdx.x * kRowPer;
    u32 len[kRowPer];
    u64 s = 0;
#pragma unroll
    for (int k = 0; k < kRowPer; ++k) {
        const u64 r = base + k;
        len[k] = r < a.n_rows ? v[r] : 0u;
        s += len[k];
    }
    u64 inc = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const u64 y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= (u32)d) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    u64 before = 0;
    for (u32 w = 0; w < warp; ++w) before += wsum[w];
    u64 o = block_sums[blockIdx.x] + before + inc - s;
#pragma unroll
    for (int k = 0; k < kRowPer; ++k) {
        const u64 r = base + k;
        if (r <= a.n_rows) v[r] = (u32)o;   // r == n_rows: the total (32 bits; larger totals were flagged)
        o += len[k];
    }
}

// Code in physical slot q of the stored stream.
template <int CODEC>
__device__ __forceinline__ u32 read_code(const uint8_t* s, u64 q) {
    if (CODEC == FP_ONPAIR16) return (u32)__ldg(s + 2 * q) | ((u32)__ldg(s + 2 * q + 1) << 8);
    if (CODEC == FP_ONPAIR12 || CODEC == FP_FSST12) {
        const u64 by = q * 3 / 2;
        const u32 lo = __ldg(s + by), hi = __ldg(s + by + 1);
        return (q & 1) ? ((lo >> 4) | (hi << 4)) : (lo | ((hi & 0xfu) << 8));
    }
    return __ldg(s + q);
}

// Pass 4: gather.  Thread g writes the group of G virtual slots [G g, G g + G)
// of the compacted stream as whole words: 8 slots of 16 or 12 bits (16 or
// 12 bytes), 16 slots of 8 bits (16 bytes).  Slots past the selected total
// (or the bound) are written as zero and never decoded.
template <int CODEC>
__global__ void __launch_bounds__(kRowBlock) rows_gather_kernel(const RowsArgs a, const u32* v, uint8_t* out,
                                                              u64 bound, const WsHeader* ws) {
    constexpr bool W12 = (CODEC == FP_ONPAIR12 || CODEC == FP_FSST12);
    constexpr int G = (CODEC == FP_FSST8) ? 16 : 8;
    const u64 total_raw = ws->rows_slots;
    // a total past 32 bits left v[] wrapped (and flagged): gather nothing
    const u64 total = total_raw > 0xffffffffull ? 0 : (total_raw < bound ? total_raw : bound);
    const u64 n_groups = (total + G - 1) / G;
    const u32 m = a.n_rows;
    for (u64 g = (u64)blockIdx.x * blockDim.x + threadIdx.x; g < n_groups; g += (u64)gridDim.x * blockDim.x) {
        const u64 v0 = g * G;
        // the row holding virtual slot v0: the last k with v[k] <= v0
        u32 lo = 0, hi = m;   // v[lo] <= v0 < v[hi] (v[m] = total > v0)
        while (hi - lo > 1) {
            const u32 mid = (lo + hi) >> 1;
            if ((u64)__ldg(v + mid) <= v0) lo = mid;
            else hi = mid;
        }
        // row k is non-empty (v[k] <= v0 < v[k+1]), so its id passed the checks
        u32 k = lo, held = lo;
        u64 row_end = __ldg(v + k + 1);
        u64 shift = (u64)__ldg(a.code_offsets + __ldg(a.row_ids + k)) - (u64)__ldg(v + k);   // physical - virtual
        u32 c[G];
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const u64 vs = v0 + j;
            u32 code = 0;
            if (vs < total) {
                // skip to the row holding vs (empty rows, bad ids among them, are passed over)
                while (vs >= row_end && k + 1 < m) row_end = __ldg(v + (++k) + 1);
                if (vs < row_end) {
                    if (k != held) {
                        shift = (u64)__ldg(a.code_offsets + __ldg(a.row_ids + k)) - (u64)__ldg(v + k);
                        held = k;
                    }
                    code = read_code<CODEC>(a.codes, vs + shift);
                }
            }
            c[j] = code;
        }
        if (CODEC == FP_ONPAIR16) {
            reinterpret_cast<uint4*>(out)[g] = make_uint4(c[0] | (c[1] << 16), c[2] | (c[3] << 16),
                                                          c[4] | (c[5] << 16), c[6] | (c[7] << 16));
        } else if (W12) {
            // 8 codes, LSB-first: 96 bits = 3 words
            u32* w = reinterpret_cast<u32*>(out) + 3 * g;
            w[0] = c[0] | (c[1] << 12) | (c[2] << 24);
            w[1] = (c[2] >> 8) | (c[3] << 4) | (c[4] << 16) | (c[5] << 28);
            w[2] = (c[5] >> 4) | (c[6] << 8) | (c[7] << 20);
        } else {
            reinterpret_cast<uint4*>(out)[g] =
                make_uint4(c[0] | (c[1] << 8) | (c[2] << 16) | (c[3] << 24), c[4] | (c[5] << 8) | (c[6] << 16) | (c[7] << 24),
                           c[8] | (c[9] << 8) | (c[10] << 16) | (c[11] << 24),
                           c[12] | (c[13] << 8) | (c[14] << 16) | (c[15] << 24));
        }
    }
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

RowsLayout rows_layout(int codec, uint32_t n_rows, uint64_t selected_slots) {
    RowsLayout L{};
    const uint64_t nb = ((uint64_t)n_rows + kRowItems - 1) / kRowItems + 1;
    L.o_v = 0;
    L.o_sums = al256(((size_t)n_rows + 1) * sizeof(u32));
    L.o_codes = L.o_sums + al256(nb * sizeof(u64));
    const uint64_t G = codec == FP_FSST8 ? 16 : 8;
    const uint64_t group_bytes = codec == FP_FSST8 ? 16 : (code_bits(codec) * 8 / 8);
    const uint64_t groups = (selected_slots + G - 1) / G;
    L.codes_bytes = (selected_slots * code_bits(codec) + 7) / 8;
    L.bytes = L.o_codes + al256(groups * group_bytes + 16);
    return L;
}

cudaError_t launch_rows_gather(int codec, const RowsArgs& a, uint64_t selected_slots, bool gather, void* scratch,
                               const RowsLayout& L, WsHeader* ws, int sms, cudaStream_t stream) {
    char* base = static_cast<char*>(scratch);
    u32* v = reinterpret_cast<u32*>(base + L.o_v);
    u64* sums = reinterpret_cast<u64*>(base + L.o_sums);
    uint8_t* codes = reinterpret_cast<uint8_t*>(base + L.o_codes);
    const u32 nb = (u32)((uint64_t)a.n_rows / kRowItems) + 1;   // the blocks of v[0 .. n_rows]
    rows_sums_kernel<<<nb, kRowBlock, 0, stream>>>(a, v, sums, &ws->status);
    rows_scan_sums_kernel<<<1, kRowBlock, 0, stream>>>(sums, nb, selected_slots, ws);
    rows_offsets_kernel<<<nb, kRowBlock, 0, stream>>>(a, v, sums);
    if (!gather) return cudaGetLastError();
    const uint64_t G = codec == FP_FSST8 ? 16 : 8;
    uint64_t grid = (selected_slots + G * kRowBlock - 1) / (G * kRowBlock);
    if (grid > (uint64_t)sms * 8) grid = (uint64_t)sms * 8;
    if (grid < 1) grid = 1;
    switch (codec) {
        case FP_ONPAIR16: rows_gather_kernel<FP_ONPAIR16><<<(unsigned)grid, kRowBlock, 0, stream>>>(a, v, codes, selected_slots, ws); break;
        case FP_ONPAIR12: rows_gather_kernel<FP_ONPAIR12><<<(unsigned)grid, kRowBlock, 0, stream>>>(a, v, codes, selected_slots, ws); break;
        case FP_FSST8: rows_gather_kernel<FP_FSST8><<<(unsigned)grid, kRowBlock, 0, stream>>>(a, v, codes, selected_slots, ws); break;
        default: rows_gather_kernel<FP_FSST12><<<(unsigned)grid, kRowBlock, 0, stream>>>(a, v, codes, selected_slots, ws); break;
    }
    return cudaGetLastError();
}

}  // namespace fp
