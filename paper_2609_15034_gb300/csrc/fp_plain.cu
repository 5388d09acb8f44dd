// Plain baseline decoder: one thread per string.
//
// Three launches: (1) every thread sums the token lengths of its string,
// (2) an exclusive prefix sum over strings gives out_offsets, (3) every
// thread walks its string again and copies token bytes one at a time from
// the dictionary's interchange layout (an offset read, then the bytes).
// This is the straightforward GPU port of a CPU decode loop; it is timed
// beside the single-pass decoder.
#include <cuda_runtime.h>
#include <cstdint>

#include "fp_internal.h"

namespace fp {
namespace {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr int kBlock = 256;
constexpr int kScanItems = 2048;   // strings per scan block (kBlock x 8)

__device__ __forceinline__ u32 read_slot(int codec, const uint8_t* s, u64 q) {
    if (codec == FP_ONPAIR16) return (u32)s[2 * q] | ((u32)s[2 * q + 1] << 8);
    if (codec == FP_ONPAIR12 || codec == FP_FSST12) {
        const u64 by = q * 3 / 2;
        const u32 a = s[by], b = s[by + 1];
        return (q & 1) ? ((a >> 4) | (b << 4)) : (a | ((b & 0xfu) << 8));
    }
    return s[q];
}

// Bytes string i decodes to; flags corrupt input.
__device__ u64 string_size(int codec, const DecodeParams& p, u32 i, u32& err) {
    u64 j = p.code_offsets[i], e = p.code_offsets[i + 1];
    if (e < j || e > p.max_slots) { err |= ERRB_CORRUPT; return 0; }
    u64 n = 0;
    while (j < e) {
        const u32 c = read_slot(codec, p.codes, j);
        if (codec == FP_FSST8 && c == 255u) {
            if (j + 1 >= e) { err |= ERRB_CORRUPT; j += 1; continue; }
            n += 1; j += 2; continue;
        }
        if (c >= p.dict.n_entries) { err |= ERRB_CORRUPT; j += 1; continue; }
        n += p.dict.offsets[c + 1] - p.dict.offsets[c];
        j += 1;
    }
    return n;
}

__global__ void plain_sizes(int codec, DecodeParams p, u32* sizes) {
    const u32 i = blockIdx.x * kBlock + threadIdx.x;
    u32 err = 0;
    if (i < p.n_strings) sizes[i] = (u32)string_size(codec, p, i, err);
    if (err) atomicOr(&p.ws->status, err);
}

// Per-block sums of kScanItems sizes.
__global__ void plain_block_sums(const u32* sizes, u32 n, u64* block_sums) {
    __shared__ u64 red[kBlock];
    const u64 base = (u64)blockIdx.x * kScanItems;
    u64 s = 0;
    for (int k = 0; k < kScanItems / kBlock; ++k) {
        const u64 i = base + (u64)k * kBlock + threadIdx.x;
        if (i < n) s += sizes[i];
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int d = kBlock / 2; d > 0; d >>= 1) {
        if (threadIdx.x < (u32)d) red[threadIdx.x] += red[threadIdx.x + d];
        __syncthreads();
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = red[0];
}

// Exclusive scan of the block sums by one block (serial over chunks).
__global__ void plain_scan_block_sums(u64* block_sums, u32 nb, DecodeParams p) {
    __shared__ u64 buf[kBlock];
    u64 carry = 0;
    for (u32 base = 0; base < nb; base += kBlock) {
        const u32 i = base + threadIdx.x;
        const u64 v = i < nb ? block_sums[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int d = 1; d < kBlock; d <<= 1) {
            const u64 x = threadIdx.x >= (u32)d ? buf[threadIdx.x - d] : 0;
            __syncthreads();
            buf[threadIdx.x] += x;
            __syncthreads();
        }
        if (i < nb) block_sums[i] = carry + buf[threadIdx.x] - v;
        const u64 tot = buf[kBlock - 1];
        __syncthreads();
        carry += tot;
    }
    if (threadIdx.x == 0) {
        p.ws->total = carry;
        if (!p.size_only && carry > p.capacity) atomicOr(&p.ws->status, ERRB_CAPACITY);
        if (carry > 0x7fffffffull) atomicOr(&p.ws->status, ERRB_OVERFLOW);
    }
}

// Exclusive offsets within each block plus the block's prefix.
__global__ void plain_offsets(const u32* sizes, u32 n, const u64* block_sums, DecodeParams p) {
    __shared__ u64 buf[kBlock];
    const u64 base = (u64)blockIdx.x * kScanItems;
    constexpr int PER = kScanItems / kBlock;
    u64 loc[PER];
    u64 s = 0;
    for (int k = 0; k < PER; ++k) {
        const u64 i = base + (u64)threadIdx.x * PER + k;
        loc[k] = s;
        s += i < n ? sizes[i] : 0;
    }
    buf[threadIdx.x] = s;
    __syncthreads();
    for (int d = 1; d < kBlock; d <<= 1) {
        const u64 x = threadIdx.x >= (u32)d ? buf[threadIdx.x - d] : 0;
        __syncthreads();
        buf[threadIdx.x] += x;
        __syncthreads();
    }
    const u64 pre = block_sums[blockIdx.x] + buf[threadIdx.x] - s;
    for (int k = 0; k < PER; ++k) {
        const u64 i = base + (u64)threadIdx.x * PER + k;
        if (i <= n && !p.size_only) p.out_offsets[i] = (u32)(pre + loc[k]);
    }
}

__global__ void plain_copy(int codec, DecodeParams p) {
    const u32 i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= p.n_strings) return;
    if (p.ws->total > p.capacity) return;
    u64 j = p.code_offsets[i], e = p.code_offsets[i + 1];
    if (e < j || e > p.max_slots) return;
    u64 pos = p.out_offsets[i];
    while (j < e) {
        const u32 c = read_slot(codec, p.codes, j);
        if (codec == FP_FSST8 && c == 255u) {
            if (j + 1 >= e) break;
            p.out[pos++] = (uint8_t)read_slot(codec, p.codes, j + 1);
            j += 2;
            continue;
        }
        if (c < p.dict.n_entries) {
            const u32 a = p.dict.offsets[c], b = p.dict.offsets[c + 1];
            for (u32 x = a; x < b; ++x) p.out[pos++] = p.dict.bytes[x];
        }
        j += 1;
    }
}

}  // namespace

size_t plain_scratch_words(uint32_t n_strings) {
    const size_t nb = ((size_t)n_strings + kScanItems) / kScanItems + 1;
    return (size_t)n_strings + 2 * nb + 4;   // sizes (u32) + block sums (u64)
}

cudaError_t launch_plain(int codec, const DecodeParams& p, uint32_t* d_scratch, size_t scratch_words,
                         cudaStream_t stream) {
    (void)scratch_words;
    const u32 n = p.n_strings;
    u32* sizes = d_scratch;
    u64* block_sums = reinterpret_cast<u64*>(d_scratch + (((size_t)n + 3) & ~(size_t)1));
    const u32 nb = (u32)(((u64)n + 1 + kScanItems - 1) / kScanItems);
    const u32 gs = (n + kBlock - 1) / kBlock;
    if (gs) plain_sizes<<<gs, kBlock, 0, stream>>>(codec, p, sizes);
    plain_block_sums<<<nb, kBlock, 0, stream>>>(sizes, n, block_sums);
    plain_scan_block_sums<<<1, kBlock, 0, stream>>>(block_sums, nb, p);
    plain_offsets<<<nb, kBlock, 0, stream>>>(sizes, n, block_sums, p);
    if (!p.size_only && gs) plain_copy<<<gs, kBlock, 0, stream>>>(codec, p);
    return cudaGetLastError();
}

}  // namespace fp
