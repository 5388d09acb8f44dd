// Single-pass column decoder for sm_103a.
//
// One stream-ordered call decodes a whole column (paper Sec. 2.1 semantics)
// into Arrow-style output (Sec. 5) with two launches:
//
//   index_kernel   one pass over code_offsets: validates it and records, for
//                  every tile of 256*K code slots, the first string boundary
//                  at or after the tile's start;
//   decode_kernel  persistent; tiles are taken from an atomic ticket counter.
//
// A decode block has 8 worker warps and 1 scan warp.  Two tiles are in flight
// per block, in a two-slot ring:
//
//   workers, front(t+1): wide code loads and in-register unpack (16-bit
//       words, the 12-bit LSB-first bitstream, FSST-8 bytes), token-length
//       gather, per-warp scan; arrive on FRONT[slot];
//   scan warp: block scan of the warp totals, publish the tile aggregate,
//       decoupled look-back over earlier tiles (Merrill & Garland, "Single-
//       pass Parallel Prefix Scan with Decoupled Look-back", 2016) with a
//       bounded wait, publish the inclusive prefix; arrive on EXCL[slot];
//   workers, back(t): assemble each thread's K tokens in a 32-byte register
//       window with funnel shifts and store whole aligned 16-byte chunks;
//       chunks shared by neighbouring threads are merged through shared
//       memory; write out_offsets of the strings that start in the tile.
//
// So the look-back of tile t overlaps the loads of tile t+1 and the
// assembly of tile t-1.  The paper instead reads stored per-batch output
// positions (a sidecar, Sec. 3.1) and stages output bytes in shared memory
// before a coalesced drain (Algorithm 1).
//
// FSST-8 escapes: each thread computes the bytes and exit state of its slots
// for both possible entry states (is the first slot a literal?); the scans
// compose these two-state elements, so escape parity crosses thread and tile
// boundaries through the same scan and look-back.
#include <cuda_runtime.h>
#include <cstdint>

#include "fp_internal.h"

namespace fp {
namespace {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr int kWorkWarps = 8;
constexpr int kWork = kWorkWarps * 32;        // worker threads per block
constexpr int kThreads = kWork + 32;          // + the scan warp
constexpr u32 kBarWork = 1;                   // named barrier: workers only
constexpr u32 kBarFront = 2;                  // + slot: workers -> scan warp
constexpr u32 kBarExcl = 4;                   // + slot: scan warp -> workers

constexpr u64 kFlagAgg = 1ull;
constexpr u64 kFlagInc = 2ull;
constexpr u64 kPayloadMask = (1ull << 36) - 1ull;
constexpr u32 kSpinLimit = 1u << 21;   // ~2 s with the backoff below

__device__ __forceinline__ void bar_sync(u32 id, u32 n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(u32 id, u32 n) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

__device__ __forceinline__ u64 status_word(u64 flag, u32 epoch, u64 payload) {
    return (flag << 62) | ((u64)(epoch & kEpochMask) << 36) | (payload & kPayloadMask);
}
__device__ __forceinline__ u64 ld_volatile(const u64* p) { return *(const volatile u64*)p; }
__device__ __forceinline__ void st_volatile(u64* p, u64 v) { *(volatile u64*)p = v; }

// Sum of the four bytes of a word.
__device__ __forceinline__ u32 byte_sum(u32 w) { return (u32)__dp4a((int)w, 0x01010101, 0); }
// Byte mask keeping bytes whose bit is set in the low 4 bits of m.
__device__ __forceinline__ u32 byte_mask4(u32 m) {
    return ((m & 1u) ? 0xffu : 0u) | ((m & 2u) ? 0xff00u : 0u) | ((m & 4u) ? 0xff0000u : 0u) |
           ((m & 8u) ? 0xff000000u : 0u);
}

// ---------------------------------------------------------------------------
// Scan elements.  For OnPair codecs only b0 is used (a byte count).  For
// FSST-8 an element maps the state entering a run of slots (1 = its first
// slot is a literal) to the bytes the run produces and the state after it:
//   element(s) = (b[s], n[s]);  "x then y"(s) = (x.b[s] + y.b[x.n[s]], y.n[x.n[s]]).
// TElem holds in-tile values (32-bit); Elem the cross-tile ones (64-bit).
// ---------------------------------------------------------------------------
struct TElem {
    u32 b0, b1, n;
};
struct Elem {
    u64 b0, b1;
    u32 n;
};

__device__ __forceinline__ TElem telem_identity() { return TElem{0u, 0u, 2u}; }
__device__ __forceinline__ Elem elem_identity() { return Elem{0, 0, 2u}; }

template <bool FSST, class E>
__device__ __forceinline__ E then(const E& x, const E& y) {
    if (!FSST) return E{x.b0 + y.b0, 0, 0};
    const u32 x0 = x.n & 1u, x1 = (x.n >> 1) & 1u;
    E r;
    r.b0 = x.b0 + (x0 ? y.b1 : y.b0);
    r.b1 = x.b1 + (x1 ? y.b1 : y.b0);
    r.n = ((y.n >> x0) & 1u) | (((y.n >> x1) & 1u) << 1);
    return r;
}

template <bool FSST, class E>
__device__ __forceinline__ E shfl_up_e(const E& e, int d) {
    E r;
    r.b0 = __shfl_up_sync(0xffffffffu, e.b0, d);
    r.b1 = FSST ? __shfl_up_sync(0xffffffffu, e.b1, d) : 0;
    r.n = FSST ? __shfl_up_sync(0xffffffffu, e.n, d) : 0u;
    return r;
}
template <bool FSST, class E>
__device__ __forceinline__ E shfl_down_e(const E& e, int d) {
    E r;
    r.b0 = __shfl_down_sync(0xffffffffu, e.b0, d);
    r.b1 = FSST ? __shfl_down_sync(0xffffffffu, e.b1, d) : 0;
    r.n = FSST ? __shfl_down_sync(0xffffffffu, e.n, d) : 0u;
    return r;
}
template <bool FSST, class E>
__device__ __forceinline__ E shfl_e(const E& e, int src) {
    E r;
    r.b0 = __shfl_sync(0xffffffffu, e.b0, src);
    r.b1 = FSST ? __shfl_sync(0xffffffffu, e.b1, src) : 0;
    r.n = FSST ? __shfl_sync(0xffffffffu, e.n, src) : 0u;
    return r;
}

// Inclusive warp scan in lane order (= stream order).
template <bool FSST, class E>
__device__ __forceinline__ E warp_scan_incl(E x, u32 lane, E ident) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        E y = shfl_up_e<FSST>(x, d);
        if (lane < (u32)d) y = ident;
        x = then<FSST>(y, x);
    }
    return x;
}

// Tile aggregate <-> 36-bit payload.
template <bool FSST>
__device__ __forceinline__ u64 agg_payload(const TElem& e) {
    if (!FSST) return e.b0;
    return ((u64)e.b0 & 0x1ffffull) | ((u64)(e.n & 1u) << 17) | (((u64)e.b1 & 0x1ffffull) << 18) |
           ((u64)((e.n >> 1) & 1u) << 35);
}
template <bool FSST>
__device__ __forceinline__ Elem agg_unpack(u64 w) {
    if (!FSST) return Elem{w & kPayloadMask, 0, 0};
    Elem e;
    e.b0 = w & 0x1ffffull;
    e.b1 = (w >> 18) & 0x1ffffull;
    e.n = (u32)((w >> 17) & 1u) | ((u32)((w >> 35) & 1u) << 1);
    return e;
}
template <bool FSST>
__device__ __forceinline__ u64 inc_payload(u64 bytes, u32 state) {
    if (!FSST) return bytes & kPayloadMask;
    return (bytes & 0x7ffffffffull) | ((u64)state << 35);
}

// ---------------------------------------------------------------------------
// Decoupled look-back, run by one full warp.  Returns the bytes before the
// tile and (FSST-8) the state entering it.  Waits are bounded: on giving up
// the status word gets ERRB_TIMEOUT and every later wait returns at once.
// ---------------------------------------------------------------------------
template <bool FSST>
__device__ void lookback(const u64* status, long long tile, u32 epoch, WsHeader* ws, u64& excl_bytes,
                         u32& excl_state) {
    const u32 lane = threadIdx.x & 31u;
    Elem acc = elem_identity();
    long long base = tile - 1;
    u32 spins = 0;
    for (;;) {
        const long long idx = base - (long long)lane;
        u64 w = 0;
        u32 flag;
        if (idx < 0) {
            flag = 2u;   // virtual inclusive prefix before the first tile: 0 bytes, state 0
        } else {
            w = ld_volatile(status + idx);
            flag = (u32)(w >> 62);
            if ((u32)((w >> 36) & kEpochMask) != (epoch & kEpochMask)) flag = 0u;
        }
        const u32 inc = __ballot_sync(0xffffffffu, flag == 2u);
        const u32 inv = __ballot_sync(0xffffffffu, flag == 0u);
        const u32 p = inc ? (u32)(__ffs(inc) - 1) : 32u;
        const u32 need = (p >= 31u) ? 0xffffffffu : ((2u << p) - 1u);
        if (inv & need) {
            bool give_up = false;
            if (lane == 0) give_up = (++spins > kSpinLimit) || (*(volatile u32*)&ws->abort != 0u);
            give_up = __shfl_sync(0xffffffffu, give_up, 0);
            if (give_up) {
                if (lane == 0) {
                    atomicOr(&ws->status, ERRB_TIMEOUT);
                    *(volatile u32*)&ws->abort = 1u;
                }
                excl_bytes = 0;
                excl_state = 0;
                return;
            }
            if (lane == 0) __nanosleep(spins < 16 ? 32u : 500u);
            __syncwarp();
            continue;
        }
        // Lanes before p hold aggregates; lane L+1 precedes lane L in the stream.
        Elem f = (lane < p) ? agg_unpack<FSST>(w & kPayloadMask) : elem_identity();
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            Elem o = shfl_down_e<FSST>(f, d);
            if (lane + (u32)d < 32u) f = then<FSST>(o, f);
        }
        const Elem win = shfl_e<FSST>(f, 0);
        acc = then<FSST>(win, acc);
        if (p < 32u) {
            const u64 iw = __shfl_sync(0xffffffffu, w, p);
            const u64 pb = FSST ? (iw & 0x7ffffffffull) : (iw & kPayloadMask);
            const u32 ps = FSST ? (u32)((iw >> 35) & 1u) : 0u;
            excl_bytes = pb + ((FSST && ps) ? acc.b1 : acc.b0);
            excl_state = FSST ? ((acc.n >> ps) & 1u) : 0u;
            return;
        }
        base -= 32;
    }
}

// ---------------------------------------------------------------------------
// Register window: 32 bytes (w[0..7]) aligned to a 16-byte output chunk.
// OR a token of up to 16 bytes (zero padded) in at byte position f < 16.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void or_shifted(u32 (&w)[8], const uint4 t, u32 f) {
    const u32 r = (f & 3u) * 8u;
    const u32 s0 = t.x << r;
    const u32 s1 = __funnelshift_l(t.x, t.y, r);
    const u32 s2 = __funnelshift_l(t.y, t.z, r);
    const u32 s3 = __funnelshift_l(t.z, t.w, r);
    const u32 s4 = __funnelshift_l(t.w, 0u, r);
    const bool q1 = (f & 4u) != 0u;
    const bool q2 = (f & 8u) != 0u;
    const u32 u0 = q1 ? 0u : s0;
    const u32 u1 = q1 ? s0 : s1;
    const u32 u2 = q1 ? s1 : s2;
    const u32 u3 = q1 ? s2 : s3;
    const u32 u4 = q1 ? s3 : s4;
    const u32 u5 = q1 ? s4 : 0u;
    w[0] |= q2 ? 0u : u0;
    w[1] |= q2 ? 0u : u1;
    w[2] |= q2 ? u0 : u2;
    w[3] |= q2 ? u1 : u3;
    w[4] |= q2 ? u2 : u4;
    w[5] |= q2 ? u3 : u5;
    w[6] |= q2 ? u4 : 0u;
    w[7] |= q2 ? u5 : 0u;
}

__device__ __forceinline__ void store_chunk(uint8_t* out, u64 chunk, uint4 v) {
    __stcs(reinterpret_cast<uint4*>(out) + chunk, v);
}

// Write bytes [lo, hi) of a 16-byte chunk with aligned pieces.
__device__ void store_partial(uint8_t* out, u64 chunk, uint4 v, u32 lo, u32 hi) {
    const u32 wv[4] = {v.x, v.y, v.z, v.w};
    uint8_t* base = out + chunk * 16;
    u32 b = lo;
    while (b < hi) {
        if ((b & 7u) == 0u && b + 8 <= hi) {
            *reinterpret_cast<u64*>(base + b) = (u64)wv[b >> 2] | ((u64)wv[(b >> 2) + 1] << 32);
            b += 8;
        } else if ((b & 3u) == 0u && b + 4 <= hi) {
            *reinterpret_cast<u32*>(base + b) = wv[b >> 2];
            b += 4;
        } else if ((b & 1u) == 0u && b + 2 <= hi) {
            *reinterpret_cast<unsigned short*>(base + b) = (unsigned short)(wv[b >> 2] >> ((b & 3u) * 8u));
            b += 2;
        } else {
            base[b] = (uint8_t)(wv[b >> 2] >> ((b & 3u) * 8u));
            b += 1;
        }
    }
}

__device__ __forceinline__ uint4 or4(uint4 a, uint4 b) {
    return make_uint4(a.x | b.x, a.y | b.y, a.z | b.z, a.w | b.w);
}

// Fragment bookkeeping bits (one word per thread).
constexpr u32 FA_VALID = 1u << 0;    // lead (or only) partial chunk present
constexpr u32 FA_LO_SHIFT = 1;       // 5 bits
constexpr u32 FA_HI_SHIFT = 6;       // 5 bits
constexpr u32 FB_VALID = 1u << 11;   // trail partial chunk present
constexpr u32 FB_HI_SHIFT = 12;      // 5 bits

// Per-thread assembly state.
struct Assembler {
    u32 w[8];
    u32 f;          // bytes of the current chunk already filled (incl. predecessors')
    u32 f0;         // first byte of this thread in its first chunk
    u64 cb;         // current chunk index
    u64 cb0;        // first chunk index
    bool head_open; // first chunk is shared with the predecessor and not yet flushed
    uint4 fa, fb;
    u32 meta;

    __device__ __forceinline__ void begin(u64 O) {
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = 0u;
        f0 = (u32)(O & 15u);
        f = f0;
        cb = O >> 4;
        cb0 = cb;
        head_open = (f0 != 0u);
        meta = 0u;
        fa = make_uint4(0, 0, 0, 0);
        fb = make_uint4(0, 0, 0, 0);
    }
    __device__ __forceinline__ void put(uint4 t, u32 len, uint8_t* out) {
        or_shifted(w, t, f);
        f += len;
        if (f >= 16u) {
            const uint4 c = make_uint4(w[0], w[1], w[2], w[3]);
            if (head_open) {
                fa = c;
                meta |= FA_VALID | (f0 << FA_LO_SHIFT) | (16u << FA_HI_SHIFT);
                head_open = false;
            } else {
                store_chunk(out, cb, c);
            }
            w[0] = w[4]; w[1] = w[5]; w[2] = w[6]; w[3] = w[7];
            w[4] = 0u; w[5] = 0u; w[6] = 0u; w[7] = 0u;
            f -= 16u;
            cb += 1;
        }
    }
    // Close the thread's range; `nonempty` = it produced at least one byte.
    __device__ __forceinline__ void finish(bool nonempty) {
        if (!nonempty) return;
        if (head_open) {
            if (f > f0) {
                fa = make_uint4(w[0], w[1], w[2], w[3]);
                meta |= FA_VALID | (f0 << FA_LO_SHIFT) | (f << FA_HI_SHIFT);
            }
        } else if (f > 0u) {
            fb = make_uint4(w[0], w[1], w[2], w[3]);
            meta |= FB_VALID | (f << FB_HI_SHIFT);
        }
    }
};

// Merge a partial chunk with the lead fragments of the following threads and
// store it.  `lo` is the first byte present, `hi` one past the last.
__device__ void combine_and_store(uint8_t* out, u64 chunk, uint4 acc, u32 lo, u32 hi, int m,
                                  const uint4* s_fa, const u32* s_meta) {
    while (hi < 16u && m < kWork) {
        const u32 mm = s_meta[m];
        if (mm & FA_VALID) {
            acc = or4(acc, s_fa[m]);
            hi = (mm >> FA_HI_SHIFT) & 31u;
        }
        ++m;
    }
    if (lo == 0u && hi == 16u) store_chunk(out, chunk, acc);
    else store_partial(out, chunk, acc, lo, hi);
}

// Column extent shared by both kernels.
struct Extent {
    u64 c_begin, c_end, first_tile, n_tiles;
    bool bad;
};
__device__ __forceinline__ Extent column_extent(const DecodeParams& p, u64 tile) {
    Extent x;
    x.c_begin = __ldg(p.code_offsets);
    x.c_end = __ldg(p.code_offsets + p.n_strings);
    x.bad = false;
    if (x.c_end > p.max_slots) { x.c_end = p.max_slots; x.bad = true; }
    if (x.c_begin > x.c_end) { x.c_begin = x.c_end; x.bad = true; }
    x.first_tile = x.c_begin / tile;
    const u64 end_tile = (x.c_end + tile - 1) / tile;
    x.n_tiles = end_tile > x.first_tile ? end_tile - x.first_tile : 1;
    return x;
}

// ---------------------------------------------------------------------------
// Index pass: first[u] = first string boundary owned by tile u (a boundary
// at slot position p belongs to the tile containing p; the column's end
// belongs to the last tile); first[n_tiles] = n_strings + 1.  Also checks
// that code_offsets is non-decreasing and inside the code buffer.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) index_kernel(const DecodeParams p, u32 tile, u32* first) {
    const Extent x = column_extent(p, tile);
    const u64 nb = (u64)p.n_strings + 1;
    u32 err = x.bad ? ERRB_CORRUPT : 0u;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (u64)gridDim.x * blockDim.x) {
        const u64 pos = __ldg(p.code_offsets + i);
        u64 pc = pos < x.c_begin ? x.c_begin : (pos > x.c_end ? x.c_end : pos);
        u64 u = pc / tile - x.first_tile;
        if (u >= x.n_tiles) u = x.n_tiles - 1;
        u64 w0 = 0;
        if (i > 0) {
            const u64 prev = __ldg(p.code_offsets + i - 1);
            if (prev > pos) err |= ERRB_CORRUPT;
            u64 qc = prev < x.c_begin ? x.c_begin : (prev > x.c_end ? x.c_end : prev);
            u64 up = qc / tile - x.first_tile;
            if (up >= x.n_tiles) up = x.n_tiles - 1;
            w0 = up + 1;
        }
        for (u64 w = w0; w <= u; ++w) first[w] = (u32)i;
        if (i == nb - 1)
            for (u64 w = u + 1; w <= x.n_tiles; ++w) first[w] = (u32)nb;
    }
    if (err) atomicOr(&p.ws->status, err);
}

// ---------------------------------------------------------------------------
// Shared memory of a decode block.
// ---------------------------------------------------------------------------
struct Slot {
    TElem wsum[kWorkWarps];   // worker-warp inclusive totals, then exclusive prefixes
    u64 tile_excl;            // bytes before the tile
    u64 tile_incl;            // bytes up to the tile's end
    u32 tile_state;           // FSST-8: state entering the tile
    u32 tile_out_state;       // FSST-8: state after the tile
    u32 ticket;
    u32 lo, hi;               // string boundaries [lo, hi) owned by the tile
};

template <int K, int DICT_BYTES, int LENS_BYTES>
struct Smem {
    uint4 dict[DICT_BYTES ? DICT_BYTES / 16 : 1];
    uint4 fa[kWork];
    uint4 fb[kWork];
    u32 meta[kWork];
    u32 thr_excl[kWork];          // tile-relative output offset of each worker thread
    u32 contrib[K / 4][kWork];    // bytes each slot produced, one byte per slot
    u32 lit_mask[kWork];          // FSST-8: bit k = slot k holds a literal byte
    uint8_t lens[LENS_BYTES ? LENS_BYTES : 16];
    Slot slot[2];
};

// Per-tile registers of a worker thread, kept from front() to back().
template <int CODEC, int K>
struct TileRegs {
    static constexpr int CW = (CODEC == FP_FSST8) ? K / 4 : K / 2;
    u32 c[CW];       // codes: two 16-bit codes per word (OnPair), four bytes per word (FSST-8)
    u32 L[K / 4];    // token length per slot, one byte each
    u32 valid;       // bit k: slot k inside the column's slot range
    TElem lex;       // scan element of the lanes before this one in its warp
    u64 tile_start;
    u32 t;
};

template <int CODEC, int K>
__device__ __forceinline__ u32 code_at(const TileRegs<CODEC, K>& R, int k) {
    if (CODEC == FP_FSST8) return (R.c[k >> 2] >> ((k & 3) * 8)) & 0xffu;
    return (R.c[k >> 1] >> ((k & 1) * 16)) & 0xffffu;
}
template <int CODEC, int K>
__device__ __forceinline__ u32 len_at(const TileRegs<CODEC, K>& R, int k) {
    return (R.L[k >> 2] >> ((k & 3) * 8)) & 0xffu;
}

// ---------------------------------------------------------------------------
// The decode kernel.
// ---------------------------------------------------------------------------
template <int CODEC, int K, bool DSMEM, int MINB>
struct Decoder {
    static constexpr bool FSST = (CODEC == FP_FSST8);
    static constexpr int TILE = kWork * K;
    static constexpr int DICT_BYTES = DSMEM ? (FSST ? 256 * 8 : 4096 * 16) : 0;
    static constexpr int LENS_BYTES = DSMEM ? (FSST ? 256 : 4096) : 0;
    typedef Smem<K, DICT_BYTES, LENS_BYTES> S;
    typedef TileRegs<CODEC, K> R;
    static_assert(K == 8 || K == 16 || K == 32, "slots per thread");
    static_assert(!DSMEM || CODEC != FP_ONPAIR16, "OnPair-16 tables do not fit in shared memory");
    static_assert(!FSST || K >= 16, "FSST-8 loads 16 slots at a time");

    // ---- front: load, unpack, lengths, per-warp scan ----------------------
    static __device__ __forceinline__ bool front(const DecodeParams& p, S& sm, int b, const Extent& x,
                                                 const u32* first, R& r, u32& err) {
        const u32 wtid = threadIdx.x;
        const u32 lane = wtid & 31u;
        const u32 warp = wtid >> 5;
        const u32 t = sm.slot[b].ticket;
        if ((u64)t >= x.n_tiles) {
            __threadfence_block();
            bar_arrive(kBarFront + b, kThreads);
            return false;
        }
        r.t = t;
        r.tile_start = (x.first_tile + t) * (u64)TILE;
        const u64 q0 = r.tile_start + (u64)wtid * K;

        // 1. codes
        if (CODEC == FP_ONPAIR16) {
            if (q0 + K <= p.max_slots) {
#pragma unroll
                for (int v = 0; v < K / 8; ++v) {
                    const uint4 a = __ldcs(reinterpret_cast<const uint4*>(p.codes + 2 * q0) + v);
                    r.c[4 * v + 0] = a.x; r.c[4 * v + 1] = a.y; r.c[4 * v + 2] = a.z; r.c[4 * v + 3] = a.w;
                }
            } else {
#pragma unroll
                for (int m = 0; m < K / 2; ++m) {
                    u32 v = 0;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const u64 q = q0 + 2 * m + h;
                        if (q < p.max_slots) v |= ((u32)p.codes[2 * q] | ((u32)p.codes[2 * q + 1] << 8)) << (16 * h);
                    }
                    r.c[m] = v;
                }
            }
        } else if (CODEC == FP_ONPAIR12) {
            const u64 byte0 = q0 / 8 * 12;
            if (byte0 + 12 * (K / 8) <= p.codes_bytes) {
                u32 wv[3 * (K / 8)];
                if (K >= 16) {
#pragma unroll
                    for (int v = 0; v < 3 * (K / 8) / 2; ++v) {
                        const uint2 a = __ldcs(reinterpret_cast<const uint2*>(p.codes + byte0) + v);
                        wv[2 * v] = a.x; wv[2 * v + 1] = a.y;
                    }
                } else {
#pragma unroll
                    for (int v = 0; v < 3 * (K / 8); ++v) wv[v] = __ldcs(reinterpret_cast<const u32*>(p.codes + byte0) + v);
                }
#pragma unroll
                for (int g = 0; g < K / 8; ++g) {
                    const u32 a = wv[3 * g], bb = wv[3 * g + 1], c = wv[3 * g + 2];
                    r.c[4 * g + 0] = (a & 0xfffu) | (((a >> 12) & 0xfffu) << 16);
                    r.c[4 * g + 1] = (__funnelshift_r(a, bb, 24) & 0xfffu) | (((bb >> 4) & 0xfffu) << 16);
                    r.c[4 * g + 2] = ((bb >> 16) & 0xfffu) | ((__funnelshift_r(bb, c, 28) & 0xfffu) << 16);
                    r.c[4 * g + 3] = ((c >> 8) & 0xfffu) | ((c >> 20) << 16);
                }
            } else {
#pragma unroll
                for (int m = 0; m < K / 2; ++m) {
                    u32 v = 0;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const u64 q = q0 + 2 * m + h;
                        if (q < p.max_slots) {
                            const u64 by = q * 3 / 2;
                            const u32 lo8 = p.codes[by], hi8 = p.codes[by + 1];
                            const u32 c = (q & 1) ? ((lo8 >> 4) | (hi8 << 4)) : (lo8 | ((hi8 & 0xfu) << 8));
                            v |= c << (16 * h);
                        }
                    }
                    r.c[m] = v;
                }
            }
        } else {
            if (q0 + K <= p.max_slots) {
#pragma unroll
                for (int v = 0; v < K / 16; ++v) {
                    const uint4 a = __ldcs(reinterpret_cast<const uint4*>(p.codes + q0) + v);
                    r.c[4 * v + 0] = a.x; r.c[4 * v + 1] = a.y; r.c[4 * v + 2] = a.z; r.c[4 * v + 3] = a.w;
                }
            } else {
#pragma unroll
                for (int m = 0; m < K / 4; ++m) {
                    u32 v = 0;
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const u64 q = q0 + 4 * m + h;
                        if (q < p.max_slots) v |= (u32)p.codes[q] << (8 * h);
                    }
                    r.c[m] = v;
                }
            }
        }

        // 2. slots inside [c_begin, c_end)
        if (q0 >= x.c_begin && q0 + K <= x.c_end) {
            r.valid = (K == 32) ? 0xffffffffu : ((1u << K) - 1u);
        } else {
            u32 v = 0;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const u64 q = q0 + k;
                v |= ((q >= x.c_begin && q < x.c_end) ? 1u : 0u) << k;
            }
            r.valid = v;
        }

        // 3. token lengths
#pragma unroll
        for (int j = 0; j < K / 4; ++j) {
            u32 w = 0;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const u32 code = code_at<CODEC, K>(r, 4 * j + h);
                u32 L;
                if (DSMEM) L = sm.lens[code];
                else L = __ldg(p.dict.lens + code);
                w |= L << (8 * h);
            }
            r.L[j] = w;
        }

        // 4. the thread's scan element
        TElem e;
        if (!FSST) {
            u32 sum = 0;
#pragma unroll
            for (int j = 0; j < K / 4; ++j) {
                const u32 vm = byte_mask4(r.valid >> (4 * j));
                sum += byte_sum(r.L[j] & vm);
                // a valid slot whose code has no token: corrupt input
                if (__vcmpeq4(r.L[j], 0u) & vm) err |= ERRB_CORRUPT;
            }
            e = TElem{sum, 0u, 0u};
        } else {
            // run the slots once per entry state
            u32 c0 = 0, c1 = 0, s0 = 0, s1 = 1;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const bool v = (r.valid >> k) & 1u;
                const u32 bt = code_at<CODEC, K>(r, k);
                const u32 L = len_at<CODEC, K>(r, k);
                const bool is255 = (bt == 255u);
                const u32 a0 = s0 ? 1u : (is255 ? 0u : L);
                const u32 n0 = s0 ? 0u : (is255 ? 1u : 0u);
                const u32 a1 = s1 ? 1u : (is255 ? 0u : L);
                const u32 n1 = s1 ? 0u : (is255 ? 1u : 0u);
                c0 += v ? a0 : 0u;
                c1 += v ? a1 : 0u;
                s0 = v ? n0 : 0u;
                s1 = v ? n1 : 0u;
            }
            e = TElem{c0, c1, s0 | (s1 << 1)};
        }

        // 5. per-warp inclusive scan; warp totals to the slot
        const TElem ident = telem_identity();
        const TElem inc = warp_scan_incl<FSST>(e, lane, ident);
        TElem lex = shfl_up_e<FSST>(inc, 1);
        if (lane == 0) lex = ident;
        r.lex = lex;
        if (lane == 31) sm.slot[b].wsum[warp] = inc;
        if (wtid == 0) {
            const u64 nb = (u64)p.n_strings + 1;
            u32 lo = __ldg(first + t), hi = __ldg(first + t + 1);
            if ((u64)lo > nb) lo = (u32)nb;
            if ((u64)hi > nb) hi = (u32)nb;
            if (hi < lo) hi = lo;
            sm.slot[b].lo = lo;
            sm.slot[b].hi = hi;
        }
        __threadfence_block();
        bar_arrive(kBarFront + b, kThreads);
        return true;
    }

    // ---- back: assemble tile r.t and write its string offsets ------------
    static __device__ __forceinline__ void back(const DecodeParams& p, S& sm, int b, const Extent& x,
                                                const R& r, u32& err) {
        const u32 wtid = threadIdx.x;
        const u32 warp = wtid >> 5;
        bar_sync(kBarExcl + b, kThreads);
        const u64 tile_excl = sm.slot[b].tile_excl;
        const u64 tile_incl = sm.slot[b].tile_incl;
        const u32 s_tile = FSST ? sm.slot[b].tile_state : 0u;
        const u32 lo = sm.slot[b].lo, hi = sm.slot[b].hi;
        const TElem tex = then<FSST>(sm.slot[b].wsum[warp], r.lex);
        const u32 s_in = FSST ? ((tex.n >> s_tile) & 1u) : 0u;
        const u32 thr = FSST ? (s_tile ? tex.b1 : tex.b0) : tex.b0;
        const bool last_tile = ((u64)r.t == x.n_tiles - 1);

        // prefetch the first boundary positions and the next ticket
        u32 pos0 = 0;
        if (lo + wtid < hi) pos0 = __ldg(p.code_offsets + lo + wtid);
        u32 next_ticket = 0;
        if (wtid == 0) next_ticket = atomicAdd(&p.ws->tile_counter, 1u);

        const bool skip = p.size_only || tile_incl > p.capacity;
        Assembler as;
        as.begin(tile_excl + thr);
        u32 produced = 0;
        if (!FSST) {
#pragma unroll
            for (int j = 0; j < K / 4; ++j) {
                const u32 cw = r.L[j] & byte_mask4(r.valid >> (4 * j));
                sm.contrib[j][wtid] = cw;
                produced += byte_sum(cw);
            }
            if (!skip) {
#pragma unroll
                for (int k0 = 0; k0 < K; k0 += 4) {
                    uint4 tok[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const u32 code = code_at<CODEC, K>(r, k0 + h);
                        if (DSMEM) tok[h] = sm.dict[code];
                        else tok[h] = __ldg(reinterpret_cast<const uint4*>(p.dict.table) + code);
                    }
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int k = k0 + h;
                        const bool v = (r.valid >> k) & 1u;
                        as.put(v ? tok[h] : make_uint4(0, 0, 0, 0), v ? len_at<CODEC, K>(r, k) : 0u, p.out);
                    }
                }
            }
        } else {
            u32 s = s_in, lit = 0;
            u32 cw[K / 4];
#pragma unroll
            for (int j = 0; j < K / 4; ++j) cw[j] = 0u;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const bool v = (r.valid >> k) & 1u;
                const u32 bt = code_at<CODEC, K>(r, k);
                lit |= (s & 1u) << k;   // state entering slot k (1 = a literal is due)
                u32 a = 0;
                if (v) {
                    if (s) { a = 1u; s = 0u; }
                    else if (bt == 255u) { s = 1u; }
                    else {
                        a = len_at<CODEC, K>(r, k);
                        if (a == 0u) err |= ERRB_CORRUPT;
                    }
                } else {
                    s = 0u;
                }
                cw[k >> 2] |= a << ((k & 3) * 8);
                produced += a;
            }
#pragma unroll
            for (int j = 0; j < K / 4; ++j) sm.contrib[j][wtid] = cw[j];
            sm.lit_mask[wtid] = lit;
            if (!skip) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const u32 bt = code_at<CODEC, K>(r, k);
                    const u32 a = (cw[k >> 2] >> ((k & 3) * 8)) & 0xffu;
                    const bool is_lit = (lit >> k) & 1u;
                    uint4 tok = make_uint4(0, 0, 0, 0);
                    if (is_lit) {
                        tok.x = bt;
                    } else {
                        uint2 d;
                        if (DSMEM) d = reinterpret_cast<const uint2*>(sm.dict)[bt];
                        else d = __ldg(reinterpret_cast<const uint2*>(p.dict.table) + bt);
                        tok.x = d.x;
                        tok.y = d.y;
                    }
                    as.put(a ? tok : make_uint4(0, 0, 0, 0), a, p.out);
                }
            }
        }
        sm.thr_excl[wtid] = thr;
        as.finish(produced > 0u && !skip);
        sm.fa[wtid] = as.fa;
        sm.fb[wtid] = as.fb;
        sm.meta[wtid] = as.meta;
        bar_sync(kBarWork, kWork);

        // merge chunks shared between threads
        if (!skip && produced > 0u) {
            if (as.meta & FB_VALID)
                combine_and_store(p.out, as.cb, as.fb, 0u, (as.meta >> FB_HI_SHIFT) & 31u, (int)wtid + 1, sm.fa,
                                  sm.meta);
            if ((as.meta & FA_VALID) && thr == 0u)
                combine_and_store(p.out, as.cb0, as.fa, (as.meta >> FA_LO_SHIFT) & 31u,
                                  (as.meta >> FA_HI_SHIFT) & 31u, (int)wtid + 1, sm.fa, sm.meta);
        }

        // string offsets of the boundaries the tile owns
        for (u32 i = lo + wtid; i < hi; i += kWork) {
            const u64 pos = (i == lo + wtid) ? (u64)pos0 : (u64)__ldg(p.code_offsets + i);
            u64 rel = 0;
            u32 st = 0;
            if (pos < r.tile_start || pos > r.tile_start + TILE) {
                err |= ERRB_CORRUPT;
            } else if (pos == r.tile_start + TILE) {
                rel = tile_incl - tile_excl;
                st = FSST ? sm.slot[b].tile_out_state : 0u;
                if (!last_tile) err |= ERRB_CORRUPT;
            } else {
                const u32 sidx = (u32)(pos - r.tile_start);
                const u32 j = sidx / K, k = sidx % K;
                u32 acc = sm.thr_excl[j];
#pragma unroll
                for (int m = 0; m < K / 4; ++m) {
                    const u32 w = sm.contrib[m][j];
                    u32 keep = 0u;
                    if ((u32)m < k / 4) keep = 0xffffffffu;
                    else if ((u32)m == k / 4 && (k & 3u)) keep = 0xffffffffu >> (32 - 8 * (k & 3u));
                    acc += byte_sum(w & keep);
                }
                rel = acc;
                if (FSST) st = (sm.lit_mask[j] >> k) & 1u;
            }
            if (st) err |= ERRB_CORRUPT;   // a string would start on a literal
            if (!p.size_only) __stcs(p.out_offsets + i, (u32)(tile_excl + rel));
        }
        if (wtid == 0) sm.slot[b].ticket = next_ticket;
        bar_sync(kBarWork, kWork);
    }

    // ---- scan warp --------------------------------------------------------
    static __device__ __forceinline__ void scan_loop(const DecodeParams& p, S& sm, const Extent& x, u32 epoch) {
        const u32 lane = threadIdx.x & 31u;
        WsHeader* ws = p.ws;
        for (int b = 0;; b ^= 1) {
            bar_sync(kBarFront + b, kThreads);
            const u32 t = sm.slot[b].ticket;
            if ((u64)t >= x.n_tiles) break;
            const TElem ident = telem_identity();
            const TElem v = (lane < (u32)kWorkWarps) ? sm.slot[b].wsum[lane] : ident;
            const TElem inc = warp_scan_incl<FSST>(v, lane, ident);
            TElem ex = shfl_up_e<FSST>(inc, 1);
            if (lane == 0) ex = ident;
            const TElem tot = shfl_e<FSST>(inc, kWorkWarps - 1);
            if (lane < (u32)kWorkWarps) sm.slot[b].wsum[lane] = ex;
            u64* st = p.tile_status + t;
            u64 excl = 0;
            u32 s_excl = 0;
            if (t != 0) {
                if (lane == 0) st_volatile(st, status_word(kFlagAgg, epoch, agg_payload<FSST>(tot)));
                lookback<FSST>(p.tile_status, (long long)t, epoch, ws, excl, s_excl);
            }
            const u64 inc_b = excl + ((FSST && s_excl) ? tot.b1 : tot.b0);
            const u32 inc_s = FSST ? ((tot.n >> s_excl) & 1u) : 0u;
            if (lane == 0) {
                st_volatile(st, status_word(kFlagInc, epoch, inc_payload<FSST>(inc_b, inc_s)));
                sm.slot[b].tile_excl = excl;
                sm.slot[b].tile_incl = inc_b;
                sm.slot[b].tile_state = s_excl;
                sm.slot[b].tile_out_state = inc_s;
                if (inc_b > p.capacity && !p.size_only) atomicOr(&ws->status, ERRB_CAPACITY);
                if (inc_b > 0x7fffffffull) atomicOr(&ws->status, ERRB_OVERFLOW);
                if ((u64)t == x.n_tiles - 1) ws->total = inc_b;
            }
            __threadfence_block();
            bar_arrive(kBarExcl + b, kThreads);
        }
    }

    static __device__ __forceinline__ void run(const DecodeParams& p, const u32* first) {
        extern __shared__ __align__(16) unsigned char smem_raw[];
        S& sm = *reinterpret_cast<S*>(smem_raw);
        WsHeader* ws = p.ws;
        if (DSMEM) {
            const uint4* src = reinterpret_cast<const uint4*>(p.dict.table);
            for (int i = threadIdx.x; i < DICT_BYTES / 16; i += kThreads) sm.dict[i] = __ldg(src + i);
            const uint4* lsrc = reinterpret_cast<const uint4*>(p.dict.lens);
            for (int i = threadIdx.x; i < LENS_BYTES / 16; i += kThreads)
                reinterpret_cast<uint4*>(sm.lens)[i] = __ldg(lsrc + i);
        }
        if (threadIdx.x == 0) {
            sm.slot[0].ticket = atomicAdd(&ws->tile_counter, 1u);
            sm.slot[1].ticket = atomicAdd(&ws->tile_counter, 1u);
        }
        const u32 epoch = *(volatile u32*)&ws->epoch;
        const Extent x = column_extent(p, TILE);
        __syncthreads();

        u32 err = 0;
        if (threadIdx.x >= (u32)kWork) {
            scan_loop(p, sm, x, epoch);
        } else {
            R ra, rb;
            if (front(p, sm, 0, x, first, ra, err)) {
                for (;;) {
                    const bool hb = front(p, sm, 1, x, first, rb, err);
                    back(p, sm, 0, x, ra, err);
                    if (!hb) break;
                    const bool ha = front(p, sm, 0, x, first, ra, err);
                    back(p, sm, 1, x, rb, err);
                    if (!ha) break;
                }
            }
        }
        if (err) atomicOr(&ws->status, err);

        // last block out: reset the counters for the next launch
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const u32 done = atomicAdd(&ws->exit_counter, 1u);
            if (done == gridDim.x - 1) {
                __threadfence();
                ws->tile_counter = 0;
                ws->exit_counter = 0;
                ws->abort = 0;
                u32 ne = (epoch + 1u) & kEpochMask;
                if (ne == 0u) ne = 1u;
                ws->epoch = ne;
                __threadfence();
            }
        }
    }
};

template <int CODEC, int K, bool DSMEM, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) decode_kernel(const DecodeParams p, const u32* first) {
    Decoder<CODEC, K, DSMEM, MINB>::run(p, first);
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

cudaError_t launch_decode(int codec, const Variant& var, const DecodeParams& p, uint32_t* first, int grid,
                          cudaStream_t stream) {
    (void)codec;
    const uint64_t tile = variant_tile(var);
    const uint64_t nb = (uint64_t)p.n_strings + 1;
    uint64_t ib = (nb + 255) / 256;
    if (ib > 4096) ib = 4096;
    index_kernel<<<(unsigned)ib, 256, 0, stream>>>(p, (u32)tile, first);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const u32* cfirst = first;
    void* args[] = {(void*)&p, (void*)&cfirst};
    return cudaLaunchKernel(var.kernel, dim3(grid), dim3(var.threads), args, var.smem_bytes, stream);
}

}  // namespace fp
