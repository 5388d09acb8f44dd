// Single-pass column decoder for sm_103a.
//
// One launch decodes a whole column (paper Sec. 2.1 semantics) and writes
// Arrow-style output (Sec. 5).  The launch is persistent: each block takes
// tiles of T*K consecutive code slots from an atomic ticket counter and, per
// tile:
//   1. unpacks its K slots per thread (16-bit words, the 12-bit LSB-first
//      bitstream, or FSST-8 bytes) with wide loads;
//   2. gathers token lengths and scans them across the block; FSST-8 tiles
//      scan a two-state element (bytes, next-slot-is-literal) per input state
//      so escapes resolve without knowing the tile's first slot;
//   3. obtains the tile's output position with a single-pass decoupled
//      look-back over earlier tiles (Merrill & Garland, "Single-pass Parallel
//      Prefix Scan with Decoupled Look-back", 2016), replacing the paper's
//      precomputed per-batch sidecar (Sec. 3.1), with a bounded wait;
//   4. assembles each thread's tokens in a 32-byte register window with
//      funnel shifts and writes whole aligned 16-byte chunks straight to
//      global memory; chunks shared between neighbouring threads are merged
//      through shared memory, so only the two chunks at a tile's edges are
//      written piecewise (the paper stages bytes in shared memory and drains
//      them, Algorithm 1);
//   5. writes out_offsets for the strings that start in the tile.
#include <cuda_runtime.h>
#include <cstdint>

#include "fp_internal.h"

namespace fp {
namespace {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr u64 kFlagAgg = 1ull;
constexpr u64 kFlagInc = 2ull;
constexpr u64 kPayloadMask = (1ull << 36) - 1ull;
constexpr u32 kSpinLimit = 1u << 21;   // ~2 s with the backoff below

__device__ __forceinline__ u64 status_word(u64 flag, u32 epoch, u64 payload) {
    return (flag << 62) | ((u64)(epoch & kEpochMask) << 36) | (payload & kPayloadMask);
}

__device__ __forceinline__ u64 ld_volatile(const u64* p) { return *(const volatile u64*)p; }
__device__ __forceinline__ void st_volatile(u64* p, u64 v) { *(volatile u64*)p = v; }

// ---------------------------------------------------------------------------
// Scan element.  For OnPair codecs only b[0] is used (a plain byte count).
// For FSST-8 an element maps the state entering a run of slots (1 = the first
// slot is a literal) to the bytes the run produces and the state after it:
//   element(s) = (b[s], n[s]).
// Composition "x then y": (x;y)(s) = (x.b[s] + y.b[x.n[s]], y.n[x.n[s]]).
// ---------------------------------------------------------------------------
struct Elem {
    u64 b0, b1;
    u32 n;   // bit0 = n[0], bit1 = n[1]
};

__device__ __forceinline__ Elem elem_identity() { return Elem{0, 0, 2u}; }

template <bool FSST>
__device__ __forceinline__ Elem elem_then(const Elem& x, const Elem& y) {
    if (!FSST) return Elem{x.b0 + y.b0, 0, 0};
    u32 x0 = x.n & 1u, x1 = (x.n >> 1) & 1u;
    Elem r;
    r.b0 = x.b0 + (x0 ? y.b1 : y.b0);
    r.b1 = x.b1 + (x1 ? y.b1 : y.b0);
    u32 n0 = (y.n >> x0) & 1u, n1 = (y.n >> x1) & 1u;
    r.n = n0 | (n1 << 1);
    return r;
}

template <bool FSST>
__device__ __forceinline__ Elem elem_shfl_up(const Elem& e, int d) {
    Elem r;
    r.b0 = __shfl_up_sync(0xffffffffu, e.b0, d);
    if (FSST) {
        r.b1 = __shfl_up_sync(0xffffffffu, e.b1, d);
        r.n = __shfl_up_sync(0xffffffffu, e.n, d);
    } else {
        r.b1 = 0;
        r.n = 0;
    }
    return r;
}

template <bool FSST>
__device__ __forceinline__ Elem elem_shfl_down(const Elem& e, int d) {
    Elem r;
    r.b0 = __shfl_down_sync(0xffffffffu, e.b0, d);
    if (FSST) {
        r.b1 = __shfl_down_sync(0xffffffffu, e.b1, d);
        r.n = __shfl_down_sync(0xffffffffu, e.n, d);
    } else {
        r.b1 = 0;
        r.n = 0;
    }
    return r;
}

template <bool FSST>
__device__ __forceinline__ Elem elem_shfl(const Elem& e, int src) {
    Elem r;
    r.b0 = __shfl_sync(0xffffffffu, e.b0, src);
    r.b1 = FSST ? __shfl_sync(0xffffffffu, e.b1, src) : 0;
    r.n = FSST ? __shfl_sync(0xffffffffu, e.n, src) : 0;
    return r;
}

// Inclusive warp scan (lane order = stream order).
template <bool FSST>
__device__ __forceinline__ Elem warp_scan_incl(Elem x, u32 lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        Elem y = elem_shfl_up<FSST>(x, d);
        if (lane >= (u32)d) x = elem_then<FSST>(y, x);
    }
    return x;
}

// Tile aggregate <-> 36-bit payload.
template <bool FSST>
__device__ __forceinline__ u64 agg_payload(const Elem& e) {
    if (!FSST) return e.b0;
    return (e.b0 & 0x1ffffull) | ((u64)(e.n & 1u) << 17) | ((e.b1 & 0x1ffffull) << 18) |
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
// Inclusive prefix (bytes, state after) <-> payload.
template <bool FSST>
__device__ __forceinline__ u64 inc_payload(u64 bytes, u32 state) {
    if (!FSST) return bytes & kPayloadMask;
    return (bytes & 0x7ffffffffull) | ((u64)state << 35);
}

// ---------------------------------------------------------------------------
// Decoupled look-back, run by one full warp.  Returns the bytes before the
// tile and (FSST-8) the state entering it.
// ---------------------------------------------------------------------------
template <bool FSST>
__device__ void lookback(u64* status, long long tile, u32 epoch, WsHeader* ws, u64& excl_bytes,
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
            if (lane == 0) __nanosleep(spins < 32 ? 64u : 1000u);
            __syncwarp();
            continue;
        }
        // Lanes before p hold aggregates (applied after the inclusive one).
        Elem f = (lane < p) ? agg_unpack<FSST>(w & kPayloadMask) : elem_identity();
        // Reduce in stream order: lane L+1 precedes lane L in the stream.
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            Elem o = elem_shfl_down<FSST>(f, d);
            if (lane + (u32)d < 32u) f = elem_then<FSST>(o, f);
        }
        Elem win = elem_shfl<FSST>(f, 0);
        acc = elem_then<FSST>(win, acc);
        if (p < 32u) {
            const u64 iw = __shfl_sync(0xffffffffu, w, p);
            const u64 pb = FSST ? (iw & 0x7ffffffffull) : (iw & kPayloadMask);
            const u32 ps = FSST ? (u32)((iw >> 35) & 1u) : 0u;
            if (FSST) {
                excl_bytes = pb + (ps ? acc.b1 : acc.b0);
                excl_state = (acc.n >> ps) & 1u;
            } else {
                excl_bytes = pb + acc.b0;
                excl_state = 0;
            }
            return;
        }
        base -= 32;
    }
}

// Warp-cooperative lower bound: smallest i in [0, n) with o[i] >= key, or n.
__device__ u64 warp_lower_bound(const u32* __restrict__ o, u64 n, u64 key) {
    const u32 lane = threadIdx.x & 31u;
    u64 lo = 0, hi = n;
    while (hi - lo > 32) {
        const u64 step = (hi - lo + 31) / 32;
        u64 q = lo + (u64)(lane + 1) * step - 1;
        if (q >= hi) q = hi - 1;
        const bool less = (u64)__ldg(o + q) < key;
        const u32 c = __popc(__ballot_sync(0xffffffffu, less));
        const u64 nlo = c ? (((lo + (u64)c * step - 1) < hi ? (lo + (u64)c * step - 1) : hi - 1) + 1) : lo;
        u64 nhi = hi;
        if (c < 32) {
            u64 qc = lo + (u64)(c + 1) * step - 1;
            nhi = qc < hi - 1 ? qc : hi - 1;
        }
        lo = nlo;
        hi = nhi < lo ? lo : nhi;
    }
    const u64 q = lo + lane;
    const bool less = (q < hi) && ((u64)__ldg(o + q) < key);
    return lo + (u64)__popc(__ballot_sync(0xffffffffu, less));
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
    u32 wv[4] = {v.x, v.y, v.z, v.w};
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
            *reinterpret_cast<unsigned short*>(base + b) =
                (unsigned short)(wv[b >> 2] >> ((b & 3u) * 8u));
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
    __device__ __forceinline__ void put(uint4 t, u32 len, uint8_t* out, bool write) {
        or_shifted(w, t, f);
        f += len;
        if (f >= 16u) {
            const uint4 c = make_uint4(w[0], w[1], w[2], w[3]);
            if (head_open) {
                fa = c;
                meta |= FA_VALID | (f0 << FA_LO_SHIFT) | (16u << FA_HI_SHIFT);
                head_open = false;
            } else if (write) {
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
template <int T>
__device__ void combine_and_store(uint8_t* out, u64 chunk, uint4 acc, u32 lo, u32 hi, int m,
                                  const uint4* s_fa, const u32* s_meta) {
    while (hi < 16u && m < T) {
        const u32 mm = s_meta[m];
        if (mm & FA_VALID) {
            acc = or4(acc, s_fa[m]);
            hi = (mm >> FA_HI_SHIFT) & 31u;
        }
        ++m;
    }
    if (lo == 0u && hi == 16u) {
        store_chunk(out, chunk, acc);
    } else {
        store_partial(out, chunk, acc, lo, hi);
    }
}

// Shared-memory layout of a block.
template <int T, int K, int DICT_BYTES, int LENS_BYTES>
struct Smem {
    uint4 dict[DICT_BYTES ? DICT_BYTES / 16 : 1];
    uint4 fa[T];
    uint4 fb[T];
    u32 off[T * K];          // per slot: tile-relative output offset (bit 31: FSST state)
    u32 meta[T];
    uint8_t lens[LENS_BYTES ? LENS_BYTES : 4];
    Elem wsum[T / 32];       // per-warp inclusive element, then exclusive
    u64 lo_string;           // first string boundary owned by the tile
    u64 tile_excl;           // bytes before the tile
    u64 tile_incl;           // bytes up to the tile's end
    u32 tile_state;          // FSST-8: state entering the tile
    u32 tile_out_state;      // FSST-8: state after the tile's last slot
    u32 ticket[2];
};

// ---------------------------------------------------------------------------
// The kernel.  CODEC is FP_ONPAIR16 / FP_ONPAIR12 / FP_FSST8; T threads per
// block; K slots per thread; DSMEM = dictionary staged in shared memory.
// ---------------------------------------------------------------------------
template <int CODEC, int T, int K, bool DSMEM, int MINB>
__global__ void __launch_bounds__(T, MINB) decode_kernel(const DecodeParams p) {
    constexpr bool FSST = (CODEC == FP_FSST8);
    constexpr int TILE = T * K;
    constexpr int NW = T / 32;
    constexpr int DICT_BYTES = DSMEM ? (FSST ? 256 * 8 : 4096 * 16) : 0;
    constexpr int LENS_BYTES = DSMEM ? (FSST ? 256 : 4096) : 0;
    static_assert(K % 8 == 0 && T % 32 == 0 && T >= 128, "tile shape");
    static_assert(!DSMEM || CODEC != FP_ONPAIR16, "OnPair-16 tables do not fit in shared memory");
    typedef Smem<T, K, DICT_BYTES, LENS_BYTES> S;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S& sm = *reinterpret_cast<S*>(smem_raw);

    const u32 tid = threadIdx.x;
    const u32 lane = tid & 31u;
    const u32 wid = tid >> 5;
    WsHeader* ws = p.ws;

    if (DSMEM) {
        const uint4* src = reinterpret_cast<const uint4*>(p.dict.table);
        for (int i = tid; i < DICT_BYTES / 16; i += T) sm.dict[i] = __ldg(src + i);
        const uint4* lsrc = reinterpret_cast<const uint4*>(p.dict.lens);
        for (int i = tid; i < LENS_BYTES / 16; i += T)
            reinterpret_cast<uint4*>(sm.lens)[i] = __ldg(lsrc + i);
    }

    const u32 epoch = *(volatile u32*)&ws->epoch;
    const u64 n_bounds = (u64)p.n_strings + 1;
    const u64 c_begin = __ldg(p.code_offsets);
    u64 c_end = __ldg(p.code_offsets + p.n_strings);
    bool bad_range = false;
    if (c_end > p.max_slots) { c_end = p.max_slots; bad_range = true; }
    if (c_end < c_begin) { c_end = c_begin; bad_range = true; }
    const u64 first_tile = c_begin / TILE;
    const u64 end_tile = (c_end + TILE - 1) / TILE;
    const u64 n_tiles = end_tile > first_tile ? end_tile - first_tile : 1;
    if (bad_range && blockIdx.x == 0 && tid == 0) atomicOr(&ws->status, ERRB_CORRUPT);

    if (tid == 0) sm.ticket[0] = atomicAdd(&ws->tile_counter, 1u);
    __syncthreads();

    u32 err = 0;
    for (u32 it = 0;; ++it) {
        const u64 t = sm.ticket[it & 1u];
        if (t >= n_tiles) break;
        const u64 tile_start = (first_tile + t) * (u64)TILE;
        const bool last_tile = (t == n_tiles - 1);
        const u64 q0 = tile_start + (u64)tid * K;

        // ---- 1. unpack this thread's K slots -----------------------------
        u32 code[K];
        if (CODEC == FP_ONPAIR16) {
            if (q0 + K <= p.max_slots) {
#pragma unroll
                for (int v = 0; v < K / 8; ++v) {
                    const uint4 x = __ldcs(reinterpret_cast<const uint4*>(p.codes + 2 * q0) + v);
                    code[8 * v + 0] = x.x & 0xffffu; code[8 * v + 1] = x.x >> 16;
                    code[8 * v + 2] = x.y & 0xffffu; code[8 * v + 3] = x.y >> 16;
                    code[8 * v + 4] = x.z & 0xffffu; code[8 * v + 5] = x.z >> 16;
                    code[8 * v + 6] = x.w & 0xffffu; code[8 * v + 7] = x.w >> 16;
                }
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const u64 q = q0 + k;
                    code[k] = q < p.max_slots ? ((u32)p.codes[2 * q] | ((u32)p.codes[2 * q + 1] << 8)) : 0u;
                }
            }
        } else if (CODEC == FP_ONPAIR12) {
            const u64 byte0 = q0 / 8 * 12;
            if (byte0 + 12 * (K / 8) <= p.codes_bytes) {
#pragma unroll
                for (int v = 0; v < K / 8; ++v) {
                    const u32* src = reinterpret_cast<const u32*>(p.codes + byte0) + 3 * v;
                    const u32 a = __ldcs(src), b = __ldcs(src + 1), c = __ldcs(src + 2);
                    code[8 * v + 0] = a & 0xfffu;
                    code[8 * v + 1] = (a >> 12) & 0xfffu;
                    code[8 * v + 2] = __funnelshift_r(a, b, 24) & 0xfffu;
                    code[8 * v + 3] = (b >> 4) & 0xfffu;
                    code[8 * v + 4] = (b >> 16) & 0xfffu;
                    code[8 * v + 5] = __funnelshift_r(b, c, 28) & 0xfffu;
                    code[8 * v + 6] = (c >> 8) & 0xfffu;
                    code[8 * v + 7] = c >> 20;
                }
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const u64 q = q0 + k;
                    u32 c = 0;
                    if (q < p.max_slots) {
                        const u64 by = q * 3 / 2;
                        const u32 lo8 = p.codes[by], hi8 = p.codes[by + 1];
                        c = (q & 1) ? ((lo8 >> 4) | (hi8 << 4)) : (lo8 | ((hi8 & 0xfu) << 8));
                    }
                    code[k] = c;
                }
            }
        } else {
            if (q0 + K <= p.max_slots) {
#pragma unroll
                for (int v = 0; v < K / 16; ++v) {
                    const uint4 x = __ldcs(reinterpret_cast<const uint4*>(p.codes + q0) + v);
                    const u32 wv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                    for (int j = 0; j < 16; ++j) code[16 * v + j] = (wv[j >> 2] >> ((j & 3) * 8)) & 0xffu;
                }
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) code[k] = (q0 + k < p.max_slots) ? (u32)p.codes[q0 + k] : 0u;
            }
        }

        // ---- 2. lengths and the thread's scan element ---------------------
        u32 lens_packed[K / 4];   // token length per slot, one byte each
#pragma unroll
        for (int k = 0; k < K / 4; ++k) lens_packed[k] = 0u;
        u32 valid_mask = 0;       // bit k: slot inside [c_begin, c_end)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const u64 q = q0 + k;
            const bool v = (q >= c_begin) && (q < c_end);
            valid_mask |= (v ? 1u : 0u) << k;
            u32 L;
            if (DSMEM) L = sm.lens[code[k]];
            else L = __ldg(p.dict.lens + code[k]);
            lens_packed[k >> 2] |= L << ((k & 3) * 8);
        }
        auto len_of = [&](int k) -> u32 { return (lens_packed[k >> 2] >> ((k & 3) * 8)) & 0xffu; };

        Elem e;
        if (!FSST) {
            u32 sum = 0;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const bool v = (valid_mask >> k) & 1u;
                const u32 L = len_of(k);
                if (v && L == 0u) err |= ERRB_CORRUPT;
                sum += v ? L : 0u;
            }
            e = Elem{sum, 0, 0};
        } else {
            // Run the slots once per entry state.
            u32 cnt[2], nxt[2];
#pragma unroll
            for (int s_in = 0; s_in < 2; ++s_in) {
                u32 s = (u32)s_in, c = 0;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const bool v = (valid_mask >> k) & 1u;
                    const u32 b = code[k];
                    if (!v) { s = 0u; continue; }
                    if (s) { c += 1u; s = 0u; }
                    else if (b == 255u) { s = 1u; }
                    else { c += len_of(k); }
                }
                cnt[s_in] = c;
                nxt[s_in] = s;
            }
            e = Elem{cnt[0], cnt[1], nxt[0] | (nxt[1] << 1)};
        }

        // ---- 3. block scan + look-back ----------------------------------
        const Elem incl = warp_scan_incl<FSST>(e, lane);
        Elem lane_excl = elem_shfl_up<FSST>(incl, 1);
        if (lane == 0) lane_excl = elem_identity();
        if (lane == 31) sm.wsum[wid] = incl;
        __syncthreads();   // (A)

        if (wid == 0) {
            Elem x = (lane < (u32)NW) ? sm.wsum[lane] : elem_identity();
            const Elem xi = warp_scan_incl<FSST>(x, lane);
            Elem xe = elem_shfl_up<FSST>(xi, 1);
            if (lane == 0) xe = elem_identity();
            const Elem tot = elem_shfl<FSST>(xi, NW - 1);
            __syncwarp();
            if (lane < (u32)NW) sm.wsum[lane] = xe;
            // publish, look back, publish the inclusive prefix
            u64* st = p.tile_status + t;
            u64 excl = 0;
            u32 s_excl = 0;
            if (t == 0) {
                excl = 0;
                s_excl = 0;
            } else {
                if (lane == 0) st_volatile(st, status_word(kFlagAgg, epoch, agg_payload<FSST>(tot)));
                lookback<FSST>(p.tile_status, (long long)t, epoch, ws, excl, s_excl);
            }
            const u64 inc_b = excl + (FSST ? (s_excl ? tot.b1 : tot.b0) : tot.b0);
            const u32 inc_s = FSST ? ((tot.n >> s_excl) & 1u) : 0u;
            if (lane == 0) {
                st_volatile(st, status_word(kFlagInc, epoch, inc_payload<FSST>(inc_b, inc_s)));
                sm.tile_excl = excl;
                sm.tile_incl = inc_b;
                sm.tile_state = s_excl;
                sm.tile_out_state = inc_s;
                if (inc_b > p.capacity && !p.size_only) atomicOr(&ws->status, ERRB_CAPACITY);
                if (inc_b > 0x7fffffffull) atomicOr(&ws->status, ERRB_OVERFLOW);
                if (last_tile) ws->total = inc_b;
            }
        } else if (wid == (u32)NW - 1) {
            const u64 lo = (t == 0) ? 0 : warp_lower_bound(p.code_offsets, n_bounds, tile_start);
            if (lane == 0) sm.lo_string = lo;
        } else if (wid == 1 && lane == 0) {
            sm.ticket[(it + 1) & 1u] = atomicAdd(&ws->tile_counter, 1u);
        }
        __syncthreads();   // (B)

        const u64 tile_excl = sm.tile_excl;
        const u32 s_tile = FSST ? sm.tile_state : 0u;
        const Elem wexcl = sm.wsum[wid];
        const Elem tex = elem_then<FSST>(wexcl, lane_excl);   // everything before this thread
        const u32 s_in = FSST ? ((tex.n >> s_tile) & 1u) : 0u;
        const u64 thr_excl = FSST ? (s_tile ? tex.b1 : tex.b0) : tex.b0;
        const u64 tile_incl = sm.tile_incl;
        // A tile whose end passes the capacity writes no bytes (the status word
        // already carries ERRB_CAPACITY), so every write stays in bounds.
        const bool skip_writes = p.size_only || tile_incl > p.capacity;

        // ---- 4. per-slot offsets and assembly ------------------------------
        Assembler as;
        const u64 O = tile_excl + thr_excl;
        as.begin(O);
        u32 produced = 0;
        if (!FSST) {
            u32 rel = (u32)thr_excl;
            u32 offs[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                offs[k] = rel;
                const bool v = (valid_mask >> k) & 1u;
                rel += v ? len_of(k) : 0u;
            }
#pragma unroll
            for (int k = 0; k < K; k += 4)
                *reinterpret_cast<uint4*>(&sm.off[tid * K + k]) = make_uint4(offs[k], offs[k + 1], offs[k + 2], offs[k + 3]);
            produced = rel - (u32)thr_excl;
        }
        if (!FSST) {
            if (!skip_writes) {
#pragma unroll
                for (int k0 = 0; k0 < K; k0 += 8) {
                    uint4 tok[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int k = k0 + j;
                        const bool v = (valid_mask >> k) & 1u;
                        uint4 x;
                        if (DSMEM) x = sm.dict[code[k]];
                        else x = __ldg(reinterpret_cast<const uint4*>(p.dict.table) + code[k]);
                        tok[j] = v ? x : make_uint4(0, 0, 0, 0);
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int k = k0 + j;
                        const bool v = (valid_mask >> k) & 1u;
                        as.put(tok[j], v ? len_of(k) : 0u, p.out, true);
                    }
                }
            }
        } else {
            u32 s = s_in;
            u32 rel = (u32)thr_excl;
            u32 offs[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                offs[k] = rel | (s << 31);
                const bool v = (valid_mask >> k) & 1u;
                const u32 b = code[k];
                if (!v) { s = 0u; continue; }
                if (s) { rel += 1u; s = 0u; }
                else if (b == 255u) { s = 1u; }
                else {
                    const u32 L = len_of(k);
                    if (L == 0u) err |= ERRB_CORRUPT;
                    rel += L;
                }
            }
#pragma unroll
            for (int k = 0; k < K; k += 4)
                *reinterpret_cast<uint4*>(&sm.off[tid * K + k]) = make_uint4(offs[k], offs[k + 1], offs[k + 2], offs[k + 3]);
            produced = rel - (u32)thr_excl;
            if (!skip_writes) {
                s = s_in;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const bool v = (valid_mask >> k) & 1u;
                    const u32 b = code[k];
                    uint4 tok = make_uint4(0, 0, 0, 0);
                    u32 L = 0;
                    if (v) {
                        if (s) { tok.x = b; L = 1u; s = 0u; }
                        else if (b == 255u) { s = 1u; }
                        else {
                            uint2 x;
                            if (DSMEM) x = reinterpret_cast<const uint2*>(sm.dict)[b];
                            else x = __ldg(reinterpret_cast<const uint2*>(p.dict.table) + b);
                            tok.x = x.x; tok.y = x.y;
                            L = len_of(k);
                        }
                    } else {
                        s = 0u;
                    }
                    as.put(tok, L, p.out, true);
                }
            }
        }
        as.finish(produced > 0u && !skip_writes);
        sm.fa[tid] = as.fa;
        sm.fb[tid] = as.fb;
        sm.meta[tid] = as.meta;
        __syncthreads();   // (C)

        // ---- merge partial chunks ------------------------------------------
        if (!skip_writes && produced > 0u) {
            if (as.meta & FB_VALID) {
                const u32 hi = (as.meta >> FB_HI_SHIFT) & 31u;
                combine_and_store<T>(p.out, as.cb, as.fb, 0u, hi, tid + 1, sm.fa, sm.meta);
            }
            if ((as.meta & FA_VALID) && thr_excl == 0) {
                const u32 lo = (as.meta >> FA_LO_SHIFT) & 31u;
                const u32 hi = (as.meta >> FA_HI_SHIFT) & 31u;
                combine_and_store<T>(p.out, as.cb0, as.fa, lo, hi, tid + 1, sm.fa, sm.meta);
            }
        }

        // ---- 5. string boundaries owned by the tile -------------------------
        {
            const u64 key_end = last_tile ? c_end + 1 : tile_start + TILE;
            u64 lo = sm.lo_string;
            u64 covered = 0;
            for (;;) {
                const u64 i = lo + tid;
                bool mine = false;
                if (i < n_bounds) {
                    const u64 pos = __ldg(p.code_offsets + i);
                    mine = pos < key_end;
                    if (mine) {
                        u32 rel;
                        u32 st;
                        if (pos < tile_start) {
                            err |= ERRB_CORRUPT;
                            rel = 0; st = 0;
                        } else if (pos - tile_start >= (u64)TILE) {
                            // boundary at the very end of the last tile
                            rel = (u32)(tile_incl - tile_excl);
                            st = FSST ? sm.tile_out_state : 0u;
                        } else {
                            const u32 w = sm.off[pos - tile_start];
                            rel = FSST ? (w & 0x7fffffffu) : w;
                            st = FSST ? (w >> 31) : 0u;
                        }
                        if (st) err |= ERRB_CORRUPT;   // a string would start on a literal
                        if (i > 0 && __ldg(p.code_offsets + i - 1) > pos) err |= ERRB_CORRUPT;
                        if (!p.size_only) __stcs(p.out_offsets + i, (u32)(tile_excl + rel));
                    }
                }
                const int cnt = __syncthreads_count(mine);
                covered += (u64)cnt;
                if (cnt < T) break;
                lo += T;
            }
            if (tid == 0 && covered) atomicAdd(&ws->covered, covered);
        }
    }

    if (err) atomicOr(&ws->status, err);

    // ---- last block out: final checks and reset for the next launch --------
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const u32 done = atomicAdd(&ws->exit_counter, 1u);
        if (done == gridDim.x - 1) {
            __threadfence();
            const u64 cov = atomicAdd(&ws->covered, 0ull);
            if (cov != n_bounds) atomicOr(&ws->status, ERRB_CORRUPT);
            ws->covered = 0;
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

}  // namespace

// ---------------------------------------------------------------------------
// Variant tables
// ---------------------------------------------------------------------------
template <int CODEC, int T, int K, bool DSMEM, int MINB>
static Variant make_variant() {
    constexpr bool FSST = (CODEC == FP_FSST8);
    constexpr int DICT_BYTES = DSMEM ? (FSST ? 256 * 8 : 4096 * 16) : 0;
    constexpr int LENS_BYTES = DSMEM ? (FSST ? 256 : 4096) : 0;
    return Variant{T, K, DSMEM ? 1 : 0, sizeof(Smem<T, K, DICT_BYTES, LENS_BYTES>),
                   (const void*)&decode_kernel<CODEC, T, K, DSMEM, MINB>};
}

static const Variant* table_for(int codec, int* n) {
    static const Variant v16[] = {
        make_variant<FP_ONPAIR16, 256, 8, false, 2>(),
        make_variant<FP_ONPAIR16, 256, 16, false, 2>(),
    };
    static const Variant v12[] = {
        make_variant<FP_ONPAIR12, 256, 8, true, 2>(),
        make_variant<FP_ONPAIR12, 256, 8, false, 2>(),
        make_variant<FP_ONPAIR12, 256, 16, true, 2>(),
    };
    static const Variant v8[] = {
        make_variant<FP_FSST8, 256, 16, true, 2>(),
        make_variant<FP_FSST8, 256, 32, true, 2>(),
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

cudaError_t launch_decode(int codec, const Variant& var, const DecodeParams& p, int grid,
                          cudaStream_t stream) {
    (void)codec;
    void* args[] = {(void*)&p};
    return cudaLaunchKernel(var.kernel, dim3(grid), dim3(var.threads), args, var.smem_bytes, stream);
}

}  // namespace fp
