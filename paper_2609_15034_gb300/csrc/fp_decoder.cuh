// The decode pipeline shared by the single-column and the batched kernels.
//
// One stream-ordered call decodes a whole column (paper Sec. 2.1 semantics)
// into Arrow-style output (Sec. 5) with two launches:
//
//   index_kernel   one pass over code_offsets: validates it and records, for
//                  every tile of 256*K code slots, the first string boundary
//                  at or after the tile's start;
//   decode_kernel  persistent; tiles are taken from an atomic ticket counter.
//
// A decode block has 8 worker warps, 1 scan warp and 1 producer warp, and a
// ring of three tile slots in shared memory:
//
//   producer: on the workers' request (made when they start assembling a
//       tile, for the tile after next) takes a ticket and bulk-copies (TMA
//       engine, cp.async.bulk) the tile's code bytes and its window of
//       code_offsets into the slot; completion is tracked by an mbarrier;
//   workers, front(t+1): unpack codes from the slot (16-bit words, the
//       12-bit LSB-first bitstream, FSST-8 bytes), gather token lengths,
//       per-warp scan; the last warp publishes the tile aggregate; arrive
//       on FRONT[slot];
//   scan warp: block scan of the warp totals, decoupled look-back over
//       earlier tiles (Merrill & Garland, "Single-pass Parallel Prefix Scan
//       with Decoupled Look-back", 2016) with bounded waits, publish the
//       inclusive prefix; arrive on EXCL[slot];
//   workers, back(t): assemble each thread's K tokens in registers with
//       funnel shifts and store whole aligned 16-byte chunks; chunks shared
//       by neighbouring threads are merged through shared memory; write
//       out_offsets of the strings that start in the tile; release the slot.
//
// So input latency, the look-back of tile t, and the assembly of tile t-1
// overlap.  The paper instead reads stored per-batch output positions (a
// sidecar, Sec. 3.1) and stages output bytes in shared memory before a
// coalesced drain (Algorithm 1).
//
// FSST-8 escapes: each thread computes the bytes and exit state of its slots
// for both possible entry states (is the first slot a literal?) with a
// bit-parallel run resolution; the scans compose these two-state elements,
// so escape parity crosses thread and tile boundaries through the same scan
// and look-back.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "fp_internal.h"

namespace fp {
namespace {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr int kWorkWarps = 8;
constexpr int kWork = kWorkWarps * 32;        // worker threads per block
constexpr int kThreads = kWork + 64;          // + the scan warp and the producer warp
constexpr int kPair = kWork + 32;             // threads on the FRONT/EXCL barriers: workers + scan warp
constexpr u32 kBarWork = 1;                   // named barrier: workers only
constexpr u32 kBarFront = 2;                  // + slot (3): workers -> scan warp
constexpr u32 kBarExcl = 5;                   // + slot (3): scan warp -> workers

constexpr u64 kFlagAgg = 1ull;
constexpr u64 kFlagInc = 2ull;
constexpr u64 kPayloadMask = (1ull << 36) - 1ull;
constexpr u32 kSpinLimit = 1u << 20;   // about a second with the backoff below

// Named barriers in their non-aligned form (barrier.sync / barrier.arrive);
// each call first reconverges its warp.
__device__ __forceinline__ void bar_sync(u32 id, u32 n) {
    __syncwarp();
    asm volatile("barrier.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(u32 id, u32 n) {
    __syncwarp();
    asm volatile("barrier.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the kernel before it on the stream still
// runs; grid_wait() returns once that kernel has completed and its writes
// are visible (at once for a kernel launched without the attribute), and
// grid_release() lets the next kernel start launching.
__device__ __forceinline__ void grid_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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
// Aggregates of large tiles (up to 2^29 bytes).  For FSST-8 the two byte
// counts of an element differ by at most 8 -- the two parses of a slot range
// (entered on a code or on a literal) produce the same bytes from the first
// slot where they meet, and before that only an alternating run of 0xFF
// slots (one byte per two slots in both) and one token-versus-literal step
// -- so b1 is stored as a 5-bit difference from b0.
template <bool FSST>
__device__ __forceinline__ u64 agg_payload_wide(const Elem& e) {
    if (!FSST) return e.b0 & kPayloadMask;
    const u64 d = (u64)((long long)e.b1 - (long long)e.b0 + 16) & 31ull;
    return (e.b0 & 0x1fffffffull) | (d << 29) | ((u64)(e.n & 3u) << 34);
}
template <bool FSST>
__device__ __forceinline__ Elem agg_unpack_wide(u64 w) {
    if (!FSST) return Elem{w & kPayloadMask, 0, 0};
    Elem e;
    e.b0 = w & 0x1fffffffull;
    e.b1 = (u64)((long long)e.b0 + (long long)((w >> 29) & 31ull) - 16);
    e.n = (u32)((w >> 34) & 3ull);
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
template <bool FSST, bool WIDE = false>
__device__ void lookback(const u64* status, long long tile, u32 epoch, WsHeader* ws, u64& excl_bytes,
                         u32& excl_state) {
    // Each lane reads 4 consecutive status words, so one round trip to L2
    // covers 128 predecessors: lane L holds tiles base-4L .. base-4L-3.
    constexpr int V = 4;
    const u32 lane = threadIdx.x & 31u;
    Elem acc = elem_identity();
    long long base = tile - 1;
    u32 spins = 0;
    const u32 lim = *(volatile u32*)&ws->spin_limit;
    const u32 limit = lim ? lim : kSpinLimit;
    for (;;) {
        u64 w[V];
        u32 fl[V];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const long long idx = base - (long long)(V * lane + j);
            if (idx < 0) {
                w[j] = 0;
                fl[j] = 2u;   // virtual inclusive prefix before the first tile: 0 bytes, state 0
            } else {
                w[j] = ld_volatile(status + idx);
                fl[j] = (u32)(w[j] >> 62);
                if ((u32)((w[j] >> 36) & kEpochMask) != (epoch & kEpochMask)) fl[j] = 0u;
            }
        }
        // first inclusive word in stream-backward order, per lane and over the warp
        u32 jinc = V;
#pragma unroll
        for (int j = V - 1; j >= 0; --j)
            if (fl[j] == 2u) jinc = (u32)j;
        const u32 inc = __ballot_sync(0xffffffffu, jinc < (u32)V);
        const u32 p = inc ? (u32)(__ffs(inc) - 1) : 32u;
        // every word before the first inclusive one must be published
        bool missing = false;
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const bool before = (lane < p) || (lane == p && (u32)j < jinc);
            if (before && fl[j] == 0u) missing = true;
        }
        if (__any_sync(0xffffffffu, missing)) {
            bool give_up = false;
            if (lane == 0) give_up = (++spins > limit) || (*(volatile u32*)&ws->abort != 0u);
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
            if (spins > 8 && lane == 0) __nanosleep(spins < 64 ? 64u : 500u);
            __syncwarp();
            continue;
        }
        // compose this lane's aggregates, oldest first (j = V-1 is the oldest)
        Elem f = elem_identity();
#pragma unroll
        for (int j = V - 1; j >= 0; --j) {
            const bool use = (lane < p) || (lane == p && (u32)j < jinc);
            if (use) f = then<FSST>(f, WIDE ? agg_unpack_wide<FSST>(w[j] & kPayloadMask)
                                            : agg_unpack<FSST>(w[j] & kPayloadMask));
        }
        // then across lanes: lane L+1 precedes lane L in the stream
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            Elem o = shfl_down_e<FSST>(f, d);
            if (lane + (u32)d < 32u) f = then<FSST>(o, f);
        }
        const Elem win = shfl_e<FSST>(f, 0);
        acc = then<FSST>(win, acc);
        if (p < 32u) {
            u64 mine = 0;
#pragma unroll
            for (int j = 0; j < V; ++j)
                if ((u32)j == jinc) mine = w[j];
            const u64 iw = __shfl_sync(0xffffffffu, mine, p);
            const u64 pb = FSST ? (iw & 0x7ffffffffull) : (iw & kPayloadMask);
            const u32 ps = FSST ? (u32)((iw >> 35) & 1u) : 0u;
            excl_bytes = pb + ((FSST && ps) ? acc.b1 : acc.b0);
            excl_state = FSST ? ((acc.n >> ps) & 1u) : 0u;
            return;
        }
        base -= 32 * V;
    }
}

// ---------------------------------------------------------------------------
// Grid barrier of a cooperative launch (every block resident): the last
// block to arrive resets the count and advances the generation the others
// wait on.  The wait is bounded like the look-back's: on giving up the
// status word gets ERRB_TIMEOUT, the abort flag is set (later barriers of the
// launch then pass at once) and the block carries on; its later writes stay
// in bounds.  Every thread of the block calls it.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void grid_barrier(WsHeader* ws) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile u32* gen = &ws->bar_gen;
        const u32 g = *gen;
        __threadfence();
        if (atomicAdd(&ws->bar_count, 1u) == gridDim.x - 1) {
            atomicExch(&ws->bar_count, 0u);
            __threadfence();
            atomicAdd(&ws->bar_gen, 1u);
        } else {
            const u32 lim = *(volatile u32*)&ws->spin_limit;
            const u32 limit = lim ? lim : kSpinLimit;
            u32 spins = 0;
            while (*gen == g) {
                if (++spins > limit || *(volatile u32*)&ws->abort != 0u) {
                    atomicOr(&ws->status, ERRB_TIMEOUT);
                    *(volatile u32*)&ws->abort = 1u;
                    break;
                }
                if (spins > 8) __nanosleep(spins < 64 ? 64u : 500u);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// A token of up to 16 bytes (zero padded, words t.x..t.w) moved to byte
// position f < 16 of a 32-byte span: s[0..7] = the span's words.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void shift_token(const uint4 t, u32 f, u32 (&s)[8]) {
    const bool q1 = (f & 4u) != 0u;
    const bool q2 = (f & 8u) != 0u;
    const u32 r = (f & 3u) * 8u;
    // whole-word moves by (f >> 2) words, then a funnel shift by r bits
    const u32 v0 = q1 ? 0u : t.x, v1 = q1 ? t.x : t.y, v2 = q1 ? t.y : t.z, v3 = q1 ? t.z : t.w,
              v4 = q1 ? t.w : 0u;
    const u32 x0 = q2 ? 0u : v0, x1 = q2 ? 0u : v1, x2 = q2 ? v0 : v2, x3 = q2 ? v1 : v3, x4 = q2 ? v2 : v4,
              x5 = q2 ? v3 : 0u, x6 = q2 ? v4 : 0u;
    s[0] = x0 << r;
    s[1] = __funnelshift_l(x0, x1, r);
    s[2] = __funnelshift_l(x1, x2, r);
    s[3] = __funnelshift_l(x2, x3, r);
    s[4] = __funnelshift_l(x3, x4, r);
    s[5] = __funnelshift_l(x4, x5, r);
    s[6] = __funnelshift_l(x5, x6, r);
    s[7] = __funnelshift_l(x6, 0u, r);
}

// Write bytes [lo, hi) of a 16-byte chunk with aligned pieces.
__device__ void store_partial(uint8_t* base, uint4 v, u32 lo, u32 hi) {
    const u32 wv[4] = {v.x, v.y, v.z, v.w};
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

// Per-thread assembly state: the current 16-byte output chunk c[0..3] and
// how many of its bytes are filled (including a predecessor's bytes when the
// thread's output starts inside the chunk).  When the thread's first chunk
// is shared with its predecessor, that chunk is stored into the thread's
// head slot in shared memory instead of global memory; `tgt` points at
// wherever the current chunk goes, so each insert stores through one
// pointer and needs no test of which chunk it completes.
struct Assembler {
    u32 c[4];
    u32 f;          // filled bytes of the current chunk
    u32 f0;         // first byte of this thread in its first chunk
    uint4* g;       // current chunk in global memory
    uint4* dst0;    // first chunk in global memory
    uint4* tgt;     // where the current chunk is stored when it completes
    uint4* head;    // the thread's head slot (shared memory, generic address)
    uint4 fb;
    u32 meta;

    __device__ __forceinline__ void begin(uint8_t* out, u64 O, uint4* head_slot) {
        c[0] = c[1] = c[2] = c[3] = 0u;
        f0 = (u32)(O & 15u);
        f = f0;
        g = reinterpret_cast<uint4*>(out) + (O >> 4);
        dst0 = g;
        head = head_slot;
        tgt = f0 != 0u ? head_slot : g;
        meta = 0u;
        fb = make_uint4(0, 0, 0, 0);
    }
    // Append a token (zero padded beyond len).  When the chunk completes it is
    // stored and the token's overflow starts the next chunk.  No branches:
    // every step runs the same instructions.
    __device__ __forceinline__ void put(uint4 t, u32 len) {
        u32 s[8];
        shift_token(t, f, s);
        f += len;
        const bool fl = f >= 16u;
        const uint4 full = make_uint4(c[0] | s[0], c[1] | s[1], c[2] | s[2], c[3] | s[3]);
        if (fl) *tgt = full;
        g += fl ? 1 : 0;
        tgt = fl ? g : tgt;
        c[0] = fl ? s[4] : full.x;
        c[1] = fl ? s[5] : full.y;
        c[2] = fl ? s[6] : full.z;
        c[3] = fl ? s[7] : full.w;
        f &= 15u;   // below 16 before the insert, below 32 after it
    }
    // Append a token of at most 8 bytes given already moved up by (f & 3)
    // bytes (y0..y2, zero elsewhere): only whole-word moves remain, no
    // funnel shifts.  Same stores and chunk handling as put().
    __device__ __forceinline__ void put3(u32 y0, u32 y1, u32 y2, u32 len) {
        const bool q1 = (f & 4u) != 0u;
        const bool q2 = (f & 8u) != 0u;
        const u32 v0 = q1 ? 0u : y0, v1 = q1 ? y0 : y1, v2 = q1 ? y1 : y2, v3 = q1 ? y2 : 0u;
        const u32 s0 = q2 ? 0u : v0, s1 = q2 ? 0u : v1, s2 = q2 ? v0 : v2, s3 = q2 ? v1 : v3, s4 = q2 ? v2 : 0u,
                  s5 = q2 ? v3 : 0u;
        f += len;
        const bool fl = f >= 16u;
        const uint4 full = make_uint4(c[0] | s0, c[1] | s1, c[2] | s2, c[3] | s3);
        if (fl) *tgt = full;
        g += fl ? 1 : 0;
        tgt = fl ? g : tgt;
        c[0] = fl ? s4 : full.x;
        c[1] = fl ? s5 : full.y;
        c[2] = fl ? 0u : full.z;
        c[3] = fl ? 0u : full.w;
        f &= 15u;
    }
    // Close the thread's range; `nonempty` = it produced at least one byte.
    // Afterwards the head slot holds the thread's lead fragment (FA_VALID).
    __device__ __forceinline__ void finish(bool nonempty) {
        if (!nonempty) return;
        const bool head_shared = f0 != 0u;
        const bool head_open = head_shared && tgt == head;   // the first chunk never completed
        if (head_shared && !head_open) meta |= FA_VALID | (f0 << FA_LO_SHIFT) | (16u << FA_HI_SHIFT);
        if (head_open) {
            if (f > f0) {
                *head = make_uint4(c[0], c[1], c[2], c[3]);
                meta |= FA_VALID | (f0 << FA_LO_SHIFT) | (f << FA_HI_SHIFT);
            }
        } else if (f > 0u) {
            fb = make_uint4(c[0], c[1], c[2], c[3]);
            meta |= FB_VALID | (f << FB_HI_SHIFT);
        }
    }
};

// Merge a partial chunk with the lead fragments of the following threads and
// store it.  `lo` is the first byte present, `hi` one past the last.
__device__ void combine_and_store(uint4* chunk, uint4 acc, u32 lo, u32 hi, int m,
                                  const uint4* s_fa, const u32* s_meta) {
    while (hi < 16u && m < kWork) {
        const u32 mm = s_meta[m];
        if (mm & FA_VALID) {
            acc = or4(acc, s_fa[m]);
            hi = (mm >> FA_HI_SHIFT) & 31u;
        }
        ++m;
    }
    if (lo == 0u && hi == 16u) __stcs(chunk, acc);
    else store_partial(reinterpret_cast<uint8_t*>(chunk), acc, lo, hi);
}

// The column's slot range [c_begin, c_end) from code_offsets[0] and
// code_offsets[n], clamped to the code buffer (x.bad when it had to be).
__device__ __forceinline__ void slot_range(const DecodeParams& p, Extent& x) {
    x.c_begin = __ldg(p.code_offsets);
    x.c_end = __ldg(p.code_offsets + p.n_strings);
    x.bad = 0u;
    if (x.c_end > p.max_slots) { x.c_end = p.max_slots; x.bad = 1u; }
    if (x.c_begin > x.c_end) { x.c_begin = x.c_end; x.bad = 1u; }
}

// Single-column tiling: the tiles that cover [c_begin, c_end).
__device__ __forceinline__ Extent column_extent(const DecodeParams& p, u64 tile) {
    Extent x;
    slot_range(p, x);
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
// Boundary i (at slot `pos`, boundary i-1 at `prev`): the tiles from the one
// after prev's tile up to pos's tile start their first string at i.  Tiles
// are a power of two slots long (1 << tile_log2).
// Slot positions are code_offsets values (32-bit), so is c_end (clamped
// to one), and tile indices are below 2^32.
__device__ __forceinline__ void index_one(const Extent& x, u32 tile_log2, u64 nb, u64 i, u32 pos, u32 prev,
                                          u32* first, u32& err) {
    const u32 cb = (u32)x.c_begin, ce = (u32)x.c_end, ft = (u32)x.first_tile, nt = (u32)x.n_tiles;
    const u32 pc = pos < cb ? cb : (pos > ce ? ce : pos);
    u32 u = (pc >> tile_log2) - ft;
    if (u >= nt) u = nt - 1;
    u32 w0 = 0;
    if (i > 0) {
        if (prev > pos) err |= ERRB_CORRUPT;
        const u32 qc = prev < cb ? cb : (prev > ce ? ce : prev);
        u32 up = (qc >> tile_log2) - ft;
        if (up >= nt) up = nt - 1;
        w0 = up + 1;
    }
    for (u32 w = w0; w <= u; ++w) first[w] = (u32)i;
    if (i == nb - 1)
        for (u64 w = (u64)u + 1; w <= x.n_tiles; ++w) first[w] = (u32)nb;
}

// Boundaries [g * 8, g * 8 + 8) for groups g = g0, g0 + gstep, ... : a
// thread's nine code_offsets loads are in flight together.
constexpr int kIdxGroup = 8;
__device__ __forceinline__ void index_groups(const DecodeParams& p, const Extent& x, u32 tile_log2, u64 i_begin,
                                             u64 i_end, u64 g0, u64 gstep, u32* first) {
    const u64 nb = (u64)p.n_strings + 1;
    if (i_end > nb) i_end = nb;
    u32 err = x.bad ? ERRB_CORRUPT : 0u;
    for (u64 i0 = i_begin + g0 * kIdxGroup; i0 < i_end; i0 += gstep * kIdxGroup) {
        u32 v[kIdxGroup + 1];
#pragma unroll
        for (int k = 0; k <= kIdxGroup; ++k) {
            const u64 i = i0 + k - 1;   // v[0] is boundary i0 - 1
            v[k] = (k > 0 || i0 > 0) && i < i_end ? __ldg(p.code_offsets + i) : 0u;
        }
#pragma unroll
        for (int k = 0; k < kIdxGroup; ++k)
            if (i0 + k < i_end) index_one(x, tile_log2, nb, i0 + k, v[k + 1], v[k], first, err);
    }
    if (err) atomicOr(p.err_word, err);
}

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA engine) and mbarriers, in inline PTX.
// ---------------------------------------------------------------------------
__device__ __forceinline__ u32 smem_u32(const void* p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ u64 global_timer_ns() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(u64* bar, u32 count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(u64* bar, u32 bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(u64* bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(u64* bar, u32 parity) {
    u32 ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0u;
}
// Copy `bytes` (a multiple of 16, both addresses 16-byte aligned) from global
// to shared memory; completion is counted on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, u32 bytes, u64* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Bounded mbarrier waits give up after 4 s: well after any look-back has
// given up (kSpinLimit), so a wait that a look-back holds up never expires
// first.  The abort flag does not end them: once a look-back has given up
// the pipeline still runs to its end (with wrong positions, every write in
// bounds), so the workers, the scan warp and the producer keep seeing the
// same ring state and every named barrier stays matched.
constexpr u64 kWaitLimitNs = 4000000000ull;

// Wait for a phase of `bar`; gives up (status ERRB_TIMEOUT, abort flag) after
// kWaitLimitNs.  Returns false on giving up.
__device__ bool mbar_wait(u64* bar, u32 parity, WsHeader* ws) {
    if (mbar_try_wait(bar, parity)) return true;
    const u64 t0 = global_timer_ns();
    for (u32 i = 0;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 63u) {
            if (global_timer_ns() - t0 > kWaitLimitNs) {
                atomicOr(&ws->status, ERRB_TIMEOUT);
                *(volatile u32*)&ws->abort = 1u;
                return false;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// FSST-8 escapes, bit-parallel.  E has bit k set when slot k holds 0xFF;
// s = 1 when slot 0 is a literal (the slot before the run was an escape
// code).  Returns the literal slots and the escape-code slots: inside a run
// of 0xFF slots that starts on a code, codes and literals alternate, and the
// slot after the run is a literal exactly when the run has odd length
// counted from that code.  The carry of a subtraction propagates along each
// run (the same device scanners of JSON use for backslash runs).
// ---------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void fsst_escapes(u32 E, u32 s, u32& lit, u32& esc) {
    constexpr u32 M = (N == 32) ? 0xffffffffu : ((1u << N) - 1u);
    constexpr u32 ODD = 0xaaaaaaaau & M;
    const u32 pot = E & ~s & M;                    // slots that may be escape codes
    const u32 t = (((pot << 1) | ODD) - pot) & M;
    const u32 tc = t ^ ODD;
    lit = (tc ^ (E | s)) & M;
    esc = tc & E & M;
}

// 0xFF-byte mask of four bytes -> 4-bit mask (bit k = byte k is 0xFF).
__device__ __forceinline__ u32 ff_bits4(u32 w) {
    const u32 eq = __vcmpeq4(w, 0xffffffffu) & 0x01010101u;
    return (eq * 0x01020408u) >> 24;
}
// 4-bit mask -> 0x01 in byte k when bit k is set.
__device__ __forceinline__ u32 ones_of4(u32 m) { return ((m & 0xfu) * 0x00204081u) & 0x01010101u; }
// 4-bit mask -> byte mask (byte k = 0xFF when bit k is set).
__device__ __forceinline__ u32 bytes_of4(u32 m) { return ones_of4(m) * 0xffu; }
// acc + sum of the bytes of w whose 0x01 marker in `ones` is set.
__device__ __forceinline__ u32 masked_byte_sum(u32 w, u32 ones, u32 acc) { return __dp4a(w, ones, acc); }
// Does any byte of w equal zero?
__device__ __forceinline__ bool has_zero_byte(u32 w) {
    return ((w - 0x01010101u) & ~w & 0x80808080u) != 0u;
}

// ---------------------------------------------------------------------------
// Shared memory of a decode block.
// ---------------------------------------------------------------------------
constexpr int kSlots = 3;      // ring of tiles in flight: produced, scanned, assembled
constexpr int kOffCap = 512;   // code_offsets entries copied per tile (more are read from global)

struct Ring {
    u64 full;                 // mbarrier: tile inputs landed (producer arrival + copy bytes)
    u64 req;                  // mbarrier: workers ask the producer to fill the slot
    TElem wsum[kWorkWarps];   // worker-warp inclusive totals, then exclusive prefixes
    u64 tile_excl;            // bytes before the tile
    u64 tile_incl;            // bytes up to the tile's end
    u32 tile_state;           // FSST-8: state entering the tile
    u32 tile_out_state;       // FSST-8: state after the tile
    u32 tile;                 // tile index within its column
    u32 stop;                 // 1: no tile (the work is exhausted); the pipeline ends here
    u32 lo, hi;               // string boundaries [lo, hi) owned by the tile
    u32 off_base, off_count;  // code_offsets[off_base, off_base + off_count) are in offbuf
    u32 codes_in_smem;        // 0: the tile's codes are read from global memory
    u32 nready;               // worker warps that finished front() for this tile
};

template <int CODE_BYTES, int K, int DICT_BYTES, int LENS_BYTES, int NSRC>
struct Smem {
    SlotSrc src[NSRC];   // batched decode: the record of each slot's chunk
    uint4 dict[DICT_BYTES ? DICT_BYTES / 16 : 1];
    uint4 lens4[LENS_BYTES ? LENS_BYTES / 16 : 1];   // token length table (bytes), staged with 16-byte stores
    uint4 codebuf[kSlots][CODE_BYTES / 16];
    u32 offbuf[kSlots][kOffCap];
    uint4 fa[kWork];
    uint4 fb[kWork];
    u32 meta[kWork];
    u32 thr_excl[kWork];          // tile-relative output offset of each worker thread
    u32 contrib[K / 4][kWork];    // bytes each slot produced, one byte per slot
    u32 lit_mask[kWork];          // FSST-8: bit k = slot k holds a literal byte
    Ring ring[kSlots];
};

__device__ __forceinline__ int next_slot(int s) { return s + 1 == kSlots ? 0 : s + 1; }

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
// The decode kernel: 8 worker warps, a scan warp and a producer warp.
// ---------------------------------------------------------------------------
// Last block out: reset the ticket counters for the next launch and advance
// the launch tag of the look-back words.  Called by every thread after the
// block's last __syncthreads().
__device__ __forceinline__ void finish_launch(WsHeader* ws, u32 epoch) {
    if (threadIdx.x == 0) {
        __threadfence();
        const u32 done = atomicAdd(&ws->exit_counter, 1u);
        if (done == gridDim.x - 1) {
            __threadfence();
            ws->tile_counter = 0;
            ws->queue_counter[0] = 0;
            ws->queue_counter[1] = 0;
            ws->queue_counter[2] = 0;
            ws->exit_counter = 0;
            ws->abort = 0;
            ws->spin_limit = 0;
            ws->bar_count = 0;
            u32 ne = (epoch + 1u) & kEpochMask;
            if (ne == 0u) ne = 1u;
            ws->epoch = ne;
            __threadfence();
        }
    }
}

// Where front/back/scan find the column of a ring slot: the kernel's
// parameters (one column) or the slot's chunk record in shared memory.
struct OneColumn {
    const DecodeParams& p;
    const Extent& x;
    __device__ __forceinline__ const DecodeParams& P(int) const { return p; }
    __device__ __forceinline__ const Extent& X(int) const { return x; }
};
struct SlotColumns {
    const SlotSrc* src;
    __device__ __forceinline__ const DecodeParams& P(int s) const { return src[s].p; }
    __device__ __forceinline__ const Extent& X(int s) const { return src[s].x; }
};

template <int CODEC, int K, bool DSMEM, int MINB, bool BATCH = false>
struct Decoder {
    static constexpr bool FSST = (CODEC == FP_FSST8);
    static constexpr int TILE = kWork * K;
    static constexpr int WBITS = (CODEC == FP_ONPAIR16) ? 16 : (CODEC == FP_ONPAIR12 ? 12 : 8);
    static constexpr int CODE_BYTES = TILE * WBITS / 8;
    static constexpr int DICT_BYTES = DSMEM ? (FSST ? 256 * 8 : 4096 * 16) : 0;
    static constexpr int LENS_BYTES = DSMEM ? (FSST ? 256 : 4096) : 0;
    typedef Smem<CODE_BYTES, K, DICT_BYTES, LENS_BYTES, BATCH ? kSlots : 1> S;
    typedef TileRegs<CODEC, K> R;
    static_assert(K == 8 || K == 16 || K == 32, "slots per thread");
    static_assert(CODE_BYTES % 16 == 0, "tile code bytes must allow 16-byte bulk copies");
    static_assert(!DSMEM || CODEC != FP_ONPAIR16, "OnPair-16 tables do not fit in shared memory");
    static_assert(!FSST || K >= 16, "FSST-8 loads 16 slots at a time");
    // Members accessed with 16-byte vector operations or bulk copies must be
    // 16-byte aligned (the block's shared memory base is); the ring holds
    // 64-bit words and mbarriers (8 bytes).
    static_assert(!BATCH || !DSMEM, "batched chunks read their dictionaries through the L1 cache");
    static_assert(offsetof(S, src) % 16 == 0 && offsetof(S, dict) % 16 == 0 && offsetof(S, lens4) % 16 == 0 && offsetof(S, codebuf) % 16 == 0 && offsetof(S, offbuf) % 16 == 0 &&
                      offsetof(S, fa) % 16 == 0 && offsetof(S, fb) % 16 == 0 && offsetof(S, ring) % 8 == 0 &&
                      (sizeof(u32) * kOffCap) % 16 == 0,
                  "shared-memory layout alignment");

    static __device__ __forceinline__ u32 full_mask() { return K == 32 ? 0xffffffffu : ((1u << K) - 1u); }

    // ---- codes of this thread: from the shared-memory copy or from global --
    static __device__ __forceinline__ void codes_from_smem(const S& sm, int s, u32 wtid, R& r) {
        if (CODEC == FP_ONPAIR16) {
            const uint4* src = reinterpret_cast<const uint4*>(sm.codebuf[s]) + wtid * (K / 8);
#pragma unroll
            for (int v = 0; v < K / 8; ++v) {
                const uint4 a = src[v];
                r.c[4 * v + 0] = a.x; r.c[4 * v + 1] = a.y; r.c[4 * v + 2] = a.z; r.c[4 * v + 3] = a.w;
            }
        } else if (CODEC == FP_ONPAIR12) {
            u32 wv[3 * (K / 8)];
            if (K >= 16) {
                const uint2* src = reinterpret_cast<const uint2*>(sm.codebuf[s]) + wtid * (3 * (K / 8) / 2);
#pragma unroll
                for (int v = 0; v < 3 * (K / 8) / 2; ++v) {
                    const uint2 a = src[v];
                    wv[2 * v] = a.x; wv[2 * v + 1] = a.y;
                }
            } else {
                const u32* src = reinterpret_cast<const u32*>(sm.codebuf[s]) + wtid * 3;
#pragma unroll
                for (int v = 0; v < 3; ++v) wv[v] = src[v];
            }
            unpack12(wv, r);
        } else {
            const uint4* src = reinterpret_cast<const uint4*>(sm.codebuf[s]) + wtid * (K / 16);
#pragma unroll
            for (int v = 0; v < K / 16; ++v) {
                const uint4 a = src[v];
                r.c[4 * v + 0] = a.x; r.c[4 * v + 1] = a.y; r.c[4 * v + 2] = a.z; r.c[4 * v + 3] = a.w;
            }
        }
    }

    static __device__ __forceinline__ void unpack12(const u32 (&wv)[3 * (K / 8)], R& r) {
#pragma unroll
        for (int g = 0; g < K / 8; ++g) {
            const u32 a = wv[3 * g], bb = wv[3 * g + 1], c = wv[3 * g + 2];
            r.c[4 * g + 0] = (a & 0xfffu) | (((a >> 12) & 0xfffu) << 16);
            r.c[4 * g + 1] = (__funnelshift_r(a, bb, 24) & 0xfffu) | (((bb >> 4) & 0xfffu) << 16);
            r.c[4 * g + 2] = ((bb >> 16) & 0xfffu) | ((__funnelshift_r(bb, c, 28) & 0xfffu) << 16);
            r.c[4 * g + 3] = ((c >> 8) & 0xfffu) | ((c >> 20) << 16);
        }
    }

    // Guarded global loads (tiles at the end of the code buffer).
    static __device__ __forceinline__ void codes_from_global(const DecodeParams& p, u64 q0, R& r) {
        if (CODEC == FP_ONPAIR16) {
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
        } else if (CODEC == FP_ONPAIR12) {
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

    // FSST-8: 0xFF mask of the thread's slots.
    static __device__ __forceinline__ u32 ff_mask(const R& r) {
        u32 E = 0;
#pragma unroll
        for (int j = 0; j < K / 4; ++j) E |= ff_bits4(r.c[j]) << (4 * j);
        return E;
    }
    // FSST-8: bytes produced by the code slots in `codes` plus one per literal.
    static __device__ __forceinline__ u32 fsst_bytes(const R& r, u32 codes, u32 lits) {
        u32 n = __popc(lits);
#pragma unroll
        for (int j = 0; j < K / 4; ++j) n += byte_sum(r.L[j] & bytes_of4(codes >> (4 * j)));
        return n;
    }

    // ---- front: inputs, lengths, per-warp scan ---------------------------
    // `p` and `x` may live in the slot (batched decode): nothing reads them
    // before the slot's inputs have landed.
    static __device__ __forceinline__ bool front(const DecodeParams& p, S& sm, int s, u32 ph, const Extent& x,
                                                 u32 epoch, WsHeader* ws, R& r, u32& err) {
        const u32 wtid = threadIdx.x;
        const u32 lane = wtid & 31u;
        const u32 warp = wtid >> 5;
        Ring& rg = sm.ring[s];
        mbar_wait(&rg.full, ph, ws);
        if (rg.stop) {
            __threadfence_block();
            bar_arrive(kBarFront + s, kPair);
            return false;
        }
        const u32 t = rg.tile;
        r.t = t;
        r.tile_start = (x.first_tile + t) * (u64)TILE;
        const u64 q0 = r.tile_start + (u64)wtid * K;

        // 1. codes
        if (rg.codes_in_smem) codes_from_smem(sm, s, wtid, r);
        else codes_from_global(p, q0, r);

        // 2. slots inside [c_begin, c_end)
        if (q0 >= x.c_begin && q0 + K <= x.c_end) {
            r.valid = full_mask();
        } else {
            u32 v = 0;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const u64 q = q0 + k;
                v |= ((q >= x.c_begin && q < x.c_end) ? 1u : 0u) << k;
            }
            r.valid = v;
        }
        const bool allv = (r.valid == full_mask());

        // 3. token lengths
#pragma unroll
        for (int j = 0; j < K / 4; ++j) {
            u32 w = 0;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const u32 code = code_at<CODEC, K>(r, 4 * j + h);
                u32 L;
                if (DSMEM) L = reinterpret_cast<const uint8_t*>(sm.lens4)[code];
                else L = __ldg(p.dict.lens + code);
                w |= L << (8 * h);
            }
            r.L[j] = w;
        }

        // 4. the thread's scan element
        TElem e;
        if (!FSST) {
            u32 sum = 0;
            if (allv) {
                bool zero = false;
#pragma unroll
                for (int j = 0; j < K / 4; ++j) {
                    sum += byte_sum(r.L[j]);
                    zero |= has_zero_byte(r.L[j]);
                }
                if (zero) err |= ERRB_CORRUPT;   // a code without a token
            } else {
#pragma unroll
                for (int j = 0; j < K / 4; ++j) {
                    const u32 vm = bytes_of4(r.valid >> (4 * j));
                    sum += byte_sum(r.L[j] & vm);
                    if (__vcmpeq4(r.L[j], 0u) & vm) err |= ERRB_CORRUPT;
                }
            }
            e = TElem{sum, 0u, 0u};
        } else if (allv) {
            const u32 E = ff_mask(r);
            u32 lit0, esc0, lit1, esc1;
            fsst_escapes<K>(E, 0u, lit0, esc0);
            fsst_escapes<K>(E, 1u, lit1, esc1);
            const u32 c0 = fsst_bytes(r, ~(lit0 | esc0) & full_mask(), lit0);
            const u32 c1 = fsst_bytes(r, ~(lit1 | esc1) & full_mask(), lit1);
            e = TElem{c0, c1, ((esc0 >> (K - 1)) & 1u) | (((esc1 >> (K - 1)) & 1u) << 1)};
        } else {
            // slots outside the column reset the state (the column starts on a code)
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

        // 5. per-warp inclusive scan; warp totals to the ring slot
        const TElem ident = telem_identity();
        const TElem inc = warp_scan_incl<FSST>(e, lane, ident);
        TElem lex = shfl_up_e<FSST>(inc, 1);
        if (lane == 0) lex = ident;
        r.lex = lex;
        if (lane == 31) rg.wsum[warp] = inc;
        // The last worker warp to get here publishes the tile aggregate at
        // once, so later tiles' look-backs never wait on this block's scan warp.
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            const u32 prior = atomicAdd(&rg.nready, 1u);
            if (prior == (u32)kWorkWarps - 1) {
                __threadfence_block();
                volatile TElem* ws_v = rg.wsum;
                TElem tot = ident;
#pragma unroll
                for (int w = 0; w < kWorkWarps; ++w) {
                    const TElem e2{ws_v[w].b0, ws_v[w].b1, ws_v[w].n};
                    tot = then<FSST>(tot, e2);
                }
                if (t != 0) st_volatile(p.tile_status + t, status_word(kFlagAgg, epoch, agg_payload<FSST>(tot)));
                rg.nready = 0u;
            }
        }
        if (err) {
            atomicOr(p.err_word, err);
            err = 0u;
        }
        __threadfence_block();
        bar_arrive(kBarFront + s, kPair);
        return true;
    }

    template <bool ALLV>
    static __device__ __forceinline__ void assemble_onpair(const DecodeParams& p, S& sm, const R& r, Assembler& as) {
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
                if (ALLV) {
                    as.put(tok[h], len_at<CODEC, K>(r, k));
                } else {
                    const bool v = (r.valid >> k) & 1u;
                    as.put(v ? tok[h] : make_uint4(0, 0, 0, 0), v ? len_at<CODEC, K>(r, k) : 0u);
                }
            }
        }
    }

    // ---- back: assemble tile r.t and write its string offsets ------------
    static __device__ __forceinline__ void back(const DecodeParams& p, S& sm, int s, const Extent& x, const R& r,
                                                u32& err) {
        const u32 wtid = threadIdx.x;
        const u32 warp = wtid >> 5;
        Ring& rg = sm.ring[s];
        bar_sync(kBarExcl + s, kPair);
        const u64 tile_excl = rg.tile_excl;
        const u64 tile_incl = rg.tile_incl;
        const u32 s_tile = FSST ? rg.tile_state : 0u;
        const u32 lo = rg.lo, hi = rg.hi;
        const u32 off_base = rg.off_base, off_count = rg.off_count;
        const TElem tex = then<FSST>(rg.wsum[warp], r.lex);
        const u32 s_in = FSST ? ((tex.n >> s_tile) & 1u) : 0u;
        const u32 thr = FSST ? (s_tile ? tex.b1 : tex.b0) : tex.b0;
        const bool last_tile = ((u64)r.t == x.n_tiles - 1);
        const bool allv = (r.valid == full_mask());
        // Ask the producer for the tile after next: it goes into the slot the
        // previous tile used, which is free now.  Taking its ticket only now
        // keeps every ticketed tile at most one step from publishing its
        // aggregate, so look-backs elsewhere rarely wait on it.
        if (wtid == 0) mbar_arrive(&sm.ring[next_slot(next_slot(s))].req);
        __syncwarp();

        const bool skip = p.size_only || tile_incl > p.capacity;
        Assembler as;
        as.begin(p.out, tile_excl + thr, &sm.fa[wtid]);
        u32 produced = 0;
        if (!FSST) {
#pragma unroll
            for (int j = 0; j < K / 4; ++j) {
                const u32 cw = allv ? r.L[j] : (r.L[j] & bytes_of4(r.valid >> (4 * j)));
                sm.contrib[j][wtid] = cw;
                produced += byte_sum(cw);
            }
            if (!skip) {
                if (allv) assemble_onpair<true>(p, sm, r, as);
                else assemble_onpair<false>(p, sm, r, as);
            }
        } else {
            u32 lit = 0;
            u32 cw[K / 4];
            if (allv) {
                u32 esc;
                fsst_escapes<K>(ff_mask(r), s_in, lit, esc);
                const u32 code_slots = ~(lit | esc) & full_mask();
#pragma unroll
                for (int j = 0; j < K / 4; ++j) {
                    cw[j] = (r.L[j] & bytes_of4(code_slots >> (4 * j))) | (bytes_of4(lit >> (4 * j)) & 0x01010101u);
                    if (has_zero_byte(r.L[j] | ~bytes_of4(code_slots >> (4 * j)))) err |= ERRB_CORRUPT;
                    produced += byte_sum(cw[j]);
                }
            } else {
                u32 st = s_in;
#pragma unroll
                for (int j = 0; j < K / 4; ++j) cw[j] = 0u;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const bool v = (r.valid >> k) & 1u;
                    const u32 bt = code_at<CODEC, K>(r, k);
                    lit |= (st & 1u) << k;   // state entering slot k (1 = a literal is due)
                    u32 a = 0;
                    if (v) {
                        if (st) { a = 1u; st = 0u; }
                        else if (bt == 255u) { st = 1u; }
                        else {
                            a = len_at<CODEC, K>(r, k);
                            if (a == 0u) err |= ERRB_CORRUPT;
                        }
                    } else {
                        st = 0u;
                    }
                    cw[k >> 2] |= a << ((k & 3) * 8);
                    produced += a;
                }
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
                    uint2 d;
                    if (DSMEM) d = reinterpret_cast<const uint2*>(sm.dict)[bt];
                    else d = __ldg(reinterpret_cast<const uint2*>(p.dict.table) + bt);
                    // literal: the byte itself; escape code or outside the column: nothing
                    const uint4 tok =
                        make_uint4(a == 0u ? 0u : (is_lit ? bt : d.x), (a == 0u || is_lit) ? 0u : d.y, 0u, 0u);
                    as.put(tok, a);
                }
            }
        }
        sm.thr_excl[wtid] = thr;
        as.finish(produced > 0u && !skip);
        sm.meta[wtid] = as.meta;
        bar_sync(kBarWork, kWork);

        // merge chunks shared between threads
        if (!skip && produced > 0u) {
            if (as.meta & FB_VALID)
                combine_and_store(as.g, as.fb, 0u, (as.meta >> FB_HI_SHIFT) & 31u, (int)wtid + 1, sm.fa, sm.meta);
            if ((as.meta & FA_VALID) && thr == 0u)
                combine_and_store(as.dst0, sm.fa[wtid], (as.meta >> FA_LO_SHIFT) & 31u,
                                  (as.meta >> FA_HI_SHIFT) & 31u, (int)wtid + 1, sm.fa, sm.meta);
        }

        // string offsets of the boundaries the tile owns
        for (u32 i = lo + wtid; i < hi; i += kWork) {
            const u32 rel_i = i - off_base;
            const u64 pos = (i >= off_base && rel_i < off_count) ? (u64)sm.offbuf[s][rel_i]
                                                                   : (u64)__ldg(p.code_offsets + i);
            u64 rel = 0;
            u32 st = 0;
            if (pos < r.tile_start || pos > r.tile_start + TILE) {
                err |= ERRB_CORRUPT;
            } else if (pos == r.tile_start + TILE) {
                rel = tile_incl - tile_excl;
                st = FSST ? rg.tile_out_state : 0u;
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
        if (err) {
            atomicOr(p.err_word, err);
            err = 0u;
        }
        bar_sync(kBarWork, kWork);
    }

    // ---- scan warp --------------------------------------------------------
    template <class SRC>
    static __device__ __forceinline__ void scan_loop(const SRC& src, S& sm, u32 epoch, WsHeader* ws) {
        const u32 lane = threadIdx.x & 31u;
        for (int s = 0;; s = next_slot(s)) {
            bar_sync(kBarFront + s, kPair);
            Ring& rg = sm.ring[s];
            if (rg.stop) break;
            const DecodeParams& p = src.P(s);
            const Extent& x = src.X(s);
            const u32 t = rg.tile;
            const TElem ident = telem_identity();
            const TElem v = (lane < (u32)kWorkWarps) ? rg.wsum[lane] : ident;
            const TElem inc = warp_scan_incl<FSST>(v, lane, ident);
            TElem ex = shfl_up_e<FSST>(inc, 1);
            if (lane == 0) ex = ident;
            const TElem tot = shfl_e<FSST>(inc, kWorkWarps - 1);
            if (lane < (u32)kWorkWarps) rg.wsum[lane] = ex;
            u64 excl = 0;
            u32 s_excl = 0;
            if (t != 0) lookback<FSST>(p.tile_status, (long long)t, epoch, ws, excl, s_excl);
            const u64 inc_b = excl + ((FSST && s_excl) ? tot.b1 : tot.b0);
            const u32 inc_s = FSST ? ((tot.n >> s_excl) & 1u) : 0u;
            if (lane == 0) {
                st_volatile(p.tile_status + t, status_word(kFlagInc, epoch, inc_payload<FSST>(inc_b, inc_s)));
                rg.tile_excl = excl;
                rg.tile_incl = inc_b;
                rg.tile_state = s_excl;
                rg.tile_out_state = inc_s;
                if (inc_b > p.capacity && !p.size_only) atomicOr(p.err_word, ERRB_CAPACITY);
                if (inc_b > 0x7fffffffull) atomicOr(p.err_word, ERRB_OVERFLOW);
                if ((u64)t == x.n_tiles - 1) *p.total_out = inc_b;
            }
            __threadfence_block();
            bar_arrive(kBarExcl + s, kPair);
        }
    }

    // ---- producer: tickets, then bulk copies of each tile's inputs --------
    // Fill ring slot s with tile t of column (p, x).
    static __device__ __forceinline__ void fill_slot(const DecodeParams& p, const Extent& x, u32 t, int s, S& sm) {
        Ring& rg = sm.ring[s];
        const u64 nb = (u64)p.n_strings + 1;
        rg.tile = t;
        rg.stop = 0u;
        const u64 tile_start = (x.first_tile + t) * (u64)TILE;
        const u64 byte0 = tile_start / 8 * WBITS;   // TILE is a multiple of 8 slots
        if (byte0 + CODE_BYTES <= p.codes_bytes) {
            rg.codes_in_smem = 1u;
            mbar_expect_tx(&rg.full, (u32)CODE_BYTES);
            bulk_g2s(sm.codebuf[s], p.codes + byte0, (u32)CODE_BYTES, &rg.full);
        } else {
            rg.codes_in_smem = 0u;
        }
        u32 lo = __ldg(p.first + t), hi = __ldg(p.first + t + 1);
        if ((u64)lo > nb) lo = (u32)nb;
        if ((u64)hi > nb) hi = (u32)nb;
        if (hi < lo) hi = lo;
        rg.lo = lo;
        rg.hi = hi;
        const u64 a0 = lo & ~3u;
        u64 a1 = ((u64)hi + 3) & ~3ull;
        if (a1 > (nb & ~3ull)) a1 = nb & ~3ull;
        if (a1 > a0 + kOffCap) a1 = a0 + kOffCap;
        const bool offs16 = (reinterpret_cast<uintptr_t>(p.code_offsets) & 15u) == 0u;
        if (offs16 && a1 > a0) {
            rg.off_base = (u32)a0;
            rg.off_count = (u32)(a1 - a0);
            mbar_expect_tx(&rg.full, (u32)((a1 - a0) * 4));
            bulk_g2s(sm.offbuf[s], p.code_offsets + a0, (u32)((a1 - a0) * 4), &rg.full);
        } else {
            rg.off_base = 0u;
            rg.off_count = 0u;
        }
    }

    // Wait until the workers ask for slot s (the first two tiles are fetched
    // at once, later ones on request).
    static __device__ __forceinline__ void await_request(S& sm, u32 i, int s, u32& req_ph, WsHeader* ws) {
        if (i >= 2u) {
            mbar_wait(&sm.ring[s].req, (req_ph >> s) & 1u, ws);
            req_ph ^= 1u << s;
        }
    }

    // One column: tickets count its tiles.
    static __device__ __forceinline__ void produce_one(const DecodeParams& p, S& sm, const Extent& x, WsHeader* ws) {
        u32 req_ph = 0;   // bit s: parity of the next wait on ring[s].req
        for (u32 i = 0;; ++i) {
            const int s = (int)(i % kSlots);
            Ring& rg = sm.ring[s];
            await_request(sm, i, s, req_ph, ws);
            const u32 t = atomicAdd(&ws->tile_counter, 1u);
            if ((u64)t >= x.n_tiles) {
                rg.stop = 1u;
                mbar_arrive(&rg.full);
                break;
            }
            fill_slot(p, x, t, s, sm);
            mbar_arrive(&rg.full);
        }
    }

    // A codec queue of a batch: a ticket names a chunk and one of its tiles;
    // the chunk's record is copied into the slot with the tile's inputs.
    static __device__ __forceinline__ void produce_queue(const BatchQueue& Q, unsigned int* counter, S& sm,
                                                         WsHeader* ws) {
        u32 req_ph = 0;
        for (u32 i = 0;; ++i) {
            const int s = (int)(i % kSlots);
            Ring& rg = sm.ring[s];
            await_request(sm, i, s, req_ph, ws);
            const u32 t = atomicAdd(counter, 1u);
            if (t >= Q.n_tiles) {
                rg.stop = 1u;
                mbar_arrive(&rg.full);
                break;
            }
            const u32 c = __ldg(Q.tile_chunk + t);
            const uint4* g = reinterpret_cast<const uint4*>(Q.src + c);
            uint4* d = reinterpret_cast<uint4*>(&sm.src[s]);
            uint4 v[sizeof(SlotSrc) / 16];
#pragma unroll
            for (int j = 0; j < (int)(sizeof(SlotSrc) / 16); ++j) v[j] = __ldg(g + j);
#pragma unroll
            for (int j = 0; j < (int)(sizeof(SlotSrc) / 16); ++j) d[j] = v[j];
            const SlotSrc& cs = sm.src[s];
            fill_slot(cs.p, cs.x, t - cs.tile_base, s, sm);
            mbar_arrive(&rg.full);
        }
    }

    // ---- block setup and the worker loop ------------------------------------
    static __device__ __forceinline__ void init_ring(S& sm) {
        if (threadIdx.x == 0) {
            for (int s = 0; s < kSlots; ++s) {
                mbar_init(&sm.ring[s].full, 1u);
                mbar_init(&sm.ring[s].req, 1u);
                sm.ring[s].nready = 0u;
            }
            mbar_init_fence();
        }
    }
    // The ring's mbarriers must be invalidated before their memory holds
    // anything else: a batch block re-lays out its shared memory for every
    // codec queue, and another queue's layout puts ordinary data (the
    // per-thread byte counts of the offsets) where these barriers were.
    // Writing over live mbarrier objects is undefined; it once showed as
    // string offsets off by a few bytes, from the threads whose counts sat on
    // the barriers.  Called by every thread after the queue's last barrier.
    static __device__ __forceinline__ void inval_ring(S& sm) {
        if (threadIdx.x == 0) {
            for (int s = 0; s < kSlots; ++s) {
                asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&sm.ring[s].full)) : "memory");
                asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&sm.ring[s].req)) : "memory");
            }
        }
    }

    // Worker warps: front of tile t+1, then back of tile t, two ring slots
    // alternating.
    template <class SRC>
    static __device__ __forceinline__ void work(const SRC& src, S& sm, u32 epoch, WsHeader* ws) {
        u32 err = 0;
        R ra, rb;
        u32 full_ph = 0;   // bit s: parity of the next wait on ring[s].full
        int sa = 0;
        bool ok = front(src.P(sa), sm, sa, 0u, src.X(sa), epoch, ws, ra, err);
        full_ph ^= 1u;
        while (ok) {
            const int sb = next_slot(sa);
            const bool hb = front(src.P(sb), sm, sb, (full_ph >> sb) & 1u, src.X(sb), epoch, ws, rb, err);
            full_ph ^= 1u << sb;
            back(src.P(sa), sm, sa, src.X(sa), ra, err);
            if (!hb) break;
            sa = next_slot(sb);
            ok = front(src.P(sa), sm, sa, (full_ph >> sa) & 1u, src.X(sa), epoch, ws, ra, err);
            full_ph ^= 1u << sa;
            back(src.P(sb), sm, sb, src.X(sb), rb, err);
        }
    }

    // ---- one column per launch ----------------------------------------------
    static __device__ __forceinline__ void run(const DecodeParams& p) {
        extern __shared__ __align__(128) unsigned char smem_raw[];
        S& sm = *reinterpret_cast<S*>(smem_raw);
        WsHeader* ws = p.ws;
        if (DSMEM) {
            const uint4* src = reinterpret_cast<const uint4*>(p.dict.table);
            for (int i = threadIdx.x; i < DICT_BYTES / 16; i += kThreads) sm.dict[i] = __ldg(src + i);
            const uint4* lsrc = reinterpret_cast<const uint4*>(p.dict.lens);
            for (int i = threadIdx.x; i < LENS_BYTES / 16; i += kThreads)
                sm.lens4[i] = __ldg(lsrc + i);
        }
        init_ring(sm);
        const u32 epoch = *(volatile u32*)&ws->epoch;
        const Extent x = column_extent(p, TILE);
        __syncthreads();

        const u32 warp = threadIdx.x >> 5;
        const OneColumn one{p, x};
        if (warp == (u32)kWorkWarps) {
            scan_loop(one, sm, epoch, ws);
        } else if (warp == (u32)kWorkWarps + 1) {
            if ((threadIdx.x & 31u) == 0u) produce_one(p, sm, x, ws);
        } else {
            work(one, sm, epoch, ws);
        }
        __syncthreads();
        finish_launch(ws, epoch);
    }

    // ---- one codec queue of a batch -------------------------------------------
    // Every thread of the block calls this; it returns with the ring's
    // barriers invalidated, so that the next queue may lay out the block's
    // shared memory differently.
    static __device__ __forceinline__ void run_queue(const BatchParams& bp, int q, u32 epoch) {
        extern __shared__ __align__(128) unsigned char smem_raw[];
        S& sm = *reinterpret_cast<S*>(smem_raw);
        WsHeader* ws = bp.ws;
        init_ring(sm);
        __syncthreads();
        const u32 warp = threadIdx.x >> 5;
        const SlotColumns cols{sm.src};
        if (warp == (u32)kWorkWarps) {
            scan_loop(cols, sm, epoch, ws);
        } else if (warp == (u32)kWorkWarps + 1) {
            if ((threadIdx.x & 31u) == 0u) produce_queue(bp.q[q], &ws->queue_counter[q], sm, ws);
        } else {
            work(cols, sm, epoch, ws);
        }
        __syncthreads();
        inval_ring(sm);   // the next init_ring (same thread) follows it in program order
    }
};

}  // namespace
}  // namespace fp
