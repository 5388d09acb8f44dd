// Warp-tile decoder: the column is cut into warp tiles of 32*K code slots,
// and a decode runs in three launches:
//
//   reduce_kernel   its first blocks run the index pass (the first string
//                   boundary of every warp tile); in the others each warp
//                   computes the scan element of a warp tile (its decoded
//                   bytes; for FSST-8 the two-state element of the escape
//                   parity) and stores it: fully parallel, the code stream
//                   is read once;
//   tiles_scan_kernel  single-pass exclusive scan of the warp-tile elements
//                   (blocks of 2,048 elements, decoupled look-back across
//                   blocks): every warp tile's output offset and entering
//                   escape state;
//   warp_decode_kernel  every warp decodes whole warp tiles on its own: code
//                   unpack, lengths, a warp scan inside the tile, assembly in
//                   registers with aligned 16-byte stores, merging of chunks
//                   shared by lanes through a per-warp shared-memory area,
//                   string offsets.  No block barrier and no wait on other
//                   warps, so the SM hides the latency of one warp's loads with
//                   the others' work.
//
// Reading the code stream twice costs its bytes (about a fifth of the
// traffic at 6 decoded bytes per 12-bit code) but removes the serial
// look-back from the decode itself; this is the paper's sidecar (Sec. 3.1)
// regenerated on the device by the first two passes.
#pragma once
#include "fp_decoder.cuh"

namespace fp {
namespace {

// Warp-tile element <-> 64-bit word (bytes of a warp tile stay below 2^20).
template <bool FSST>
__device__ __forceinline__ u64 wt_pack(const TElem& e) {
    if (!FSST) return e.b0;
    return (u64)e.b0 | ((u64)e.b1 << 24) | ((u64)(e.n & 3u) << 48);
}
template <bool FSST>
__device__ __forceinline__ Elem wt_unpack(u64 w) {
    if (!FSST) return Elem{w, 0, 0};
    return Elem{w & 0xffffffull, (w >> 24) & 0xffffffull, (u32)((w >> 48) & 3u)};
}

// A chunk of which only bytes [lo, hi) may be written (shared with a
// neighbouring warp tile).
struct Partial {
    uint4 v;
    uint4* chunk;
    u32 lo, hi;
    bool pending;
};

// Merge a partial chunk with the lead fragments of the following lanes of
// the same warp tile; store it if it is complete, else leave it pending for
// store_partials().
__device__ __forceinline__ void combine_lanes(uint4* chunk, uint4 acc, u32 lo, u32 hi, int m, const uint4* s_fa,
                                              const u32* s_meta, Partial& pend) {
    while (hi < 16u && m < 32) {
        const u32 mm = s_meta[m];
        if (mm & FA_VALID) {
            acc = or4(acc, s_fa[m]);
            hi = (mm >> FA_HI_SHIFT) & 31u;
        }
        ++m;
    }
    if (lo == 0u && hi == 16u) {
        __stcs(chunk, acc);
    } else {
        pend.v = acc;
        pend.chunk = chunk;
        pend.lo = lo;
        pend.hi = hi;
        pend.pending = true;
    }
}

// The warp writes its lanes' pending partial chunks together: lane b stores
// byte b of a chunk when b is in [lo, hi), one byte store per chunk.
__device__ __forceinline__ void store_partials(const Partial& pd) {
    const u32 lane = threadIdx.x & 31u;
    u32 ball = __ballot_sync(0xffffffffu, pd.pending);
    while (ball) {
        const int src = __ffs(ball) - 1;
        ball &= ball - 1u;
        const u32 x = __shfl_sync(0xffffffffu, pd.v.x, src), y = __shfl_sync(0xffffffffu, pd.v.y, src);
        const u32 z = __shfl_sync(0xffffffffu, pd.v.z, src), w = __shfl_sync(0xffffffffu, pd.v.w, src);
        const u32 lo = __shfl_sync(0xffffffffu, pd.lo, src), hi = __shfl_sync(0xffffffffu, pd.hi, src);
        const unsigned long long a = __shfl_sync(0xffffffffu, (unsigned long long)pd.chunk, src);
        const u32 q = lane >> 2;
        const u32 word = q == 0 ? x : (q == 1 ? y : (q == 2 ? z : w));
        if (lane >= lo && lane < hi) reinterpret_cast<uint8_t*>(a)[lane] = (uint8_t)(word >> ((lane & 3u) * 8u));
    }
}

// Per-warp shared-memory area of the decode kernel.
template <int K>
struct WarpArea {
    uint4 fa[32];
    uint4 fb[32];
    u32 meta[32];
    u32 pre[K / 4][32];     // tile-relative output offset of slot 4m of each lane
    u32 contrib[K / 4][32]; // bytes each slot produced, one byte per slot
    u32 lit_mask[32];       // FSST-8: bit k = slot k holds a literal byte
};

// W: dictionary read width of the OnPair codecs (paper Sec. 3.2 and 4.3):
// 16 reads whole 16-byte entries, 8 reads the low plane (bytes 0-7) for
// every token and the high plane (bytes 8-15) only for longer tokens.  The
// FSST codecs have 8-byte entries (W = 8).
// PACKED: the codes are stored bit-packed at p.packed_bits bits per code
// (LSB-first, 1..16) instead of the codec's own layout -- the cascade layer
// the paper removes on the host (Sec. 5), unpacked here inside the kernels.
template <int CODEC, int K, bool DSMEM, int W = (CODEC == FP_ONPAIR16 || CODEC == FP_ONPAIR12) ? 16 : 8,
          bool PACKED = false>
struct WarpCore {
    static constexpr bool FSST = (CODEC == FP_FSST8);   // escape codec: two-state scan elements
    static constexpr bool TOK8 = (CODEC == FP_FSST8 || CODEC == FP_FSST12);   // 8-byte table entries
    static constexpr bool W12 = (CODEC == FP_ONPAIR12 || CODEC == FP_FSST12);  // 12-bit codes
    static constexpr int TILE = 32 * K;
    static constexpr int WBITS = (CODEC == FP_ONPAIR16) ? 16 : (W12 ? 12 : 8);
    static constexpr int LANE_BYTES = K * WBITS / 8;   // code bytes of one lane
    // words a lane loads: its code bytes, or for packed codes the 32-bit
    // words covering K codes of up to 16 bits at any bit offset
    static constexpr int LANE_WORDS = PACKED ? (K * 16 + 31) / 32 + 1 : LANE_BYTES / 4;
    // per-lane scratch: word i next to word i + 1, as 8-byte pairs; a stride
    // of 2 * LANE_WORDS words keeps the 16 lanes of each half-warp's 8-byte
    // accesses on distinct banks
    static constexpr int PK_STRIDE = 2 * LANE_WORDS;
    // entries of the table (a staged table, or the global planes)
    static constexpr int kTable = (CODEC == FP_FSST8) ? 256 : (CODEC == FP_ONPAIR16 ? 65536 : 4096);
    // FSST-8 with a staged table: every symbol and every literal byte kept
    // moved up by 0..3 bytes (entry lit * 1024 + r * 256 + b, 16 bytes
    // each), so an insert at byte position f reads the copy for r = f & 3
    // and needs only whole-word moves.
    static constexpr bool PRESHIFT = FSST && DSMEM;
    static constexpr int DICT_BYTES = DSMEM ? (PRESHIFT ? 2 * 4 * 256 * 16 : kTable * (TOK8 ? 8 : 16)) : 0;
    static constexpr int LENS_BYTES = kTable;
    typedef TileRegs<CODEC, K> R;
    static_assert(K == 8 || K == 16 || K == 32, "slots per lane");
    static_assert(!FSST || K >= 16, "FSST-8 handles 16 slots at a time");
    static_assert(!DSMEM || CODEC != FP_ONPAIR16, "OnPair-16 tables do not fit in shared memory");
    static_assert(LANE_BYTES % 8 == 0, "lane code bytes are read in 8-byte words");
    static_assert(W == 16 || W == 8, "read width");
    static_assert(!TOK8 || W == 8, "FSST entries are 8 bytes");
    static_assert(!PACKED || (!FSST && K == 16), "packed codes: escape-free codecs, 16 slots per lane");

    static __device__ __forceinline__ u32 full_mask() { return K == 32 ? 0xffffffffu : ((1u << K) - 1u); }

    // ---- codes of slots [q0, q0 + K) ---------------------------------------
    static __device__ __forceinline__ void unpack_words(const u32* wv, R& r) {
        if (W12) {
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
            for (int m = 0; m < R::CW; ++m) r.c[m] = wv[m];
        }
    }

    // Raw code words of the lane (LANE_WORDS words); false if they run past
    // the buffer (then load_guarded() is used).
    static __device__ __forceinline__ bool load_fast(const DecodeParams& p, u64 q0, u32 (&wv)[LANE_WORDS]) {
        if (PACKED) {
            const u64 w0 = (q0 * p.packed_bits) >> 5;   // the word holding the lane's first bit
            if ((w0 + LANE_WORDS) * 4 > p.codes_bytes) return false;
            const u32* src = reinterpret_cast<const u32*>(p.codes) + w0;
#pragma unroll
            for (int i = 0; i < LANE_WORDS; ++i) wv[i] = __ldcs(src + i);
            return true;
        }
        const u64 b0 = q0 * WBITS / 8;   // q0 is a multiple of K, K a multiple of 8
        if (b0 + LANE_BYTES > p.codes_bytes) return false;
        if (LANE_BYTES % 16 == 0) {
            const uint4* src = reinterpret_cast<const uint4*>(p.codes + b0);
#pragma unroll
            for (int v = 0; v < LANE_BYTES / 16; ++v) {
                const uint4 a = __ldcs(src + v);
                wv[4 * v] = a.x; wv[4 * v + 1] = a.y; wv[4 * v + 2] = a.z; wv[4 * v + 3] = a.w;
            }
        } else {
            const uint2* src = reinterpret_cast<const uint2*>(p.codes + b0);
#pragma unroll
            for (int v = 0; v < LANE_BYTES / 8; ++v) {
                const uint2 a = __ldcs(src + v);
                wv[2 * v] = a.x; wv[2 * v + 1] = a.y;
            }
        }
        return true;
    }

    static __device__ void load_guarded(const DecodeParams& p, u64 q0, R& r) {
        if (PACKED) {
            // bit-packed codes near the end of the buffer: byte by byte
            const u32 b = p.packed_bits, mask = (1u << b) - 1u;
#pragma unroll
            for (int m = 0; m < K / 2; ++m) {
                u32 v = 0;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const u64 q = q0 + 2 * m + h;
                    if (q < p.max_slots) {
                        const u64 P = q * b, by = P >> 3;
                        u32 x = 0;
#pragma unroll
                        for (int e = 0; e < 3; ++e)
                            if (by + e < p.codes_bytes) x |= (u32)p.codes[by + e] << (8 * e);
                        v |= ((x >> (P & 7u)) & mask) << (16 * h);
                    }
                }
                r.c[m] = v;
            }
            return;
        }
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
        } else if (W12) {
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

    // Packed codes: the lane's words go to its shared-memory scratch `pk`
    // (a run-time bit offset cannot index registers), then each code is one
    // funnel shift of the two words that hold it.
    static __device__ __forceinline__ void unpack_packed(const u32 (&wv)[LANE_WORDS], u32 o, u32 b, u32* pk, R& r) {
        uint2* pairs = reinterpret_cast<uint2*>(pk);
#pragma unroll
        for (int i = 0; i < LANE_WORDS; ++i) pairs[i] = make_uint2(wv[i], i + 1 < LANE_WORDS ? wv[i + 1] : 0u);
        const u32 mask = (1u << b) - 1u;
#pragma unroll
        for (int m = 0; m < K / 2; ++m) {
            u32 v = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const u32 P = o + (u32)(2 * m + h) * b;   // < 32 + 15 * 16
                const uint2 w = pairs[P >> 5];
                v |= (__funnelshift_r(w.x, w.y, P) & mask) << (16 * h);
            }
            r.c[m] = v;
        }
    }

    // Codes (from words load_fast() fetched, or guarded loads), the slots
    // inside the column and their token lengths.  `pk`: the lane's scratch
    // (packed codes only).
    static __device__ __forceinline__ void finish_load(const DecodeParams& p, const Extent& x, u64 q0,
                                                       const u32 (&wv)[LANE_WORDS], bool fast, const uint8_t* lens,
                                                       R& r, u32* pk = nullptr) {
        if (fast) {
            if (PACKED) unpack_packed(wv, (u32)((q0 * p.packed_bits) & 31u), p.packed_bits, pk, r);
            else unpack_words(wv, r);
        } else {
            load_guarded(p, q0, r);
        }
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
#pragma unroll
        for (int j = 0; j < K / 4; ++j) {
            u32 w = 0;
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const u32 code = code_at<CODEC, K>(r, 4 * j + h);
                const u32 L = DSMEM ? (u32)lens[code] : (u32)__ldg(lens + code);
                w |= L << (8 * h);
            }
            r.L[j] = w;
        }
    }

    // FSST-8 helpers on the lane's registers.
    static __device__ __forceinline__ u32 ff_mask(const R& r) {
        u32 E = 0;
#pragma unroll
        for (int j = 0; j < K / 4; ++j) E |= ff_bits4(r.c[j]) << (4 * j);
        return E;
    }
    static __device__ __forceinline__ u32 fsst_bytes(const R& r, u32 codes, u32 lits) {
        u32 n = __popc(lits);
#pragma unroll
        for (int j = 0; j < K / 4; ++j) n = masked_byte_sum(r.L[j], ones_of4(codes >> (4 * j)), n);
        return n;
    }

    // FSST-8 escape state across lanes.  A lane maps the state entering it
    // (1: its first slot is a literal) to the state after it.  For a lane
    // whose K slots are all 0xFF that map is the identity (codes and
    // literals alternate, K is even); for any other lane it is constant: a
    // slot that is not 0xFF (or lies outside the column, which resets the
    // state) fixes the parity of every later slot.  x0 is the state after
    // the lane entered with 0; `ident` marks the identity lanes.
    static __device__ __forceinline__ void lane_state(const R& r, bool allv, u32 E, u32& x0, bool& ident) {
        if (allv) {
            u32 lit, esc;
            fsst_escapes<K>(E, 0u, lit, esc);
            x0 = (esc >> (K - 1)) & 1u;
            ident = (E == full_mask());
            return;
        }
        u32 st = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const bool v = (r.valid >> k) & 1u;
            st = v ? (st ? 0u : (code_at<CODEC, K>(r, k) == 255u ? 1u : 0u)) : 0u;
        }
        x0 = st;
        ident = false;
    }
    // The state entering this lane when s_tile enters the tile: the exit of
    // the nearest lower lane whose map is constant, else s_tile (only
    // identity lanes before it).  One ballot and one shuffle; every lane of
    // the warp calls it.
    static __device__ __forceinline__ u32 enter_state(u32 cmask, u32 x0, u32 s_tile, u32 lane) {
        const u32 below = cmask & ((1u << lane) - 1u);
        const u32 src = below ? 31u - (u32)__clz(below) : 0u;
        const u32 xk = __shfl_sync(0xffffffffu, x0, src);
        return below ? xk : s_tile;
    }
    // Bytes of an all-inside lane entered in state s (lit/esc: its literal
    // and escape-code slots).
    static __device__ __forceinline__ u32 fsst_lane_bytes(const R& r, u32 E, u32 s) {
        u32 lit, esc;
        fsst_escapes<K>(E, s, lit, esc);
        return fsst_bytes(r, ~(lit | esc) & full_mask(), lit);
    }
    // Bytes of an edge lane (some slots outside the column) entered in state s.
    static __device__ __forceinline__ u32 fsst_edge_bytes(const R& r, u32 s) {
        u32 n = 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const bool v = (r.valid >> k) & 1u;
            const bool is255 = code_at<CODEC, K>(r, k) == 255u;
            n += v ? (s ? 1u : (is255 ? 0u : len_at<CODEC, K>(r, k))) : 0u;
            s = v ? (s ? 0u : (is255 ? 1u : 0u)) : 0u;
        }
        return n;
    }

    // The warp tile's scan element; every lane of the warp calls it.  OnPair:
    // the tile's byte count (the same for both entry states; corrupt codes
    // set ERRB_CORRUPT).  FSST-8: for each escape state entering the tile,
    // the bytes it produces and the state after it.
    static __device__ __forceinline__ TElem tile_element(const R& r, u32 lane, u32& err) {
        const bool allv = (r.valid == full_mask());
        if (!FSST) {
            u32 sum = 0;
            if (allv) {
                bool zero = false;
#pragma unroll
                for (int j = 0; j < K / 4; ++j) {
                    sum += byte_sum(r.L[j]);
                    zero |= has_zero_byte(r.L[j]);
                }
                if (zero) err |= ERRB_CORRUPT;
            } else {
#pragma unroll
                for (int j = 0; j < K / 4; ++j) {
                    const u32 vm = bytes_of4(r.valid >> (4 * j));
                    sum += byte_sum(r.L[j] & vm);
                    if (__vcmpeq4(r.L[j], 0u) & vm) err |= ERRB_CORRUPT;
                }
            }
            sum = __reduce_add_sync(0xffffffffu, sum);
            return TElem{sum, sum, 2u};
        }
        const u32 E = allv ? ff_mask(r) : 0u;
        u32 x0;
        bool ident;
        lane_state(r, allv, E, x0, ident);
        // states entering this lane when the tile is entered with 0 and with 1:
        // they differ only for lanes that only identity lanes precede
        const u32 below = __ballot_sync(0xffffffffu, !ident) & ((1u << lane) - 1u);
        const u32 xk = __shfl_sync(0xffffffffu, x0, below ? 31u - (u32)__clz(below) : 0u);
        const u32 s0 = below ? xk : 0u, s1 = below ? xk : 1u;
        u32 b0 = allv ? fsst_lane_bytes(r, E, s0) : fsst_edge_bytes(r, s0);
        u32 b1 = b0;
        if (__any_sync(0xffffffffu, s0 != s1) && s0 != s1) b1 = allv ? fsst_lane_bytes(r, E, s1) : fsst_edge_bytes(r, s1);
        b0 = __reduce_add_sync(0xffffffffu, b0);
        b1 = __reduce_add_sync(0xffffffffu, b1);
        const u32 e = (ident ? s0 : x0) | ((ident ? s1 : x0) << 1);
        return TElem{b0, b1, __shfl_sync(0xffffffffu, e, 31)};
    }

    // Token of `code` (zero padded to 16 bytes), from the table staged in
    // shared memory (DSMEM) or through L1.  OnPair: the whole 16-byte entry
    // (W = 16) or the low plane and, for longer tokens, the high plane
    // (W = 8).  FSST: 8-byte entries.
    static __device__ __forceinline__ uint4 token(const DecodeParams& p, const uint4* dict, u32 code, u32 len) {
        if (TOK8) {
            const uint2 d = DSMEM ? reinterpret_cast<const uint2*>(dict)[code]
                                  : __ldg(reinterpret_cast<const uint2*>(p.dict.table) + code);
            return make_uint4(d.x, d.y, 0u, 0u);
        }
        // W = 16: whole 16-byte entries, one load (staged as the table is laid out)
        if (W == 16) return DSMEM ? dict[code] : __ldg(reinterpret_cast<const uint4*>(p.dict.table) + code);
        const uint2* lo = DSMEM ? reinterpret_cast<const uint2*>(dict) : reinterpret_cast<const uint2*>(p.dict.planes);
        const uint2 a = DSMEM ? lo[code] : __ldg(lo + code);
        uint2 b = make_uint2(0u, 0u);
        // split read: the high plane only for longer tokens (W = 8), always for W = 16
        if (W == 16 || len > 8u) b = DSMEM ? lo[kTable + code] : __ldg(lo + kTable + code);
        return make_uint4(a.x, a.y, b.x, b.y);
    }

    template <bool ALLV>
    static __device__ __forceinline__ void assemble_onpair(const DecodeParams& p, const uint4* dict, const R& r,
                                                           Assembler& as) {
#pragma unroll
        for (int k0 = 0; k0 < K; k0 += 4) {
            uint4 tok[4];
#pragma unroll
            for (int h = 0; h < 4; ++h)
                tok[h] = token(p, dict, code_at<CODEC, K>(r, k0 + h), len_at<CODEC, K>(r, k0 + h));
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

    // FSST-8 slots: a literal's byte, else the symbol; cw holds each slot's
    // byte count.  In a lane whose slots are all inside the column a slot
    // that yields no byte is an escape or a corrupt code, whose table entries
    // (255, and those past the dictionary) are all zero, so only literals
    // need a select there.
    template <bool ALLV>
    static __device__ __forceinline__ void assemble_fsst(const DecodeParams& p, const uint4* dict, const R& r,
                                                         const u32 (&cw)[K / 4], u32 lit, Assembler& as) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const u32 bt = code_at<CODEC, K>(r, k);
            const u32 a = (cw[k >> 2] >> ((k & 3) * 8)) & 0xffu;
            const bool is_lit = (lit >> k) & 1u;
            if (PRESHIFT) {
                // the copy of the symbol (or literal) moved up by the insert position's byte offset
                uint4 y = dict[(((lit >> k) & 1u) << 10) | ((as.f & 3u) << 8) | bt];
                if (!ALLV && a == 0u) y = make_uint4(0u, 0u, 0u, 0u);
                as.put3(y.x, y.y, y.z, a);
                continue;
            }
            uint2 d;
            if (DSMEM) d = reinterpret_cast<const uint2*>(dict)[bt];
            else d = __ldg(reinterpret_cast<const uint2*>(p.dict.table) + bt);
            uint4 tok;
            if (ALLV) tok = make_uint4(is_lit ? bt : d.x, is_lit ? 0u : d.y, 0u, 0u);
            else tok = make_uint4(a == 0u ? 0u : (is_lit ? bt : d.x), (a == 0u || is_lit) ? 0u : d.y, 0u, 0u);
            as.put(tok, a);
        }
    }

    // Stage the dictionary and the token lengths in shared memory (every
    // thread of the block; the caller synchronises).  FSST: the 8-byte
    // entries, or for FSST-8 the moved-up copies (PRESHIFT); OnPair read
    // whole (W = 16): the 16-byte entries; OnPair split read (W = 8): the two
    // planes (entry e's bytes 0..7 at low-plane word e, bytes 8..15 at
    // high-plane word e).
    static __device__ __forceinline__ void stage_dict(const DecodeParams& p, uint4* s_dict, uint8_t* s_lens,
                                                      int nthreads) {
        if (!DSMEM) return;
        if (PRESHIFT) {
            const uint2* tab = reinterpret_cast<const uint2*>(p.dict.table);
            for (int i = threadIdx.x; i < DICT_BYTES / 16; i += nthreads) {
                const u32 b = (u32)i & 255u, r8 = (((u32)i >> 8) & 3u) * 8u;
                u32 lo = b, hi = 0u;   // a literal byte
                if (i < 1024) {
                    const uint2 d = __ldg(tab + b);
                    lo = d.x;
                    hi = d.y;
                }
                s_dict[i] = make_uint4(lo << r8, __funnelshift_l(lo, hi, r8), __funnelshift_l(hi, 0u, r8), 0u);
            }
        } else {
            const uint4* src = reinterpret_cast<const uint4*>((TOK8 || W == 16) ? p.dict.table : p.dict.planes);
            for (int i = threadIdx.x; i < DICT_BYTES / 16; i += nthreads) s_dict[i] = __ldg(src + i);
        }
        const uint4* lsrc = reinterpret_cast<const uint4*>(p.dict.lens);
        for (int i = threadIdx.x; i < LENS_BYTES / 16; i += nthreads) reinterpret_cast<uint4*>(s_lens)[i] = __ldg(lsrc + i);
    }

    // The same staging by the bulk-copy engine where the staged layout is the
    // stored one (no planes, no moved-up copies): thread 0 issues the two
    // copies (cp.async.bulk, completion counted on one mbarrier) and every
    // thread waits for them, bounded (a wait that gives up sets
    // ERRB_TIMEOUT).  Falls back to the loads above for tables that are not
    // 16-byte aligned.  Every thread of the block calls it; returns synchronised.
    static constexpr bool BULK_STAGE = DSMEM && !PRESHIFT && (TOK8 || W == 16);
    static __device__ __forceinline__ void stage_dict_bulk(const DecodeParams& p, uint4* s_dict, uint8_t* s_lens,
                                                           u64* bar, int nthreads) {
        const bool aligned =
            ((reinterpret_cast<uintptr_t>(p.dict.table) | reinterpret_cast<uintptr_t>(p.dict.lens)) & 15u) == 0u;
        if (!aligned) {
            stage_dict(p, s_dict, s_lens, nthreads);
            __syncthreads();
            return;
        }
        if (threadIdx.x == 0) {
            mbar_init(bar, 1u);
            mbar_init_fence();
            mbar_expect_tx(bar, (u32)(DICT_BYTES + LENS_BYTES));
            bulk_g2s(s_dict, p.dict.table, (u32)DICT_BYTES, bar);
            bulk_g2s(s_lens, p.dict.lens, (u32)LENS_BYTES, bar);
            mbar_arrive(bar);
        }
        __syncthreads();   // the barrier is initialised before anyone waits on it
        mbar_wait(bar, 0u, p.ws);
    }

    // Byte count of an escape-free lane whose K slots all lie inside the
    // column, straight from its code words (constant bit positions): one
    // extract, one length load and one add per code; a code without a token
    // (length 0) raises ERRB_CORRUPT.
    static __device__ __forceinline__ u32 lane_length_sum(const u32 (&wv)[LANE_WORDS], const uint8_t* lens,
                                                          u32& err) {
        static_assert(!FSST && !PACKED, "escape-free codecs in their own layout");
        constexpr u32 MASK = (1u << WBITS) - 1u;
        u32 sum = 0, mn = 0xffu;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int bit = k * WBITS, w = bit >> 5, sh = bit & 31;
            const u32 code = (sh + WBITS <= 32) ? ((wv[w] >> sh) & MASK) : (__funnelshift_r(wv[w], wv[w + 1], sh) & MASK);
            const u32 L = DSMEM ? (u32)lens[code] : (u32)__ldg(lens + code);
            sum += L;
            mn = min(mn, L);
        }
        if (mn == 0u) err |= ERRB_CORRUPT;
        return sum;
    }

    static __device__ __forceinline__ u64 lane_q0(const Extent& x, u64 t) {
        return (x.first_tile + t) * (u64)TILE + (u64)(threadIdx.x & 31u) * K;
    }

    // Inputs of a warp tile fetched ahead of its decode: the lane's code
    // words, the tile's scanned offset, its string boundaries [lo, hi) and
    // the first PB*32 of their code_offsets (one per lane and round).
    static constexpr int PB = FSST ? 2 : 1;
    struct Fetch {
        u32 wv[LANE_WORDS];
        bool fast;
        u64 ex;
        u32 lo, hi;
        u32 pos[PB];
    };

    // Loads of data written by this launch's earlier phases (the one-launch
    // decode, CG) bypass L1; otherwise the read-only path.
    template <bool CG, class T>
    static __device__ __forceinline__ T ld(const T* a) { return CG ? __ldcg(a) : __ldg(a); }

    // Issue the loads of tile t whose boundaries [lo, hi) are already known.
    template <bool CG = false>
    static __device__ __forceinline__ void fetch(const DecodeParams& p, const Extent& x, const u64* ex, u64 t, u32 lo,
                                                 u32 hi, Fetch& f) {
        const u32 lane = threadIdx.x & 31u;
        f.fast = load_fast(p, lane_q0(x, t), f.wv);
        f.ex = ld<CG>(ex + t);
        f.lo = lo;
        f.hi = hi;
#pragma unroll
        for (int j = 0; j < PB; ++j) {
            const u32 i = lo + lane + 32u * j;
            f.pos[j] = i < hi ? __ldg(p.code_offsets + i) : 0u;
        }
    }

    // Boundaries [lo, hi) of tile t, clamped to the column's.
    template <bool CG = false>
    static __device__ __forceinline__ void bounds(const DecodeParams& p, u64 t, u32& lo, u32& hi) {
        const u64 nb = (u64)p.n_strings + 1;
        lo = ld<CG>(p.first + t);
        hi = ld<CG>(p.first + t + 1);
        if ((u64)lo > nb) lo = (u32)nb;
        if ((u64)hi > nb) hi = (u32)nb;
        if (hi < lo) hi = lo;
    }

    // Decode warp tile t of column (p, x) from its fetched inputs: offset
    // and entering escape state (from the tile scan), code words, string
    // boundaries.  `area` is the warp's scratch.  `ex_tiles` holds the
    // column's scanned tile offsets (f.ex = ex_tiles[t]): the tile's own
    // byte total, recomputed here, must bring it to ex_tiles[t + 1], else
    // ERRB_MISMATCH is raised (a self-check of the two passes, one load
    // per tile).
    template <bool CG = false>
    static __device__ __forceinline__ void decode_tile(const DecodeParams& p, const Extent& x, u64 t, const Fetch& f,
                                                       const u64* ex_tiles, const uint4* dict, const uint8_t* lens,
                                                       WarpArea<K>& area, u32& err, u32* pk = nullptr) {
        const u32 lane = threadIdx.x & 31u;
        const u64 tile_start = (x.first_tile + t) * (u64)TILE;
        const u64 q0 = tile_start + (u64)lane * K;
        const u64 ex = f.ex;
        // low word of the next tile's offset (lane 0 checks), in flight during the tile
        const bool chk = lane == 0u && t + 1 < x.n_tiles;
        const u32 ex_next = chk ? ld<CG>(reinterpret_cast<const u32*>(ex_tiles + t + 1)) : 0u;
        R r;
        finish_load(p, x, q0, f.wv, f.fast, lens, r, pk);
        r.t = (u32)t;
        r.tile_start = tile_start;
        const bool allv = (r.valid == full_mask());
        const u64 tile_excl = ex & 0x7fffffffffffffffull;
        const u32 s_tile = FSST ? (u32)(ex >> 63) : 0u;

        // bytes of each slot (cw, one byte per slot) and of the lane; FSST-8:
        // the lane's entering escape state first, then its literals
        u32 cw[K / 4];
        u32 produced = 0;
        u32 lit = 0, exit_state = 0;
        if (!FSST) {
#pragma unroll
            for (int j = 0; j < K / 4; ++j) {
                // a code without a token (length 0) is corrupt input
                if (allv) {
                    cw[j] = r.L[j];
                    if (has_zero_byte(cw[j])) err |= ERRB_CORRUPT;
                } else {
                    const u32 vm = bytes_of4(r.valid >> (4 * j));
                    cw[j] = r.L[j] & vm;
                    if (__vcmpeq4(r.L[j], 0u) & vm) err |= ERRB_CORRUPT;
                }
                produced += byte_sum(cw[j]);
            }
        } else {
            const u32 E = allv ? ff_mask(r) : 0u;
            u32 x0;
            bool ident;
            lane_state(r, allv, E, x0, ident);
            const u32 s_in = enter_state(__ballot_sync(0xffffffffu, !ident), x0, s_tile, lane);
            exit_state = ident ? s_in : x0;
            if (allv) {
                u32 esc;
                fsst_escapes<K>(E, s_in, lit, esc);
                const u32 code_slots = ~(lit | esc) & full_mask();
#pragma unroll
                for (int j = 0; j < K / 4; ++j) {
                    const u32 code_ff = bytes_of4(code_slots >> (4 * j));
                    cw[j] = (r.L[j] & code_ff) | ones_of4(lit >> (4 * j));
                    if (has_zero_byte(r.L[j] | ~code_ff)) err |= ERRB_CORRUPT;
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
                    lit |= (st & 1u) << k;
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
            area.lit_mask[lane] = lit;
        }

        // the lane's output offset in the tile: one warp scan of byte counts
        u32 inc = produced;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const u32 y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= (u32)d) inc += y;
        }
        const u32 thr = inc - produced;
        const u32 tot = __shfl_sync(0xffffffffu, inc, 31);
        const u64 tile_incl = tile_excl + tot;
        const u32 tile_out_state = FSST ? __shfl_sync(0xffffffffu, exit_state, 31) : 0u;
        const bool last_tile = (t == x.n_tiles - 1);
        const bool skip = p.size_only || tile_incl > p.capacity;

        // per-slot bytes and the offsets of every fourth slot, for the string offsets
        {
            u32 o = thr;
#pragma unroll
            for (int j = 0; j < K / 4; ++j) {
                area.contrib[j][lane] = cw[j];
                area.pre[j][lane] = o;
                o += byte_sum(cw[j]);
            }
        }
        Assembler as;
        as.begin(p.out, tile_excl + thr, &area.fa[lane]);
        if (!skip) {
            if (!FSST) {
                if (allv) assemble_onpair<true>(p, dict, r, as);
                else assemble_onpair<false>(p, dict, r, as);
            } else {
                if (allv) assemble_fsst<true>(p, dict, r, cw, lit, as);
                else assemble_fsst<false>(p, dict, r, cw, lit, as);
            }
        }
        as.finish(produced > 0u && !skip);
        area.meta[lane] = as.meta;
        __syncwarp();

        // chunks shared between lanes; the tile's edge chunks, shared with
        // the neighbouring tiles, are written bytewise by the whole warp
        const bool wrote = !skip && produced > 0u;
        Partial pd;
        pd.pending = false;
        if (wrote && (as.meta & FB_VALID))
            combine_lanes(as.g, as.fb, 0u, (as.meta >> FB_HI_SHIFT) & 31u, (int)lane + 1, area.fa, area.meta, pd);
        store_partials(pd);
        pd.pending = false;
        if (wrote && (as.meta & FA_VALID) && thr == 0u)
            combine_lanes(as.dst0, area.fa[lane], (as.meta >> FA_LO_SHIFT) & 31u, (as.meta >> FA_HI_SHIFT) & 31u,
                          (int)lane + 1, area.fa, area.meta, pd);
        store_partials(pd);

        // offsets of the strings whose boundaries the tile owns (the first
        // PB*32 positions were fetched with the tile)
        for (u32 i = f.lo + lane, j = 0; i < f.hi; i += 32, ++j) {
            u64 pos;
            if (j < (u32)PB) {
                u32 v = f.pos[0];
#pragma unroll
                for (int m = 1; m < PB; ++m)
                    if (j == (u32)m) v = f.pos[m];
                pos = v;
            } else {
                pos = __ldg(p.code_offsets + i);
            }
            u64 rel = 0;
            u32 st = 0;
            if (pos < tile_start || pos > tile_start + TILE) {
                err |= ERRB_CORRUPT;
            } else if (pos == tile_start + TILE) {
                rel = tile_incl - tile_excl;
                st = tile_out_state;
                if (!last_tile) err |= ERRB_CORRUPT;
            } else {
                const u32 sidx = (u32)(pos - tile_start);
                const u32 j = sidx / K, k = sidx % K;
                // offset of slot k's group of four, then the group's slots before k
                rel = area.pre[k >> 2][j] + byte_sum(area.contrib[k >> 2][j] & ((1u << (8u * (k & 3u))) - 1u));
                if (FSST) st = (area.lit_mask[j] >> k) & 1u;
            }
            if (st) err |= ERRB_CORRUPT;   // a string would start on a literal
            if (!p.size_only) __stcs(p.out_offsets + i, (u32)(tile_excl + rel));
        }
        if (chk && ex_next != (u32)tile_incl) err |= ERRB_MISMATCH;
        __syncwarp();   // the area is reused by the next tile
    }

    // Decode the tiles t0, t0 + step, ... of the column (every lane of the
    // warp).  Software pipeline: while tile t decodes, the inputs of
    // t + step are in flight and the boundaries of t + 2 step are being read.
    template <bool CG = false>
    static __device__ __forceinline__ void decode_tiles(const DecodeParams& p, const Extent& x, const u64* ex, u64 t,
                                                        u64 step, const uint4* dict, const uint8_t* lens,
                                                        WarpArea<K>& area, u32& err, u32* pk) {
        if (t >= x.n_tiles) return;
        Fetch cur;
        u32 lo, hi, lo1 = 0, hi1 = 0;
        bounds<CG>(p, t, lo, hi);
        fetch<CG>(p, x, ex, t, lo, hi, cur);
        if (t + step < x.n_tiles) bounds<CG>(p, t + step, lo1, hi1);
        for (; t < x.n_tiles; t += step) {
            Fetch nxt;
            const u64 tn = t + step, t2 = t + 2 * step;
            u32 lo2 = 0, hi2 = 0;
            if (tn < x.n_tiles) fetch<CG>(p, x, ex, tn, lo1, hi1, nxt);
            if (t2 < x.n_tiles) bounds<CG>(p, t2, lo2, hi2);
            decode_tile<CG>(p, x, t, cur, ex, dict, lens, area, err, pk);
            cur = nxt;
            lo1 = lo2;
            hi1 = hi2;
        }
    }
};

// ---------------------------------------------------------------------------
// Pass 1: warp-tile elements.
// ---------------------------------------------------------------------------
// Blocks [0, index_blocks) run the index pass (first string of every warp
// tile; block 0 also stores the column's extent for the later passes), the
// others the reduce: the two overlap in one launch.
// Reduce shape per codec, from an A/B on GB300 (10M-16M strings): rounds of
// kReduceU tiles in flight, kReduceMinB blocks of 256 threads per SM.
// OnPair-12: 2 x 4 (1,515 GB/s per call against 1,498 at 2 x 3); FSST-8,
// whose 32-slot lanes spill at fewer than 128 registers: 2 x 2 (1,051
// against 1,038); FSST-12: 1 x 4 (1,188 against 1,171).
template <int CODEC, int K>
struct ReduceShape {
    static constexpr int U = CODEC == FP_FSST12 ? 1 : 2;
    static constexpr int MINB = (CODEC == FP_FSST8 && K == 32) ? 2 : 4;
};

template <int CODEC, int K, bool DSMEM, bool PACKED = false>
__global__ void __launch_bounds__(256, ReduceShape<CODEC, K>::MINB) reduce_kernel(const DecodeParams p, Extent* xp,
                                                                                  u64* agg, u32 index_blocks) {
    typedef WarpCore<CODEC, K, DSMEM, WarpCore<CODEC, K, DSMEM>::TOK8 ? 8 : 16, PACKED> C;
    __shared__ __align__(16) uint8_t s_lens[DSMEM ? C::LENS_BYTES : 16];
    __shared__ __align__(16) u32 s_pk[PACKED ? 256 * C::PK_STRIDE : 2];   // packed codes: per-lane scratch
    grid_release();   // the next launch may be scheduled as these blocks retire (it waits for their results)
    if (blockIdx.x < index_blocks) {
        const Extent x = column_extent(p, C::TILE);
        if (blockIdx.x == 0 && threadIdx.x == 0) *xp = x;
        index_groups(p, x, (u32)(__ffs(C::TILE) - 1), 0, (u64)p.n_strings + 1,
                     (u64)blockIdx.x * blockDim.x + threadIdx.x, (u64)index_blocks * blockDim.x,
                     const_cast<u32*>(p.first));
        return;
    }
    if (DSMEM) {
        const uint4* src = reinterpret_cast<const uint4*>(p.dict.lens);
        for (int i = threadIdx.x; i < C::LENS_BYTES / 16; i += blockDim.x) reinterpret_cast<uint4*>(s_lens)[i] = __ldg(src + i);
        __syncthreads();
    }
    const Extent x = column_extent(p, C::TILE);
    const uint8_t* lens = DSMEM ? s_lens : p.dict.lens;
    const u32 lane = threadIdx.x & 31u;
    const u32 rblock = blockIdx.x - index_blocks;
    const u64 warps = (u64)(gridDim.x - index_blocks) * (blockDim.x / 32);
    u32 err = 0;
    // rounds of U tiles; the next round's loads are in flight while this one computes
    constexpr int U = ReduceShape<CODEC, K>::U;
    if constexpr (!C::FSST && !PACKED) {
        // Escape-free codes in their own layout: tiles [t_lo, t_hi) lie wholly
        // inside the column and the code buffer; their lanes load their code
        // words at a fixed stride and sum their lengths straight from them
        // (32-bit tile indices: fewer than 2^32 tiles).  Edge tiles take the
        // general path.
        constexpr u32 TB = C::TILE * C::WBITS / 8;   // code bytes of a tile
        const u32 nt = (u32)x.n_tiles, W = (u32)warps;
        const u64 buf_slots = p.codes_bytes * 8 / C::WBITS;
        const u64 end = x.c_end < buf_slots ? x.c_end : buf_slots;
        const u64 lo64 = (x.c_begin + C::TILE - 1) / C::TILE, hi64 = end / C::TILE;
        const u32 t_lo = (u32)(lo64 - x.first_tile);
        const u32 t_hi = hi64 > lo64 ? (u32)(hi64 - x.first_tile) : t_lo;
        const uint8_t* base = p.codes + x.first_tile * (u64)TB + (u64)lane * C::LANE_BYTES;
        auto load = [&](u32 t, u32 (&w)[C::LANE_WORDS]) {
            if (C::LANE_BYTES % 16 == 0) {
                const uint4* src = reinterpret_cast<const uint4*>(base + (u64)t * TB);
#pragma unroll
                for (int v = 0; v < C::LANE_WORDS / 4; ++v) {
                    const uint4 a = __ldcs(src + v);
                    w[4 * v] = a.x; w[4 * v + 1] = a.y; w[4 * v + 2] = a.z; w[4 * v + 3] = a.w;
                }
            } else {
                const uint2* src = reinterpret_cast<const uint2*>(base + (u64)t * TB);
#pragma unroll
                for (int v = 0; v < C::LANE_WORDS / 2; ++v) {
                    const uint2 a = __ldcs(src + v);
                    w[2 * v] = a.x;
                    w[2 * v + 1] = a.y;
                }
            }
        };
        u32 t = (u32)rblock * (blockDim.x / 32) + (threadIdx.x >> 5);
        u32 wv[U][C::LANE_WORDS];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const u32 tt = t + u * W;
            if (tt >= t_lo && tt < t_hi) load(tt, wv[u]);
        }
        for (; t < nt; t += U * W) {
            u32 nv[U][C::LANE_WORDS];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const u32 tt = t + (U + u) * W;
                if (tt >= t_lo && tt < t_hi) load(tt, nv[u]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const u32 tt = t + u * W;
                if (tt >= nt) continue;
                if (tt >= t_lo && tt < t_hi) {
                    const u32 tot = __reduce_add_sync(0xffffffffu, C::lane_length_sum(wv[u], lens, err));
                    if (lane == 31) agg[tt] = tot;
                } else {
                    u32 gw[C::LANE_WORDS];
                    const bool fast = C::load_fast(p, C::lane_q0(x, tt), gw);
                    typename C::R r;
                    C::finish_load(p, x, C::lane_q0(x, tt), gw, fast, lens, r);
                    const TElem e = C::tile_element(r, lane, err);
                    if (lane == 31) agg[tt] = wt_pack<false>(e);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int i = 0; i < C::LANE_WORDS; ++i) wv[u][i] = nv[u][i];
        }
        if (err) atomicOr(p.err_word, err);
        return;
    }
    u64 t0 = (u64)rblock * (blockDim.x / 32) + (threadIdx.x >> 5);
    u32 wv[U][C::LANE_WORDS];
    bool fast[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const u64 t = t0 + u * warps;
        fast[u] = t < x.n_tiles && C::load_fast(p, C::lane_q0(x, t), wv[u]);
    }
    for (; t0 < x.n_tiles; t0 += U * warps) {
        u32 nv[U][C::LANE_WORDS];
        bool nfast[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const u64 t = t0 + (U + u) * warps;
            nfast[u] = t < x.n_tiles && C::load_fast(p, C::lane_q0(x, t), nv[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const u64 t = t0 + u * warps;
            if (t < x.n_tiles) {
                typename C::R r;
                C::finish_load(p, x, C::lane_q0(x, t), wv[u], fast[u], lens, r, s_pk + threadIdx.x * C::PK_STRIDE);
                const TElem e = C::tile_element(r, lane, err);
                if (lane == 31) agg[t] = wt_pack<C::FSST>(e);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int i = 0; i < C::LANE_WORDS; ++i) wv[u][i] = nv[u][i];
            fast[u] = nfast[u];
        }
    }
    if (err) atomicOr(p.err_word, err);
}

// ---------------------------------------------------------------------------
// Pass 2: exclusive scan of the warp-tile elements.  Blocks of 256 threads
// take 2,048 consecutive elements by ticket; decoupled look-back across
// blocks.  Writes ex[t] = bytes before warp tile t | entering state << 63.
// ---------------------------------------------------------------------------
constexpr int kScanPerThread = 8;
constexpr int kScanTile = 256 * kScanPerThread;

// Shared state of a tile-scan block.
struct ScanShared {
    Elem wsum[8];
    u64 excl_b;
    u32 excl_s;
    u32 ticket;
};

// Scan block b (of n_blocks) over elements agg[0, n) of one column: writes
// ex[] for its 2,048 elements, publishes its look-back word in status[b]
// (status words of this column only), and at the column's last block its
// decoded size and size errors.  Every thread of the block calls this.
template <bool FSST>
__device__ __forceinline__ void scan_block(const DecodeParams& p, const u64* agg, u64* ex, u64 n, u64 b, u64 n_blocks,
                                           unsigned long long* status, u32 epoch, WsHeader* ws, ScanShared& sh) {
    const u32 lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const u64 pad = FSST ? wt_pack<true>(telem_identity()) : 0ull;
    const u64 i0 = b * kScanTile + (u64)threadIdx.x * kScanPerThread;
    u64 w[kScanPerThread];
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) w[k] = (i0 + k < n) ? agg[i0 + k] : pad;
    // this thread's elements composed, then a block scan of 64-bit elements
    Elem e = elem_identity();
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) e = then<FSST>(e, wt_unpack<FSST>(w[k]));
    Elem inc = e;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        Elem y = shfl_up_e<FSST>(inc, d);
        if (lane < (u32)d) y = elem_identity();
        inc = then<FSST>(y, inc);
    }
    if (lane == 31) sh.wsum[warp] = inc;
    __syncthreads();
    Elem wex = elem_identity(), tot = elem_identity();
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const Elem sv = sh.wsum[v];
        if ((u32)v < warp) wex = then<FSST>(wex, sv);
        tot = then<FSST>(tot, sv);
    }
    Elem lex = shfl_up_e<FSST>(inc, 1);
    if (lane == 0) lex = elem_identity();
    lex = then<FSST>(wex, lex);   // the block's elements before this thread's
    if (warp == 0) {
        // publish the aggregate first, so later blocks need not wait for this look-back
        if (b > 0 && lane == 0) st_volatile(status + b, status_word(kFlagAgg, epoch, agg_payload_wide<FSST>(tot)));
        u64 eb = 0;
        u32 es = 0;
        if (b > 0) lookback<FSST, true>(status, (long long)b, epoch, ws, eb, es);
        if (lane == 0) {
            const u64 ib = eb + ((FSST && es) ? tot.b1 : tot.b0);
            const u32 is = FSST ? ((tot.n >> es) & 1u) : 0u;
            st_volatile(status + b, status_word(kFlagInc, epoch, inc_payload<FSST>(ib, is)));
            sh.excl_b = eb;
            sh.excl_s = es;
            if (b == n_blocks - 1) {
                *p.total_out = ib;
                if (ib > p.capacity && !p.size_only) atomicOr(p.err_word, ERRB_CAPACITY);
                if (ib > 0x7fffffffull) atomicOr(p.err_word, ERRB_OVERFLOW);
            }
        }
    }
    __syncthreads();
    const u64 eb = sh.excl_b;
    const u32 es = sh.excl_s;
    // each element's exclusive offset and entering state
    u64 ob = eb + ((FSST && es) ? lex.b1 : lex.b0);
    u32 os = FSST ? ((lex.n >> es) & 1u) : 0u;
#pragma unroll
    for (int k = 0; k < kScanPerThread; ++k) {
        if (i0 + k < n) ex[i0 + k] = ob | ((u64)os << 63);
        const Elem ek = wt_unpack<FSST>(w[k]);
        ob += (FSST && os) ? ek.b1 : ek.b0;
        os = FSST ? ((ek.n >> os) & 1u) : 0u;
    }
    __syncthreads();   // shared words are rewritten for the next ticket
}

template <bool FSST>
__global__ void __launch_bounds__(256) tiles_scan_kernel(const DecodeParams p, const Extent* xp, const u64* agg,
                                                         u64* ex, unsigned long long* status) {
    __shared__ ScanShared sh;
    WsHeader* ws = p.ws;
    grid_release();   // the decode may start launching (its blocks stage the dictionary, then wait)
    grid_wait();      // the reduce's elements and extent
    const Extent x = *xp;
    const u32 epoch = *(volatile u32*)&ws->epoch;
    const u64 n = x.n_tiles;
    const u64 n_blocks = (n + kScanTile - 1) / kScanTile;
    for (;;) {
        if (threadIdx.x == 0) sh.ticket = atomicAdd(&ws->tile_counter, 1u);
        __syncthreads();
        const u64 b = sh.ticket;
        if (b >= n_blocks) break;
        scan_block<FSST>(p, agg, ex, n, b, n_blocks, status, epoch, ws, sh);
        // with a block per scan block the first tickets cover them all: no
        // second ticket (one atomic round trip less at the end of the scan)
        if ((u64)gridDim.x >= n_blocks) break;
    }
    finish_launch(ws, epoch);
}

// ---------------------------------------------------------------------------
// Pass 3: every warp decodes warp tiles on its own (grid-stride order).
// ---------------------------------------------------------------------------
template <int CODEC, int K, bool DSMEM, int NW, int MINB, int W = WarpCore<CODEC, K, DSMEM>::TOK8 ? 8 : 16,
          bool PACKED = false>
__global__ void __launch_bounds__(NW * 32, MINB) warp_decode_kernel(const DecodeParams p, const Extent* xp,
                                                                     const u64* ex) {
    typedef WarpCore<CODEC, K, DSMEM, W, PACKED> C;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint4* s_dict = reinterpret_cast<uint4*>(smem_raw);
    uint8_t* s_lens = smem_raw + C::DICT_BYTES;
    WarpArea<K>* areas = reinterpret_cast<WarpArea<K>*>(smem_raw + C::DICT_BYTES + (DSMEM ? C::LENS_BYTES : 0));
    // packed codes: a scratch of PK_STRIDE words per lane after the warp areas
    u32* pk = PACKED ? reinterpret_cast<u32*>(areas + NW) + threadIdx.x * C::PK_STRIDE : nullptr;
    __shared__ __align__(8) u64 s_bar;
    if (C::BULK_STAGE) {
        C::stage_dict_bulk(p, s_dict, s_lens, &s_bar, NW * 32);
    } else if (DSMEM) {
        C::stage_dict(p, s_dict, s_lens, NW * 32);
        __syncthreads();
    }
    grid_wait();   // the tile scan's offsets (the dictionary staging above overlapped it)
    const Extent x = *xp;
    const uint8_t* lens = DSMEM ? s_lens : p.dict.lens;
    u32 err = 0;
    C::decode_tiles(p, x, ex, (u64)blockIdx.x * NW + (threadIdx.x >> 5), (u64)gridDim.x * NW, s_dict, lens,
                    areas[threadIdx.x >> 5], err, pk);
    if (err) atomicOr(p.err_word, err);
}


// ---------------------------------------------------------------------------
// Small columns in one cooperative launch: the three passes above as phases
// of one kernel, separated by grid barriers (bounded waits), so a column of
// a few thousand warp tiles pays one launch instead of three.
//   phase 1  index pass (every thread) and tile elements (every warp);
//   phase 2  block 0 scans the tile elements (one block is enough for the
//            sizes this path takes) and checks the decoded size;
//   phase 3  every warp decodes tiles, as warp_decode_kernel.
// Data written by earlier phases is read through L2 (ld.global.cg).
// ---------------------------------------------------------------------------
// Exclusive scan of n tile elements by one block of NT threads: ex[t] =
// bytes before tile t | entering state << 63; the decoded size and its
// checks as the tile scan's last block.
template <bool FSST, int NT>
__device__ __forceinline__ void block_scan_tiles(const DecodeParams& p, const u64* agg, u64* ex, u64 n, Elem* s_w) {
    const u32 lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const u64 per = (n + NT - 1) / NT;
    const u64 i0 = (u64)threadIdx.x * per, i1 = i0 + per < n ? i0 + per : n;
    Elem e = elem_identity();
    for (u64 i = i0; i < i1; ++i) e = then<FSST>(e, wt_unpack<FSST>(__ldcg(agg + i)));
    Elem inc = e;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        Elem y = shfl_up_e<FSST>(inc, d);
        if (lane < (u32)d) y = elem_identity();
        inc = then<FSST>(y, inc);
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    Elem before = elem_identity(), tot = elem_identity();
    for (int w = 0; w < NT / 32; ++w) {
        if ((u32)w < warp) before = then<FSST>(before, s_w[w]);
        tot = then<FSST>(tot, s_w[w]);
    }
    Elem lex = shfl_up_e<FSST>(inc, 1);
    if (lane == 0) lex = elem_identity();
    lex = then<FSST>(before, lex);
    u64 ob = lex.b0;   // the column is entered on a code: state 0
    u32 os = FSST ? (lex.n & 1u) : 0u;
    for (u64 i = i0; i < i1; ++i) {
        ex[i] = ob | ((u64)os << 63);
        const Elem ek = wt_unpack<FSST>(__ldcg(agg + i));
        ob += (FSST && os) ? ek.b1 : ek.b0;
        os = FSST ? ((ek.n >> os) & 1u) : 0u;
    }
    if (threadIdx.x == 0) {
        const u64 total = tot.b0;
        *p.total_out = total;
        if (total > p.capacity && !p.size_only) atomicOr(p.err_word, ERRB_CAPACITY);
        if (total > 0x7fffffffull) atomicOr(p.err_word, ERRB_OVERFLOW);
    }
}

template <int CODEC, int K, bool DSMEM, int NW, int W = WarpCore<CODEC, K, DSMEM>::TOK8 ? 8 : 16>
__global__ void __launch_bounds__(NW * 32, 1) fused_decode_kernel(const DecodeParams p, Extent* xp, u64* agg,
                                                                   u64* ex) {
    typedef WarpCore<CODEC, K, DSMEM, W> C;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ Elem s_w[NW];
    uint4* s_dict = reinterpret_cast<uint4*>(smem_raw);
    uint8_t* s_lens = smem_raw + C::DICT_BYTES;
    WarpArea<K>* areas = reinterpret_cast<WarpArea<K>*>(smem_raw + C::DICT_BYTES + (DSMEM ? C::LENS_BYTES : 0));
    if (DSMEM) {
        C::stage_dict(p, s_dict, s_lens, NW * 32);
        __syncthreads();
    }
    const uint8_t* lens = DSMEM ? s_lens : p.dict.lens;
    const u32 epoch = *(volatile u32*)&p.ws->epoch;
    const Extent x = column_extent(p, C::TILE);
    if (blockIdx.x == 0 && threadIdx.x == 0) *xp = x;
    const u32 lane = threadIdx.x & 31u;
    const u64 gwarp = (u64)blockIdx.x * NW + (threadIdx.x >> 5), gwarps = (u64)gridDim.x * NW;
    u32 err = 0;
    // phase 1
    index_groups(p, x, (u32)(__ffs(C::TILE) - 1), 0, (u64)p.n_strings + 1, (u64)blockIdx.x * blockDim.x + threadIdx.x,
                 (u64)gridDim.x * blockDim.x, const_cast<u32*>(p.first));
    for (u64 t = gwarp; t < x.n_tiles; t += gwarps) {
        u32 wv[C::LANE_WORDS];
        const u64 q0 = C::lane_q0(x, t);
        const bool fast = C::load_fast(p, q0, wv);
        typename C::R r;
        C::finish_load(p, x, q0, wv, fast, lens, r);
        const TElem e = C::tile_element(r, lane, err);
        if (lane == 31) agg[t] = wt_pack<C::FSST>(e);
    }
    grid_barrier(p.ws);
    // phase 2
    if (blockIdx.x == 0) block_scan_tiles<C::FSST, NW * 32>(p, agg, ex, x.n_tiles, s_w);
    grid_barrier(p.ws);
    // phase 3
    C::template decode_tiles<true>(p, x, ex, gwarp, gwarps, s_dict, lens, areas[threadIdx.x >> 5], err, nullptr);
    if (err) atomicOr(p.err_word, err);
    __syncthreads();
    finish_launch(p.ws, epoch);   // the last block out clears the abort flag and the stall settings
}

}  // namespace
}  // namespace fp
