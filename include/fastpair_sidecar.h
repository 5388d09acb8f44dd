/*
 * fastpair_sidecar.h -- decoding with a stored sidecar of output positions.
 *
 * The paper's decoder does not compute where each part of the output goes
 * while it decodes: it reads those positions from a small table written
 * when the column was compressed (the "sidecar", Sec. 3.1), and reports
 * that computing them at decode time instead costs about 20-35 %.  fp_decode
 * computes them on the device in two passes before it decodes (reduce and
 * tile scan).  These calls split that work: fp_sidecar_build computes the
 * table once and stores it in a caller buffer; fp_decode_sidecar decodes
 * from a stored table and runs neither pass.
 *
 * Sidecar format (uint64 entries, little-endian, in device memory):
 *   S = fp_sidecar_tile_slots(codec) code slots per tile (512 for OnPair-16,
 *   OnPair-12 and FSST-12, 1024 for FSST-8).  With c0 = code_offsets[0] and
 *   c1 = code_offsets[n_strings], the column's tiles are
 *   u = 0 .. T-1, T = max(1, ceil(c1 / S) - floor(c0 / S)), tile u starting
 *   at slot s_u = (floor(c0 / S) + u) * S.
 *     entry 0       total decoded bytes of the column;
 *     entry 1 + u   bytes produced by the column's slots before
 *                   max(s_u, c0), in bits 0..62; bit 63 = 1 if slot s_u is
 *                   the literal byte of an FSST-8 escape (always 0 for
 *                   OnPair and for u = 0).
 *   Entries after entry T are not read.  The table depends only on the
 *   codes, code_offsets and the dictionary's token lengths.
 *
 * Scratch: both calls take a caller-owned device scratch buffer of at least
 * fp_sidecar_scratch_bytes(codec, codes_bytes) bytes, 16-byte aligned, and
 * allocate nothing.  Calls that overlap on the GPU must not share a scratch
 * buffer or a status word.
 *
 * Status: d_status is one device uint32 that the call clears and then ORs
 * its data-error bits into, stream-ordered: 1 = corrupt input (as
 * fp_decode), 2 = decoded size above out_capacity, 4 = above 2^31-1, 8 = a
 * bounded device wait gave up, 16 = the table disagrees with the code
 * stream (fp_decode_sidecar: some tile's byte total, recomputed from its
 * codes, does not bring its entry to the next one).  The host-side return
 * value covers argument errors and launch failures only, as for fp_decode.
 *
 * A sidecar that does not belong to the column gives wrong output: the
 * decode places bytes where the table says, as the paper's does, and flags
 * the disagreement with bit 16 (it does not catch a table whose entries are
 * consistent with the codes but belong to other string boundaries).  Every
 * write still stays inside [0, out_capacity) of d_out_bytes and inside the
 * n_strings + 1 entries of d_out_offsets.
 */
#ifndef FASTPAIR_SIDECAR_H
#define FASTPAIR_SIDECAR_H

#include "fastpair.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Code slots per sidecar tile for `codec` (0 for an unknown codec). */
uint32_t fp_sidecar_tile_slots(fp_codec codec);

/* Entries a sidecar needs for any column whose code buffer has codes_bytes
 * bytes (an upper bound on 1 + T; 0 for an unknown codec). */
uint64_t fp_sidecar_entries(fp_codec codec, uint64_t codes_bytes);

/* Scratch bytes both calls need for a code buffer of codes_bytes bytes. */
uint64_t fp_sidecar_scratch_bytes(fp_codec codec, uint64_t codes_bytes);

/*
 * fp_sidecar_build -- compute the sidecar of a column.
 *
 * Inputs as fp_decode (dict, d_codes, codes_bytes, d_code_offsets,
 * n_strings).  d_sidecar: device, sidecar_entries >= fp_sidecar_entries()
 * uint64 entries, 8-byte aligned, written in the format above.  Two
 * launches, those that fp_decode runs before its decode (index pass and
 * reduce in one grid, tile scan); asynchronous.
 */
fp_status fp_sidecar_build(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                           const uint32_t* d_code_offsets, uint32_t n_strings, uint64_t* d_sidecar,
                           uint64_t sidecar_entries, void* d_scratch, uint64_t scratch_bytes,
                           uint32_t* d_status, fp_stream_t stream);

/*
 * fp_decode_sidecar -- fp_decode from a stored sidecar.
 *
 * Inputs and outputs as fp_decode, plus the sidecar (read only) and the
 * scratch.  Three launches: the index pass (the first string of every
 * tile), a size check against out_capacity, the warp-tile decode; no reduce
 * and no tile scan.  Asynchronous.
 */
fp_status fp_decode_sidecar(fp_codec codec, const fp_dict* dict, const void* d_codes, uint64_t codes_bytes,
                            const uint32_t* d_code_offsets, uint32_t n_strings, const uint64_t* d_sidecar,
                            uint64_t sidecar_entries, uint8_t* d_out_bytes, uint64_t out_capacity,
                            uint32_t* d_out_offsets, void* d_scratch, uint64_t scratch_bytes,
                            uint32_t* d_status, fp_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* FASTPAIR_SIDECAR_H */
