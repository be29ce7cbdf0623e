// Launch parameters of the Jiffy kernels, shared by the kernels and the
// host-side API in this directory.
//
// A call codes one or more segments: a segment is one stream's part of the
// call (T consecutive scans of one stream). Row items (scan t, attribute a,
// row r) and sections (scan t, attribute a) are numbered globally across the
// segments of a call, segment after segment. Within a segment, sections are
// ordered (t, a); the encoder's row items are ordered (a, t, r) (attribute-
// major), and so are the decoder's.
#pragma once

#include <cstdint>

#include "jiffy_types.h"

namespace jiffy {

struct EncSeg {
  uint32_t H, W, A, T;
  uint32_t nw, ncls;             // mask words per row, class words per row (0 without the mask stage)
  uint32_t stages;               // kStage* switches of the stream
  uint32_t frame0;               // scan index of the segment's first frame
  uint32_t shdr;                 // stream header bytes at the start of out (0 or 16 + 8A)
  uint32_t fhdr;                 // frame header bytes (8 + 12A)
  uint32_t test_lines;
  int32_t force_mode;
  uint32_t item_base;            // first global row item of the segment
  uint32_t sec_base;             // first global section of the segment
  uint32_t slot_bytes;           // per-row slot size (row_bound(W) rounded to 16)
  unsigned long long slot_base;  // byte offset of the segment's first slot
  const AttrDev* attrs;          // [A]
  const uint8_t* const* cur;     // [T*A] current planes
  const uint8_t* const* prev;    // [T*A] previous planes: t = 0 -> stored scan (or null), else raw t-1
  uint8_t* const* state_next;    // [A] receives the last scan as decoded (q * P)
  uint8_t* out;
  unsigned long long cap;
  unsigned long long* frame_off; // [T+1]
  uint32_t* err;                 // the segment's error word
  // Zstandard mask (stages & kStageZstdMask): each section's coded mask
  // bytes (rows of zm_rb = ceil(W/8) bytes) at zm_base + section * zm_stride
  // in EncParams::zmask, its zm_nblk blocks in slots zb_base + section *
  // zm_nblk + j of EncParams::zblk
  uint32_t zm_rb, zm_nblk;
  unsigned long long zm_base, zm_stride, zb_base;
};

struct EncParams {
  uint32_t n_seg;
  uint32_t n_items;              // row items of all segments
  uint32_t n_sec;                // sections of all segments
  uint32_t max_W;                // widest row (per-warp shared memory)
  uint32_t trial_rows;           // most distinct test rows of a segment (0: no trial)
  const EncSeg* seg;             // [n_seg]
  const uint32_t* seg_item_base; // [n_seg] (search key for row items)
  const uint32_t* seg_sec_base;  // [n_seg] (search key for sections)
  uint32_t* cost;                // [2 n_sec] trial bytes of I and P (zeroed)
  uint32_t* modes;               // [n_sec]
  uint32_t* row_bytes;           // [n_items] chunk bytes
  uint32_t* row_nnz;             // [n_items]
  uint32_t* row_carry;           // [n_items]
  unsigned long long* st_carry;  // [n_items] look-back status, delta carry (zeroed)
  uint8_t* slots;                // packed row chunks, slot_base + local item * slot_bytes
  unsigned long long* sec_bytes; // [n_sec] section bytes (row table + chunks)
  uint32_t* sec_nnz;             // [n_sec]
  uint32_t* ticket;
  uint32_t wpc;                  // rows kernel: warps per CTA (1, 2, 4; 0 = by shared memory)
  uint32_t ctas_per_sm;          // rows kernel: resident CTAs per SM (0 = occupancy limit)
  uint32_t staged;               // 1: launch the rows kernel that reads stage switches and the test hook
  uint32_t withhold;             // test hook: 1 + the row item that does not publish its carry status (0: none)
  // rows kernel launches: items [item_lo, n_items) from ticket word ticket[0];
  // split > 0: the launcher runs two rows launches, items [0, split) sized for
  // rows of at most split_W columns, then [split, n_items) from ticket[1]
  uint32_t item_lo;
  uint32_t split, split_W;
  // Zstandard mask sections (null when no segment codes its mask that way)
  uint8_t* zmask;                // coded mask bytes of the sections
  uint8_t* zblk;                 // block slots, kZSlot bytes each
  uint32_t* zblk_bytes;          // [blocks] bytes of each block (header included)
  uint32_t* zfr_bytes;           // [n_sec] frame bytes of each section
  uint32_t zmax_blk;             // most blocks of a section
};

struct DecSeg {
  uint32_t H, W, A, T;
  uint32_t nw, ncls;             // as in EncSeg
  uint32_t stages;
  uint32_t frame0;
  uint32_t fhdr;
  uint32_t check_shdr;           // validate the stream header at in[0]
  uint32_t item_base;
  const AttrDev* attrs;
  const uint8_t* in;
  unsigned long long in_len;
  const unsigned long long* off; // [T+1] frame offsets in `in`
  uint8_t* const* outp;          // [T*A] output planes
  const uint8_t* const* state;   // [A] previous decoded planes (for the segment's first frame)
  uint8_t* const* state_next;    // [A] receives the last frame's planes
  uint32_t* err;                 // the segment's error word
  unsigned long long mask_base;  // word offset of the segment's first row in DecParams::masks
  uint32_t sec_base;             // first global section (scan t, attribute a) of the segment
  uint32_t zm_rb, zm_nblk;       // Zstandard mask: bytes per row, blocks per section
  unsigned long long zm_base, zm_stride;  // its decoded mask bytes in DecParams::zdec
};

struct DecParams {
  uint32_t n_seg;
  uint32_t n_items;
  uint32_t max_W;
  const DecSeg* seg;             // [n_seg]
  const uint32_t* seg_item_base; // [n_seg]
  uint32_t* done;                // [n_items] row-done flags
  uint32_t* masks;               // decoded zero masks, nw words per row item (read by the next frame's P rows)
  uint32_t* ticket;
  uint32_t wpc;                  // warps per CTA (1, 2, 4, 8; 0 = by shared memory)
  uint32_t ctas_per_sm;          // resident CTAs per SM (0 = occupancy limit)
  uint32_t items_per_ticket;     // row items a warp takes per ticket (0 = 4)
  uint32_t staged;               // as in EncParams
  uint32_t withhold;             // test hook: 1 + the row item that does not publish its done flag (0: none)
  // Zstandard mask sections (null when no segment codes its mask that way)
  uint32_t n_sec;                // sections of all segments
  const uint32_t* seg_sec_base;  // [n_seg] (search key for sections)
  uint8_t* zdec;                 // decoded (still XORed) mask bytes of the sections
  uint32_t zmax_blk;             // most blocks of a section
};

// Launch configuration of a rows kernel as resolved for given parameters
// (requests clamped to what fits the device).
struct RowsLaunch {
  uint32_t wpc, ctas_per_sm, items_per_ticket, grid;
};

size_t enc_smem_bytes_host(uint32_t W);
size_t trial_smem_bytes_host(uint32_t W);
size_t dec_smem_bytes_host(uint32_t W);
// Return a cudaError_t as int; *out receives the configuration.
int encode_rows_launch(const EncParams& p, RowsLaunch* out);
int decode_rows_launch(const DecParams& p, RowsLaunch* out);

// Launchers (return a cudaError_t as int). ev: null, or events (cudaEvent_t
// as void*) recorded before each kernel and after the last one (encode: 4,
// decode: 2).
int launch_encode(const EncParams& p, void* stream, void* const* ev);
int launch_decode(const DecParams& p, void* stream, void* const* ev);

// Zstandard mask kernels (jiffy_zstd.cu): the writer of every block of the
// Zstandard sections (after the rows kernel, before the placement kernels)
// and the reader of them (before the rows kernel of a decode).
int launch_zstd_encode(const EncParams& p, void* stream);
int launch_zstd_decode(const DecParams& p, void* stream);

}  // namespace jiffy
