// Constants and plain types shared by the Jiffy kernels and the host API.
#pragma once

#include <cstddef>
#include <cstdint>

#if defined(__CUDACC__)
#define JIFFY_HD __host__ __device__
#else
#define JIFFY_HD
#endif

namespace jiffy {

constexpr int kThreads = 256;          // threads per CTA of the per-section kernels
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kMaxW = 16384;      // columns
constexpr uint32_t kMaxH = 4096;       // rows
constexpr uint32_t kMaxAttr = 64;
constexpr uint32_t kBlockN = 128;      // values per packing block (Sec. II frames of 128)

// Stage switches of a stream: the first three each remove one step of the
// codec, for the ablated codecs of Sec. IV-H (Table IV); kStageZstdMask codes
// the zero mask the way Sec. III-C does, one Zstandard frame per section,
// instead of the per-row class words. 0 = the full codec with class words.
enum : uint32_t { kStageNoMask = 1u, kStageNoDelta = 2u, kStageNoZigzag = 4u, kStageZstdMask = 8u, kStageAll = 15u };

// First word of an attribute's stream-header entry: dtype bytes, ZigZag
// variant (1 = Eq. 1, 0 = none), stage flags (bit 0 no mask, bit 1 no delta,
// bit 2 Zstandard mask), 0.
JIFFY_HD inline uint32_t attr_header_word(uint32_t s, uint32_t stages) {
  const uint32_t flags = (stages & (kStageNoMask | kStageNoDelta)) | ((stages & kStageZstdMask) ? 4u : 0u);
  return s | (((stages & kStageNoZigzag) ? 0u : 1u) << 8) | (flags << 16);
}

// Zstandard mask (RFC 8878 frames): mask bytes per block, bytes of the frame
// header (magic, descriptor, 4-byte content size), bytes of a block's slot in
// the encoder's scratch (the largest block, Raw, is 3 + kZBlock bytes).
constexpr uint32_t kZBlock = 8192;
constexpr uint32_t kZFrameHdr = 9;
constexpr uint32_t kZSlot = kZBlock + 16;

// Zstandard mask part of a section: u32 frame bytes, u32 end of each block,
// the frame, zero bytes up to a multiple of 4.
JIFFY_HD inline uint32_t zmask_blocks(uint32_t H, uint32_t W) {
  const uint32_t n = H * ((W + 7u) / 8u);
  return n ? (n + kZBlock - 1u) / kZBlock : 1u;
}
JIFFY_HD inline uint32_t zmask_part_bytes(uint32_t nblk, uint32_t frame_bytes) {
  return (4u + 4u * nblk + frame_bytes + 3u) & ~3u;
}

// bits of the device error word
enum : uint32_t { kErrCorrupt = 1u, kErrCapacity = 2u, kErrTimeout = 4u };

// Wall-clock bound of every spin-wait (ns); a wait that runs out sets
// kErrTimeout and the kernel returns instead of hanging.
constexpr unsigned long long kSpinLimitNs = 2000000000ull;

// Quantizer of one attribute (Sec. III-B): q = min(floor((v + half) / P), qmax).
//   qkind 0: P = 1, q = v.
//   qkind 1: q = umulhi(min(v, lim) + half, m32) >> sh. lim = the largest v
//            whose q is not clamped (capped so that lim + half < 2^32); any
//            larger v gives q = qmax, and so does lim. (m32, sh) divides
//            every 32-bit dividend exactly: m32 = ceil(2^(32+sh) / P) with
//            m32 P - 2^(32+sh) <= 2^sh (Granlund and Montgomery, "Division by
//            invariant integers using multiplication", 1994, Thm. 4.2).
//   qkind 2: no 32-bit multiplier exists: 64-bit reciprocal `magic` =
//            ceil(2^64 / P).
struct AttrDev {
  uint32_t s;                 // bytes per sample: 1, 2 or 4
  uint32_t P;                 // precision
  uint32_t qmax;              // floor(max_sample / P)
  uint32_t qkind;
  unsigned long long magic;   // ceil(2^64 / P), for 2 <= P <= 2^31
  uint32_t m32, sh;           // qkind 1 multiplier and shift
  uint32_t half;              // floor(P / 2)
  uint32_t lim;               // qkind 1 input clamp
};

inline AttrDev make_attr(uint32_t s, uint32_t P) {
  AttrDev d{};
  d.s = s;
  d.P = P;
  const uint32_t maxv = s == 4 ? 0xffffffffu : ((1u << (8 * s)) - 1u);
  d.qmax = maxv / P;
  d.half = P >> 1;
  d.magic = (P >= 2 && P <= 0x80000000u) ? (~0ull) / P + 1ull : 0ull;
  d.qkind = 2;
  if (P == 1) {
    d.qkind = 0;
    return d;
  }
  for (uint32_t l = 0; l < 32; l++) {
    const unsigned __int128 two = (unsigned __int128)1 << (32 + l);
    const unsigned __int128 m = (two + P - 1) / P;
    if (m >> 32) break;  // multipliers only grow with l
    if (m * P - two <= ((unsigned __int128)1 << l)) {
      d.qkind = 1;
      d.m32 = (uint32_t)m;
      d.sh = l;
      const unsigned long long top = (unsigned long long)d.qmax * P + (P - 1) - d.half;
      const unsigned long long cap = 0xffffffffull - d.half;
      d.lim = (uint32_t)(top < cap ? top : cap);
      break;
    }
  }
  return d;
}

JIFFY_HD inline uint32_t ceil_div_u32(uint32_t a, uint32_t b) { return (a + b - 1) / b; }

// Worst-case bytes of one row chunk: class words, literals, block headers and
// bodies (with b = wmax a block of m values never exceeds 4m bytes and the
// chosen b never needs more).
JIFFY_HD inline uint32_t row_bound_bytes(uint32_t W) {
  uint32_t nw = ceil_div_u32(W, 32);
  return 4u * ceil_div_u32(nw, 16) + 4u * nw + 4u * ceil_div_u32(W, kBlockN) + 4u * W;
}

}  // namespace jiffy
