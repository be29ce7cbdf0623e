// Jiffy encoder kernels (sm_103a).
//
// One call codes T consecutive scans of each of one or more streams (the
// segments of the call), all in parallel: the P prediction of scan t uses the
// *input* of scan t-1 (Sec. III-D), so no scan waits for another's output.
// Launches:
//   k_trial     one warp per (section, test row): I and P residuals of the
//               scanline, delta chained across the test rows, priced with
//               the block-width choice below; the bytes add up per section
//               and mode (trial compression, mask excluded, Sec. III-E, IV-E).
//   k_encode    one warp per row item (scan, attribute, row), items taken in
//               ticket order. Per row:
//     pass A    8 consecutive pixels per lane per 256-pixel step: quantize
//               (Sec. III-B), zero bitmask (Sec. III-C), mask XOR with the
//               previous scan for P (Sec. III-D), residual (I: q, P: q - q'),
//               compaction of the kept samples (warp scan of counts) into a
//               padded shared buffer.
//     steps     1024 compacted values at a time, 32 consecutive ones per
//               lane (a block of 128 = 4 lanes): delta (Sec. III-C) from the
//               previous row's last residual, ZigZag (Eq. 1), the
//               byte-minimal width of every block (Sec. II, PFOR: counts of
//               the values wider than b for all b at once, carry-save adders
//               over unary width codes, bit-sliced across the block's 4
//               lanes), then each lane packs its 32 values' low bits -- b
//               words exactly -- and its exceptions (positions, high parts)
//               straight into the row's chunk in global memory. No lane
//               waits for another lane's words: the only words two lanes
//               share (the ends of their high-part runs) are merged in
//               registers through shuffles.
//     The mask code and block headers complete the chunk, which goes to the
//     row's slot; rows never wait for one another's sizes (sections differ a
//     lot in cost, and an in-order prefix over rows would queue fast rows
//     behind slow ones).
//   k_sec_sizes one CTA per section: its bytes and nonzero count.
//   k_place     one CTA per section: offset (sum over the earlier sections),
//               row table, frame and stream headers, and the copy of every
//               row chunk from its slot to its place in the stream.
#include "jiffy_device.cuh"
#include "jiffy_kernels.h"

namespace jiffy {

namespace {

constexpr uint32_t kStepPx = 256;    // pixels per warp step of pass A (8 per lane)
constexpr uint32_t kStepVal = 1024;  // values per warp step of the packing (32 per lane)
constexpr uint32_t kFull = 0xffffffffu;

// Compacted-value buffer: value k at word k + 4 floor(k / 32), i.e. every
// 32-value segment is followed by 4 pad words (segment stride 144 bytes).
// A lane reading a whole segment as 8 16-byte vectors and lanes storing
// consecutive values both spread over all 32 banks.
constexpr uint32_t kSegWords = 36;
__device__ __forceinline__ uint32_t zaddr(uint32_t k) { return k + ((k >> 5) << 2); }
__host__ __device__ inline uint32_t zbuf_words(uint32_t W) {
  return ceil_div_u32(W, kStepVal) * (kStepVal / 32u) * kSegWords;
}

__device__ __forceinline__ uint32_t find_seg(const uint32_t* base, uint32_t n, uint32_t key) {
  uint32_t lo = 0, hi = n;  // base[lo] <= key < base[hi] (base[n] = infinity)
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(base + mid) <= key) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Row items of a segment are numbered attribute-major, (a, t, r): the rows a
// warp takes next are of the attribute it just coded, so resident warps run
// the same code (the kernel is large; mixing attributes thrashes instruction
// fetch), and a section's rows stay consecutive for the carry look-back.
__device__ __forceinline__ uint32_t enc_item(const EncSeg& sg, uint32_t t, uint32_t a, uint32_t r) {
  return (a * sg.T + t) * sg.H + r;
}

// Bulk prefetch of [p, p + bytes) into L2 (the 16-byte aligned part of it).
__device__ __forceinline__ void prefetch_l2(const uint8_t* p, size_t bytes) {
  const uintptr_t c0 = reinterpret_cast<uintptr_t>(p), c1 = c0 + bytes;
  const uintptr_t a0 = (c0 + 15u) & ~uintptr_t(15), a1 = c1 & ~uintptr_t(15);
  if (a1 > a0) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"((uint32_t)(a1 - a0)) : "memory");
}

__device__ __forceinline__ uint32_t mask_class(uint32_t c, uint32_t valid) {
  return c == 0u ? 0u : (c == valid ? 1u : 2u);
}

__device__ __forceinline__ uint32_t valid_bits(uint32_t W, uint32_t nw, uint32_t j) {
  return (j + 1 < nw || (W & 31u) == 0) ? 0xffffffffu : ((1u << (W & 31u)) - 1u);
}

// Mode of section (scan t, attribute a): the first frame after create/reset
// is I; forced modes; else P iff the trial priced P strictly cheaper.
__device__ __forceinline__ uint32_t section_mode(const EncParams& p, const EncSeg& sg, uint32_t sec, uint32_t t) {
  if (sg.frame0 + t == 0 || sg.force_mode == 0) return 0u;
  if (sg.force_mode == 1) return 1u;
  return p.cost[2 * sec + 1] < p.cost[2 * sec] ? 1u : 0u;
}

// Loads / stores 8 samples with the width fixed at compile time (S = 1, 2,
// 4) or read at run time (S = 0).
template <uint32_t S>
__device__ __forceinline__ void ld8(const uint8_t* row, uint32_t s, uint32_t x0, uint32_t nv, bool vec,
                                    uint32_t (&v)[8]) {
  if constexpr (S == 0) load8<false>(row, s, x0, nv, vec, v);
  else load8s<S, false>(row, x0, nv, vec, v);
}
template <uint32_t S>
__device__ __forceinline__ void st8(uint8_t* row, uint32_t s, uint32_t x0, uint32_t nv, bool vec,
                                    const uint32_t (&v)[8]) {
  if constexpr (S == 0) store8(row, s, x0, nv, vec, v);
  else store8s<S>(row, x0, nv, vec, v);
}

// ZigZag of a delta known to satisfy |d| < 2^30: with t = 2d, Eq. 1 gives
// t for d >= 0 and 1 - t for d < 0, and in that range the wanted one is the
// smaller as an unsigned number (d >= 0: 1 - t wraps above 2^31 unless d = 0,
// where 0 < 1; d < 0: t wraps above 2^31, 1 - t = 2|d| + 1 < 2^31 + 1).
// Three adds and a min, none of them on the logic/shift pipe.
__device__ __forceinline__ uint32_t zigzag_small(uint32_t d) {
  const uint32_t t = d + d;
  return min(t, 1u - t);
}

__device__ __forceinline__ void quant8(uint32_t (&v)[8], const AttrDev& at) {
  if (at.qkind == 1) {
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = quant<1>(v[i], at);
  } else if (at.qkind == 2) {
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] = quant<2>(v[i], at);
  }
}

// ---------------------------------------------------------------------------
// Pass A (one row): returns the number n of kept samples (the nonzero ones;
// all samples with kz = 0, i.e. without the mask stage); their residuals (I:
// q, P with prv: q - q', Sec. III-D) go to zb in row-major order (padded
// layout), the coded mask bytes (M, or M xor M_prev for P, Sec. III-C/D) to
// mb. qhi receives the largest quantized sample of the row (current and
// previous scan) for 4-byte samples (0 otherwise). One copy of the code
// serves every sample width, quantizer and mode (warp-uniform branches
// around small blocks): the kernel is bound by instruction fetch, so its
// footprint matters more than a few uniform branches per step.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t pass_a(const uint8_t* cur, const uint8_t* prv, const AttrDev& at, uint32_t W,
                                           uint32_t kz, uint32_t* zb, uint8_t* mb, uint32_t& qhi) {
  const uint32_t lane = lane_id(), s = at.s;
  const bool vc = vec_ok(cur, s), vp = prv && vec_ok(prv, s);
  const uint32_t Wm = (W + 31u) & ~31u;
  uint32_t n = 0, qm = 0;
  for (uint32_t base = 0; base < W; base += kStepPx) {
    const uint32_t x0 = base + 8u * lane;
    const uint32_t nv = x0 < W ? min(8u, W - x0) : 0u;
    uint32_t v[8];
    load8<false>(cur, s, x0, nv, vc, v);
    quant8(v, at);
    uint32_t keep = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) keep += min(v[i], 1u) << i;  // 1 = nonzero
    if (s == 4) {
#pragma unroll
      for (int i = 0; i < 8; i++) qm = max(qm, v[i]);
    }
    const uint32_t vm = (1u << nv) - 1u;
    uint32_t code = ~keep & vm & kz;  // 1 = zero sample
    if (prv) {
      uint32_t pv[8];
      load8<false>(prv, s, x0, nv, vp, pv);
      quant8(pv, at);
      uint32_t pkeep = 0;
#pragma unroll
      for (int i = 0; i < 8; i++) {
        pkeep += min(pv[i], 1u) << i;
        if (s == 4) qm = max(qm, pv[i]);
        v[i] -= pv[i];  // modulo 2^32
      }
      code ^= ~pkeep & vm & kz;
    }
    keep = kz ? (keep & vm) : vm;
    if (x0 < Wm) mb[x0 >> 3] = (uint8_t)code;
    uint32_t tot;
    uint32_t kk = n + warp_excl_scan(__popc(keep), tot);
#pragma unroll
    for (int i = 0; i < 8; i++) {
      if ((keep >> i) & 1u) {
        zb[zaddr(kk)] = v[i];
        kk++;
      }
    }
    n += tot;
  }
  qhi = __reduce_max_sync(kFull, qm);
  return n;
}

// The call's last scan of a row, dequantized (q * P) as the decoder holds it:
// the next call's previous scan.
__device__ __noinline__ void state_row(const uint8_t* cur, uint8_t* st_row, const AttrDev at, uint32_t W) {
  const uint32_t lane = lane_id(), s = at.s;
  const bool vc = vec_ok(cur, s), vs = vec_ok(st_row, s);
  for (uint32_t base = 0; base < W; base += kStepPx) {
    const uint32_t x0 = base + 8u * lane;
    const uint32_t nv = x0 < W ? min(8u, W - x0) : 0u;
    if (!nv) continue;
    uint32_t v[8];
    load8<false>(cur, s, x0, nv, vc, v);
    quant8(v, at);
#pragma unroll
    for (int i = 0; i < 8; i++) v[i] *= at.P;
    store8(st_row, s, x0, nv, vs, v);
  }
}

// Pass A of the trial: the residuals of the row's kept samples both ways (I
// to zi, P to zp).
template <int QU>
__device__ __forceinline__ uint32_t pass_a_trial(const uint8_t* cur, const uint8_t* prv, const AttrDev at, uint32_t W,
                                              uint32_t kz, bool pmode, uint32_t* zb) {
  const uint32_t lane = lane_id(), S = at.s;
  const bool vc = vec_ok(cur, S), vp = vec_ok(prv, S);
  uint32_t n = 0;
  for (uint32_t base = 0; base < W; base += kStepPx) {
    const uint32_t x0 = base + 8u * lane;
    const uint32_t nv = x0 < W ? min(8u, W - x0) : 0u;
    uint32_t v[8], pv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    load8<false>(cur, S, x0, nv, vc, v);
    if (pmode) load8<false>(prv, S, x0, nv, vp, pv);
    uint32_t zm = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      v[i] = quant<QU>(v[i], at);
      if (pmode) pv[i] = v[i] - quant<QU>(pv[i], at);
      zm |= (v[i] == 0u ? 1u : 0u) << i;
    }
    const uint32_t nz = ~(zm & kz) & ((1u << nv) - 1u);
    uint32_t tot;
    uint32_t kk = n + warp_excl_scan(__popc(nz), tot);
#pragma unroll
    for (int i = 0; i < 8; i++) {
      if ((nz >> i) & 1u) {
        zb[zaddr(kk)] = pmode ? pv[i] : v[i];
        kk++;
      }
    }
    n += tot;
  }
  return n;
}

// The residuals (I and, with prv, P) of the last nonzero sample (with all,
// the last sample) among the row's last max_steps 256-pixel steps. Returns
// false if there is none.
template <int QU>
__device__ __noinline__ bool row_last(const uint8_t* cur, const uint8_t* prv, const AttrDev at, uint32_t W,
                                      uint32_t max_steps, bool all, uint32_t* e_i, uint32_t* e_p) {
  const uint32_t lane = lane_id(), S = at.s;
  const uint32_t nsteps = ceil_div_u32(W, kStepPx);
  const bool vc = vec_ok(cur, S), vp = prv && vec_ok(prv, S);
  for (uint32_t si = 0; si < min(nsteps, max_steps); si++) {
    const uint32_t x0 = kStepPx * (nsteps - 1u - si) + 8u * lane;
    const uint32_t nv = x0 < W ? min(8u, W - x0) : 0u;
    uint32_t v[8], pv[8];
    load8<false>(cur, S, x0, nv, vc, v);
    if (prv) load8<false>(prv, S, x0, nv, vp, pv);
    bool has = false;
    uint32_t li = 0, lp = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      const uint32_t q = quant<QU>(v[i], at);
      if ((uint32_t)i < nv && (q != 0u || all)) {
        has = true;
        li = q;
        lp = prv ? q - quant<QU>(pv[i], at) : q;
      }
    }
    const uint32_t hm = __ballot_sync(kFull, has);
    if (hm) {
      const uint32_t src = 31u - __clz(hm);
      *e_i = __shfl_sync(kFull, li, src);
      *e_p = __shfl_sync(kFull, lp, src);
      return true;
    }
  }
  return false;
}

// Values n .. (end of the last 1024-value step) repeat `last` (the last
// residual, or 0 without the delta stage), so that their deltas are 0 and
// they count as zero-width values.
__device__ __forceinline__ void fill_tail(uint32_t* zb, uint32_t n, uint32_t last) {
  const uint32_t end = (n + kStepVal - 1) / kStepVal * kStepVal;
  for (uint32_t k = n + lane_id(); k < end; k += 32u) zb[zaddr(k)] = last;
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Block width (Sec. II, PFOR): b in [0, wmax] minimising the block's body
// bytes, ties to the smallest b. Warp-wide: lane l holds the 32 consecutive
// values z of its segment, the 4 lanes 4g'..4g'+3 (j = l & 3) hold one block
// of m values (the values past m are 0). For each value, its unary width
// code has bit b set iff the value needs more than b bits, so the column
// sums of a block's unary codes are e_b = #values wider than b, for all b at
// once: carry-save adders give each lane its 6 bit planes (counts <= 32),
// two bit-sliced additions across the block's 4 lanes give 8 planes (counts
// <= 128). Each lane then prices the candidates b = j, j+4, ... Returns
// f << 14 | b << 8 | e (f = body bytes), the same in the block's 4 lanes
// (all ones for m = 0); wmax = the bits of the block's widest value.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t block_width(const uint32_t (&z)[32], uint32_t j, uint32_t m, uint32_t& wmax) {
  // per-lane column counts of the unary width codes: 6 bit planes
  uint32_t p1, p2, p4, p8, p16, p32;
  {
    uint32_t ones = 0, twos = 0, fours = 0, eights = 0, sixteens[2];
#pragma unroll
    for (int h = 0; h < 2; h++) {
      uint32_t ta, tb, fa, fb, ea, eb;
      const int o = 16 * h;
      csa(ta, ones, ones, width_unary(z[o + 0]), width_unary(z[o + 1]));
      csa(tb, ones, ones, width_unary(z[o + 2]), width_unary(z[o + 3]));
      csa(fa, twos, twos, ta, tb);
      csa(ta, ones, ones, width_unary(z[o + 4]), width_unary(z[o + 5]));
      csa(tb, ones, ones, width_unary(z[o + 6]), width_unary(z[o + 7]));
      csa(fb, twos, twos, ta, tb);
      csa(ea, fours, fours, fa, fb);
      csa(ta, ones, ones, width_unary(z[o + 8]), width_unary(z[o + 9]));
      csa(tb, ones, ones, width_unary(z[o + 10]), width_unary(z[o + 11]));
      csa(fa, twos, twos, ta, tb);
      csa(ta, ones, ones, width_unary(z[o + 12]), width_unary(z[o + 13]));
      csa(tb, ones, ones, width_unary(z[o + 14]), width_unary(z[o + 15]));
      csa(fb, twos, twos, ta, tb);
      csa(eb, fours, fours, fa, fb);
      csa(sixteens[h], eights, eights, ea, eb);
    }
    p1 = ones; p2 = twos; p4 = fours; p8 = eights;
    p16 = sixteens[0] ^ sixteens[1];
    p32 = sixteens[0] & sixteens[1];
  }
  // bit-sliced sums across the block's 4 lanes: 8 planes E[0..7]
  uint32_t E[8];
  {
    uint32_t A[6] = {p1, p2, p4, p8, p16, p32}, B[7];
#pragma unroll
    for (int k = 0; k < 6; k++) B[k] = __shfl_xor_sync(kFull, A[k], 1);
    uint32_t C[7], c = 0;
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const uint32_t u = A[k] ^ B[k];
      C[k] = u ^ c;
      c = (A[k] & B[k]) | (u & c);
    }
    C[6] = c;
#pragma unroll
    for (int k = 0; k < 7; k++) B[k] = __shfl_xor_sync(kFull, C[k], 2);
    c = 0;
#pragma unroll
    for (int k = 0; k < 7; k++) {
      const uint32_t u = C[k] ^ B[k];
      E[k] = u ^ c;
      c = (C[k] & B[k]) | (u & c);
    }
    E[7] = c;
  }
  const uint32_t anyb = E[0] | E[1] | E[2] | E[3] | E[4] | E[5] | E[6] | E[7];
  wmax = 32u - __clz(anyb);  // e_b > 0 exactly for b < wmax
  // e_b for b = j + 4i: nibble i of lo (low 4 bits) and hi (high 4 bits)
  uint32_t lo4, hi4;
  {
    uint32_t F[8];
#pragma unroll
    for (int k = 0; k < 8; k++) F[k] = (E[k] >> j) & 0x11111111u;
    lo4 = F[0] + 2u * F[1] + 4u * F[2] + 8u * F[3];
    hi4 = F[4] + 2u * F[5] + 4u * F[6] + 8u * F[7];
  }
  // candidates in increasing b; the low-bit words alone, 4 ceil(mb/32),
  // bound a candidate's bytes from below, so once that bound reaches the
  // lane's best so far no larger b can win (ties go to the smaller b)
  uint32_t key = 0xffffffffu;
#pragma unroll
  for (uint32_t i = 0; i < 9; i++) {
    const uint32_t b = j + 4u * i;
    const uint32_t low = 4u * ((m * b + 31u) >> 5);
    const bool live = m != 0u && b <= wmax && low < (key >> 14);
    if (!__any_sync(kFull, live)) break;
    if (live) {
      const uint32_t e = i < 8 ? ((lo4 >> (4 * i)) & 15u) | (((hi4 >> (4 * i)) & 15u) << 4) : 0u;
      const uint32_t f = low + ((e + 3u) & ~3u) + 4u * ((e * (wmax - b) + 31u) >> 5);
      key = min(key, (f << 14) | (b << 8) | e);
    }
  }
  key = min(key, __shfl_xor_sync(kFull, key, 1));
  key = min(key, __shfl_xor_sync(kFull, key, 2));
  return key;
}

// Delta (Sec. III-C) and ZigZag (Eq. 1) of a lane's 32 consecutive residuals
// in place; pred = the residual before the first. FAST: every delta is below
// 2^30 in magnitude (zigzag_small). st: stage switches (delta and ZigZag may
// be off, Sec. IV-H).
template <bool STAGED, bool FAST>
__device__ __forceinline__ void delta_zigzag(uint32_t (&z)[32], uint32_t pred, uint32_t st) {
  if (!STAGED || !(st & (kStageNoDelta | kStageNoZigzag))) {
#pragma unroll
    for (int i = 31; i >= 0; i--) {
      const uint32_t d = z[i] - (i ? z[i - 1] : pred);
      z[i] = FAST ? zigzag_small(d) : zigzag(d);
    }
  } else {  // ablated codecs (Sec. IV-H); values past n are 0 without the delta
#pragma unroll
    for (int i = 31; i >= 0; i--) {
      const uint32_t d = (st & kStageNoDelta) ? z[i] : z[i] - (i ? z[i - 1] : pred);
      z[i] = (st & kStageNoZigzag) ? d : zigzag(d);
    }
  }
}

// Loads a lane's segment (32 consecutive values) from the padded buffer.
__device__ __forceinline__ void load_seg(const uint32_t* zb, uint32_t seg, uint32_t (&z)[32]) {
  const uint4* sp = reinterpret_cast<const uint4*>(zb + kSegWords * seg);
#pragma unroll
  for (uint32_t c = 0; c < 8; c++) {
    const uint4 v = sp[c];
    z[4 * c] = v.x; z[4 * c + 1] = v.y; z[4 * c + 2] = v.z; z[4 * c + 3] = v.w;
  }
}

// Bytes of the blocks of a row's n residuals (trial pricing, Sec. III-E):
// header + body bytes summed over the blocks, delta chained from carry.
__device__ __forceinline__ uint32_t price_row(const uint32_t* zb, uint32_t n, uint32_t carry, uint32_t st) {
  const uint32_t lane = lane_id(), j = lane & 3u;
  uint32_t pred_step = carry;
  uint32_t total = 0;
  for (uint32_t s0 = 0; s0 < n; s0 += kStepVal) {
    const uint32_t seg = (s0 >> 5) + lane;
    uint32_t z[32];
    load_seg(zb, seg, z);
    uint32_t pred = __shfl_up_sync(kFull, z[31], 1);
    if (lane == 0) pred = pred_step;
    pred_step = __shfl_sync(kFull, z[31], 31);
    delta_zigzag<true, false>(z, pred, st);
    const uint32_t g = seg >> 2;
    const uint32_t m = n > 128u * g ? min(128u, n - 128u * g) : 0u;
    uint32_t wmax;
    const uint32_t key = block_width(z, j, m, wmax);
    if (m && j == 0) total += 4u + (key >> 14);
  }
  return __reduce_add_sync(kFull, total);
}

// ---------------------------------------------------------------------------
// Low bits of a lane's 32 values (Sec. II, PFOR: value i at bit i b of the
// block's bit stream, LSB first). 32 values of b bits are exactly b words,
// so a lane owns words [j b, j b + b) of its block. Words k >= lim are not
// stored (the lane's share past the block's last value). Values wider than
// b are cut (masked) when the block has exceptions. Each word is assembled
// in a 64-bit accumulator (multiply-adds place the bits) and stored once.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pack_low(const uint32_t (&z)[32], const uint32_t* zseg, uint32_t b, uint32_t lim,
                                         bool masked, uint32_t* wp) {
  unsigned long long acc = 0;
  uint32_t nbit = 0, k = 0;
  if (__all_sync(kFull, b <= 8u)) {
    // quads: 4 values = 4b <= 32 bits, at most one word completes per quad
    const uint32_t bm = (1u << b) - 1u, m1 = 1u << b, u4 = 4u * b;
    const bool anym = __any_sync(kFull, masked);
#pragma unroll
    for (int q = 0; q < 8; q++) {
      uint32_t a0 = z[4 * q], a1 = z[4 * q + 1], a2 = z[4 * q + 2], a3 = z[4 * q + 3];
      if (anym) { a0 &= bm; a1 &= bm; a2 &= bm; a3 &= bm; }
      const uint32_t x = ((a3 * m1 + a2) * m1 + a1) * m1 + a0;
      acc += (unsigned long long)x * (1u << nbit);
      nbit += u4;
      if (nbit >= 32u) {
        if (k < lim) wp[k] = (uint32_t)acc;
        k++;
        acc >>= 32;
        nbit -= 32u;
      }
    }
  } else {  // some block of the step is wider than 8 bits (rare): one value at a time, rolled
    const uint32_t bm = b >= 32u ? 0xffffffffu : ((1u << b) - 1u);
#pragma unroll 1
    for (uint32_t i = 0; i < 32; i++) {
      acc += (unsigned long long)(zseg[i] & bm) * (1u << nbit);
      nbit += b;
      if (nbit >= 32u) {
        if (k < lim) wp[k] = (uint32_t)acc;
        k++;
        acc >>= 32;
        nbit -= 32u;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Exceptions of a block (Sec. II, PFOR: the values wider than b): e position
// bytes in ascending order, zero-padded to 4 bytes, then the high parts
// (value >> b) as a bit stream of hb bits each. Lane j of the block handles
// its own exceptions: ranks r0 .. r0 + c - 1 (prefix of the counts over the
// block's lanes), position bytes stored one by one, high parts appended to
// its run of bits [r0 hb, (r0 + c) hb). Words inside a run are stored by its
// lane; a word where runs meet belongs to the lane whose run holds its first
// bit, which ORs in the later lanes' leading bits (shuffles) and stores it.
// zseg: the lane's 32 ZigZag values in shared memory (dynamic indexing).
// Warp-wide (shuffles).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pack_exceptions(const uint32_t (&z)[32], const uint32_t* zseg, uint32_t j, uint32_t b,
                                                uint32_t e, uint32_t hb, uint8_t* blk, uint32_t low_words) {
  uint32_t xm = 0;
  if (e) {  // e > 0 implies b < 32
#pragma unroll
    for (int i = 0; i < 32; i++) xm |= (z[i] >> b ? 1u : 0u) << i;
  }
  const uint32_t c = __popc(xm);
  uint32_t incl = c;
  {
    const uint32_t t1 = __shfl_up_sync(kFull, incl, 1);
    if (j >= 1) incl += t1;
    const uint32_t t2 = __shfl_up_sync(kFull, incl, 2);
    if (j >= 2) incl += t2;
  }
  const uint32_t r0 = incl - c;
  uint8_t* pb = blk + 4u * low_words;                                              // position bytes
  uint32_t* hw = reinterpret_cast<uint32_t*>(blk + 4u * low_words + ((e + 3u) & ~3u));  // high parts
  const uint32_t S0 = r0 * hb;
  uint32_t q = S0 >> 5, nbit = S0 & 31u;
  const bool unaligned = nbit != 0u;
  bool first = true;
  uint32_t F = 0, Fq = 0xffffffffu;  // a first word that starts in an earlier lane's run
  unsigned long long acc = 0;
  uint32_t rank = r0, xs = xm;
  while (xs) {
    const uint32_t i = __ffs(xs) - 1u;
    xs &= xs - 1u;
    pb[rank++] = (uint8_t)(32u * j + i);
    const uint32_t h = zseg[i] >> b;
    acc += (unsigned long long)h * (1u << nbit);
    nbit += hb;
    if (nbit >= 32u) {
      if (first && unaligned) { F = (uint32_t)acc; Fq = q; }
      else hw[q] = (uint32_t)acc;
      first = false;
      q++;
      acc >>= 32;
      nbit -= 32u;
    }
  }
  uint32_t Bw = 0, Bq = 0xffffffffu;  // the run's last, partial word
  if (c && nbit) {
    if (first && unaligned) { F = (uint32_t)acc; Fq = q; }
    else { Bw = (uint32_t)acc; Bq = q; }
  }
  if (j == 3u && e) {  // zero padding of the position bytes
    for (uint32_t t = e; t < ((e + 3u) & ~3u); t++) pb[t] = 0;
  }
#pragma unroll
  for (uint32_t d = 1; d <= 3; d++) {
    const uint32_t oq = __shfl_down_sync(kFull, Fq, d), ov = __shfl_down_sync(kFull, F, d);
    if (j + d <= 3u && Bq != 0xffffffffu && oq == Bq) Bw |= ov;
  }
  if (Bq != 0xffffffffu) hw[Bq] = Bw;
}

// ---------------------------------------------------------------------------
// One step of a row: compacted values [s0, s0 + 1024) of n (lane l: segment
// s0/32 + l, block g = segment/4 of the row, j = l & 3). Delta from
// pred_step (updated to the step's last residual), ZigZag, widths, block
// headers to hdr[g], bodies from body + boff (bytes). Returns the step's
// body bytes.
// ---------------------------------------------------------------------------
template <bool STAGED>
__device__ __forceinline__ uint32_t code_step(uint32_t* zb, uint32_t s0, uint32_t n, uint32_t& pred_step, bool fast,
                                              uint32_t st, uint32_t* hdr, uint8_t* body, uint32_t boff) {
  const uint32_t lane = lane_id(), j = lane & 3u;
  const uint32_t seg = (s0 >> 5) + lane;
  uint32_t z[32];
  load_seg(zb, seg, z);
  uint32_t pred = __shfl_up_sync(kFull, z[31], 1);
  if (lane == 0) pred = pred_step;
  pred_step = __shfl_sync(kFull, z[31], 31);
  uint4* sp = reinterpret_cast<uint4*>(zb + kSegWords * seg);  // ZigZag values back, for the exceptions
  if (!STAGED && fast) {
    delta_zigzag<false, true>(z, pred, st);
#pragma unroll
    for (uint32_t c = 0; c < 8; c++) sp[c] = make_uint4(z[4 * c], z[4 * c + 1], z[4 * c + 2], z[4 * c + 3]);
  } else {  // deltas of 2^30 or more, or ablated codecs (Sec. IV-H; rare): rolled, through shared memory
    uint32_t* zs = zb + kSegWords * seg;
    uint32_t prev = pred;
#pragma unroll 1
    for (uint32_t i = 0; i < 32; i++) {
      const uint32_t e = zs[i];
      const uint32_t d = (STAGED && (st & kStageNoDelta)) ? e : e - prev;
      zs[i] = (STAGED && (st & kStageNoZigzag)) ? d : zigzag(d);
      prev = e;
    }
    load_seg(zb, seg, z);
  }
  const uint32_t g = seg >> 2;
  const uint32_t m = n > 128u * g ? min(128u, n - 128u * g) : 0u;
  uint32_t wmax;
  const uint32_t key = block_width(z, j, m, wmax);
  const uint32_t b = m ? (key >> 8) & 63u : 0u, e = m ? key & 255u : 0u, f = m ? key >> 14 : 0u;
  const uint32_t hb = e ? wmax - b : 0u;
  // the block's body offset: prefix of the sizes over the step's blocks
  uint32_t tot;
  const uint32_t pre = warp_excl_scan(j == 0u ? f : 0u, tot);
  const uint32_t off = boff + __shfl_sync(kFull, pre, lane & ~3u);
  if (j == 0u && m) hdr[g] = b | (e << 8) | (hb << 16);
  const uint32_t low_words = (m * b + 31u) >> 5;
  const uint32_t lim = min(b, low_words > j * b ? low_words - j * b : 0u);
  uint8_t* blk = body + off;
  pack_low(z, zb + kSegWords * seg, b, lim, e != 0u, reinterpret_cast<uint32_t*>(blk) + j * b);
  if (__any_sync(kFull, e != 0u)) pack_exceptions(z, zb + kSegWords * seg, j, b, e, hb, blk, low_words);
  return tot;
}

}  // namespace

// ----------------------------------------------------------------------------
// k_trial: Sec. III-E. For sections with a predecessor and no forced mode,
// one warp per test row floor((2k+1)H/(2L)) (de-duplicated): the I and P
// residuals of the row, delta-chained from the last residual of the earlier
// test rows (the test rows' residuals form one flat vector starting from 0),
// priced per block. cost[2 sec + mode] += the row's block bytes.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(32) k_trial(EncParams p) {
  extern __shared__ __align__(16) uint32_t smem[];
  // one mode per CTA (I: even blocks, P: odd), so a CTA needs one buffer and
  // twice as many fit an SM
  const bool pmode = (blockIdx.x & 1u) != 0u;
  const uint32_t gsr = blockIdx.x >> 1;
  const uint32_t gs = gsr / p.trial_rows, ti = gsr % p.trial_rows;
  const EncSeg& sg = p.seg[find_seg(p.seg_sec_base, p.n_seg, gs)];
  const uint32_t ta = gs - sg.sec_base;
  const uint32_t t = ta / sg.A, a = ta % sg.A;
  if (sg.frame0 + t == 0 || sg.force_mode >= 0) return;
  // the distinct test rows, ascending: floor((2k+1)H/(2L)) are distinct for
  // L <= H, and for L >= H they are every row (brute force over the data)
  const uint32_t L = sg.test_lines, H = sg.H;
  const uint32_t nr = min(L, H);
  if (ti >= nr) return;
  auto test_row = [&](uint32_t k) -> uint32_t {
    return L >= H ? k : (uint32_t)(((unsigned long long)(2 * k + 1) * H) / (2ull * L));
  };
  const AttrDev at = sg.attrs[a];
  const uint32_t W = sg.W;
  const size_t rowb = (size_t)W * at.s;
  const uint8_t* cur = sg.cur[ta];
  const uint8_t* prv = sg.prev[ta];
  const uint32_t st = sg.stages;
  const bool all = (st & kStageNoMask) != 0u;
  uint32_t* zb = smem;
  if (lane_id() == 0) {  // fetch the test row and the earlier test row's tail into L2 at once
    prefetch_l2(cur + test_row(ti) * rowb, rowb);
    if (pmode) prefetch_l2(prv + test_row(ti) * rowb, rowb);
    if (ti > 0) {
      const size_t tail = min(rowb, (size_t)kStepPx * at.s);
      prefetch_l2(cur + test_row(ti - 1) * rowb + rowb - tail, tail);
      if (pmode) prefetch_l2(prv + test_row(ti - 1) * rowb + rowb - tail, tail);
    }
  }
  // carry: the last residual of the nearest earlier test row that has one
  uint32_t ci = 0, cp = 0;
  for (int k = (int)ti - 1; k >= 0; k--) {
    const uint8_t* c0 = cur + test_row(k) * rowb;
    const uint8_t* p0 = prv + test_row(k) * rowb;
    bool f;
    if (at.qkind == 0) f = row_last<0>(c0, p0, at, W, 0xffffffffu, all, &ci, &cp);
    else if (at.qkind == 1) f = row_last<1>(c0, p0, at, W, 0xffffffffu, all, &ci, &cp);
    else f = row_last<2>(c0, p0, at, W, 0xffffffffu, all, &ci, &cp);
    if (f) break;
  }
  const uint8_t* c1 = cur + test_row(ti) * rowb;
  const uint8_t* p1 = prv + test_row(ti) * rowb;
  uint32_t n;
  const uint32_t kz = all ? 0u : 0xffu;
  if (at.qkind == 0) n = pass_a_trial<0>(c1, p1, at, W, kz, pmode, zb);
  else if (at.qkind == 1) n = pass_a_trial<1>(c1, p1, at, W, kz, pmode, zb);
  else n = pass_a_trial<2>(c1, p1, at, W, kz, pmode, zb);
  __syncwarp();
  const bool nd = (st & kStageNoDelta) != 0u;
  if (n) fill_tail(zb, n, nd ? 0u : zb[zaddr(n - 1)]);
  const uint32_t cost = price_row(zb, n, pmode ? cp : ci, st);
  if (lane_id() == 0) atomicAdd(p.cost + 2 * gs + (pmode ? 1u : 0u), cost);
}

// ----------------------------------------------------------------------------
// k_encode: one warp per row item k = (t, a, r), items taken one at a time
// from an atomic ticket so that every item a warp waits on (look-backs over
// earlier items) was handed out earlier. No CTA-wide barrier.
// ----------------------------------------------------------------------------

// Per-warp shared memory (byte offsets): compacted residuals / ZigZag values
// (padded layout, whole 1024-value steps), coded mask bytes.
struct EncWarpLayout {
  uint32_t zb, mb, bytes;
};

__host__ __device__ inline EncWarpLayout enc_warp_layout(uint32_t W) {
  auto a16 = [](uint32_t x) { return (x + 15u) & ~15u; };
  EncWarpLayout L;
  L.zb = 0;
  L.mb = 4u * zbuf_words(W);
  L.bytes = a16(L.mb + ceil_div_u32(W, 32) * 4u);
  return L;
}

struct EncWarp {
  uint32_t* zb;
  uint8_t* mb;
};

// The last kept sample among the 8 (nv valid) in v / pv, across the warp:
// its residual (P: q - q', I: q). Returns false if there is none.
__device__ __forceinline__ bool tail_residual(uint32_t (&v)[8], uint32_t (&pv)[8], uint32_t nv, bool pm, bool all,
                                              const AttrDev& at, uint32_t& e_last) {
  quant8(v, at);
  if (pm) quant8(pv, at);
  bool has = false;
  uint32_t last = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    if ((uint32_t)i < nv && (v[i] != 0u || all)) {
      has = true;
      last = pm ? v[i] - pv[i] : v[i];
    }
  }
  const uint32_t hm = __ballot_sync(kFull, has);
  if (!hm) return false;
  e_last = __shfl_sync(kFull, last, 31u - __clz(hm));
  return true;
}

// STAGED: the segments may have stage switches, or the test hook may be set
// (else both are read as 0 and the full codec's code is all that is compiled
// in).
template <bool STAGED>
__device__ __forceinline__ void encode_item(const EncParams& p, const uint32_t k, const EncWarp& w) {
  const EncSeg& sg = p.seg[find_seg(p.seg_item_base, p.n_seg, k)];
  const uint32_t lane = lane_id();
  const uint32_t H = sg.H, W = sg.W, A = sg.A, ncls = sg.ncls;
  const uint32_t nw = (!STAGED || ncls) ? sg.nw : 0u;  // coded mask words (none without the mask stage)
  const uint32_t st = STAGED ? sg.stages : 0u, kz = (st & kStageNoMask) ? 0u : 0xffu;
  const uint32_t kl = k - sg.item_base;  // item within the segment, attribute-major (enc_item)
  const uint32_t r = kl % H, at_idx = kl / H, a = at_idx / sg.T, t = at_idx % sg.T;
  const uint32_t ta = t * A + a;     // section (scan t, attribute a)
  const uint32_t sec = sg.sec_base + ta;
  const uint32_t sec_start = k - r;  // global item of row 0 of this attribute-scan
  const AttrDev at = sg.attrs[a];
  const uint32_t mode = section_mode(p, sg, sec, t);
  if (r == 0 && lane == 0) p.modes[sec] = mode;
  const size_t rowb = (size_t)W * at.s;
  const uint8_t* cur = sg.cur[ta] + r * rowb;
  const uint8_t* prv = mode ? sg.prev[ta] + r * rowb : nullptr;
  if (lane == 0) {  // fetch the row(s) into L2 ahead of the 256-pixel steps
    prefetch_l2(cur, rowb);
    if (prv) prefetch_l2(prv, rowb);
  }
  // the previous row's last 256-pixel step, loaded now and read after pass A:
  // its last kept residual is this row's delta carry (Sec. III-C)
  const uint32_t nsteps = ceil_div_u32(W, kStepPx);
  const uint32_t tx0 = kStepPx * (nsteps - 1u) + 8u * lane;
  const uint32_t tnv = tx0 < W ? min(8u, W - tx0) : 0u;
  uint32_t tv[8], tpv[8];
  if (r > 0) {
    load8<false>(cur - rowb, at.s, tx0, tnv, vec_ok(cur - rowb, at.s), tv);
    if (prv) load8<false>(prv - rowb, at.s, tx0, tnv, vec_ok(prv - rowb, at.s), tpv);
  }

  // ---- pass A
  uint32_t qhi;
  const uint32_t n = pass_a(cur, prv, at, W, kz, w.zb, w.mb, qhi);
  if (t + 1 == sg.T) state_row(cur, sg.state_next[a] + r * rowb, at, W);
  __syncwarp();
  if (STAGED && (st & kStageZstdMask)) {  // the row's coded mask bytes, for the section's Zstandard frame
    const uint32_t rb = sg.zm_rb;
    uint8_t* zrow = p.zmask + sg.zm_base + (size_t)ta * sg.zm_stride + (size_t)r * rb;
    if ((rb & 3u) == 0u) {
      for (uint32_t i = lane; i < rb / 4u; i += 32u)
        reinterpret_cast<uint32_t*>(zrow)[i] = reinterpret_cast<const uint32_t*>(w.mb)[i];
    } else {
      for (uint32_t i = lane; i < rb; i += 32u) zrow[i] = w.mb[i];
    }
  }
  const uint32_t last_e = n ? w.zb[zaddr(n - 1)] : 0u;
  // (the failure-detection test hook, read by the STAGED instance only, may
  // withhold this row's status)
  const bool publish = !STAGED || k + 1u != p.withhold;
  if (lane == 0 && publish) {  // this row's last residual, for the rows after it (one word: no fence)
    st_store(p.st_carry + k, kStAgg | ((unsigned long long)(n ? 1 : 0) << 32) | last_e);
  }
  if (n) fill_tail(w.zb, n, (st & kStageNoDelta) ? 0u : last_e);

  // ---- delta carry
  uint32_t carry = 0;
  bool known = r == 0;  // e[-1] = 0 at the start of the attribute-scan
  if (r > 0) {
    known = tail_residual(tv, tpv, tnv, prv != nullptr, kz == 0u, at, carry);
  }
  if (!known) {  // the previous rows' "last residual" words decide
    const bool ok = lookback_last(p.st_carry, k, sec_start, carry);
    if (!ok) {
      if (lane == 0) {
        atomicOr(sg.err, kErrTimeout);
        st_store(p.st_carry + k, kStErr);
      }
      return;
    }
  }

  // ---- mask part: 2-bit class per word (16 per class word), literals
  uint32_t* dst = reinterpret_cast<uint32_t*>(p.slots + sg.slot_base + (size_t)kl * sg.slot_bytes);
  const uint32_t* mbw = reinterpret_cast<const uint32_t*>(w.mb);
  const uint32_t below = (1u << lane) - 1u;
  uint32_t nlit = 0;
  for (uint32_t jb = 0; jb < nw; jb += 32) {
    const uint32_t jw = jb + lane;
    const bool lit = jw < nw && mask_class(mbw[jw], valid_bits(W, nw, jw)) == 2u;
    nlit += __popc(__ballot_sync(kFull, lit));
  }
  uint32_t litbase = 0;
  for (uint32_t jb = 0; jb < nw; jb += 32) {
    const uint32_t jw = jb + lane;
    const uint32_t c = jw < nw ? mbw[jw] : 0u;
    const uint32_t cls = jw < nw ? mask_class(c, valid_bits(W, nw, jw)) : 0u;
    uint32_t cw = cls << (2u * (lane & 15u));
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) cw |= __shfl_xor_sync(kFull, cw, o);
    const uint32_t ci = (jb >> 4) + (lane >> 4);
    if ((lane & 15u) == 0 && ci < ncls) dst[ci] = cw;
    const uint32_t litm = __ballot_sync(kFull, cls == 2u);
    if (cls == 2u) dst[ncls + litbase + __popc(litm & below)] = c;
    litbase += __popc(litm);
  }

  // ---- block headers and bodies, 1024 values per step
  const uint32_t nb = ceil_div_u32(n, kBlockN);
  uint32_t* hdr = dst + ncls + nlit;
  uint8_t* body = reinterpret_cast<uint8_t*>(hdr + nb);
  // every delta below 2^30 in magnitude: 1- and 2-byte samples always (D5),
  // 4-byte ones when the quantized samples and the carry stay below 2^29
  const bool fast = at.s <= 2u || (qhi < (1u << 29) && carry + (1u << 29) < (1u << 30));
  uint32_t body_bytes = 0, pred = carry;
  for (uint32_t s0 = 0; s0 < n; s0 += kStepVal)
    body_bytes += code_step<STAGED>(w.zb, s0, n, pred, fast, st, hdr, body, body_bytes);
  if (lane == 0) {
    p.row_bytes[k] = 4u * (ncls + nlit + nb) + body_bytes;
    p.row_nnz[k] = n;
    p.row_carry[k] = carry;
  }
  __syncwarp();
}

template <int WPC, bool STAGED>
__global__ void __launch_bounds__(WPC * 32, 24 / WPC) k_encode(EncParams p) {
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t lane = lane_id();
  const EncWarpLayout lay = enc_warp_layout(p.max_W);
  uint8_t* wb = reinterpret_cast<uint8_t*>(smem) + warp_id() * lay.bytes;
  EncWarp w;
  w.zb = reinterpret_cast<uint32_t*>(wb + lay.zb);
  w.mb = wb + lay.mb;
  // the next ticket is requested before the current item is coded, so its
  // round trip overlaps the work (an item still waits only on items handed
  // out before it: a warp holding an unstarted ticket is coding a smaller one)
  uint32_t k = 0;
  if (lane == 0) k = p.item_lo + atomicAdd(p.ticket, 1u);
  k = __shfl_sync(kFull, k, 0);
  while (k < p.n_items) {
    uint32_t next = 0;
    if (lane == 0) next = p.item_lo + atomicAdd(p.ticket, 1u);
    encode_item<STAGED>(p, k, w);
    k = __shfl_sync(kFull, next, 0);
  }
}

// ----------------------------------------------------------------------------
// k_sec_sizes: one CTA per section (scan t, attribute a): its bytes (row
// table + row chunks) and nonzero count.
// k_place: one CTA per section: the section's offset in the stream (sum over
// the segment's earlier sections), its row table (end offsets + carries),
// the copy of each row chunk from its slot and, for attribute 0, the frame
// header and frame offset; section 0 also writes the stream header. Every
// write is checked against the output capacity.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void put_u32_guarded(uint8_t* out, unsigned long long cap, unsigned long long at,
                                                uint32_t v, uint32_t* err) {
  if (at + 4 <= cap) *reinterpret_cast<uint32_t*>(out + at) = v;
  else atomicOr(err, kErrCapacity);
}

__device__ __forceinline__ void put_u8_guarded(uint8_t* out, unsigned long long cap, unsigned long long at, uint32_t v,
                                               uint32_t* err) {
  if (at < cap) out[at] = (uint8_t)v;
  else atomicOr(err, kErrCapacity);
}

__device__ __forceinline__ unsigned long long cta_sum_u64(unsigned long long v, unsigned long long* s_red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane_id() == 0) s_red[warp_id()] = v;
  __syncthreads();
  unsigned long long tot = 0;
  for (uint32_t w2 = 0; w2 < blockDim.x / 32u; w2++) tot += s_red[w2];
  __syncthreads();
  return tot;
}

__global__ void __launch_bounds__(kThreads) k_sec_sizes(EncParams p) {
  __shared__ unsigned long long s_red[kWarps];
  const uint32_t gs = blockIdx.x;
  const EncSeg& sg = p.seg[find_seg(p.seg_sec_base, p.n_seg, gs)];
  const uint32_t H = sg.H, ta = gs - sg.sec_base;
  const uint32_t item0 = sg.item_base + enc_item(sg, ta / sg.A, ta % sg.A, 0);
  unsigned long long bytes = 0, nnz = 0;
  for (uint32_t r = threadIdx.x; r < H; r += kThreads) {
    bytes += p.row_bytes[item0 + r];
    nnz += p.row_nnz[item0 + r];
  }
  bytes = cta_sum_u64(bytes, s_red);
  nnz = cta_sum_u64(nnz, s_red);
  unsigned long long zpart = 0;
  if (sg.stages & kStageZstdMask) {  // the Zstandard mask part: index, frame, padding
    const uint32_t nblk = sg.zm_nblk;
    unsigned long long fb = 0;
    for (uint32_t j = threadIdx.x; j < nblk; j += kThreads) fb += p.zblk_bytes[sg.zb_base + (size_t)ta * nblk + j];
    fb = cta_sum_u64(fb, s_red) + kZFrameHdr;
    zpart = zmask_part_bytes(nblk, (uint32_t)fb);
    if (threadIdx.x == 0) p.zfr_bytes[gs] = (uint32_t)fb;
  }
  if (threadIdx.x == 0) {
    p.sec_bytes[gs] = 8ull * H + zpart + bytes;
    p.sec_nnz[gs] = (uint32_t)nnz;
  }
}

constexpr uint32_t kPlaceSplit = 4;  // CTAs per section in k_place (rows dealt round robin)

__global__ void __launch_bounds__(kThreads) k_place(EncParams p) {
  extern __shared__ __align__(16) uint32_t smem[];  // [H] row chunk starts
  __shared__ unsigned long long s_red[kWarps];
  __shared__ uint32_t s_tmp[kWarps + 1];
  const uint32_t gs = blockIdx.x / kPlaceSplit, part = blockIdx.x % kPlaceSplit;
  const EncSeg& sg = p.seg[find_seg(p.seg_sec_base, p.n_seg, gs)];
  const uint32_t H = sg.H, A = sg.A;
  const uint32_t ta = gs - sg.sec_base, t = ta / A, a = ta % A;
  const uint32_t local0 = enc_item(sg, t, a, 0);
  const uint32_t item0 = sg.item_base + local0;
  uint8_t* out = sg.out;
  const unsigned long long cap = sg.cap;
  // bytes of the segment's earlier sections: of earlier frames (frame_before)
  // and of this frame's earlier attributes
  unsigned long long frame_before = 0, attr_before = 0;
  for (uint32_t i = threadIdx.x; i < ta; i += kThreads) {
    if (i < t * A) frame_before += p.sec_bytes[sg.sec_base + i];
    else attr_before += p.sec_bytes[sg.sec_base + i];
  }
  frame_before = cta_sum_u64(frame_before, s_red);
  attr_before = cta_sum_u64(attr_before, s_red);
  const unsigned long long frame_at = sg.shdr + (unsigned long long)t * sg.fhdr + frame_before;
  const unsigned long long sec_at = frame_at + sg.fhdr + attr_before;
  // the Zstandard mask part after the row table: u32 frame bytes, u32 end of
  // each block, the frame (header, then the blocks from their slots), zero
  // bytes up to a multiple of 4
  uint32_t zpart = 0;
  if (sg.stages & kStageZstdMask) {
    const uint32_t nblk = sg.zm_nblk, fb = p.zfr_bytes[gs];
    const size_t b0 = sg.zb_base + (size_t)ta * nblk;
    uint32_t* bstart = smem + kMaxH;
    zpart = zmask_part_bytes(nblk, fb);
    for (uint32_t j = threadIdx.x; j < nblk; j += kThreads) bstart[j] = p.zblk_bytes[b0 + j];
    __syncthreads();
    block_excl_scan(bstart, nblk, s_tmp);
    const unsigned long long zp = sec_at + 8ull * H, fz = zp + 4ull + 4ull * nblk;
    if (part == 0) {
      for (uint32_t j = threadIdx.x; j < nblk; j += kThreads)
        put_u32_guarded(out, cap, zp + 4ull + 4ull * j, kZFrameHdr + bstart[j] + p.zblk_bytes[b0 + j], sg.err);
      if (threadIdx.x == 0) {
        put_u32_guarded(out, cap, zp, fb, sg.err);
        const uint32_t hdr[9] = {0x28, 0xB5, 0x2F, 0xFD, 0xA0, 0, 0, 0, 0};
        const uint32_t n = sg.H * sg.zm_rb;
        for (uint32_t i = 0; i < 9; i++) put_u8_guarded(out, cap, fz + i, i < 5 ? hdr[i] : (n >> (8 * (i - 5))) & 0xffu, sg.err);
        for (unsigned long long i = fz + fb; i < zp + zpart; i++) put_u8_guarded(out, cap, i, 0u, sg.err);
      }
    }
    for (uint32_t j = part; j < nblk; j += kPlaceSplit) {
      const uint32_t nb = p.zblk_bytes[b0 + j];
      const unsigned long long at = fz + kZFrameHdr + bstart[j];
      const uint8_t* src = p.zblk + (b0 + j) * (size_t)kZSlot;
      if (at + nb > cap) {
        if (threadIdx.x == 0) atomicOr(sg.err, kErrCapacity);
        continue;
      }
      for (uint32_t i = threadIdx.x; i < nb; i += kThreads) out[at + i] = src[i];
    }
  }
  // row table: end offsets (prefix of chunk sizes) and carries
  for (uint32_t r = threadIdx.x; r < H; r += kThreads) smem[r] = p.row_bytes[item0 + r];
  __syncthreads();
  const uint32_t data = block_excl_scan(smem, H, s_tmp);  // smem = row starts
  if (part == 0) {
    for (uint32_t r = threadIdx.x; r < H; r += kThreads) {
      const uint32_t end = (r + 1 < H) ? smem[r + 1] : data;
      put_u32_guarded(out, cap, sec_at + 8ull * r, end, sg.err);
      put_u32_guarded(out, cap, sec_at + 8ull * r + 4, p.row_carry[item0 + r], sg.err);
    }
  }
  // row chunks: slot -> stream, a warp per two rows at a time, 4 words of
  // each in flight per lane
  const unsigned long long data_at = sec_at + 8ull * H + zpart;
  const uint32_t lane = lane_id();
  auto row_span = [&](uint32_t r, const uint32_t*& src, uint32_t*& dst) -> uint32_t {
    const uint32_t words = p.row_bytes[item0 + r] / 4u;
    const unsigned long long at = data_at + smem[r];
    if (at + 4ull * words > cap) {
      if (lane == 0) atomicOr(sg.err, kErrCapacity);
      return 0u;
    }
    src = reinterpret_cast<const uint32_t*>(p.slots + sg.slot_base + (size_t)(local0 + r) * sg.slot_bytes);
    dst = reinterpret_cast<uint32_t*>(out + at);
    return words;
  };
  constexpr uint32_t kRowStride = kWarps * kPlaceSplit;
  for (uint32_t r = part * kWarps + warp_id(); r < H; r += 2u * kRowStride) {
    const uint32_t* sa = nullptr;
    const uint32_t* sb = nullptr;
    uint32_t* da = nullptr;
    uint32_t* db = nullptr;
    const uint32_t wa = row_span(r, sa, da);
    const uint32_t wb = r + kRowStride < H ? row_span(r + kRowStride, sb, db) : 0u;
    const uint32_t wmax = max(wa, wb);
    for (uint32_t i = lane; i < wmax; i += 128u) {
      uint32_t va[4], vb[4];
#pragma unroll
      for (uint32_t q = 0; q < 4; q++) {
        va[q] = i + 32u * q < wa ? __ldcs(sa + i + 32u * q) : 0u;
        vb[q] = i + 32u * q < wb ? __ldcs(sb + i + 32u * q) : 0u;
      }
#pragma unroll
      for (uint32_t q = 0; q < 4; q++) {
        if (i + 32u * q < wa) da[i + 32u * q] = va[q];
        if (i + 32u * q < wb) db[i + 32u * q] = vb[q];
      }
    }
  }
  if (part == 0 && a == 0 && threadIdx.x == 0) {
    const uint32_t f0 = sg.sec_base + t * A;
    unsigned long long fbytes = sg.fhdr;
    for (uint32_t aa = 0; aa < A; aa++) fbytes += p.sec_bytes[f0 + aa];
    put_u32_guarded(out, cap, frame_at, (uint32_t)fbytes, sg.err);
    put_u32_guarded(out, cap, frame_at + 4, sg.frame0 + t, sg.err);
    for (uint32_t aa = 0; aa < A; aa++) {
      const unsigned long long h = frame_at + 8ull + 12ull * aa;
      put_u32_guarded(out, cap, h, p.modes[f0 + aa], sg.err);
      put_u32_guarded(out, cap, h + 4, (uint32_t)p.sec_bytes[f0 + aa], sg.err);
      put_u32_guarded(out, cap, h + 8, p.sec_nnz[f0 + aa], sg.err);
    }
    sg.frame_off[t] = frame_at;
    if (t + 1 == sg.T) sg.frame_off[sg.T] = frame_at + fbytes;
    if (t == 0 && sg.shdr) {
      put_u32_guarded(out, cap, 0, 0x3159464Au, sg.err);  // "JFY1"
      put_u32_guarded(out, cap, 4, 1u | (A << 16), sg.err);
      put_u32_guarded(out, cap, 8, H, sg.err);
      put_u32_guarded(out, cap, 12, sg.W, sg.err);
      for (uint32_t aa = 0; aa < A; aa++) {
        put_u32_guarded(out, cap, 16 + 8ull * aa, attr_header_word(sg.attrs[aa].s, sg.stages), sg.err);
        put_u32_guarded(out, cap, 20 + 8ull * aa, sg.attrs[aa].P, sg.err);
      }
    }
  }
}

size_t enc_smem_bytes_host(uint32_t W) { return enc_warp_layout(W).bytes; }

constexpr size_t kRowsSmemAuto = 100 * 1024;  // per CTA when picking warps per CTA by itself
constexpr size_t kRowsSmemMax = 227 * 1024;

template <int WPC>
static cudaError_t rows_occupancy(size_t smem, bool staged, int* per_sm) {
  auto f = staged ? k_encode<WPC, true> : k_encode<WPC, false>;
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, f, WPC * 32, smem);
}

int encode_rows_launch(const EncParams& p, RowsLaunch* out) {
  const EncWarpLayout L = enc_warp_layout(p.max_W);
  if ((L.mb | L.bytes) & 15u) return (int)cudaErrorInvalidValue;  // 16-byte aligned regions
  uint32_t wpc = p.wpc;
  if ((wpc != 1 && wpc != 2 && wpc != 4) || wpc * L.bytes > kRowsSmemMax) wpc = 0;
  if (!wpc) wpc = 4 * L.bytes <= kRowsSmemAuto ? 4u : (2 * L.bytes <= kRowsSmemAuto ? 2u : 1u);
  const size_t smem = (size_t)wpc * L.bytes;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    if (wpc == 4) e = rows_occupancy<4>(smem, p.staged != 0, &per_sm);
    else if (wpc == 2) e = rows_occupancy<2>(smem, p.staged != 0, &per_sm);
    else e = rows_occupancy<1>(smem, p.staged != 0, &per_sm);
  }
  if (e != cudaSuccess) return (int)e;
  uint32_t ctas = (uint32_t)max(per_sm, 1);
  if (p.ctas_per_sm) ctas = min(ctas, p.ctas_per_sm);
  // enough warps to fill the GPU; warps beyond the work find the ticket spent
  const uint32_t want = ceil_div_u32(p.n_items - p.item_lo, wpc);
  out->wpc = wpc;
  out->ctas_per_sm = ctas;
  out->items_per_ticket = 1;
  out->grid = max(1u, min(want, ctas * (uint32_t)sms));
  return 0;
}

size_t trial_smem_bytes_host(uint32_t W) { return 4ull * zbuf_words(W); }

int launch_encode(const EncParams& p, void* stream, void* const* ev) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t s_trial = trial_smem_bytes_host(p.max_W);
  RowsLaunch rl{};
  int rc = encode_rows_launch(p, &rl);
  if (rc != 0) return rc;
  const size_t s_place = 4ull * kMaxH + 4ull * zmask_blocks(kMaxH, kMaxW);  // row starts, block starts
  cudaError_t e = cudaFuncSetAttribute(k_trial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_trial);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_place, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_place);
  if (e != cudaSuccess) return (int)e;
  auto mark = [&](int i) {
    if (ev) record_event(ev[i], st);
  };
  mark(0);
  if (p.trial_rows) k_trial<<<2u * p.n_sec * p.trial_rows, 32, s_trial, st>>>(p);
  mark(1);
  // rows of narrow segments first, with shared memory (and so occupancy) for
  // their own width, then the wider ones: one rows launch per width class
  // (each launch sets its own shared-memory limit first: resolving another
  // launch's configuration changes it)
  auto rows = [&](const EncParams& q, const RowsLaunch& r) -> cudaError_t {
    const size_t smem = (size_t)r.wpc * enc_warp_layout(q.max_W).bytes;
    void (*f)(EncParams) = q.staged ? (r.wpc == 4 ? k_encode<4, true> : r.wpc == 2 ? k_encode<2, true> : k_encode<1, true>)
                                    : (r.wpc == 4 ? k_encode<4, false> : r.wpc == 2 ? k_encode<2, false> : k_encode<1, false>);
    cudaError_t ce = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ce != cudaSuccess) return ce;
    f<<<r.grid, r.wpc * 32, smem, st>>>(q);
    return cudaGetLastError();
  };
  if (p.split > 0 && p.split < p.n_items) {
    EncParams lo = p, hi = p;
    lo.n_items = p.split;
    lo.max_W = p.split_W;
    hi.item_lo = p.split;
    hi.ticket = p.ticket + 1;
    RowsLaunch rlo{};
    rc = encode_rows_launch(lo, &rlo);
    if (rc != 0) return rc;
    e = rows(lo, rlo);
    if (e == cudaSuccess) e = rows(hi, rl);
  } else {
    e = rows(p, rl);
  }
  if (e != cudaSuccess) return (int)e;  // the placement kernels would read row sizes never written
  mark(2);
  rc = launch_zstd_encode(p, st);
  if (rc != 0) return rc;
  k_sec_sizes<<<p.n_sec, kThreads, 0, st>>>(p);
  k_place<<<p.n_sec * kPlaceSplit, kThreads, s_place, st>>>(p);
  mark(3);
  return (int)cudaGetLastError();
}

}  // namespace jiffy
