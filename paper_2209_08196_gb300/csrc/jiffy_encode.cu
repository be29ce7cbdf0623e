// Jiffy encoder kernels (sm_103a).
//
// One call codes T consecutive scans of each of one or more streams (the
// segments of the call), all in parallel: the P prediction of scan t uses the
// *input* of scan t-1 (Sec. III-D), so no scan waits for another's output.
// Three launches:
//   k_trial     one warp per (section, test row): I and P residuals of the
//               scanline, delta chained across the test rows, priced with
//               the block-width pass below; the bytes add up per section and
//               mode (trial compression, mask excluded, Sec. III-E, IV-E).
//   k_encode    one warp per row item (scan, attribute, row), items taken in
//               ticket order. Per row:
//     pass A    8 consecutive pixels per lane per 256-pixel step: quantize
//               (Sec. III-B), zero bitmask (Sec. III-C), mask XOR with the
//               previous scan for P (Sec. III-D), residual (I: q, P: q - q'),
//               compaction of the nonzero samples (warp scan of counts) into
//               a swizzled shared buffer.
//     pass B1   32 consecutive values per lane (8 blocks of 128 per warp
//               step): delta (Sec. III-C) from the previous row's last
//               residual, ZigZag (Eq. 1), then per block the count of values
//               wider than b for every b at once -- carry-save adders over
//               the values' unary width codes, bit-sliced across the 4 lanes
//               of a block -- and the byte-minimal width (Sec. II, PFOR).
//     pass B2   one block at a time, 4 consecutive values per lane: low bits
//               joined with funnel shifts, each body word written once by
//               the lane holding its first bit, exceptions listed and packed
//               the same way; then the mask code, block headers and bodies
//               go to the row's slot. Rows never wait for one another's
//               sizes (sections differ a lot in cost, and an in-order prefix
//               over rows would queue fast rows behind slow ones).
//   k_sec_sizes one CTA per section: its bytes and nonzero count.
//   k_place     one CTA per section: offset (sum over the earlier sections),
//               row table, frame and stream headers, and the copy of every
//               row chunk from its slot to its place in the stream.
#include "jiffy_device.cuh"
#include "jiffy_kernels.h"

namespace jiffy {

namespace {

constexpr uint32_t kStepPx = 256;    // pixels per warp step of pass A (8 per lane)
constexpr uint32_t kStepVal = 1024;  // values per warp step of pass B1 (32 per lane)

// Residual buffer layout: value k lives in 32-value segment k >> 5; the
// segment's 16-byte chunks are XOR-swizzled by the segment index so that a
// lane reading a whole segment and a lane reading 4 consecutive values both
// hit distinct banks.
__device__ __forceinline__ uint32_t swz(uint32_t k) { return k ^ (((k >> 5) & 7u) << 2); }

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

// ---------------------------------------------------------------------------
// Pass A (one row): returns the number n of nonzero samples; their residuals
// go to zb in row-major order (swizzled), the coded mask bytes (M, or M xor
// M_prev for P) to mb, and, for the call's last scan, q * P to st_row. kz =
// 0xff, or 0 without the mask stage (every sample kept, mask bytes 0).
// ---------------------------------------------------------------------------
template <bool PM, int QU, uint32_t S>
__device__ __forceinline__ uint32_t pass_a(const uint8_t* cur, const uint8_t* prv, uint8_t* st_row, const AttrDev& at,
                                           uint32_t W, uint32_t kz, uint32_t* zb, uint8_t* mb) {
  const uint32_t lane = lane_id(), s = at.s;
  const bool vc = vec_ok(cur, s), vp = PM && vec_ok(prv, s), vs = st_row && vec_ok(st_row, s);
  const uint32_t Wm = (W + 31u) & ~31u;
  uint32_t n = 0;
  for (uint32_t base = 0; base < W; base += kStepPx) {
    const uint32_t x0 = base + 8u * lane;
    const uint32_t nv = x0 < W ? min(8u, W - x0) : 0u;
    uint32_t v[8], pv[8];
    ld8<S>(cur, s, x0, nv, vc, v);
    if (PM) ld8<S>(prv, s, x0, nv, vp, pv);
    uint32_t e[8], zm = 0, pm = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      const uint32_t q = quant<QU>(v[i], at);
      v[i] = q;
      zm |= (q == 0u ? 1u : 0u) << i;  // Sec. III-C: 1 = zero sample
      if (PM) {
        const uint32_t pq = quant<QU>(pv[i], at);
        pm |= (pq == 0u ? 1u : 0u) << i;
        e[i] = q - pq;  // Sec. III-D, modulo 2^32
      } else {
        e[i] = q;
      }
    }
    zm &= kz;
    const uint32_t vm = (1u << nv) - 1u;
    const uint32_t nz = ~zm & vm;
    if (x0 < Wm) mb[x0 >> 3] = (uint8_t)((PM ? (zm ^ (pm & kz)) : zm) & vm);
    if (st_row && nv) {  // the next call's previous scan, dequantized as the decoder holds it
      uint32_t sv[8];
#pragma unroll
      for (int i = 0; i < 8; i++) sv[i] = v[i] * at.P;
      st8<S>(st_row, s, x0, nv, vs, sv);
    }
    uint32_t tot;
    uint32_t kk = n + warp_excl_scan(__popc(nz), tot);
#pragma unroll
    for (int i = 0; i < 8; i++) {
      if ((nz >> i) & 1u) {
        zb[swz(kk)] = e[i];
        kk++;
      }
    }
    n += tot;
  }
  return n;
}

// Pass A of the trial: the residuals of the row's nonzero samples (all
// samples with kz = 0) both ways (I to zi, P to zp).
template <int QU>
__device__ __forceinline__ uint32_t pass_a_trial(const uint8_t* cur, const uint8_t* prv, const AttrDev at, uint32_t W,
                                              uint32_t kz, uint32_t* zi, uint32_t* zp) {
  const uint32_t lane = lane_id(), S = at.s;
  const bool vc = vec_ok(cur, S), vp = vec_ok(prv, S);
  uint32_t n = 0;
  for (uint32_t base = 0; base < W; base += kStepPx) {
    const uint32_t x0 = base + 8u * lane;
    const uint32_t nv = x0 < W ? min(8u, W - x0) : 0u;
    uint32_t v[8], pv[8];
    load8<false>(cur, S, x0, nv, vc, v);
    load8<false>(prv, S, x0, nv, vp, pv);
    uint32_t zm = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      v[i] = quant<QU>(v[i], at);
      pv[i] = v[i] - quant<QU>(pv[i], at);
      zm |= (v[i] == 0u ? 1u : 0u) << i;
    }
    const uint32_t nz = ~(zm & kz) & ((1u << nv) - 1u);
    uint32_t tot;
    uint32_t kk = n + warp_excl_scan(__popc(nz), tot);
#pragma unroll
    for (int i = 0; i < 8; i++) {
      if ((nz >> i) & 1u) {
        zi[swz(kk)] = v[i];
        zp[swz(kk)] = pv[i];
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
    const uint32_t hm = __ballot_sync(0xffffffffu, has);
    if (hm) {
      const uint32_t src = 31u - __clz(hm);
      *e_i = __shfl_sync(0xffffffffu, li, src);
      *e_p = __shfl_sync(0xffffffffu, lp, src);
      return true;
    }
  }
  return false;
}

// Repeats the last residual (0 without the delta stage) from n up to the end
// of pass B1's last step, so that those slots code to 0 (and count as
// zero-width values).
__device__ __forceinline__ void fill_tail(uint32_t* zb, uint32_t n, bool no_delta) {
  if (n == 0) return;
  const uint32_t last = no_delta ? 0u : zb[swz(n - 1)];
  const uint32_t end = (n + kStepVal - 1) / kStepVal * kStepVal;
  for (uint32_t k = n + lane_id(); k < end; k += 32u) zb[swz(k)] = last;
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Pass B1: delta + ZigZag in place and the width of every block (Sec. II:
// b in [0, wmax] minimising the block's body bytes, ties to the smallest b).
// Lane l of a warp step holds values 32l .. 32l+31 of the step: the 4 lanes
// 4g'..4g'+3 hold block g' of the step. For each value, its unary width code
// has bit b set iff the value needs more than b bits, so the column sums of
// a block's unary codes are e_b = #values wider than b, for all b at once:
// carry-save adders give each lane its 6 bit planes (counts <= 32), two
// bit-sliced additions across the block's 4 lanes give 8 planes (counts <=
// 128). Each lane then prices the candidates b = j, j+4, ... (j = lane & 3).
// meta[g] = {b | e << 8 | hb << 16, body bytes}. Returns the sum over blocks
// of header + body bytes. st: the stream's stage switches (delta and ZigZag
// may be off).
// ---------------------------------------------------------------------------
template <bool WRITE>
__device__ __forceinline__ uint32_t pass_b1(uint32_t* zb, uint32_t n, uint32_t carry, uint2* meta, uint32_t st) {
  const uint32_t lane = lane_id(), j = lane & 3u;
  uint32_t pred_step = carry;  // the residual before the step's first value
  uint32_t total = 0;
  for (uint32_t s0 = 0; s0 < n; s0 += kStepVal) {
    const uint32_t seg = (s0 >> 5) + lane;
    uint4* sp = reinterpret_cast<uint4*>(zb + 32u * seg);
    uint32_t z[32];
#pragma unroll
    for (uint32_t c = 0; c < 8; c++) {
      const uint4 v = sp[c ^ (seg & 7u)];
      z[4 * c] = v.x; z[4 * c + 1] = v.y; z[4 * c + 2] = v.z; z[4 * c + 3] = v.w;
    }
    uint32_t pred = __shfl_up_sync(0xffffffffu, z[31], 1);
    if (lane == 0) pred = pred_step;
    pred_step = __shfl_sync(0xffffffffu, z[31], 31);
    // delta (Sec. III-C) and ZigZag (Eq. 1); values past n repeat the last
    // residual (fill_tail), so their ZigZag values are 0
    if (!(st & (kStageNoDelta | kStageNoZigzag))) {
#pragma unroll
      for (int i = 31; i >= 0; i--) z[i] = zigzag(z[i] - (i ? z[i - 1] : pred));
    } else {  // ablated codecs (Sec. IV-H); values past n are 0 without the delta
#pragma unroll
      for (int i = 31; i >= 0; i--) {
        const uint32_t d = (st & kStageNoDelta) ? z[i] : z[i] - (i ? z[i - 1] : pred);
        z[i] = (st & kStageNoZigzag) ? d : zigzag(d);
      }
    }
    if (WRITE) {
#pragma unroll
      for (uint32_t c = 0; c < 8; c++) sp[c ^ (seg & 7u)] = make_uint4(z[4 * c], z[4 * c + 1], z[4 * c + 2], z[4 * c + 3]);
    }
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
      for (int k = 0; k < 6; k++) B[k] = __shfl_xor_sync(0xffffffffu, A[k], 1);
      uint32_t C[7], c = 0;
#pragma unroll
      for (int k = 0; k < 6; k++) {
        const uint32_t u = A[k] ^ B[k];
        C[k] = u ^ c;
        c = (A[k] & B[k]) | (u & c);
      }
      C[6] = c;
#pragma unroll
      for (int k = 0; k < 7; k++) B[k] = __shfl_xor_sync(0xffffffffu, C[k], 2);
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
    const uint32_t wmax = 32u - __clz(anyb);  // e_b > 0 exactly for b < wmax
    const uint32_t g = (s0 >> 7) + (lane >> 2);
    const uint32_t m = n > 128u * g ? min(128u, n - 128u * g) : 0u;
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
      if (!__any_sync(0xffffffffu, live)) break;
      if (live) {
        const uint32_t e = i < 8 ? ((lo4 >> (4 * i)) & 15u) | (((hi4 >> (4 * i)) & 15u) << 4) : 0u;
        const uint32_t f = low + ((e + 3u) & ~3u) + 4u * ((e * (wmax - b) + 31u) >> 5);
        key = min(key, (f << 14) | (b << 8) | e);
      }
    }
    key = min(key, __shfl_xor_sync(0xffffffffu, key, 1));
    key = min(key, __shfl_xor_sync(0xffffffffu, key, 2));
    if (m && j == 0) {
      const uint32_t b = (key >> 8) & 63u, e = key & 255u, f = key >> 14;
      if (WRITE) meta[g] = make_uint2(b | (e << 8) | ((e ? wmax - b : 0u) << 16), f);
      total += 4u + f;
    }
  }
  return __reduce_add_sync(0xffffffffu, total);
}

// ---------------------------------------------------------------------------
// Packs 128 values of b bits, value i at bit i b (Sec. II, a block's low-bit
// stream), into words [0, nwords) of dst, which must be zero. Lane l holds
// values 4l .. 4l+3, bits [4lb, 4lb + 4b) of the stream, joined in registers
// with funnel shifts. For b <= 8 (a word spans up to 8 lanes) the lanes OR
// their 4b bits into the (at most 2) words they touch; for b > 8 each word is
// written once, by the lane holding its first bit, completed with the next
// lane's bits (one shuffle). Bits of the values above b are dropped.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pack4(uint32_t* dst, uint32_t b, uint32_t nwords, uint32_t z0, uint32_t z1,
                                      uint32_t z2, uint32_t z3) {
  const uint32_t lane = lane_id();
  const uint32_t S = 4u * lane * b;           // the lane's first bit
  if (b == 0) return;
  if (b <= 8u) {
    const uint32_t bm = (1u << b) - 1u;
    const uint32_t x = (z0 & bm) | ((z1 & bm) << b) | ((z2 & bm) << (2u * b)) | ((z3 & bm) << (3u * b));
    const uint32_t sh = S & 31u, w = S >> 5;
    const uint32_t y0 = x << sh, y1 = __funnelshift_l(x, 0u, sh);
    if (y0) atomicOr(dst + w, y0);
    if (y1) atomicOr(dst + w + 1u, y1);
    return;
  }
  const uint32_t o = (32u - (S & 31u)) & 31u;  // the lane's first word start, relative to S
  const uint32_t w = (S + o) >> 5;            // that word
  if (b <= 16u) {
    const uint32_t bm = (1u << b) - 1u;
    const unsigned long long x = (unsigned long long)(z0 & bm) | ((unsigned long long)(z1 & bm) << b) |
                                 ((unsigned long long)(z2 & bm) << (2u * b)) |
                                 ((unsigned long long)(z3 & bm) << (3u * b));
    uint32_t N = __shfl_down_sync(0xffffffffu, (uint32_t)x, 1);
    if (lane == 31u) N = 0u;
    const uint32_t sN = 4u * b - 32u;  // the next lane's bits start at word 1, bit sN (4..32)
    const uint32_t Z0 = (uint32_t)x, Z1 = (uint32_t)(x >> 32) | __funnelshift_lc(0u, N, sN),
                   Z2 = __funnelshift_lc(N, 0u, sN);
    if (w < nwords) dst[w] = __funnelshift_r(Z0, Z1, o);
    if (o + 32u < 4u * b && w + 1u < nwords) dst[w + 1] = __funnelshift_r(Z1, Z2, o);
  } else {
    const uint32_t bm = b >= 32u ? 0xffffffffu : ((1u << b) - 1u);
    const unsigned long long lo = (unsigned long long)(z0 & bm) | ((unsigned long long)(z1 & bm) << b);
    const unsigned long long hi = (unsigned long long)(z2 & bm) | ((unsigned long long)(z3 & bm) << b);
    const uint32_t s2 = 2u * b - 32u;  // hi starts at word 1, bit s2 (2..32)
    const uint32_t h0 = (uint32_t)hi, h1 = (uint32_t)(hi >> 32);
    uint32_t X0 = (uint32_t)lo, X1 = (uint32_t)(lo >> 32) | __funnelshift_lc(0u, h0, s2),
             X2 = __funnelshift_lc(h0, h1, s2), X3 = __funnelshift_lc(h1, 0u, s2), X4 = 0u;
    uint32_t N = __shfl_down_sync(0xffffffffu, X0, 1);
    if (lane == 31u) N = 0u;
    if (4u * b <= 96u) {  // the next lane's bits start at word 2, bit 4b - 64 (4..32)
      const uint32_t sN = 4u * b - 64u;
      X2 |= __funnelshift_lc(0u, N, sN);
      X3 |= __funnelshift_lc(N, 0u, sN);
    } else {  // word 3, bit 4b - 96 (4..32)
      const uint32_t sN = 4u * b - 96u;
      X3 |= __funnelshift_lc(0u, N, sN);
      X4 = __funnelshift_lc(N, 0u, sN);
    }
    if (w < nwords) dst[w] = __funnelshift_r(X0, X1, o);
    if (o + 32u < 4u * b && w + 1u < nwords) dst[w + 1] = __funnelshift_r(X1, X2, o);
    if (o + 64u < 4u * b && w + 2u < nwords) dst[w + 2] = __funnelshift_r(X2, X3, o);
    if (o + 96u < 4u * b && w + 3u < nwords) dst[w + 3] = __funnelshift_r(X3, X4, o);
  }
}

// ---------------------------------------------------------------------------
// Pass B2: packs every block's body into zb, in place and unswizzled (block
// g's body lands in words [off_g, off_g + size_g) with off_g + size_g <=
// 128 (g + 1), so it never reaches a value still to be read): the low b
// bits of all values, then the exceptions (values wider than b) as e
// position bytes in ascending order and their high parts of hb bits (Sec. II,
// PFOR). The body is zeroed first. The exceptions are listed in order in
// xpos / xhv (a warp scan of the lanes' counts gives the ranks); lane x then
// ORs the high part of exception x into place and lane l writes position
// bytes 4l .. 4l+3 as one word.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pass_b2(uint32_t* zb, uint32_t n, uint32_t nb, const uint2* meta, uint8_t* xpos,
                                        uint32_t* xhv) {
  const uint32_t lane = lane_id();
  for (uint32_t g = 0; g < nb; g++) {
    const uint2 md = meta[g];  // .x header, .y body byte offset
    const uint32_t b = md.x & 0xffu, e = (md.x >> 8) & 0xffu, hb = (md.x >> 16) & 0xffu;
    const uint32_t m = min(128u, n - 128u * g);
    uint32_t* body = zb + (md.y >> 2);
    const uint32_t low_words = (m * b + 31u) >> 5;
    const uint32_t pw = (e + 3u) >> 2, size_words = low_words + (e ? pw + ((e * hb + 31u) >> 5) : 0u);
    const uint32_t sgi = 4u * g + (lane >> 3);
    const uint4 zz = reinterpret_cast<const uint4*>(zb + 32u * sgi)[(lane & 7u) ^ (sgi & 7u)];
    const uint32_t z0 = zz.x, z1 = zz.y, z2 = zz.z, z3 = zz.w;  // 0 past m
    __syncwarp();
    for (uint32_t i = lane; i < size_words; i += 32u) body[i] = 0u;
    __syncwarp();
    pack4(body, b, low_words, z0, z1, z2, z3);
    if (e) {  // e > 0 implies b < 32
      const uint32_t xm = ((z0 >> b) != 0u ? 1u : 0u) | ((z1 >> b) != 0u ? 2u : 0u) |
                          ((z2 >> b) != 0u ? 4u : 0u) | ((z3 >> b) != 0u ? 8u : 0u);
      uint32_t unused;
      uint32_t rank = warp_excl_scan(__popc(xm), unused);
      if (xm & 1u) { xpos[rank] = (uint8_t)(4u * lane); xhv[rank] = z0 >> b; rank++; }
      if (xm & 2u) { xpos[rank] = (uint8_t)(4u * lane + 1u); xhv[rank] = z1 >> b; rank++; }
      if (xm & 4u) { xpos[rank] = (uint8_t)(4u * lane + 2u); xhv[rank] = z2 >> b; rank++; }
      if (xm & 8u) { xpos[rank] = (uint8_t)(4u * lane + 3u); xhv[rank] = z3 >> b; }
      __syncwarp();
      uint32_t pword = reinterpret_cast<const uint32_t*>(xpos)[lane];
      if (4u * lane + 4u > e) pword &= 4u * lane >= e ? 0u : ((1u << (8u * (e - 4u * lane))) - 1u);
      if (lane < pw) body[low_words + lane] = pword;
      uint32_t* hp = body + low_words + pw;
      for (uint32_t x = lane; x < e; x += 32u) {
        const uint32_t hv = xhv[x], hbit = x * hb, hs = hbit & 31u;
        atomicOr(hp + (hbit >> 5), hv << hs);
        if (hs + hb > 32u) atomicOr(hp + (hbit >> 5) + 1u, hv >> (32u - hs));
      }
    }
    __syncwarp();
  }
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
  const uint32_t gs = blockIdx.x / p.trial_rows, ti = blockIdx.x % p.trial_rows;
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
  uint32_t* zi = smem;
  uint32_t* zp = smem + ((W + kStepVal - 1) / kStepVal) * kStepVal;
  if (lane_id() == 0) {  // fetch the test row (both scans) and the earlier test row's tail into L2 at once
    prefetch_l2(cur + test_row(ti) * rowb, rowb);
    prefetch_l2(prv + test_row(ti) * rowb, rowb);
    if (ti > 0) {
      const size_t tail = min(rowb, (size_t)kStepPx * at.s);
      prefetch_l2(cur + test_row(ti - 1) * rowb + rowb - tail, tail);
      prefetch_l2(prv + test_row(ti - 1) * rowb + rowb - tail, tail);
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
  if (at.qkind == 0) n = pass_a_trial<0>(c1, p1, at, W, kz, zi, zp);
  else if (at.qkind == 1) n = pass_a_trial<1>(c1, p1, at, W, kz, zi, zp);
  else n = pass_a_trial<2>(c1, p1, at, W, kz, zi, zp);
  __syncwarp();
  fill_tail(zi, n, st & kStageNoDelta);
  fill_tail(zp, n, st & kStageNoDelta);
  const uint32_t cost_i = pass_b1<false>(zi, n, ci, nullptr, st);
  const uint32_t cost_p = pass_b1<false>(zp, n, cp, nullptr, st);
  if (lane_id() == 0) {
    atomicAdd(p.cost + 2 * gs, cost_i);
    atomicAdd(p.cost + 2 * gs + 1, cost_p);
  }
}

// ----------------------------------------------------------------------------
// k_encode: one warp per row item k = (t, a, r), items taken one at a time
// from an atomic ticket so that every item a warp waits on (look-backs over
// earlier items) was handed out earlier. No CTA-wide barrier.
// ----------------------------------------------------------------------------

// Per-warp shared memory (byte offsets): residual / ZigZag / packed-body
// buffer (values rounded up to whole pass-B1 steps), coded mask bytes, block
// metadata.
struct EncWarpLayout {
  uint32_t zb, mb, meta, xpos, xhv, bytes;
};

__host__ __device__ inline EncWarpLayout enc_warp_layout(uint32_t W) {
  const uint32_t nbmax = ceil_div_u32(W, kBlockN);
  auto a16 = [](uint32_t x) { return (x + 15u) & ~15u; };
  EncWarpLayout L;
  L.zb = 0;
  L.mb = 4u * ceil_div_u32(W, kStepVal) * kStepVal;
  L.meta = a16(L.mb + ceil_div_u32(W, 32) * 4u);
  L.xpos = a16(L.meta + 8u * nbmax);
  L.xhv = L.xpos + kBlockN;
  L.bytes = a16(L.xhv + 4u * kBlockN);
  return L;
}

struct EncWarp {
  uint32_t* zb;
  uint8_t* mb;
  uint2* meta;
  uint8_t* xpos;
  uint32_t* xhv;
};

// The last nonzero sample (with all, the last sample) among the 8 (nv valid)
// in v / pv, across the warp: its residual (P: q - q', I: q). Returns false
// if there is none.
template <int QU>
__device__ __forceinline__ bool tail_residual(const uint32_t (&v)[8], const uint32_t (&pv)[8], uint32_t nv, bool pm,
                                              bool all, const AttrDev& at, uint32_t& e_last) {
  bool has = false;
  uint32_t last = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const uint32_t q = quant<QU>(v[i], at);
    if ((uint32_t)i < nv && (q != 0u || all)) {
      has = true;
      last = pm ? q - quant<QU>(pv[i], at) : q;
    }
  }
  const uint32_t hm = __ballot_sync(0xffffffffu, has);
  if (!hm) return false;
  e_last = __shfl_sync(0xffffffffu, last, 31u - __clz(hm));
  return true;
}

template <bool PM, int QU>
__device__ __forceinline__ uint32_t pass_a_any(const uint8_t* cur, const uint8_t* prv, uint8_t* st_row,
                                               const AttrDev& at, uint32_t W, uint32_t kz, uint32_t* zb,
                                               uint8_t* mb) {
  if constexpr (QU == 2) {
    return pass_a<PM, QU, 0>(cur, prv, st_row, at, W, kz, zb, mb);
  } else {
    if (at.s == 4) return pass_a<PM, QU, 4>(cur, prv, st_row, at, W, kz, zb, mb);
    if (at.s == 2) return pass_a<PM, QU, 2>(cur, prv, st_row, at, W, kz, zb, mb);
    return pass_a<PM, QU, 1>(cur, prv, st_row, at, W, kz, zb, mb);
  }
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
  uint8_t* st_row = (t + 1 == sg.T) ? sg.state_next[a] + r * rowb : nullptr;
  const int qk = (int)at.qkind;
  if (lane == 0) {  // fetch the row(s) into L2 ahead of the 256-pixel steps
    const uintptr_t c0 = reinterpret_cast<uintptr_t>(cur), c1 = c0 + rowb;
    const uintptr_t a0 = (c0 + 15u) & ~uintptr_t(15), a1 = c1 & ~uintptr_t(15);
    if (a1 > a0) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"((uint32_t)(a1 - a0)) : "memory");
    if (prv) {
      const uintptr_t p0 = reinterpret_cast<uintptr_t>(prv), p1 = p0 + rowb;
      const uintptr_t b0 = (p0 + 15u) & ~uintptr_t(15), b1 = p1 & ~uintptr_t(15);
      if (b1 > b0) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b0), "r"((uint32_t)(b1 - b0)) : "memory");
    }
  }
  // the previous row's last 256-pixel step, loaded now and read after pass A:
  // its last nonzero residual is this row's delta carry (Sec. III-C)
  const uint32_t nsteps = ceil_div_u32(W, kStepPx);
  const uint32_t tx0 = kStepPx * (nsteps - 1u) + 8u * lane;
  const uint32_t tnv = tx0 < W ? min(8u, W - tx0) : 0u;
  uint32_t tv[8], tpv[8];
  if (r > 0) {
    load8<false>(cur - rowb, at.s, tx0, tnv, vec_ok(cur - rowb, at.s), tv);
    if (prv) load8<false>(prv - rowb, at.s, tx0, tnv, vec_ok(prv - rowb, at.s), tpv);
  }

  // ---- pass A
  uint32_t n;
  if (mode) {
    if (qk == 0) n = pass_a_any<true, 0>(cur, prv, st_row, at, W, kz, w.zb, w.mb);
    else if (qk == 1) n = pass_a_any<true, 1>(cur, prv, st_row, at, W, kz, w.zb, w.mb);
    else n = pass_a_any<true, 2>(cur, prv, st_row, at, W, kz, w.zb, w.mb);
  } else {
    if (qk == 0) n = pass_a_any<false, 0>(cur, nullptr, st_row, at, W, kz, w.zb, w.mb);
    else if (qk == 1) n = pass_a_any<false, 1>(cur, nullptr, st_row, at, W, kz, w.zb, w.mb);
    else n = pass_a_any<false, 2>(cur, nullptr, st_row, at, W, kz, w.zb, w.mb);
  }
  __syncwarp();
  const uint32_t last_e = n ? w.zb[swz(n - 1)] : 0u;
  // (the failure-detection test hook, read by the STAGED instance only, may
  // withhold this row's status)
  const bool publish = !STAGED || k + 1u != p.withhold;
  if (lane == 0 && publish) {  // this row's last residual, for the rows after it
    st_publish(p.st_carry + k, kStAgg | ((unsigned long long)(n ? 1 : 0) << 32) | last_e);
  }
  fill_tail(w.zb, n, st & kStageNoDelta);

  // ---- delta carry
  uint32_t carry = 0;
  bool known = r == 0;  // e[-1] = 0 at the start of the attribute-scan
  if (r > 0) {
    if (qk == 0) known = tail_residual<0>(tv, tpv, tnv, prv != nullptr, kz == 0u, at, carry);
    else if (qk == 1) known = tail_residual<1>(tv, tpv, tnv, prv != nullptr, kz == 0u, at, carry);
    else known = tail_residual<2>(tv, tpv, tnv, prv != nullptr, kz == 0u, at, carry);
  }
  if (!known) {  // the previous rows' "last residual" words decide
    const bool ok = lookback_last(p.st_carry, k, sec_start, carry);
    if (!ok) {
      if (lane == 0) {
        atomicOr(sg.err, kErrTimeout);
        st_publish(p.st_carry + k, kStErr);
      }
      return;
    }
  }
  if (lane == 0 && publish) st_publish(p.st_carry + k, kStInc | (1ull << 32) | (n ? last_e : carry));

  // ---- mask part size: literal words
  const uint32_t* mbw = reinterpret_cast<const uint32_t*>(w.mb);
  uint32_t nlit = 0;
  for (uint32_t jb = 0; jb < nw; jb += 32) {
    const uint32_t jw = jb + lane;
    const bool lit = jw < nw && mask_class(mbw[jw], valid_bits(W, nw, jw)) == 2u;
    nlit += __popc(__ballot_sync(0xffffffffu, lit));
  }

  // ---- pass B1: delta, ZigZag, block widths
  const uint32_t nb = ceil_div_u32(n, kBlockN);
  pass_b1<true>(w.zb, n, carry, w.meta, st);
  __syncwarp();
  // body offsets: exclusive prefix of the block bytes (lane l: 4l..4l+3)
  uint32_t body = 0;
  {
    uint32_t bsz[4], mysum = 0;
#pragma unroll
    for (uint32_t q = 0; q < 4; q++) {
      const uint32_t blk = 4u * lane + q;
      bsz[q] = blk < nb ? w.meta[blk].y : 0u;
      mysum += bsz[q];
    }
    uint32_t o = warp_excl_scan(mysum, body);
#pragma unroll
    for (uint32_t q = 0; q < 4; q++) {
      const uint32_t blk = 4u * lane + q;
      if (blk < nb) w.meta[blk].y = o;
      o += bsz[q];
    }
  }
  __syncwarp();
  const uint32_t head_words = ncls + nlit + nb;
  const uint32_t chunk = 4u * head_words + body;
  if (lane == 0) {
    p.row_bytes[k] = chunk;
    p.row_nnz[k] = n;
    p.row_carry[k] = carry;
  }

  // ---- pass B2: block bodies, packed in shared memory
  pass_b2(w.zb, n, nb, w.meta, w.xpos, w.xhv);

  // ---- the chunk goes to this row's slot; k_place moves it to its offset
  uint32_t* dst = reinterpret_cast<uint32_t*>(p.slots + sg.slot_base + (size_t)kl * sg.slot_bytes);

  // ---- mask part: 2-bit class per word (16 per class word), literals
  const uint32_t below = (1u << lane) - 1u;
  uint32_t litbase = 0;
  for (uint32_t jb = 0; jb < nw; jb += 32) {
    const uint32_t jw = jb + lane;
    const uint32_t c = jw < nw ? mbw[jw] : 0u;
    const uint32_t cls = jw < nw ? mask_class(c, valid_bits(W, nw, jw)) : 0u;
    uint32_t cw = cls << (2u * (lane & 15u));
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) cw |= __shfl_xor_sync(0xffffffffu, cw, o);
    const uint32_t ci = (jb >> 4) + (lane >> 4);
    if ((lane & 15u) == 0 && ci < ncls) dst[ci] = cw;
    const uint32_t litm = __ballot_sync(0xffffffffu, cls == 2u);
    if (cls == 2u) dst[ncls + litbase + __popc(litm & below)] = c;
    litbase += __popc(litm);
  }
  // ---- block headers and bodies
  for (uint32_t blk = lane; blk < nb; blk += 32) dst[ncls + nlit + blk] = w.meta[blk].x;
  uint32_t* bd = dst + head_words;
  for (uint32_t i = lane; i < body / 4u; i += 32u) bd[i] = w.zb[i];
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
  w.meta = reinterpret_cast<uint2*>(wb + lay.meta);
  w.xpos = wb + lay.xpos;
  w.xhv = reinterpret_cast<uint32_t*>(wb + lay.xhv);
  while (true) {
    uint32_t k = 0;
    if (lane == 0) k = atomicAdd(p.ticket, 1u);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (k >= p.n_items) break;
    encode_item<STAGED>(p, k, w);
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
  if (threadIdx.x == 0) {
    p.sec_bytes[gs] = 8ull * H + bytes;
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
  // row chunks: a warp per row, slot -> stream, 4 words in flight per lane
  const unsigned long long data_at = sec_at + 8ull * H;
  const uint32_t lane = lane_id();
  for (uint32_t r = part * kWarps + warp_id(); r < H; r += kWarps * kPlaceSplit) {
    const uint32_t words = p.row_bytes[item0 + r] / 4u;
    const unsigned long long at = data_at + smem[r];
    if (at + 4ull * words > cap) {
      if (lane == 0) atomicOr(sg.err, kErrCapacity);
      continue;
    }
    const uint32_t* src =
        reinterpret_cast<const uint32_t*>(p.slots + sg.slot_base + (size_t)(local0 + r) * sg.slot_bytes);
    uint32_t* dst = reinterpret_cast<uint32_t*>(out + at);
    for (uint32_t i = lane; i < words; i += 128u) {
      uint32_t v[4];
#pragma unroll
      for (uint32_t q = 0; q < 4; q++) v[q] = i + 32u * q < words ? __ldcs(src + i + 32u * q) : 0u;
#pragma unroll
      for (uint32_t q = 0; q < 4; q++)
        if (i + 32u * q < words) dst[i + 32u * q] = v[q];
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
  if ((L.mb | L.meta | L.xpos | L.xhv | L.bytes) & 15u) return (int)cudaErrorInvalidValue;  // 16-byte aligned regions
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
  const uint32_t want = ceil_div_u32(p.n_items, wpc);
  out->wpc = wpc;
  out->ctas_per_sm = ctas;
  out->items_per_ticket = 1;
  out->grid = max(1u, min(want, ctas * (uint32_t)sms));
  return 0;
}

size_t trial_smem_bytes_host(uint32_t W) { return 2ull * 4u * ceil_div_u32(W, kStepVal) * kStepVal; }

int launch_encode(const EncParams& p, void* stream, void* const* ev) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t s_trial = trial_smem_bytes_host(p.max_W);
  RowsLaunch rl{};
  int rc = encode_rows_launch(p, &rl);
  if (rc != 0) return rc;
  const size_t s_place = 4ull * kMaxH;
  cudaError_t e = cudaFuncSetAttribute(k_trial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_trial);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_place, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_place);
  if (e != cudaSuccess) return (int)e;
  auto mark = [&](int i) {
    if (ev) record_event(ev[i], st);
  };
  mark(0);
  if (p.trial_rows) k_trial<<<p.n_sec * p.trial_rows, 32, s_trial, st>>>(p);
  mark(1);
  const size_t smem = (size_t)rl.wpc * enc_warp_layout(p.max_W).bytes;
  if (p.staged) {
    if (rl.wpc == 4) k_encode<4, true><<<rl.grid, 4 * 32, smem, st>>>(p);
    else if (rl.wpc == 2) k_encode<2, true><<<rl.grid, 2 * 32, smem, st>>>(p);
    else k_encode<1, true><<<rl.grid, 32, smem, st>>>(p);
  } else {
    if (rl.wpc == 4) k_encode<4, false><<<rl.grid, 4 * 32, smem, st>>>(p);
    else if (rl.wpc == 2) k_encode<2, false><<<rl.grid, 2 * 32, smem, st>>>(p);
    else k_encode<1, false><<<rl.grid, 32, smem, st>>>(p);
  }
  mark(2);
  k_sec_sizes<<<p.n_sec, kThreads, 0, st>>>(p);
  k_place<<<p.n_sec * kPlaceSplit, kThreads, s_place, st>>>(p);
  mark(3);
  return (int)cudaGetLastError();
}

}  // namespace jiffy
