// Jiffy encoder kernels (sm_103a).
//
// One call codes T consecutive scans of each of one or more streams (the
// segments of the call), all in parallel: the P prediction of scan t uses the
// *input* of scan t-1 (Sec. III-D), so no scan waits for another's output.
// Four launches:
//   k_trial      one CTA per section (scan, attribute): I/P choice by trial
//                compression of a few scanlines, mask excluded (Sec. III-E,
//                Sec. IV-E).
//   k_encode     one warp per row item (scan, attribute, row), ticket order:
//                stage the row -> quantize (Sec. III-B) -> zero bitmask
//                (Sec. III-C) -> mask XOR with the previous scan for P
//                (Sec. III-D) -> compaction -> residual -> delta (the carry
//                from the previous row's tail, else a look-back) -> ZigZag
//                (Eq. 1) -> block widths and packing of 128-value blocks
//                (Sec. II) into the row's slot.
//   k_sec_sizes  one CTA per section: its bytes and nonzero count.
//   k_place      one CTA per section: offsets, row table, chunk copies, frame
//                and stream headers.
#include "jiffy_device.cuh"
#include "jiffy_kernels.h"

namespace jiffy {

// ----------------------------------------------------------------------------
// Row load: quantize the samples of one row (and of the previous scan's row),
// build the zero bitmask words, and compact the residuals of the nonzero
// samples into shared memory in row-major order.
//   want_i / want_p: write I residuals (q) to eI and/or P residuals (q - pq)
//   to eP. coded (nullable): receives per word M (mode I) or M ^ Mprev (P).
//   Both rows hold raw samples (the stored previous scan is dequantized, and
//   quantizing q * P gives q back), so one quantizer serves both.
// Returns the row's nonzero count. Every thread calls it.
// ----------------------------------------------------------------------------
struct RowLoad {
  const uint8_t* cur;   // row of the current scan (raw samples)
  const uint8_t* prev;  // row of the previous scan, or null
  AttrDev at;           // quantizer
  uint32_t W, nw;
};

__device__ uint32_t load_compact_row(const RowLoad& L, bool want_i, bool want_p, bool xor_prev,
                                     uint32_t* eI, uint32_t* eP, uint32_t* coded, uint32_t* s_cnt) {
  const uint32_t lane = lane_id(), warp = warp_id();
  const uint32_t s = L.at.s;
  uint32_t total = 0;
  for (uint32_t wbase = 0; wbase < L.nw; wbase += kWarps * kSegWords) {
    uint32_t v[kSegWords], pv[kSegWords];
#pragma unroll
    for (uint32_t i = 0; i < kSegWords; i++) {
      uint32_t j = wbase + warp * kSegWords + i;
      uint32_t x = j * 32u + lane;
      bool in = j < L.nw && x < L.W;
      v[i] = in ? load_sample(L.cur, s, x) : 0u;
      pv[i] = (in && L.prev) ? load_sample(L.prev, s, x) : 0u;
    }
    uint32_t ei[kSegWords], ep[kSegWords], nzm[kSegWords];
    uint32_t cnt = 0;
#pragma unroll
    for (uint32_t i = 0; i < kSegWords; i++) {
      uint32_t j = wbase + warp * kSegWords + i;
      uint32_t x = j * 32u + lane;
      bool in = j < L.nw && x < L.W;
      uint32_t q = quantize(v[i], L.at);
      uint32_t pq = L.prev ? quantize(pv[i], L.at) : 0u;
      uint32_t nz = __ballot_sync(0xffffffffu, in && q != 0u);
      if (coded) {
        uint32_t m = __ballot_sync(0xffffffffu, in && q == 0u);  // Sec. III-C: 1 = zero sample
        if (xor_prev) m ^= __ballot_sync(0xffffffffu, in && pq == 0u);  // Sec. III-D
        if (lane == 0 && j < L.nw) coded[j] = m;
      }
      ei[i] = q;
      ep[i] = q - pq;  // modulo 2^32
      nzm[i] = nz;
      cnt += __popc(nz);
    }
    if (lane == 0) s_cnt[warp] = cnt;
    __syncthreads();
    uint32_t base = total, seg = 0;
#pragma unroll
    for (int w2 = 0; w2 < kWarps; w2++) {
      uint32_t c = s_cnt[w2];
      if ((uint32_t)w2 < warp) base += c;
      seg += c;
    }
    const uint32_t below = (1u << lane) - 1u;
#pragma unroll
    for (uint32_t i = 0; i < kSegWords; i++) {
      uint32_t nz = nzm[i];
      if ((nz >> lane) & 1u) {
        uint32_t k = base + __popc(nz & below);
        if (want_i) eI[k] = ei[i];
        if (want_p) eP[k] = ep[i];
      }
      base += __popc(nz);
    }
    total += seg;
    __syncthreads();
  }
  return total;
}

// Warp-wide: loads block blk of z (n values) into lanes (4 per lane).
__device__ __forceinline__ void load_block(const uint32_t* z, uint32_t n, uint32_t (&r)[4]) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (int m = 0; m < 4; m++) {
    uint32_t i = lane + 32u * m;
    r[m] = i < n ? z[i] : 0u;
  }
}

// Index of the segment holding global index key: the last i with base[i] <= key.
__device__ __forceinline__ uint32_t find_seg(const uint32_t* base, uint32_t n, uint32_t key) {
  uint32_t lo = 0, hi = n;  // base[lo] <= key < base[hi] (base[n] = infinity)
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(base + mid) <= key) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ----------------------------------------------------------------------------
// k_trial: Sec. III-E. For scans with a predecessor and no forced mode, codes
// the test rows floor((2k+1)H/(2L)) (de-duplicated) both ways, the residuals
// of the test rows delta-coded as one flat vector from 0 and packed per row,
// and picks P iff its packed bytes are strictly fewer.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_trial(EncParams p) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_cnt[kWarps + 1];
  __shared__ unsigned long long s_cost[2];
  __shared__ uint32_t s_rows[kMaxTestLines];
  __shared__ uint32_t s_nrows;
  __shared__ uint32_t s_hist[kWarps][33];

  const uint32_t gs = blockIdx.x;
  const EncSeg& sg = p.seg[find_seg(p.seg_sec_base, p.n_seg, gs)];
  const uint32_t ta = gs - sg.sec_base;
  const uint32_t t = ta / sg.A, a = ta % sg.A;
  uint32_t* eI = smem;
  uint32_t* eP = smem + sg.W;
  if (sg.frame0 + t == 0 || sg.force_mode == 0) {
    if (threadIdx.x == 0) p.modes[gs] = 0;
    return;
  }
  if (sg.force_mode == 1) {
    if (threadIdx.x == 0) p.modes[gs] = 1;
    return;
  }
  const AttrDev at = sg.attrs[a];
  if (threadIdx.x == 0) {
    uint32_t n = 0;
    for (uint32_t k = 0; k < sg.test_lines; k++) {
      uint32_t r = (uint32_t)(((unsigned long long)(2 * k + 1) * sg.H) / (2ull * sg.test_lines));
      if (n == 0 || s_rows[n - 1] != r) s_rows[n++] = r;
    }
    s_nrows = n;
    s_cost[0] = s_cost[1] = 0;
  }
  __syncthreads();
  const size_t rowb = (size_t)sg.W * at.s;
  uint32_t carry_i = 0, carry_p = 0;  // flat vector starts from 0
  unsigned long long cost_i = 0, cost_p = 0;  // per-warp partial sums (lane 0)
  for (uint32_t ri = 0; ri < s_nrows; ri++) {
    const uint32_t r = s_rows[ri];
    RowLoad L{sg.cur[ta] + r * rowb, sg.prev[ta] + r * rowb, at, sg.W, sg.nw};
    uint32_t n = load_compact_row(L, true, true, false, eI, eP, nullptr, s_cnt);
    // residuals -> delta -> ZigZag -> block costs, both modes
    const uint32_t nb = ceil_div_u32(n, kBlockN);
    for (uint32_t blk = warp_id(); blk < 2 * nb; blk += kWarps) {
      const uint32_t mode = blk / nb, bi = blk % nb;
      const uint32_t* e = mode ? eP : eI;
      const uint32_t carry = mode ? carry_p : carry_i;
      const uint32_t base = bi * kBlockN, m = min(kBlockN, n - base);
      uint32_t z[4];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        uint32_t i = base + lane_id() + 32u * q;
        z[q] = (i - base) < m ? zigzag(e[i] - (i ? e[i - 1] : carry)) : 0u;
      }
      BlockChoice c = choose_block(z, m, s_hist[warp_id()]);
      if (lane_id() == 0) {
        if (mode) cost_p += 4u + c.bytes;
        else cost_i += 4u + c.bytes;
      }
    }
    if (n > 0) { carry_i = eI[n - 1]; carry_p = eP[n - 1]; }
    __syncthreads();  // e arrays are rewritten by the next row
  }
  if (lane_id() == 0) {
    atomicAdd(&s_cost[0], cost_i);
    atomicAdd(&s_cost[1], cost_p);
  }
  __syncthreads();
  if (threadIdx.x == 0) p.modes[gs] = s_cost[1] < s_cost[0] ? 1u : 0u;
}

// ----------------------------------------------------------------------------
// k_encode: one warp per row item k = (t, a, r), items taken one at a time
// from an atomic ticket so that every item a warp waits on (look-backs over
// earlier items) was handed out earlier. No CTA-wide barrier.
// ----------------------------------------------------------------------------

// Per-warp shared memory (byte offsets): ZigZag values of the row, coded mask
// words, per-block {header, body byte offset}, width histogram, and the body
// of the block being packed.
struct EncWarpLayout {
  uint32_t z, coded, meta, hist, pbuf, bytes;
};

__host__ __device__ inline EncWarpLayout enc_warp_layout(uint32_t W) {
  const uint32_t nbmax = ceil_div_u32(W, kBlockN), nw = ceil_div_u32(W, 32);
  auto a16 = [](uint32_t x) { return (x + 15u) & ~15u; };
  EncWarpLayout L;
  L.z = 0;
  L.coded = a16(4u * W);
  L.meta = a16(L.coded + 4u * nw);
  L.hist = a16(L.meta + 8u * nbmax);
  L.pbuf = a16(L.hist + 4u * 36u);
  L.bytes = a16(L.pbuf + 4u * 192u);  // a packed block body never exceeds 162 words
  return L;
}

__device__ __forceinline__ uint32_t mask_class(uint32_t c, uint32_t valid) {
  return c == 0u ? 0u : (c == valid ? 1u : 2u);
}

struct EncWarp {
  uint32_t* zbuf;
  uint32_t* coded;
  uint8_t* coded_b;
  uint2* meta;
  uint32_t* hist;
  uint32_t* pbuf;
};

// One row item, samples of S bytes (compile-time, so each warp runs one
// compact path).
__device__ __forceinline__ void encode_item(const EncParams& p, const uint32_t k, const EncWarp& w) {
  const EncSeg& sg = p.seg[find_seg(p.seg_item_base, p.n_seg, k)];
  const uint32_t lane = lane_id();
  const uint32_t H = sg.H, W = sg.W, A = sg.A, nw = sg.nw, ncls = sg.ncls;
  const uint32_t niter = ceil_div_u32(W, 256u);
  const uint32_t below = (1u << lane) - 1u;
  uint32_t* zbuf = w.zbuf;
  uint32_t* coded = w.coded;
  const uint32_t kl = k - sg.item_base;  // item within the segment
  const uint32_t r = kl % H, ta = kl / H, a = ta % A, t = ta / A;
  const uint32_t sec_start = k - r;  // global item of row 0 of this attribute-scan
  const AttrDev at = sg.attrs[a];
  const uint32_t S = at.s;
  const uint32_t mode = p.modes[sg.sec_base + ta];
  const size_t rowb = (size_t)W * S;
  const uint8_t* cur = sg.cur[ta] + r * rowb;
  const uint8_t* prv = mode ? sg.prev[ta] + r * rowb : nullptr;
  uint8_t* st_row = (t + 1 == sg.T) ? sg.state_next[a] + r * rowb : nullptr;
  const bool vec_prv = prv && vec_ok(prv, S), vec_st = st_row && vec_ok(st_row, S);

  for (uint32_t j = lane; j < nw; j += 32) coded[j] = 0u;
  // stage the row in one round of loads, at the top of the ZigZag buffer:
  // ZigZag values fill it from the bottom and, with every lane reading its
  // pixels of a step before any value of that step is written, never reach
  // a pixel that is still to be read (raw row at byte (4 - S) * W)
  uint8_t* raw = reinterpret_cast<uint8_t*>(zbuf) + (4u - S) * W;
  stage_bytes(raw, cur, W * S);
  if (prv) prefetch_l1(prv, (uint32_t)rowb);
  const bool vec_cur = vec_ok(raw, S);
  // the previous row's last 256 pixels, for the delta carry (read now, used
  // after pass A)
  const uint32_t px0 = W > 256u ? W - 256u : 0u;
  const uint32_t pnv = px0 + 8u * lane < W ? min(8u, W - (px0 + 8u * lane)) : 0u;
  uint32_t tv[8], tpv[8];
  if (r > 0) {
    const bool tvec = (px0 & 7u) == 0;
    load8<false>(cur - rowb, S, px0 + 8u * lane, pnv, tvec && vec_ok(cur - rowb, S), tv);
    if (prv) load8<false>(prv - rowb, S, px0 + 8u * lane, pnv, tvec && vec_ok(prv - rowb, S), tpv);
  }
  __syncwarp();

  // ---- delta carry: the residual preceding this row in the attribute-scan's
  //      flat vector (Sec. III-C). The previous row's tail usually holds it;
  //      otherwise a "last valid" look-back over the earlier rows decides.
  uint32_t carry = 0;
  bool known = r == 0;  // e[-1] = 0 at the start of the attribute-scan
  if (r > 0) {
    uint32_t tnz = 0, tlast = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      const uint32_t q = quantize(tv[i], at);
      const uint32_t pq = prv ? quantize(tpv[i], at) : 0u;
      if ((uint32_t)i < pnv && q != 0u) {
        tnz = 1u;
        tlast = q - pq;
      }
    }
    const uint32_t has = __ballot_sync(0xffffffffu, tnz != 0u);
    if (has) {
      carry = __shfl_sync(0xffffffffu, tlast, 31u - __clz(has));
      known = true;
    }
  }
  // ---- pass A: quantize (Sec. III-B), zero mask (Sec. III-C), mask XOR
  //      (Sec. III-D), compaction, residual, delta, ZigZag (Eq. 1)
  uint32_t n = 0;          // nonzero samples so far (uniform)
  uint32_t last_e = 0;     // last residual so far (uniform, valid when n > 0)
  uint32_t e_first = 0;    // the row's first residual (uniform)
  for (uint32_t it = 0; it < niter; it++) {
    const uint32_t x0 = 256u * it + 8u * lane;
    const uint32_t nv = x0 < W ? min(8u, W - x0) : 0u;
    uint32_t v[8], pv[8];
    load8<false>(raw, S, x0, nv, vec_cur, v);
    if (prv) load8<false>(prv, S, x0, nv, vec_prv, pv);
    __syncwarp();  // every lane has its pixels of this step before values are written
    uint32_t e[8];
    uint32_t mb = 0, pm = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      const uint32_t q = quantize(v[i], at);
      v[i] = q;
      const uint32_t pq = prv ? quantize(pv[i], at) : 0u;
      mb |= (uint32_t)((uint32_t)i < nv && q == 0u) << i;
      pm |= (uint32_t)((uint32_t)i < nv && pq == 0u) << i;
      e[i] = q - pq;  // I: q (pq = 0); P: q - pq, modulo 2^32
    }
    if (st_row && nv) {  // the next call's previous scan, dequantized as the decoder holds it
      uint32_t sv[8];
#pragma unroll
      for (int i = 0; i < 8; i++) sv[i] = v[i] * at.P;
      store8(st_row, S, x0, nv, vec_st, sv);
    }
    if (nv) w.coded_b[x0 >> 3] = (uint8_t)(mode ? (mb ^ pm) : mb);
    const uint32_t nz = ~mb & ((1u << nv) - 1u);
    const uint32_t c = __popc(nz);
    uint32_t tot;
    const uint32_t k0 = n + warp_excl_scan(c, tot);
    // the residual before this lane's first nonzero: the last one of the
    // nearest lower lane that has any, else the last one so far
    uint32_t my_last = 0, my_first = 0;
#pragma unroll
    for (int i = 7; i >= 0; i--)
      if ((nz >> i) & 1u) my_first = e[i];
#pragma unroll
    for (int i = 0; i < 8; i++)
      if ((nz >> i) & 1u) my_last = e[i];
    const uint32_t has = __ballot_sync(0xffffffffu, c != 0u);
    const uint32_t lower = has & below;
    const uint32_t src = lower ? 31u - __clz(lower) : 0u;
    const uint32_t from_lane = __shfl_sync(0xffffffffu, my_last, src);
    uint32_t pe = lower ? from_lane : last_e;  // (n == 0: placeholder, fixed after the carry)
    uint32_t kk = k0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      if ((nz >> i) & 1u) {
        zbuf[kk++] = zigzag(e[i] - pe);
        pe = e[i];
      }
    }
    if (has) {
      const uint32_t hi = 31u - __clz(has), lo = __ffs(has) - 1u;
      const uint32_t lastv = __shfl_sync(0xffffffffu, my_last, hi);
      const uint32_t firstv = __shfl_sync(0xffffffffu, my_first, lo);
      if (n == 0) e_first = firstv;
      last_e = lastv;
    }
    n += tot;
  }
  if (lane == 0) {
    const unsigned long long lastv = n ? last_e : carry;
    if (known) st_publish(p.st_carry + k, kStInc | (1ull << 32) | lastv);
    else st_publish(p.st_carry + k, kStAgg | ((unsigned long long)(n ? 1 : 0) << 32) | last_e);
  }

  // ---- block widths (Sec. II) of blocks 1.. first: only block 0 depends on
  //      the carry, so a fallback wait overlaps this work
  const uint32_t nb = ceil_div_u32(n, kBlockN);
  auto width_of = [&](uint32_t blk) {
    const uint32_t base = blk * kBlockN, m = min(kBlockN, n - base);
    uint32_t z[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint32_t i = lane + 32u * q;
      z[q] = i < m ? zbuf[base + i] : 0u;
    }
    const BlockChoice bc = choose_block(z, m, w.hist);
    if (lane == 0) w.meta[blk] = make_uint2(bc.b | (bc.e << 8) | (bc.hb << 16), bc.bytes);
  };
  for (uint32_t blk = 1; blk < nb; blk++) width_of(blk);
  if (!known) {
    const bool ok = lookback_last(p.st_carry, k, sec_start, carry);
    if (lane == 0) st_publish(p.st_carry + k, ok ? (kStInc | (1ull << 32) | (n ? last_e : carry)) : kStErr);
    if (!ok) {
      if (lane == 0) atomicOr(sg.err, kErrTimeout);
      return;
    }
  }
  if (n) {
    if (lane == 0) zbuf[0] = zigzag(e_first - carry);
    __syncwarp();
    width_of(0);
  }
  __syncwarp();

  // ---- body offsets: exclusive prefix of the block bytes (lane l: 4l..4l+3)
  uint32_t body = 0;
  {
    uint32_t bsz[4], mysum = 0;
#pragma unroll
    for (uint32_t q = 0; q < 4; q++) {
      const uint32_t blk = 4u * lane + q;
      bsz[q] = blk < nb ? w.meta[blk].y : 0u;
      mysum += bsz[q];
    }
    uint32_t off = warp_excl_scan(mysum, body);
#pragma unroll
    for (uint32_t q = 0; q < 4; q++) {
      const uint32_t blk = 4u * lane + q;
      if (blk < nb) w.meta[blk].y = off;
      off += bsz[q];
    }
  }

  // ---- mask part size: literal words
  uint32_t nlit = 0;
  for (uint32_t jb = 0; jb < nw; jb += 32) {
    const uint32_t j = jb + lane;
    const uint32_t valid = (j + 1 < nw || (W & 31u) == 0) ? 0xffffffffu : ((1u << (W & 31u)) - 1u);
    const bool lit = j < nw && mask_class(coded[j], valid) == 2u;
    nlit += __popc(__ballot_sync(0xffffffffu, lit));
  }
  __syncwarp();
  const uint32_t head_words = ncls + nlit + nb;
  const uint32_t chunk = 4u * head_words + body;
  if (lane == 0) {
    p.row_bytes[k] = chunk;
    p.row_nnz[k] = n;
    p.row_carry[k] = carry;
  }
  // the chunk goes to this row's slot; k_place moves it to its offset
  uint32_t* dst = reinterpret_cast<uint32_t*>(p.slots + sg.slot_base + (size_t)kl * sg.slot_bytes);

  // ---- mask part: 2-bit class per word (16 per class word), literals
  uint32_t litbase = 0;
  for (uint32_t jb = 0; jb < nw; jb += 32) {
    const uint32_t j = jb + lane;
    const uint32_t valid = (j + 1 < nw || (W & 31u) == 0) ? 0xffffffffu : ((1u << (W & 31u)) - 1u);
    const uint32_t c = j < nw ? coded[j] : 0u;
    const uint32_t cls = j < nw ? mask_class(c, valid) : 0u;
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
  for (uint32_t blk = 0; blk < nb; blk++) {
    const uint32_t base = blk * kBlockN, m = min(kBlockN, n - base);
    const uint2 md = w.meta[blk];
    const uint32_t b = md.x & 0xffu, ex = (md.x >> 8) & 0xffu, hb = (md.x >> 16) & 0xffu;
    const uint32_t low_words = (m * b + 31u) >> 5;
    const uint32_t high0 = low_words + ((ex + 3u) >> 2);  // first word of the high parts
    const uint32_t body_words = block_body_bytes(m, b, ex, b + hb) / 4u;
    uint32_t* pb = w.pbuf;
    for (uint32_t i = lane; i < body_words; i += 32) pb[i] = 0u;
    __syncwarp();
    // value-centric packing into shared memory: low b bits of every value at
    // bit i*b; exceptions: position byte and high part (hb bits) by rank
    const uint32_t bmask = b >= 32u ? 0xffffffffu : ((1u << b) - 1u);
    const uint32_t* zb = zbuf + base;
    uint32_t xi = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const uint32_t i = lane + 32u * q;
      const bool valid = i < m;
      const uint32_t vz = valid ? zb[i] : 0u;
      if (valid && b) {
        const uint32_t bit = i * b, wi = bit >> 5, sh = bit & 31u, lo = vz & bmask;
        atomicOr(pb + wi, lo << sh);
        if (sh + b > 32u) atomicOr(pb + wi + 1u, lo >> (32u - sh));
      }
      if (ex) {
        const bool isx = valid && bit_width(vz) > b;
        const uint32_t bal = __ballot_sync(0xffffffffu, isx);
        if (isx) {
          const uint32_t slot = xi + __popc(bal & below);
          atomicOr(pb + low_words + (slot >> 2), i << (8u * (slot & 3u)));
          const uint32_t hv = vz >> b, hbit = slot * hb, hw = high0 + (hbit >> 5), hs = hbit & 31u;
          atomicOr(pb + hw, hv << hs);
          if (hs + hb > 32u) atomicOr(pb + hw + 1u, hv >> (32u - hs));
        }
        xi += __popc(bal);
      }
    }
    __syncwarp();
    uint32_t* bd = dst + head_words + md.y / 4u;
    for (uint32_t i = lane; i < body_words; i += 32) bd[i] = pb[i];
    __syncwarp();
  }
  __syncwarp();
}

template <int WPC>
__global__ void __launch_bounds__(WPC * 32) k_encode(EncParams p) {
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t lane = lane_id();
  const EncWarpLayout lay = enc_warp_layout(p.max_W);
  uint8_t* wb = reinterpret_cast<uint8_t*>(smem) + warp_id() * lay.bytes;
  EncWarp w;
  w.zbuf = reinterpret_cast<uint32_t*>(wb + lay.z);
  w.coded = reinterpret_cast<uint32_t*>(wb + lay.coded);
  w.coded_b = wb + lay.coded;
  w.meta = reinterpret_cast<uint2*>(wb + lay.meta);
  w.hist = reinterpret_cast<uint32_t*>(wb + lay.hist);
  w.pbuf = reinterpret_cast<uint32_t*>(wb + lay.pbuf);
  while (true) {
    uint32_t k = 0;
    if (lane == 0) k = atomicAdd(p.ticket, 1u);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (k >= p.n_items) break;
    encode_item(p, k, w);
  }
}

// ----------------------------------------------------------------------------
// k_sec_sizes: one CTA per section (scan t, attribute a): its bytes (row
// table + row chunks) and nonzero count.
// k_place: one CTA per section: the section's offset in the stream (prefix
// over the earlier sections), its row table (end offsets + carries), the copy
// of each row chunk from its slot, and, for attribute 0, the frame header and
// frame offset; section 0 also writes the stream header. Every write is
// checked against the output capacity.
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
  const uint32_t H = sg.H;
  const uint32_t item0 = sg.item_base + (gs - sg.sec_base) * H;
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

__global__ void __launch_bounds__(kThreads) k_place(EncParams p) {
  extern __shared__ __align__(16) uint32_t smem[];  // [H] row chunk starts
  __shared__ unsigned long long s_red[kWarps];
  __shared__ uint32_t s_tmp[kWarps + 1];
  const uint32_t gs = blockIdx.x;
  const EncSeg& sg = p.seg[find_seg(p.seg_sec_base, p.n_seg, gs)];
  const uint32_t H = sg.H, A = sg.A;
  const uint32_t ta = gs - sg.sec_base, t = ta / A, a = ta % A;
  const uint32_t item0 = sg.item_base + ta * H;
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
  for (uint32_t r = threadIdx.x; r < H; r += kThreads) {
    const uint32_t end = (r + 1 < H) ? smem[r + 1] : data;
    put_u32_guarded(out, cap, sec_at + 8ull * r, end, sg.err);
    put_u32_guarded(out, cap, sec_at + 8ull * r + 4, p.row_carry[item0 + r], sg.err);
  }
  // row chunks: warp per row, slot -> stream (4-byte aligned words)
  const unsigned long long data_at = sec_at + 8ull * H;
  for (uint32_t r = warp_id(); r < H; r += kWarps) {
    const uint32_t words = p.row_bytes[item0 + r] / 4u;
    const unsigned long long at = data_at + smem[r];
    if (at + 4ull * words > cap) {
      if (lane_id() == 0) atomicOr(sg.err, kErrCapacity);
      continue;
    }
    const uint32_t* src =
        reinterpret_cast<const uint32_t*>(p.slots + sg.slot_base + (size_t)(ta * H + r) * sg.slot_bytes);
    uint32_t* dst = reinterpret_cast<uint32_t*>(out + at);
    for (uint32_t i = lane_id(); i < words; i += 32u) dst[i] = src[i];
  }
  if (a == 0 && threadIdx.x == 0) {
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
        put_u32_guarded(out, cap, 16 + 8ull * aa, sg.attrs[aa].s | (1u << 8), sg.err);
        put_u32_guarded(out, cap, 20 + 8ull * aa, sg.attrs[aa].P, sg.err);
      }
    }
  }
}

size_t enc_smem_bytes_host(uint32_t W) { return enc_warp_layout(W).bytes; }

constexpr size_t kRowsSmemAuto = 100 * 1024;  // per CTA when picking warps per CTA by itself
constexpr size_t kRowsSmemMax = 227 * 1024;

template <int WPC>
static cudaError_t rows_occupancy(size_t smem, int* per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_encode<WPC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_encode<WPC>, WPC * 32, smem);
}

int encode_rows_launch(const EncParams& p, RowsLaunch* out) {
  const EncWarpLayout L = enc_warp_layout(p.max_W);
  if ((L.coded | L.meta | L.hist | L.pbuf | L.bytes) & 15u)
    return (int)cudaErrorInvalidValue;  // every per-warp region starts 16-byte aligned
  uint32_t wpc = p.wpc;
  if ((wpc != 1 && wpc != 2 && wpc != 4) || wpc * L.bytes > kRowsSmemMax) wpc = 0;
  if (!wpc) wpc = 4 * L.bytes <= kRowsSmemAuto ? 4u : (2 * L.bytes <= kRowsSmemAuto ? 2u : 1u);
  const size_t smem = (size_t)wpc * L.bytes;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    if (wpc == 4) e = rows_occupancy<4>(smem, &per_sm);
    else if (wpc == 2) e = rows_occupancy<2>(smem, &per_sm);
    else e = rows_occupancy<1>(smem, &per_sm);
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

int launch_encode(const EncParams& p, void* stream, void* const* ev) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t s_trial = 8ull * p.max_W, s_place = 4ull * kMaxH;
  RowsLaunch rl{};
  int rc = encode_rows_launch(p, &rl);
  if (rc != 0) return rc;
  cudaError_t e = cudaFuncSetAttribute(k_trial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_trial);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_place, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_place);
  if (e != cudaSuccess) return (int)e;
  auto mark = [&](int i) {
    if (ev) cudaEventRecord(reinterpret_cast<cudaEvent_t>(ev[i]), st);
  };
  mark(0);
  k_trial<<<p.n_sec, kThreads, s_trial, st>>>(p);
  mark(1);
  const size_t smem = (size_t)rl.wpc * enc_warp_layout(p.max_W).bytes;
  if (rl.wpc == 4) k_encode<4><<<rl.grid, 4 * 32, smem, st>>>(p);
  else if (rl.wpc == 2) k_encode<2><<<rl.grid, 2 * 32, smem, st>>>(p);
  else k_encode<1><<<rl.grid, 32, smem, st>>>(p);
  mark(2);
  k_sec_sizes<<<p.n_sec, kThreads, 0, st>>>(p);
  k_place<<<p.n_sec, kThreads, s_place, st>>>(p);
  mark(3);
  return (int)cudaGetLastError();
}

}  // namespace jiffy
