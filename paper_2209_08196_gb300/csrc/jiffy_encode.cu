// Jiffy encoder kernels (sm_103a).
//
// One call codes T consecutive scans of one stream, all in parallel: the P
// prediction of scan t uses the *input* of scan t-1 (Sec. III-D), so no scan
// waits for another's output. Three launches:
//   k_trial     one CTA per (scan, attribute): I/P choice by trial compression
//               of a few scanlines, mask excluded (Sec. III-E, Sec. IV-E).
//   k_encode    one CTA per (scan, attribute, row), taken in ticket order:
//               quantize (Sec. III-B) -> zero bitmask by __ballot_sync
//               (Sec. III-C) -> mask XOR with the previous scan for P
//               (Sec. III-D) -> mask class code -> compaction -> residual ->
//               delta carried across rows by a look-back -> ZigZag (Eq. 1) ->
//               block width choice and funnel packing of 128-value blocks
//               (Sec. II) in shared memory -> byte offset by decoupled
//               look-back -> coalesced copy to the output.
//   k_finalize  one CTA per frame: row tables, frame headers, stream header,
//               frame offsets.
#include "jiffy_device.cuh"
#include "jiffy_kernels.h"

namespace jiffy {

// ----------------------------------------------------------------------------
// Row load: quantize the samples of one row (and of the previous scan's row),
// build the zero bitmask words, and compact the residuals of the nonzero
// samples into shared memory in row-major order.
//   want_i / want_p: write I residuals (q) to eI and/or P residuals (q - pq)
//   to eP. coded (nullable): receives per word M (mode I) or M ^ Mprev (P).
//   st_row (nullable): receives q (state of the next call).
// Returns the row's nonzero count. Every thread calls it.
// ----------------------------------------------------------------------------
struct RowLoad {
  const uint8_t* cur;   // row of the current scan (raw samples)
  const uint8_t* prev;  // row of the previous scan, or null
  AttrDev at;           // quantizer of cur
  AttrDev pat;          // quantizer of prev (identity when prev is stored q)
  uint32_t W, nw;
};

__device__ uint32_t load_compact_row(const RowLoad& L, bool want_i, bool want_p, bool xor_prev,
                                     uint32_t* eI, uint32_t* eP, uint32_t* coded, uint8_t* st_row,
                                     uint32_t* s_cnt) {
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
      uint32_t pq = L.prev ? quantize(pv[i], L.pat) : 0u;
      if (st_row && in) store_sample(st_row, s, x, q);
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

// ----------------------------------------------------------------------------
// k_trial: Sec. III-E. For scans with a predecessor and no forced mode, codes
// the test rows floor((2k+1)H/(2L)) (de-duplicated) both ways, the residuals
// of the test rows delta-coded as one flat vector from 0 and packed per row,
// and picks P iff its packed bytes are strictly fewer.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_trial(EncParams p) {
  extern __shared__ __align__(16) uint32_t smem[];
  uint32_t* eI = smem;
  uint32_t* eP = smem + p.W;
  __shared__ uint32_t s_cnt[kWarps + 1];
  __shared__ unsigned long long s_cost[2];
  __shared__ uint32_t s_rows[kMaxTestLines];
  __shared__ uint32_t s_nrows;

  const uint32_t ta = blockIdx.x;
  const uint32_t t = ta / p.A, a = ta % p.A;
  if (p.frame0 + t == 0 || p.force_mode == 0) {
    if (threadIdx.x == 0) p.modes[ta] = 0;
    return;
  }
  if (p.force_mode == 1) {
    if (threadIdx.x == 0) p.modes[ta] = 1;
    return;
  }
  const AttrDev at = p.attrs[a];
  AttrDev pat = at;
  if (t == 0) { pat.P = 1; pat.qmax = 0xffffffffu; }  // previous scan stored quantized
  if (threadIdx.x == 0) {
    uint32_t n = 0;
    for (uint32_t k = 0; k < p.test_lines; k++) {
      uint32_t r = (uint32_t)(((unsigned long long)(2 * k + 1) * p.H) / (2ull * p.test_lines));
      if (n == 0 || s_rows[n - 1] != r) s_rows[n++] = r;
    }
    s_nrows = n;
    s_cost[0] = s_cost[1] = 0;
  }
  __syncthreads();
  const size_t rowb = (size_t)p.W * at.s;
  uint32_t carry_i = 0, carry_p = 0;  // flat vector starts from 0
  unsigned long long cost_i = 0, cost_p = 0;  // per-warp partial sums (lane 0)
  for (uint32_t ri = 0; ri < s_nrows; ri++) {
    const uint32_t r = s_rows[ri];
    RowLoad L{p.cur[ta] + r * rowb, p.prev[ta] + r * rowb, at, pat, p.W, p.nw};
    uint32_t n = load_compact_row(L, true, true, false, eI, eP, nullptr, nullptr, s_cnt);
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
      BlockChoice c = choose_block(z, m);
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
  if (threadIdx.x == 0) p.modes[ta] = s_cost[1] < s_cost[0] ? 1u : 0u;
}

// ----------------------------------------------------------------------------
// k_encode: one CTA per row item k = (t, a, r), ticket order.
// ----------------------------------------------------------------------------
struct EncSmem {
  uint32_t* e;      // compacted residuals [W]
  uint32_t* z;      // ZigZag deltas [W]
  uint32_t* coded;  // coded mask words [nw]
  uint32_t* aux;    // literal prefix scratch [nw]
  uint32_t* bhdr;   // block headers [nbmax]
  uint32_t* boff;   // block body bytes -> offsets [nbmax]
  uint32_t* xhigh;  // per-warp exception high parts [kWarps][128]
  uint8_t* xpos;    // per-warp exception positions [kWarps][128]
  uint32_t* stage;  // staged row chunk [row_bound/4]
};

__host__ __device__ inline size_t enc_smem_bytes(uint32_t W) {
  uint32_t nw = ceil_div_u32(W, 32), nbmax = ceil_div_u32(W, kBlockN);
  size_t words = 2ull * W + 2ull * nw + 2ull * nbmax + kWarps * 128ull + kWarps * 32ull +
                 row_bound_bytes(W) / 4u;
  return words * 4u;
}

__device__ inline EncSmem enc_smem_carve(uint32_t* base, uint32_t W) {
  uint32_t nw = ceil_div_u32(W, 32), nbmax = ceil_div_u32(W, kBlockN);
  EncSmem S;
  S.e = base; base += W;
  S.z = base; base += W;
  S.coded = base; base += nw;
  S.aux = base; base += nw;
  S.bhdr = base; base += nbmax;
  S.boff = base; base += nbmax;
  S.xhigh = base; base += kWarps * 128;
  S.xpos = reinterpret_cast<uint8_t*>(base); base += kWarps * 32;
  S.stage = base;
  return S;
}

// Warp-wide funnel packing of nbits-wide values src[0..n) into dst words
// (bit stream, least significant bit first).
__device__ __forceinline__ void pack_bits(const uint32_t* src, uint32_t n, uint32_t nbits, uint32_t mask,
                                          uint32_t* dst) {
  const uint32_t nwords = (n * nbits + 31u) >> 5;
  for (uint32_t wi = lane_id(); wi < nwords; wi += 32) {
    const uint32_t bit0 = wi * 32u;
    const uint32_t i0 = bit0 / nbits;
    const uint32_t i1 = min(n - 1u, (bit0 + 31u) / nbits);
    uint32_t word = 0;
    for (uint32_t i = i0; i <= i1; i++) {
      const uint32_t v = src[i] & mask;
      const int32_t sh = (int32_t)(i * nbits) - (int32_t)bit0;
      word |= sh >= 0 ? (v << sh) : (v >> (uint32_t)(-sh));
    }
    dst[wi] = word;
  }
}

__global__ void __launch_bounds__(kThreads) k_encode(EncParams p) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_tmp[kWarps + 1];
  __shared__ uint32_t s_item, s_carry, s_ok;
  __shared__ unsigned long long s_off;

  if (threadIdx.x == 0) s_item = atomicAdd(p.ticket, 1u);
  __syncthreads();
  const uint32_t k = s_item;
  const uint32_t H = p.H, W = p.W, A = p.A, nw = p.nw;
  const uint32_t r = k % H, ta = k / H, a = ta % A, t = ta / A;
  const uint32_t sec_start = ta * H;  // first item of this attribute-scan
  const AttrDev at = p.attrs[a];
  AttrDev pat = at;
  if (t == 0) { pat.P = 1; pat.qmax = 0xffffffffu; }
  const uint32_t mode = p.modes[ta];
  const size_t rowb = (size_t)W * at.s;
  EncSmem S = enc_smem_carve(smem, W);

  // 1. quantize, mask, compaction, residual (Sec. III-B, III-C, III-D)
  RowLoad L{p.cur[ta] + r * rowb, mode ? p.prev[ta] + r * rowb : nullptr, at, pat, W, nw};
  uint8_t* st_row = (t + 1 == p.T) ? p.state_next[a] + r * rowb : nullptr;
  const uint32_t n = load_compact_row(L, mode == 0, mode == 1, mode == 1, S.e, S.e, S.coded, st_row, s_tmp);
  const uint32_t e_last = n ? S.e[n - 1] : 0u;

  // 2. delta carry: the residual preceding this row in the flat vector of the
  //    attribute-scan (Sec. III-C), by a "last valid" look-back over rows.
  if (threadIdx.x < 32) {
    uint32_t carry = 0;
    bool ok = true;
    if (r == 0) {
      if (threadIdx.x == 0) st_publish(p.st_carry + k, kStInc | (1ull << 32) | e_last);
    } else {
      if (threadIdx.x == 0) st_publish(p.st_carry + k, kStAgg | ((unsigned long long)(n ? 1 : 0) << 32) | e_last);
      ok = lookback_last(p.st_carry, k, sec_start, carry);
      if (threadIdx.x == 0)
        st_publish(p.st_carry + k, ok ? (kStInc | (1ull << 32) | (n ? e_last : carry)) : kStErr);
    }
    if (threadIdx.x == 0) { s_carry = carry; s_ok = ok; }
  }
  __syncthreads();
  if (!s_ok) {
    if (threadIdx.x == 0) {
      atomicOr(p.err, kErrTimeout);
      st_publish(p.st_bytes + k, kStErr);
    }
    return;
  }
  const uint32_t carry = s_carry;

  // 3. delta over the flat vector + ZigZag (Eq. 1)
  for (uint32_t i = threadIdx.x; i < n; i += kThreads) S.z[i] = zigzag(S.e[i] - (i ? S.e[i - 1] : carry));

  // 4. mask part: 2-bit class per word, literals in order
  const uint32_t ncls = p.ncls;
  for (uint32_t j = threadIdx.x; j < nw; j += kThreads) {
    const uint32_t c = S.coded[j];
    const uint32_t valid = (j + 1 < nw || (W & 31u) == 0) ? 0xffffffffu : ((1u << (W & 31u)) - 1u);
    S.aux[j] = (c != 0u && c != valid) ? 1u : 0u;
  }
  __syncthreads();
  const uint32_t nlit = block_excl_scan(S.aux, nw, s_tmp);
  for (uint32_t i = threadIdx.x; i < ncls; i += kThreads) {
    uint32_t word = 0;
    for (uint32_t j = 16u * i; j < min(nw, 16u * i + 16u); j++) {
      const uint32_t c = S.coded[j];
      const uint32_t valid = (j + 1 < nw || (W & 31u) == 0) ? 0xffffffffu : ((1u << (W & 31u)) - 1u);
      const uint32_t cls = c == 0u ? 0u : (c == valid ? 1u : 2u);
      word |= cls << (2u * (j - 16u * i));
    }
    S.stage[i] = word;
  }
  for (uint32_t j = threadIdx.x; j < nw; j += kThreads) {
    const uint32_t c = S.coded[j];
    const uint32_t valid = (j + 1 < nw || (W & 31u) == 0) ? 0xffffffffu : ((1u << (W & 31u)) - 1u);
    if (c != 0u && c != valid) S.stage[ncls + S.aux[j]] = c;
  }

  // 5. block widths (Sec. II): warp per block
  const uint32_t nb = ceil_div_u32(n, kBlockN);
  for (uint32_t blk = warp_id(); blk < nb; blk += kWarps) {
    const uint32_t base = blk * kBlockN, m = min(kBlockN, n - base);
    uint32_t z[4];
    load_block(S.z + base, m, z);
    BlockChoice c = choose_block(z, m);
    if (lane_id() == 0) {
      S.bhdr[blk] = c.b | (c.e << 8) | (c.hb << 16);
      S.boff[blk] = c.bytes;
    }
  }
  __syncthreads();
  const uint32_t body_total = block_excl_scan(S.boff, nb, s_tmp);
  const uint32_t head_words = ncls + nlit + nb;
  const uint32_t chunk = 4u * head_words + body_total;

  // 6. publish this row's byte aggregate, then pack while predecessors finish
  if (threadIdx.x == 0) {
    if (k == sec_start && ta == 0) st_publish(p.st_bytes + k, kStInc | chunk);
    else st_publish(p.st_bytes + k, kStAgg | chunk);
  }
  for (uint32_t blk = warp_id(); blk < nb; blk += kWarps) {
    const uint32_t base = blk * kBlockN, m = min(kBlockN, n - base);
    const uint32_t h = S.bhdr[blk];
    const uint32_t b = h & 0xffu, ex = (h >> 8) & 0xffu, hb = (h >> 16) & 0xffu;
    if (lane_id() == 0) S.stage[ncls + nlit + blk] = h;
    uint32_t* body = S.stage + head_words + S.boff[blk] / 4u;
    const uint32_t* zb = S.z + base;
    pack_bits(zb, m, b, b >= 32u ? 0xffffffffu : ((1u << b) - 1u), body);
    if (ex) {
      uint32_t* xh = S.xhigh + warp_id() * 128u;
      uint8_t* xp = S.xpos + warp_id() * 128u;
      uint32_t xi = 0;
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const uint32_t i = lane_id() + 32u * q;
        const uint32_t v = i < m ? zb[i] : 0u;
        const bool isx = i < m && bit_width(v) > b;
        const uint32_t bal = __ballot_sync(0xffffffffu, isx);
        if (isx) {
          const uint32_t slot = xi + __popc(bal & ((1u << lane_id()) - 1u));
          xp[slot] = (uint8_t)i;
          xh[slot] = v >> b;
        }
        xi += __popc(bal);
      }
      __syncwarp();
      const uint32_t low_words = (m * b + 31u) >> 5;
      const uint32_t pos_words = (ex + 3u) >> 2;
      for (uint32_t wi = lane_id(); wi < pos_words; wi += 32) {
        uint32_t word = 0;
#pragma unroll
        for (uint32_t q = 0; q < 4; q++) {
          const uint32_t idx = 4u * wi + q;
          if (idx < ex) word |= (uint32_t)xp[idx] << (8u * q);
        }
        body[low_words + wi] = word;
      }
      pack_bits(xh, ex, hb, hb >= 32u ? 0xffffffffu : ((1u << hb) - 1u), body + low_words + pos_words);
      __syncwarp();
    }
  }

  // 7. byte offset by decoupled look-back over all rows of the call
  if (threadIdx.x < 32) {
    unsigned long long excl = 0;
    bool ok = true;
    if (!(k == 0)) {
      ok = lookback_sum(p.st_bytes, k, 0, excl);
      if (threadIdx.x == 0) st_publish(p.st_bytes + k, ok ? (kStInc | (excl + chunk)) : kStErr);
    }
    if (threadIdx.x == 0) { s_off = excl; s_ok = ok; }
  }
  __syncthreads();
  if (!s_ok) {
    if (threadIdx.x == 0) atomicOr(p.err, kErrTimeout);
    return;
  }
  const unsigned long long off = p.shdr + (unsigned long long)(t + 1) * p.fhdr +
                                 (unsigned long long)(ta + 1) * 8ull * H + s_off;
  if (threadIdx.x == 0) {
    p.row_bytes[k] = chunk;
    p.row_nnz[k] = n;
    p.row_carry[k] = carry;
  }
  // 8. copy the staged chunk out (4-byte aligned)
  if (off + chunk <= p.cap) {
    uint32_t* dst = reinterpret_cast<uint32_t*>(p.out + off);
    for (uint32_t i = threadIdx.x; i < chunk / 4u; i += kThreads) dst[i] = S.stage[i];
  } else if (threadIdx.x == 0) {
    atomicOr(p.err, kErrCapacity);
  }
}

// ----------------------------------------------------------------------------
// k_finalize: one CTA per frame: row tables (end offsets + carries), frame
// header, stream header, frame offsets and the total length.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void put_u32_guarded(uint8_t* out, unsigned long long cap, unsigned long long at,
                                                uint32_t v, uint32_t* err) {
  if (at + 4 <= cap) *reinterpret_cast<uint32_t*>(out + at) = v;
  else atomicOr(err, kErrCapacity);
}

__global__ void __launch_bounds__(kThreads) k_finalize(EncParams p) {
  extern __shared__ __align__(16) uint32_t smem[];  // [H] row ends
  __shared__ uint32_t s_tmp[kWarps + 1];
  __shared__ uint32_t s_sec[kMaxAttr], s_nnz[kMaxAttr];
  const uint32_t t = blockIdx.x, H = p.H, A = p.A;
  // every status word is an inclusive prefix now
  const uint32_t first = t * A * H;
  const unsigned long long before = first ? (p.st_bytes[first - 1] & kStValMask) : 0ull;
  const unsigned long long fstart = p.shdr + (unsigned long long)t * (p.fhdr + 8ull * A * H) + before;
  unsigned long long sec_at = fstart + p.fhdr;
  for (uint32_t a = 0; a < A; a++) {
    const uint32_t ta = t * A + a;
    for (uint32_t r = threadIdx.x; r < H; r += kThreads) smem[r] = p.row_bytes[ta * H + r];
    __syncthreads();
    const uint32_t data = block_excl_scan(smem, H, s_tmp);  // smem = row starts
    uint32_t nnz = 0;
    for (uint32_t r = threadIdx.x; r < H; r += kThreads) {
      const uint32_t end = (r + 1 < H) ? smem[r + 1] : data;
      put_u32_guarded(p.out, p.cap, sec_at + 8ull * r, end, p.err);
      put_u32_guarded(p.out, p.cap, sec_at + 8ull * r + 4, p.row_carry[ta * H + r], p.err);
      nnz += p.row_nnz[ta * H + r];
    }
    nnz = warp_sum(nnz);
    if (lane_id() == 0) s_tmp[warp_id()] = nnz;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t tot = 0;
      for (int w = 0; w < kWarps; w++) tot += s_tmp[w];
      s_nnz[a] = tot;
      s_sec[a] = 8u * H + data;
    }
    __syncthreads();
    sec_at += s_sec[a];
  }
  if (threadIdx.x == 0) {
    const uint32_t frame_bytes = (uint32_t)(sec_at - fstart);
    put_u32_guarded(p.out, p.cap, fstart, frame_bytes, p.err);
    put_u32_guarded(p.out, p.cap, fstart + 4, p.frame0 + t, p.err);
    for (uint32_t a = 0; a < A; a++) {
      const unsigned long long h = fstart + 8ull + 12ull * a;
      put_u32_guarded(p.out, p.cap, h, p.modes[t * A + a], p.err);
      put_u32_guarded(p.out, p.cap, h + 4, s_sec[a], p.err);
      put_u32_guarded(p.out, p.cap, h + 8, s_nnz[a], p.err);
    }
    p.frame_off[t] = fstart;
    if (t + 1 == p.T) p.frame_off[p.T] = sec_at;
    if (t == 0 && p.shdr) {
      put_u32_guarded(p.out, p.cap, 0, 0x3159464Au, p.err);  // "JFY1"
      put_u32_guarded(p.out, p.cap, 4, 1u | (A << 16), p.err);
      put_u32_guarded(p.out, p.cap, 8, H, p.err);
      put_u32_guarded(p.out, p.cap, 12, p.W, p.err);
      for (uint32_t a = 0; a < A; a++) {
        put_u32_guarded(p.out, p.cap, 16 + 8ull * a, p.attrs[a].s | (1u << 8), p.err);
        put_u32_guarded(p.out, p.cap, 20 + 8ull * a, p.attrs[a].P, p.err);
      }
    }
  }
}

size_t enc_smem_bytes_host(uint32_t W) { return enc_smem_bytes(W); }
size_t trial_smem_bytes_host(uint32_t W) { return 8ull * W; }

int launch_encode(const EncParams& p, void* stream, void* const* ev) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t s_enc = enc_smem_bytes(p.W), s_trial = 8ull * p.W, s_fin = 4ull * p.H;
  cudaError_t e = cudaFuncSetAttribute(k_encode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_enc);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_trial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_trial);
  if (e != cudaSuccess) return (int)e;
  auto mark = [&](int i) {
    if (ev) cudaEventRecord(reinterpret_cast<cudaEvent_t>(ev[i]), st);
  };
  mark(0);
  k_trial<<<p.T * p.A, kThreads, s_trial, st>>>(p);
  mark(1);
  k_encode<<<p.n_items, kThreads, s_enc, st>>>(p);
  mark(2);
  k_finalize<<<p.T, kThreads, s_fin, st>>>(p);
  mark(3);
  return (int)cudaGetLastError();
}

}  // namespace jiffy
