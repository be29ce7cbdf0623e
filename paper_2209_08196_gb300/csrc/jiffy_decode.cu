// Jiffy decoder kernel (sm_103a): the encoder's steps run backwards
// ("straightforward reversal", Sec. III-C).
//
// One warp per row item (scan t, attribute a, row r). Warps take items in
// batches from an atomic ticket, in increasing order, so every item a warp
// may wait on was handed out earlier. Rows decode independently: the row
// table gives each row's chunk and the residual its first delta continues
// from. A P row (Sec. III-D) waits for the same row of scan t-1 (bounded spin
// on a done flag) and reads it back from the previous frame's output. There
// is no CTA-wide barrier: a warp never waits for another warp of its CTA.
//
// Per row:
//   lane 0   parses and bounds-checks the frame header and row-table entry
//   lanes    class words -> literal prefix (Sec. III-C mask code)
//   mask     a mask word (32 pixels) per lane at a time: its class code or
//            literal, XOR with the previous scan's word for P (Sec. III-D);
//            one warp scan per 32 words gives each word's first compacted
//            index
//   lanes    block headers validated and sized (Sec. II, PFOR blocks)
//   then, per 256-pixel step (lane l owning the 8 consecutive pixels
//   8l .. 8l+7 of the step), interleaved:
//   unpack   the blocks the step needs, lane l owning the 4 consecutive
//            values 4l..4l+3: a window of the body words they occupy,
//            funnel-shift extraction, exception high parts via a patch
//            buffer, inverse ZigZag (Eq. 1), into a ring of deltas
//   scatter  compacted index of each own pixel from its mask word's; the
//            lane's running sum of its deltas + a warp scan of the lanes'
//            sums from the row's carry = the residuals (inverse delta); +
//            previous pixel for P; x precision (Sec. III-A); vector stores
// The row chunk is read through L1 (bulk-prefetched into L2 at the start of
// the row); deltas pass through a small ring buffer in shared memory.
#include "jiffy_device.cuh"
#include "jiffy_kernels.h"

namespace jiffy {

namespace {

constexpr uint32_t kDecBatch = 1;  // row items per ticket unless the launch asks otherwise (1 balances the tail best)

__device__ __forceinline__ uint32_t ld_in_u32(const uint8_t* in, unsigned long long at) {
  return __ldg(reinterpret_cast<const unsigned int*>(in + at));
}

__device__ __forceinline__ uint32_t valid_word_bits(uint32_t W, uint32_t nw, uint32_t j) {
  return (j + 1 < nw || (W & 31u) == 0) ? 0xffffffffu : ((1u << (W & 31u)) - 1u);
}

__device__ __forceinline__ uint32_t literal_bits(uint32_t cwd) { return (cwd >> 1) & ~cwd & 0x55555555u; }

// Index of the segment holding global row item key: the last i with base[i] <= key.
__device__ __forceinline__ uint32_t find_seg(const uint32_t* base, uint32_t n, uint32_t key) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(base + mid) <= key) lo = mid;
    else hi = mid;
  }
  return lo;
}

}  // namespace

// Per-warp shared memory (byte offsets): a ring of 512 deltas (unpacked
// ahead of the scatter), a 128-word exception patch buffer, the row's block
// descriptors, zero mask words (1 = zero sample), each mask word's first
// compacted index and literal mask words.
constexpr uint32_t kRing = 512;

struct DecWarpLayout {
  uint32_t ring, patch, desc, mw, wbase, lits, bytes;
};

__host__ __device__ inline DecWarpLayout dec_warp_layout(uint32_t W) {
  DecWarpLayout L;
  L.ring = 0;
  L.patch = L.ring + 4u * kRing;
  L.desc = L.patch + 4u * kBlockN;
  L.mw = L.desc + ((8u * ceil_div_u32(W, kBlockN) + 15u) & ~15u);
  L.wbase = L.mw + ((4u * ceil_div_u32(W, 32u) + 15u) & ~15u);
  L.lits = L.wbase + ((4u * ceil_div_u32(W, 32u) + 15u) & ~15u);
  L.bytes = (L.lits + 4u * ceil_div_u32(W, 32u) + 15u) & ~15u;
  return L;
}

// One row item, samples of S bytes (compile-time, so each warp runs one
// compact path).
// The frame- and section-level part of a row's parse, shared by the rows of
// one section (a warp's consecutive items are mostly of one section).
struct SecCache {
  unsigned long long key;       // (1 + segment) << 32 | section in the segment; 0 = empty
  uint32_t mode, bad;           // the section's mode; 1 = malformed frame header
  uint32_t data_len;            // bytes of the section's row chunks
  uint32_t next_p;              // the call's next frame codes this attribute as P (its rows read this frame's masks)
  uint32_t zpart;               // bytes of the Zstandard mask part after the row table (0 without it)
  unsigned long long sec;       // byte offset of the section (its row table)
};

// STAGED: the segments may have stage switches, or the test hook may be set
// (else both are read as 0).
template <bool STAGED>
__device__ __forceinline__ void decode_item(const DecParams& p, const uint32_t k, uint32_t* ring,
                                            uint32_t* patch, uint2* desc, uint32_t* mw, uint32_t* wbase,
                                            uint32_t* lits, SecCache& sc) {
  const uint32_t si = find_seg(p.seg_item_base, p.n_seg, k);
  const DecSeg& sg = p.seg[si];
  const uint32_t lane = lane_id();
  const uint32_t H = sg.H, W = sg.W, A = sg.A, nw = sg.nw, ncls = sg.ncls;
  const uint32_t stages = STAGED ? sg.stages : 0u;
  const uint32_t niter = ceil_div_u32(W, 256u);
  const uint32_t kl = k - sg.item_base;  // item within the segment
  // items of a segment are numbered attribute-major, (a, t, r): resident warps
  // decode one attribute's rows at a time, and a P row's dependency, the same
  // row of the previous scan, is the item H before it
  const uint32_t r = kl % H, at_idx = kl / H, a = at_idx / sg.T, t = at_idx % sg.T;
  const uint32_t ta = t * A + a;
  const AttrDev at = sg.attrs[a];
  const uint32_t S = at.s;
  const size_t rowb = (size_t)W * S;

  // ---- frame header (once per section); status 1 = malformed, 2 = timed out
  const unsigned long long key = ((unsigned long long)(si + 1u) << 32) | ta;
  if (sc.key != key) {
    const unsigned long long f0 = sg.off[t], f1 = sg.off[t + 1];
    // offsets in range before any read: 4-byte aligned, a whole frame header,
    // inside `in`, after the stream header for a stream's first frame
    const unsigned long long first = (t == 0 && sg.check_shdr) ? 16ull + 8ull * A : 0ull;
    bool hbad = f0 < first || (f0 & 3ull) || f1 < f0 + sg.fhdr || f1 > sg.in_len || ((f1 - f0) >> 32);
    unsigned long long sb_before = 0, sb_total = 0;
    uint32_t my_mode = 0, my_sb = 0;
    for (uint32_t aa = lane; aa < A && !hbad; aa += 32) {
      const uint32_t m = ld_in_u32(sg.in, f0 + 8ull + 12ull * aa);
      const uint32_t sb = ld_in_u32(sg.in, f0 + 12ull + 12ull * aa);
      if ((m & 0xffffff00u) || (m & 0xffu) > 1u || sb < 8u * H || (sb & 3u)) hbad = true;
      sb_total += sb;
      if (aa < a) sb_before += sb;
      if (aa == a) { my_mode = m & 0xffu; my_sb = sb; }
    }
    hbad = __any_sync(0xffffffffu, hbad);
    for (int o = 16; o > 0; o >>= 1) {
      sb_total += __shfl_xor_sync(0xffffffffu, sb_total, o);
      sb_before += __shfl_xor_sync(0xffffffffu, sb_before, o);
    }
    sc.mode = __shfl_sync(0xffffffffu, my_mode, a & 31u);
    my_sb = __shfl_sync(0xffffffffu, my_sb, a & 31u);
    if (!hbad) {
      const uint32_t frame_bytes = ld_in_u32(sg.in, f0);
      const uint32_t scan = ld_in_u32(sg.in, f0 + 4);
      if (frame_bytes != f1 - f0 || scan != sg.frame0 + t || sb_total + sg.fhdr != frame_bytes) hbad = true;
    }
    if (sc.mode == 1u && sg.frame0 + t == 0) hbad = true;
    sc.next_p = 1u;  // unless the next frame's header says I (or there is none)
    if (t + 1 == sg.T) {
      sc.next_p = 0u;
    } else if (!hbad) {
      const unsigned long long g1 = sg.off[t + 2];
      if (g1 >= f1 + sg.fhdr && g1 <= sg.in_len && !(g1 & 3ull)) sc.next_p = ld_in_u32(sg.in, f1 + 8ull + 12ull * a) == 1u;
    }
    sc.zpart = 0;
    if (STAGED && (stages & kStageZstdMask) && !hbad) {  // index + frame + padding before the row chunks
      const unsigned long long idx = 4ull + 4ull * sg.zm_nblk;
      if (my_sb - 8ull * H < idx) {
        hbad = true;
      } else {
        const uint32_t F = ld_in_u32(sg.in, f0 + sg.fhdr + sb_before + 8ull * H);
        const unsigned long long part = (idx + F + 3ull) & ~3ull;
        if (part > my_sb - 8ull * H) hbad = true;
        else sc.zpart = (uint32_t)part;
      }
    }
    sc.bad = hbad ? 1u : 0u;
    sc.sec = f0 + sg.fhdr + sb_before;
    sc.data_len = my_sb - 8u * H - sc.zpart;
    sc.key = key;
  }
  const uint32_t mode = sc.mode;
  uint32_t status = 0, clen = 0, carry = 0;
  unsigned long long chunk_off = 0;
  if (lane == 0) {
    bool bad = sc.bad != 0;
    if (!bad) {  // the row-table entry
      const unsigned long long sec = sc.sec;
      const uint32_t data_len = sc.data_len;
      const uint32_t end = ld_in_u32(sg.in, sec + 8ull * r);
      carry = ld_in_u32(sg.in, sec + 8ull * r + 4);
      const uint32_t start = r ? ld_in_u32(sg.in, sec + 8ull * (r - 1)) : 0u;
      if (start > end || end > data_len || (r + 1 == H && end != data_len) || ((start | end) & 3u) ||
          end - start > row_bound_bytes(W) || end - start < 4u * ncls)
        bad = true;
      clen = end - start;
      chunk_off = sec + 8ull * H + sc.zpart + start;
    }
    if (kl == 0 && sg.check_shdr && !bad) {  // stream header: shape, dtypes, precisions
      if (ld_in_u32(sg.in, 0) != 0x3159464Au || ld_in_u32(sg.in, 4) != (1u | (A << 16)) ||
          ld_in_u32(sg.in, 8) != H || ld_in_u32(sg.in, 12) != W)
        bad = true;
      for (uint32_t aa = 0; aa < A && !bad; aa++) {
        if (ld_in_u32(sg.in, 16 + 8ull * aa) != attr_header_word(sg.attrs[aa].s, stages) ||
            ld_in_u32(sg.in, 20 + 8ull * aa) != sg.attrs[aa].P)
          bad = true;
      }
    }
    status = bad ? 1u : 0u;
    // a P row waits for the same row of the previous frame (bounded)
    if (!bad && mode == 1u && t > 0) {
      const volatile uint32_t* flag = p.done + (k - H);
      if (!*flag) {
        const unsigned long long t0 = global_timer_ns();
        uint32_t ns = 32;
        while (!*flag) {
          __nanosleep(ns);
          if (ns < 1024) ns <<= 1;
          if (global_timer_ns() - t0 > kSpinLimitNs) {
            atomicOr(sg.err, kErrTimeout);
            status = 2u;
            break;
          }
        }
      }
      __threadfence();
    }
  }
  status = __shfl_sync(0xffffffffu, status, 0);
  clen = __shfl_sync(0xffffffffu, clen, 0);
  carry = __shfl_sync(0xffffffffu, carry, 0);
  chunk_off = __shfl_sync(0xffffffffu, chunk_off, 0);
  if (mode == 1u) __threadfence();  // every lane orders its reads of the previous row after the flag

  bool bad = status != 0;
  // ---- the chunk is read through L1: fetched into L2 in one bulk request,
  //      its lines requested for L1 by the lanes (one round)
  const uint32_t* chunk = reinterpret_cast<const uint32_t*>(sg.in + chunk_off);
  if (!bad) {
    if (lane == 0) {
      const uintptr_t c0 = reinterpret_cast<uintptr_t>(chunk), c1 = c0 + clen;
      const uintptr_t a0 = (c0 + 15u) & ~uintptr_t(15), a1 = c1 & ~uintptr_t(15);
      if (a1 > a0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"((uint32_t)(a1 - a0)) : "memory");
    }
    prefetch_l1(chunk, clen);
  }
  // ---- class words: class 3 and bits past nw are invalid; literal prefix
  uint32_t cw = 0, lit = 0;
  if (!bad && lane < ncls) {
    cw = chunk[lane];
    uint32_t used = 0xffffffffu;
    const uint32_t nslots = min(16u, nw - 16u * lane);
    if (nslots < 16u) used = (1u << (2u * nslots)) - 1u;
    lit = __popc(literal_bits(cw));
    if (((cw >> 1) & cw & 0x55555555u) || (cw & ~used)) bad = true;
  }
  const uint32_t litincl = warp_incl_scan(lit);
  const uint32_t litpre = litincl - lit;
  const uint32_t nlit = __shfl_sync(0xffffffffu, litincl, 31);
  bad = __any_sync(0xffffffffu, bad) || 4u * (ncls + nlit) > clen;
  if (!bad) {  // the row's literal mask words, one coalesced read into shared memory
    for (uint32_t i = lane; i < nlit; i += 32u) lits[i] = chunk[ncls + i];
    __syncwarp();
  }
  {  // a literal last mask word may not set bits past W
    const uint32_t j = nw - 1;
    const uint32_t cwj = __shfl_sync(0xffffffffu, cw, (j >> 4) & 31u);
    const uint32_t lpj = __shfl_sync(0xffffffffu, litpre, (j >> 4) & 31u);
    if (!bad && (W & 31u) && ((cwj >> (2u * (j & 15u))) & 3u) == 2u) {
      const uint32_t li = lpj + __popc(literal_bits(cwj) & ((1u << (2u * (j & 15u))) - 1u));
      if (lits[li] & ~valid_word_bits(W, nw, j)) bad = true;
    }
  }

  uint8_t* orow = sg.outp[ta] + r * rowb;
  uint8_t* srow = (t + 1 == sg.T) ? sg.state_next[a] + r * rowb : nullptr;
  const uint8_t* prow = mode == 1u ? (t > 0 ? sg.outp[(t - 1) * A + a] : sg.state[a]) + r * rowb : nullptr;
  const bool vec_prev = prow && vec_ok(prow, S);
  if (!bad && prow && lane == 0) {  // the previous scan's row, for the P sums of the scatter
    const uintptr_t c0 = reinterpret_cast<uintptr_t>(prow), c1 = c0 + rowb;
    const uintptr_t a0 = (c0 + 15u) & ~uintptr_t(15), a1 = c1 & ~uintptr_t(15);
    if (a1 > a0)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"((uint32_t)(a1 - a0)) : "memory");
  }
  const bool vec_out = vec_ok(orow, S) && (!srow || vec_ok(srow, S));

  // ---- zero mask, a word (32 pixels) per lane at a time: class code or
  //      literal (Sec. III-C); for P (Sec. III-D) the XOR with the previous
  //      scan's mask is undone, that mask taken from the words the previous
  //      frame's row wrote in this call, else from its samples. Without the
  //      mask stage (no class words) every sample is coded. One warp scan per
  //      32 words gives each word's first compacted index.
  uint32_t n = 0;
  bool zbad = false;
  if (!bad) {
    const bool xor_prev = mode == 1u && !(stages & kStageNoMask);
    const uint32_t* pmask = (xor_prev && t > 0) ? p.masks + sg.mask_base + (size_t)(kl - H) * nw : nullptr;
    uint32_t* omask = (sc.next_p && !(stages & kStageNoMask)) ? p.masks + sg.mask_base + (size_t)kl * nw : nullptr;
    const bool prev_samples = xor_prev && !pmask;
    // the row's coded mask bytes from the section's Zstandard frame (decoded
    // by k_zstd_dec); a bit past W is malformed
    const uint8_t* zrow = (STAGED && (stages & kStageZstdMask))
                              ? p.zdec + sg.zm_base + (size_t)ta * sg.zm_stride + (size_t)r * sg.zm_rb
                              : nullptr;
    const uint32_t zrb = sg.zm_rb;
    if (prev_samples) {  // the previous scan's zero bits, 8 pixels per lane per step, into mw
      uint8_t* pb = reinterpret_cast<uint8_t*>(mw);
      for (uint32_t it = 0; it < niter; it++) {
        const uint32_t x0 = 256u * it + 8u * lane;
        if (x0 < W) {
          const uint32_t nv = min(8u, W - x0);
          uint32_t pv[8];
          load8<true>(prow, S, x0, nv, vec_prev, pv);
          uint32_t pm = 0;
#pragma unroll
          for (int i = 0; i < 8; i++) pm |= (uint32_t)(pv[i] == 0u) << i;
          pb[x0 >> 3] = (uint8_t)pm;
        }
      }
      __syncwarp();
    }
    for (uint32_t j0 = 0; j0 < nw; j0 += 32u) {
      const uint32_t j = j0 + lane;
      const uint32_t cwj = __shfl_sync(0xffffffffu, cw, (j >> 4) & 31u);
      const uint32_t lpj = __shfl_sync(0xffffffffu, litpre, (j >> 4) & 31u);
      uint32_t kept = 0;
      if (j < nw) {
        const uint32_t valid = valid_word_bits(W, nw, j);
        uint32_t X = 0;
        if (ncls) {
          const uint32_t sl = 2u * (j & 15u), cls = (cwj >> sl) & 3u;
          if (cls == 1u) X = valid;
          else if (cls == 2u) X = lits[lpj + __popc(literal_bits(cwj) & ((1u << sl) - 1u))];
          if (pmask) X ^= __ldcg(pmask + j);
          else if (prev_samples) X ^= mw[j];  // bits past W are cleared below
          X &= valid;
          if (omask) omask[j] = X;
        } else if (zrow) {
          if ((zrb & 3u) == 0u) {
            X = __ldcg(reinterpret_cast<const uint32_t*>(zrow) + j);
          } else {
            for (uint32_t q = 0; q < 4u && 4u * j + q < zrb; q++) X |= (uint32_t)__ldcg(zrow + 4u * j + q) << (8u * q);
          }
          zbad |= (X & ~valid) != 0u;
          if (pmask) X ^= __ldcg(pmask + j);
          else if (prev_samples) X ^= mw[j];
          X &= valid;
          if (omask) omask[j] = X;
        }
        mw[j] = X;
        kept = __popc(~X & valid);
      }
      uint32_t tot;
      const uint32_t ex = warp_excl_scan(kept, tot);
      if (j < nw) wbase[j] = n + ex;
      n += tot;
    }
  }
  bad = bad || __any_sync(0xffffffffu, zbad);
  __syncwarp();
  const uint32_t nb = ceil_div_u32(n, kBlockN);

  // ---- block headers (lane l: blocks 4l .. 4l+3): validate, size the
  //      bodies, check they fill the chunk exactly; descriptors {body word,
  //      b | e << 8 | hb << 16 | m << 24} for the unpack
  const uint32_t hdr0 = ncls + nlit;
  if (!bad && 4u * (hdr0 + nb) > clen) bad = true;
  {
    uint32_t sz[4], hv[4], mysum = 0;
    bool lbad = false;
#pragma unroll
    for (uint32_t q = 0; q < 4; q++) {
      const uint32_t blk = 4u * lane + q;
      sz[q] = 0;
      hv[q] = 0;
      if (!bad && blk < nb) {
        const uint32_t h = chunk[hdr0 + blk];
        const uint32_t b = h & 0xffu, e = (h >> 8) & 0xffu, hb = (h >> 16) & 0xffu;
        const uint32_t m = min(kBlockN, n - blk * kBlockN);
        if ((h >> 24) || b > 32u || hb > 32u || b + hb > 32u || e > m || ((e == 0u) != (hb == 0u))) lbad = true;
        sz[q] = block_body_bytes(m, min(b, 32u), min(e, m), min(b + hb, 32u)) / 4u;
        hv[q] = (h & 0x00ffffffu) | (m << 24);
        mysum += sz[q];
      }
    }
    bad = __any_sync(0xffffffffu, bad || lbad);
    uint32_t total;
    uint32_t o = hdr0 + nb + warp_excl_scan(mysum, total);
    if (!bad && 4u * (hdr0 + nb + total) != clen) bad = true;
#pragma unroll
    for (uint32_t q = 0; q < 4; q++) {
      const uint32_t blk = 4u * lane + q;
      if (blk < nb) desc[blk] = make_uint2(o, hv[q]);
      o += sz[q];
    }
  }
  __syncwarp();

  // ---- unpack, block by block (lane l: the 4 consecutive values 4l..4l+3,
  //      a register window of the body words they occupy, funnel-shift
  //      extraction; exceptions' high parts through the patch buffer;
  //      inverse ZigZag, Eq. 1) into a ring of deltas, interleaved with the
  //      scatter by position: per 256-pixel step a warp scan of the lanes'
  //      delta sums from the running residual is the inverse delta; + the
  //      previous pixel for P, x precision (Sec. III-A)
  if (!bad) {
    const uint32_t Pq = at.P;
    const bool no_delta = (stages & kStageNoDelta) != 0u, no_zz = (stages & kStageNoZigzag) != 0u;
    const uint32_t last_word = clen / 4u - 1u;
    uint32_t erun = carry, blk = 0, unpacked = 0;
    bool xbad = false;
    for (uint32_t it = 0; it < niter && !xbad; it++) {
      const uint32_t x0 = 256u * it + 8u * lane;
      const uint32_t nv = x0 < W ? min(8u, W - x0) : 0u;
      // own pixels' mask byte (pixels past W count as zero samples) and the
      // compacted index of the first; the step ends at the next word group
      const uint32_t X = nv ? mw[x0 >> 5] : 0xffffffffu;
      const uint32_t nzm = ~(X >> (x0 & 31u)) & ((1u << nv) - 1u);
      uint32_t kk = nv ? wbase[x0 >> 5] + __popc(~X & ((1u << (x0 & 31u)) - 1u)) : n;
      const uint32_t kend = 8u * it + 8u < nw ? wbase[8u * it + 8u] : n;
      while (unpacked < kend) {
        const uint2 dsc = desc[blk];
        const uint32_t b = dsc.y & 0xffu, e = (dsc.y >> 8) & 0xffu, hb = (dsc.y >> 16) & 0xffu;
        const uint32_t bm = b >= 32u ? 0xffffffffu : ((1u << b) - 1u);
        const uint32_t bit0 = 4u * lane * b, sh = bit0 & 31u;
        const uint32_t w0 = dsc.x + (bit0 >> 5);
        uint32_t v0 = 0, v1 = 0, v2 = 0, v3 = 0;
        if (b) {
          const uint32_t W0 = chunk[min(w0, last_word)], W1 = chunk[min(w0 + 1u, last_word)],
                         W2 = chunk[min(w0 + 2u, last_word)];
          const uint32_t A = __funnelshift_r(W0, W1, sh), B = __funnelshift_r(W1, W2, sh);
          if (b <= 8u) {
            v0 = A; v1 = A >> b; v2 = A >> (2u * b); v3 = A >> (3u * b);
          } else if (b <= 16u) {
            const unsigned long long Y = ((unsigned long long)B << 32) | A;
            v0 = A; v1 = __funnelshift_r(A, B, b); v2 = __funnelshift_rc(A, B, 2u * b);
            v3 = (uint32_t)(Y >> (3u * b));
          } else {
            const uint32_t W3 = chunk[min(w0 + 3u, last_word)], W4 = chunk[min(w0 + 4u, last_word)];
            const uint32_t C = __funnelshift_r(W2, W3, sh), D = __funnelshift_r(W3, W4, sh);
            v0 = A; v1 = __funnelshift_rc(A, B, b); v2 = __funnelshift_rc(B, C, 2u * b - 32u);
            v3 = 3u * b <= 64u ? __funnelshift_rc(B, C, 3u * b - 32u) : __funnelshift_rc(C, D, 3u * b - 64u);
          }
          v0 &= bm; v1 &= bm; v2 &= bm; v3 &= bm;
        }
        if (e) {  // exceptions: positions (ascending, < m), high parts of hb bits
          const uint32_t m = dsc.y >> 24;
          reinterpret_cast<uint4*>(patch)[lane] = make_uint4(0u, 0u, 0u, 0u);
          __syncwarp();
          const uint32_t lw = dsc.x + ((m * b + 31u) >> 5);
          const uint8_t* pos = reinterpret_cast<const uint8_t*>(chunk + lw);
          const uint32_t hw = lw + ((e + 3u) >> 2);
          const uint32_t hmask = hb >= 32u ? 0xffffffffu : ((1u << hb) - 1u);
          for (uint32_t jx = lane; jx < e; jx += 32) {
            const uint32_t ps = pos[jx];
            if (ps >= m || (jx > 0 && ps <= pos[jx - 1])) {
              xbad = true;
            } else {
              const uint32_t bit = jx * hb, wi = hw + (bit >> 5);
              const uint32_t lo = chunk[min(wi, last_word)], hi = chunk[min(wi + 1u, last_word)];
              patch[ps] = (__funnelshift_r(lo, hi, bit & 31u) & hmask) << b;
            }
          }
          __syncwarp();
          const uint4 pt = reinterpret_cast<const uint4*>(patch)[lane];
          v0 |= pt.x; v1 |= pt.y; v2 |= pt.z; v3 |= pt.w;
        }
        if (!no_zz) {
          v0 = unzigzag(v0); v1 = unzigzag(v1); v2 = unzigzag(v2); v3 = unzigzag(v3);
        }
        reinterpret_cast<uint4*>(ring)[((128u * blk + 4u * lane) & (kRing - 1u)) >> 2] = make_uint4(v0, v1, v2, v3);
        unpacked += min(kBlockN, n - 128u * blk);
        blk++;
      }
      xbad = __any_sync(0xffffffffu, xbad);
      __syncwarp();
      if (xbad) break;
      uint32_t pv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      if (mode == 1u && nv) load8<true>(prow, S, x0, nv, vec_prev, pv);
      // residuals: running sum of the deltas from the step's start (without
      // the delta stage the values are the residuals)
      uint32_t d[8], ebase = 0;
      if (!no_delta) {
        uint32_t lsum = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const bool nzb = (nzm >> i) & 1u;
          d[i] = nzb ? ring[kk & (kRing - 1u)] : 0u;
          kk += nzb ? 1u : 0u;
          lsum += d[i];
          d[i] = lsum;
        }
        uint32_t stot;
        ebase = erun + warp_excl_scan(lsum, stot);
        erun += stot;
      } else {
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const bool nzb = (nzm >> i) & 1u;
          d[i] = nzb ? ring[kk & (kRing - 1u)] : 0u;
          kk += nzb ? 1u : 0u;
        }
      }
      uint32_t out[8];
#pragma unroll
      for (int i = 0; i < 8; i++) out[i] = ((nzm >> i) & 1u) ? (ebase + d[i]) * Pq + pv[i] : 0u;
      if (nv) {
        store8(orow, S, x0, nv, vec_out, out);
        if (srow) store8(srow, S, x0, nv, vec_out, out);
      }
      __syncwarp();
    }
    bad = xbad;
  }
  if (lane == 0 && bad && status != 2u) atomicOr(sg.err, kErrCorrupt);
  __threadfence();
  __syncwarp();
  if (lane == 0 && (!STAGED || k + 1u != p.withhold)) atomicExch(p.done + k, 1u);
}

template <int WPC, bool STAGED>
__global__ void __launch_bounds__(WPC * 32) k_decode(DecParams p) {
  extern __shared__ __align__(16) uint32_t smem[];
  const uint32_t lane = lane_id();
  const DecWarpLayout lay = dec_warp_layout(p.max_W);
  uint8_t* wb = reinterpret_cast<uint8_t*>(smem) + warp_id() * lay.bytes;
  uint32_t* ring = reinterpret_cast<uint32_t*>(wb + lay.ring);
  uint32_t* patch = reinterpret_cast<uint32_t*>(wb + lay.patch);
  uint2* desc = reinterpret_cast<uint2*>(wb + lay.desc);
  uint32_t* mw = reinterpret_cast<uint32_t*>(wb + lay.mw);
  uint32_t* wbase = reinterpret_cast<uint32_t*>(wb + lay.wbase);
  uint32_t* lits = reinterpret_cast<uint32_t*>(wb + lay.lits);
  SecCache sc{0ull, 0u, 0u, 0u, 0u, 0ull};
  while (true) {
    uint32_t kb = 0;
    if (lane == 0) kb = atomicAdd(p.ticket, p.items_per_ticket);
    kb = __shfl_sync(0xffffffffu, kb, 0);
    if (kb >= p.n_items) break;
    const uint32_t kend = min(kb + p.items_per_ticket, p.n_items);
    for (uint32_t k = kb; k < kend; k++) {
      decode_item<STAGED>(p, k, ring, patch, desc, mw, wbase, lits, sc);
    }
  }
}

size_t dec_smem_bytes_host(uint32_t W) { return dec_warp_layout(W).bytes; }

constexpr size_t kDecSmemAuto = 48 * 1024;  // per CTA when picking warps per CTA by itself
constexpr size_t kDecSmemMax = 227 * 1024;

template <int WPC>
static cudaError_t dec_occupancy(size_t smem, bool staged, int* per_sm) {
  auto f = staged ? k_decode<WPC, true> : k_decode<WPC, false>;
  cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, f, WPC * 32, smem);
}

int decode_rows_launch(const DecParams& p, RowsLaunch* out) {
  const DecWarpLayout L = dec_warp_layout(p.max_W);
  if ((L.ring | L.patch | L.desc | L.mw | L.wbase | L.lits | L.bytes) & 15u) return (int)cudaErrorInvalidValue;  // 16-byte aligned regions
  uint32_t wpc = p.wpc;
  if ((wpc != 1 && wpc != 2 && wpc != 4 && wpc != 8) || wpc * L.bytes > kDecSmemMax) wpc = 0;
  if (!wpc) wpc = 4 * L.bytes <= kDecSmemAuto ? 4u : (2 * L.bytes <= kDecSmemAuto ? 2u : 1u);
  const size_t smem = (size_t)wpc * L.bytes;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    const bool sd = p.staged != 0;
    if (wpc == 8) e = dec_occupancy<8>(smem, sd, &per_sm);
    else if (wpc == 4) e = dec_occupancy<4>(smem, sd, &per_sm);
    else if (wpc == 2) e = dec_occupancy<2>(smem, sd, &per_sm);
    else e = dec_occupancy<1>(smem, sd, &per_sm);
  }
  if (e != cudaSuccess) return (int)e;
  uint32_t ctas = (uint32_t)max(per_sm, 1);
  if (p.ctas_per_sm) ctas = min(ctas, p.ctas_per_sm);
  const uint32_t ipt = p.items_per_ticket ? min(p.items_per_ticket, 64u) : kDecBatch;
  // enough warps to fill the GPU; warps beyond the work find the ticket spent
  const uint32_t want = ceil_div_u32(p.n_items, ipt * wpc);
  out->wpc = wpc;
  out->ctas_per_sm = ctas;
  out->items_per_ticket = ipt;
  out->grid = max(1u, min(want, ctas * (uint32_t)sms));
  return 0;
}

int launch_decode(const DecParams& p0, void* stream, void* const* ev) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  RowsLaunch rl{};
  int rc = decode_rows_launch(p0, &rl);
  if (rc != 0) return rc;
  DecParams p = p0;
  p.items_per_ticket = rl.items_per_ticket;
  const size_t smem = (size_t)rl.wpc * dec_warp_layout(p.max_W).bytes;
  if (ev) record_event(ev[0], st);
  rc = launch_zstd_decode(p, st);
  if (rc != 0) return rc;
  if (p.staged) {
    if (rl.wpc == 8) k_decode<8, true><<<rl.grid, 8 * 32, smem, st>>>(p);
    else if (rl.wpc == 4) k_decode<4, true><<<rl.grid, 4 * 32, smem, st>>>(p);
    else if (rl.wpc == 2) k_decode<2, true><<<rl.grid, 2 * 32, smem, st>>>(p);
    else k_decode<1, true><<<rl.grid, 32, smem, st>>>(p);
  } else {
    if (rl.wpc == 8) k_decode<8, false><<<rl.grid, 8 * 32, smem, st>>>(p);
    else if (rl.wpc == 4) k_decode<4, false><<<rl.grid, 4 * 32, smem, st>>>(p);
    else if (rl.wpc == 2) k_decode<2, false><<<rl.grid, 2 * 32, smem, st>>>(p);
    else k_decode<1, false><<<rl.grid, 32, smem, st>>>(p);
  }
  if (ev) record_event(ev[1], st);
  return (int)cudaGetLastError();
}

}  // namespace jiffy
