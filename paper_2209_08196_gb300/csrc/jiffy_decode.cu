// Jiffy decoder kernel (sm_103a): the encoder's steps run backwards
// ("straightforward reversal", Sec. III-C).
//
// One CTA per row item (scan t, attribute a, row r), taken in ticket order so
// that every item it may wait on started earlier. Rows decode independently:
// the row table gives each row's chunk and the residual its first delta
// continues from. A P row (Sec. III-D) waits for the same row of scan t-1
// (bounded spin on a done flag) and reads it back from the previous frame's
// output. Per row: bounds-checked header and row-table parse -> chunk staged
// in shared memory -> mask words from class codes and literals, XOR with the
// previous scan's mask for P -> nonzero counts and positions (popc) -> block
// headers -> unpack low bits and patch exceptions (Sec. II) -> inverse
// ZigZag (Eq. 1) -> inclusive prefix sum from the carry (inverse delta,
// mod 2^32) -> + previous value for P -> scatter into the dense row and scale
// by the precision (Sec. III-A).
#include "jiffy_device.cuh"
#include "jiffy_kernels.h"

namespace jiffy {

struct DecSmem {
  uint32_t* stage;  // row chunk words [row_bound/4]
  uint32_t* z;      // values [W]
  uint32_t* vprev;  // previous scan's row [W]
  uint32_t* mask;   // mask words [nw]
  uint32_t* base;   // per word nonzero count -> exclusive base [nw]
  uint32_t* boff;   // per block body bytes -> offsets [nbmax]
};

__host__ __device__ inline size_t dec_smem_bytes(uint32_t W) {
  uint32_t nw = ceil_div_u32(W, 32), nbmax = ceil_div_u32(W, kBlockN);
  return 4ull * (row_bound_bytes(W) / 4u + 2ull * W + 2ull * nw + nbmax);
}

__device__ inline DecSmem dec_smem_carve(uint32_t* p, uint32_t W) {
  uint32_t nw = ceil_div_u32(W, 32), nbmax = ceil_div_u32(W, kBlockN);
  DecSmem S;
  S.stage = p; p += row_bound_bytes(W) / 4u;
  S.z = p; p += W;
  S.vprev = p; p += W;
  S.mask = p; p += nw;
  S.base = p; p += nw;
  S.boff = p; p += nbmax;
  (void)p;
  return S;
}

__device__ __forceinline__ uint32_t ld_in_u32(const uint8_t* in, unsigned long long at) {
  return *reinterpret_cast<const uint32_t*>(in + at);
}

// Bits [bitpos, bitpos + nbits) of a least-significant-bit-first word stream.
__device__ __forceinline__ uint32_t extract_bits(const uint32_t* w, uint32_t bitpos, uint32_t nbits) {
  if (nbits == 0) return 0u;
  const uint32_t i = bitpos >> 5, sh = bitpos & 31u;
  uint32_t v = w[i] >> sh;
  if (sh + nbits > 32u) v |= w[i + 1] << (32u - sh);
  return nbits >= 32u ? v : (v & ((1u << nbits) - 1u));
}

__global__ void __launch_bounds__(kThreads) k_decode(DecParams p) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint32_t s_tmp[kWarps + 1];
  __shared__ uint32_t s_item, s_bad, s_mode, s_clen, s_carry, s_nlit, s_litpre[33];
  __shared__ unsigned long long s_chunk;

  if (threadIdx.x == 0) {
    s_item = atomicAdd(p.ticket, 1u);
    s_bad = 0;
  }
  __syncthreads();
  const uint32_t k = s_item;
  const uint32_t H = p.H, W = p.W, A = p.A, nw = p.nw, ncls = p.ncls;
  const uint32_t r = k % H, ta = k / H, a = ta % A, t = ta / A;
  const AttrDev at = p.attrs[a];
  const size_t rowb = (size_t)W * at.s;
  DecSmem S = dec_smem_carve(smem, W);

  // ---- frame header and row table (warp 0), every field bounds-checked
  if (threadIdx.x < 32) {
    const uint32_t lane = lane_id();
    const unsigned long long f0 = p.off[t], f1 = p.off[t + 1];
    bool bad = false;
    // per-attribute header fields, lane l covers attributes l and l + 32
    unsigned long long sb_before = 0, sb_total = 0;
    uint32_t my_mode = 0, my_sb = 0;
    for (uint32_t aa = lane; aa < A; aa += 32) {
      const uint32_t m = ld_in_u32(p.in, f0 + 8ull + 12ull * aa);
      const uint32_t sb = ld_in_u32(p.in, f0 + 12ull + 12ull * aa);
      if ((m & 0xffffff00u) || (m & 0xffu) > 1u) bad = true;
      sb_total += sb;  // sections are small: no wrap for valid frames; checked below
      if (aa < a) sb_before += sb;
      if (aa == a) { my_mode = m & 0xffu; my_sb = sb; }
      if (sb < 8u * H || (sb & 3u)) bad = true;
    }
    bad = __any_sync(0xffffffffu, bad);
    unsigned long long tot = sb_total;
    for (int o = 16; o > 0; o >>= 1) {
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
      sb_before += __shfl_xor_sync(0xffffffffu, sb_before, o);
    }
    my_mode = __shfl_sync(0xffffffffu, my_mode, a & 31u);
    my_sb = __shfl_sync(0xffffffffu, my_sb, a & 31u);
    if (lane == 0) {
      const uint32_t frame_bytes = ld_in_u32(p.in, f0);
      const uint32_t scan = ld_in_u32(p.in, f0 + 4);
      if (frame_bytes != f1 - f0 || scan != p.frame0 + t || tot + p.fhdr != frame_bytes) bad = true;
      if (my_mode == 1u && p.frame0 + t == 0) bad = true;
      uint32_t clen = 0, carry = 0;
      unsigned long long chunk = 0;
      if (!bad) {
        const unsigned long long sec = f0 + p.fhdr + sb_before;
        const uint32_t data_len = my_sb - 8u * H;
        const uint32_t end = ld_in_u32(p.in, sec + 8ull * r);
        carry = ld_in_u32(p.in, sec + 8ull * r + 4);
        const uint32_t start = r ? ld_in_u32(p.in, sec + 8ull * (r - 1)) : 0u;
        if (start > end || end > data_len || (r + 1 == H && end != data_len) || ((start | end) & 3u) ||
            end - start > row_bound_bytes(W) || end - start < 4u * ncls)
          bad = true;
        clen = end - start;
        chunk = sec + 8ull * H + start;
      }
      if (k == 0 && p.check_shdr && !bad) {  // stream header: shape, dtypes, precisions
        if (ld_in_u32(p.in, 0) != 0x3159464Au || ld_in_u32(p.in, 4) != (1u | (A << 16)) ||
            ld_in_u32(p.in, 8) != H || ld_in_u32(p.in, 12) != W)
          bad = true;
        for (uint32_t aa = 0; aa < A && !bad; aa++) {
          if (ld_in_u32(p.in, 16 + 8ull * aa) != (p.attrs[aa].s | (1u << 8)) ||
              ld_in_u32(p.in, 20 + 8ull * aa) != p.attrs[aa].P)
            bad = true;
        }
      }
      s_bad = bad;
      s_mode = my_mode;
      s_clen = clen;
      s_carry = carry;
      s_chunk = chunk;
    }
  }
  __syncthreads();
  const uint32_t mode = s_mode;
  bool ok = !s_bad;

  // ---- P rows wait for the same row of the previous frame (bounded)
  if (ok && mode == 1u && t > 0 && threadIdx.x == 0) {
    const uint32_t* flag = p.done + (k - A * H);
    if (!*reinterpret_cast<const volatile uint32_t*>(flag)) {
      const unsigned long long t0 = global_timer_ns();
      uint32_t ns = 32;
      while (!*reinterpret_cast<const volatile uint32_t*>(flag)) {
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
        if (global_timer_ns() - t0 > kSpinLimitNs) {
          atomicOr(p.err, kErrTimeout);
          s_bad = 2;
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  ok = !s_bad;

  uint32_t n = 0, nlit = 0, nb = 0;
  if (ok) {
    // ---- stage the chunk and (P) the previous row
    const uint32_t clen = s_clen;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(p.in + s_chunk);
    for (uint32_t i = threadIdx.x; i < clen / 4u; i += kThreads) S.stage[i] = src[i];
    if (mode == 1u) {
      const uint8_t* prow = (t > 0 ? p.outp[(t - 1) * A + a] : p.state[a]) + r * rowb;
      for (uint32_t x = threadIdx.x; x < W; x += kThreads) S.vprev[x] = load_sample_cg(prow, at.s, x);
    }
    __syncthreads();
    // ---- literal counts per class word (2-bit class 2 = literal, 3 = invalid)
    if (threadIdx.x < 32) {
      const uint32_t lane = lane_id();
      uint32_t lit = 0;
      bool bad = false;
      if (lane < ncls) {
        const uint32_t cw = S.stage[lane];
        uint32_t used = 0xffffffffu;  // class slots past nw must be 0
        const uint32_t nslots = min(16u, nw - 16u * lane);
        if (nslots < 16u) used = (1u << (2u * nslots)) - 1u;
        lit = __popc((cw >> 1) & ~cw & 0x55555555u);
        if (((cw >> 1) & cw & 0x55555555u) || (cw & ~used)) bad = true;
      }
      const uint32_t incl = warp_incl_scan(lit);
      if (lane < ncls) s_litpre[lane] = incl - lit;
      bad = __any_sync(0xffffffffu, bad);
      if (lane == 31) {
        s_nlit = incl;
        if (bad || 4u * (ncls + incl) > clen) s_bad = 1;
      }
    }
    __syncthreads();
    ok = !s_bad;
  }
  if (ok) {
    nlit = s_nlit;
    // ---- mask words: decoded class/literal, XOR previous mask for P
    for (uint32_t j = warp_id(); j < nw; j += kWarps) {
      const uint32_t x = 32u * j + lane_id();
      const uint32_t valid = (j + 1 < nw || (W & 31u) == 0) ? 0xffffffffu : ((1u << (W & 31u)) - 1u);
      const uint32_t cw = S.stage[j >> 4];
      const uint32_t sl = 2u * (j & 15u);
      const uint32_t cls = (cw >> sl) & 3u;
      uint32_t X = 0;
      if (cls == 1u) X = valid;
      else if (cls == 2u) {
        const uint32_t li = s_litpre[j >> 4] + __popc((cw >> 1) & ~cw & 0x55555555u & ((1u << sl) - 1u));
        X = S.stage[ncls + li];
        if (X & ~valid) s_bad = 1;
      }
      uint32_t M = X;
      if (mode == 1u) M ^= __ballot_sync(0xffffffffu, x < W && S.vprev[x] == 0u);
      if (lane_id() == 0) {
        S.mask[j] = M;
        S.base[j] = __popc(~M & valid);
      }
    }
    __syncthreads();
    n = block_excl_scan(S.base, nw, s_tmp);
    nb = ceil_div_u32(n, kBlockN);
    if (4u * (ncls + nlit + nb) > s_clen) s_bad = 1;
    __syncthreads();
    ok = !s_bad;
  }
  if (ok) {
    // ---- block headers
    const uint32_t* hdr = S.stage + ncls + nlit;
    for (uint32_t blk = threadIdx.x; blk < nb; blk += kThreads) {
      const uint32_t h = hdr[blk];
      const uint32_t b = h & 0xffu, e = (h >> 8) & 0xffu, hb = (h >> 16) & 0xffu;
      const uint32_t m = min(kBlockN, n - blk * kBlockN);
      if ((h >> 24) || b > 32u || hb > 32u || b + hb > 32u || e > m || ((e == 0u) != (hb == 0u))) s_bad = 1;
      S.boff[blk] = block_body_bytes(m, min(b, 32u), min(e, m), min(b + hb, 32u));
    }
    __syncthreads();
    const uint32_t body = block_excl_scan(S.boff, nb, s_tmp);
    if (4u * (ncls + nlit + nb) + body != s_clen) s_bad = 1;
    __syncthreads();
    ok = !s_bad;
  }
  if (ok) {
    // ---- unpack: warp per block
    const uint32_t* hdr = S.stage + ncls + nlit;
    for (uint32_t blk = warp_id(); blk < nb; blk += kWarps) {
      const uint32_t h = hdr[blk];
      const uint32_t b = h & 0xffu, e = (h >> 8) & 0xffu, hb = (h >> 16) & 0xffu;
      const uint32_t base = blk * kBlockN, m = min(kBlockN, n - base);
      const uint32_t* body = S.stage + ncls + nlit + nb + S.boff[blk] / 4u;
      for (uint32_t i = lane_id(); i < m; i += 32) S.z[base + i] = extract_bits(body, i * b, b);
      __syncwarp();
      if (e) {
        const uint32_t low_words = (m * b + 31u) >> 5;
        const uint8_t* pos = reinterpret_cast<const uint8_t*>(body + low_words);
        const uint32_t* high = body + low_words + ((e + 3u) >> 2);
        for (uint32_t j = lane_id(); j < e; j += 32) {
          const uint32_t ps = pos[j];
          if (ps >= m || (j > 0 && ps <= pos[j - 1])) s_bad = 1;
          else S.z[base + ps] |= extract_bits(high, j * hb, hb) << b;
        }
      }
      __syncwarp();
    }
    __syncthreads();
    ok = !s_bad;
  }
  if (ok) {
    // ---- inverse ZigZag + inclusive prefix from the carry (mod 2^32)
    const uint32_t per = (n + kThreads - 1) / kThreads;
    const uint32_t beg = min(threadIdx.x * per, n), end = min(beg + per, n);
    uint32_t sum = 0;
    for (uint32_t i = beg; i < end; i++) sum += unzigzag(S.z[i]);
    const uint32_t incl = warp_incl_scan(sum);
    if (lane_id() == 31) s_tmp[warp_id()] = incl;
    __syncthreads();
    if (threadIdx.x < 32) {
      const uint32_t w = threadIdx.x < (uint32_t)kWarps ? s_tmp[threadIdx.x] : 0u;
      const uint32_t wi = warp_incl_scan(w);
      if (threadIdx.x < (uint32_t)kWarps) s_tmp[threadIdx.x] = wi - w;
    }
    __syncthreads();
    uint32_t run = s_carry + s_tmp[warp_id()] + incl - sum;
    for (uint32_t i = beg; i < end; i++) {
      run += unzigzag(S.z[i]);
      S.z[i] = run;
    }
    __syncthreads();
    // ---- scatter, + previous value (P), times the precision
    uint8_t* orow = p.outp[ta] + r * rowb;
    uint8_t* srow = (t + 1 == p.T) ? p.state_next[a] + r * rowb : nullptr;
    const uint32_t P = at.P;
    for (uint32_t j = warp_id(); j < nw; j += kWarps) {
      const uint32_t x = 32u * j + lane_id();
      if (x < W) {
        const uint32_t M = S.mask[j];
        uint32_t v = 0;
        if (!((M >> lane_id()) & 1u)) {
          const uint32_t kk = S.base[j] + __popc(~M & ((1u << lane_id()) - 1u));
          v = S.z[kk] * P;
          if (mode == 1u) v += S.vprev[x];
        }
        store_sample(orow, at.s, x, v);
        if (srow) store_sample(srow, at.s, x, v);
      }
    }
  } else if (threadIdx.x == 0 && s_bad == 1) {
    atomicOr(p.err, kErrCorrupt);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicExch(p.done + k, 1u);
  }
}

size_t dec_smem_bytes_host(uint32_t W) { return dec_smem_bytes(W); }

int launch_decode(const DecParams& p, void* stream, void* const* ev) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t smem = dec_smem_bytes(p.W);
  cudaError_t e = cudaFuncSetAttribute(k_decode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  if (ev) cudaEventRecord(reinterpret_cast<cudaEvent_t>(ev[0]), st);
  k_decode<<<p.n_items, kThreads, smem, st>>>(p);
  if (ev) cudaEventRecord(reinterpret_cast<cudaEvent_t>(ev[1]), st);
  return (int)cudaGetLastError();
}

}  // namespace jiffy
