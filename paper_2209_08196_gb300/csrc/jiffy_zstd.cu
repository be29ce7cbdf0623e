// Zstandard mask kernels (sm_103a). Sec. III-C packs the zero bitmask into
// bytes and compresses it with Zstd; for a P scan (Sec. III-D) the mask is
// the XOR with the previous scan's first. A stream with kStageZstdMask codes
// each section's mask that way: the rows' coded mask bits, LSB first, rows of
// ceil(W/8) bytes, as one Zstandard frame (RFC 8878) that any Zstandard
// decoder restores. The part of the format written here:
//   frame header: magic, descriptor 0xA0 (single segment, 4-byte content
//     size), the content size; one block per 8192 mask bytes, each
//     RLE         when its bytes are all equal,
//     Compressed  a Huffman-coded literals section and no sequences, when
//                 that is smaller than the input,
//     Raw         otherwise;
//   Huffman code lengths: the two-queue construction over the present byte
//     values sorted by (count, value), a tie taking the leaf; while a code is
//     longer than 11 bits every count c becomes ceil(c/2) and the
//     construction is repeated;
//   tree description: 4-bit weights when at most 128 weights are listed,
//     else FSE-compressed weights (accuracy log 6, two interleaved states,
//     normalised counts max(1, floor(64 c / N)) with the rest on the most
//     frequent weight value, the smaller one among ties; initial states at the
//     lowest table position of their symbol); a block whose weights fit
//     neither form is Raw;
//   one Huffman stream for blocks of at most 1023 bytes, four above.
// Beside the frame the section keeps the end of every block, so that each
// block is located, and decoded, on its own.
//
// k_zstd_enc: one CTA of 128 threads per (section, block), after the rows
//   kernel has stored the section's coded mask bytes. Each thread owns 64
//   consecutive bytes of the block (all requested at once for the histogram,
//   re-read from L1 by the later passes); code lengths (a bitonic sort of the
//   present symbols, the merge on thread 0) and the tree description (FSE
//   steps on thread 0: at most 256 symbols and 255 weights); then each thread
//   codes its literals: their bit positions from a CTA-wide scan of the code
//   lengths, their codes ORed into the block image in shared memory. The image goes to the block's slot; the placement kernel
//   assembles the frame. (Small CTAs: the serial steps of many blocks
//   overlap on an SM.)
// k_zstd_dec: one warp per (section, block), before the rows kernel. Checks
//   the block-end index, the frame and block headers, stages a Compressed
//   block in shared memory, reads the tree (lane 0), builds the decoding
//   table (warp ballots per weight class) and decodes the streams, one lane
//   per stream, each through a 64-bit window of its bits held in registers,
//   into the section's mask bytes; the rows kernel reads its rows from there.
//   Anything that is not what the writer can produce sets the segment's
//   CORRUPT flag.
#include "jiffy_device.cuh"
#include "jiffy_kernels.h"

namespace jiffy {

namespace {

constexpr uint32_t kZT = 128;               // threads of a writer CTA
constexpr uint32_t kZW = kZT / 32;          // its warps
constexpr uint32_t kZPer = kZBlock / kZT;   // literals of one writer thread (64)
constexpr uint32_t kZMaxBits = 11;          // longest Huffman code (RFC 8878)
constexpr uint32_t kZFseLog = 6;            // accuracy log of the weights' FSE table
constexpr uint32_t kZTree = 136;            // tree description buffer (a description is at most 128 bytes)

__device__ __forceinline__ uint32_t hibit(uint32_t x) { return 31u - __clz(x); }

__device__ __forceinline__ uint32_t sec_segment(const uint32_t* base, uint32_t n, uint32_t key) {
  uint32_t lo = 0, hi = n;  // base[lo] <= key < base[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(base + mid) <= key) lo = mid;
    else hi = mid;
  }
  return lo;
}

// ----------------------------------------------------------------------------
// FSE decoding table of a normalised distribution (RFC 8878 4.1.1): symbols
// spread with step 64/2 + 64/8 + 3; position u holding symbol s gets the next
// of s's counters x (from norm[s]), nb = 6 - highbit(x), base = (x << nb) - 64.
// next: 16 words of scratch.
// ----------------------------------------------------------------------------
struct FseTable {
  uint8_t sym[64], nb[64];
  uint16_t base[64];
};

__device__ void fse_table(const uint32_t* norm, uint32_t nsym, FseTable& t, uint32_t* next) {
  uint32_t pos = 0;
  for (uint32_t s = 0; s < nsym; s++) {
    for (uint32_t i = 0; i < norm[s]; i++) {
      t.sym[pos] = (uint8_t)s;
      pos = (pos + 43u) & 63u;
    }
  }
  for (uint32_t s = 0; s < 16; s++) next[s] = s < nsym ? norm[s] : 0u;
  for (uint32_t u = 0; u < 64; u++) {
    const uint32_t x = next[t.sym[u]]++;
    t.nb[u] = (uint8_t)(kZFseLog - hibit(x));
    t.base[u] = (uint16_t)((x << t.nb[u]) - 64u);
  }
}

// Bit writer (bits LSB first, fields of at most 16 bits): whole bytes leave a
// register accumulator in order; bytes past cap are dropped (counted).
struct BitPut {
  uint8_t* buf;
  uint32_t cap, nbytes;
  unsigned long long acc;
  uint32_t nacc;
  __device__ void put(uint32_t v, uint32_t n) {
    acc |= (unsigned long long)(v & ((1u << n) - 1u)) << nacc;
    nacc += n;
    while (nacc >= 8u) {
      if (nbytes < cap) buf[nbytes] = (uint8_t)acc;
      nbytes++;
      acc >>= 8;
      nacc -= 8u;
    }
  }
  __device__ uint32_t close() {  // zero bits up to the byte boundary; returns the bytes
    if (nacc) {
      if (nbytes < cap) buf[nbytes] = (uint8_t)acc;
      nbytes++;
      acc = 0;
      nacc = 0;
    }
    return nbytes;
  }
};

// ----------------------------------------------------------------------------
// Writer
// ----------------------------------------------------------------------------
struct ZEnc {
  uint32_t img[kZSlot / 4];       // the block being assembled (header first)
  uint32_t hist[kZW][256];        // per-warp histograms
  uint32_t cnt[256], len[256], code[256];
  uint32_t key[256];              // count << 8 | value of the present symbols, sorted; then absent ones
  uint32_t wnode[511];            // Huffman internal node weights (index >= number of leaves)
  uint16_t parent[511];
  uint8_t depth[511];
  uint8_t weight[256];
  uint8_t tree[kZTree];
  uint8_t fenc[16][64];           // FSE encoding: (symbol, next state) -> state
  FseTable ft;
  uint32_t fhist[16], fnorm[16], fnext[16];
  uint32_t gcnt[8][kZMaxBits + 1];  // symbols of each weight per group of 32 values
  uint32_t wsum[kZW];             // scan scratch
  uint32_t pb[5];                 // literal bits before each stream boundary
  uint32_t maxd, last, tree_len, fnsym, fok;
};

// FSE-compressed Huffman weights (RFC 8878 4.2.1.2) of weight[0..n), in
// three steps: fse_prepare (thread 0; z.fhist holds the weights' histogram)
// normalises and builds the table, or clears z.fok when the weights cannot be
// written that way; fse_fill (threads 0..63) builds the encoding table;
// fse_write (thread 0) writes the description into z.tree (header byte first)
// and returns its bytes, or 0.
__device__ void fse_prepare(ZEnc& z, uint32_t n) {
  const uint32_t* hist = z.fhist;
  uint32_t* norm = z.fnorm;
  uint32_t distinct = 0, nsym = 0, best = 0;
  for (uint32_t v = 0; v < 16; v++) {
    if (!hist[v]) continue;
    distinct++;
    nsym = v + 1;
    if (hist[v] > hist[best]) best = v;
  }
  z.fok = 0;
  if (distinct < 2 || n < 2) return;
  uint32_t sum = 0;
  for (uint32_t v = 0; v < 16; v++) {
    norm[v] = 0;
    if (!hist[v]) continue;
    norm[v] = max(1u, (hist[v] << kZFseLog) / n);
    sum += norm[v];
  }
  const int rest = (int)norm[best] + 64 - (int)sum;
  if (rest < 1) return;
  norm[best] = (uint32_t)rest;
  fse_table(norm, nsym, z.ft, z.fnext);
  z.fnsym = nsym;
  z.fok = 1;
}

__device__ __forceinline__ void fse_fill(ZEnc& z, uint32_t u) {
  const uint32_t lo = z.ft.base[u], hi = lo + (1u << z.ft.nb[u]);
  for (uint32_t v = lo; v < hi && v < 64u; v++) z.fenc[z.ft.sym[u]][v] = (uint8_t)u;
}

__device__ uint32_t fse_write(ZEnc& z, uint32_t n) {
  const uint32_t* norm = z.fnorm;
  const uint32_t nsym = z.fnsym;
  // table description, forward: log - 5, then count + 1 per value with the
  // variable-size code the reader expects, repeat flags after a zero count
  BitPut w{z.tree + 1, 127u, 0u, 0ull, 0u};
  w.put(kZFseLog - 5u, 4u);
  uint32_t remaining = 65, s = 0;
  while (remaining > 1 && s < nsym) {
    const uint32_t v = norm[s] + 1u, nbits = hibit(remaining) + 1u, thr = 1u << (nbits - 1u);
    const uint32_t lo = 2u * thr - 1u - remaining;
    if (v < lo) w.put(v, nbits - 1u);
    else if (v < thr) w.put(v, nbits);
    else w.put(v + lo, nbits);
    remaining -= norm[s];
    s++;
    if (norm[s - 1] == 0) {
      uint32_t zr = 0;
      while (s + zr < nsym && norm[s + zr] == 0) zr++;
      s += zr;
      while (zr >= 3) {
        w.put(3u, 2u);
        zr -= 3;
      }
      w.put(zr, 2u);
    }
  }
  const uint32_t head = w.close();
  if (head >= 127u) return 0;
  // two states from the last weight back: weight i is emitted by state i%2;
  // the fields come out in the order they are written
  BitPut b{z.tree + 1 + head, 127u - head, 0u, 0ull, 0u};
  uint32_t st[2] = {0, 0};
  for (int i = (int)n - 1; i >= 0; i--) {
    const uint32_t q = (uint32_t)i & 1u, sy = z.weight[i];
    if (i >= (int)n - 2) {
      uint32_t u = 0;
      while (z.ft.sym[u] != sy) u++;
      st[q] = u;
      continue;
    }
    const uint32_t v = st[q], u = z.fenc[sy][v];
    b.put(v - z.ft.base[u], z.ft.nb[u]);
    st[q] = u;
  }
  b.put(st[1], kZFseLog);
  b.put(st[0], kZFseLog);
  b.put(1u, 1u);
  const uint32_t body = b.close();
  if (head + body >= 128u) return 0;
  z.tree[0] = (uint8_t)(head + body);
  return 1u + head + body;
}

// In-place ascending bitonic sort of 256 words in shared memory (all threads).
__device__ __forceinline__ void bitonic256(uint32_t* key) {
  for (uint32_t k = 2; k <= 256u; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      const uint32_t t = threadIdx.x;
      const uint32_t i = 2u * t - (t & (j - 1u)), l = i + j;
      const uint32_t a = key[i], c = key[l];
      if ((a > c) == ((i & k) == 0u)) {
        key[i] = c;
        key[l] = a;
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ void img_put_bytes(uint8_t* img, uint32_t at, unsigned long long v, uint32_t nbytes) {
  for (uint32_t i = 0; i < nbytes; i++) img[at + i] = (uint8_t)(v >> (8u * i));
}

// Word k of a writer thread's literals, bytes i0 + 4k .. i0 + 4k + 3 of the
// block (bytes past its end m read as 0; the thread's bytes are re-read from
// L1 by each pass).
__device__ __forceinline__ uint32_t chunk_word(const uint8_t* src, uint32_t i0, uint32_t m, uint32_t k) {
  const uint32_t at = i0 + 4u * k;
  if (at + 4u <= m) return __ldg(reinterpret_cast<const uint32_t*>(src + at));
  uint32_t v = 0;
  for (uint32_t b = 0; b < 4u; b++)
    if (at + b < m) v |= (uint32_t)__ldg(src + at + b) << (8u * b);
  return v;
}

// Exclusive prefix of v over the CTA's threads; *total receives the sum.
__device__ __forceinline__ uint32_t cta_excl_scan(uint32_t v, uint32_t* wsum, uint32_t* total) {
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const uint32_t incl = warp_incl_scan(v);
  if (lane == 31u) wsum[w] = incl;
  __syncthreads();
  uint32_t off = 0, tot = 0;
#pragma unroll
  for (uint32_t i = 0; i < kZW; i++) {
    const uint32_t x = wsum[i];
    off += i < w ? x : 0u;
    tot += x;
  }
  *total = tot;
  return off + incl - v;
}

__global__ void __launch_bounds__(kZT, 8) k_zstd_enc(EncParams p) {
  __shared__ ZEnc z;
  const uint32_t gs = blockIdx.x, j = blockIdx.y, tid = threadIdx.x;
  const EncSeg& sg = p.seg[sec_segment(p.seg_sec_base, p.n_seg, gs)];
  if (!(sg.stages & kStageZstdMask) || j >= sg.zm_nblk) return;  // the whole CTA
  const uint32_t ta = gs - sg.sec_base;
  const uint32_t n = sg.H * sg.zm_rb, lo = j * kZBlock, m = min(kZBlock, n - lo);
  // (section strides and block starts are multiples of 16 bytes)
  const uint8_t* src = p.zmask + sg.zm_base + (size_t)ta * sg.zm_stride + lo;
  const size_t slot = sg.zb_base + (size_t)ta * sg.zm_nblk + j;
  uint32_t* dst = reinterpret_cast<uint32_t*>(p.zblk + slot * kZSlot);
  const uint32_t last_blk = j + 1 == sg.zm_nblk ? 1u : 0u;
  uint8_t* img = reinterpret_cast<uint8_t*>(z.img);
  const uint32_t i0 = kZPer * tid;
  const uint32_t nmine = i0 < m ? min(kZPer, m - i0) : 0u;

  // ---- clear the image and the histograms; one pass over the thread's
  //      bytes (all 16 words requested at once): histogram, and are the
  //      block's bytes all equal?
  const uint32_t nw4 = (nmine + 3u) / 4u;
  for (uint32_t i = tid; i < kZSlot / 4; i += kZT) z.img[i] = 0;
  for (uint32_t i = tid; i < kZW * 256; i += kZT) (&z.hist[0][0])[i] = 0;
  const uint8_t b0 = __ldg(src);
  __syncthreads();
  int diff = 0;
  {
    uint32_t wv[kZPer / 4];
#pragma unroll
    for (uint32_t k = 0; k < kZPer / 4; k++) wv[k] = k < nw4 ? chunk_word(src, i0, m, k) : 0u;
#pragma unroll
    for (uint32_t k = 0; k < kZPer / 4; k++) {
#pragma unroll
      for (uint32_t b = 0; b < 4u; b++) {
        if (4u * k + b < nmine) {
          const uint32_t v = (wv[k] >> (8u * b)) & 0xffu;
          diff |= v != b0;
          atomicAdd(&z.hist[tid >> 5][v], 1u);
        }
      }
    }
  }
  if (!__syncthreads_or(diff)) {  // RLE block: header + the byte
    if (tid == 0) {
      dst[0] = last_blk | (1u << 1) | (m << 3) | ((uint32_t)b0 << 24);
      p.zblk_bytes[slot] = 4;
    }
    return;
  }

  // ---- counts of the block
  for (uint32_t s = tid; s < 256; s += kZT) {
    uint32_t c = 0;
    for (uint32_t w = 0; w < kZW; w++) c += z.hist[w][s];
    z.cnt[s] = c;
  }
  __syncthreads();

  // ---- code lengths: the present symbols sorted by (count, value) (a
  //      bitonic sort of count << 8 | value), merged on thread 0 with the
  //      queue heads in registers, internal depths top-down; each leaf's
  //      length is its parent's depth + 1. Counts halved while too deep.
  for (;;) {
    uint32_t c2[2];
    for (uint32_t h = 0; h < 2; h++) {
      const uint32_t s = tid + kZT * h, c = z.cnt[s];
      c2[h] = c;
      z.len[s] = 0;
      z.key[s] = c ? (c << 8) | s : 0xffffffffu;
    }
    if (tid == 0) z.maxd = 0;
    const uint32_t nsym = (uint32_t)__syncthreads_count(c2[0] != 0u) + (uint32_t)__syncthreads_count(c2[1] != 0u);
    bitonic256(z.key);
    if (tid == 0) {
      uint32_t lf = 0, nd = nsym, next = nsym;
      uint32_t lw = z.key[0] >> 8, ndw = 0;
      for (uint32_t k = 0; k + 1 < nsym; k++) {
        uint32_t pk[2], pw[2];
#pragma unroll
        for (uint32_t q = 0; q < 2; q++) {
          if (lf < nsym && (nd >= next || lw <= ndw)) {
            pk[q] = lf;
            pw[q] = lw;
            lf++;
            lw = lf < nsym ? (z.key[lf] >> 8) : 0u;
          } else {
            pk[q] = nd;
            pw[q] = ndw;
            nd++;
            ndw = nd < next ? z.wnode[nd] : 0u;
          }
        }
        const uint32_t ws = pw[0] + pw[1];
        z.wnode[next] = ws;
        z.parent[pk[0]] = (uint16_t)next;
        z.parent[pk[1]] = (uint16_t)next;
        if (nd == next) ndw = ws;  // the node queue was empty: the new node heads it
        next++;
      }
      z.depth[next - 1] = 0;
      for (int i = (int)next - 2; i >= (int)nsym; i--) z.depth[i] = (uint8_t)(z.depth[z.parent[i]] + 1u);
    }
    __syncthreads();
    for (uint32_t i = tid; i < nsym; i += kZT) {
      const uint32_t L = z.depth[z.parent[i]] + 1u;
      z.len[z.key[i] & 0xffu] = L;
      atomicMax(&z.maxd, L);
    }
    __syncthreads();
    if (z.maxd <= kZMaxBits) break;
    z.cnt[tid] = (c2[0] + 1u) >> 1;
    z.cnt[tid + kZT] = (c2[1] + 1u) >> 1;
    __syncthreads();
  }

  // ---- weights; canonical codes (symbols by weight then value take
  //      consecutive ranges of the 2^maxbits decoding entries from entry 0):
  //      a symbol's range starts after all lower weights and the symbols of
  //      its own weight with smaller values (warp ballots per group of 32)
  const uint32_t maxb = z.maxd, lane = tid & 31u, wp = tid >> 5;
  if (tid == 0) z.last = 0;
  uint32_t wt2[2];
  for (uint32_t h = 0; h < 2; h++) {
    const uint32_t s = tid + kZT * h, L = z.len[s];
    wt2[h] = L ? maxb + 1u - L : 0u;
    z.weight[s] = (uint8_t)wt2[h];
  }
  if (tid < 16) z.fhist[tid] = 0;
  __syncthreads();
  uint32_t rank2[2];
  for (uint32_t h = 0; h < 2; h++) {
    const uint32_t g = 4u * h + wp;  // group of symbols 32g .. 32g + 31
    rank2[h] = 0;
    for (uint32_t w = 1; w <= maxb; w++) {
      const uint32_t msk = __ballot_sync(0xffffffffu, wt2[h] == w);
      if (wt2[h] == w) rank2[h] = __popc(msk & ((1u << lane) - 1u));
      if (lane == 0) z.gcnt[g][w] = __popc(msk);
    }
    if (wt2[h]) atomicMax(&z.last, tid + kZT * h);
  }
  __syncthreads();
  const uint32_t last = z.last;
  for (uint32_t h = 0; h < 2; h++) {
    const uint32_t s = tid + kZT * h, w = wt2[h];
    if (s < last) atomicAdd(&z.fhist[w], 1u);
    if (!w) continue;
    uint32_t base = 0, before = 0;
    for (uint32_t w2 = 1; w2 <= maxb; w2++) {
      uint32_t tot = 0;
      for (uint32_t g = 0; g < 8; g++) {
        const uint32_t c = z.gcnt[g][w2];
        tot += c;
        if (w2 == w && g < 4u * h + wp) before += c;
      }
      if (w2 < w) base += tot << (w2 - 1u);
    }
    z.code[s] = (base + ((before + rank2[h]) << (w - 1u))) >> (w - 1u);
  }
  __syncthreads();
  // tree description: weights of symbols 0 .. last-1 (the last is implied)
  if (last <= 128u) {
    if (tid == 0) {
      for (uint32_t i = 0; i < kZTree; i++) z.tree[i] = 0;
      z.tree[0] = (uint8_t)(127u + last);
      for (uint32_t i = 0; i < last; i++) z.tree[1 + i / 2] |= (uint8_t)(z.weight[i] << ((i & 1u) ? 0 : 4));
      z.tree_len = 1u + (last + 1u) / 2u;
    }
  } else {
    if (tid == 0) fse_prepare(z, last);
    __syncthreads();
    if (z.fok && tid < 64u) fse_fill(z, tid);
    __syncthreads();
    if (tid == 0) z.tree_len = z.fok ? fse_write(z, last) : 0u;
  }

  // ---- literal bit counts: per-thread sums, CTA scan, stream boundaries
  const bool four = m > 1023u;
  const uint32_t seg = four ? (m + 3u) / 4u : m, ns = four ? 4u : 1u;
  uint32_t sum = 0;
  for (uint32_t k = 0; k < nw4; k++) {
    const uint32_t w = chunk_word(src, i0, m, k);
#pragma unroll
    for (uint32_t b = 0; b < 4u; b++)
      if (4u * k + b < nmine) sum += z.len[(w >> (8u * b)) & 0xffu];
  }
  uint32_t total;
  const uint32_t P0 = cta_excl_scan(sum, z.wsum, &total);
  if (four) {  // the stream boundaries a thread's literals cross
    uint32_t P = P0;
    for (uint32_t k = 0; k < nw4; k++) {
      const uint32_t w = chunk_word(src, i0, m, k);
#pragma unroll
      for (uint32_t b = 0; b < 4u; b++) {
        const uint32_t i = i0 + 4u * k + b;
        if (4u * k + b >= nmine) break;
        if (i % seg == 0 && i > 0) z.pb[i / seg] = P;
        P += z.len[(w >> (8u * b)) & 0xffu];
      }
    }
  }
  {
    if (tid == 0) {
      z.pb[0] = 0;
      z.pb[ns] = total;
    }
  }
  __syncthreads();
  const uint32_t tl = z.tree_len, lhdr = four ? 4u : 3u;
  uint32_t soff[4], bytes_k[4], cs = tl + (four ? 6u : 0u);
  bool jump_ok = true;
  for (uint32_t k = 0; k < ns; k++) {
    bytes_k[k] = (z.pb[k + 1] - z.pb[k] + 8u) >> 3;  // bits + end mark, whole bytes
    soff[k] = 3u + lhdr + cs;
    cs += bytes_k[k];
    if (k < 3 && bytes_k[k] > 0xFFFFu) jump_ok = false;
  }
  const uint32_t content = lhdr + cs + 1u;  // literals section + Number_of_Sequences = 0
  const bool compressed = tl != 0u && jump_ok && content < m;

  uint32_t blk_bytes;
  if (compressed) {
    if (tid == 0) {
      img_put_bytes(img, 0, last_blk | (2u << 1) | (content << 3), 3);
      const unsigned long long h = four ? (2ull | (2ull << 2) | ((unsigned long long)m << 4) | ((unsigned long long)cs << 18))
                                        : (2ull | ((unsigned long long)m << 4) | ((unsigned long long)cs << 14));
      img_put_bytes(img, 3, h, lhdr);
      for (uint32_t i = 0; i < tl; i++) img[3 + lhdr + i] = z.tree[i];
      if (four)
        for (uint32_t k = 0; k < 3; k++) img_put_bytes(img, 3 + lhdr + tl + 2 * k, bytes_k[k], 2);
    }
    __syncthreads();  // header bytes before the streams' bits (they may share words)
    // each stream is read from its end: literal i of stream k sits after the
    // codes of the stream's later literals; end mark after the last field
    uint32_t P = P0;
    for (uint32_t kw = 0; kw < nw4; kw++) {
      const uint32_t w = chunk_word(src, i0, m, kw);
#pragma unroll
      for (uint32_t b = 0; b < 4u; b++) {
        if (4u * kw + b >= nmine) break;
        const uint32_t i = i0 + 4u * kw + b, s = (w >> (8u * b)) & 0xffu;
        const uint32_t l = z.len[s], k = four ? min(i / seg, 3u) : 0u;
        const uint32_t g = 8u * soff[k] + (z.pb[k + 1] - P - l);
        const uint32_t c = z.code[s], sh = g & 31u;
        atomicOr(&z.img[g >> 5], c << sh);
        if (sh + l > 32u) atomicOr(&z.img[(g >> 5) + 1u], c >> (32u - sh));
        P += l;
      }
    }
    if (tid < ns) {
      const uint32_t g = 8u * soff[tid] + (z.pb[tid + 1] - z.pb[tid]);
      atomicOr(&z.img[g >> 5], 1u << (g & 31u));
    }
    blk_bytes = 3u + content;
  } else {  // Raw block
    if (tid == 0) img_put_bytes(img, 0, last_blk | (m << 3), 3);
    for (uint32_t k = 0; k < nw4; k++) {
      const uint32_t w = chunk_word(src, i0, m, k);
#pragma unroll
      for (uint32_t b = 0; b < 4u; b++)
        if (4u * k + b < nmine) img[3 + i0 + 4u * k + b] = (uint8_t)(w >> (8u * b));
    }
    blk_bytes = 3u + m;
  }
  __syncthreads();
  for (uint32_t i = tid; i < (blk_bytes + 3u) / 4u; i += kZT) dst[i] = z.img[i];
  if (tid == 0) p.zblk_bytes[slot] = blk_bytes;
}

// ----------------------------------------------------------------------------
// Reader
// ----------------------------------------------------------------------------
constexpr uint32_t kBlkWords = (kZBlock + 128) / 4;  // a block's content (<= 8192 bytes from byte 0..3) + slack

struct ZDec {
  uint32_t blkw[kBlkWords];   // a Compressed block's content (from byte blk_at), zero slack for the peeks
  uint16_t dt[1u << kZMaxBits];  // decoding table: symbol | code bits << 8
  uint8_t weight[256];
  uint8_t sorted[256];        // symbols with a weight, by (weight, value)
  uint32_t cls_base[kZMaxBits + 1], cls_pos[kZMaxBits + 1], cls_cnt[kZMaxBits + 1];
  uint32_t fnext[16];
  uint32_t fpack[64];         // FSE decoding table packed: symbol | bits << 8 | baseline << 16
  FseTable ft;
  uint32_t ok, maxbits, tree_len, sf, cs, lhdr, nweights;
};

__device__ __forceinline__ uint8_t in_byte(const uint8_t* in, unsigned long long at) { return __ldg(in + at); }

// Huffman tree description at s[0..len) (lane 0): the listed weights into
// z.weight[0 .. n) (z.weight zeroed beforehand), n into z.nweights; returns
// its bytes or 0. The FSE-coded form is read through a 64-bit window of its
// bit stream, as the literal streams are; the weights are checked afterwards
// by the whole warp (tree_weights).
__device__ uint32_t read_tree(ZDec& z, const uint8_t* s, uint32_t len) {
  if (len < 1) return 0;
  const uint32_t hb = s[0];
  uint32_t n = 0, used;
  if (hb >= 128u) {
    n = hb - 127u;
    used = 1u + (n + 1u) / 2u;
    if (used > len) return 0;
    for (uint32_t i = 0; i < n; i++) z.weight[i] = (uint8_t)((s[1 + i / 2] >> ((i & 1u) ? 0 : 4)) & 15u);
  } else {
    used = 1u + hb;
    if (used > len || hb == 0) return 0;
    const uint8_t* f = s + 1;
    const uint32_t fbits = 8u * hb;
    auto get = [&](uint32_t at, uint32_t nb) -> uint32_t {
      uint32_t v = 0;
      for (uint32_t i = 0; i < nb; i++) v |= (uint32_t)((f[(at + i) >> 3] >> ((at + i) & 7u)) & 1u) << i;
      return v;
    };
    const uint32_t log = (f[0] & 15u) + 5u;
    if (log != kZFseLog) return 0;  // only the writer's accuracy log
    uint32_t bp = 4, norm[16], nsym = 0, remaining = 65;
    while (remaining > 1) {
      if (nsym >= 16) return 0;
      const uint32_t nbits = hibit(remaining) + 1u, thr = 1u << (nbits - 1u), lo = 2u * thr - 1u - remaining;
      if (bp + nbits > fbits) return 0;
      uint32_t v = get(bp, nbits);
      if ((v & (thr - 1u)) < lo) {
        v &= thr - 1u;
        bp += nbits - 1u;
      } else {
        if (v >= thr) v -= lo;
        bp += nbits;
      }
      if (v == 0 || v - 1u > remaining - 1u) return 0;
      const uint32_t cnt = v - 1u;
      norm[nsym++] = cnt;
      remaining -= cnt;
      if (cnt == 0) {
        for (;;) {
          if (bp + 2u > fbits) return 0;
          const uint32_t rep = get(bp, 2u);
          bp += 2u;
          if (nsym + rep > 16u) return 0;
          for (uint32_t i = 0; i < rep; i++) norm[nsym++] = 0;
          if (rep != 3u) break;
        }
      }
    }
    const uint32_t head = (bp + 7u) >> 3;
    if (head >= hb) return 0;
    fse_table(norm, nsym, z.ft, z.fnext);
    for (uint32_t u = 0; u < 64; u++) z.fpack[u] = z.ft.sym[u] | ((uint32_t)z.ft.nb[u] << 8) | ((uint32_t)z.ft.base[u] << 16);
    // the weights' bit stream, read from its end through a 64-bit window
    // (bits [bot, bot + k) in its low k bits; below the start: zeros)
    const uint8_t* bs = f + head;
    const uint32_t blen = hb - head;
    if (bs[blen - 1] == 0) return 0;
    const int p0 = (int)(8u * (blen - 1u) + hibit(bs[blen - 1]));
    if (p0 < (int)(2u * kZFseLog)) return 0;
    int bot = p0 & ~7, k = p0 - bot;
    unsigned long long win = bs[bot >> 3] & ((1u << k) - 1u);
    auto refill = [&]() {
      if (k < 32) {
        const int b = (bot >> 3) - 4;
        uint32_t w = 0;
#pragma unroll
        for (int q = 0; q < 4; q++) w |= (b + q >= 0 ? (uint32_t)bs[b + q] : 0u) << (8 * q);
        win = (win << 32) | w;
        bot -= 32;
        k += 32;
      }
    };
    auto take = [&](uint32_t nb) -> uint32_t {  // nb <= 6 <= k after a refill
      const uint32_t v = (uint32_t)(win >> (k - (int)nb)) & ((1u << nb) - 1u);
      k -= (int)nb;
      return v;
    };
    refill();
    uint32_t st[2];
    st[0] = take(kZFseLog);
    refill();
    st[1] = take(kZFseLog);
    for (uint32_t q = 0;; q ^= 1u) {
      if (n >= 255u) return 0;
      const uint32_t e = z.fpack[st[q]];
      z.weight[n++] = (uint8_t)e;
      const uint32_t nb = (e >> 8) & 0xffu;
      if (bot + k < (int)nb) {  // past the start: the other state gives the last weight
        if (n >= 255u) return 0;
        z.weight[n++] = (uint8_t)z.fpack[st[q ^ 1u]];
        break;
      }
      refill();
      st[q] = (e >> 16) + take(nb);
    }
  }
  z.nweights = n;
  return used;
}

// The weights read by read_tree, checked by the whole warp: every weight at
// most 11, their sum (of 2^(w-1)) completed to a power of two by the implied
// last weight, whose symbol is n. Sets z.maxbits; false if malformed.
__device__ bool tree_weights(ZDec& z, uint32_t lane) {
  const uint32_t n = z.nweights;
  uint32_t sum = 0;
  bool bad = false;
  for (uint32_t i = lane; i < n; i += 32) {
    const uint32_t w = z.weight[i];
    bad |= w > kZMaxBits;
    sum += w ? 1u << (w - 1u) : 0u;
  }
  sum = __reduce_add_sync(0xffffffffu, sum);
  if (__any_sync(0xffffffffu, bad) || sum == 0 || n > 255u) return false;
  const uint32_t mb = hibit(sum) + 1u, rest = (1u << mb) - sum;
  if (mb > kZMaxBits || (rest & (rest - 1u))) return false;
  __syncwarp();
  if (lane == 0) {
    z.weight[n] = (uint8_t)(hibit(rest) + 1u);
    z.maxbits = mb;
  }
  __syncwarp();
  return true;
}

// One stream of cnt literals (lanes 0..3); false if malformed. The bits
// below the read position sit in a 64-bit window (bits [bot, bot + k) of the
// stream in its low k bits); whenever fewer than 32 remain it takes the 32
// bits below it (bytes before the stream's start read as zero), then two
// literals are decoded. The stream is well formed if the last literal ends
// exactly at bit 0. Loads and refills are predicated, so the lanes of
// different streams do not diverge.
__device__ bool read_stream(const ZDec& z, const uint8_t* s, uint32_t len, uint8_t* out, uint32_t cnt) {
  if (len == 0 || s[len - 1] == 0) return false;
  const int p0 = (int)(8u * (len - 1u) + hibit(s[len - 1]));
  const uint32_t mb = z.maxbits, mask = (1u << mb) - 1u;
  int bot = p0 & ~7;
  unsigned long long win = s[bot >> 3] & ((1u << (p0 - bot)) - 1u);
  int k = p0 - bot;
  auto refill = [&]() {
    const int b = (bot >> 3) - 4;
    uint32_t w = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) w |= (b + q >= 0 ? (uint32_t)s[b + q] : 0u) << (8 * q);
    const bool need = k < 32;
    win = need ? (win << 32) | w : win;
    bot = need ? bot - 32 : bot;
    k = need ? k + 32 : k;
  };
  auto one = [&](uint32_t i) {
    const uint32_t e = z.dt[(uint32_t)(win >> (k - (int)mb)) & mask];
    out[i] = (uint8_t)e;
    k -= (int)(e >> 8);
  };
  uint32_t i = 0;
  for (; i + 1u < cnt; i += 2u) {
    refill();
    one(i);
    one(i + 1u);
  }
  if (i < cnt) {
    refill();
    one(i);
  }
  return bot + k == 0;
}

__global__ void __launch_bounds__(32) k_zstd_dec(DecParams p) {
  __shared__ ZDec z;
  const uint32_t gs = blockIdx.x, j = blockIdx.y, lane = threadIdx.x;
  const DecSeg& sg = p.seg[sec_segment(p.seg_sec_base, p.n_seg, gs)];
  if (!(sg.stages & kStageZstdMask) || j >= sg.zm_nblk) return;
  const uint32_t ta = gs - sg.sec_base, A = sg.A, t = ta / A, a = ta % A, H = sg.H, nblk = sg.zm_nblk;
  const uint32_t n = H * sg.zm_rb, lo = j * kZBlock, m = min(kZBlock, n - lo);
  uint8_t* dst = p.zdec + sg.zm_base + (size_t)ta * sg.zm_stride + lo;
  const uint8_t* in = sg.in;
  auto fail = [&]() {
    if (lane == 0) atomicOr(sg.err, kErrCorrupt);
  };
  // ---- the section: frame offsets checked before any read, then the sum of
  //      the earlier attributes' section bytes
  const unsigned long long f0 = sg.off[t], f1 = sg.off[t + 1];
  const unsigned long long first = (t == 0 && sg.check_shdr) ? 16ull + 8ull * A : 0ull;
  if (f0 < first || (f0 & 3ull) || f1 < f0 + sg.fhdr || f1 > sg.in_len) return fail();
  unsigned long long before = 0, mine = 0;
  for (uint32_t aa = lane; aa <= a; aa += 32) {
    const unsigned long long sb = __ldg(reinterpret_cast<const unsigned int*>(in + f0 + 12ull + 12ull * aa));
    if (aa < a) before += sb;
    else mine = sb;
  }
  for (int o = 16; o > 0; o >>= 1) {
    before += __shfl_xor_sync(0xffffffffu, before, o);
    mine += __shfl_xor_sync(0xffffffffu, mine, o);
  }
  const unsigned long long sec = f0 + sg.fhdr + before;
  const unsigned long long zp = sec + 8ull * H, idx = 4ull + 4ull * nblk;
  if (sec + mine > f1 || mine < 8ull * H + idx || ((sec + mine) & 3ull)) return fail();
  const unsigned long long F = __ldg(reinterpret_cast<const unsigned int*>(in + zp));
  if (idx + F > mine - 8ull * H) return fail();
  const unsigned long long fz = zp + idx;  // the frame
  const uint32_t e1 = __ldg(reinterpret_cast<const unsigned int*>(in + zp + 4ull + 4ull * j));
  const uint32_t e0 = j ? __ldg(reinterpret_cast<const unsigned int*>(in + zp + 4ull * j)) : kZFrameHdr;
  if (e0 < kZFrameHdr || e1 <= e0 || e1 > F || e1 - e0 < 4u || e1 - e0 > 3u + kZBlock || (j + 1 == nblk && e1 != F))
    return fail();
  if (j == 0) {
    bool hb = false;
    const uint8_t want[5] = {0x28, 0xB5, 0x2F, 0xFD, 0xA0};
    for (uint32_t i = 0; i < 5; i++) hb |= in_byte(in, fz + i) != want[i];
    uint32_t fcs = 0;
    for (uint32_t i = 0; i < 4; i++) fcs |= (uint32_t)in_byte(in, fz + 5 + i) << (8 * i);
    if (hb || fcs != n) return fail();
  }
  const unsigned long long b = fz + e0;
  const uint32_t bh = in_byte(in, b) | ((uint32_t)in_byte(in, b + 1) << 8) | ((uint32_t)in_byte(in, b + 2) << 16);
  const uint32_t last = bh & 1u, type = (bh >> 1) & 3u, bsize = bh >> 3;
  if (last != (j + 1 == nblk ? 1u : 0u)) return fail();
  if (type == 0u) {  // Raw
    if (bsize != m || e1 - e0 != 3u + m) return fail();
    for (uint32_t i = lane; i < m; i += 32) dst[i] = in_byte(in, b + 3 + i);
    return;
  }
  if (type == 1u) {  // RLE
    if (bsize != m || e1 - e0 != 4u) return fail();
    const uint8_t v = in_byte(in, b + 3);
    for (uint32_t i = lane; i < m; i += 32) dst[i] = v;
    return;
  }
  if (type != 2u || e1 - e0 != 3u + bsize) return fail();
  // ---- Compressed: stage the content (the aligned words that hold it: the
  //      section, and so its last word, ends on a 4-byte boundary inside in),
  //      headers and tree on lane 0
  const unsigned long long c0 = b + 3;
  const uint32_t blk_at = (uint32_t)(c0 & 3ull), nwords = (blk_at + bsize + 3u) / 4u;
  const unsigned int* cw = reinterpret_cast<const unsigned int*>(in + (c0 - blk_at));
#pragma unroll 8
  for (uint32_t i = lane; i < nwords; i += 32) z.blkw[i] = __ldg(cw + i);
  for (uint32_t i = nwords + lane; i < nwords + 24u && i < kBlkWords; i += 32) z.blkw[i] = 0u;  // zero slack for the peeks
  __syncwarp();
  uint8_t* blk = reinterpret_cast<uint8_t*>(z.blkw) + blk_at;
  for (uint32_t i = lane; i < 256; i += 32) z.weight[i] = 0;
  __syncwarp();
  if (lane == 0) {
    uint32_t ok = 0;
    const uint32_t lt = blk[0] & 3u, sf = (blk[0] >> 2) & 3u;
    const uint32_t lhdr = sf <= 1u ? 3u : (sf == 2u ? 4u : 5u), bits = sf <= 1u ? 10u : (sf == 2u ? 14u : 18u);
    if (lt == 2u && lhdr + 1u <= bsize) {
      unsigned long long h = 0;
      for (uint32_t i = 0; i < lhdr; i++) h |= (unsigned long long)blk[i] << (8 * i);
      const uint32_t rs = (uint32_t)((h >> 4) & ((1u << bits) - 1u));
      const uint32_t cs = (uint32_t)((h >> (4 + bits)) & ((1u << bits) - 1u));
      if (rs == m && lhdr + cs + 1u == bsize && blk[lhdr + cs] == 0) {
        const uint32_t tu = read_tree(z, blk + lhdr, cs);
        if (tu) {
          ok = 1;
          z.tree_len = tu;
          z.sf = sf;
          z.cs = cs;
          z.lhdr = lhdr;
        }
      }
    }
    z.ok = ok;
  }
  __syncwarp();
  if (!z.ok || !tree_weights(z, lane)) return fail();
  // decoding table: the symbols of weight w, by value, take consecutive
  // ranges of 2^(w-1) entries after those of the lower weights
  const uint32_t mb = z.maxbits;
  {
    uint32_t base = 0, pos = 0;
    for (uint32_t w = 1; w <= mb; w++) {
      uint32_t cw = 0;
      for (uint32_t r = 0; r < 8; r++) {
        const uint32_t s = 32u * r + lane;
        const bool is = z.weight[s] == w;
        const uint32_t msk = __ballot_sync(0xffffffffu, is);
        if (is) z.sorted[pos + cw + __popc(msk & ((1u << lane) - 1u))] = (uint8_t)s;
        cw += __popc(msk);
      }
      if (lane == 0) {
        z.cls_base[w] = base;
        z.cls_pos[w] = pos;
        z.cls_cnt[w] = cw;
      }
      base += cw << (w - 1u);
      pos += cw;
    }
    if (base != (1u << mb)) return fail();
  }
  __syncwarp();
  for (uint32_t w = 1; w <= mb; w++) {
    const uint32_t sh = w - 1u, total = z.cls_cnt[w] << sh, b = z.cls_base[w], p0 = z.cls_pos[w];
    const uint32_t lenbits = (mb + 1u - w) << 8;
    for (uint32_t e = lane; e < total; e += 32u) z.dt[b + e] = (uint16_t)(z.sorted[p0 + (e >> sh)] | lenbits);
  }
  __syncwarp();
  // ---- the streams, one lane each
  const uint8_t* lit = blk + z.lhdr;
  const uint32_t tl = z.tree_len, cs = z.cs;
  bool ok = true;
  if (z.sf == 0u) {
    if (lane == 0) ok = read_stream(z, lit + tl, cs - tl, dst, m);
  } else {
    if (tl + 6u > cs) return fail();
    uint32_t sz[4];
    for (uint32_t k = 0; k < 3; k++) sz[k] = lit[tl + 2 * k] | ((uint32_t)lit[tl + 2 * k + 1] << 8);
    const uint32_t rest = cs - tl - 6u;
    const uint32_t seg = (m + 3u) / 4u;
    if (sz[0] + sz[1] + sz[2] > rest || 3u * seg > m) return fail();
    sz[3] = rest - sz[0] - sz[1] - sz[2];
    if (lane < 4) {
      uint32_t off = tl + 6u;
      for (uint32_t k = 0; k < lane; k++) off += sz[k];
      const uint32_t l0 = lane * seg, l1 = lane < 3 ? l0 + seg : m;
      ok = read_stream(z, lit + off, sz[lane], dst + l0, l1 - l0);
    }
  }
  if (__any_sync(0xffffffffu, !ok)) fail();
}

}  // namespace

int launch_zstd_encode(const EncParams& p, void* stream) {
  if (!p.zblk || !p.zmax_blk) return 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_zstd_enc<<<dim3(p.n_sec, p.zmax_blk), kZT, 0, st>>>(p);
  return (int)cudaGetLastError();
}

int launch_zstd_decode(const DecParams& p, void* stream) {
  if (!p.zdec || !p.zmax_blk) return 0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_zstd_dec<<<dim3(p.n_sec, p.zmax_blk), 32, 0, st>>>(p);
  return (int)cudaGetLastError();
}

}  // namespace jiffy
