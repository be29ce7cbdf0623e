/*
 * Zstandard frames for the zero mask: a plain writer and reader of the part
 * of the Zstandard format (RFC 8878) that the Jiffy oracle uses.
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of the oracle: the test suite, the
 * smoke check and the benchmark's CPU baseline load it; the library never
 * calls it, and it shares nothing with the CUDA path.
 *
 * The paper packs the zero bitmask into bytes and compresses it with Zstd
 * (Sec. III-C); a P scan's mask is XORed with the previous scan's first
 * (Sec. III-D). The frames written here are ordinary Zstandard frames, so any
 * Zstandard decoder restores them (the tests check every one with libzstd's
 * ZSTD_decompress). They use this subset of the format:
 *   frame header: magic, a descriptor with Single_Segment_flag set and a
 *     4-byte Frame_Content_Size, no checksum, no dictionary (RFC 8878 3.1.1.1)
 *   one block per 8192 input bytes (the last one shorter), each of them
 *     RLE     if all its bytes are equal,
 *     Compressed, made of a Huffman-coded literals section and no sequences
 *             (Number_of_Sequences = 0), if that is smaller than the input,
 *     Raw     otherwise (RFC 8878 3.1.1.2)
 *   literals: one Huffman stream for blocks of at most 1023 bytes, four
 *     streams with a jump table above that (RFC 8878 3.1.1.3.1)
 *   Huffman tree description: weights written directly (4 bits each) when at
 *     most 128 weights are listed, else FSE-compressed with accuracy log 6
 *     and two interleaved states (RFC 8878 4.2.1); a block whose weights
 *     cannot be written either way is stored Raw.
 * Every choice the format leaves to the writer is fixed below so that another
 * implementation of the same rules writes the same bytes:
 *   - Huffman code lengths: two-queue Huffman construction over the present
 *     symbols sorted by (count, value), a tie taking the leaf; if a length
 *     exceeds 11 every count c becomes ceil(c/2) and the construction is
 *     repeated;
 *   - FSE normalisation of the weight histogram (table size 64): each present
 *     weight value gets max(1, floor(64 c / N)); the value with the largest
 *     count (the smallest value among equal counts) takes the rest, and the
 *     block is stored Raw if that leaves it below 1;
 *   - FSE initial states: the lowest table position holding the symbol.
 * The reader accepts exactly what the writer can produce (and the parts of
 * the literals-section header any writer may choose) and rejects the rest;
 * in particular block j must hold input bytes 8192 j .. 8192 (j+1) - 1, so
 * that a block-end index lets every block be decoded on its own.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define JZ_BLOCK 8192u  /* input bytes per block */
#define JZ_MAXBITS 11u  /* longest Huffman code (RFC 8878: Max_Number_of_Bits <= 11) */
#define JZ_FSE_LOG 6u   /* accuracy log of the weights' FSE table (at most 6 for weights) */
#define JZ_FRAME_HDR 9u /* magic (4) + descriptor (1) + Frame_Content_Size (4) */

static uint32_t highbit(uint32_t x) { /* index of the highest set bit, x > 0 */
  uint32_t h = 0;
  while (x >>= 1) h++;
  return h;
}

/* ------------------------------------------------------------------ */
/* Bit streams. A Zstandard "backward" bit stream is laid out forward,  */
/* least significant bit first, and read from its end: the last field   */
/* written is the first one read, and a field read as n bits has its    */
/* most significant bit at the higher position. The writer closes it    */
/* with a single 1 bit and zero bits up to the next byte.               */
/* ------------------------------------------------------------------ */
typedef struct {
  uint8_t* buf;
  size_t cap;    /* bytes */
  uint64_t bits; /* bits written */
  int full;      /* a write went past cap */
} bitw;

static void bw_put(bitw* w, uint32_t value, uint32_t n) {
  for (uint32_t i = 0; i < n; i++) {
    uint64_t at = w->bits + i;
    if (at / 8 >= w->cap) { w->full = 1; continue; }
    if ((value >> i) & 1u) w->buf[at / 8] |= (uint8_t)(1u << (at % 8));
  }
  w->bits += n;
}

static size_t bw_close(bitw* w) { /* end mark, returns the bytes used */
  bw_put(w, 1u, 1u);
  return (size_t)((w->bits + 7) / 8);
}

/* n bits ending at bit position p (exclusive) of a backward stream, bits
 * below position 0 read as zero */
static uint32_t br_peek(const uint8_t* s, int64_t p, uint32_t n) {
  uint32_t v = 0;
  for (uint32_t i = 0; i < n; i++) {
    int64_t at = p - 1 - (int64_t)i; /* the i-th bit read, most significant first */
    uint32_t bit = at >= 0 ? (s[at / 8] >> (at % 8)) & 1u : 0u;
    v = (v << 1) | bit;
  }
  return v;
}

/* payload bits of a backward stream (position of its end mark), or -1 */
static int64_t br_start(const uint8_t* s, size_t len) {
  if (len == 0 || s[len - 1] == 0) return -1;
  return (int64_t)(8 * (len - 1) + highbit(s[len - 1]));
}

/* ------------------------------------------------------------------ */
/* Huffman code lengths (RFC 8878 4.2.1 fixes the code given lengths;   */
/* the lengths are the writer's choice, fixed in the header comment).   */
/* ------------------------------------------------------------------ */
static void huff_lengths(const uint32_t* count, uint8_t* len) {
  uint64_t c[256];
  for (int s = 0; s < 256; s++) c[s] = count[s];
  for (;;) {
    int sym[256], n = 0;
    for (int s = 0; s < 256; s++) {
      if (!c[s]) continue;
      int i = n++; /* insertion sort by (count, value) */
      while (i > 0 && c[sym[i - 1]] > c[s]) { sym[i] = sym[i - 1]; i--; }
      sym[i] = s;
    }
    uint64_t w[511];
    int parent[511], depth[511];
    for (int i = 0; i < n; i++) w[i] = c[sym[i]];
    int leaf = 0, node = n, next = n; /* leaf queue head, internal queue head, next node */
    for (int k = 0; k < n - 1; k++) {
      int pick[2];
      for (int j = 0; j < 2; j++) {
        if (leaf < n && (node >= next || w[leaf] <= w[node])) pick[j] = leaf++;
        else pick[j] = node++;
      }
      w[next] = w[pick[0]] + w[pick[1]];
      parent[pick[0]] = parent[pick[1]] = next;
      next++;
    }
    depth[next - 1] = 0;
    for (int i = next - 2; i >= 0; i--) depth[i] = depth[parent[i]] + 1;
    int maxd = 0;
    memset(len, 0, 256);
    for (int i = 0; i < n; i++) {
      len[sym[i]] = (uint8_t)depth[i];
      if (depth[i] > maxd) maxd = depth[i];
    }
    if (maxd <= (int)JZ_MAXBITS) return;
    for (int s = 0; s < 256; s++) c[s] = (c[s] + 1) / 2;
  }
}

/* Canonical codes from weights (RFC 8878 4.2.1): the symbols with a
 * nonzero weight, sorted by weight then value, take consecutive ranges of
 * the 2^maxbits-entry decoding table, 2^(weight-1) entries each, starting at
 * entry 0; a symbol's code is its first entry >> (weight - 1). */
static void huff_codes(const uint8_t* weight, uint32_t maxbits, uint32_t* code) {
  uint32_t pos = 0;
  for (uint32_t wt = 1; wt <= maxbits; wt++) {
    for (int s = 0; s < 256; s++) {
      if (weight[s] != wt) continue;
      code[s] = pos >> (wt - 1);
      pos += 1u << (wt - 1);
    }
  }
}

/* ------------------------------------------------------------------ */
/* FSE (RFC 8878 4.1). The decoding table of a normalised distribution   */
/* (counts summing to 2^log, no "less than 1" entries): symbols spread   */
/* with step (size/2 + size/8 + 3); position u holding symbol s gets the */
/* next of s's counters x (starting at count[s]), nb = log - highbit(x)  */
/* bits and baseline (x << nb) - size.                                   */
/* ------------------------------------------------------------------ */
typedef struct {
  uint8_t sym[64], nb[64];
  uint16_t base[64];
} fse_table;

static void fse_build(const uint32_t* norm, uint32_t nsym, uint32_t log, fse_table* t) {
  uint32_t size = 1u << log, step = (size >> 1) + (size >> 3) + 3, pos = 0;
  for (uint32_t s = 0; s < nsym; s++) {
    for (uint32_t i = 0; i < norm[s]; i++) {
      t->sym[pos] = (uint8_t)s;
      pos = (pos + step) & (size - 1);
    }
  }
  uint32_t next[16];
  for (uint32_t s = 0; s < nsym; s++) next[s] = norm[s];
  for (uint32_t u = 0; u < size; u++) {
    uint32_t x = next[t->sym[u]]++;
    t->nb[u] = (uint8_t)(log - highbit(x));
    t->base[u] = (uint16_t)((x << t->nb[u]) - size);
  }
}

/* FSE table description (RFC 8878 4.1.1), written forward (LSB first):
 * accuracy log - 5 in 4 bits, then count + 1 per symbol value with the
 * variable-size code the decoder expects given the probability points left,
 * a zero count followed by 2-bit repeat flags for the run of zero counts
 * after it. Stops once all points are given out. */
static void fse_write_ncount(bitw* w, const uint32_t* norm, uint32_t nsym, uint32_t log) {
  bw_put(w, log - 5u, 4u);
  uint32_t remaining = (1u << log) + 1u; /* the largest value count + 1 can still take, plus one */
  uint32_t s = 0;
  while (remaining > 1 && s < nsym) {
    uint32_t v = norm[s] + 1u; /* value written: count + 1 */
    uint32_t nbits = highbit(remaining) + 1u, thr = 1u << (nbits - 1);
    uint32_t lo = 2u * thr - 1u - remaining; /* values below lo take nbits - 1 bits */
    if (v < lo) bw_put(w, v, nbits - 1u);
    else if (v < thr) bw_put(w, v, nbits);
    else bw_put(w, v + lo, nbits);
    remaining -= norm[s];
    s++;
    if (norm[s - 1] == 0) { /* repeat flags: the zero counts that follow */
      uint32_t z = 0;
      while (s + z < nsym && norm[s + z] == 0) z++;
      s += z;
      while (z >= 24) { bw_put(w, 0xFFFFu, 16u); z -= 24; }
      while (z >= 3) { bw_put(w, 3u, 2u); z -= 3; }
      bw_put(w, z, 2u);
    }
  }
}

/* Huffman tree description with FSE-compressed weights (RFC 8878 4.2.1.2):
 * returns its bytes in out (header byte first), or 0 if it cannot be
 * written (fewer than two distinct values, normalisation failure, or 128
 * bytes or more). */
static size_t fse_weights(const uint8_t* wt, uint32_t n, uint8_t* out) {
  uint32_t hist[16] = {0}, nsym = 0, best = 0;
  for (uint32_t i = 0; i < n; i++) hist[wt[i]]++;
  uint32_t distinct = 0;
  for (uint32_t v = 0; v < 16; v++) {
    if (!hist[v]) continue;
    distinct++;
    nsym = v + 1;
    if (hist[v] > hist[best]) best = v;
  }
  if (distinct < 2 || n < 2) return 0;
  uint32_t norm[16] = {0}, sum = 0;
  for (uint32_t v = 0; v < nsym; v++) {
    if (!hist[v]) continue;
    norm[v] = (uint32_t)(((uint64_t)hist[v] << JZ_FSE_LOG) / n);
    if (norm[v] < 1) norm[v] = 1;
    sum += norm[v];
  }
  int64_t rest = (int64_t)norm[best] + (int64_t)(1u << JZ_FSE_LOG) - (int64_t)sum;
  if (rest < 1) return 0;
  norm[best] = (uint32_t)rest;
  fse_table t;
  fse_build(norm, nsym, JZ_FSE_LOG, &t);
  uint8_t tmp[256];
  memset(tmp, 0, sizeof tmp);
  bitw w = {tmp, 127, 0, 0};
  fse_write_ncount(&w, norm, nsym, JZ_FSE_LOG);
  size_t head = (size_t)((w.bits + 7) / 8);
  /* the two states, walked from the last weight back to the first: weight
   * i is emitted by state i % 2; each emitted weight's state was reached
   * from the next state of the same parity */
  uint32_t state[2] = {0, 0}, fv[256], fn[256];
  for (int64_t i = (int64_t)n - 1; i >= 0; i--) {
    uint32_t p = (uint32_t)i & 1u, s = wt[i];
    if (i >= (int64_t)n - 2) {
      uint32_t u = 0;
      while (t.sym[u] != s) u++;
      state[p] = u;
      continue;
    }
    uint32_t v = state[p], u = 0;
    while (!(t.sym[u] == s && t.base[u] <= v && v < (uint32_t)t.base[u] + (1u << t.nb[u]))) u++;
    fv[i] = v - t.base[u];
    fn[i] = t.nb[u];
    state[p] = u;
  }
  /* read order: state of weight 0, state of weight 1, then the bits after
   * weights 0, 1, ..., n-3; written in the reverse order */
  bitw b = {tmp + head, 127 - head, 0, 0};
  for (int64_t i = (int64_t)n - 3; i >= 0; i--) bw_put(&b, fv[i], fn[i]);
  bw_put(&b, state[1], JZ_FSE_LOG);
  bw_put(&b, state[0], JZ_FSE_LOG);
  size_t body = bw_close(&b);
  if (w.full || b.full || head + body >= 128) return 0;
  out[0] = (uint8_t)(head + body);
  memcpy(out + 1, tmp, head + body);
  return 1 + head + body;
}

/* One Huffman stream of literals lit[0..n) (read from the end: the first
 * literal's code is the last field written). */
static size_t huff_stream(const uint8_t* lit, uint32_t n, const uint32_t* code, const uint8_t* len, uint8_t* out,
                          size_t cap, int* full) {
  bitw w = {out, cap, 0, 0};
  for (int64_t i = (int64_t)n - 1; i >= 0; i--) bw_put(&w, code[lit[i]], len[lit[i]]);
  size_t k = bw_close(&w);
  if (w.full) *full = 1;
  return k;
}

static void put_le(uint8_t* p, uint64_t v, uint32_t bytes) {
  for (uint32_t i = 0; i < bytes; i++) p[i] = (uint8_t)(v >> (8 * i));
}
static uint64_t get_le(const uint8_t* p, uint32_t bytes) {
  uint64_t v = 0;
  for (uint32_t i = 0; i < bytes; i++) v |= (uint64_t)p[i] << (8 * i);
  return v;
}

/* Content of a Compressed block holding src[0..n) as Huffman literals and no
 * sequences, or 0 if it cannot be written or is not smaller than n. */
static size_t compressed_block(const uint8_t* src, uint32_t n, uint8_t* out) {
  uint32_t count[256] = {0};
  for (uint32_t i = 0; i < n; i++) count[src[i]]++;
  uint8_t len[256];
  huff_lengths(count, len);
  uint32_t maxbits = 0, last = 0;
  for (uint32_t s = 0; s < 256; s++) {
    if (len[s] > maxbits) maxbits = len[s];
    if (len[s]) last = s;
  }
  uint8_t weight[256];
  for (uint32_t s = 0; s < 256; s++) weight[s] = len[s] ? (uint8_t)(maxbits + 1u - len[s]) : 0;
  uint32_t code[256] = {0};
  huff_codes(weight, maxbits, code);
  /* tree description: weights of symbols 0 .. last-1 (the last one is implied) */
  uint8_t* lit = (uint8_t*)calloc((size_t)n + 256u, 1);
  size_t tree;
  if (last <= 128) {
    lit[0] = (uint8_t)(127u + last);
    for (uint32_t i = 0; i < last; i++) lit[1 + i / 2] |= (uint8_t)(weight[i] << ((i % 2) ? 0 : 4));
    tree = 1u + (last + 1u) / 2u;
  } else {
    tree = fse_weights(weight, last, lit);
    if (!tree) { free(lit); return 0; }
  }
  int four = n > 1023u, full = 0;
  size_t pos = tree;
  if (!four) {
    pos += huff_stream(src, n, code, len, lit + pos, n - pos > n ? 0 : n - pos, &full);
  } else {
    uint32_t seg = (n + 3u) / 4u;
    size_t jt = pos;
    pos += 6;
    for (uint32_t k = 0; k < 4 && !full; k++) {
      uint32_t lo = k * seg, hi = k < 3 ? lo + seg : n;
      size_t room = pos < n ? n - pos : 0;
      size_t sz = huff_stream(src + lo, hi - lo, code, len, lit + pos, room, &full);
      if (k < 3) {
        if (sz > 0xFFFFu) full = 1;
        put_le(lit + jt + 2u * k, sz, 2);
      }
      pos += sz;
    }
  }
  size_t lhdr = four ? (n <= 16383u ? 4u : 5u) : 3u;
  size_t content = lhdr + pos + 1u; /* literals section + Number_of_Sequences = 0 */
  if (full || content >= n) { free(lit); return 0; }
  uint64_t h;
  if (!four) h = 2u | (0u << 2) | ((uint64_t)n << 4) | ((uint64_t)pos << 14);
  else if (lhdr == 4) h = 2u | (2u << 2) | ((uint64_t)n << 4) | ((uint64_t)pos << 18);
  else h = 2u | (3u << 2) | ((uint64_t)n << 4) | ((uint64_t)pos << 22);
  put_le(out, h, (uint32_t)lhdr);
  memcpy(out + lhdr, lit, pos);
  out[lhdr + pos] = 0;
  free(lit);
  return content;
}

/* Bytes jz_write_frame may need for n input bytes. */
size_t jz_frame_bound(size_t n) {
  size_t nblk = n ? (n + JZ_BLOCK - 1) / JZ_BLOCK : 1;
  return JZ_FRAME_HDR + 3u * nblk + n;
}

size_t jz_block_count(size_t n) { return n ? (n + JZ_BLOCK - 1) / JZ_BLOCK : 1; }

/* Writes src[0..n) (1 <= n < 2^32) as one frame; returns its bytes (at most
 * jz_frame_bound(n)); ends (nullable) receives the end of each block, in
 * bytes from the frame's start. */
size_t jz_write_frame(const uint8_t* src, size_t n, uint8_t* dst, uint32_t* ends) {
  put_le(dst, 0xFD2FB528u, 4);
  dst[4] = 0xA0; /* Frame_Content_Size_flag 2 (4 bytes), Single_Segment_flag */
  put_le(dst + 5, n, 4);
  size_t pos = JZ_FRAME_HDR;
  size_t nblk = jz_block_count(n);
  uint8_t* tmp = (uint8_t*)malloc(JZ_BLOCK + 64u);
  for (size_t j = 0; j < nblk; j++) {
    const uint8_t* b = src + j * JZ_BLOCK;
    uint32_t m = (uint32_t)(n - j * JZ_BLOCK < JZ_BLOCK ? n - j * JZ_BLOCK : JZ_BLOCK);
    uint32_t last = j + 1 == nblk ? 1u : 0u;
    int same = 1;
    for (uint32_t i = 1; i < m; i++) if (b[i] != b[0]) { same = 0; break; }
    if (same) {
      put_le(dst + pos, last | (1u << 1) | ((uint64_t)m << 3), 3);
      dst[pos + 3] = b[0];
      pos += 4;
    } else {
      memset(tmp, 0, JZ_BLOCK + 64u);
      size_t c = compressed_block(b, m, tmp);
      if (c) {
        put_le(dst + pos, last | (2u << 1) | ((uint64_t)c << 3), 3);
        memcpy(dst + pos + 3, tmp, c);
        pos += 3 + c;
      } else {
        put_le(dst + pos, last | (0u << 1) | ((uint64_t)m << 3), 3);
        memcpy(dst + pos + 3, b, m);
        pos += 3 + m;
      }
    }
    if (ends) ends[j] = (uint32_t)pos;
  }
  free(tmp);
  return pos;
}

/* ------------------------------------------------------------------ */
/* Reader                                                               */
/* ------------------------------------------------------------------ */

/* Huffman weights: direct or FSE-compressed. Returns the bytes used, 0 on
 * error; weight[0..255] receives all weights (the implied one included),
 * *maxbits the code length limit. */
static size_t read_tree(const uint8_t* s, size_t len, uint8_t* weight, uint32_t* maxbits) {
  if (len < 1) return 0;
  uint32_t hb = s[0], n;
  size_t used;
  memset(weight, 0, 256);
  if (hb >= 128) {
    n = hb - 127u;
    used = 1u + (n + 1u) / 2u;
    if (used > len) return 0;
    for (uint32_t i = 0; i < n; i++) weight[i] = (uint8_t)((s[1 + i / 2] >> ((i % 2) ? 0 : 4)) & 15u);
  } else {
    used = 1u + hb;
    if (used > len || hb == 0) return 0;
    const uint8_t* f = s + 1;
    /* table description, read forward */
    uint64_t bp = 0, fbits = 8ull * hb;
    uint32_t log = (uint32_t)(f[0] & 15u) + 5u;
    bp = 4;
    if (log > JZ_FSE_LOG) return 0;
    uint32_t norm[16] = {0}, nsym = 0, remaining = (1u << log) + 1u;
    while (remaining > 1) {
      if (nsym >= 16) return 0;
      uint32_t nbits = highbit(remaining) + 1u, thr = 1u << (nbits - 1), lo = 2u * thr - 1u - remaining, v = 0;
      if (bp + nbits > fbits) return 0;
      for (uint32_t i = 0; i < nbits; i++) v |= (uint32_t)((f[(bp + i) / 8] >> ((bp + i) % 8)) & 1u) << i;
      if ((v & (thr - 1u)) < lo) { v &= thr - 1u; bp += nbits - 1; }
      else { if (v >= thr) v -= lo; bp += nbits; }
      if (v == 0) return 0; /* "less than 1" probabilities are not written */
      uint32_t cnt = v - 1u;
      if (cnt > remaining - 1u) return 0;
      norm[nsym++] = cnt;
      remaining -= cnt;
      if (cnt == 0) {
        for (;;) {
          if (bp + 2 > fbits) return 0;
          uint32_t rep = (f[bp / 8] >> (bp % 8)) & 1u;
          rep |= (uint32_t)((f[(bp + 1) / 8] >> ((bp + 1) % 8)) & 1u) << 1;
          bp += 2;
          if (nsym + rep > 16) return 0;
          for (uint32_t i = 0; i < rep; i++) norm[nsym++] = 0;
          if (rep != 3) break;
        }
      }
    }
    if (remaining != 1) return 0;
    size_t head = (size_t)((bp + 7) / 8);
    if (head >= hb) return 0;
    fse_table t;
    fse_build(norm, nsym, log, &t);
    const uint8_t* bs = f + head;
    int64_t p = br_start(bs, hb - head);
    if (p < 2 * (int64_t)log) return 0;
    uint32_t st[2];
    st[0] = br_peek(bs, p, log); p -= log;
    st[1] = br_peek(bs, p, log); p -= log;
    n = 0;
    for (uint32_t k = 0;; k ^= 1u) {
      if (n >= 255) return 0;
      weight[n++] = t.sym[st[k]];
      uint32_t nb = t.nb[st[k]];
      if (p < (int64_t)nb) { /* past the start: the other state gives the last weight */
        if (n >= 255) return 0;
        weight[n++] = t.sym[st[k ^ 1u]];
        break;
      }
      st[k] = t.base[st[k]] + br_peek(bs, p, nb);
      p -= nb;
    }
  }
  uint32_t sum = 0;
  for (uint32_t i = 0; i < n; i++) {
    if (weight[i] > JZ_MAXBITS) return 0;
    if (weight[i]) sum += 1u << (weight[i] - 1u);
  }
  if (sum == 0 || n > 255) return 0;
  uint32_t mb = highbit(sum) + 1u, rest = (1u << mb) - sum;
  if (mb > JZ_MAXBITS || (rest & (rest - 1u))) return 0;
  weight[n] = (uint8_t)(highbit(rest) + 1u);
  *maxbits = mb;
  return used;
}

static int read_stream(const uint8_t* s, size_t len, const uint8_t* dsym, const uint8_t* dlen, uint32_t maxbits,
                       uint8_t* out, uint32_t n) {
  int64_t p = br_start(s, len);
  if (p < 0) return -1;
  for (uint32_t i = 0; i < n; i++) {
    uint32_t v = br_peek(s, p, maxbits);
    out[i] = dsym[v];
    p -= dlen[v];
    if (p < 0) return -1;
  }
  return p == 0 ? 0 : -1;
}

/* Reads one frame of the subset above holding exactly n bytes into dst.
 * Returns the frame's bytes, or 0 if it is malformed or outside the subset.
 * ends (nullable, one entry per block) receives the end of each block. */
size_t jz_read_frame(const uint8_t* src, size_t len, uint8_t* dst, size_t n, uint32_t* ends, size_t max_blocks) {
  if (len < JZ_FRAME_HDR || get_le(src, 4) != 0xFD2FB528u || src[4] != 0xA0 || get_le(src + 5, 4) != n) return 0;
  size_t pos = JZ_FRAME_HDR, out = 0, nb = 0;
  for (;;) {
    if (pos + 3 > len || nb >= max_blocks) return 0;
    uint32_t bh = (uint32_t)get_le(src + pos, 3);
    uint32_t last = bh & 1u, type = (bh >> 1) & 3u, bsize = bh >> 3;
    size_t want = n - out < JZ_BLOCK ? n - out : JZ_BLOCK; /* this block's share of the input */
    if (want == 0 || last != (out + want == n)) return 0;
    pos += 3;
    if (type == 0) {
      if (bsize != want || bsize > len - pos) return 0;
      memcpy(dst + out, src + pos, bsize);
      out += bsize;
      pos += bsize;
    } else if (type == 1) {
      if (bsize != want || pos + 1 > len) return 0;
      memset(dst + out, src[pos], bsize);
      out += bsize;
      pos += 1;
    } else if (type == 2) {
      if (bsize > len - pos || bsize < 4) return 0;
      const uint8_t* b = src + pos;
      uint32_t lt = b[0] & 3u, sf = (b[0] >> 2) & 3u, lhdr, rs, cs;
      if (lt != 2) return 0;
      lhdr = sf <= 1 ? 3u : (sf == 2 ? 4u : 5u);
      if (lhdr > bsize) return 0;
      uint64_t h = get_le(b, lhdr);
      uint32_t bits = sf <= 1 ? 10u : (sf == 2 ? 14u : 18u);
      rs = (uint32_t)((h >> 4) & ((1u << bits) - 1u));
      cs = (uint32_t)((h >> (4 + bits)) & ((1u << bits) - 1u));
      if (rs != want || (uint64_t)lhdr + cs + 1u != bsize || b[lhdr + cs] != 0) return 0;
      const uint8_t* l = b + lhdr;
      uint8_t weight[256];
      uint32_t maxbits = 0;
      size_t tu = read_tree(l, cs, weight, &maxbits);
      if (!tu) return 0;
      /* decoding table: 2^maxbits entries, symbols by weight then value */
      uint8_t dsym[1u << JZ_MAXBITS], dlen[1u << JZ_MAXBITS];
      uint32_t e = 0;
      for (uint32_t wt = 1; wt <= maxbits; wt++) {
        for (uint32_t s = 0; s < 256; s++) {
          if (weight[s] != wt) continue;
          for (uint32_t i = 0; i < (1u << (wt - 1)); i++) {
            dsym[e] = (uint8_t)s;
            dlen[e] = (uint8_t)(maxbits + 1u - wt);
            e++;
          }
        }
      }
      if (e != (1u << maxbits)) return 0;
      if (sf == 0) {
        if (read_stream(l + tu, cs - tu, dsym, dlen, maxbits, dst + out, rs)) return 0;
      } else {
        if (tu + 6 > cs) return 0;
        const uint8_t* jt = l + tu;
        size_t sz[4], at = tu + 6;
        sz[0] = get_le(jt, 2); sz[1] = get_le(jt + 2, 2); sz[2] = get_le(jt + 4, 2);
        if (sz[0] + sz[1] + sz[2] > cs - at) return 0;
        sz[3] = cs - at - sz[0] - sz[1] - sz[2];
        uint32_t seg = (rs + 3u) / 4u;
        if (3u * seg > rs) return 0; /* every stream holds a literal */
        for (uint32_t k = 0; k < 4; k++) {
          uint32_t lo = k * seg, hi = k < 3 ? lo + seg : rs;
          if (read_stream(l + at, sz[k], dsym, dlen, maxbits, dst + out + lo, hi - lo)) return 0;
          at += sz[k];
        }
      }
      out += rs;
      pos += bsize;
    } else {
      return 0;
    }
    if (ends) ends[nb] = (uint32_t)pos;
    nb++;
    if (last) break;
  }
  return out == n ? pos : 0;
}
