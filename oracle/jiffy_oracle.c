/*
 * Jiffy oracle: a plain, slow, single-threaded CPU encoder and decoder for the
 * Jiffy LiDAR range/attribute scan codec (Ford & Ford, arXiv 2209.08196).
 *
 * TEST INFRASTRUCTURE ONLY. This is the reference the CUDA path is checked
 * against. Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg load it; the library's encode/decode path never calls it. It
 * shares no code, header, table or constant with the CUDA implementation.
 *
 * One whole-array pass per step, in the paper's order:
 *   quantize          Sec. III-A / III-B
 *   zero bitmask      Sec. III-C (bit = 1 for an out-of-range, zero sample)
 *   I/P mode          Sec. III-E (trial compression of a few scanlines,
 *                     mask excluded), validated in Sec. IV-E (4 test lines)
 *   mask section      Sec. III-C (I) and Sec. III-D (P: XOR with the
 *                     previous scan's mask)
 *   compaction        Sec. III-C (remove masked samples -> flat 1D vector)
 *   residual          I: the value; P: value minus the previous scan's value
 *                     at the same pixel, Sec. III-D
 *   delta             Sec. III-C (each sample minus its left neighbour in
 *                     the flat vector)
 *   ZigZag            Eq. 1, taken modulo 2^32
 *   integer packing   frames of 128 integers, low bits packed, wide values
 *                     in a separate exception list (PFOR, Sec. II)
 * The decoder runs the same steps backwards (Sec. III-C, "straightforward
 * reversal").
 *
 * Ablation switches (Sec. IV-H, Table IV): a stream may drop the zero mask
 * (every sample is coded, zeros included), the horizontal delta (residuals
 * packed as they are) or ZigZag (deltas packed as 32-bit two's complement
 * words); with I forced as well, the four ablated codecs of Table IV are
 * SIMD-PFOR alone, Delta -> PFOR, Delta -> ZigZag -> PFOR and
 * Mask -> Delta -> ZigZag -> PFOR.
 *
 * The paper does not fix a byte layout; the layout written here (stream
 * header, frame header, per-attribute section with a row table, per-row
 * chunks, mask class words, block headers and bodies) is this project's and
 * is spelled out next to each writer below. All multi-byte fields are
 * little-endian; bit streams are least-significant-bit first.
 *
 * Parity: pinned by the tests in tests/test_oracle_pins.py (Eq. 1 values,
 * quantization error bound, round trips, hand-derived golden bytes, trial ==
 * brute force for H <= test lines, exhaustive block-width choice).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define JO_MAX_ATTR 64

enum { JO_OK = 0, JO_ERR_INVALID_ARG = 1, JO_ERR_CAPACITY = 2, JO_ERR_CORRUPT = 3 };

/* Stage switches of a stream (Table IV ablations); 0 = the full codec.
 * JO_ZSTD_MASK is not an ablation: it codes the mask the paper's way, one
 * Zstandard frame per section (Sec. III-C), instead of per-row class words. */
enum { JO_NO_MASK = 1, JO_NO_DELTA = 2, JO_NO_ZIGZAG = 4, JO_ZSTD_MASK = 8 };

/* the Zstandard writer and reader (jiffy_zstd_oracle.c) */
size_t jz_frame_bound(size_t n);
size_t jz_block_count(size_t n);
size_t jz_write_frame(const uint8_t* src, size_t n, uint8_t* dst, uint32_t* ends);
size_t jz_read_frame(const uint8_t* src, size_t len, uint8_t* dst, size_t n, uint32_t* ends, size_t max_blocks);

/* stage-flag byte of the stream header: bit 0 no mask, bit 1 no delta,
 * bit 2 Zstandard mask */
static uint8_t header_flags(uint32_t stages) {
  return (uint8_t)((stages & (JO_NO_MASK | JO_NO_DELTA)) | ((stages & JO_ZSTD_MASK) ? 4u : 0u));
}

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

static uint32_t dtype_max(uint32_t s) {
  return s == 4 ? 0xFFFFFFFFu : ((1u << (8 * s)) - 1u);
}

static uint32_t load_sample(const void* plane, uint32_t s, size_t i) {
  if (s == 1) return ((const uint8_t*)plane)[i];
  if (s == 2) return ((const uint16_t*)plane)[i];
  return ((const uint32_t*)plane)[i];
}

static void store_sample(void* plane, uint32_t s, size_t i, uint32_t v) {
  if (s == 1) ((uint8_t*)plane)[i] = (uint8_t)v;
  else if (s == 2) ((uint16_t*)plane)[i] = (uint16_t)v;
  else ((uint32_t*)plane)[i] = v;
}

static uint32_t ceil_div(uint32_t a, uint32_t b) { return (a + b - 1) / b; }

/* Number of bits needed to write x (0 for x == 0). */
static uint32_t bit_width(uint32_t x) {
  uint32_t w = 0;
  while (x) { w++; x >>= 1; }
  return w;
}

static void put_u16(uint8_t* p, uint32_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void put_u32(uint8_t* p, uint32_t v) {
  p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); p[2] = (uint8_t)(v >> 16); p[3] = (uint8_t)(v >> 24);
}
static uint32_t get_u16(const uint8_t* p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
static uint32_t get_u32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

/* Write the low nbits of value into a zeroed bit stream, one bit at a time,
 * least significant bit first: stream bit k is bit (k % 8) of byte k / 8. */
static void put_bits(uint8_t* base, uint64_t bitpos, uint32_t value, uint32_t nbits) {
  for (uint32_t k = 0; k < nbits; k++) {
    if ((value >> k) & 1u) {
      uint64_t p = bitpos + k;
      base[p / 8] |= (uint8_t)(1u << (p % 8));
    }
  }
}

static uint32_t get_bits(const uint8_t* base, uint64_t bitpos, uint32_t nbits) {
  uint32_t v = 0;
  for (uint32_t k = 0; k < nbits; k++) {
    uint64_t p = bitpos + k;
    if ((base[p / 8] >> (p % 8)) & 1u) v |= (1u << k);
  }
  return v;
}

/* ------------------------------------------------------------------ */
/* Quantization (Sec. III-A, III-B; error bound Sec. IV-G, Fig. 4)     */
/* q = floor((v + floor(P/2)) / P), i.e. round half up, computed in 64  */
/* bits, then clamped so that q * P still fits the sample type. The     */
/* decoder restores q * P.                                              */
/* ------------------------------------------------------------------ */

uint32_t jo_quantize(uint32_t v, uint32_t P, uint32_t s) {
  uint64_t q = ((uint64_t)v + (uint64_t)(P / 2)) / (uint64_t)P;
  uint64_t qmax = (uint64_t)dtype_max(s) / (uint64_t)P;
  if (q > qmax) q = qmax;
  return (uint32_t)q;
}

/* ------------------------------------------------------------------ */
/* ZigZag, Eq. 1: 2|x| + (1 if x < 0 else 0), taken modulo 2^32.       */
/* Residuals are 32-bit two's complement values; |-2^31| = 2^31, so     */
/* ZigZag(-2^31) = 2^32 + 1 = 1 (mod 2^32), the only odd value below 3. */
/* ------------------------------------------------------------------ */

uint32_t jo_zigzag(int32_t x) {
  uint32_t mag = x < 0 ? (uint32_t)(-(int64_t)x) : (uint32_t)x; /* |x| as an integer */
  return 2u * mag + (x < 0 ? 1u : 0u);                           /* modulo 2^32 */
}

int32_t jo_unzigzag(uint32_t z) {
  if ((z & 1u) == 0) return (int32_t)(z / 2u);
  if (z == 1u) return INT32_MIN;
  return (int32_t)(-(int64_t)((z - 1u) / 2u));
}

/* ------------------------------------------------------------------ */
/* PFOR-style block of up to 128 values (Sec. II: frames of 128         */
/* integers; values wider than the frame's bit width go to a separate   */
/* list). Layout of one block:                                          */
/*   header (4 bytes): b, e, hb, 0                                      */
/*     b  = bits kept for every value, e = number of exceptions         */
/*     hb = bits of each exception's high part (wmax - b, 0 if e == 0)  */
/*   body:                                                              */
/*     low part: the low b bits of each of the n values, bit stream,    */
/*               4*ceil(n*b/32) bytes                                   */
/*     if e > 0: e one-byte positions (ascending), zero-padded to a     */
/*               multiple of 4, then the high parts (z >> b) of the     */
/*               exceptions, hb bits each, 4*ceil(e*hb/32) bytes         */
/* b minimises the body size over 0..wmax; ties go to the smallest b.   */
/* ------------------------------------------------------------------ */

static uint32_t max_width(const uint32_t* z, uint32_t n) {
  uint32_t w = 0;
  for (uint32_t i = 0; i < n; i++) { uint32_t bw = bit_width(z[i]); if (bw > w) w = bw; }
  return w;
}

uint32_t jo_block_body_bytes(const uint32_t* z, uint32_t n, uint32_t b) {
  uint32_t wmax = max_width(z, n);
  uint32_t e = 0;
  for (uint32_t i = 0; i < n; i++) if (bit_width(z[i]) > b) e++;
  uint32_t bytes = 4u * ceil_div(n * b, 32u);
  if (e > 0) bytes += 4u * ceil_div(e, 4u) + 4u * ceil_div(e * (wmax - b), 32u);
  return bytes;
}

uint32_t jo_best_b(const uint32_t* z, uint32_t n) {
  uint32_t wmax = max_width(z, n);
  uint32_t best = 0, best_bytes = jo_block_body_bytes(z, n, 0);
  for (uint32_t b = 1; b <= wmax; b++) {
    uint32_t c = jo_block_body_bytes(z, n, b);
    if (c < best_bytes) { best = b; best_bytes = c; }
  }
  return best;
}

/* Writes header + body of one block packed with width b (any b with
 * b >= 0 and b <= 32; b >= wmax means no exceptions). out must be zeroed.
 * Returns the bytes written (4 + body). */
uint32_t jo_pack_block(const uint32_t* z, uint32_t n, uint32_t b, uint8_t* out) {
  uint32_t wmax = max_width(z, n);
  uint32_t e = 0;
  for (uint32_t i = 0; i < n; i++) if (bit_width(z[i]) > b) e++;
  uint32_t hb = e > 0 ? wmax - b : 0;
  out[0] = (uint8_t)b; out[1] = (uint8_t)e; out[2] = (uint8_t)hb; out[3] = 0;
  uint8_t* body = out + 4;
  uint32_t low_mask = b >= 32 ? 0xFFFFFFFFu : ((1u << b) - 1u);
  for (uint32_t i = 0; i < n; i++) put_bits(body, (uint64_t)i * b, z[i] & low_mask, b);
  uint32_t pos = 4u * ceil_div(n * b, 32u);
  if (e > 0) {
    uint8_t* positions = body + pos;
    uint32_t j = 0;
    for (uint32_t i = 0; i < n; i++) if (bit_width(z[i]) > b) positions[j++] = (uint8_t)i;
    pos += 4u * ceil_div(e, 4u);
    uint8_t* highs = body + pos;
    j = 0;
    for (uint32_t i = 0; i < n; i++)
      if (bit_width(z[i]) > b) { put_bits(highs, (uint64_t)j * hb, z[i] >> b, hb); j++; }
    pos += 4u * ceil_div(e * hb, 32u);
  }
  return 4u + pos;
}

/* Parses one block of n values given its 4-byte header and its body
 * (avail bytes left in the row). Returns 1 + the body bytes consumed (a
 * block with b = 0 and no exceptions has an empty body), or 0 on a
 * malformed block. */
static uint32_t unpack_block(const uint8_t* hdr, const uint8_t* body, size_t avail, uint32_t n, uint32_t* z) {
  uint32_t b = hdr[0], e = hdr[1], hb = hdr[2];
  if (hdr[3] != 0 || b > 32 || e > n || hb > 32 || b + hb > 32) return 0;
  if ((e == 0) != (hb == 0)) return 0;
  uint32_t low_bytes = 4u * ceil_div(n * b, 32u);
  uint32_t total = low_bytes;
  if (e > 0) total += 4u * ceil_div(e, 4u) + 4u * ceil_div(e * hb, 32u);
  if (total > avail) return 0;
  for (uint32_t i = 0; i < n; i++) z[i] = get_bits(body, (uint64_t)i * b, b);
  if (e > 0) {
    const uint8_t* positions = body + low_bytes;
    const uint8_t* highs = positions + 4u * ceil_div(e, 4u);
    for (uint32_t j = 0; j < e; j++) {
      uint32_t i = positions[j];
      if (i >= n || (j > 0 && i <= positions[j - 1])) return 0;
      z[i] |= get_bits(highs, (uint64_t)j * hb, hb) << b;
    }
  }
  return total + 1u;
}

/* ------------------------------------------------------------------ */
/* Residual sequence of one attribute-scan (Sec. III-C, III-D)          */
/* ------------------------------------------------------------------ */

/* Compacts the nonzero samples of the listed rows in row-major order and
 * forms residuals: e = q (I) or e = q - pq (P), modulo 2^32, with pq the
 * previous scan's quantized value at the same pixel (Sec. III-D: both scans
 * are masked with the current scan's mask). Without the mask stage every
 * sample is kept. row_start[k] receives the index of the first residual of
 * listed row k; row_start[nrows] the total. */
static uint32_t residuals(uint32_t W, const uint32_t* q, const uint32_t* pq, int mode, uint32_t stages,
                          const uint32_t* rows, uint32_t nrows, uint32_t* e, uint32_t* row_start) {
  uint32_t k = 0;
  for (uint32_t ri = 0; ri < nrows; ri++) {
    row_start[ri] = k;
    uint32_t r = rows[ri];
    for (uint32_t x = 0; x < W; x++) {
      size_t i = (size_t)r * W + x;
      if (q[i] == 0 && !(stages & JO_NO_MASK)) continue; /* masked out (Sec. III-C) */
      e[k++] = mode == 0 ? q[i] : q[i] - pq[i];
    }
  }
  row_start[nrows] = k;
  return k;
}

/* Horizontal delta over the flat vector (Sec. III-C), e[-1] = 0, then ZigZag
 * (Eq. 1); each step only if the stream keeps it. */
static void delta_zigzag(const uint32_t* e, uint32_t n, uint32_t stages, uint32_t* z) {
  uint32_t prev = 0;
  for (uint32_t k = 0; k < n; k++) {
    uint32_t d = (stages & JO_NO_DELTA) ? e[k] : e[k] - prev; /* modulo 2^32 */
    z[k] = (stages & JO_NO_ZIGZAG) ? d : jo_zigzag((int32_t)d);
    prev = e[k];
  }
}

/* Bytes of the packed blocks (headers included) of a row's values. */
static uint64_t row_block_bytes(const uint32_t* z, uint32_t n) {
  uint64_t bytes = 0;
  for (uint32_t s = 0; s < n; s += 128) {
    uint32_t m = n - s < 128 ? n - s : 128;
    bytes += 4u + jo_block_body_bytes(z + s, m, jo_best_b(z + s, m));
  }
  return bytes;
}

/* ------------------------------------------------------------------ */
/* Trial compression I/P selection (Sec. III-E, Sec. IV-E)              */
/* Test rows r_k = floor((2k+1) H / (2L)), k = 0..L-1, de-duplicated.    */
/* The residuals of the test rows (mask excluded) are delta coded as    */
/* one flat vector starting from 0 and packed per row; the cost is the  */
/* packed bytes. For H <= L the test rows are all rows and the cost      */
/* equals the full scan's packed data bytes.                            */
/* ------------------------------------------------------------------ */

static uint32_t test_rows(uint32_t H, uint32_t L, uint32_t* rows) {
  uint32_t n = 0;
  for (uint32_t k = 0; k < L; k++) {
    uint32_t r = (uint32_t)(((uint64_t)(2 * k + 1) * H) / (2ull * L));
    if (n == 0 || rows[n - 1] != r) rows[n++] = r;
  }
  return n;
}

static uint64_t trial_cost(uint32_t H, uint32_t W, const uint32_t* q, const uint32_t* pq, int mode,
                           uint32_t L, uint32_t stages) {
  uint32_t* rows = (uint32_t*)calloc(L ? L : 1, sizeof(uint32_t));
  uint32_t nrows = test_rows(H, L, rows);
  uint32_t* e = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)nrows * W + 1));
  uint32_t* z = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)nrows * W + 1));
  uint32_t* start = (uint32_t*)malloc(sizeof(uint32_t) * (nrows + 1));
  uint32_t n = residuals(W, q, pq, mode, stages, rows, nrows, e, start);
  delta_zigzag(e, n, stages, z);
  uint64_t cost = 0;
  for (uint32_t k = 0; k < nrows; k++) cost += row_block_bytes(z + start[k], start[k + 1] - start[k]);
  free(rows); free(e); free(z); free(start);
  return cost;
}

/* ------------------------------------------------------------------ */
/* Section = one attribute of one scan.                                 */
/*   row table: H entries of 8 bytes {u32 end, u32 carry}               */
/*     end   = end of row r's chunk, in bytes from the first chunk      */
/*     carry = the residual just before row r's first residual in the   */
/*             flat vector (0 if none): the value row r's first delta   */
/*             subtracts. Redundant, it lets rows decode independently. */
/*   row chunks, r = 0..H-1:                                            */
/*     (mask part, absent without the mask stage:)                      */
/*     mask class words: ceil(nw/16) u32, nw = ceil(W/32); word j's     */
/*       2-bit class sits at bits 2*(j%16) of class word j/16:           */
/*       0: coded word is 0, 1: coded word has every valid bit set,     */
/*       2: coded word stored as a literal, 3: invalid                   */
/*     literal words, ascending j                                       */
/*     block headers of the row's ceil(n_r/128) blocks                  */
/*     block bodies, same order                                         */
/*   Mask words: bit x%32 of word x/32 is 1 where sample x of the row is */
/*   zero; bits past W are 0. The coded word is the mask word (I) or     */
/*   the mask word XOR the previous scan's (P).                          */
/* With the Zstandard mask (JO_ZSTD_MASK) the rows carry no mask part;   */
/* the mask of the whole section follows the row table instead:         */
/*     u32 frame bytes F                                                 */
/*     u32 end of each of the frame's B = ceil(H ceil(W/8) / 8192) blocks, */
/*       in bytes from the frame's start                                */
/*     the Zstandard frame of the section's mask bytes: row r's bits,   */
/*       LSB first, in bytes r*ceil(W/8) .. (r+1)*ceil(W/8)-1 (padding   */
/*       bits 0), XORed with the previous scan's for P                  */
/*     zero bytes up to a multiple of 4                                  */
/*   and the row ends count from the first row chunk after it.          */
/* ------------------------------------------------------------------ */

static uint32_t valid_bits(uint32_t W, uint32_t j) {
  uint32_t nw = ceil_div(W, 32u);
  if (j + 1 < nw || W % 32 == 0) return 0xFFFFFFFFu;
  return (1u << (W % 32)) - 1u;
}

static size_t section_bound(uint32_t H, uint32_t W) {
  uint32_t nw = ceil_div(W, 32u);
  /* class words + literals + block headers + bodies; with b = wmax a block
   * of m values has no exceptions and needs at most 4*m bytes, and the
   * chosen b never needs more than that */
  size_t row = 4u * ceil_div(nw, 16u) + 4u * nw + 4u * ceil_div(W, 128u) + (size_t)W * 4u;
  size_t zm = (size_t)H * ((W + 7u) / 8u);
  return (size_t)H * 8u + (size_t)H * row + 8u + 4u * jz_block_count(zm) + jz_frame_bound(zm);
}

/* Zstandard mask part of a section (layout above); returns its bytes */
static size_t write_zstd_mask(uint32_t H, uint32_t W, const uint8_t* M, const uint32_t* pq, int mode, uint8_t* out) {
  size_t rb = (W + 7u) / 8u, n = (size_t)H * rb;
  uint8_t* bytes = (uint8_t*)calloc(n, 1);
  for (uint32_t r = 0; r < H; r++) {
    for (uint32_t x = 0; x < W; x++) {
      size_t i = (size_t)r * W + x;
      uint32_t bit = M[i];
      if (mode == 1) bit ^= (pq[i] == 0); /* Sec. III-D */
      bytes[(size_t)r * rb + x / 8u] |= (uint8_t)(bit << (x % 8u));
    }
  }
  size_t nblk = jz_block_count(n);
  uint32_t* ends = (uint32_t*)malloc(sizeof(uint32_t) * nblk);
  uint8_t* f = out + 4u + 4u * nblk;
  size_t fb = jz_write_frame(bytes, n, f, ends);
  put_u32(out, (uint32_t)fb);
  for (size_t j = 0; j < nblk; j++) put_u32(out + 4u + 4u * j, ends[j]);
  free(bytes); free(ends);
  return (4u + 4u * nblk + fb + 3u) & ~(size_t)3u; /* the caller's buffer is zeroed: pad bytes are 0 */
}

/* Encodes one section into out (zeroed by the caller, at least
 * section_bound bytes). Returns its size; mask_bytes / data_bytes receive
 * the mask-part and block (header + body) byte counts. */
static size_t encode_section(uint32_t H, uint32_t W, const uint32_t* q, const uint32_t* pq, int mode,
                             uint32_t stages, uint8_t* out, uint32_t* nnz_out, uint64_t* mask_bytes,
                             uint64_t* data_bytes) {
  uint32_t nw = (stages & (JO_NO_MASK | JO_ZSTD_MASK)) ? 0u : ceil_div(W, 32u); /* class-coded mask words per row */
  size_t HW = (size_t)H * W;
  /* zero bitmask, one entry per sample (Sec. III-C): 1 = zero sample */
  uint8_t* M = (uint8_t*)malloc(HW ? HW : 1);
  for (size_t i = 0; i < HW; i++) M[i] = q[i] == 0;
  /* compaction + residual over all rows (Sec. III-C, III-D) */
  uint32_t* rows = (uint32_t*)malloc(sizeof(uint32_t) * (H ? H : 1));
  for (uint32_t r = 0; r < H; r++) rows[r] = r;
  uint32_t* e = (uint32_t*)malloc(sizeof(uint32_t) * (HW + 1));
  uint32_t* z = (uint32_t*)malloc(sizeof(uint32_t) * (HW + 1));
  uint32_t* start = (uint32_t*)malloc(sizeof(uint32_t) * (H + 1));
  uint32_t nnz = residuals(W, q, pq, mode, stages, rows, H, e, start);
  /* delta over the flat vector, then ZigZag (Sec. III-C, Eq. 1) */
  delta_zigzag(e, nnz, stages, z);

  uint8_t* table = out;
  uint8_t* data = out + (size_t)H * 8u;
  size_t pos = 0, zpart = 0;
  uint64_t mbytes = 0, dbytes = 0;
  if (stages & JO_ZSTD_MASK) {
    zpart = write_zstd_mask(H, W, M, pq, mode, data);
    data += zpart;
    mbytes += zpart;
  }
  for (uint32_t r = 0; r < H; r++) {
    /* mask part */
    uint32_t ncls = ceil_div(nw, 16u);
    uint8_t* cls = data + pos;
    size_t lit = pos + 4u * ncls;
    for (uint32_t j = 0; j < nw; j++) {
      uint32_t word = 0;
      for (uint32_t k = 0; k < 32; k++) {
        uint32_t x = 32u * j + k;
        if (x >= W) break;
        size_t i = (size_t)r * W + x;
        uint32_t bit = M[i];
        if (mode == 1) bit ^= (pq[i] == 0); /* Sec. III-D: XOR with the previous mask */
        word |= bit << k;
      }
      uint32_t c;
      if (word == 0) c = 0;
      else if (word == valid_bits(W, j)) c = 1;
      else { c = 2; put_u32(data + lit, word); lit += 4; }
      cls[4u * (j / 16u) + (2u * (j % 16u)) / 8u] |= (uint8_t)(c << ((2u * (j % 16u)) % 8u));
    }
    mbytes += lit - pos;
    pos = lit;
    /* blocks: headers, then bodies */
    uint32_t n = start[r + 1] - start[r];
    uint32_t nb = ceil_div(n, 128u);
    uint8_t* headers = data + pos;
    size_t body = pos + 4u * nb;
    for (uint32_t k = 0; k < nb; k++) {
      uint32_t s = start[r] + 128u * k;
      uint32_t m = n - 128u * k < 128u ? n - 128u * k : 128u;
      uint8_t* tmp = (uint8_t*)calloc(4u + 4u * 128u + 4u * 32u + 4u * 128u, 1);
      uint32_t sz = jo_pack_block(z + s, m, jo_best_b(z + s, m), tmp);
      memcpy(headers + 4u * k, tmp, 4);
      memcpy(data + body, tmp + 4, sz - 4u);
      body += sz - 4u;
      free(tmp);
    }
    dbytes += body - pos;
    pos = body;
    put_u32(table + 8u * r, (uint32_t)pos);
    put_u32(table + 8u * r + 4u, start[r] > 0 ? e[start[r] - 1] : 0u);
  }
  free(M); free(rows); free(e); free(z); free(start);
  if (nnz_out) *nnz_out = nnz;
  if (mask_bytes) *mask_bytes = mbytes;
  if (data_bytes) *data_bytes = dbytes;
  return (size_t)H * 8u + zpart + pos;
}

/* Decodes one section into q_out. Returns 0 or JO_ERR_CORRUPT. */
static int decode_section(uint32_t H, uint32_t W, const uint8_t* sec, size_t len, int mode, uint32_t stages,
                          const uint32_t* pq, uint32_t* q_out, uint32_t expect_nnz) {
  uint32_t nw = ceil_div(W, 32u);
  uint32_t nmw = (stages & (JO_NO_MASK | JO_ZSTD_MASK)) ? 0u : nw; /* class-coded mask words per row */
  if (len < (size_t)H * 8u) return JO_ERR_CORRUPT;
  const uint8_t* table = sec;
  const uint8_t* data = sec + (size_t)H * 8u;
  size_t data_len = len - (size_t)H * 8u;
  uint8_t* zm = NULL; /* Zstandard mask bytes of the section (the coded, XORed form) */
  size_t rb = (W + 7u) / 8u;
  if (stages & JO_ZSTD_MASK) {
    size_t n = (size_t)H * rb, nblk = jz_block_count(n);
    if (data_len < 4u + 4u * nblk) return JO_ERR_CORRUPT;
    size_t fb = get_u32(data), part = (4u + 4u * nblk + fb + 3u) & ~(size_t)3u;
    if (fb > data_len || part > data_len) return JO_ERR_CORRUPT;
    zm = (uint8_t*)malloc(n);
    uint32_t* ends = (uint32_t*)malloc(sizeof(uint32_t) * nblk);
    size_t got = jz_read_frame(data + 4u + 4u * nblk, fb, zm, n, ends, nblk);
    int bad = got != fb;
    for (size_t j = 0; j < nblk && !bad; j++) bad = ends[j] != get_u32(data + 4u + 4u * j);
    for (size_t i = 4u + 4u * nblk + fb; i < part && !bad; i++) bad = data[i] != 0;
    free(ends);
    if (bad) { free(zm); return JO_ERR_CORRUPT; }
    data += part;
    data_len -= part;
  }
  uint32_t* z = (uint32_t*)malloc(sizeof(uint32_t) * (W + 128u));
  uint32_t* word = (uint32_t*)malloc(sizeof(uint32_t) * (nw ? nw : 1));
  size_t begin = 0;
  uint32_t last_e = 0, total = 0;
  int rc = JO_OK;
  for (uint32_t r = 0; r < H && rc == JO_OK; r++) {
    size_t end = get_u32(table + 8u * r);
    uint32_t carry = get_u32(table + 8u * r + 4u);
    if (end < begin || end > data_len || carry != last_e) { rc = JO_ERR_CORRUPT; break; }
    const uint8_t* chunk = data + begin;
    size_t clen = end - begin, p = 0;
    /* mask part */
    uint32_t ncls = ceil_div(nmw, 16u);
    if (4u * ncls > clen) { rc = JO_ERR_CORRUPT; break; }
    p = 4u * ncls;
    uint32_t n = 0;
    if (nmw == 0 && !zm) { /* no mask stage: every sample was coded */
      for (uint32_t j = 0; j < nw; j++) word[j] = 0;
      n = W;
    }
    if (zm) { /* the row's bits from the section's Zstandard mask */
      for (uint32_t j = 0; j < nw; j++) word[j] = 0;
      for (uint32_t x = 0; x < W; x++) {
        uint32_t bit = (zm[(size_t)r * rb + x / 8u] >> (x % 8u)) & 1u;
        if (mode == 1) bit ^= (pq[(size_t)r * W + x] == 0); /* undo the XOR with the previous mask */
        word[x / 32u] |= bit << (x % 32u);
        n += bit == 0;
      }
      for (uint32_t x = W; x < 8u * (uint32_t)rb; x++)
        if ((zm[(size_t)r * rb + x / 8u] >> (x % 8u)) & 1u) rc = JO_ERR_CORRUPT; /* padding bits are 0 */
      if (rc != JO_OK) break;
    }
    for (uint32_t j = 0; j < nmw && rc == JO_OK; j++) {
      uint32_t c = (get_u32(chunk + 4u * (j / 16u)) >> (2u * (j % 16u))) & 3u;
      uint32_t w;
      if (c == 0) w = 0;
      else if (c == 1) w = valid_bits(W, j);
      else if (c == 2) {
        if (p + 4 > clen) { rc = JO_ERR_CORRUPT; break; }
        w = get_u32(chunk + p); p += 4;
        if (w & ~valid_bits(W, j)) { rc = JO_ERR_CORRUPT; break; }
      } else { rc = JO_ERR_CORRUPT; break; }
      if (mode == 1) { /* undo the XOR with the previous scan's mask */
        uint32_t prev = 0;
        for (uint32_t k = 0; k < 32 && 32u * j + k < W; k++)
          prev |= (uint32_t)(pq[(size_t)r * W + 32u * j + k] == 0) << k;
        w ^= prev;
      }
      word[j] = w;
      for (uint32_t k = 0; k < 32 && 32u * j + k < W; k++) n += ((w >> k) & 1u) == 0;
    }
    if (rc != JO_OK) break;
    /* blocks */
    uint32_t nb = ceil_div(n, 128u);
    if (p + 4u * nb > clen) { rc = JO_ERR_CORRUPT; break; }
    const uint8_t* headers = chunk + p;
    p += 4u * nb;
    for (uint32_t k = 0; k < nb; k++) {
      uint32_t m = n - 128u * k < 128u ? n - 128u * k : 128u;
      uint32_t used = unpack_block(headers + 4u * k, chunk + p, clen - p, m, z + 128u * k);
      if (used == 0) { rc = JO_ERR_CORRUPT; break; }
      p += used - 1u;
    }
    if (rc != JO_OK) break;
    if (p != clen) { rc = JO_ERR_CORRUPT; break; }
    /* un-ZigZag, inverse delta starting from the carry, inverse residual,
     * scatter into the nonzero positions */
    uint32_t prev = carry, k = 0;
    for (uint32_t x = 0; x < W; x++) {
      size_t i = (size_t)r * W + x;
      if ((word[x / 32u] >> (x % 32u)) & 1u) { q_out[i] = 0; continue; }
      uint32_t d = (stages & JO_NO_ZIGZAG) ? z[k++] : (uint32_t)jo_unzigzag(z[k++]);
      uint32_t e = (stages & JO_NO_DELTA) ? d : prev + d; /* modulo 2^32 */
      prev = e;
      q_out[i] = mode == 0 ? e : e + pq[i];
    }
    if (n > 0) last_e = prev;
    total += n;
    begin = end;
  }
  if (rc == JO_OK && (begin != data_len || total != expect_nnz)) rc = JO_ERR_CORRUPT;
  free(z); free(word); free(zm);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Stream codec                                                         */
/*   stream header (first frame after create/reset), 16 + 8A bytes:     */
/*     "JFY1", u16 version = 1, u16 A, u32 H, u32 W,                     */
/*     per attribute: u8 dtype_bytes, u8 zigzag variant (1 = Eq. 1,      */
/*     0 = none), u8 stage flags (bit 0: no zero mask, bit 1: no delta, */
/*     bit 2: Zstandard mask), u8 0, u32 precision (Sec. III-A: the      */
/*     precision is stored)                                             */
/*   frame, header 8 + 12A bytes:                                       */
/*     u32 frame_bytes (header included), u32 scan_index,               */
/*     per attribute: u8 mode (0 = I, 1 = P), 3 bytes 0,                 */
/*     u32 section_bytes, u32 nnz                                       */
/*   then the A sections back to back.                                  */
/* ------------------------------------------------------------------ */

typedef struct {
  uint32_t H, W, A, L;
  int32_t force_mode;
  uint32_t stages; /* JO_NO_* switches */
  uint8_t dtype[JO_MAX_ATTR];
  uint32_t prec[JO_MAX_ATTR];
  uint32_t frame;
  uint32_t* prev_q[JO_MAX_ATTR];
} jo_codec;

jo_codec* jo_create(uint32_t H, uint32_t W, uint32_t A, const uint8_t* dtypes, const uint32_t* precs,
                    uint32_t test_lines, int32_t force_mode, uint32_t stages) {
  if (H == 0 || W == 0 || A == 0 || A > JO_MAX_ATTR || test_lines == 0 || stages > 15u) return NULL;
  if ((stages & JO_NO_MASK) && (stages & JO_ZSTD_MASK)) return NULL; /* no mask to code */
  for (uint32_t a = 0; a < A; a++) {
    if (!(dtypes[a] == 1 || dtypes[a] == 2 || dtypes[a] == 4) || precs[a] == 0) return NULL;
  }
  jo_codec* c = (jo_codec*)calloc(1, sizeof(jo_codec));
  c->H = H; c->W = W; c->A = A; c->L = test_lines; c->force_mode = force_mode; c->stages = stages;
  for (uint32_t a = 0; a < A; a++) {
    c->dtype[a] = dtypes[a]; c->prec[a] = precs[a];
    c->prev_q[a] = (uint32_t*)calloc((size_t)H * W, sizeof(uint32_t));
  }
  return c;
}

void jo_destroy(jo_codec* c) {
  if (!c) return;
  for (uint32_t a = 0; a < c->A; a++) free(c->prev_q[a]);
  free(c);
}

void jo_reset(jo_codec* c) { c->frame = 0; }

static size_t stream_header_bytes(uint32_t A) { return 16u + 8u * A; }
static size_t frame_header_bytes(uint32_t A) { return 8u + 12u * A; }

/* Encodes one scan (A planes of H x W samples). Returns the bytes written
 * (the stream header is included before the first frame), or -JO_ERR_*.
 * modes_out (nullable) receives the A chosen modes. */
int64_t jo_encode(jo_codec* c, const void* const* planes, uint8_t* out, size_t cap, uint8_t* modes_out) {
  size_t HW = (size_t)c->H * c->W;
  size_t bound = stream_header_bytes(c->A) + frame_header_bytes(c->A) + c->A * section_bound(c->H, c->W);
  uint8_t* buf = (uint8_t*)calloc(bound, 1);
  uint32_t** q = (uint32_t**)calloc(c->A, sizeof(uint32_t*));
  size_t pos = 0;
  if (c->frame == 0) {
    memcpy(buf, "JFY1", 4);
    put_u16(buf + 4, 1); put_u16(buf + 6, c->A); put_u32(buf + 8, c->H); put_u32(buf + 12, c->W);
    for (uint32_t a = 0; a < c->A; a++) {
      uint8_t* p = buf + 16 + 8 * a;
      p[0] = c->dtype[a];
      p[1] = (c->stages & JO_NO_ZIGZAG) ? 0 : 1;
      p[2] = header_flags(c->stages);
      p[3] = 0;
      put_u32(p + 4, c->prec[a]);
    }
    pos = stream_header_bytes(c->A);
  }
  size_t frame_start = pos;
  pos += frame_header_bytes(c->A);
  for (uint32_t a = 0; a < c->A; a++) {
    q[a] = (uint32_t*)malloc(sizeof(uint32_t) * (HW ? HW : 1));
    for (size_t i = 0; i < HW; i++) q[a][i] = jo_quantize(load_sample(planes[a], c->dtype[a], i), c->prec[a], c->dtype[a]);
    int mode;
    if (c->frame == 0) mode = 0;
    else if (c->force_mode == 0 || c->force_mode == 1) mode = c->force_mode;
    else {
      uint64_t ci = trial_cost(c->H, c->W, q[a], c->prev_q[a], 0, c->L, c->stages);
      uint64_t cp = trial_cost(c->H, c->W, q[a], c->prev_q[a], 1, c->L, c->stages);
      mode = cp < ci ? 1 : 0;
    }
    uint32_t nnz = 0;
    size_t sec = encode_section(c->H, c->W, q[a], c->prev_q[a], mode, c->stages, buf + pos, &nnz, NULL, NULL);
    uint8_t* h = buf + frame_start + 8 + 12 * a;
    h[0] = (uint8_t)mode; put_u32(h + 4, (uint32_t)sec); put_u32(h + 8, nnz);
    if (modes_out) modes_out[a] = (uint8_t)mode;
    pos += sec;
  }
  put_u32(buf + frame_start, (uint32_t)(pos - frame_start));
  put_u32(buf + frame_start + 4, c->frame);
  int64_t rc;
  if (pos > cap) {
    rc = -JO_ERR_CAPACITY; /* state does not advance */
  } else {
    memcpy(out, buf, pos);
    for (uint32_t a = 0; a < c->A; a++) memcpy(c->prev_q[a], q[a], sizeof(uint32_t) * HW);
    c->frame++;
    rc = (int64_t)pos;
  }
  for (uint32_t a = 0; a < c->A; a++) free(q[a]);
  free(q); free(buf);
  return rc;
}

/* Decodes one frame (preceded by the stream header for the first frame
 * after create/reset). Returns the bytes consumed or -JO_ERR_*. */
int64_t jo_decode(jo_codec* c, const uint8_t* in, size_t len, void* const* planes_out) {
  size_t HW = (size_t)c->H * c->W;
  size_t pos = 0;
  if (c->frame == 0) {
    if (len < stream_header_bytes(c->A)) return -JO_ERR_CORRUPT;
    if (memcmp(in, "JFY1", 4) != 0 || get_u16(in + 4) != 1 || get_u16(in + 6) != c->A ||
        get_u32(in + 8) != c->H || get_u32(in + 12) != c->W)
      return -JO_ERR_CORRUPT;
    for (uint32_t a = 0; a < c->A; a++) {
      const uint8_t* p = in + 16 + 8 * a;
      if (p[0] != c->dtype[a] || p[1] != ((c->stages & JO_NO_ZIGZAG) ? 0 : 1) ||
          p[2] != header_flags(c->stages) || p[3] != 0 || get_u32(p + 4) != c->prec[a])
        return -JO_ERR_CORRUPT;
    }
    pos = stream_header_bytes(c->A);
  }
  if (len - pos < frame_header_bytes(c->A)) return -JO_ERR_CORRUPT;
  const uint8_t* fh = in + pos;
  size_t frame_bytes = get_u32(fh);
  if (frame_bytes > len - pos || get_u32(fh + 4) != c->frame) return -JO_ERR_CORRUPT;
  size_t sp = pos + frame_header_bytes(c->A);
  uint32_t** q = (uint32_t**)calloc(c->A, sizeof(uint32_t*));
  int rc = JO_OK;
  for (uint32_t a = 0; a < c->A && rc == JO_OK; a++) {
    const uint8_t* h = fh + 8 + 12 * a;
    int mode = h[0];
    size_t sec = get_u32(h + 4);
    uint32_t nnz = get_u32(h + 8);
    if (mode > 1 || h[1] || h[2] || h[3] || (mode == 1 && c->frame == 0) || sec > pos + frame_bytes - sp) {
      rc = JO_ERR_CORRUPT; break;
    }
    q[a] = (uint32_t*)malloc(sizeof(uint32_t) * (HW ? HW : 1));
    rc = decode_section(c->H, c->W, in + sp, sec, mode, c->stages, c->prev_q[a], q[a], nnz);
    if (rc == JO_OK) {
      uint32_t qmax = dtype_max(c->dtype[a]) / c->prec[a];
      for (size_t i = 0; i < HW; i++) if (q[a][i] > qmax) { rc = JO_ERR_CORRUPT; break; }
    }
    sp += sec;
  }
  if (rc == JO_OK && sp != pos + frame_bytes) rc = JO_ERR_CORRUPT;
  if (rc == JO_OK) {
    for (uint32_t a = 0; a < c->A; a++) {
      for (size_t i = 0; i < HW; i++) store_sample(planes_out[a], c->dtype[a], i, q[a][i] * c->prec[a]);
      memcpy(c->prev_q[a], q[a], sizeof(uint32_t) * HW);
    }
    c->frame++;
  }
  for (uint32_t a = 0; a < c->A; a++) free(q[a]);
  free(q);
  return rc == JO_OK ? (int64_t)(sp) : -(int64_t)rc;
}

/* ------------------------------------------------------------------ */
/* Probes used by the pins: trial cost and full-encode byte split for a */
/* single attribute-scan given its raw plane and the previous raw plane. */
/* ------------------------------------------------------------------ */

static uint32_t* quantize_plane(const void* plane, uint32_t s, uint32_t P, size_t HW) {
  uint32_t* q = (uint32_t*)malloc(sizeof(uint32_t) * (HW ? HW : 1));
  for (size_t i = 0; i < HW; i++) q[i] = jo_quantize(load_sample(plane, s, i), P, s);
  return q;
}

uint64_t jo_trial_cost(uint32_t H, uint32_t W, uint32_t s, uint32_t P, uint32_t L, const void* cur,
                       const void* prev, int mode) {
  size_t HW = (size_t)H * W;
  uint32_t* q = quantize_plane(cur, s, P, HW);
  uint32_t* pq = quantize_plane(prev, s, P, HW);
  uint64_t c = trial_cost(H, W, q, pq, mode, L, 0u);
  free(q); free(pq);
  return c;
}

/* Full encode of one section in a forced mode; reports the mask-part bytes
 * and the block bytes (headers + bodies); returns the section bytes. */
uint64_t jo_section_split(uint32_t H, uint32_t W, uint32_t s, uint32_t P, const void* cur, const void* prev,
                          int mode, uint64_t* mask_bytes, uint64_t* data_bytes) {
  size_t HW = (size_t)H * W;
  uint32_t* q = quantize_plane(cur, s, P, HW);
  uint32_t* pq = quantize_plane(prev, s, P, HW);
  uint8_t* buf = (uint8_t*)calloc(section_bound(H, W), 1);
  uint32_t nnz = 0;
  size_t sec = encode_section(H, W, q, pq, mode, 0u, buf, &nnz, mask_bytes, data_bytes);
  free(q); free(pq); free(buf);
  return sec;
}
