/*
 * Standardization oracle: Cartesian points -> H x W range image (Sec. III-A).
 *
 * TEST INFRASTRUCTURE ONLY, like jiffy_oracle.c: the test suite and the
 * benchmark's CPU leg load it; the library never calls it, and it shares no
 * code, header, table or constant with the CUDA implementation.
 *
 * Sec. III-A: points given as floating-point Cartesian coordinates are
 * converted to spherical coordinates, sorted by altitude and azimuth into the
 * scan's rows and columns, and quantized to unsigned integers; invalid or
 * out-of-range measurements become the sentinel 0. Attributes are arranged
 * and quantized the same way. The paper fixes no arithmetic for this step;
 * this project defines it in integers so that every decision (which pixel,
 * which point) is exact and reproducible:
 *
 *   1. coordinates: X = round-half-even(x * k) with the product rounded to
 *      float32 (k = units per metre, e.g. 1000 for millimetres); a point
 *      with |x * k| >= 2^31 (or NaN) is invalid;
 *   2. range R = X^2 + Y^2 + Z^2 square-rooted and rounded to the nearest
 *      integer (exact integer square root);
 *   3. angles as binary angles, 2^32 units per turn, by CORDIC vectoring
 *      (Volder, "The CORDIC trigonometric computing technique", 1959) in
 *      32-bit integers, 30 iterations, on the vector scaled by a power of
 *      two (arithmetic shifts) so that its larger component has 29 bits:
 *      azimuth of (X, Y) in [0, 2^32) counterclockwise from +x (clockwise
 *      sensors negate Y; 0 for X = Y = 0), elevation of (rho, Z) with rho =
 *      floor(sqrt(X^2 + Y^2) 2^f) and Z 2^f (floor), f the largest (possibly
 *      negative) integer that keeps both below 2^29 (0 for X = Y = Z = 0);
 *      the arctangent table atan(2^-i) is rounded from the C library's atan;
 *   4. row = nearest beam: beam altitudes (radians within +-pi/2, strictly
 *      decreasing, row 0 on top) as binary angles; row r covers elevations from the midpoint
 *      with the beam below up to the midpoint with the beam above (the top
 *      and bottom rows extend half their spacing outwards; points beyond are
 *      dropped); column c = floor(((az - az0) mod 2^48) * W / 2^48);
 *   5. a pixel hit by several points keeps the nearest one (smallest R, then
 *      smallest point index); pixels without a valid point are 0;
 *   6. attribute value q = round-half-even(v * scale) with the product
 *      rounded to float32, clamped to [0, max of the sample type], NaN -> 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define JS_PI 3.14159265358979323846
#define JS_ITER 30
#define JS_NORM_BITS 29

enum { JS_OK = 0, JS_ERR_INVALID_ARG = 1 };

static int32_t js_atan_table[JS_ITER];
static int js_table_ready = 0;

/* atan(2^-i) as a binary angle (2^32 per turn), rounded to nearest. */
static void js_init_table(void) {
  if (js_table_ready) return;
  for (int i = 0; i < JS_ITER; i++) {
    double a = atan(ldexp(1.0, -i)); /* radians */
    js_atan_table[i] = (int32_t)llround(a / (2.0 * JS_PI) * 4294967296.0);
  }
  js_table_ready = 1;
}

/* Vectoring CORDIC: the angle of (x, y) for x >= 0, components below 2^29,
 * as a signed binary angle; y is driven to 0 by micro-rotations of
 * +-atan(2^-i). |x| stays below 1.65 * sqrt(2) * 2^29 < 2^31. */
static int32_t js_cordic_vec(int32_t x, int32_t y) {
  int32_t ang = 0;
  for (int i = 0; i < JS_ITER; i++) {
    int32_t xs = x >> i, ys = y >> i; /* arithmetic shifts */
    if (y > 0) {
      x = x + ys; y = y - xs; ang += js_atan_table[i];
    } else {
      x = x - ys; y = y + xs; ang -= js_atan_table[i];
    }
  }
  return ang;
}

static int js_bits(uint64_t m) {
  int bits = 0;
  while (bits < 64 && (m >> bits)) bits++;
  return bits;
}

/* v * 2^s, with floor division for s < 0 (arithmetic shift). */
static int64_t js_scale(int64_t v, int s) {
  return s >= 0 ? v * ((int64_t)1 << s) : (v >> (-s));
}

uint32_t js_azimuth(int64_t X, int64_t Y) {
  js_init_table();
  if (X == 0 && Y == 0) return 0;
  uint64_t m = (uint64_t)(X < 0 ? -X : X) | (uint64_t)(Y < 0 ? -Y : Y);
  int s = JS_NORM_BITS - js_bits(m);
  int32_t x = (int32_t)js_scale(X, s), y = (int32_t)js_scale(Y, s);
  uint32_t base = 0;
  if (x < 0) { x = -x; y = -y; base = 0x80000000u; } /* a half turn first */
  return base + (uint32_t)js_cordic_vec(x, y);       /* modulo 2^32 */
}

/* floor(sqrt(n)) for n < 2^126. */
static uint64_t js_isqrt128(unsigned __int128 n) {
  uint64_t r = (uint64_t)sqrt((double)n);
  while ((unsigned __int128)r * r > n) r--;
  while ((unsigned __int128)(r + 1) * (r + 1) <= n) r++;
  return r;
}

uint64_t js_isqrt(uint64_t hi, uint64_t lo) {
  return js_isqrt128(((unsigned __int128)hi << 64) | lo);
}

int32_t js_elevation(int64_t X, int64_t Y, int64_t Z) {
  js_init_table();
  uint64_t h = (uint64_t)(X * X) + (uint64_t)(Y * Y); /* < 2^63 */
  uint64_t z2 = (uint64_t)(Z * Z);
  uint64_t m = h > z2 ? h : z2;
  if (m == 0) return 0;
  int e = js_bits(m);
  /* largest f with m * 4^f < 2^58 */
  int f = e <= 2 * JS_NORM_BITS ? (2 * JS_NORM_BITS - e) / 2 : -((e - 2 * JS_NORM_BITS + 1) / 2);
  uint64_t hs = f >= 0 ? h << (2 * f) : h >> (-2 * f);
  int32_t rho = (int32_t)js_isqrt128(hs); /* floor(sqrt(h) * 2^f), below 2^29 */
  return js_cordic_vec(rho, (int32_t)js_scale(Z, f));
}

static int64_t js_binary_angle(double rad) {
  return (int64_t)llround(rad / (2.0 * JS_PI) * 4294967296.0);
}

/* Float -> integer coordinate (step 1); returns 0 if invalid. */
static int js_coord(float v, float k, int64_t* out) {
  float p = v * k;
  if (!(fabsf(p) < 2147483648.0f)) return 0; /* also NaN */
  *out = (int64_t)rintf(p);                /* round half to even */
  return 1;
}

static uint32_t js_max_of(uint32_t bytes) {
  return bytes == 4 ? 0xFFFFFFFFu : ((1u << (8 * bytes)) - 1u);
}

static void js_store(void* p, uint32_t bytes, size_t i, uint32_t v) {
  if (bytes == 1) ((uint8_t*)p)[i] = (uint8_t)v;
  else if (bytes == 2) ((uint16_t*)p)[i] = (uint16_t)v;
  else ((uint32_t*)p)[i] = v;
}

uint32_t js_quantize_attr(float v, float scale, uint32_t bytes) {
  float p = v * scale;
  uint32_t mx = js_max_of(bytes);
  if (!(p > 0.0f)) return 0; /* also NaN */
  if (p >= (float)mx) return mx;
  float r = rintf(p);
  return r >= (float)mx ? mx : (uint32_t)r;
}

/* Pixel of one point, or -1 if dropped; *range receives R (steps 1-4). */
int64_t js_pixel(float x, float y, float z, float k, uint32_t H, uint32_t W, const int64_t* alt, uint32_t az0,
                 int clockwise, uint32_t rmin, uint32_t rmax, uint32_t* range) {
  int64_t X, Y, Z;
  if (!js_coord(x, k, &X) || !js_coord(y, k, &Y) || !js_coord(z, k, &Z)) return -1;
  if (clockwise) Y = -Y;
  uint64_t n = (uint64_t)(X * X) + (uint64_t)(Y * Y) + (uint64_t)(Z * Z); /* < 3 * 2^62 */
  uint64_t r = js_isqrt128(n);
  uint64_t R = r + ((n - r * r) > r ? 1u : 0u); /* nearest integer */
  if (R < 1 || R < rmin || R > rmax) return -1;
  *range = (uint32_t)R;
  /* row: nearest beam */
  int64_t el = js_elevation(X, Y, Z);
  uint32_t row = 0;
  if (H > 1) {
    if (el > alt[0] + (alt[0] - alt[1]) / 2) return -1;
    if (el < alt[H - 1] - (alt[H - 2] - alt[H - 1]) / 2) return -1;
    for (uint32_t b = 0; b + 1 < H; b++) {
      int64_t mid = alt[b + 1] + (alt[b] - alt[b + 1]) / 2;
      if (el < mid) row = b + 1;
    }
  }
  /* column */
  uint32_t a = js_azimuth(X, Y) - az0; /* modulo 2^32 */
  uint64_t col = ((uint64_t)a * W) >> 32;
  return (int64_t)row * W + (int64_t)col;
}

/*
 * Standardizes one scan of n points (xyz: 3n floats, x y z per point, in
 * metres) into range_out (H x W samples of range_bytes, units of 1/k m) and
 * n_attr attribute images (attr[a]: n floats, nullable when n_attr = 0).
 * beam_alt: H radians, strictly decreasing. Returns 0 or JS_ERR_INVALID_ARG.
 */
int js_standardize(const float* xyz, uint32_t n, uint32_t H, uint32_t W, const double* beam_alt, double az0,
                   int clockwise, float k, uint32_t range_bytes, uint32_t rmin, uint32_t rmax, void* range_out,
                   uint32_t n_attr, const float* const* attr, const uint32_t* attr_bytes,
                   const float* attr_scale, void* const* attr_out) {
  if (H == 0 || W == 0 || !(range_bytes == 2 || range_bytes == 4) || !(k > 0.0f)) return JS_ERR_INVALID_ARG;
  for (uint32_t a = 0; a < n_attr; a++)
    if (!(attr_bytes[a] == 1 || attr_bytes[a] == 2 || attr_bytes[a] == 4)) return JS_ERR_INVALID_ARG;
  int64_t* alt = (int64_t*)malloc(sizeof(int64_t) * H);
  for (uint32_t b = 0; b < H; b++) {
    alt[b] = js_binary_angle(beam_alt[b]);
    if (alt[b] > (1 << 30) || alt[b] < -(1 << 30) || (b > 0 && alt[b] >= alt[b - 1])) { /* within +-90 deg */
      free(alt);
      return JS_ERR_INVALID_ARG;
    }
  }
  uint32_t a0 = (uint32_t)(uint64_t)js_binary_angle(az0); /* modulo 2^32 */
  uint32_t rcap = rmax < js_max_of(range_bytes) ? rmax : js_max_of(range_bytes);
  size_t HW = (size_t)H * W;
  uint64_t* best = (uint64_t*)malloc(sizeof(uint64_t) * HW); /* (R << 32) | point index */
  for (size_t i = 0; i < HW; i++) best[i] = UINT64_MAX;
  for (uint32_t i = 0; i < n; i++) {
    uint32_t R;
    int64_t pix = js_pixel(xyz[3 * (size_t)i], xyz[3 * (size_t)i + 1], xyz[3 * (size_t)i + 2], k, H, W, alt, a0,
                           clockwise, rmin, rcap, &R);
    if (pix < 0) continue;
    uint64_t key = ((uint64_t)R << 32) | i;
    if (key < best[pix]) best[pix] = key; /* the nearest point wins */
  }
  for (size_t p = 0; p < HW; p++) {
    int hit = best[p] != UINT64_MAX;
    uint32_t idx = (uint32_t)best[p];
    js_store(range_out, range_bytes, p, hit ? (uint32_t)(best[p] >> 32) : 0u);
    for (uint32_t a = 0; a < n_attr; a++)
      js_store(attr_out[a], attr_bytes[a], p, hit ? js_quantize_attr(attr[a][idx], attr_scale[a], attr_bytes[a]) : 0u);
  }
  free(best);
  free(alt);
  return JS_OK;
}
