// Input standardization (Sec. III-A): one scan of floating-point Cartesian
// points -> an H x W range image (rows by altitude, columns by azimuth) and
// attribute images, quantized to unsigned integers, 0 where no valid point.
//
// The paper leaves the arithmetic open; this library fixes it in integers so
// that every decision is exact (no floating-point rounding can move a point
// to another pixel between two implementations):
//   coordinates  X = round-half-even(x * k), the product rounded to float32
//                (k = range units per metre); |x * k| >= 2^31 or NaN drops
//                the point
//   range        R = nearest integer to sqrt(X^2 + Y^2 + Z^2) (exact integer
//                square root)
//   angles       binary angles, 2^32 per turn, by CORDIC vectoring (Volder,
//                1959) in 32-bit integers: 30 micro-rotations of atan(2^-i)
//                on the vector scaled by a power of two (arithmetic shifts)
//                so that its larger component has 29 bits. Azimuth of (X, Y)
//                (counterclockwise from +x, 0 for X = Y = 0); elevation of
//                (rho, Z 2^f), rho = floor(sqrt(X^2 + Y^2) 2^f), f the
//                largest (possibly negative) integer keeping both below 2^29
//   pixel        row = nearest beam (midpoints between the beams' binary
//                altitudes; beyond half a spacing outside the first or last
//                beam the point is dropped), column = floor(((az - az0) mod
//                2^32) W / 2^32)
//   collisions   the nearest point wins (smallest R, then smallest index)
//   attributes   round-half-even(v * scale), the product rounded to float32,
//                clamped to the sample type, NaN and v * scale <= 0 -> 0
//
// Two launches per call of up to 256 scans: k_std_points (one thread per
// point, one grid row per scan: pixel and an atomicMin of the key (R << 32 |
// index in the scan) into a per-pixel word, L2-resident for a few scans) and
// k_std_pixels (one thread per pixel of every scan, grid-stride: the winning
// point's range and attributes, and the key word reset for the next call).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "jiffy.h"
#include "jiffy_types.h"

namespace jiffy {
namespace {

constexpr int kStdIter = 30;         // CORDIC micro-rotations
constexpr int kNormBits = 29;        // CORDIC inputs scaled to this many bits
constexpr uint32_t kStdMaxAttr = 16;
constexpr uint32_t kStdMaxScans = 256;  // scans per call
constexpr double kPi = 3.14159265358979323846;

struct StdAttr {
  const float* v;
  void* out;
  float scale;
  uint32_t bytes;
};

struct StdParams {
  uint32_t H, W, T, clockwise, range_bytes, rmin, rmax, n_attr;
  float k;
  uint32_t az0;          // binary angle (2^32 per turn)
  int top, bottom;       // elevation limits (H > 1)
  const int* mid;        // [H - 1] midpoints between beams, decreasing
  int atan_t[kStdIter];
  const float* xyz;
  unsigned long long* keys;  // [T][H * W]
  void* range_out;           // [T][H * W]
  StdAttr attr[kStdMaxAttr];
  unsigned long long off[kStdMaxScans + 1];  // scan t's points: [off[t], off[t + 1])
};

__device__ __forceinline__ bool coord(float v, float k, long long& out) {
  const float p = __fmul_rn(v, k);
  if (!(fabsf(p) < 2147483648.0f)) return false;  // also NaN
  out = (long long)rintf(p);                     // round half to even
  return true;
}

// floor(sqrt(n)) for n < 2^63.6 (n < 3 2^62): a float32 estimate (the FP64
// units of this GPU are few), one Newton correction r += (n - r^2) / 2r in
// float32 (leaves r within one of the root), then exact integer corrections.
__device__ __forceinline__ unsigned long long isqrt64(unsigned long long n) {
  if (n == 0ull) return 0ull;
  unsigned long long r = (unsigned long long)__fsqrt_rn(__ull2float_rn(n));
  const long long e = (long long)(n - r * r);  // |e| < 2^42
  r = (unsigned long long)((long long)r + __float2ll_rn(__fdividef((float)e, 2.0f * (float)r)));
  while (r * r > n) r--;
  while ((r + 1) * (r + 1) <= n) r++;
  return r;
}

__device__ __forceinline__ int cordic_vec(int x, int y, const int* t) {
  int ang = 0;
#pragma unroll
  for (int i = 0; i < kStdIter; i++) {
    const int xs = x >> i, ys = y >> i;
    const bool up = y > 0;
    x += up ? ys : -ys;
    y += up ? -xs : xs;
    ang += up ? t[i] : -t[i];
  }
  return ang;
}

__device__ __forceinline__ int bit_length(unsigned long long m) { return 64 - __clzll(m); }

// v 2^s, floor division (arithmetic shift) for s < 0
__device__ __forceinline__ long long scale2(long long v, int s) { return s >= 0 ? v * (1ll << s) : (v >> (-s)); }

__device__ __forceinline__ uint32_t azimuth(long long X, long long Y, const int* t) {
  if (X == 0 && Y == 0) return 0u;
  const unsigned long long m = (unsigned long long)(X < 0 ? -X : X) | (unsigned long long)(Y < 0 ? -Y : Y);
  const int s = kNormBits - bit_length(m);
  int x = (int)scale2(X, s), y = (int)scale2(Y, s);
  uint32_t base = 0u;
  if (x < 0) {  // a half turn first
    x = -x;
    y = -y;
    base = 0x80000000u;
  }
  return base + (uint32_t)cordic_vec(x, y, t);  // modulo 2^32
}

__device__ __forceinline__ int elevation(long long X, long long Y, long long Z, const int* t) {
  const unsigned long long h = (unsigned long long)(X * X) + (unsigned long long)(Y * Y);
  const unsigned long long z2 = (unsigned long long)(Z * Z);
  const unsigned long long m = h > z2 ? h : z2;
  if (m == 0) return 0;
  const int e = bit_length(m);
  const int f = e <= 2 * kNormBits ? (2 * kNormBits - e) / 2 : -((e - 2 * kNormBits + 1) / 2);  // m 4^f < 2^58
  const unsigned long long hs = f >= 0 ? h << (2 * f) : h >> (-2 * f);
  return cordic_vec((int)isqrt64(hs), (int)scale2(Z, f), t);
}

__device__ __forceinline__ void store_sample(void* p, uint32_t bytes, size_t i, uint32_t v) {
  if (bytes == 4) static_cast<uint32_t*>(p)[i] = v;
  else if (bytes == 2) static_cast<uint16_t*>(p)[i] = (uint16_t)v;
  else static_cast<uint8_t*>(p)[i] = (uint8_t)v;
}

__device__ __forceinline__ uint32_t quantize_attr(float v, float scale, uint32_t bytes) {
  const float p = __fmul_rn(v, scale);
  const uint32_t mx = bytes == 4 ? 0xffffffffu : ((1u << (8 * bytes)) - 1u);
  if (!(p > 0.0f)) return 0u;  // also NaN
  if (p >= (float)mx) return mx;
  const float r = rintf(p);
  return r >= (float)mx ? mx : (uint32_t)r;
}

__global__ void __launch_bounds__(256) k_std_points(const __grid_constant__ StdParams p) {
  __shared__ int t[kStdIter];
  for (int i = threadIdx.x; i < kStdIter; i += blockDim.x) t[i] = p.atan_t[i];
  __syncthreads();
  const uint32_t scan = blockIdx.y;
  const unsigned long long p0 = p.off[scan], n = p.off[scan + 1] - p0;
  unsigned long long* keys = p.keys + (size_t)scan * p.H * p.W;
  for (unsigned long long ii = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; ii < n;
       ii += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)ii;  // index within the scan (< 2^32)
    long long X, Y, Z;
    const float* q = p.xyz + 3ull * (p0 + ii);
    if (!coord(__ldg(q), p.k, X) || !coord(__ldg(q + 1), p.k, Y) || !coord(__ldg(q + 2), p.k, Z)) continue;
    if (p.clockwise) Y = -Y;
    const unsigned long long n = (unsigned long long)(X * X) + (unsigned long long)(Y * Y) +
                                 (unsigned long long)(Z * Z);  // < 3 2^62
    const unsigned long long r = isqrt64(n);
    const unsigned long long R = r + ((n - r * r) > r ? 1ull : 0ull);
    if (R < 1 || R < p.rmin || R > p.rmax) continue;
    uint32_t row = 0;
    if (p.H > 1) {
      const int el = elevation(X, Y, Z, t);
      if (el > p.top || el < p.bottom) continue;
      uint32_t lo = 0, hi = p.H - 1;  // row = number of midpoints above el
      while (lo < hi) {
        const uint32_t m = (lo + hi) >> 1;
        if (__ldg(p.mid + m) > el) lo = m + 1;
        else hi = m;
      }
      row = lo;
    }
    const uint32_t a = azimuth(X, Y, t) - p.az0;  // modulo 2^32
    const uint32_t col = (uint32_t)(((unsigned long long)a * p.W) >> 32);
    atomicMin(keys + (size_t)row * p.W + col, (R << 32) | i);
  }
}

__global__ void __launch_bounds__(256) k_std_pixels(const __grid_constant__ StdParams p) {
  const uint32_t HW = p.H * p.W;  // <= 2^26
  const size_t total = (size_t)HW * p.T;
  const uint32_t G = gridDim.x * blockDim.x, g0 = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t dt = G / HW, dr = G % HW;  // the stride as (scans, pixels)
  uint32_t t = g0 / HW, r = g0 % HW;        // this thread's scan and pixel
  for (size_t px = g0; px < total; px += G) {
    const unsigned long long key = p.keys[px];
    const bool hit = key != ~0ull;
    if (hit) p.keys[px] = ~0ull;  // ready for the next call
    const unsigned long long idx = p.off[t] + (uint32_t)key;  // the point, across the call
    store_sample(p.range_out, p.range_bytes, px, hit ? (uint32_t)(key >> 32) : 0u);
    for (uint32_t a = 0; a < p.n_attr; a++) {
      const StdAttr& at = p.attr[a];
      store_sample(at.out, at.bytes, px, hit ? quantize_attr(__ldg(at.v + idx), at.scale, at.bytes) : 0u);
    }
    t += dt;
    r += dr;
    if (r >= HW) {
      r -= HW;
      t++;
    }
  }
}

long long binary_angle(double rad) {
  return std::llround(rad / (2.0 * kPi) * 4294967296.0);  // 2^32 per turn
}

}  // namespace
}  // namespace jiffy

struct jiffy_standardizer {
  int device = 0;
  uint32_t H = 0, W = 0;
  jiffy::StdParams base{};
  int* d_mid = nullptr;
  unsigned long long* d_keys = nullptr;  // key_scans x H x W, all ~0 between calls
  uint32_t key_scans = 0;
  int sms = 0;
};

extern "C" {

jiffy_status jiffy_standardizer_create(jiffy_standardizer** out, const jiffy_sensor_desc* sd, int device) {
  using namespace jiffy;
  if (!out || !sd) return JIFFY_ERR_INVALID_ARG;
  *out = nullptr;
  const uint32_t H = sd->H, W = sd->W;
  if (H == 0 || H > kMaxH || W == 0 || W > kMaxW || !sd->beam_altitude || !(sd->units_per_m > 0.0f) ||
      !(sd->range_bytes == 2 || sd->range_bytes == 4) || !std::isfinite(sd->azimuth0))
    return JIFFY_ERR_INVALID_ARG;
  std::vector<long long> alt(H);
  std::vector<int> mid(H > 1 ? H - 1 : 1, 0);
  for (uint32_t b = 0; b < H; b++) {
    if (!std::isfinite(sd->beam_altitude[b])) return JIFFY_ERR_INVALID_ARG;
    alt[b] = binary_angle(sd->beam_altitude[b]);
    if (alt[b] > (1ll << 30) || alt[b] < -(1ll << 30) || (b > 0 && alt[b] >= alt[b - 1]))  // within +-90 deg
      return JIFFY_ERR_INVALID_ARG;
  }
  for (uint32_t b = 0; b + 1 < H; b++) mid[b] = (int)(alt[b + 1] + (alt[b] - alt[b + 1]) / 2);
  int prev = 0, ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return JIFFY_ERR_CUDA;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return JIFFY_ERR_CUDA;
  jiffy_standardizer* s = new (std::nothrow) jiffy_standardizer();
  jiffy_status st = s ? JIFFY_OK : JIFFY_ERR_NOMEM;
  if (st == JIFFY_OK) {
    s->device = device;
    s->H = H;
    s->W = W;
    StdParams& p = s->base;
    p.H = H;
    p.W = W;
    p.clockwise = sd->clockwise ? 1u : 0u;
    p.range_bytes = sd->range_bytes;
    p.rmin = sd->min_range;
    const uint32_t dmax = sd->range_bytes == 4 ? 0xffffffffu : 0xffffu;
    p.rmax = sd->max_range < dmax ? sd->max_range : dmax;
    p.k = sd->units_per_m;
    p.az0 = (uint32_t)(unsigned long long)binary_angle(sd->azimuth0);  // modulo 2^32
    if (H > 1) {
      p.top = (int)std::min<long long>(alt[0] + (alt[0] - alt[1]) / 2, 0x7fffffffll);
      p.bottom = (int)std::max<long long>(alt[H - 1] - (alt[H - 2] - alt[H - 1]) / 2, -0x7fffffffll - 1);
    }
    for (int i = 0; i < kStdIter; i++)
      p.atan_t[i] = (int)std::llround(std::atan(std::ldexp(1.0, -i)) / (2.0 * kPi) * 4294967296.0);
    if (cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaMalloc(&s->d_mid, sizeof(int) * mid.size()) != cudaSuccess ||
        cudaMalloc(&s->d_keys, sizeof(unsigned long long) * (size_t)H * W) != cudaSuccess ||
        cudaMemcpy(s->d_mid, mid.data(), sizeof(int) * mid.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(s->d_keys, 0xff, sizeof(unsigned long long) * (size_t)H * W) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess)
      st = JIFFY_ERR_CUDA;
    p.mid = s->d_mid;
    s->key_scans = 1;
  }
  if (st != JIFFY_OK && s) {
    cudaFree(s->d_mid);
    cudaFree(s->d_keys);
    delete s;
    s = nullptr;
  }
  cudaSetDevice(prev);
  *out = s;
  return st;
}

void jiffy_standardizer_destroy(jiffy_standardizer* s) {
  if (!s) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  cudaFree(s->d_mid);
  cudaFree(s->d_keys);
  cudaSetDevice(prev);
  delete s;
}

jiffy_status jiffy_standardize_seq(jiffy_standardizer* s, uint32_t n_scans, const float* xyz,
                                   const uint64_t* point_offsets, void* range_out, uint32_t n_attr,
                                   const jiffy_point_attr* attrs, void* cuda_stream) {
  using namespace jiffy;
  if (!s || n_scans == 0 || n_scans > kStdMaxScans || !point_offsets || !range_out || n_attr > kStdMaxAttr ||
      (n_attr && !attrs))
    return JIFFY_ERR_INVALID_ARG;
  StdParams p = s->base;
  unsigned long long max_n = 0;
  for (uint32_t t = 0; t < n_scans; t++) {
    if (point_offsets[t + 1] < point_offsets[t] || point_offsets[t + 1] - point_offsets[t] > 0xffffffffull)
      return JIFFY_ERR_INVALID_ARG;
    max_n = std::max<unsigned long long>(max_n, point_offsets[t + 1] - point_offsets[t]);
  }
  for (uint32_t t = 0; t <= n_scans; t++) p.off[t] = point_offsets[t];
  if (max_n && !xyz) return JIFFY_ERR_INVALID_ARG;
  p.T = n_scans;
  p.xyz = xyz;
  p.range_out = range_out;
  p.n_attr = n_attr;
  for (uint32_t a = 0; a < n_attr; a++) {
    const uint32_t b = attrs[a].dtype_bytes;
    if (!(b == 1 || b == 2 || b == 4) || !attrs[a].out || (max_n && !attrs[a].values)) return JIFFY_ERR_INVALID_ARG;
    p.attr[a] = StdAttr{attrs[a].values, attrs[a].out, attrs[a].scale, b};
  }
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(s->device) != cudaSuccess) return JIFFY_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const size_t HW = (size_t)s->H * s->W;
  jiffy_status rc = JIFFY_OK;
  if (n_scans > s->key_scans || !s->d_keys) {  // a larger pixel table: wait for the calls using the old one
    if (cudaStreamSynchronize(st) != cudaSuccess) rc = JIFFY_ERR_CUDA;
    cudaFree(s->d_keys);
    s->d_keys = nullptr;
    s->key_scans = 0;
    if (rc == JIFFY_OK) {
      const size_t bytes = sizeof(unsigned long long) * HW * n_scans;
      const cudaError_t me = cudaMalloc(&s->d_keys, bytes);
      if (me != cudaSuccess) rc = me == cudaErrorMemoryAllocation ? JIFFY_ERR_NOMEM : JIFFY_ERR_CUDA;
      else if (cudaMemsetAsync(s->d_keys, 0xff, bytes, st) != cudaSuccess) rc = JIFFY_ERR_CUDA;
      else s->key_scans = n_scans;
    }
  }
  if (rc == JIFFY_OK) {
    p.keys = s->d_keys;
    const uint32_t target = 16u * (uint32_t)s->sms;  // CTAs of 256 threads in flight, grid-stride beyond
    if (max_n) {
      const unsigned long long need = (max_n + 255u) / 256u;
      const uint32_t bx = (uint32_t)std::max<unsigned long long>(
          1ull, std::min<unsigned long long>(need, (target + n_scans - 1) / n_scans));
      k_std_points<<<dim3(bx, n_scans), 256, 0, st>>>(p);
    }
    k_std_pixels<<<(uint32_t)std::min<size_t>(target, (HW * n_scans + 255) / 256), 256, 0, st>>>(p);
    if (cudaGetLastError() != cudaSuccess) rc = JIFFY_ERR_CUDA;
  }
  cudaSetDevice(prev);
  return rc;
}

jiffy_status jiffy_standardize(jiffy_standardizer* s, const float* xyz, uint32_t n_points, void* range_out,
                               uint32_t n_attr, const jiffy_point_attr* attrs, void* cuda_stream) {
  const uint64_t off[2] = {0, n_points};
  return jiffy_standardize_seq(s, 1, xyz, off, range_out, n_attr, attrs, cuda_stream);
}

}  // extern "C"
