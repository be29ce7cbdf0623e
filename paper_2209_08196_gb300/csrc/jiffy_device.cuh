// Device-side building blocks of the Jiffy codec kernels (sm_103a).
//
// Jiffy: Ford & Ford, arXiv 2209.08196. Quantization (Sec. III-B), ZigZag
// (Eq. 1), PFOR-style block sizing (Sec. II) and the prefix/look-back
// machinery the encoder and decoder kernels share.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "jiffy_types.h"

namespace jiffy {

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Host: records a timing event on st; inside a stream capture it becomes an
// event-record node of the graph, so replays time their kernels too.
inline cudaError_t record_event(void* ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    return cudaEventRecordWithFlags(reinterpret_cast<cudaEvent_t>(ev), st, cudaEventRecordExternal);
  return cudaEventRecord(reinterpret_cast<cudaEvent_t>(ev), st);
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t warp_id() { return threadIdx.x >> 5; }

__device__ __forceinline__ uint32_t load_sample(const uint8_t* row, uint32_t s, uint32_t x) {
  if (s == 4) return reinterpret_cast<const uint32_t*>(row)[x];
  if (s == 2) return reinterpret_cast<const uint16_t*>(row)[x];
  return row[x];
}

// Loads that bypass L1: used for data another CTA wrote during this kernel.
__device__ __forceinline__ uint32_t load_sample_cg(const uint8_t* row, uint32_t s, uint32_t x) {
  if (s == 4) return __ldcg(reinterpret_cast<const unsigned int*>(row) + x);
  if (s == 2) return __ldcg(reinterpret_cast<const unsigned short*>(row) + x);
  return __ldcg(reinterpret_cast<const unsigned char*>(row) + x);
}

__device__ __forceinline__ void store_sample(uint8_t* row, uint32_t s, uint32_t x, uint32_t v) {
  if (s == 4) reinterpret_cast<uint32_t*>(row)[x] = v;
  else if (s == 2) reinterpret_cast<uint16_t*>(row)[x] = (uint16_t)v;
  else row[x] = (uint8_t)v;
}

__device__ __forceinline__ uint32_t warp_incl_scan_fwd(uint32_t v) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= (uint32_t)o) v += t;
  }
  return v;
}

// Warp-wide prefetch of [p, p + bytes) into L1, one 128-byte line per lane per
// round: a single round of independent requests instead of many dependent
// ones later.
__device__ __forceinline__ void prefetch_l1(const void* p, uint32_t bytes) {
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(p) & ~uintptr_t(127);
  const uintptr_t a1 = reinterpret_cast<uintptr_t>(p) + bytes;
  for (uintptr_t a = a0 + 128u * (threadIdx.x & 31u); a < a1; a += 32u * 128u)
    asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
}

// Groups of 8 consecutive samples move as one vector when the group is
// aligned: 32 bytes (u32), 16 bytes (u16) or 8 bytes (u8). Group starts are
// multiples of 8 samples, so a vector-aligned row base suffices.
__device__ __forceinline__ bool vec_ok(const void* row, uint32_t s) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(row);
  return s == 1 ? (a & 7u) == 0 : (a & 15u) == 0;
}

// Loads the nvalid (<= 8) samples from pixel x0 (missing ones read as 0);
// CG bypasses L1 (data other CTAs wrote during this kernel).
// Scalar paths for ragged or unaligned groups (rare), kept out of line so the
// hot loops stay small.
template <bool CG>
static __device__ __noinline__ void load8_slow(const uint8_t* row, uint32_t s, uint32_t x0, uint32_t nvalid, uint32_t* v) {
  for (uint32_t i = 0; i < 8; i++)
    v[i] = i < nvalid ? (CG ? load_sample_cg(row, s, x0 + i) : load_sample(row, s, x0 + i)) : 0u;
}

static __device__ __noinline__ void store8_slow(uint8_t* row, uint32_t s, uint32_t x0, uint32_t nvalid, const uint32_t* v) {
  for (uint32_t i = 0; i < nvalid; i++) store_sample(row, s, x0 + i, v[i]);
}

template <bool CG>
__device__ __forceinline__ void load8(const uint8_t* row, uint32_t s, uint32_t x0, uint32_t nvalid, bool vec,
                                      uint32_t (&v)[8]) {
  if (vec && nvalid == 8) {
    if (s == 4) {
      const uint4* q = reinterpret_cast<const uint4*>(row + 4ull * x0);
      const uint4 a = CG ? __ldcg(q) : q[0];
      const uint4 b = CG ? __ldcg(q + 1) : q[1];
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else if (s == 2) {
      const uint4* q = reinterpret_cast<const uint4*>(row + 2ull * x0);
      const uint4 a = CG ? __ldcg(q) : q[0];
      const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int i = 0; i < 4; i++) { v[2 * i] = w[i] & 0xffffu; v[2 * i + 1] = w[i] >> 16; }
    } else {
      const uint2* q = reinterpret_cast<const uint2*>(row + x0);
      const uint2 a = CG ? __ldcg(q) : q[0];
#pragma unroll
      for (int i = 0; i < 4; i++) { v[i] = (a.x >> (8 * i)) & 0xffu; v[4 + i] = (a.y >> (8 * i)) & 0xffu; }
    }
    return;
  }
  uint32_t tmp[8];
  load8_slow<CG>(row, s, x0, nvalid, tmp);
#pragma unroll
  for (int i = 0; i < 8; i++) v[i] = tmp[i];
}

__device__ __forceinline__ void store8(uint8_t* row, uint32_t s, uint32_t x0, uint32_t nvalid, bool vec,
                                       const uint32_t (&v)[8]) {
  if (vec && nvalid == 8) {
    if (s == 4) {
      uint4* q = reinterpret_cast<uint4*>(row + 4ull * x0);
      q[0] = make_uint4(v[0], v[1], v[2], v[3]);
      q[1] = make_uint4(v[4], v[5], v[6], v[7]);
    } else if (s == 2) {
      uint4* q = reinterpret_cast<uint4*>(row + 2ull * x0);
      q[0] = make_uint4((v[0] & 0xffffu) | (v[1] << 16), (v[2] & 0xffffu) | (v[3] << 16),
                        (v[4] & 0xffffu) | (v[5] << 16), (v[6] & 0xffffu) | (v[7] << 16));
    } else {
      uint2* q = reinterpret_cast<uint2*>(row + x0);
      q[0] = make_uint2((v[0] & 0xffu) | ((v[1] & 0xffu) << 8) | ((v[2] & 0xffu) << 16) | (v[3] << 24),
                        (v[4] & 0xffu) | ((v[5] & 0xffu) << 8) | ((v[6] & 0xffu) << 16) | (v[7] << 24));
    }
    return;
  }
  uint32_t tmp[8];
#pragma unroll
  for (int i = 0; i < 8; i++) tmp[i] = v[i];
  store8_slow(row, s, x0, nvalid, tmp);
}

// Compile-time sample width variants (S = 1, 2 or 4 bytes).
template <uint32_t S, bool CG>
__device__ __forceinline__ void load8s(const uint8_t* row, uint32_t x0, uint32_t nvalid, bool vec, uint32_t (&v)[8]) {
  if (vec && nvalid == 8) {
    if constexpr (S == 4) {
      const uint4* q = reinterpret_cast<const uint4*>(row + 4ull * x0);
      const uint4 a = CG ? __ldcg(q) : q[0];
      const uint4 b = CG ? __ldcg(q + 1) : q[1];
      v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else if constexpr (S == 2) {
      const uint4* q = reinterpret_cast<const uint4*>(row + 2ull * x0);
      const uint4 a = CG ? __ldcg(q) : q[0];
      const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int i = 0; i < 4; i++) { v[2 * i] = w[i] & 0xffffu; v[2 * i + 1] = w[i] >> 16; }
    } else {
      const uint2* q = reinterpret_cast<const uint2*>(row + x0);
      const uint2 a = CG ? __ldcg(q) : q[0];
#pragma unroll
      for (int i = 0; i < 4; i++) { v[i] = (a.x >> (8 * i)) & 0xffu; v[4 + i] = (a.y >> (8 * i)) & 0xffu; }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 8; i++)
    v[i] = (uint32_t)i < nvalid ? (CG ? load_sample_cg(row, S, x0 + i) : load_sample(row, S, x0 + i)) : 0u;
}

template <uint32_t S>
__device__ __forceinline__ void store8s(uint8_t* row, uint32_t x0, uint32_t nvalid, bool vec, const uint32_t (&v)[8]) {
  if (vec && nvalid == 8) {
    if constexpr (S == 4) {
      uint4* q = reinterpret_cast<uint4*>(row + 4ull * x0);
      q[0] = make_uint4(v[0], v[1], v[2], v[3]);
      q[1] = make_uint4(v[4], v[5], v[6], v[7]);
    } else if constexpr (S == 2) {
      uint4* q = reinterpret_cast<uint4*>(row + 2ull * x0);
      q[0] = make_uint4((v[0] & 0xffffu) | (v[1] << 16), (v[2] & 0xffffu) | (v[3] << 16),
                        (v[4] & 0xffffu) | (v[5] << 16), (v[6] & 0xffffu) | (v[7] << 16));
    } else {
      uint2* q = reinterpret_cast<uint2*>(row + x0);
      q[0] = make_uint2((v[0] & 0xffu) | ((v[1] & 0xffu) << 8) | ((v[2] & 0xffu) << 16) | (v[3] << 24),
                        (v[4] & 0xffu) | ((v[5] & 0xffu) << 8) | ((v[6] & 0xffu) << 16) | (v[7] << 24));
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 8; i++)
    if ((uint32_t)i < nvalid) store_sample(row, S, x0 + i, v[i]);
}

__device__ __forceinline__ uint32_t warp_excl_scan(uint32_t v, uint32_t& total) {
  const uint32_t incl = warp_incl_scan_fwd(v);
  total = __shfl_sync(0xffffffffu, incl, 31);
  return incl - v;
}

// Quantization, Sec. III-B: q = min(floor((v + floor(P/2)) / P), floor(max/P)).
// qkind 2 divides with the round-up reciprocal m = ceil(2^64/P) (Granlund and
// Montgomery, "Division by invariant integers using multiplication", 1994):
// for a dividend n < 2^33 the product n*m/2^64 exceeds n/P by less than
// 2^-31 <= 1/P, which never crosses the next integer, so the high word of
// n*m is exactly floor(n/P) for P <= 2^31. Larger P leave q in {0, 1, 2}.
__device__ __forceinline__ uint32_t quantize(uint32_t v, const AttrDev& a) {
  if (a.P == 1) return v;
  unsigned long long n = (unsigned long long)v + (a.P >> 1);
  uint32_t q;
  if (a.P <= 0x80000000u) q = (uint32_t)__umul64hi(n, a.magic);
  else q = (uint32_t)(n >= a.P) + (uint32_t)(n >= 2ull * a.P);
  return q < a.qmax ? q : a.qmax;
}

// Compile-time quantizer kind (AttrDev::qkind): 0 identity, 1 32-bit
// multiply-high and shift on the clamped input, 2 the 64-bit form above.
template <int QU>
__device__ __forceinline__ uint32_t quant(uint32_t v, const AttrDev& a) {
  if constexpr (QU == 0) {
    return v;
  } else if constexpr (QU == 1) {
    return __umulhi(min(v, a.lim) + a.half, a.m32) >> a.sh;
  } else {
    return quantize(v, a);
  }
}

// ZigZag, Eq. 1: 2|x| + [x < 0] with x the residual read as a signed 32-bit
// value; everything modulo 2^32 (so ZigZag(-2^31) = 1).
__device__ __forceinline__ uint32_t zigzag(uint32_t d) {
  bool neg = (int32_t)d < 0;
  uint32_t mag = neg ? 0u - d : d;
  return (mag << 1) + (neg ? 1u : 0u);
}

// Inverse of Eq. 1: even z -> z/2; odd z -> -(z >> 1), except z = 1, whose
// magnitude 2^31 wrapped to 0 in the forward map.
__device__ __forceinline__ uint32_t unzigzag(uint32_t z) {
  uint32_t m = z >> 1;
  if (z & 1u) return 0u - (m ? m : 0x80000000u);
  return m;
}

// Body bytes of a block of n values coded with width b, e exceptions and
// widest value wmax bits (Sec. II, PFOR: low bits for all, exceptions apart).
__device__ __forceinline__ uint32_t block_body_bytes(uint32_t n, uint32_t b, uint32_t e, uint32_t wmax) {
  uint32_t bytes = 4u * ((n * b + 31u) >> 5);
  if (e) bytes += 4u * ((e + 3u) >> 2) + 4u * ((e * (wmax - b) + 31u) >> 5);
  return bytes;
}

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const uint32_t lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= (uint32_t)o) v += t;
  }
  return v;
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v) { return __reduce_add_sync(0xffffffffu, v); }

// In-place exclusive prefix sum of a[0..n) in shared memory; returns the
// total. Every thread of the CTA calls it. tmp: kWarps + 1 words.
__device__ inline uint32_t block_excl_scan(uint32_t* a, uint32_t n, uint32_t* tmp) {
  const uint32_t per = (n + kThreads - 1) / kThreads;
  const uint32_t beg = min(threadIdx.x * per, n), end = min(beg + per, n);
  uint32_t sum = 0;
  for (uint32_t i = beg; i < end; i++) sum += a[i];
  uint32_t incl = warp_incl_scan(sum);
  if (lane_id() == 31) tmp[warp_id()] = incl;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t w = threadIdx.x < (uint32_t)kWarps ? tmp[threadIdx.x] : 0u;
    uint32_t wi = warp_incl_scan(w);
    if (threadIdx.x < (uint32_t)kWarps) tmp[threadIdx.x] = wi - w;
    if (threadIdx.x == kWarps - 1) tmp[kWarps] = wi;
  }
  __syncthreads();
  uint32_t run = tmp[warp_id()] + incl - sum;
  for (uint32_t i = beg; i < end; i++) {
    uint32_t v = a[i];
    a[i] = run;
    run += v;
  }
  uint32_t total = tmp[kWarps];
  __syncthreads();
  return total;
}

// ---- decoupled look-back (Merrill & Garland, "Single-pass Parallel Prefix
// Scan with Decoupled Look-back", 2016) over 64-bit status words:
// bits 62..63 = flag (0 empty, 1 aggregate, 2 inclusive prefix, 3 error),
// bits 0..61 = value.
constexpr unsigned long long kStAgg = 1ull << 62;
constexpr unsigned long long kStInc = 2ull << 62;
constexpr unsigned long long kStErr = 3ull << 62;
constexpr unsigned long long kStValMask = (1ull << 62) - 1;

__device__ __forceinline__ unsigned long long st_load(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}
// A status word carries its value with its flag, so nothing has to become
// visible before it: one relaxed 64-bit store, no fence.
__device__ __forceinline__ void st_store(unsigned long long* p, unsigned long long v) {
  *reinterpret_cast<volatile unsigned long long*>(p) = v;
}

// Outcome of a look-back step.
enum : int { kLbFail = 0, kLbOk = 1 };

// Warp-wide window read for the look-back: kLookQ x 32 status words per
// round, entry (q, lane) = word j - 32q - lane (nearest first), `beyond` past
// the segment start. Finds the nearest entry that decides the look-back,
// re-reading while an entry nearer than it is still empty; gives up after
// kSpinLimitNs. stop = kLookQ * 32: no decision in this window.
constexpr uint32_t kLookQ = 4;

template <typename Decides>
__device__ __forceinline__ int lookback_window(const unsigned long long* st, int64_t j, uint32_t seg_start,
                                               unsigned long long beyond, Decides decides,
                                               unsigned long long (&s)[kLookQ], uint32_t& stop) {
  const uint32_t lane = lane_id();
  unsigned long long t0 = 0;
  uint32_t ns = 32;
  while (true) {
#pragma unroll
    for (uint32_t q = 0; q < kLookQ; q++) {
      const int64_t idx = j - (int64_t)(32u * q + lane);
      s[q] = idx >= (int64_t)seg_start ? st_load(st + idx) : beyond;
    }
    bool err = false, waiting = false;
    stop = kLookQ * 32u;
#pragma unroll
    for (uint32_t q = 0; q < kLookQ; q++) {
      const uint32_t flag = (uint32_t)(s[q] >> 62);
      err |= flag == 3u;
      const uint32_t dec = __ballot_sync(0xffffffffu, flag != 0u && decides(s[q]));
      const uint32_t empty = __ballot_sync(0xffffffffu, flag == 0u);
      if (stop == kLookQ * 32u) {
        const uint32_t first = dec ? (uint32_t)(__ffs(dec) - 1) : 32u;
        if (empty & (first == 32u ? 0xffffffffu : ((1u << first) - 1u))) waiting = true;
        if (first < 32u) stop = 32u * q + first;
      }
    }
    if (__any_sync(0xffffffffu, err)) return kLbFail;  // an upstream error
    if (!waiting) return kLbOk;
    if (t0 == 0) t0 = global_timer_ns();
    else if (global_timer_ns() - t0 > kSpinLimitNs) return kLbFail;
    __nanosleep(ns);
    if (ns < 512) ns <<= 1;
  }
}

// Warp-wide. "Last valid" look-back for the delta carry: value bit 32 =
// has-a-residual, bits 0..31 = the last residual. The nearest predecessor
// that has a residual or holds an inclusive value decides; the segment start
// counts as a residual of 0 (e[-1] = 0).
__device__ inline bool lookback_last(const unsigned long long* st, uint32_t k, uint32_t seg_start,
                                     uint32_t& carry) {
  int64_t j = (int64_t)k - 1;
  while (true) {
    unsigned long long s[kLookQ];
    uint32_t stop;
    if (lookback_window(st, j, seg_start, kStInc | (1ull << 32),
                        [](unsigned long long x) { return ((x >> 62) == 2ull) || ((x >> 32) & 1ull); }, s,
                        stop) != kLbOk)
      return false;
    if (stop < kLookQ * 32u) {
      uint32_t c = 0;
#pragma unroll
      for (uint32_t q = 0; q < kLookQ; q++) {
        const uint32_t v = __shfl_sync(0xffffffffu, (uint32_t)s[q], stop & 31u);
        if (q == stop / 32u) c = v;
      }
      carry = c;
      return true;
    }
    j -= kLookQ * 32;
  }
}

// ---- bit-sliced counting (carry-save adders, as in the Harley-Seal
// population count: Warren, "Hacker's Delight", 2nd ed., Sec. 5-1).
// csa: per bit position, a + b + c = 2 * hi + lo.
__device__ __forceinline__ void csa(uint32_t& hi, uint32_t& lo, uint32_t a, uint32_t b, uint32_t c) {
  const uint32_t u = a ^ b;
  hi = (a & b) | (u & c);
  lo = u ^ c;
}

// Unary code of a value's bit width: bits 0 .. W(z)-1 set, W(z) = bits
// needed to write z (0 for z = 0). Bit b is set exactly when z needs more
// than b bits. (PTX shr clamps the shift amount at 32, giving 0 for z = 0.)
__device__ __forceinline__ uint32_t width_unary(uint32_t z) {
  uint32_t u;
  asm("shr.b32 %0, %1, %2;" : "=r"(u) : "r"(0xffffffffu), "r"((uint32_t)__clz(z)));
  return u;
}

}  // namespace jiffy
