// Host side of the Jiffy C ABI (include/jiffy.h): stream handles, device
// state and scratch, argument checks, kernel launches and status mapping.
// Every step of the codec itself runs in the kernels of jiffy_encode.cu and
// jiffy_decode.cu; this file only marshals pointers and sizes.
#include "jiffy.h"

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "jiffy_kernels.h"

using jiffy::AttrDev;

struct jiffy_stream {
  int device = 0;
  jiffy_role role = JIFFY_ENCODER;
  uint32_t H = 0, W = 0, A = 0;
  jiffy_options opt{4, -1};
  std::vector<AttrDev> attrs;
  AttrDev* d_attrs = nullptr;
  uint8_t* d_state[2] = {nullptr, nullptr};  // previous scan, ping-pong
  std::vector<size_t> plane_off;              // byte offset of attribute a in a state buffer
  int cur = 0;                                // state buffer holding the previous scan
  uint32_t frame = 0;                         // frames since create/reset
  uint8_t* d_scratch = nullptr;
  size_t scratch_cap = 0;
  uint8_t* h_pinned = nullptr;
  size_t pinned_cap = 0;
  bool profile = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  float kernel_ms[3] = {0, 0, 0};
  uint32_t n_kernel_ms = 0;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves consecutive 256-byte aligned regions out of one buffer.
struct Carver {
  size_t off = 0;
  size_t take(size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  }
};

uint64_t magic_for(uint32_t P) {
  if (P < 2 || P > 0x80000000u) return 0;
  // ceil(2^64 / P) = floor((2^64 - 1) / P) + 1
  return (~0ull) / P + 1ull;
}

jiffy_status ensure_scratch(jiffy_stream* s, size_t dev_bytes, size_t host_bytes) {
  if (dev_bytes > s->scratch_cap) {
    if (s->d_scratch) cudaFree(s->d_scratch);
    s->d_scratch = nullptr;
    s->scratch_cap = 0;
    size_t cap = align_up(dev_bytes + dev_bytes / 4, 1 << 20);
    if (cudaMalloc(&s->d_scratch, cap) != cudaSuccess) return JIFFY_ERR_NOMEM;
    s->scratch_cap = cap;
  }
  if (host_bytes > s->pinned_cap) {
    if (s->h_pinned) cudaFreeHost(s->h_pinned);
    s->h_pinned = nullptr;
    s->pinned_cap = 0;
    size_t cap = align_up(host_bytes + host_bytes / 4, 1 << 16);
    if (cudaMallocHost(&s->h_pinned, cap) != cudaSuccess) return JIFFY_ERR_NOMEM;
    s->pinned_cap = cap;
  }
  return JIFFY_OK;
}

jiffy_status map_device_error(uint32_t err) {
  if (err & jiffy::kErrTimeout) return JIFFY_ERR_TIMEOUT;
  if (err & jiffy::kErrCorrupt) return JIFFY_ERR_CORRUPT;
  if (err & jiffy::kErrCapacity) return JIFFY_ERR_CAPACITY;
  return JIFFY_OK;
}

// Reads the event intervals of the last call (after its synchronize).
void read_kernel_times(jiffy_stream* s, uint32_t n_kernels) {
  s->n_kernel_ms = 0;
  if (!s->profile) return;
  for (uint32_t i = 0; i < n_kernels; i++) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, s->ev[i], s->ev[i + 1]) != cudaSuccess) return;
    s->kernel_ms[i] = ms;
  }
  s->n_kernel_ms = n_kernels;
}

uint32_t stream_header_bytes(uint32_t A) { return 16u + 8u * A; }
uint32_t frame_header_bytes(uint32_t A) { return 8u + 12u * A; }

}  // namespace

extern "C" {

const char* jiffy_status_string(jiffy_status st) {
  switch (st) {
    case JIFFY_OK: return "ok";
    case JIFFY_ERR_INVALID_ARG: return "invalid argument";
    case JIFFY_ERR_CAPACITY: return "output capacity too small";
    case JIFFY_ERR_CORRUPT: return "corrupt or mismatching stream";
    case JIFFY_ERR_STATE: return "invalid stream state";
    case JIFFY_ERR_TIMEOUT: return "device wait timed out";
    case JIFFY_ERR_CUDA: return "CUDA error";
    case JIFFY_ERR_NOMEM: return "out of memory";
  }
  return "unknown status";
}

size_t jiffy_max_encoded_size(uint32_t H, uint32_t W, uint32_t n_attr, const jiffy_attr_desc* attrs,
                              uint32_t n_scans) {
  (void)attrs;
  if (H == 0 || W == 0 || n_attr == 0) return 0;
  const size_t section = 8ull * H + (size_t)H * jiffy::row_bound_bytes(W);
  const size_t frame = frame_header_bytes(n_attr) + (size_t)n_attr * section;
  return stream_header_bytes(n_attr) + (size_t)n_scans * frame;
}

jiffy_status jiffy_stream_create(jiffy_stream** out, jiffy_role role, uint32_t H, uint32_t W, uint32_t n_attr,
                                 const jiffy_attr_desc* attrs, const jiffy_options* opt, int device) {
  if (!out || !attrs) return JIFFY_ERR_INVALID_ARG;
  *out = nullptr;
  if (role != JIFFY_ENCODER && role != JIFFY_DECODER) return JIFFY_ERR_INVALID_ARG;
  if (H == 0 || H > jiffy::kMaxH || W == 0 || W > jiffy::kMaxW || n_attr == 0 || n_attr > jiffy::kMaxAttr)
    return JIFFY_ERR_INVALID_ARG;
  jiffy_options o{4, -1};
  if (opt) o = *opt;
  if (o.test_lines == 0 || o.test_lines > jiffy::kMaxTestLines || o.force_mode < -1 || o.force_mode > 1)
    return JIFFY_ERR_INVALID_ARG;
  for (uint32_t a = 0; a < n_attr; a++) {
    const uint32_t sz = attrs[a].dtype_bytes;
    if (!(sz == 1 || sz == 2 || sz == 4) || attrs[a].precision == 0) return JIFFY_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return JIFFY_ERR_CUDA;
  DeviceGuard g(device);
  if (!g.ok) return JIFFY_ERR_CUDA;
  jiffy_stream* s = new (std::nothrow) jiffy_stream();
  if (!s) return JIFFY_ERR_NOMEM;
  s->device = device;
  s->role = role;
  s->H = H;
  s->W = W;
  s->A = n_attr;
  s->opt = o;
  size_t state_bytes = 0;
  for (uint32_t a = 0; a < n_attr; a++) {
    AttrDev d{};
    d.s = attrs[a].dtype_bytes;
    d.P = attrs[a].precision;
    const uint32_t maxv = d.s == 4 ? 0xffffffffu : ((1u << (8 * d.s)) - 1u);
    d.qmax = maxv / d.P;
    d.magic = magic_for(d.P);
    s->attrs.push_back(d);
    s->plane_off.push_back(state_bytes);
    state_bytes = align_up(state_bytes + (size_t)H * W * d.s, 256);
  }
  jiffy_status st = JIFFY_OK;
  if (cudaMalloc(&s->d_attrs, sizeof(AttrDev) * n_attr) != cudaSuccess ||
      cudaMalloc(&s->d_state[0], state_bytes) != cudaSuccess ||
      cudaMalloc(&s->d_state[1], state_bytes) != cudaSuccess) {
    st = JIFFY_ERR_NOMEM;
  } else if (cudaMemcpy(s->d_attrs, s->attrs.data(), sizeof(AttrDev) * n_attr, cudaMemcpyHostToDevice) !=
                 cudaSuccess ||
             cudaMemset(s->d_state[0], 0, state_bytes) != cudaSuccess ||
             cudaMemset(s->d_state[1], 0, state_bytes) != cudaSuccess) {
    st = JIFFY_ERR_CUDA;
  }
  if (st != JIFFY_OK) {
    jiffy_stream_destroy(s);
    return st;
  }
  *out = s;
  return JIFFY_OK;
}

void jiffy_stream_destroy(jiffy_stream* s) {
  if (!s) return;
  DeviceGuard g(s->device);
  cudaDeviceSynchronize();
  if (s->d_attrs) cudaFree(s->d_attrs);
  if (s->d_state[0]) cudaFree(s->d_state[0]);
  if (s->d_state[1]) cudaFree(s->d_state[1]);
  if (s->d_scratch) cudaFree(s->d_scratch);
  if (s->h_pinned) cudaFreeHost(s->h_pinned);
  for (cudaEvent_t e : s->ev)
    if (e) cudaEventDestroy(e);
  delete s;
}

jiffy_status jiffy_stream_reset(jiffy_stream* s) {
  if (!s) return JIFFY_ERR_INVALID_ARG;
  s->frame = 0;
  return JIFFY_OK;
}

uint32_t jiffy_stream_frame_index(const jiffy_stream* s) { return s ? s->frame : 0u; }

jiffy_status jiffy_stream_set_profiling(jiffy_stream* s, int enable) {
  if (!s) return JIFFY_ERR_INVALID_ARG;
  if (enable && !s->ev[0]) {
    DeviceGuard g(s->device);
    if (!g.ok) return JIFFY_ERR_CUDA;
    for (cudaEvent_t& e : s->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return JIFFY_ERR_CUDA;
  }
  s->profile = enable != 0;
  s->n_kernel_ms = 0;
  return JIFFY_OK;
}

uint32_t jiffy_stream_kernel_times(const jiffy_stream* s, float* ms, uint32_t n) {
  if (!s) return 0;
  for (uint32_t i = 0; i < n && i < s->n_kernel_ms; i++) ms[i] = s->kernel_ms[i];
  return s->n_kernel_ms;
}

jiffy_status jiffy_encode_seq(jiffy_stream* s, uint32_t n_scans, const void* const* planes, void* out,
                              size_t out_capacity, uint64_t* frame_offsets, size_t* out_len, void* cuda_stream) {
  if (!s || !planes || !out || !out_len || n_scans == 0) return JIFFY_ERR_INVALID_ARG;
  if (s->role != JIFFY_ENCODER) return JIFFY_ERR_STATE;
  if (reinterpret_cast<uintptr_t>(out) & 15u) return JIFFY_ERR_INVALID_ARG;
  const uint32_t T = n_scans, A = s->A, H = s->H, W = s->W;
  for (size_t i = 0; i < (size_t)T * A; i++)
    if (!planes[i]) return JIFFY_ERR_INVALID_ARG;
  const unsigned long long items = (unsigned long long)T * A * H;
  if (items > 0x7fffffffull) return JIFFY_ERR_INVALID_ARG;
  DeviceGuard g(s->device);
  if (!g.ok) return JIFFY_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);

  // device scratch layout
  Carver c;
  const size_t o_cur = c.take(8ull * T * A), o_prev = c.take(8ull * T * A), o_next = c.take(8ull * A);
  const size_t o_modes = c.take(4ull * T * A);
  const size_t o_rb = c.take(4ull * items), o_rn = c.take(4ull * items), o_rc = c.take(4ull * items);
  const size_t o_secb = c.take(8ull * T * A), o_secn = c.take(4ull * T * A);
  const size_t o_zero = c.take(0);
  const size_t o_stc = c.take(8ull * items), o_tick = c.take(8);
  const size_t zero_bytes = c.off - o_zero;
  const size_t o_foff = c.take(8ull * (T + 1));
  const uint32_t slot_bytes = (jiffy::row_bound_bytes(W) + 15u) & ~15u;
  const size_t o_slots = c.take((size_t)slot_bytes * items);
  const size_t dev_bytes = c.off;
  // pinned host layout: pointer arrays (upload), then results (download)
  const size_t h_ptrs = 8ull * (2ull * T * A + A);
  const size_t h_res = align_up(h_ptrs, 64);
  const size_t host_bytes = h_res + 16 + 8ull * (T + 1);
  jiffy_status rs = ensure_scratch(s, dev_bytes, host_bytes);
  if (rs != JIFFY_OK) return rs;
  uint8_t* d = s->d_scratch;
  uint64_t* hp = reinterpret_cast<uint64_t*>(s->h_pinned);
  for (uint32_t t = 0; t < T; t++) {
    for (uint32_t a = 0; a < A; a++) {
      hp[t * A + a] = reinterpret_cast<uint64_t>(planes[t * A + a]);
      uint64_t prev = 0;
      if (t > 0) prev = reinterpret_cast<uint64_t>(planes[(t - 1) * A + a]);
      else if (s->frame > 0) prev = reinterpret_cast<uint64_t>(s->d_state[s->cur] + s->plane_off[a]);
      hp[(size_t)T * A + t * A + a] = prev;
    }
  }
  for (uint32_t a = 0; a < A; a++)
    hp[2ull * T * A + a] = reinterpret_cast<uint64_t>(s->d_state[1 - s->cur] + s->plane_off[a]);

  cudaError_t ce = cudaMemcpyAsync(d + o_cur, hp, 8ull * T * A, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(d + o_prev, hp + (size_t)T * A, 8ull * T * A, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(d + o_next, hp + 2ull * T * A, 8ull * A, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(d + o_zero, 0, zero_bytes, st);
  if (ce != cudaSuccess) return JIFFY_ERR_CUDA;

  jiffy::EncParams p{};
  p.H = H; p.W = W; p.A = A; p.T = T;
  p.nw = (W + 31) / 32;
  p.ncls = (p.nw + 15) / 16;
  p.frame0 = s->frame;
  p.shdr = s->frame == 0 ? stream_header_bytes(A) : 0u;
  p.fhdr = frame_header_bytes(A);
  p.test_lines = s->opt.test_lines;
  p.force_mode = s->opt.force_mode;
  p.n_items = (uint32_t)items;
  p.attrs = s->d_attrs;
  p.cur = reinterpret_cast<const uint8_t* const*>(d + o_cur);
  p.prev = reinterpret_cast<const uint8_t* const*>(d + o_prev);
  p.state_next = reinterpret_cast<uint8_t* const*>(d + o_next);
  p.out = static_cast<uint8_t*>(out);
  p.cap = out_capacity;
  p.modes = reinterpret_cast<uint32_t*>(d + o_modes);
  p.row_bytes = reinterpret_cast<uint32_t*>(d + o_rb);
  p.row_nnz = reinterpret_cast<uint32_t*>(d + o_rn);
  p.row_carry = reinterpret_cast<uint32_t*>(d + o_rc);
  p.st_carry = reinterpret_cast<unsigned long long*>(d + o_stc);
  p.slots = d + o_slots;
  p.slot_bytes = slot_bytes;
  p.sec_bytes = reinterpret_cast<unsigned long long*>(d + o_secb);
  p.sec_nnz = reinterpret_cast<uint32_t*>(d + o_secn);
  p.ticket = reinterpret_cast<uint32_t*>(d + o_tick);
  p.err = reinterpret_cast<uint32_t*>(d + o_tick + 4);
  p.frame_off = reinterpret_cast<unsigned long long*>(d + o_foff);
  void* evs[4] = {s->ev[0], s->ev[1], s->ev[2], s->ev[3]};
  if (jiffy::launch_encode(p, cuda_stream, s->profile ? evs : nullptr) != 0) return JIFFY_ERR_CUDA;

  uint8_t* hr = s->h_pinned + h_res;
  ce = cudaMemcpyAsync(hr, d + o_tick, 8, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(hr + 16, d + o_foff, 8ull * (T + 1), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return JIFFY_ERR_CUDA;
  uint32_t err = 0;
  std::memcpy(&err, hr + 4, 4);
  const uint64_t* foff = reinterpret_cast<const uint64_t*>(hr + 16);
  jiffy_status res = map_device_error(err);
  *out_len = foff[T];
  if (res != JIFFY_OK) return res;
  read_kernel_times(s, 3);
  if (frame_offsets) std::memcpy(frame_offsets, foff, 8ull * (T + 1));
  s->cur = 1 - s->cur;
  s->frame += T;
  return JIFFY_OK;
}

jiffy_status jiffy_encode(jiffy_stream* s, const void* const* planes, void* out, size_t out_capacity,
                          size_t* out_len, void* cuda_stream) {
  return jiffy_encode_seq(s, 1, planes, out, out_capacity, nullptr, out_len, cuda_stream);
}

jiffy_status jiffy_decode_seq(jiffy_stream* s, uint32_t n_scans, const void* in, size_t in_len,
                              const uint64_t* frame_offsets, void* const* planes_out, void* cuda_stream) {
  if (!s || !in || !frame_offsets || !planes_out || n_scans == 0) return JIFFY_ERR_INVALID_ARG;
  if (s->role != JIFFY_DECODER) return JIFFY_ERR_STATE;
  if (reinterpret_cast<uintptr_t>(in) & 3u) return JIFFY_ERR_INVALID_ARG;
  const uint32_t T = n_scans, A = s->A, H = s->H, W = s->W;
  for (size_t i = 0; i < (size_t)T * A; i++)
    if (!planes_out[i]) return JIFFY_ERR_INVALID_ARG;
  const unsigned long long items = (unsigned long long)T * A * H;
  if (items > 0x7fffffffull) return JIFFY_ERR_INVALID_ARG;
  // frame offsets: aligned, increasing by at least a frame header, inside `in`
  const uint32_t fh = frame_header_bytes(A);
  const uint64_t first = s->frame == 0 ? stream_header_bytes(A) : 0u;
  if (frame_offsets[0] < first) return JIFFY_ERR_CORRUPT;
  for (uint32_t t = 0; t < T; t++) {
    if ((frame_offsets[t] & 3u) || frame_offsets[t + 1] < frame_offsets[t] + fh) return JIFFY_ERR_CORRUPT;
    if (frame_offsets[t + 1] - frame_offsets[t] > 0xffffffffull) return JIFFY_ERR_CORRUPT;
  }
  if (frame_offsets[T] > in_len || (frame_offsets[T] & 3u)) return JIFFY_ERR_CORRUPT;
  DeviceGuard g(s->device);
  if (!g.ok) return JIFFY_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);

  Carver c;
  const size_t o_out = c.take(8ull * T * A), o_state = c.take(8ull * A), o_next = c.take(8ull * A);
  const size_t o_off = c.take(8ull * (T + 1));
  const size_t o_zero = c.take(0);
  const size_t o_done = c.take(4ull * items), o_tick = c.take(8);
  const size_t zero_bytes = c.off - o_zero;
  const size_t dev_bytes = c.off;
  const size_t n_up = (size_t)T * A + 2ull * A + (T + 1);
  const size_t h_res = align_up(8ull * n_up, 64);
  jiffy_status rs = ensure_scratch(s, dev_bytes, h_res + 16);
  if (rs != JIFFY_OK) return rs;
  uint8_t* d = s->d_scratch;
  uint64_t* hp = reinterpret_cast<uint64_t*>(s->h_pinned);
  for (size_t i = 0; i < (size_t)T * A; i++) hp[i] = reinterpret_cast<uint64_t>(planes_out[i]);
  for (uint32_t a = 0; a < A; a++) {
    hp[(size_t)T * A + a] = reinterpret_cast<uint64_t>(s->d_state[s->cur] + s->plane_off[a]);
    hp[(size_t)T * A + A + a] = reinterpret_cast<uint64_t>(s->d_state[1 - s->cur] + s->plane_off[a]);
  }
  std::memcpy(hp + (size_t)T * A + 2ull * A, frame_offsets, 8ull * (T + 1));
  cudaError_t ce = cudaMemcpyAsync(d + o_out, hp, 8ull * T * A, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(d + o_state, hp + (size_t)T * A, 8ull * A, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(d + o_next, hp + (size_t)T * A + A, 8ull * A, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(d + o_off, hp + (size_t)T * A + 2ull * A, 8ull * (T + 1), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(d + o_zero, 0, zero_bytes, st);
  if (ce != cudaSuccess) return JIFFY_ERR_CUDA;

  jiffy::DecParams p{};
  p.H = H; p.W = W; p.A = A; p.T = T;
  p.nw = (W + 31) / 32;
  p.ncls = (p.nw + 15) / 16;
  p.frame0 = s->frame;
  p.fhdr = fh;
  p.check_shdr = s->frame == 0;
  p.n_items = (uint32_t)items;
  p.attrs = s->d_attrs;
  p.in = static_cast<const uint8_t*>(in);
  p.in_len = in_len;
  p.off = reinterpret_cast<const unsigned long long*>(d + o_off);
  p.outp = reinterpret_cast<uint8_t* const*>(d + o_out);
  p.state = reinterpret_cast<const uint8_t* const*>(d + o_state);
  p.state_next = reinterpret_cast<uint8_t* const*>(d + o_next);
  p.done = reinterpret_cast<uint32_t*>(d + o_done);
  p.ticket = reinterpret_cast<uint32_t*>(d + o_tick);
  p.err = reinterpret_cast<uint32_t*>(d + o_tick + 4);
  void* evs[2] = {s->ev[0], s->ev[1]};
  if (jiffy::launch_decode(p, cuda_stream, s->profile ? evs : nullptr) != 0) return JIFFY_ERR_CUDA;
  uint8_t* hr = s->h_pinned + h_res;
  ce = cudaMemcpyAsync(hr, d + o_tick, 8, cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return JIFFY_ERR_CUDA;
  uint32_t err = 0;
  std::memcpy(&err, hr + 4, 4);
  jiffy_status res = map_device_error(err);
  if (res != JIFFY_OK) return res;
  read_kernel_times(s, 1);
  s->cur = 1 - s->cur;
  s->frame += T;
  return JIFFY_OK;
}

jiffy_status jiffy_decode(jiffy_stream* s, const void* in, size_t in_len, void* const* planes_out,
                          void* cuda_stream) {
  if (!s) return JIFFY_ERR_INVALID_ARG;
  const uint64_t off[2] = {s->frame == 0 ? stream_header_bytes(s->A) : 0u, in_len};
  return jiffy_decode_seq(s, 1, in, in_len, off, planes_out, cuda_stream);
}

}  // extern "C"
