// Allocation-free decode of one frame: jiffy_decode_frame_noalloc.
//
// Some callers cannot allocate device memory while they run: hard real-time
// perception stacks fix their device memory footprint at start-up and forbid
// allocation afterwards (an allocation can block, fail or fragment memory in
// the middle of a drive), and hosts whose own allocator has already reserved
// the whole HBM pool have nothing left for a library to take. Such callers
// cannot create a jiffy_stream (it allocates its state and scratch). This
// entry point decodes a frame with nothing but the caller's buffers plus a
// fixed scratch array that lives in this file: it calls no cudaMalloc,
// cudaFree, pinned-host allocation or allocating library routine.
//
// The scratch is a file-scope __device__ array (kNoAllocScratchBytes). Every
// GPU that loads the library holds it until the process exits. Every call
// shares it and it keeps the previous call's contents, so the parts that must
// start at zero are cleared on each call; calls that overlap on the GPU (on
// different streams, or from several host threads) race on it.
//
// In-place decode (prev_planes[a] == planes_out[a]) is allowed: a row's
// previous-scan pixels are read by the warp that writes the same pixels of
// that row, each before it is overwritten (the mask pass reads the whole
// previous row first, then every 256-pixel step loads before it stores).
//
// Set-up: the first call on a device looks up the array's device address with
// cudaGetSymbolAddress while that device is current (in host code the array's
// name is only a host-side stand-in, not a device address) and caches it.
// Make that first call before any stream capture begins.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "jiffy.h"
#include "jiffy_kernels.h"

namespace jiffy {
namespace {

// Limits of the allocation-free entry point.
constexpr uint32_t kNoAllocMaxAttr = 16;
constexpr uint32_t kNoAllocMaxRows = 16384;  // n_attr * H
constexpr uint32_t kMaxDevices = 64;

// Layout of the scratch array (byte offsets, 256-byte aligned regions).
constexpr size_t kOffAttrs = 0;                                          // AttrDev[kNoAllocMaxAttr]
constexpr size_t kOffPtrs = 1024;                                        // 3 x kNoAllocMaxAttr pointers
constexpr size_t kOffFrameOff = kOffPtrs + 3 * kNoAllocMaxAttr * 8;      // 2 x u64 frame offsets
constexpr size_t kOffSeg = kOffFrameOff + 256;                           // the call's one DecSeg
constexpr size_t kOffSegKey = kOffSeg + 256;                             // its first item (0)
constexpr size_t kOffZero = kOffSegKey + 256;                            // cleared every call:
constexpr size_t kOffTicket = kOffZero;                                  //   ticket, error word
constexpr size_t kOffDone = kOffZero + 256;                              //   row-done flags
constexpr size_t kNoAllocScratchBytes = kOffDone + 4ull * kNoAllocMaxRows;

static_assert(sizeof(AttrDev) * kNoAllocMaxAttr <= kOffPtrs, "attribute table overlaps");
static_assert(sizeof(DecSeg) <= 256, "segment record overlaps");

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `device` (current), looked up once.
cudaError_t scratch_address(int device, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

}  // namespace
}  // namespace jiffy

extern "C" jiffy_status jiffy_decode_frame_noalloc(const void* in, size_t in_len, uint32_t H, uint32_t W,
                                                   uint32_t n_attr, const jiffy_attr_desc* attrs,
                                                   uint32_t scan_index, uint32_t stages,
                                                   const void* const* prev_planes, void* const* planes_out,
                                                   void* cuda_stream) {
  using namespace jiffy;
  if (!in || !attrs || !planes_out || H == 0 || W == 0 || n_attr == 0) return JIFFY_ERR_INVALID_ARG;
  if ((stages & ~kStageAll) || (stages & kStageZstdMask)) return JIFFY_ERR_INVALID_ARG;  // no scratch for the frames
  if (H > kMaxH || W > kMaxW || n_attr > kNoAllocMaxAttr || (uint64_t)n_attr * H > kNoAllocMaxRows)
    return JIFFY_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(in) & 3u) return JIFFY_ERR_INVALID_ARG;
  AttrDev ad[kNoAllocMaxAttr] = {};
  for (uint32_t a = 0; a < n_attr; a++) {
    const uint32_t s = attrs[a].dtype_bytes, P = attrs[a].precision;
    if (!(s == 1 || s == 2 || s == 4) || P == 0 || !planes_out[a]) return JIFFY_ERR_INVALID_ARG;
    if (prev_planes && !prev_planes[a]) return JIFFY_ERR_INVALID_ARG;
    ad[a] = make_attr(s, P);
  }
  const uint32_t shdr = scan_index == 0 ? 16u + 8u * n_attr : 0u;
  const uint32_t fhdr = 8u + 12u * n_attr;
  if (in_len < (uint64_t)shdr + fhdr || (in_len & 3u) || in_len - shdr > 0xffffffffull) return JIFFY_ERR_CORRUPT;

  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= (int)kMaxDevices) return JIFFY_ERR_CUDA;
  unsigned char* scratch = nullptr;
  if (scratch_address(device, &scratch) != cudaSuccess) return JIFFY_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);

  // A P frame needs the previous frame's planes: read the modes first.
  uint32_t hdr[8 + 3 * kNoAllocMaxAttr];
  if (cudaMemcpyAsync(hdr, static_cast<const uint8_t*>(in) + shdr, fhdr, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return JIFFY_ERR_CUDA;
  for (uint32_t a = 0; a < n_attr; a++) {
    const uint32_t mode = hdr[2 + 3 * a] & 0xffu;
    if (mode == 1u && !prev_planes) return JIFFY_ERR_STATE;
  }

  // Small tables into the scratch array (host stack -> device, no allocation).
  uint64_t ptrs[3 * kNoAllocMaxAttr];
  for (uint32_t a = 0; a < n_attr; a++) {
    ptrs[a] = reinterpret_cast<uint64_t>(planes_out[a]);
    // without a previous frame (all attributes I) nothing reads the state
    ptrs[kNoAllocMaxAttr + a] = reinterpret_cast<uint64_t>(prev_planes ? prev_planes[a] : planes_out[a]);
    // the kernel copies the last frame to its "next state": point it at the
    // output itself, which receives the same values
    ptrs[2 * kNoAllocMaxAttr + a] = reinterpret_cast<uint64_t>(planes_out[a]);
  }
  const uint64_t offs[2] = {shdr, in_len};
  cudaError_t ce = cudaMemcpyAsync(scratch + kOffAttrs, ad, sizeof(AttrDev) * n_attr, cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(scratch + kOffPtrs, ptrs, sizeof(ptrs), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(scratch + kOffFrameOff, offs, sizeof(offs), cudaMemcpyHostToDevice, st);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(scratch + kOffZero, 0, kOffDone - kOffZero + 4ull * n_attr * H, st);
  if (ce != cudaSuccess) return JIFFY_ERR_CUDA;

  DecSeg g{};
  g.H = H; g.W = W; g.A = n_attr; g.T = 1;
  g.nw = (W + 31) / 32;
  g.ncls = (stages & kStageNoMask) ? 0u : (g.nw + 15) / 16;
  g.stages = stages;
  g.frame0 = scan_index;
  g.fhdr = fhdr;
  g.check_shdr = scan_index == 0;
  g.item_base = 0;
  g.attrs = reinterpret_cast<const AttrDev*>(scratch + kOffAttrs);
  g.in = static_cast<const uint8_t*>(in);
  g.in_len = in_len;
  g.off = reinterpret_cast<const unsigned long long*>(scratch + kOffFrameOff);
  g.outp = reinterpret_cast<uint8_t* const*>(scratch + kOffPtrs);
  g.state = reinterpret_cast<const uint8_t* const*>(scratch + kOffPtrs + 8 * kNoAllocMaxAttr);
  g.state_next = reinterpret_cast<uint8_t* const*>(scratch + kOffPtrs + 16 * kNoAllocMaxAttr);
  g.err = reinterpret_cast<uint32_t*>(scratch + kOffTicket + 4);
  const uint32_t key = 0;
  cudaError_t ce2 = cudaMemcpyAsync(scratch + kOffSeg, &g, sizeof(g), cudaMemcpyHostToDevice, st);
  if (ce2 == cudaSuccess) ce2 = cudaMemcpyAsync(scratch + kOffSegKey, &key, 4, cudaMemcpyHostToDevice, st);
  if (ce2 != cudaSuccess) return JIFFY_ERR_CUDA;

  DecParams p{};
  p.n_seg = 1;
  p.n_items = n_attr * H;
  p.max_W = W;
  p.seg = reinterpret_cast<const DecSeg*>(scratch + kOffSeg);
  p.seg_item_base = reinterpret_cast<const uint32_t*>(scratch + kOffSegKey);
  p.done = reinterpret_cast<uint32_t*>(scratch + kOffDone);
  p.ticket = reinterpret_cast<uint32_t*>(scratch + kOffTicket);
  p.staged = stages ? 1u : 0u;  // the decoder instance that reads the stage switches
  if (launch_decode(p, cuda_stream, nullptr) != 0) return JIFFY_ERR_CUDA;

  uint32_t res[2] = {0, 0};
  if (cudaMemcpyAsync(res, scratch + kOffTicket, sizeof(res), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return JIFFY_ERR_CUDA;
  if (res[1] & kErrTimeout) return JIFFY_ERR_TIMEOUT;
  if (res[1] & kErrCorrupt) return JIFFY_ERR_CORRUPT;
  return JIFFY_OK;
}
