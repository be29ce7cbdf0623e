// Host side of the Jiffy C ABI (include/jiffy.h): stream and batch handles,
// device state and scratch, argument checks, kernel launches and status
// mapping. Every step of the codec itself runs in the kernels of
// jiffy_encode.cu and jiffy_decode.cu; this file only marshals pointers and
// sizes, and schedules the launches.
//
// A call codes one segment per stream: jiffy_encode(_seq) and
// jiffy_decode(_seq) are one-segment calls, the batch calls code many. A call
// is enqueued (upload of the segment table, clearing of the counters, the
// kernels, download of the per-segment results) and then finished (wait,
// statuses, state roll-back of failed streams). Batch contexts can replay the
// enqueued sequence from a captured CUDA graph and pick the rows kernels'
// launch configuration by timing the candidates on the first call of a shape.
#include "jiffy.h"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <new>
#include <vector>

#include "jiffy_kernels.h"

using jiffy::AttrDev;
using jiffy::RowsLaunch;

namespace {

struct EncJob {
  jiffy_stream* s;
  uint32_t T;
  const void* const* planes;  // T*A device pointers
  void* out;
  size_t cap;
  uint64_t* frame_offsets;    // host, T+1, nullable
  size_t* out_len;            // host
  jiffy_status* status;       // host
  bool async = false;         // enqueue only: errors to the stream's device word
  uint64_t* dev_offsets = nullptr;  // device, T+1, nullable (async)
};

struct DecJob {
  jiffy_stream* s;
  uint32_t T;
  const void* in;
  size_t in_len;
  const uint64_t* frame_offsets;  // host, T+1 (device with async)
  void* const* planes_out;        // T*A device pointers
  jiffy_status* status;           // host
  bool async = false;             // enqueue only: offsets on the device, checked by the kernel
};

// A call enqueued on the device whose results are not read yet.
struct Pending {
  int kind = 0;  // 0 none, 1 encode, 2 decode
  std::vector<EncJob> enc;
  std::vector<DecJob> dec;
  std::vector<size_t> r_err, r_off;  // offsets in the results image
  uint8_t* hres = nullptr;           // results image (pinned)
  uint32_t n_kernels = 0;            // timed kernels (0: none)
};

struct GraphCache {
  std::vector<uint64_t> key;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;            // kept while exec lives: its nodes address the exec's
  std::vector<cudaGraphNode_t> ev_nodes;  // the event record nodes of the kernel timing events
  std::vector<cudaEvent_t> ev_now;        // the events they record in the exec
};

// Device scratch, pinned host staging, timing events, graph cache and tuned
// launch configurations of a handle.
struct Workspace {
  int device = 0;
  uint8_t* d_scratch = nullptr;
  size_t scratch_cap = 0;
  uint8_t* h_pinned = nullptr;
  size_t pinned_cap = 0;
  bool profile = false;
  bool graphs = false;
  bool autotune = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t done = nullptr;
  cudaStream_t capture = nullptr;
  float kernel_ms[3] = {0, 0, 0};
  uint32_t n_kernel_ms = 0;
  GraphCache g_enc[2], g_dec[2];  // one captured sequence per segment-table slot
  std::map<std::vector<uint32_t>, RowsLaunch> tuned;
  RowsLaunch last{};
  RowsLaunch fixed[2] = {};  // launch requests set by the caller (encode, decode); 0 = automatic
  uint64_t calls = 0, captures = 0, replays = 0, tunings = 0;
  Pending pend;
  cudaEvent_t uploaded = nullptr;  // the last call's segment table has reached the device
  bool upload_pending = false;     // an enqueue-only call may still read the pinned table
  // Segment tables go to two device slots in turn (a table points into its
  // own slot). Per slot, the table last copied there and where it went: a
  // call whose table is the same bytes for the same place skips the copy
  // (the host waits for the previous copy before it writes a new table, so
  // every earlier copy is complete on the device). Calls that repeat, whose
  // tables alternate with the stream's ping-pong state planes, find theirs in
  // place.
  std::vector<uint8_t> up_last[2];
  const uint8_t* up_dev[2] = {nullptr, nullptr};
  uint32_t up_slot = 1;  // slot of the last call
  int slots = 0;         // 1 or 2 table slots, decided at the first call (0: not yet)
  // kernel timing of enqueue-only calls: a ring of event sets, harvested as
  // they complete and averaged at jiffy_stream_wait
  struct EvSet {
    cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
    uint32_t nk = 0;
  };
  std::vector<EvSet> ring;
  size_t ring_tail = 0, ring_count = 0;
  double acc_ms[3] = {0, 0, 0};
  uint32_t acc_calls = 0, acc_nk = 0;
};

}  // namespace

struct jiffy_stream {
  Workspace ws;
  jiffy_role role = JIFFY_ENCODER;
  uint32_t H = 0, W = 0, A = 0;
  jiffy_options opt{4, -1, 0};
  std::vector<AttrDev> attrs;
  AttrDev* d_attrs = nullptr;
  uint8_t* d_state[2] = {nullptr, nullptr};  // previous scan (as decoded, q * P), ping-pong
  std::vector<size_t> plane_off;              // byte offset of attribute a in a state buffer
  size_t state_bytes = 0;
  int cur = 0;                                // state buffer holding the previous scan
  uint32_t frame = 0;                         // frames since create/reset
  bool in_flight = false;                     // part of an enqueued, unfinished call
  uint32_t withhold = UINT32_MAX;             // test hook: row item of the next decode call left unpublished
  uint32_t* d_err = nullptr;                  // error bits of enqueue-only calls (device)
  cudaEvent_t async_done = nullptr;           // recorded after the last enqueue-only call
  bool async_out = false;                     // enqueue-only calls not yet waited for
};

struct jiffy_batch {
  Workspace ws;
};

namespace {

// A named range around a public call, for timeline tools (NVTX: no cost
// unless a tool is attached).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

// Rows of at most this many columns fit 6 encoder CTAs of 4 warps per SM;
// a call that also codes wider rows runs them in a rows launch of their own.
constexpr uint32_t kNarrowW = 2048;

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

void drop_graph(GraphCache& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
  g.exec = nullptr;
  g.graph = nullptr;
  g.ev_nodes.clear();
  g.ev_now.clear();
  g.key.clear();
}

// Workspaces of a process that use two segment-table slots. Alternating
// launch sequences cost device-side graph state: with a few hundred streams
// in one process (256 streams, one call each per step: 11.2 -> 8.0 Gpoints/s)
// that outweighed the copies saved, while up to 64 streams gained (+8 %).
// Workspaces beyond the first 64 keep one slot.
constexpr int kTwoSlotWorkspaces = 64;
std::atomic<int> g_two_slot_ws{0};

// The table slot of a workspace's next call.
uint32_t next_slot(Workspace& w) {
  if (!w.slots) {
    w.slots = g_two_slot_ws.fetch_add(1) < kTwoSlotWorkspaces ? 2 : 1;
    if (w.slots == 1) g_two_slot_ws.fetch_sub(1);
  }
  return w.slots == 2 ? 1u - w.up_slot : 0u;
}

void drop_graphs(Workspace& w) {
  for (int k = 0; k < 2; k++) {
    drop_graph(w.g_enc[k]);
    drop_graph(w.g_dec[k]);
  }
}

jiffy_status ensure_scratch(Workspace& w, size_t dev_bytes, size_t host_bytes) {
  // enqueue-only calls may still use the buffers about to be replaced
  if ((dev_bytes > w.scratch_cap || host_bytes > w.pinned_cap) && w.upload_pending) cudaDeviceSynchronize();
  if (dev_bytes > w.scratch_cap) {
    drop_graphs(w);  // the captured sequences point into the old buffers
    if (w.d_scratch) cudaFree(w.d_scratch);
    w.d_scratch = nullptr;
    w.scratch_cap = 0;
    for (int k = 0; k < 2; k++) {  // the tables on the device go with the buffer
      w.up_last[k].clear();
      w.up_dev[k] = nullptr;
    }
    size_t cap = align_up(dev_bytes + dev_bytes / 4, 1 << 20);
    if (cudaMalloc(&w.d_scratch, cap) != cudaSuccess) return JIFFY_ERR_NOMEM;
    w.scratch_cap = cap;
  }
  if (host_bytes > w.pinned_cap) {
    drop_graphs(w);
    if (w.h_pinned) cudaFreeHost(w.h_pinned);
    w.h_pinned = nullptr;
    w.pinned_cap = 0;
    size_t cap = align_up(host_bytes + host_bytes / 4, 1 << 16);
    if (cudaMallocHost(&w.h_pinned, cap) != cudaSuccess) return JIFFY_ERR_NOMEM;
    w.pinned_cap = cap;
  }
  if (!w.done && cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming) != cudaSuccess) return JIFFY_ERR_CUDA;
  if (!w.uploaded && cudaEventCreateWithFlags(&w.uploaded, cudaEventDisableTiming) != cudaSuccess)
    return JIFFY_ERR_CUDA;
  return JIFFY_OK;
}

// Moves the kernel times of completed enqueue-only calls into the running
// sums (block: wait for all of them).
void harvest(Workspace& w, bool block) {
  while (w.ring_count) {
    Workspace::EvSet& es = w.ring[w.ring_tail];
    const cudaError_t q = block ? cudaEventSynchronize(es.e[es.nk]) : cudaEventQuery(es.e[es.nk]);
    if (q != cudaSuccess) break;
    for (uint32_t k = 0; k < es.nk; k++) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, es.e[k], es.e[k + 1]) == cudaSuccess) w.acc_ms[k] += ms;
    }
    w.acc_nk = es.nk;
    w.acc_calls++;
    w.ring_tail = (w.ring_tail + 1) % w.ring.size();
    w.ring_count--;
  }
}

// An event set for the next timed enqueue-only call of nk kernels.
void* const* next_evset(Workspace& w, uint32_t nk) {
  if (w.ring.empty()) {
    w.ring.resize(16);
    for (Workspace::EvSet& es : w.ring)
      for (cudaEvent_t& e : es.e)
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  }
  harvest(w, false);
  if (w.ring_count == w.ring.size()) {  // the device is 16 calls behind: wait for the oldest
    Workspace::EvSet& old = w.ring[w.ring_tail];
    cudaEventSynchronize(old.e[old.nk]);
    harvest(w, false);
  }
  Workspace::EvSet& es = w.ring[(w.ring_tail + w.ring_count) % w.ring.size()];
  es.nk = nk;
  w.ring_count++;
  return reinterpret_cast<void* const*>(es.e);
}

// Records ev on st; inside a stream capture it becomes an event-record node
// of the graph, so a replay records it too.
cudaError_t record_ev(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    return cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
  return cudaEventRecord(ev, st);
}

// Before the host rewrites the pinned segment table: an enqueue-only call
// may not have copied it to the device yet.
jiffy_status wait_upload(Workspace& w) {
  if (!w.upload_pending) return JIFFY_OK;
  if (cudaEventSynchronize(w.uploaded) != cudaSuccess) return JIFFY_ERR_CUDA;
  w.upload_pending = false;
  return JIFFY_OK;
}

// Is the call's segment table (h, bytes) already on the device at dev? (the
// previous table went there, with the same bytes; wait_upload has made sure
// its copy is complete)
bool table_resident(const Workspace& w, uint32_t slot, const uint8_t* dev, const uint8_t* h, size_t bytes) {
  return w.up_dev[slot] == dev && w.up_last[slot].size() == bytes &&
         std::memcmp(w.up_last[slot].data(), h, bytes) == 0;
}

// Records the table a call put on the device (ok), or forgets it (a failed
// call may not have copied it).
void table_uploaded(Workspace& w, uint32_t slot, bool ok, bool skipped, const uint8_t* dev, const uint8_t* h,
                    size_t bytes) {
  w.up_slot = slot;
  if (!ok) {
    w.up_last[slot].clear();
    w.up_dev[slot] = nullptr;
  } else if (!skipped) {
    w.up_last[slot].assign(h, h + bytes);
    w.up_dev[slot] = dev;
  }
}

void release(Workspace& w) {
  drop_graphs(w);
  if (w.slots == 2) g_two_slot_ws.fetch_sub(1);
  w.slots = 0;
  if (w.d_scratch) cudaFree(w.d_scratch);
  if (w.h_pinned) cudaFreeHost(w.h_pinned);
  for (cudaEvent_t e : w.ev)
    if (e) cudaEventDestroy(e);
  if (w.done) cudaEventDestroy(w.done);
  if (w.capture) cudaStreamDestroy(w.capture);
  if (w.uploaded) cudaEventDestroy(w.uploaded);
  for (Workspace::EvSet& es : w.ring)
    for (cudaEvent_t e : es.e)
      if (e) cudaEventDestroy(e);
  w = Workspace{};
}

jiffy_status ensure_events(Workspace& w) {
  if (w.ev[0]) return JIFFY_OK;
  for (cudaEvent_t& e : w.ev)
    if (cudaEventCreate(&e) != cudaSuccess) return JIFFY_ERR_CUDA;
  return JIFFY_OK;
}

jiffy_status set_profiling(Workspace& w, int enable) {
  if (enable) {
    DeviceGuard g(w.device);
    if (!g.ok || ensure_events(w) != JIFFY_OK) return JIFFY_ERR_CUDA;
  }
  w.profile = enable != 0;
  w.n_kernel_ms = 0;
  return JIFFY_OK;
}

jiffy_status map_device_error(uint32_t err) {
  if (err & jiffy::kErrTimeout) return JIFFY_ERR_TIMEOUT;
  if (err & jiffy::kErrCorrupt) return JIFFY_ERR_CORRUPT;
  if (err & jiffy::kErrCapacity) return JIFFY_ERR_CAPACITY;
  return JIFFY_OK;
}

uint32_t stream_header_bytes(uint32_t A) { return 16u + 8u * A; }
uint32_t frame_header_bytes(uint32_t A) { return 8u + 12u * A; }
uint32_t slot_bytes_for(uint32_t W) { return (jiffy::row_bound_bytes(W) + 15u) & ~15u; }

// Number of distinct test rows floor((2k+1)H/(2L)), k < L (Sec. III-E): the
// rows are distinct while L <= H, and cover every row once L >= H.
uint32_t distinct_test_rows(uint32_t H, uint32_t L) { return L < H ? L : H; }

jiffy_status check_distinct(const std::vector<jiffy_stream*>& ss) {
  for (size_t i = 0; i < ss.size(); i++)
    for (size_t k = i + 1; k < ss.size(); k++)
      if (ss[i] == ss[k]) return JIFFY_ERR_INVALID_ARG;  // a stream at most once per call
  return JIFFY_OK;
}

// Tuned launch configurations kept across processes in the file named by
// JIFFY_TUNE_CACHE: one line per shape class, "jiffy-tune 1 <device> <n>
// <n key words> <warps per CTA> <CTAs per SM> <items per ticket>", device =
// SM count * 1000 + compute capability (lines of another device are ignored;
// a configuration that does not fit falls back to the automatic one).
using TuneKey = std::pair<uint32_t, std::vector<uint32_t>>;

const char* tune_cache_path() {
  const char* p = std::getenv("JIFFY_TUNE_CACHE");
  return (p && *p) ? p : nullptr;
}

uint32_t device_tag(int dev) {
  int sms = 0, maj = 0, mnr = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&mnr, cudaDevAttrComputeCapabilityMinor, dev);
  return (uint32_t)sms * 1000u + (uint32_t)(maj * 10 + mnr);
}

std::map<TuneKey, RowsLaunch> tune_cache_read(const char* path) {
  std::map<TuneKey, RowsLaunch> out;
  FILE* f = std::fopen(path, "r");
  if (!f) return out;
  char tag[16];
  unsigned ver, dev, n;
  while (std::fscanf(f, "%15s %u %u %u", tag, &ver, &dev, &n) == 4) {
    if (std::strcmp(tag, "jiffy-tune") != 0 || ver != 1u || n > 16u) break;
    std::vector<uint32_t> key(n);
    bool ok = true;
    for (uint32_t& x : key) ok = ok && std::fscanf(f, "%u", &x) == 1;
    unsigned w = 0, c = 0, ipt = 0;
    ok = ok && std::fscanf(f, "%u %u %u", &w, &c, &ipt) == 3;
    if (!ok) break;
    out[TuneKey(dev, key)] = RowsLaunch{w, c, ipt, 0};
  }
  std::fclose(f);
  return out;
}

void tune_cache_load(Workspace& ws) {
  const char* path = tune_cache_path();
  if (!path) return;
  const uint32_t tag = device_tag(ws.device);
  for (const auto& kv : tune_cache_read(path))
    if (kv.first.first == tag) ws.tuned.emplace(kv.first.second, kv.second);
}

void tune_cache_store(const Workspace& ws) {
  const char* path = tune_cache_path();
  if (!path) return;
  std::map<TuneKey, RowsLaunch> all = tune_cache_read(path);
  const uint32_t tag = device_tag(ws.device);
  for (const auto& kv : ws.tuned) all[TuneKey(tag, kv.first)] = kv.second;
  const std::string tmp = std::string(path) + ".tmp." + std::to_string((long)getpid());
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  for (const auto& kv : all) {
    std::fprintf(f, "jiffy-tune 1 %u %u", kv.first.first, (unsigned)kv.first.second.size());
    for (uint32_t x : kv.first.second) std::fprintf(f, " %u", x);
    std::fprintf(f, " %u %u %u\n", kv.second.wpc, kv.second.ctas_per_sm, kv.second.items_per_ticket);
  }
  const bool ok = std::fclose(f) == 0;
  if (ok) std::rename(tmp.c_str(), path);
  else std::remove(tmp.c_str());
}

uint32_t log2_ceil(uint64_t x) {
  uint32_t l = 0;
  while ((1ull << l) < x) l++;
  return l;
}

// Candidate launch configurations of the rows kernels, tried by the tuner.
std::vector<RowsLaunch> candidates(bool encode) {
  std::vector<RowsLaunch> c;
  const uint32_t wpcs_e[] = {4, 2, 1}, wpcs_d[] = {8, 4, 2, 1};
  const uint32_t ctas[] = {0, 2, 1};
  const uint32_t ipts[] = {1, 4, 16};
  if (encode) {
    for (uint32_t w : wpcs_e)
      for (uint32_t k : ctas) c.push_back(RowsLaunch{w, k, 1, 0});
  } else {
    for (uint32_t w : wpcs_d)
      for (uint32_t k : ctas)
        for (uint32_t i : ipts) c.push_back(RowsLaunch{w, k, i, 0});
  }
  return c;
}

void apply_ticket(jiffy::EncParams&, uint32_t) {}
void apply_ticket(jiffy::DecParams& p, uint32_t ipt) { p.items_per_ticket = ipt; }

bool same_launch(const RowsLaunch& a, const RowsLaunch& b) {
  return a.wpc == b.wpc && a.ctas_per_sm == b.ctas_per_sm && a.items_per_ticket == b.items_per_ticket &&
         a.grid == b.grid;
}

// Runs `enqueue` (the whole call on stream st) for every distinct candidate
// configuration, timing the rows kernel with the workspace's events between
// ev[e0] and ev[e1]; returns the fastest candidate. The call's kernels are
// idempotent: repeating them with the same inputs writes the same outputs.
template <class Params, class Resolve, class Enqueue>
jiffy_status tune(Workspace& ws, bool encode, const Params& p0, cudaStream_t st, Resolve resolve, Enqueue enqueue,
                  RowsLaunch* best_cand) {
  if (ensure_events(ws) != JIFFY_OK) return JIFFY_ERR_CUDA;
  std::vector<RowsLaunch> seen;
  float best = 1e30f;
  *best_cand = RowsLaunch{0, 0, 0, 0};
  const int e0 = encode ? 1 : 0, e1 = encode ? 2 : 1;
  for (const RowsLaunch& c : candidates(encode)) {
    Params p = p0;
    p.wpc = c.wpc;
    p.ctas_per_sm = c.ctas_per_sm;
    apply_ticket(p, c.items_per_ticket);
    RowsLaunch r{};
    if (resolve(p, &r) != 0) continue;
    bool dup = false;
    for (const RowsLaunch& s : seen) dup |= same_launch(s, r);
    if (dup) continue;
    seen.push_back(r);
    float t_min = 1e30f;
    for (int rep = 0; rep < 2; rep++) {
      void* evs[4] = {ws.ev[0], ws.ev[1], ws.ev[2], ws.ev[3]};
      if (enqueue(st, p, evs) != 0) return JIFFY_ERR_CUDA;
      if (cudaStreamSynchronize(st) != cudaSuccess) return JIFFY_ERR_CUDA;
      float ms = 0;
      if (cudaEventElapsedTime(&ms, ws.ev[e0], ws.ev[e1]) != cudaSuccess) return JIFFY_ERR_CUDA;
      t_min = std::min(t_min, ms);
    }
    if (t_min < best) {
      best = t_min;
      *best_cand = c;
    }
  }
  ws.tunings++;
  return JIFFY_OK;
}

// Enqueues the call through the graph cache when graphs are on: replays the
// captured sequence if the call's shape and buffers match the last capture,
// else captures it anew on the workspace's capture stream. tev: the call's n_tev
// kernel timing events (or null); a replay points the graph's timing event
// nodes at them, so calls that time their kernels with different event sets
// (enqueue-only calls take the next set of a ring) share one graph.
template <class Enqueue>
jiffy_status run_sequence(Workspace& ws, GraphCache& gc, const std::vector<uint64_t>& key, cudaStream_t st,
                          bool use_graph, void* const* tev, uint32_t n_tev, Enqueue enqueue) {
  if (!use_graph) return enqueue(st) == 0 ? JIFFY_OK : JIFFY_ERR_CUDA;
  if (!(gc.exec && gc.key == key)) {
    drop_graph(gc);
    if (!ws.capture && cudaStreamCreateWithFlags(&ws.capture, cudaStreamNonBlocking) != cudaSuccess)
      return JIFFY_ERR_CUDA;
    if (cudaStreamBeginCapture(ws.capture, cudaStreamCaptureModeRelaxed) != cudaSuccess) return JIFFY_ERR_CUDA;
    const int rc = enqueue(ws.capture);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(ws.capture, &graph);
    if (rc != 0 || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return JIFFY_ERR_CUDA;
    }
    // the timing events' record nodes, in the order of tev
    gc.ev_nodes.assign(n_tev, nullptr);
    gc.ev_now.assign(n_tev, nullptr);
    if (n_tev) {
      size_t nn = 0;
      std::vector<cudaGraphNode_t> nodes;
      bool ok = cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess;
      if (ok) {
        nodes.resize(nn);
        ok = cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess;
      }
      for (size_t i = 0; ok && i < nn; i++) {
        cudaGraphNodeType ty;
        cudaEvent_t e = nullptr;
        if (cudaGraphNodeGetType(nodes[i], &ty) != cudaSuccess) ok = false;
        else if (ty == cudaGraphNodeTypeEventRecord && cudaGraphEventRecordNodeGetEvent(nodes[i], &e) == cudaSuccess)
          for (uint32_t k = 0; k < n_tev; k++)
            if (e == static_cast<cudaEvent_t>(tev[k])) {
              gc.ev_nodes[k] = nodes[i];
              gc.ev_now[k] = e;
            }
      }
      for (uint32_t k = 0; k < n_tev; k++) ok = ok && gc.ev_nodes[k] != nullptr;
      if (!ok) {
        cudaGraphDestroy(graph);
        gc.ev_nodes.clear();
        gc.ev_now.clear();
        return JIFFY_ERR_CUDA;
      }
    }
    const cudaError_t ie = cudaGraphInstantiate(&gc.exec, graph, 0);
    if (ie != cudaSuccess) {
      cudaGraphDestroy(graph);
      gc.exec = nullptr;
      return JIFFY_ERR_CUDA;
    }
    gc.graph = graph;
    gc.key = key;
    ws.captures++;
  } else {
    for (uint32_t k = 0; k < n_tev && k < gc.ev_nodes.size(); k++) {
      cudaEvent_t e = static_cast<cudaEvent_t>(tev[k]);
      if (gc.ev_now[k] != e) {
        if (cudaGraphExecEventRecordNodeSetEvent(gc.exec, gc.ev_nodes[k], e) != cudaSuccess) return JIFFY_ERR_CUDA;
        gc.ev_now[k] = e;
      }
    }
    ws.replays++;
  }
  return cudaGraphLaunch(gc.exec, st) == cudaSuccess ? JIFFY_OK : JIFFY_ERR_CUDA;
}

// ---------------------------------------------------------------- encode
jiffy_status enqueue_encode(Workspace& ws, std::vector<EncJob>& jobs, cudaStream_t st) {
  const uint32_t n = (uint32_t)jobs.size();
  if (ws.pend.kind) return JIFFY_ERR_STATE;  // the previous call is not finished
  // ---- argument checks and totals
  unsigned long long items = 0, secs = 0;
  uint32_t max_W = 1;
  std::vector<jiffy_stream*> ss(n);
  for (uint32_t i = 0; i < n; i++) {
    EncJob& j = jobs[i];
    *j.status = JIFFY_OK;
    jiffy_stream* s = j.s;
    ss[i] = s;
    if (!s || !j.planes || !j.out || (!j.out_len && !j.async) || j.T == 0) return JIFFY_ERR_INVALID_ARG;
    if (s->role != JIFFY_ENCODER || s->ws.device != ws.device || s->in_flight) return JIFFY_ERR_STATE;
    if (j.async && (reinterpret_cast<uintptr_t>(j.dev_offsets) & 7u)) return JIFFY_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(j.out) & 15u) return JIFFY_ERR_INVALID_ARG;
    for (size_t q = 0; q < (size_t)j.T * s->A; q++)
      if (!j.planes[q]) return JIFFY_ERR_INVALID_ARG;
    items += (unsigned long long)j.T * s->A * s->H;
    secs += (unsigned long long)j.T * s->A;
    if (s->W > max_W) max_W = s->W;
  }
  if (check_distinct(ss) != JIFFY_OK) return JIFFY_ERR_INVALID_ARG;
  if (items > 0x7fffffffull) return JIFFY_ERR_INVALID_ARG;
  // most distinct test rows of a stream that may run the trial (the kernel
  // skips first frames itself, so the launch shape does not depend on the
  // streams' frame counters and captured graphs stay valid)
  uint32_t trial_rows = 0;
  for (uint32_t i = 0; i < n; i++) {
    const jiffy_stream* s = jobs[i].s;
    if (s->opt.force_mode >= 0) continue;
    trial_rows = std::max(trial_rows, distinct_test_rows(s->H, s->opt.test_lines));
  }

  // ---- upload image: segments, search keys, per-segment pointer arrays
  Carver up;
  const size_t u_seg = up.take(sizeof(jiffy::EncSeg) * n);
  const size_t u_ib = up.take(4ull * n), u_sb = up.take(4ull * n);
  std::vector<size_t> u_ptrs(n);
  for (uint32_t i = 0; i < n; i++) u_ptrs[i] = up.take(8ull * (2ull * jobs[i].T + 1) * jobs[i].s->A);
  // ---- results image: per-segment error word and frame offsets
  Carver rs;
  std::vector<size_t> r_err(n), r_off(n);
  for (uint32_t i = 0; i < n; i++) {
    r_err[i] = rs.take(8);
    r_off[i] = rs.take(8ull * (jobs[i].T + 1));
  }
  // ---- device scratch: upload, zeroed region (look-back words, trial
  //      costs, ticket, results), work arrays, row slots
  Carver c;
  const uint32_t slot = next_slot(ws);  // segment-table slots alternate
  const size_t o_up_slot[2] = {c.take(up.off), c.take(up.off)};
  const size_t o_up = o_up_slot[slot];
  const size_t o_zero = c.take(0);
  const size_t o_stc = c.take(8ull * items);
  const size_t o_cost = c.take(8ull * secs), o_tick = c.take(8);
  const size_t o_res = c.take(rs.off);
  const size_t zero_bytes = c.off - o_zero;
  const size_t o_modes = c.take(4ull * secs);
  const size_t o_rb = c.take(4ull * items), o_rn = c.take(4ull * items), o_rc = c.take(4ull * items);
  const size_t o_secb = c.take(8ull * secs), o_secn = c.take(4ull * secs);
  std::vector<unsigned long long> slot_base(n);
  unsigned long long slots_total = 0;
  for (uint32_t i = 0; i < n; i++) {
    const jiffy_stream* s = jobs[i].s;
    slot_base[i] = slots_total;
    slots_total += (unsigned long long)slot_bytes_for(s->W) * jobs[i].T * s->A * s->H;
  }
  const size_t o_slots = c.take(slots_total);
  // Zstandard mask sections: coded mask bytes, block slots and sizes
  std::vector<unsigned long long> zm_base(n), zb_base(n);
  unsigned long long zm_total = 0, zb_total = 0;
  uint32_t zmax_blk = 0;
  for (uint32_t i = 0; i < n; i++) {
    const jiffy_stream* s = jobs[i].s;
    if (!(s->opt.stages & jiffy::kStageZstdMask)) continue;
    const uint32_t nblk = jiffy::zmask_blocks(s->H, s->W);
    zm_base[i] = zm_total;
    zb_base[i] = zb_total;
    zm_total += align_up((size_t)s->H * ((s->W + 7) / 8), 16) * jobs[i].T * s->A;
    zb_total += (unsigned long long)nblk * jobs[i].T * s->A;
    zmax_blk = std::max(zmax_blk, nblk);
  }
  const size_t o_zm = c.take(zm_total), o_zblk = c.take(zb_total * jiffy::kZSlot);
  const size_t o_zbb = c.take(4ull * zb_total), o_zfr = c.take(zmax_blk ? 4ull * secs : 0ull);
  const size_t h_res = align_up(up.off, 256);
  jiffy_status r = ensure_scratch(ws, c.off, h_res + rs.off);
  if (r == JIFFY_OK) r = wait_upload(ws);
  if (r != JIFFY_OK) return r;
  uint8_t* d = ws.d_scratch;
  uint8_t* h = ws.h_pinned;

  jiffy::EncSeg* segs = reinterpret_cast<jiffy::EncSeg*>(h + u_seg);
  uint32_t* ib = reinterpret_cast<uint32_t*>(h + u_ib);
  uint32_t* sb = reinterpret_cast<uint32_t*>(h + u_sb);
  std::vector<uint64_t> key{1, n, (uint64_t)(uintptr_t)d, (uint64_t)(uintptr_t)h};
  std::vector<uint32_t> sig{1, max_W, log2_ceil(items)};
  uint32_t staged = 0, withhold = 0;
  uint32_t item_base = 0, sec_base = 0;
  // segment order: streams of rows up to kNarrowW columns first, so that the
  // rows kernel can run them in a launch of its own with shared memory (and
  // so occupancy) sized for them (segments are independent; the search keys
  // stay ascending)
  std::vector<uint32_t> ord;
  uint32_t split = 0, split_W = 1;
  for (int pass = 0; pass < 2; pass++)
    for (uint32_t i = 0; i < n; i++)
      if ((jobs[i].s->W <= kNarrowW) == (pass == 0)) {
        ord.push_back(i);
        if (pass == 0) {
          split += jobs[i].T * jobs[i].s->A * jobs[i].s->H;
          split_W = std::max(split_W, jobs[i].s->W);
        }
      }
  if (split == items) split = 0;  // one width class: one launch
  for (uint32_t si = 0; si < n; si++) {
    const uint32_t i = ord[si];
    EncJob& j = jobs[i];
    jiffy_stream* s = j.s;
    const uint32_t T = j.T, A = s->A;
    uint64_t* hp = reinterpret_cast<uint64_t*>(h + u_ptrs[i]);
    for (uint32_t t = 0; t < T; t++) {
      for (uint32_t a = 0; a < A; a++) {
        hp[t * A + a] = reinterpret_cast<uint64_t>(j.planes[t * A + a]);
        uint64_t prev = 0;
        if (t > 0) prev = reinterpret_cast<uint64_t>(j.planes[(t - 1) * A + a]);
        else if (s->frame > 0) prev = reinterpret_cast<uint64_t>(s->d_state[s->cur] + s->plane_off[a]);
        hp[(size_t)T * A + t * A + a] = prev;
      }
    }
    for (uint32_t a = 0; a < A; a++)
      hp[2ull * T * A + a] = reinterpret_cast<uint64_t>(s->d_state[1 - s->cur] + s->plane_off[a]);
    const uint8_t* dp = d + o_up + u_ptrs[i];
    jiffy::EncSeg g{};
    g.H = s->H;
    g.W = s->W;
    g.A = A;
    g.T = T;
    g.nw = (s->W + 31) / 32;
    g.ncls = (s->opt.stages & (jiffy::kStageNoMask | jiffy::kStageZstdMask)) ? 0u : (g.nw + 15) / 16;
    g.stages = s->opt.stages;
    if (s->opt.stages & jiffy::kStageZstdMask) {
      g.zm_rb = (s->W + 7) / 8;
      g.zm_nblk = jiffy::zmask_blocks(s->H, s->W);
      g.zm_stride = align_up((size_t)s->H * g.zm_rb, 16);
      g.zm_base = zm_base[i];
      g.zb_base = zb_base[i];
    }
    g.frame0 = s->frame;
    g.shdr = s->frame == 0 ? stream_header_bytes(A) : 0u;
    g.fhdr = frame_header_bytes(A);
    g.test_lines = s->opt.test_lines;
    g.force_mode = s->opt.force_mode;
    g.item_base = item_base;
    g.sec_base = sec_base;
    g.slot_bytes = slot_bytes_for(s->W);
    g.slot_base = slot_base[i];
    g.attrs = s->d_attrs;
    g.cur = reinterpret_cast<const uint8_t* const*>(dp);
    g.prev = reinterpret_cast<const uint8_t* const*>(dp + 8ull * T * A);
    g.state_next = reinterpret_cast<uint8_t* const*>(dp + 16ull * T * A);
    g.out = static_cast<uint8_t*>(j.out);
    g.cap = j.cap;
    g.frame_off = (j.async && j.dev_offsets) ? reinterpret_cast<unsigned long long*>(j.dev_offsets)
                                             : reinterpret_cast<unsigned long long*>(d + o_res + r_off[i]);
    g.err = j.async ? s->d_err : reinterpret_cast<uint32_t*>(d + o_res + r_err[i]);
    segs[si] = g;
    ib[si] = item_base;
    sb[si] = sec_base;
    if (s->withhold < T * A * s->H) withhold = item_base + s->withhold + 1u;
    s->withhold = UINT32_MAX;  // one call
    item_base += T * A * s->H;
    sec_base += T * A;
    staged |= s->opt.stages ? 1u : 0u;
    key.push_back(((uint64_t)s->H << 32) | s->W);
    key.push_back(((uint64_t)A << 32) | T);
    key.push_back(s->opt.stages);
  }
  key.push_back(staged);
  key.push_back(withhold);
  sig.push_back(staged);
  bool async = false;
  for (const EncJob& j : jobs) async |= j.async;

  jiffy::EncParams p{};
  p.n_seg = n;
  p.n_items = (uint32_t)items;
  p.n_sec = (uint32_t)secs;
  p.max_W = max_W;
  p.split = split;
  p.split_W = split_W;
  p.seg = reinterpret_cast<const jiffy::EncSeg*>(d + o_up + u_seg);
  p.seg_item_base = reinterpret_cast<const uint32_t*>(d + o_up + u_ib);
  p.seg_sec_base = reinterpret_cast<const uint32_t*>(d + o_up + u_sb);
  p.trial_rows = trial_rows;
  p.cost = reinterpret_cast<uint32_t*>(d + o_cost);
  p.modes = reinterpret_cast<uint32_t*>(d + o_modes);
  p.row_bytes = reinterpret_cast<uint32_t*>(d + o_rb);
  p.row_nnz = reinterpret_cast<uint32_t*>(d + o_rn);
  p.row_carry = reinterpret_cast<uint32_t*>(d + o_rc);
  p.st_carry = reinterpret_cast<unsigned long long*>(d + o_stc);
  p.slots = d + o_slots;
  p.sec_bytes = reinterpret_cast<unsigned long long*>(d + o_secb);
  p.sec_nnz = reinterpret_cast<uint32_t*>(d + o_secn);
  p.ticket = reinterpret_cast<uint32_t*>(d + o_tick);
  p.staged = staged | (withhold ? 1u : 0u);
  p.withhold = withhold;
  if (zmax_blk) {
    p.zmask = d + o_zm;
    p.zblk = d + o_zblk;
    p.zblk_bytes = reinterpret_cast<uint32_t*>(d + o_zbb);
    p.zfr_bytes = reinterpret_cast<uint32_t*>(d + o_zfr);
    p.zmax_blk = zmax_blk;
  }
  uint8_t* hres = h + h_res;
  // the segment table, copied on the call's stream ahead of the rest (and
  // outside any captured sequence) unless it is in its slot already
  const bool up_same = table_resident(ws, slot, d + o_up, h, up.off);
  if (!up_same && cudaMemcpyAsync(d + o_up, h, up.off, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    table_uploaded(ws, slot, false, up_same, d + o_up, h, up.off);
    return JIFFY_ERR_CUDA;
  }
  // (the event marks the host table's last copy: calls that copy nothing leave it)
  if (!up_same && async && record_ev(ws.uploaded, st) != cudaSuccess) return JIFFY_ERR_CUDA;

  // the rest of the call on one stream: clear, kernels, results
  auto enqueue = [&](cudaStream_t s, const jiffy::EncParams& pp, void* const* evs) -> int {
    const cudaError_t ce = cudaMemsetAsync(d + o_zero, 0, zero_bytes, s);
    if (ce != cudaSuccess) return (int)ce;
    const int rc = jiffy::launch_encode(pp, s, evs);
    if (rc != 0 || async) return rc;  // enqueue-only: offsets and errors stay on the device
    return (int)cudaMemcpyAsync(hres, d + o_res, rs.off, cudaMemcpyDeviceToHost, s);
  };
  if (ws.autotune) {
    auto it = ws.tuned.find(sig);
    if (it == ws.tuned.end()) {
      RowsLaunch best{};
      r = tune(ws, true, p, st, [](const jiffy::EncParams& pp, RowsLaunch* o) { return jiffy::encode_rows_launch(pp, o); },
               enqueue, &best);
      if (r != JIFFY_OK) return r;
      it = ws.tuned.emplace(sig, best).first;
      tune_cache_store(ws);
    }
    p.wpc = it->second.wpc;
    p.ctas_per_sm = it->second.ctas_per_sm;
  }
  if (ws.fixed[0].wpc) p.wpc = ws.fixed[0].wpc;
  if (ws.fixed[0].ctas_per_sm) p.ctas_per_sm = ws.fixed[0].ctas_per_sm;
  if (jiffy::encode_rows_launch(p, &ws.last) != 0) return JIFFY_ERR_CUDA;
  key.push_back(((uint64_t)p.wpc << 32) | p.ctas_per_sm);
  key.push_back(trial_rows);
  key.push_back(async ? 1u : 0u);
  for (const EncJob& j : jobs) key.push_back((uint64_t)(uintptr_t)j.dev_offsets);
  const bool timed = ws.profile;
  key.push_back(timed ? 1u : 0u);
  void* evs[4] = {ws.ev[0], ws.ev[1], ws.ev[2], ws.ev[3]};
  void* const* tev = timed ? (async ? next_evset(ws, 3) : evs) : nullptr;
  if (timed && !tev) return JIFFY_ERR_CUDA;
  // (a timed enqueue-only call uses the next event set of the ring)
  r = run_sequence(ws, ws.g_enc[slot], key, st, ws.graphs, tev, timed ? 4u : 0u,
                   [&](cudaStream_t s) { return enqueue(s, p, tev); });
  table_uploaded(ws, slot, r == JIFFY_OK, up_same, d + o_up, h, up.off);
  if (r != JIFFY_OK) return r;
  if (cudaEventRecord(ws.done, st) != cudaSuccess) return JIFFY_ERR_CUDA;
  ws.calls++;
  if (async) {  // enqueue only: nothing to read back; errors go to the stream's device word
    ws.upload_pending = true;
    for (EncJob& j : jobs) {
      j.s->cur = 1 - j.s->cur;
      j.s->frame += j.T;
      j.s->async_out = true;
      if (cudaEventRecord(j.s->async_done, st) != cudaSuccess) return JIFFY_ERR_CUDA;
    }
    ws.n_kernel_ms = 0;
    return JIFFY_OK;
  }
  // the streams advance now; finish() rolls back those that failed
  for (EncJob& j : jobs) {
    j.s->cur = 1 - j.s->cur;
    j.s->frame += j.T;
    j.s->in_flight = true;
  }
  ws.pend.kind = 1;
  ws.pend.enc = jobs;
  ws.pend.r_err = r_err;
  ws.pend.r_off = r_off;
  ws.pend.hres = hres;
  ws.pend.n_kernels = timed ? 3 : 0;
  return JIFFY_OK;
}

// ---------------------------------------------------------------- decode
jiffy_status enqueue_decode(Workspace& ws, std::vector<DecJob>& jobs, cudaStream_t st) {
  const uint32_t n = (uint32_t)jobs.size();
  if (ws.pend.kind) return JIFFY_ERR_STATE;
  unsigned long long items = 0;
  uint32_t max_W = 1;
  std::vector<jiffy_stream*> ss(n);
  for (uint32_t i = 0; i < n; i++) {
    DecJob& j = jobs[i];
    *j.status = JIFFY_OK;
    jiffy_stream* s = j.s;
    ss[i] = s;
    if (!s || !j.in || !j.frame_offsets || !j.planes_out || j.T == 0) return JIFFY_ERR_INVALID_ARG;
    if (s->role != JIFFY_DECODER || s->ws.device != ws.device || s->in_flight) return JIFFY_ERR_STATE;
    if (reinterpret_cast<uintptr_t>(j.in) & 3u) return JIFFY_ERR_INVALID_ARG;
    for (size_t q = 0; q < (size_t)j.T * s->A; q++)
      if (!j.planes_out[q]) return JIFFY_ERR_INVALID_ARG;
    if (j.async) {  // the offsets are on the device: the kernel checks them
      if (reinterpret_cast<uintptr_t>(j.frame_offsets) & 7u) return JIFFY_ERR_INVALID_ARG;
      items += (unsigned long long)j.T * s->A * s->H;
      if (s->W > max_W) max_W = s->W;
      continue;
    }
    // frame offsets: aligned, increasing by at least a frame header, inside `in`
    const uint64_t* fo = j.frame_offsets;
    const uint32_t fh = frame_header_bytes(s->A);
    const uint64_t first = s->frame == 0 ? stream_header_bytes(s->A) : 0u;
    jiffy_status bad = JIFFY_OK;
    if (fo[0] < first) bad = JIFFY_ERR_CORRUPT;
    for (uint32_t t = 0; t < j.T && bad == JIFFY_OK; t++) {
      if ((fo[t] & 3u) || fo[t + 1] < fo[t] + fh) bad = JIFFY_ERR_CORRUPT;
      else if (fo[t + 1] - fo[t] > 0xffffffffull) bad = JIFFY_ERR_CORRUPT;
    }
    if (fo[j.T] > j.in_len || (fo[j.T] & 3u)) bad = JIFFY_ERR_CORRUPT;
    if (bad != JIFFY_OK) {
      *j.status = bad;
      return bad;
    }
    items += (unsigned long long)j.T * s->A * s->H;
    if (s->W > max_W) max_W = s->W;
  }
  if (check_distinct(ss) != JIFFY_OK) return JIFFY_ERR_INVALID_ARG;
  if (items > 0x7fffffffull) return JIFFY_ERR_INVALID_ARG;

  Carver up;
  const size_t u_seg = up.take(sizeof(jiffy::DecSeg) * n), u_ib = up.take(4ull * n), u_sb = up.take(4ull * n);
  std::vector<size_t> u_ptrs(n);
  for (uint32_t i = 0; i < n; i++)
    u_ptrs[i] = up.take(8ull * ((size_t)(jobs[i].T + 2) * jobs[i].s->A + jobs[i].T + 1));
  Carver rs;
  std::vector<size_t> r_err(n);
  for (uint32_t i = 0; i < n; i++) r_err[i] = rs.take(8);
  Carver c;
  const uint32_t slot = next_slot(ws);  // segment-table slots alternate
  const size_t o_up_slot[2] = {c.take(up.off), c.take(up.off)};
  const size_t o_up = o_up_slot[slot];
  const size_t o_zero = c.take(0);
  const size_t o_done = c.take(4ull * items), o_tick = c.take(8);
  const size_t o_res = c.take(rs.off);
  const size_t zero_bytes = c.off - o_zero;
  std::vector<unsigned long long> mask_base(n);
  unsigned long long mask_words = 0;
  for (uint32_t i = 0; i < n; i++) {
    const jiffy_stream* s = jobs[i].s;
    mask_base[i] = mask_words;
    mask_words += (unsigned long long)jobs[i].T * s->A * s->H * ((s->W + 31) / 32);
  }
  const size_t o_masks = c.take(4ull * mask_words);
  // Zstandard mask sections: their decoded (still XORed) mask bytes
  std::vector<unsigned long long> zm_base(n);
  unsigned long long zm_total = 0, n_sec = 0;
  uint32_t zmax_blk = 0;
  for (uint32_t i = 0; i < n; i++) {
    const jiffy_stream* s = jobs[i].s;
    n_sec += (unsigned long long)jobs[i].T * s->A;
    if (!(s->opt.stages & jiffy::kStageZstdMask)) continue;
    zm_base[i] = zm_total;
    zm_total += align_up((size_t)s->H * ((s->W + 7) / 8), 16) * jobs[i].T * s->A;
    zmax_blk = std::max(zmax_blk, jiffy::zmask_blocks(s->H, s->W));
  }
  const size_t o_zdec = c.take(zm_total);
  const size_t h_res = align_up(up.off, 256);
  jiffy_status r = ensure_scratch(ws, c.off, h_res + rs.off);
  if (r == JIFFY_OK) r = wait_upload(ws);
  if (r != JIFFY_OK) return r;
  uint8_t* d = ws.d_scratch;
  uint8_t* h = ws.h_pinned;

  jiffy::DecSeg* segs = reinterpret_cast<jiffy::DecSeg*>(h + u_seg);
  uint32_t* ib = reinterpret_cast<uint32_t*>(h + u_ib);
  uint32_t* sbk = reinterpret_cast<uint32_t*>(h + u_sb);
  std::vector<uint64_t> key{2, n, (uint64_t)(uintptr_t)d, (uint64_t)(uintptr_t)h};
  std::vector<uint32_t> sig{2, max_W, log2_ceil(items)};
  uint32_t staged = 0, withhold = 0;
  uint32_t item_base = 0, sec_base = 0;
  for (uint32_t i = 0; i < n; i++) {
    DecJob& j = jobs[i];
    jiffy_stream* s = j.s;
    const uint32_t T = j.T, A = s->A;
    uint64_t* hp = reinterpret_cast<uint64_t*>(h + u_ptrs[i]);
    for (size_t q = 0; q < (size_t)T * A; q++) hp[q] = reinterpret_cast<uint64_t>(j.planes_out[q]);
    for (uint32_t a = 0; a < A; a++) {
      hp[(size_t)T * A + a] = reinterpret_cast<uint64_t>(s->d_state[s->cur] + s->plane_off[a]);
      hp[(size_t)T * A + A + a] = reinterpret_cast<uint64_t>(s->d_state[1 - s->cur] + s->plane_off[a]);
    }
    if (!j.async) std::memcpy(hp + (size_t)(T + 2) * A, j.frame_offsets, 8ull * (T + 1));
    const uint8_t* dp = d + o_up + u_ptrs[i];
    jiffy::DecSeg g{};
    g.H = s->H;
    g.W = s->W;
    g.A = A;
    g.T = T;
    g.nw = (s->W + 31) / 32;
    g.ncls = (s->opt.stages & (jiffy::kStageNoMask | jiffy::kStageZstdMask)) ? 0u : (g.nw + 15) / 16;
    g.stages = s->opt.stages;
    g.sec_base = sec_base;
    if (s->opt.stages & jiffy::kStageZstdMask) {
      g.zm_rb = (s->W + 7) / 8;
      g.zm_nblk = jiffy::zmask_blocks(s->H, s->W);
      g.zm_stride = align_up((size_t)s->H * g.zm_rb, 16);
      g.zm_base = zm_base[i];
    }
    g.frame0 = s->frame;
    g.fhdr = frame_header_bytes(A);
    g.check_shdr = s->frame == 0;
    g.item_base = item_base;
    g.attrs = s->d_attrs;
    g.in = static_cast<const uint8_t*>(j.in);
    g.in_len = j.in_len;
    g.outp = reinterpret_cast<uint8_t* const*>(dp);
    g.state = reinterpret_cast<const uint8_t* const*>(dp + 8ull * T * A);
    g.state_next = reinterpret_cast<uint8_t* const*>(dp + 8ull * (T + 1) * A);
    g.off = j.async ? reinterpret_cast<const unsigned long long*>(j.frame_offsets)
                    : reinterpret_cast<const unsigned long long*>(dp + 8ull * (T + 2) * A);
    g.err = j.async ? s->d_err : reinterpret_cast<uint32_t*>(d + o_res + r_err[i]);
    g.mask_base = mask_base[i];
    segs[i] = g;
    ib[i] = item_base;
    sbk[i] = sec_base;
    if (s->withhold < T * A * s->H) withhold = item_base + s->withhold + 1u;
    s->withhold = UINT32_MAX;  // one call
    item_base += T * A * s->H;
    sec_base += T * A;
    staged |= s->opt.stages ? 1u : 0u;
    key.push_back(((uint64_t)s->H << 32) | s->W);
    key.push_back(((uint64_t)A << 32) | T);
    key.push_back(s->opt.stages);
  }
  key.push_back(staged);
  sig.push_back(staged);
  bool async = false;
  for (const DecJob& j : jobs) {
    async |= j.async;
    if (j.async) key.push_back((uint64_t)(uintptr_t)j.frame_offsets);
  }
  key.push_back(async ? 1u : 0u);

  jiffy::DecParams p{};
  p.n_seg = n;
  p.n_items = (uint32_t)items;
  p.max_W = max_W;
  p.seg = reinterpret_cast<const jiffy::DecSeg*>(d + o_up + u_seg);
  p.seg_item_base = reinterpret_cast<const uint32_t*>(d + o_up + u_ib);
  p.done = reinterpret_cast<uint32_t*>(d + o_done);
  p.masks = reinterpret_cast<uint32_t*>(d + o_masks);
  p.ticket = reinterpret_cast<uint32_t*>(d + o_tick);
  p.staged = staged | (withhold ? 1u : 0u);
  p.withhold = withhold;
  p.n_sec = (uint32_t)n_sec;
  p.seg_sec_base = reinterpret_cast<const uint32_t*>(d + o_up + u_sb);
  if (zmax_blk) {
    p.zdec = d + o_zdec;
    p.zmax_blk = zmax_blk;
  }
  key.push_back(withhold);
  uint8_t* hres = h + h_res;
  // the segment table, copied on the call's stream ahead of the rest (and
  // outside any captured sequence) unless it is in its slot already
  const bool up_same = table_resident(ws, slot, d + o_up, h, up.off);
  if (!up_same && cudaMemcpyAsync(d + o_up, h, up.off, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    table_uploaded(ws, slot, false, up_same, d + o_up, h, up.off);
    return JIFFY_ERR_CUDA;
  }
  // (the event marks the host table's last copy: calls that copy nothing leave it)
  if (!up_same && async && record_ev(ws.uploaded, st) != cudaSuccess) return JIFFY_ERR_CUDA;

  auto enqueue = [&](cudaStream_t s, const jiffy::DecParams& pp, void* const* evs) -> int {
    const cudaError_t ce = cudaMemsetAsync(d + o_zero, 0, zero_bytes, s);
    if (ce != cudaSuccess) return (int)ce;
    const int rc = jiffy::launch_decode(pp, s, evs);
    if (rc != 0 || async) return rc;  // enqueue-only: errors stay on the device
    return (int)cudaMemcpyAsync(hres, d + o_res, rs.off, cudaMemcpyDeviceToHost, s);
  };
  if (ws.autotune) {
    auto it = ws.tuned.find(sig);
    if (it == ws.tuned.end()) {
      RowsLaunch best{};
      r = tune(ws, false, p, st, [](const jiffy::DecParams& pp, RowsLaunch* o) { return jiffy::decode_rows_launch(pp, o); },
               enqueue, &best);
      if (r != JIFFY_OK) return r;
      it = ws.tuned.emplace(sig, best).first;
      tune_cache_store(ws);
    }
    p.wpc = it->second.wpc;
    p.ctas_per_sm = it->second.ctas_per_sm;
    p.items_per_ticket = it->second.items_per_ticket;
  }
  if (ws.fixed[1].wpc) p.wpc = ws.fixed[1].wpc;
  if (ws.fixed[1].ctas_per_sm) p.ctas_per_sm = ws.fixed[1].ctas_per_sm;
  if (ws.fixed[1].items_per_ticket) p.items_per_ticket = ws.fixed[1].items_per_ticket;
  if (jiffy::decode_rows_launch(p, &ws.last) != 0) return JIFFY_ERR_CUDA;
  key.push_back(((uint64_t)p.wpc << 32) | p.ctas_per_sm);
  key.push_back(p.items_per_ticket);
  const bool timed = ws.profile;
  key.push_back(timed ? 1u : 0u);
  void* evs[2] = {ws.ev[0], ws.ev[1]};
  void* const* tev = timed ? (async ? next_evset(ws, 1) : evs) : nullptr;
  if (timed && !tev) return JIFFY_ERR_CUDA;
  r = run_sequence(ws, ws.g_dec[slot], key, st, ws.graphs, tev, timed ? 2u : 0u,
                   [&](cudaStream_t s) { return enqueue(s, p, tev); });
  table_uploaded(ws, slot, r == JIFFY_OK, up_same, d + o_up, h, up.off);
  if (r != JIFFY_OK) return r;
  if (cudaEventRecord(ws.done, st) != cudaSuccess) return JIFFY_ERR_CUDA;
  ws.calls++;
  if (async) {  // enqueue only: nothing to read back; errors go to the stream's device word
    ws.upload_pending = true;
    for (DecJob& j : jobs) {
      j.s->cur = 1 - j.s->cur;
      j.s->frame += j.T;
      j.s->async_out = true;
      if (cudaEventRecord(j.s->async_done, st) != cudaSuccess) return JIFFY_ERR_CUDA;
    }
    ws.n_kernel_ms = 0;
    return JIFFY_OK;
  }
  for (DecJob& j : jobs) {
    j.s->cur = 1 - j.s->cur;
    j.s->frame += j.T;
    j.s->in_flight = true;
  }
  ws.pend.kind = 2;
  ws.pend.dec = jobs;
  ws.pend.r_err = r_err;
  ws.pend.hres = hres;
  ws.pend.n_kernels = timed ? 1 : 0;
  return JIFFY_OK;
}

// Waits for the pending call, reports per-stream results and rolls back the
// streams that failed. Returns the first failing status.
jiffy_status finish(Workspace& ws) {
  Pending& pd = ws.pend;
  if (!pd.kind) return JIFFY_OK;
  const cudaError_t ce = cudaEventSynchronize(ws.done);
  jiffy_status first = JIFFY_OK;
  auto settle = [&](jiffy_stream* s, uint32_t T, jiffy_status res) {
    s->in_flight = false;
    if (res != JIFFY_OK) {
      s->cur = 1 - s->cur;
      s->frame -= T;
      if (first == JIFFY_OK) first = res;
    }
  };
  if (pd.kind == 1) {
    for (size_t i = 0; i < pd.enc.size(); i++) {
      EncJob& j = pd.enc[i];
      uint32_t err = 0;
      std::memcpy(&err, pd.hres + pd.r_err[i], 4);
      const uint64_t* foff = reinterpret_cast<const uint64_t*>(pd.hres + pd.r_off[i]);
      const jiffy_status res = ce != cudaSuccess ? JIFFY_ERR_CUDA : map_device_error(err);
      *j.status = res;
      if (ce == cudaSuccess) *j.out_len = foff[j.T];
      if (res == JIFFY_OK && j.frame_offsets) std::memcpy(j.frame_offsets, foff, 8ull * (j.T + 1));
      settle(j.s, j.T, res);
    }
  } else {
    for (size_t i = 0; i < pd.dec.size(); i++) {
      DecJob& j = pd.dec[i];
      uint32_t err = 0;
      std::memcpy(&err, pd.hres + pd.r_err[i], 4);
      const jiffy_status res = ce != cudaSuccess ? JIFFY_ERR_CUDA : map_device_error(err);
      *j.status = res;
      settle(j.s, j.T, res);
    }
  }
  ws.n_kernel_ms = 0;
  if (pd.n_kernels && ce == cudaSuccess) {
    uint32_t k = 0;
    for (; k < pd.n_kernels; k++) {
      float ms = 0;
      if (cudaEventElapsedTime(&ms, ws.ev[k], ws.ev[k + 1]) != cudaSuccess) break;
      ws.kernel_ms[k] = ms;
    }
    if (k == pd.n_kernels) ws.n_kernel_ms = k;
  }
  pd = Pending{};
  return first;
}

jiffy_status run_encode(Workspace& ws, std::vector<EncJob>& jobs, cudaStream_t st) {
  const jiffy_status r = enqueue_encode(ws, jobs, st);
  return r != JIFFY_OK ? r : finish(ws);
}

jiffy_status run_decode(Workspace& ws, std::vector<DecJob>& jobs, cudaStream_t st) {
  const jiffy_status r = enqueue_decode(ws, jobs, st);
  return r != JIFFY_OK ? r : finish(ws);
}

bool same_config(const jiffy_stream* a, const jiffy_stream* b) {
  if (a->H != b->H || a->W != b->W || a->A != b->A || a->opt.stages != b->opt.stages) return false;
  for (uint32_t i = 0; i < a->A; i++)
    if (a->attrs[i].s != b->attrs[i].s || a->attrs[i].P != b->attrs[i].P) return false;
  return true;
}

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
  // (with the Zstandard mask the rows carry no mask words; its index, frame
  // header, block headers and padding stay within the 16 + 8 per block added)
  const size_t section = 8ull * H + (size_t)H * jiffy::row_bound_bytes(W) + 16ull + 8ull * jiffy::zmask_blocks(H, W);
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
  jiffy_options o{4, -1, 0};
  if (opt) o = *opt;
  if (o.test_lines == 0 || o.force_mode < -1 || o.force_mode > 1 || (o.stages & ~jiffy::kStageAll))
    return JIFFY_ERR_INVALID_ARG;
  if ((o.stages & jiffy::kStageNoMask) && (o.stages & jiffy::kStageZstdMask)) return JIFFY_ERR_INVALID_ARG;
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
  s->ws.device = device;
  s->ws.graphs = true;  // a stream replays its call sequence while the call's shape repeats
  s->role = role;
  s->H = H;
  s->W = W;
  s->A = n_attr;
  s->opt = o;
  size_t state_bytes = 0;
  for (uint32_t a = 0; a < n_attr; a++) {
    const AttrDev d = jiffy::make_attr(attrs[a].dtype_bytes, attrs[a].precision);
    s->attrs.push_back(d);
    s->plane_off.push_back(state_bytes);
    state_bytes = align_up(state_bytes + (size_t)H * W * d.s, 256);
  }
  s->state_bytes = state_bytes;
  jiffy_status st = JIFFY_OK;
  if (cudaMalloc(&s->d_attrs, sizeof(AttrDev) * n_attr) != cudaSuccess ||
      cudaMalloc(&s->d_state[0], state_bytes) != cudaSuccess ||
      cudaMalloc(&s->d_state[1], state_bytes) != cudaSuccess || cudaMalloc(&s->d_err, 4) != cudaSuccess) {
    st = JIFFY_ERR_NOMEM;
  } else if (cudaEventCreateWithFlags(&s->async_done, cudaEventDisableTiming) != cudaSuccess ||
             cudaMemset(s->d_err, 0, 4) != cudaSuccess) {
    st = JIFFY_ERR_CUDA;
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
  DeviceGuard g(s->ws.device);
  cudaDeviceSynchronize();
  if (s->d_attrs) cudaFree(s->d_attrs);
  if (s->d_state[0]) cudaFree(s->d_state[0]);
  if (s->d_state[1]) cudaFree(s->d_state[1]);
  if (s->d_err) cudaFree(s->d_err);
  if (s->async_done) cudaEventDestroy(s->async_done);
  release(s->ws);
  delete s;
}

jiffy_status jiffy_stream_reset(jiffy_stream* s) {
  if (!s) return JIFFY_ERR_INVALID_ARG;
  if (s->in_flight) return JIFFY_ERR_STATE;
  s->frame = 0;
  return JIFFY_OK;
}

uint32_t jiffy_stream_frame_index(const jiffy_stream* s) { return s ? s->frame : 0u; }

size_t jiffy_stream_device_bytes(const jiffy_stream* s) {
  if (!s) return 0;
  return 2 * s->state_bytes + sizeof(AttrDev) * s->A + s->ws.scratch_cap;
}

jiffy_status jiffy_stream_copy_state(jiffy_stream* dst, const jiffy_stream* src, void* cuda_stream) {
  if (!dst || !src) return JIFFY_ERR_INVALID_ARG;
  if (dst == src) return JIFFY_OK;
  if (!same_config(dst, src) || dst->ws.device != src->ws.device) return JIFFY_ERR_INVALID_ARG;
  if (dst->in_flight || src->in_flight) return JIFFY_ERR_STATE;
  DeviceGuard g(dst->ws.device);
  if (!g.ok) return JIFFY_ERR_CUDA;
  if (cudaMemcpyAsync(dst->d_state[dst->cur], src->d_state[src->cur], src->state_bytes, cudaMemcpyDeviceToDevice,
                      reinterpret_cast<cudaStream_t>(cuda_stream)) != cudaSuccess)
    return JIFFY_ERR_CUDA;
  dst->frame = src->frame;
  return JIFFY_OK;
}

// Saved state: "JFYS", version 1, H, W, A, stages, frame counter (u32 each),
// then (bytes per sample, precision) per attribute, then the state planes as
// they lie in the state buffer.
namespace {
constexpr uint32_t kStateMagic = 0x5359464Au;  // "JFYS"
size_t state_header_bytes(uint32_t A) { return 28ull + 8ull * A; }
void put32(uint8_t* b, size_t at, uint32_t v) { std::memcpy(b + at, &v, 4); }
uint32_t get32(const uint8_t* b, size_t at) {
  uint32_t v;
  std::memcpy(&v, b + at, 4);
  return v;
}
}  // namespace

size_t jiffy_stream_state_size(const jiffy_stream* s) {
  return s ? state_header_bytes(s->A) + s->state_bytes : 0;
}

jiffy_status jiffy_stream_save_state(jiffy_stream* s, void* host_buf, size_t capacity) {
  if (!s || !host_buf) return JIFFY_ERR_INVALID_ARG;
  if (capacity < jiffy_stream_state_size(s)) return JIFFY_ERR_CAPACITY;
  if (s->in_flight || s->async_out) return JIFFY_ERR_STATE;
  DeviceGuard g(s->ws.device);
  if (!g.ok) return JIFFY_ERR_CUDA;
  uint8_t* b = static_cast<uint8_t*>(host_buf);
  const uint32_t head[7] = {kStateMagic, 1u, s->H, s->W, s->A, s->opt.stages, s->frame};
  for (uint32_t i = 0; i < 7; i++) put32(b, 4ull * i, head[i]);
  for (uint32_t a = 0; a < s->A; a++) {
    put32(b, 28ull + 8ull * a, s->attrs[a].s);
    put32(b, 32ull + 8ull * a, s->attrs[a].P);
  }
  if (cudaMemcpy(b + state_header_bytes(s->A), s->d_state[s->cur], s->state_bytes, cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return JIFFY_ERR_CUDA;
  return JIFFY_OK;
}

jiffy_status jiffy_stream_load_state(jiffy_stream* s, const void* host_buf, size_t len) {
  if (!s || !host_buf) return JIFFY_ERR_INVALID_ARG;
  if (s->in_flight || s->async_out) return JIFFY_ERR_STATE;
  const uint8_t* b = static_cast<const uint8_t*>(host_buf);
  if (len < 28 || get32(b, 0) != kStateMagic || get32(b, 4) != 1u) return JIFFY_ERR_CORRUPT;
  if (get32(b, 8) != s->H || get32(b, 12) != s->W || get32(b, 16) != s->A || get32(b, 20) != s->opt.stages)
    return JIFFY_ERR_INVALID_ARG;
  if (len != jiffy_stream_state_size(s)) return JIFFY_ERR_CORRUPT;
  for (uint32_t a = 0; a < s->A; a++)
    if (get32(b, 28ull + 8ull * a) != s->attrs[a].s || get32(b, 32ull + 8ull * a) != s->attrs[a].P)
      return JIFFY_ERR_INVALID_ARG;
  DeviceGuard g(s->ws.device);
  if (!g.ok) return JIFFY_ERR_CUDA;
  if (cudaMemcpy(s->d_state[s->cur], b + state_header_bytes(s->A), s->state_bytes, cudaMemcpyHostToDevice) !=
      cudaSuccess)
    return JIFFY_ERR_CUDA;
  s->frame = get32(b, 24);
  return JIFFY_OK;
}

jiffy_status jiffy_stream_test_withhold_row(jiffy_stream* s, uint32_t row_item) {
  if (!s) return JIFFY_ERR_INVALID_ARG;
  s->withhold = row_item;
  return JIFFY_OK;
}

jiffy_status jiffy_stream_set_profiling(jiffy_stream* s, int enable) {
  if (!s) return JIFFY_ERR_INVALID_ARG;
  return set_profiling(s->ws, enable);
}

uint32_t jiffy_stream_kernel_times(const jiffy_stream* s, float* ms, uint32_t n) {
  if (!s) return 0;
  for (uint32_t i = 0; i < n && i < s->ws.n_kernel_ms; i++) ms[i] = s->ws.kernel_ms[i];
  return s->ws.n_kernel_ms;
}

jiffy_status jiffy_stream_wait(jiffy_stream* s) {
  TraceRange trace("jiffy_stream_wait");
  if (!s) return JIFFY_ERR_INVALID_ARG;
  if (!s->async_out) return JIFFY_OK;
  DeviceGuard g(s->ws.device);
  if (!g.ok) return JIFFY_ERR_CUDA;
  uint32_t err = 0;
  if (cudaEventSynchronize(s->async_done) != cudaSuccess || cudaMemcpy(&err, s->d_err, 4, cudaMemcpyDeviceToHost) !=
      cudaSuccess || cudaMemset(s->d_err, 0, 4) != cudaSuccess)
    return JIFFY_ERR_CUDA;
  s->async_out = false;
  s->ws.upload_pending = false;
  Workspace& w = s->ws;  // kernel times: averages over the calls since the last wait
  harvest(w, true);
  if (w.acc_calls) {
    for (uint32_t k = 0; k < w.acc_nk; k++) w.kernel_ms[k] = (float)(w.acc_ms[k] / w.acc_calls);
    w.n_kernel_ms = w.acc_nk;
  }
  w.acc_ms[0] = w.acc_ms[1] = w.acc_ms[2] = 0;
  w.acc_calls = 0;
  return map_device_error(err);
}

jiffy_status jiffy_encode_seq_async(jiffy_stream* s, uint32_t n_scans, const void* const* planes, void* out,
                                    size_t out_capacity, uint64_t* frame_offsets_dev, void* cuda_stream) {
  TraceRange trace("jiffy_encode_seq_async");
  if (!s) return JIFFY_ERR_INVALID_ARG;
  DeviceGuard g(s->ws.device);
  if (!g.ok) return JIFFY_ERR_CUDA;
  jiffy_status st = JIFFY_OK;
  EncJob job{s, n_scans, planes, out, out_capacity, nullptr, nullptr, &st};
  job.async = true;
  job.dev_offsets = frame_offsets_dev;
  std::vector<EncJob> jobs{job};
  return enqueue_encode(s->ws, jobs, reinterpret_cast<cudaStream_t>(cuda_stream));
}

jiffy_status jiffy_decode_seq_async(jiffy_stream* s, uint32_t n_scans, const void* in, size_t in_capacity,
                                    const uint64_t* frame_offsets_dev, void* const* planes_out, void* cuda_stream) {
  TraceRange trace("jiffy_decode_seq_async");
  if (!s) return JIFFY_ERR_INVALID_ARG;
  DeviceGuard g(s->ws.device);
  if (!g.ok) return JIFFY_ERR_CUDA;
  jiffy_status st = JIFFY_OK;
  DecJob job{s, n_scans, in, in_capacity, frame_offsets_dev, planes_out, &st};
  job.async = true;
  std::vector<DecJob> jobs{job};
  return enqueue_decode(s->ws, jobs, reinterpret_cast<cudaStream_t>(cuda_stream));
}

jiffy_status jiffy_encode_seq(jiffy_stream* s, uint32_t n_scans, const void* const* planes, void* out,
                              size_t out_capacity, uint64_t* frame_offsets, size_t* out_len, void* cuda_stream) {
  TraceRange trace("jiffy_encode_seq");
  if (!s) return JIFFY_ERR_INVALID_ARG;
  DeviceGuard g(s->ws.device);
  if (!g.ok) return JIFFY_ERR_CUDA;
  if (s->async_out) {  // earlier enqueue-only calls first
    const jiffy_status w = jiffy_stream_wait(s);
    if (w != JIFFY_OK) return w;
  }
  jiffy_status st = JIFFY_OK;
  std::vector<EncJob> jobs{EncJob{s, n_scans, planes, out, out_capacity, frame_offsets, out_len, &st}};
  return run_encode(s->ws, jobs, reinterpret_cast<cudaStream_t>(cuda_stream));
}

jiffy_status jiffy_encode(jiffy_stream* s, const void* const* planes, void* out, size_t out_capacity,
                          size_t* out_len, void* cuda_stream) {
  TraceRange trace("jiffy_encode");
  return jiffy_encode_seq(s, 1, planes, out, out_capacity, nullptr, out_len, cuda_stream);
}

jiffy_status jiffy_decode_seq(jiffy_stream* s, uint32_t n_scans, const void* in, size_t in_len,
                              const uint64_t* frame_offsets, void* const* planes_out, void* cuda_stream) {
  TraceRange trace("jiffy_decode_seq");
  if (!s) return JIFFY_ERR_INVALID_ARG;
  DeviceGuard g(s->ws.device);
  if (!g.ok) return JIFFY_ERR_CUDA;
  if (s->async_out) {  // earlier enqueue-only calls first
    const jiffy_status w = jiffy_stream_wait(s);
    if (w != JIFFY_OK) return w;
  }
  jiffy_status st = JIFFY_OK;
  std::vector<DecJob> jobs{DecJob{s, n_scans, in, in_len, frame_offsets, planes_out, &st}};
  return run_decode(s->ws, jobs, reinterpret_cast<cudaStream_t>(cuda_stream));
}

jiffy_status jiffy_decode(jiffy_stream* s, const void* in, size_t in_len, void* const* planes_out,
                          void* cuda_stream) {
  TraceRange trace("jiffy_decode");
  if (!s) return JIFFY_ERR_INVALID_ARG;
  const uint64_t off[2] = {s->frame == 0 ? stream_header_bytes(s->A) : 0u, in_len};
  return jiffy_decode_seq(s, 1, in, in_len, off, planes_out, cuda_stream);
}

jiffy_status jiffy_batch_create(jiffy_batch** out, int device) {
  if (!out) return JIFFY_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return JIFFY_ERR_CUDA;
  jiffy_batch* b = new (std::nothrow) jiffy_batch();
  if (!b) return JIFFY_ERR_NOMEM;
  b->ws.device = device;
  *out = b;
  return JIFFY_OK;
}

void jiffy_batch_destroy(jiffy_batch* b) {
  if (!b) return;
  DeviceGuard g(b->ws.device);
  finish(b->ws);
  cudaDeviceSynchronize();
  release(b->ws);
  delete b;
}

jiffy_status jiffy_batch_set_profiling(jiffy_batch* b, int enable) {
  if (!b) return JIFFY_ERR_INVALID_ARG;
  return set_profiling(b->ws, enable);
}

uint32_t jiffy_batch_kernel_times(const jiffy_batch* b, float* ms, uint32_t n) {
  if (!b) return 0;
  for (uint32_t i = 0; i < n && i < b->ws.n_kernel_ms; i++) ms[i] = b->ws.kernel_ms[i];
  return b->ws.n_kernel_ms;
}

jiffy_status jiffy_batch_set_graphs(jiffy_batch* b, int enable) {
  if (!b) return JIFFY_ERR_INVALID_ARG;
  if (b->ws.pend.kind) return JIFFY_ERR_STATE;
  b->ws.graphs = enable != 0;
  if (!b->ws.graphs) {
    DeviceGuard g(b->ws.device);
    drop_graphs(b->ws);
  }
  return JIFFY_OK;
}

jiffy_status jiffy_batch_set_autotune(jiffy_batch* b, int enable) {
  if (!b) return JIFFY_ERR_INVALID_ARG;
  b->ws.autotune = enable != 0;
  if (b->ws.autotune) {  // configurations an earlier process tuned on this kind of device
    DeviceGuard g(b->ws.device);
    if (!g.ok) return JIFFY_ERR_CUDA;
    tune_cache_load(b->ws);
  }
  return JIFFY_OK;
}

jiffy_status jiffy_batch_set_launch(jiffy_batch* b, jiffy_role role, uint32_t warps_per_cta,
                                    uint32_t ctas_per_sm, uint32_t items_per_ticket) {
  if (!b || (role != JIFFY_ENCODER && role != JIFFY_DECODER)) return JIFFY_ERR_INVALID_ARG;
  if (warps_per_cta > 8 || ctas_per_sm > 64 || items_per_ticket > 64) return JIFFY_ERR_INVALID_ARG;
  if (b->ws.pend.kind) return JIFFY_ERR_STATE;
  b->ws.fixed[role == JIFFY_ENCODER ? 0 : 1] = RowsLaunch{warps_per_cta, ctas_per_sm, items_per_ticket, 0};
  return JIFFY_OK;
}

jiffy_status jiffy_batch_info(const jiffy_batch* b, uint64_t* info, uint32_t n) {
  if (!b || (!info && n)) return JIFFY_ERR_INVALID_ARG;
  const Workspace& w = b->ws;
  const uint64_t v[9] = {w.calls, w.captures, w.replays, w.tunings, (uint64_t)w.tuned.size(),
                         w.last.wpc, w.last.ctas_per_sm, w.last.items_per_ticket, w.last.grid};
  for (uint32_t i = 0; i < n && i < 9; i++) info[i] = v[i];
  return JIFFY_OK;
}

jiffy_status jiffy_encode_batch_async(jiffy_batch* b, uint32_t n, jiffy_stream* const* streams,
                                      const uint32_t* n_scans, const void* const* const* planes, void* const* outs,
                                      const size_t* caps, uint64_t* const* frame_offsets, size_t* out_lens,
                                      jiffy_status* statuses, void* cuda_stream) {
  TraceRange trace("jiffy_encode_batch_async");
  if (!b || n == 0 || !streams || !n_scans || !planes || !outs || !caps || !out_lens || !statuses)
    return JIFFY_ERR_INVALID_ARG;
  DeviceGuard g(b->ws.device);
  if (!g.ok) return JIFFY_ERR_CUDA;
  std::vector<EncJob> jobs(n);
  for (uint32_t i = 0; i < n; i++)
    jobs[i] = EncJob{streams[i], n_scans[i], planes[i], outs[i], caps[i],
                     frame_offsets ? frame_offsets[i] : nullptr, &out_lens[i], &statuses[i]};
  return enqueue_encode(b->ws, jobs, reinterpret_cast<cudaStream_t>(cuda_stream));
}

jiffy_status jiffy_decode_batch_async(jiffy_batch* b, uint32_t n, jiffy_stream* const* streams,
                                      const uint32_t* n_frames, const void* const* ins, const size_t* in_lens,
                                      const uint64_t* const* frame_offsets, void* const* const* planes_out,
                                      jiffy_status* statuses, void* cuda_stream) {
  TraceRange trace("jiffy_decode_batch_async");
  if (!b || n == 0 || !streams || !n_frames || !ins || !in_lens || !frame_offsets || !planes_out || !statuses)
    return JIFFY_ERR_INVALID_ARG;
  DeviceGuard g(b->ws.device);
  if (!g.ok) return JIFFY_ERR_CUDA;
  std::vector<DecJob> jobs(n);
  for (uint32_t i = 0; i < n; i++)
    jobs[i] = DecJob{streams[i], n_frames[i], ins[i], in_lens[i], frame_offsets[i], planes_out[i], &statuses[i]};
  return enqueue_decode(b->ws, jobs, reinterpret_cast<cudaStream_t>(cuda_stream));
}

jiffy_status jiffy_batch_wait(jiffy_batch* b) {
  TraceRange trace("jiffy_batch_wait");
  if (!b) return JIFFY_ERR_INVALID_ARG;
  DeviceGuard g(b->ws.device);
  if (!g.ok) return JIFFY_ERR_CUDA;
  return finish(b->ws);
}

jiffy_status jiffy_encode_batch(jiffy_batch* b, uint32_t n, jiffy_stream* const* streams, const uint32_t* n_scans,
                                const void* const* const* planes, void* const* outs, const size_t* caps,
                                uint64_t* const* frame_offsets, size_t* out_lens, jiffy_status* statuses,
                                void* cuda_stream) {
  TraceRange trace("jiffy_encode_batch");
  const jiffy_status r = jiffy_encode_batch_async(b, n, streams, n_scans, planes, outs, caps, frame_offsets,
                                                  out_lens, statuses, cuda_stream);
  return r != JIFFY_OK ? r : jiffy_batch_wait(b);
}

jiffy_status jiffy_decode_batch(jiffy_batch* b, uint32_t n, jiffy_stream* const* streams, const uint32_t* n_frames,
                                const void* const* ins, const size_t* in_lens, const uint64_t* const* frame_offsets,
                                void* const* const* planes_out, jiffy_status* statuses, void* cuda_stream) {
  TraceRange trace("jiffy_decode_batch");
  const jiffy_status r = jiffy_decode_batch_async(b, n, streams, n_frames, ins, in_lens, frame_offsets, planes_out,
                                                  statuses, cuda_stream);
  return r != JIFFY_OK ? r : jiffy_batch_wait(b);
}

}  // extern "C"
