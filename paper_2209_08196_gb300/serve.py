"""Serving loop: continuous batching of scans from many sensors.

Scans arrive from many simulated sensors (Poisson arrivals per sensor). The
server keeps each admitted sensor's encoder (and its decoder for decode
requests) on the device, so the previous scan used by P prediction
(Sec. III-D) never leaves HBM, and codes arrived scans in batched calls
(jiffy_encode_batch_async / jiffy_decode_batch_async): every scan in flight
shares the same kernel launches, and a sensor with a backlog puts up to
max_group of its queued scans into one batch as one segment (consecutive
scans of one stream in one call), so the work per launch sequence grows with
the load. Two batch contexts alternate on two CUDA streams, so the host
admits and marshals the next batch while the previous one runs; scans that
arrive while a batch is on the GPU join the next one as soon as a context
frees up (continuous batching, not a queue in front of a single-scan codec).

Admission: a sensor is admitted on its first scan if its device footprint
(encoder and decoder state, output and decode buffers) fits the HBM budget
that the engine's fixed reserve leaves; otherwise its scans wait (counted as
deferred) until memory frees up.

Decode requests: a scan flagged for decode is decoded right after it is
encoded, from the encoder's state before that scan (copied into the
sensor's decoder first: encoder and decoder hold the same state, the
previous scan as decoded), so serving a decode needs no replay of the
sensor's earlier frames. Such a scan therefore always starts its group.

The scheduler is host logic over a backend; GpuBackend drives the C ABI.
Tests drive the scheduler with a fake backend on the CPU.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Sensor:
    sid: int
    H: int
    W: int
    attrs: list              # [(bytes per sample, precision)]
    rate_hz: float
    pool: int = 0            # index of the scan pool it draws from
    pool_offset: int = 0


@dataclass
class Request:
    sensor: int
    seq: int                 # scan number within the sensor
    t_arrival: float         # seconds from the start
    decode: bool = False
    t_admit: float | None = None
    t_encoded: float | None = None
    t_decoded: float | None = None
    nbytes: int = 0
    status: int = 0


def poisson_arrivals(sensors, duration_s, decode_frac, seed):
    """Per-sensor Poisson arrivals over [0, duration_s); each scan is flagged
    for decode with probability decode_frac. Returns requests by time."""
    rng = np.random.default_rng(seed)
    reqs = []
    for s in sensors:
        t, k = 0.0, 0
        while True:
            t += rng.exponential(1.0 / s.rate_hz)
            if t >= duration_s:
                break
            reqs.append(Request(s.sid, k, t, bool(rng.random() < decode_frac)))
            k += 1
    reqs.sort(key=lambda r: (r.t_arrival, r.sensor))
    return reqs


@dataclass
class Stats:
    encoded: int = 0
    decoded: int = 0
    points: int = 0           # pixels encoded
    decoded_points: int = 0
    bytes_out: int = 0
    raw_bytes: int = 0
    batches: int = 0
    segments: int = 0         # sensor groups over all batches
    batch_sizes: list = field(default_factory=list)   # scans per batch
    deferred: int = 0         # scan-waits caused by the HBM budget
    rejected: int = 0         # scans of sensors that can never fit the budget
    admitted: int = 0
    failed: int = 0
    wall_s: float = 0.0
    enc_latency_ms: list = field(default_factory=list)
    dec_latency_ms: list = field(default_factory=list)

    def summary(self):
        def pct(v, q):
            return float(np.percentile(v, q)) if v else None
        return {
            "scans_encoded": self.encoded, "scans_decoded": self.decoded, "batches": self.batches,
            "mean_batch": float(np.mean(self.batch_sizes)) if self.batch_sizes else 0.0,
            "mean_group": float(np.sum(self.batch_sizes)) / self.segments if self.segments else 0.0,
            "sensors_admitted": self.admitted, "deferred_waits": self.deferred, "rejected": self.rejected,
            "failed": self.failed,
            "wall_s": self.wall_s,
            "gpoints_s": (self.points + self.decoded_points) / self.wall_s / 1e9 if self.wall_s else None,
            "encode_gpoints_s": self.points / self.wall_s / 1e9 if self.wall_s else None,
            "ratio": self.raw_bytes / self.bytes_out if self.bytes_out else None,
            "p50_ms": pct(self.enc_latency_ms, 50), "p99_ms": pct(self.enc_latency_ms, 99),
            "decode_p50_ms": pct(self.dec_latency_ms, 50), "decode_p99_ms": pct(self.dec_latency_ms, 99),
        }


class Server:
    """Continuous-batching scheduler over a backend.

    A batch holds at most one group per sensor: the sensor's queued scans in
    order, up to max_group of them (one segment of the batched call, so a
    backlog is coded in one launch sequence), and a scan flagged for decode
    only ever starts a group, so its decode is frame 0 of the group.

    backend interface:
      footprint(sensor) -> device bytes the sensor needs once admitted
      reserve() -> fixed device bytes of the engine (batch scratch)
      admit(sensor), release(sensor); optional trim(limit_bytes): give back
        cached memory beyond limit_bytes, and reusable(sensor): admitting the
        sensor reuses cached memory (needs none new)
      n_contexts -> number of batch contexts that may be in flight
      max_group -> most scans of one sensor per batch (optional, default 1)
      submit_encode(ctx, [(sensor, [requests])]) ; ready(ctx) -> bool
      finish_encode(ctx) -> [([nbytes per request], status)] in submission order
      submit_decode(ctx, [(sensor, request)]) -> decode of the request's
        frame, the first of its group ; finish_decode(ctx) -> [status]
    """

    def __init__(self, backend, sensors, budget_bytes, max_batch=512, max_group=None, clock=time.perf_counter,
                 sleep=time.sleep):
        self.be = backend
        self.sleep = sleep
        self.sensors = {s.sid: s for s in sensors}
        self.budget = budget_bytes
        self.max_batch = max_batch      # sensors (segments) per batch
        # consecutive queued scans of one sensor coded as one segment of a batch
        self.max_group = max_group or getattr(backend, "max_group", 1)
        self.clock = clock
        self.used = backend.reserve()
        self.admitted = set()
        self.queue = {}           # sensor -> FIFO of requests
        self.ready = {}           # sensors with queued requests and none in flight, in arrival order
        self.busy = set()         # sensors with a request in flight
        self.ctx_state = {}       # ctx -> ("encode"|"decode", [(sensor, request)])
        self.remaining = {}       # sensor -> requests not yet finished
        self.stats = Stats()

    def _try_admit(self, sid):
        if sid in self.admitted:
            return True
        need = self.be.footprint(self.sensors[sid])
        if self.used + need > self.budget:
            return False
        trim = getattr(self.be, "trim", None)
        reusable = getattr(self.be, "reusable", None)
        if trim is not None and not (reusable is not None and reusable(self.sensors[sid])):
            # memory the backend keeps from released sensors counts against the
            # budget: a sensor that cannot reuse some of it makes room first
            trim(self.budget - self.used - need)
        self.be.admit(self.sensors[sid])
        self.used += need
        self.admitted.add(sid)
        self.stats.admitted += 1
        return True

    def _done(self, sid, k=1, free=True):
        """k requests of sensor sid finished (free: nothing of it is in flight
        any more); a sensor with nothing left to serve gives its device
        memory back."""
        if free:
            self.busy.discard(sid)
            if self.queue.get(sid):
                self.ready[sid] = None
        self.remaining[sid] -= k
        if self.remaining[sid] == 0 and sid in self.admitted:
            self.be.release(self.sensors[sid])
            self.used -= self.be.footprint(self.sensors[sid])
            self.admitted.discard(sid)

    def _ready_batch(self, now):
        batch = []
        taken = []
        for sid in self.ready:
            q = self.queue[sid]
            if not self._try_admit(sid):
                if self.be.footprint(self.sensors[sid]) > self.budget - self.be.reserve():
                    self.stats.rejected += len(q)  # never fits: its scans are turned away
                    self.remaining[sid] -= len(q)
                    q.clear()
                    taken.append(sid)
                else:
                    self.stats.deferred += 1
                continue
            # the sensor's backlog, up to max_group scans; a scan to be decoded
            # only ever starts a group (its decoder takes the state before it)
            reqs = [q.popleft()]
            while q and len(reqs) < self.max_group and not q[0].decode:
                reqs.append(q.popleft())
            for r in reqs:
                r.t_admit = now
            batch.append((sid, reqs))
            taken.append(sid)
            if len(batch) >= self.max_batch:
                break
        for sid in taken:
            del self.ready[sid]
        return batch

    def _complete(self, ctx, now):
        kind, items = self.ctx_state.pop(ctx)
        if kind == "encode":
            res = self.be.finish_encode(ctx)
            decodes = []
            for (sid, reqs), (sizes, status) in zip(items, res):
                if status != 0:
                    for r in reqs:
                        r.status, r.t_encoded = status, now
                    self.stats.failed += len(reqs)
                    self._done(sid, len(reqs))
                    continue
                s = self.sensors[sid]
                for r, nbytes in zip(reqs, sizes):
                    r.nbytes, r.status, r.t_encoded = nbytes, 0, now
                    self.stats.enc_latency_ms.append((now - r.t_arrival) * 1e3)
                    self.stats.bytes_out += nbytes
                self.stats.encoded += len(reqs)
                self.stats.points += s.H * s.W * len(reqs)
                self.stats.raw_bytes += s.H * s.W * sum(b for b, _ in s.attrs) * len(reqs)
                if reqs[0].decode:
                    decodes.append((sid, reqs[0]))
                    self._done(sid, len(reqs) - 1, free=False)
                else:
                    self._done(sid, len(reqs))
            if decodes:
                self.be.submit_decode(ctx, decodes)
                self.ctx_state[ctx] = ("decode", decodes)
        else:
            res = self.be.finish_decode(ctx)
            for (sid, r), status in zip(items, res):
                r.t_decoded = now
                self._done(sid)
                if status != 0:
                    self.stats.failed += 1
                    continue
                s = self.sensors[sid]
                self.stats.decoded += 1
                self.stats.decoded_points += s.H * s.W
                self.stats.dec_latency_ms.append((now - r.t_arrival) * 1e3)

    def run(self, requests, realtime=True, poll_sleep_s=0.0):
        """Serves the requests (sorted by arrival). realtime: a request
        becomes available at its arrival time on the wall clock; otherwise
        all are available at once (saturation). poll_sleep_s: pause when a
        pass made no progress while work is on the device (0: poll without
        pausing, the lowest latency; the loop then keeps one host core
        busy). Returns the statistics."""
        pending = list(requests)
        pending.reverse()
        for r in pending:
            self.remaining[r.sensor] = self.remaining.get(r.sensor, 0) + 1
        t0 = self.clock()
        free = list(range(self.be.n_contexts))
        while pending or self.ready or self.ctx_state:
            now = self.clock() - t0
            while pending and (not realtime or pending[-1].t_arrival <= now):
                r = pending.pop()
                if not realtime:
                    r.t_arrival = now
                q = self.queue.get(r.sensor)
                if q is None:
                    q = self.queue[r.sensor] = deque()
                q.append(r)
                if r.sensor not in self.busy:
                    self.ready[r.sensor] = None
            progressed = False
            for ctx in list(self.ctx_state):
                if self.be.ready(ctx):
                    self._complete(ctx, self.clock() - t0)
                    if ctx not in self.ctx_state:
                        free.append(ctx)
                    progressed = True
            while free:
                batch = self._ready_batch(self.clock() - t0)
                if not batch:
                    break
                ctx = free.pop()
                for sid, _ in batch:
                    self.busy.add(sid)
                self.be.submit_encode(ctx, batch)
                self.ctx_state[ctx] = ("encode", batch)
                self.stats.batches += 1
                self.stats.batch_sizes.append(sum(len(reqs) for _, reqs in batch))
                self.stats.segments += len(batch)
                progressed = True
            if not progressed:
                if realtime and pending and not self.ctx_state and not self.ready:
                    self.sleep(max(0.0, min(pending[-1].t_arrival - now, 0.002)))
                elif poll_sleep_s:
                    self.sleep(poll_sleep_s)
        self.stats.wall_s = self.clock() - t0
        return self.stats


class GpuBackend:
    """Backend over the C ABI: per admitted sensor an encoder and a decoder
    stream, a one-frame output buffer and decode planes; scans drawn from
    per-class pools of device planes; n_contexts batch contexts on their own
    CUDA streams.

    Host cost per batch is kept to a few array operations: the plane pointer
    tables of every pool scan and of every sensor's decode planes are built
    once, and a batch is marshalled as numpy arrays of addresses
    (jiffy_*_batch_async_arrays). A released sensor's handles and buffers are
    kept for the next sensor of the same shape and attribute set (reset, not
    freed: freeing device memory waits for the whole device); the server
    hands cached memory back whenever the HBM budget needs it (trim)."""

    def __init__(self, pools, n_contexts=2, device=0, graphs=False, autotune=False, max_batch_px=None,
                 keep=False, max_group=8):
        import ctypes

        import torch

        from paper_2209_08196_gb300 import jiffy as J
        self.J, self.torch, self.ctypes = J, torch, ctypes
        self.pools = pools          # pool index -> list of scans (lists of device planes)
        self.device = device
        self.n_contexts = n_contexts
        self.batches = [J.jiffy_batch_create(device) for _ in range(n_contexts)]
        for b in self.batches:
            if graphs:
                J.jiffy_batch_set_graphs(b, True)
            if autotune:
                J.jiffy_batch_set_autotune(b, True)
        self.streams = [torch.cuda.Stream(device=device) for _ in range(n_contexts)]
        self.stream_ptrs = [st.cuda_stream for st in self.streams]
        self.events = [None] * n_contexts
        self.max_batch_px = max_batch_px or 0
        self.max_group = max_group
        # plane pointer table of each pool, its scans repeated so that any
        # max_group consecutive scans (modulo the pool) are one contiguous run
        self.pool_tables = []
        for pool in pools:
            L = len(pool)
            self.pool_tables.append(J.plane_table([p for k in range(L * (1 + -(-max_group // L)))
                                                   for p in pool[k % L]]))
        self.checked_pools = set()
        self.s = {}                 # sensor id -> slot (handles, buffers, addresses)
        self.free = {}              # (H, W, attrs) -> released slots
        self.cached_bytes = 0
        self._fp = {}               # (H, W, attrs) -> footprint
        self.n_decode = [0] * n_contexts
        self.items = [None] * n_contexts
        self.last = [None] * n_contexts   # frame offsets of the context's last encode
        self.keep = keep            # copy every frame and decoded scan to the host (tests)
        self.frames = {}            # (sensor, seq) -> bytes
        self.decoded = {}           # (sensor, seq) -> [numpy planes]

    @staticmethod
    def sensor_bytes(sensor, max_group=1):
        raw = sensor.H * sensor.W * sum(b for b, _ in sensor.attrs)
        from paper_2209_08196_gb300 import jiffy as J
        out = J.jiffy_max_encoded_size(sensor.H, sensor.W, sensor.attrs, max_group)
        # encoder + decoder state (two planes sets each), output bound of a group, decode planes
        return 4 * raw + out + raw

    def footprint(self, sensor):
        k = self._key(sensor)
        fp = self._fp.get(k)
        if fp is None:
            fp = self._fp[k] = self.sensor_bytes(sensor, self.max_group)
        return fp

    def reserve(self):
        # batch scratch of each context: row slots (about the row bound per
        # row) plus work arrays, for the largest batch expected
        return self.n_contexts * 3 * self.max_batch_px * 13

    @staticmethod
    def _key(sensor):
        return sensor.H, sensor.W, tuple(tuple(a) for a in sensor.attrs)

    def _check_pool(self, sensor):
        if sensor.pool in self.checked_pools:
            return
        for scan in self.pools[sensor.pool]:
            if len(scan) != len(sensor.attrs):
                raise ValueError("pool %d: scans have %d planes, sensor %d has %d attributes"
                                 % (sensor.pool, len(scan), sensor.sid, len(sensor.attrs)))
            for k, (p, (b, _)) in enumerate(zip(scan, sensor.attrs)):
                self.J._check_plane(p, sensor.H, sensor.W, b, "pool %d plane %d" % (sensor.pool, k))
        self.checked_pools.add(sensor.pool)

    def admit(self, sensor):
        J, torch = self.J, self.torch
        self._check_pool(sensor)
        cached = self.free.get(self._key(sensor))
        if cached:
            d = cached.pop()
            self.cached_bytes -= d["bytes"]
            J.jiffy_stream_reset(d["enc"])
            J.jiffy_stream_reset(d["dec"])
        else:
            enc = J.jiffy_stream_create(J.JIFFY_ENCODER, sensor.H, sensor.W, sensor.attrs, device=self.device)
            dec = J.jiffy_stream_create(J.JIFFY_DECODER, sensor.H, sensor.W, sensor.attrs, device=self.device)
            out = torch.empty(J.jiffy_max_encoded_size(sensor.H, sensor.W, sensor.attrs, self.max_group),
                              dtype=torch.uint8, device="cuda:%d" % self.device)
            planes = J.empty_planes(dec)
            dtab = J.plane_table(planes)
            d = {"enc": enc, "dec": dec, "out": out, "planes": planes, "dtab": dtab, "enc_ptr": enc.ptr,
                 "dec_ptr": dec.ptr, "out_ptr": out.data_ptr(), "cap": out.numel(),
                 "dtab_addr": self.ctypes.addressof(dtab), "bytes": self.footprint(sensor),
                 "hdr": 16 + 8 * len(sensor.attrs)}
        d["sensor"] = sensor
        d["pbase"] = self.ctypes.addressof(self.pool_tables[sensor.pool])
        d["pstride"] = 8 * len(sensor.attrs)   # bytes of one scan's pointers
        d["plen"] = len(self.pools[sensor.pool])
        self.s[sensor.sid] = d
        return d

    def reusable(self, sensor):
        return bool(self.free.get(self._key(sensor)))

    def release(self, sensor):
        d = self.s.pop(sensor.sid, None)
        if d is not None:
            self.free.setdefault(self._key(sensor), []).append(d)
            self.cached_bytes += d["bytes"]

    def trim(self, limit_bytes):
        """Frees cached handles and buffers until at most limit_bytes stay
        cached."""
        for lst in self.free.values():
            while lst and self.cached_bytes > limit_bytes:
                d = lst.pop()
                self.cached_bytes -= d["bytes"]
                self.J.jiffy_stream_destroy(d["enc"])
                self.J.jiffy_stream_destroy(d["dec"])
                d.clear()

    def scan(self, sensor, seq):
        pool = self.pools[sensor.pool]
        return pool[(sensor.pool_offset + seq) % len(pool)]

    def submit_encode(self, ctx, batch):
        J = self.J
        sp = self.stream_ptrs[ctx]
        rows = []
        for sid, reqs in batch:
            if len(reqs) > self.max_group:  # the pool tables hold max_group consecutive scans
                raise ValueError("a group of %d scans exceeds max_group = %d" % (len(reqs), self.max_group))
            d = self.s[sid]
            if reqs[0].decode:  # the decoder takes the encoder's state before this group
                J.jiffy_stream_copy_state(d["dec"], d["enc"], stream=sp)
            k = (d["sensor"].pool_offset + reqs[0].seq) % d["plen"]
            rows.append((d["enc_ptr"], d["pbase"] + d["pstride"] * k, d["out_ptr"], d["cap"], len(reqs)))
        a = np.array(rows, dtype=np.uint64).reshape(-1, 5)
        J.jiffy_encode_batch_async_arrays(self.batches[ctx], a[:, 0], a[:, 4], a[:, 1], a[:, 2], a[:, 3], stream=sp)
        ev = self.torch.cuda.Event()
        ev.record(self.streams[ctx])
        self.events[ctx] = ev
        self.items[ctx] = batch

    def ready(self, ctx):
        return self.events[ctx] is None or self.events[ctx].query()

    def finish_encode(self, ctx):
        J = self.J
        batch = self.items[ctx]
        self.events[ctx] = None
        try:
            _, offs, starts = J.jiffy_batch_wait(self.batches[ctx])
            sts = [0] * len(batch)
        except J.BatchError as e:  # the other streams of the batch succeeded and advanced
            if e.result is None:
                return [([0] * len(reqs), st) for (_, reqs), st in zip(batch, e.statuses)]
            _, offs, starts = e.result
            sts = e.statuses
        o = offs.astype(np.int64)
        out = []
        for (sid, reqs), s0, st in zip(batch, starts.tolist(), sts):
            if st != 0:
                out.append(([0] * len(reqs), st))
                continue
            f = o[s0:s0 + len(reqs) + 1].copy()
            f[0] = 0  # the first frame's bytes include the stream header when there is one
            out.append((np.diff(f).tolist(), 0))
            if self.keep:
                buf = self.s[sid]["out"][:int(f[-1])].cpu().numpy().tobytes()
                for t, r in enumerate(reqs):
                    self.frames[(sid, r.seq)] = buf[int(f[t]):int(f[t + 1])]
        self.last[ctx] = (o, dict(zip((sid for sid, _ in batch), starts.tolist())))
        return out

    def submit_decode(self, ctx, items):
        J = self.J
        o, start = self.last[ctx]
        rows = []
        for sid, r in items:
            d = self.s[sid]
            s0 = start[sid]
            # frame 0 of the sensor's group: from its offset (after the stream
            # header on a stream's first frame) to the next
            rows.append((d["dec_ptr"], d["out_ptr"], o[s0 + 1], d["dtab_addr"], o[s0], o[s0 + 1]))
        a = np.array(rows, dtype=np.uint64).reshape(-1, 6)
        n = len(rows)
        J.jiffy_decode_batch_async_arrays(self.batches[ctx], a[:, 0], np.ones(n, np.uint32), a[:, 1], a[:, 2],
                                          a[:, 4:6].reshape(-1), np.arange(n, dtype=np.int64) * 2, a[:, 3],
                                          stream=self.stream_ptrs[ctx])
        ev = self.torch.cuda.Event()
        ev.record(self.streams[ctx])
        self.events[ctx] = ev
        self.n_decode[ctx] = n
        self.items[ctx] = items

    def finish_decode(self, ctx):
        J = self.J
        self.events[ctx] = None
        try:
            J.jiffy_batch_wait(self.batches[ctx])
            res = [0] * self.n_decode[ctx]
        except J.BatchError as e:
            res = list(e.statuses)
        if self.keep:
            for (sid, r), st in zip(self.items[ctx], res):
                if st == 0:
                    self.decoded[(sid, r.seq)] = [p.cpu().clone() for p in self.s[sid]["planes"]]
        return res
