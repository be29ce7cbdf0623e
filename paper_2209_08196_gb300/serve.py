"""Serving loop: continuous batching of scans from many sensors.

Scans arrive from many simulated sensors (Poisson arrivals per sensor). The
server keeps each admitted sensor's encoder (and its decoder for decode
requests) on the device, so the previous scan used by P prediction
(Sec. III-D) never leaves HBM, and codes arrived scans in batched calls
(jiffy_encode_batch_async / jiffy_decode_batch_async): every scan in flight
shares the same kernel launches. Two batch contexts alternate on two CUDA
streams, so the host admits and marshals the next batch while the previous
one runs; scans that arrive while a batch is on the GPU join the next one as
soon as a context frees up (continuous batching, not a queue in front of a
single-scan codec).

Admission: a sensor is admitted on its first scan if its device footprint
(encoder and decoder state, output and decode buffers) fits the HBM budget
that the engine's fixed reserve leaves; otherwise its scans wait (counted as
deferred) until memory frees up.

Decode requests: a scan flagged for decode is decoded right after it is
encoded, from the encoder's state before that scan (copied into the
sensor's decoder first: encoder and decoder hold the same state, the
previous scan as decoded), so serving a decode needs no replay of the
sensor's earlier frames.

The scheduler is host logic over a backend; GpuBackend drives the C ABI.
Tests drive the scheduler with a fake backend on the CPU.
"""
from __future__ import annotations

import time
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
    batch_sizes: list = field(default_factory=list)
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

    backend interface:
      footprint(sensor) -> device bytes the sensor needs once admitted
      reserve() -> fixed device bytes of the engine (batch scratch)
      admit(sensor), release(sensor)
      n_contexts -> number of batch contexts that may be in flight
      submit_encode(ctx, [(sensor, request)]) ; ready(ctx) -> bool
      finish_encode(ctx) -> [(nbytes, status)] in submission order
      submit_decode(ctx, [(sensor, request)]) ; finish_decode(ctx) -> [status]
    """

    def __init__(self, backend, sensors, budget_bytes, max_batch=512, clock=time.perf_counter, sleep=time.sleep):
        self.be = backend
        self.sleep = sleep
        self.sensors = {s.sid: s for s in sensors}
        self.budget = budget_bytes
        self.max_batch = max_batch
        self.clock = clock
        self.used = backend.reserve()
        self.admitted = set()
        self.queue = {}           # sensor -> FIFO of requests
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
        self.be.admit(self.sensors[sid])
        self.used += need
        self.admitted.add(sid)
        self.stats.admitted += 1
        return True

    def _done(self, sid):
        """A request of sensor sid finished; a sensor with nothing left to
        serve gives its device memory back."""
        self.busy.discard(sid)
        self.remaining[sid] -= 1
        if self.remaining[sid] == 0 and sid in self.admitted:
            self.be.release(self.sensors[sid])
            self.used -= self.be.footprint(self.sensors[sid])
            self.admitted.discard(sid)

    def _ready_batch(self, now):
        batch = []
        for sid, q in self.queue.items():
            if not q or sid in self.busy:
                continue
            if not self._try_admit(sid):
                if self.be.footprint(self.sensors[sid]) > self.budget - self.be.reserve():
                    self.stats.rejected += len(q)  # never fits: its scans are turned away
                    self.remaining[sid] -= len(q)
                    q.clear()
                else:
                    self.stats.deferred += 1
                continue
            r = q[0]
            q.pop(0)
            r.t_admit = now
            batch.append((sid, r))
            if len(batch) >= self.max_batch:
                break
        return batch

    def _complete(self, ctx, now):
        kind, items = self.ctx_state.pop(ctx)
        if kind == "encode":
            res = self.be.finish_encode(ctx)
            decodes = []
            for (sid, r), (nbytes, status) in zip(items, res):
                r.nbytes, r.status = nbytes, status
                r.t_encoded = now
                if status != 0:
                    self.stats.failed += 1
                    self._done(sid)
                    continue
                s = self.sensors[sid]
                self.stats.encoded += 1
                self.stats.points += s.H * s.W
                self.stats.raw_bytes += s.H * s.W * sum(b for b, _ in s.attrs)
                self.stats.bytes_out += nbytes
                self.stats.enc_latency_ms.append((now - r.t_arrival) * 1e3)
                if r.decode:
                    decodes.append((sid, r))
                else:
                    self._done(sid)
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

    def run(self, requests, realtime=True, poll_sleep_s=0.0002):
        """Serves the requests (sorted by arrival). realtime: a request
        becomes available at its arrival time on the wall clock; otherwise
        all are available at once (saturation). Returns the statistics."""
        pending = list(requests)
        pending.reverse()
        for r in pending:
            self.remaining[r.sensor] = self.remaining.get(r.sensor, 0) + 1
        t0 = self.clock()
        free = list(range(self.be.n_contexts))
        while pending or any(self.queue.values()) or self.ctx_state:
            now = self.clock() - t0
            while pending and (not realtime or pending[-1].t_arrival <= now):
                r = pending.pop()
                if not realtime:
                    r.t_arrival = now
                self.queue.setdefault(r.sensor, []).append(r)
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
                self.stats.batch_sizes.append(len(batch))
                progressed = True
            if not progressed:
                if realtime and pending and not self.ctx_state and not any(self.queue.values()):
                    self.sleep(max(0.0, min(pending[-1].t_arrival - now, 0.002)))
                elif poll_sleep_s:
                    self.sleep(poll_sleep_s)
        self.stats.wall_s = self.clock() - t0
        return self.stats


class GpuBackend:
    """Backend over the C ABI: per sensor an encoder and a decoder stream,
    a one-frame output buffer and decode planes; scans drawn from per-class
    pools of device planes; n_contexts batch contexts on their own CUDA
    streams."""

    def __init__(self, pools, n_contexts=2, device=0, graphs=False, autotune=False, max_batch_px=None,
                 keep=False):
        import torch

        from paper_2209_08196_gb300 import jiffy as J
        self.J, self.torch = J, torch
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
        self.events = [None] * n_contexts
        self.max_batch_px = max_batch_px or 0
        self.s = {}                 # sensor id -> dict of handles and buffers
        self.n_decode = [0] * n_contexts
        self.items = [None] * n_contexts
        self.keep = keep            # copy every frame and decoded scan to the host (tests)
        self.frames = {}            # (sensor, seq) -> bytes
        self.decoded = {}           # (sensor, seq) -> [numpy planes]

    @staticmethod
    def sensor_bytes(sensor):
        raw = sensor.H * sensor.W * sum(b for b, _ in sensor.attrs)
        from paper_2209_08196_gb300 import jiffy as J
        out = J.jiffy_max_encoded_size(sensor.H, sensor.W, sensor.attrs, 1)
        # encoder + decoder state (two planes sets each), output bound, decode planes
        return 4 * raw + out + raw

    def footprint(self, sensor):
        return self.sensor_bytes(sensor)

    def reserve(self):
        # batch scratch of each context: row slots (about the row bound per
        # row) plus work arrays, for the largest batch expected
        return self.n_contexts * 3 * self.max_batch_px * 13

    def admit(self, sensor):
        J, torch = self.J, self.torch
        enc = J.jiffy_stream_create(J.JIFFY_ENCODER, sensor.H, sensor.W, sensor.attrs, device=self.device)
        dec = J.jiffy_stream_create(J.JIFFY_DECODER, sensor.H, sensor.W, sensor.attrs, device=self.device)
        out = torch.empty(J.jiffy_max_encoded_size(sensor.H, sensor.W, sensor.attrs, 1), dtype=torch.uint8,
                          device="cuda:%d" % self.device)
        planes = J.empty_planes(dec)
        self.s[sensor.sid] = {"enc": enc, "dec": dec, "out": out, "planes": planes, "sensor": sensor}

    def release(self, sensor):
        self.s.pop(sensor.sid, None)

    def scan(self, sensor, seq):
        pool = self.pools[sensor.pool]
        return pool[(sensor.pool_offset + seq) % len(pool)]

    def submit_encode(self, ctx, batch):
        J = self.J
        st = self.streams[ctx]
        with self.torch.cuda.stream(st):
            for sid, r in batch:
                if r.decode:
                    d = self.s[sid]
                    J.jiffy_stream_copy_state(d["dec"], d["enc"], stream=st)
            J.jiffy_encode_batch_async(self.batches[ctx], [self.s[sid]["enc"] for sid, _ in batch],
                                       [[self.scan(self.s[sid]["sensor"], r.seq)] for sid, r in batch],
                                       [self.s[sid]["out"] for sid, _ in batch], stream=st)
            ev = self.torch.cuda.Event()
            ev.record(st)
        self.events[ctx] = ev
        self.items[ctx] = batch

    def ready(self, ctx):
        return self.events[ctx] is None or self.events[ctx].query()

    def finish_encode(self, ctx):
        J = self.J
        try:
            res = J.jiffy_batch_wait(self.batches[ctx])
            out = [(n, 0) for n, _ in res]
        except J.BatchError as e:
            out = [((e.required or [0] * len(e.statuses))[i], st) for i, st in enumerate(e.statuses)]
        self.events[ctx] = None
        if self.keep:
            for (sid, r), (n, st) in zip(self.items[ctx], out):
                if st == 0:
                    self.frames[(sid, r.seq)] = self.s[sid]["out"][:n].cpu().numpy().tobytes()
        return out

    def submit_decode(self, ctx, items):
        J = self.J
        st = self.streams[ctx]
        handles, bufs, lens, offs, planes = [], [], [], [], []
        for sid, r in items:
            d = self.s[sid]
            # the stream header precedes frame 0
            first = 16 + 8 * len(d["sensor"].attrs) if J.jiffy_stream_frame_index(d["dec"]) == 0 else 0
            handles.append(d["dec"])
            bufs.append(d["out"])
            lens.append(r.nbytes)
            offs.append([first, r.nbytes])
            planes.append([p.unsqueeze(0) for p in d["planes"]])
        with self.torch.cuda.stream(st):
            J.jiffy_decode_batch_async(self.batches[ctx], handles, bufs, lens, offs, planes, stream=st)
            ev = self.torch.cuda.Event()
            ev.record(st)
        self.events[ctx] = ev
        self.n_decode[ctx] = len(items)
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
