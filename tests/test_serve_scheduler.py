"""The serving loop's scheduler (continuous batching, HBM-budget admission,
one request in flight per sensor, decode after encode) on the CPU, driven by
a fake backend with a simulated clock. The GPU backend is exercised by the
GPU serving test."""
import numpy as np

from paper_2209_08196_gb300.serve import Request, Sensor, Server, poisson_arrivals


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-6  # every look at the clock costs a little time
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class FakeBackend:
    """Each context finishes its call `latency` seconds after submission."""

    def __init__(self, clock, n_contexts=2, latency=0.004, fail=(), max_group=4):
        self.clock, self.n_contexts, self.latency, self.max_group = clock, n_contexts, latency, max_group
        self.done_at = {}
        self.calls = []              # (kind, ctx, [(sid, seq)], t_submit)
        self.admitted, self.peak_used, self.used = set(), 0, 0
        self.fail = set(fail)        # (sid, seq) whose encode fails
        self.in_flight = {}

    def footprint(self, s):
        return s.H * s.W

    def reserve(self):
        return 0

    def admit(self, s):
        assert s.sid not in self.admitted
        self.admitted.add(s.sid)
        self.used += self.footprint(s)
        self.peak_used = max(self.peak_used, self.used)

    def release(self, s):
        self.admitted.remove(s.sid)
        self.used -= self.footprint(s)

    def _submit(self, kind, ctx, items, pairs):
        assert ctx not in self.in_flight, "context reused while busy"
        for sid, _ in items:
            assert sid in self.admitted
            for other in self.in_flight.values():
                assert sid not in [x for x, _ in other], "sensor in two contexts at once"
        assert len({sid for sid, _ in items}) == len(items), "sensor twice in one batch"
        self.in_flight[ctx] = items
        self.done_at[ctx] = self.clock.t + self.latency
        self.calls.append((kind, ctx, pairs, self.clock.t))

    def submit_encode(self, ctx, items):
        for sid, reqs in items:
            assert 1 <= len(reqs) <= self.max_group
            assert [r.seq for r in reqs] == list(range(reqs[0].seq, reqs[0].seq + len(reqs)))
            assert not any(r.decode for r in reqs[1:]), "a scan to decode must start its group"
        self._submit("encode", ctx, items, [(sid, r.seq) for sid, reqs in items for r in reqs])

    def submit_decode(self, ctx, items):
        self._submit("decode", ctx, items, [(sid, r.seq) for sid, r in items])

    def ready(self, ctx):
        return self.clock.t >= self.done_at[ctx]

    def finish_encode(self, ctx):
        items = self.in_flight.pop(ctx)
        return [([100] * len(reqs), 3 if any((sid, r.seq) in self.fail for r in reqs) else 0) for sid, reqs in items]

    def finish_decode(self, ctx):
        return [0 for _ in self.in_flight.pop(ctx)]


def _sensors(n, seed=0):
    rng = np.random.default_rng(seed)
    shapes = [(16, 1024), (64, 2048), (128, 4096)]
    out = []
    for i in range(n):
        H, W = shapes[rng.integers(len(shapes))]
        out.append(Sensor(i, H, W, [(4, 10)], float(rng.uniform(10, 20))))
    return out


def test_every_scan_served_once_in_order_with_decodes():
    clock = FakeClock()
    sensors = _sensors(20)
    reqs = poisson_arrivals(sensors, 2.0, 0.1, seed=1)
    be = FakeBackend(clock)
    st = Server(be, sensors, budget_bytes=1 << 40, clock=clock, sleep=clock.sleep).run(reqs, realtime=True)
    assert st.encoded == len(reqs) and st.failed == 0
    assert st.decoded == sum(r.decode for r in reqs) > 0
    seen = {}
    for kind, _, items, _ in be.calls:
        if kind == "encode":
            for sid, seq in items:
                assert seq == seen.get(sid, -1) + 1, "sensor %d out of order" % sid
                seen[sid] = seq
    # decodes come right after the encode of the same scan, on the same context
    for i, (kind, ctx, items, _) in enumerate(be.calls):
        if kind == "decode":
            enc = [c for c in be.calls[:i] if c[1] == ctx][-1]
            assert enc[0] == "encode" and set(items) <= set(enc[2])
    assert all(r.t_encoded >= r.t_arrival for r in reqs)
    s = st.summary()
    assert s["p50_ms"] <= s["p99_ms"]


def test_continuous_batching_overlaps_contexts_and_grows_batches():
    clock = FakeClock()
    sensors = _sensors(64, seed=2)
    reqs = poisson_arrivals(sensors, 1.0, 0.0, seed=3)
    be = FakeBackend(clock, latency=0.02)  # slow device: arrivals pile up
    st = Server(be, sensors, budget_bytes=1 << 40, clock=clock, sleep=clock.sleep).run(reqs, realtime=True)
    assert st.encoded == len(reqs)
    # both contexts were busy at the same time at some point
    busy = sorted((t, t + 0.02, ctx) for _, ctx, _, t in be.calls)
    assert any(a[2] != b[2] and b[0] < a[1] for a, b in zip(busy, busy[1:]))
    assert max(st.batch_sizes) > 1


def test_admission_respects_the_hbm_budget():
    clock = FakeClock()
    sensors = [Sensor(i, 64, 1024, [(4, 1)], 15.0) for i in range(12)]
    reqs = poisson_arrivals(sensors, 1.0, 0.2, seed=4)
    be = FakeBackend(clock)
    budget = 3 * 64 * 1024  # three sensors at a time
    st = Server(be, sensors, budget_bytes=budget, clock=clock, sleep=clock.sleep).run(reqs, realtime=False)
    assert be.peak_used <= budget
    assert st.encoded == len(reqs) and st.deferred > 0
    assert st.admitted == 12 and not be.admitted  # everyone served, memory given back


def test_sensor_that_never_fits_is_rejected_not_waited_for():
    clock = FakeClock()
    sensors = [Sensor(0, 16, 1024, [(4, 1)], 15.0), Sensor(1, 128, 4096, [(4, 1)], 15.0)]
    reqs = poisson_arrivals(sensors, 1.0, 0.0, seed=5)
    be = FakeBackend(clock)
    st = Server(be, sensors, budget_bytes=16 * 1024 * 4, clock=clock, sleep=clock.sleep).run(reqs, realtime=False)
    n1 = sum(r.sensor == 1 for r in reqs)
    assert st.rejected == n1 and st.encoded == len(reqs) - n1


def test_failed_encode_is_counted_and_does_not_stall():
    clock = FakeClock()
    sensors = _sensors(4, seed=6)
    reqs = poisson_arrivals(sensors, 0.5, 0.5, seed=7)
    bad = (reqs[0].sensor, reqs[0].seq)
    be = FakeBackend(clock, fail={bad})
    st = Server(be, sensors, budget_bytes=1 << 40, clock=clock, sleep=clock.sleep).run(reqs, realtime=True)
    # the failing scan's group fails with it; everything else is served
    assert st.failed >= 1 and st.encoded + st.failed == len(reqs)
    assert reqs[0].status == 3


def test_backlog_is_coded_in_groups_when_the_device_is_slow():
    # saturation: every scan is available at once; each batch takes up to
    # max_group queued scans per sensor (one segment), in order, with decode
    # scans only at the start of a group
    clock = FakeClock()
    sensors = _sensors(16, seed=9)
    reqs = poisson_arrivals(sensors, 2.0, 0.1, seed=10)
    be = FakeBackend(clock, latency=0.01, max_group=4)
    st = Server(be, sensors, budget_bytes=1 << 40, clock=clock, sleep=clock.sleep).run(reqs, realtime=False)
    assert st.encoded == len(reqs) and st.failed == 0
    assert st.decoded == sum(r.decode for r in reqs)
    s = st.summary()
    assert s["mean_group"] > 2.0
    seen = {}
    for kind, _, items, _ in be.calls:
        if kind == "encode":
            for sid, seq in items:
                assert seq == seen.get(sid, -1) + 1
                seen[sid] = seq
    # max_group = 1 keeps one scan per sensor per batch
    clock = FakeClock()
    be1 = FakeBackend(clock, latency=0.01, max_group=1)
    st1 = Server(be1, sensors, budget_bytes=1 << 40, clock=clock, sleep=clock.sleep).run(
        poisson_arrivals(sensors, 2.0, 0.1, seed=10), realtime=False)
    assert st1.encoded == len(reqs) and st1.summary()["mean_group"] == 1.0
    assert st1.batches > st.batches


class CachingBackend(FakeBackend):
    """Keeps a released sensor's memory for the next sensor of the same shape
    (as the GPU backend keeps its handles) and frees it when trimmed."""

    def __init__(self, clock, **kw):
        super().__init__(clock, **kw)
        self.cache = {}              # shape -> cached footprints
        self.cached = 0
        self.peak_held = 0           # admitted + cached
        self.reused = self.trimmed = 0

    def _held(self):
        self.peak_held = max(self.peak_held, self.used + self.cached)

    def admit(self, s):
        key = (s.H, s.W)
        if self.cache.get(key):
            self.cache[key].pop()
            self.cached -= self.footprint(s)
            self.reused += 1
        super().admit(s)
        self._held()

    def release(self, s):
        super().release(s)
        self.cache.setdefault((s.H, s.W), []).append(self.footprint(s))
        self.cached += self.footprint(s)
        self._held()

    def reusable(self, s):
        return bool(self.cache.get((s.H, s.W)))

    def trim(self, limit):
        for lst in self.cache.values():
            while lst and self.cached > limit:
                self.cached -= lst.pop()
                self.trimmed += 1


def test_cached_memory_counts_against_the_budget():
    # sensors come and go under a budget of three at a time; released memory
    # is cached for reuse, and the server trims the cache whenever a new
    # admission would otherwise exceed the budget
    clock = FakeClock()
    shapes = [(64, 1024), (32, 1024), (64, 2048)]
    sensors = [Sensor(i, *shapes[i % 3], [(4, 1)], 15.0) for i in range(12)]
    reqs = poisson_arrivals(sensors, 1.0, 0.1, seed=12)
    budget = 2 * 64 * 2048 + 64 * 1024
    be = CachingBackend(clock)
    st = Server(be, sensors, budget_bytes=budget, clock=clock, sleep=clock.sleep).run(reqs, realtime=False)
    assert st.encoded == len(reqs) and st.failed == 0
    assert be.peak_held <= budget
    assert be.reused > 0 and be.trimmed > 0 and st.deferred > 0


def test_arrivals_are_poisson_at_the_sensor_rates():
    sensors = [Sensor(i, 16, 1024, [(4, 1)], r) for i, r in enumerate([10.0, 20.0])]
    reqs = poisson_arrivals(sensors, 200.0, 0.1, seed=8)
    for s in sensors:
        t = np.array([r.t_arrival for r in reqs if r.sensor == s.sid])
        assert abs(len(t) / 200.0 - s.rate_hz) < 0.1 * s.rate_hz
        gaps = np.diff(t)
        assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1  # exponential gaps: CV = 1
    frac = np.mean([r.decode for r in reqs])
    assert 0.08 < frac < 0.12
    assert all(a.t_arrival <= b.t_arrival for a, b in zip(reqs, reqs[1:]))
    assert isinstance(reqs[0], Request)
