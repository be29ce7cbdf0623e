"""Benchmark of the Jiffy GB300 codec: encode + decode throughput.

Workload (one step): one sensor stream of 100 scans of 128 x 2048 pixels with
five attribute planes -- range and second-return range (uint32 mm, 10 mm
precision), signal (uint16), reflectivity (uint8) and ambient (uint16) -- all
scans encoded in one pass (jiffy_encode_seq) and decoded in one pass
(jiffy_decode_seq); 341 MB of raw samples, larger than the 129 MB L2, so no
flush is needed between steps. Synthetic, seeded scans stand in for the
paper's driving datasets (Sec. IV-B).

Prints one JSON line. value = pixels encoded and decoded per second (Gpoints/s)
with inputs resident in HBM; e2e = the same through host buffers (H2D of the
scans and of the stream, D2H of the stream and of the decoded scans inside
the timed region); roofline = the dominant kernel's algorithmic bytes
(bytes in + bytes out) per launch over its CUDA-event duration against the
measured HBM copy bandwidth; cpu_baseline = the oracle on host cores on a
bounded sample of the same scans.

Further legs, each in its own key (compact copies of their headline figures
sit inside `roofline` and `e2e`): the small single-stream case (16 scans of
64 x 1024, CUDA-graph replay), the stream-size sweep of the low-coherence
workload (64 MiB to 4 GiB of raw planes), the many-stream batch, the serving
loop, the trial heuristic against brute force, the precision sweep, the
ablated codecs and point-cloud standardization.

--impl reference times the oracle alone (the reference arm).
Multi-GPU (torchrun): independent replicas, one stream per GPU, no collective
on the data path; value = all ranks' pixels / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Encode+decode Gpoints/s vs HBM roofline (bit-exact); served p50/p99 scan latency"
UNIT = "Gpoints/s"
WORKLOAD = ("single stream, 100 scans x 128 beams x 2048 columns; range u32 (10 mm), range2 u32 (10 mm), "
            "signal u16, reflectivity u8, ambient u16")


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# each rows kernel on the default workload (100 scans of 128 x 2048, five
# attributes), from a single-pass ncu capture of the full-size launch. It holds
# only for the kernel sources it was taken on (sha256 prefix of the files
# listed) and is reported as null for any other source or workload.
TRAFFIC = {
    "k_encode": (343708672 + 53618432, ("jiffy_encode.cu", "jiffy_device.cuh", "jiffy_kernels.h", "jiffy_types.h"),
                 "516bf26415d088ed"),
    "k_decode": (78800640 + 292559872, ("jiffy_decode.cu", "jiffy_device.cuh", "jiffy_kernels.h", "jiffy_types.h"),
                 "6c08fca6995251b8"),
}


def traffic(kernel: str, scans: int):
    import hashlib
    if kernel not in TRAFFIC or scans != 100:
        return None
    nbytes, files, digest = TRAFFIC[kernel]
    m = hashlib.sha256()
    try:
        for f in files:
            with open(os.path.join(ROOT, "paper_2209_08196_gb300", "csrc", f), "rb") as fh:
                m.update(fh.read())
    except OSError:
        return None
    return nbytes if m.hexdigest()[:16] == digest else None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Samples the SM clock and the clock event (throttle) reasons during a
    region: NVML read through ctypes from a background thread every 5 ms
    (reads only; nothing is set), else nvidia-smi every 200 ms."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, device_index: int):
        self.dev = device_index
        self.samples = []
        self.smax = None
        self.mode = None
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), "jiffy_bench_clocks_%d_rank%d.csv" % (os.getpid(), device_index))

    def _nvml(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        h = ctypes.c_void_p()
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.dev), ctypes.byref(h)) != 0:
            raise OSError("no NVML handle")
        fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0:
            self.smax = float(mx.value)
        return lib, h, fn

    def start(self):
        import threading
        try:
            lib, h, fn = self._nvml()
            import ctypes
            self.stop_flag = threading.Event()

            def loop():
                mhz, rs = ctypes.c_uint(), ctypes.c_ulonglong()
                while not self.stop_flag.is_set():
                    if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(mhz)) == 0 and \
                            fn(h, ctypes.byref(rs)) == 0:
                        self.samples.append((float(mhz.value), int(rs.value)))
                    time.sleep(0.005)
            self.thread = threading.Thread(target=loop, daemon=True)
            self.thread.start()
            self.mode = "nvml"
            return
        except Exception:
            pass
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            self.mode = "nvidia-smi"
        except Exception:
            self.proc = None

    def stop(self):
        if self.mode == "nvml":
            self.stop_flag.set()
            self.thread.join()
            sm = [m for m, _ in self.samples]
            reasons = sorted({n for _, r in self.samples for bit, n in self.REASONS.items() if r & bit})
            smax = self.smax
        elif self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()
            sm, mx, rset = [], [], set()
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        rset.add(n)
            reasons, smax = sorted(rset), (max(mx) if mx else None)
        else:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no clock reader"]}
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": smax, "reasons": ["no samples"]}
        loaded = [x for x in sm if x >= 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(sm), "source": self.mode}


def make_workload(device: str, seed: int, n_scans: int = 100):
    from paper_2209_08196_gb300 import synth
    cfg = synth.config_multi_attr(seed=seed, n_scans=n_scans)
    seq = synth.ScanSequence(cfg, device=device)
    scans = [seq.scan(t, as_numpy=False) for t in range(cfg.n_scans)]
    return cfg, synth.attr_descs(cfg), scans


def cpu_baseline(cfg, attrs, scans, budget_s: float = 12.0):
    """The oracle, as it stands, single-threaded, on the first scans of the
    same workload: encode + decode until about budget_s of CPU work."""
    import numpy as np
    import oracle
    DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}
    enc = oracle.Codec(cfg.H, cfg.W, attrs)
    dec = oracle.Codec(cfg.H, cfg.W, attrs)
    n_scans, t_enc, t_dec = 0, 0.0, 0.0
    for t, planes in enumerate(scans):
        host = [p.cpu().numpy().view(DT[s]) for p, (s, _) in zip(planes, attrs)]
        t0 = time.perf_counter()
        b = enc.encode(host)
        t1 = time.perf_counter()
        dec.decode(b)
        t2 = time.perf_counter()
        t_enc += t1 - t0
        t_dec += t2 - t1
        n_scans += 1
        if t_enc + t_dec >= budget_s:
            break
    px = n_scans * cfg.H * cfg.W
    return {"value": px / (t_enc + t_dec) / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "first %d of the %d scans, encode + decode, single-threaded plain C" % (n_scans, len(scans)),
            "encode_mpoints_s": px / t_enc / 1e6, "decode_mpoints_s": px / t_dec / 1e6}


def _oracle_worker(conn, start, H, W, attrs, repeats):
    """One host core of the N-core oracle figure: receives its scans (an
    independent stream), waits for the start signal, encodes + decodes them
    `repeats` times, reports the busy time."""
    import oracle
    scans = conn.recv()
    enc = oracle.Codec(H, W, attrs)
    dec = oracle.Codec(H, W, attrs)
    dec.decode(enc.encode(scans[0]))  # load the library, touch the pages
    conn.send("ready")
    start.wait()
    t0 = time.perf_counter()
    for _ in range(repeats):
        enc.reset()
        dec.reset()
        for planes in scans:
            dec.decode(enc.encode(planes))
    conn.send(time.perf_counter() - t0)
    conn.close()


def cpu_baseline_configs(budget_s: float = 4.0):
    """The oracle, single-threaded, on the small single-stream case (16 x
    64x1024 range at 10 mm) and on the low-coherence case (128x2048 range at
    1 mm + reflectivity, 40 % zeros in discs): scans generated on the host,
    encode then decode of each, until about budget_s of CPU work per case."""
    import oracle
    from paper_2209_08196_gb300 import synth
    out = {}
    for name, cfg in (("16 x 64x1024 range", synth.config_small_range(seed=0)),
                      ("128x2048 low coherence", synth.config_low_coherence(seed=7, n_scans=12))):
        attrs = synth.attr_descs(cfg)
        seq = synth.ScanSequence(cfg)
        enc = oracle.Codec(cfg.H, cfg.W, attrs)
        dec = oracle.Codec(cfg.H, cfg.W, attrs)
        n_scans, t_enc, t_dec = 0, 0.0, 0.0
        for t in range(cfg.n_scans):
            planes = seq.scan(t)
            t0 = time.perf_counter()
            b = enc.encode(planes)
            t1 = time.perf_counter()
            dec.decode(b)
            t2 = time.perf_counter()
            t_enc += t1 - t0
            t_dec += t2 - t1
            n_scans += 1
            if t_enc + t_dec >= budget_s:
                break
        px = n_scans * cfg.H * cfg.W
        out[name] = {"scans": n_scans, "cores": 1, "mpoints_s": px / (t_enc + t_dec) / 1e6,
                     "encode_mpoints_s": px / t_enc / 1e6, "decode_mpoints_s": px / t_dec / 1e6}
    return out


def cpu_baseline_ncore(cfg, attrs, scans, repeats: int = 6):
    """The oracle, as it stands, on every host core at once: the scans split
    into one independent stream per core (spawned processes, so no forked
    CUDA context), each encoded + decoded `repeats` times; whole-host
    points/s over the wall time of the parallel region."""
    import multiprocessing as mp
    import numpy as np
    DT = {1: np.uint8, 2: np.uint16, 4: np.uint32}
    n = max(1, min(os.cpu_count() or 1, len(scans)))
    host = [[p.cpu().numpy().view(DT[s]) for p, (s, _) in zip(planes, attrs)] for planes in scans]
    per = [host[i::n] for i in range(n)]
    ctx = mp.get_context("spawn")
    start = ctx.Event()
    procs, conns = [], []
    for i in range(n):
        a, b = ctx.Pipe()
        pr = ctx.Process(target=_oracle_worker, args=(b, start, cfg.H, cfg.W, attrs, repeats), daemon=True)
        pr.start()
        a.send(per[i])
        procs.append(pr)
        conns.append(a)
    for c in conns:
        if c.recv() != "ready":
            raise RuntimeError("oracle worker failed to start")
    t0 = time.perf_counter()
    start.set()
    busy = [c.recv() for c in conns]
    wall = time.perf_counter() - t0
    for pr in procs:
        pr.join(timeout=30)
    px = repeats * len(scans) * cfg.H * cfg.W
    return {"value": px / wall / 1e9, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": "the %d scans as %d independent streams (one per core, spawned processes), encode + decode, "
                      "%d passes; max busy %.2f s of %.2f s wall" % (len(scans), n, repeats, max(busy), wall)}


def run_reference(args, rank, world):
    """Reference arm: the oracle, timed on the host cores, one bounded sample
    of the workload (3 scans encoded and decoded) per step."""
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2209_08196_gb300 import synth
    cfg = synth.config_multi_attr(n_scans=3 + 1)
    scans = synth.ScanSequence(cfg).scans()
    attrs = synth.attr_descs(cfg)
    per = 3

    def step():
        enc = oracle.Codec(cfg.H, cfg.W, attrs)
        dec = oracle.Codec(cfg.H, cfg.W, attrs)
        for planes in scans[:per]:
            dec.decode(enc.encode(planes))

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    px = per * cfg.H * cfg.W * args.steps
    v = px / dt / 1e9
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_scans_per_step": per},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d scans encoded + decoded per step, single-threaded plain C" % per},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_leg(J, torch, dev, local, steps, warmup, n_streams=256, n_scans=8, base_seed=1000):
    """Many streams in one pass: n_streams sensors of uneven shapes and
    attribute sets, n_scans scans each, encoded by one batched call and
    decoded by another (CUDA-graph replay, autotuned launches), against the
    same scans coded one call per stream (jiffy_*_seq_async, all of a
    stream's scans in one call) and one scan per launch (jiffy_encode /
    jiffy_decode, a host round trip each)."""
    from paper_2209_08196_gb300 import synth
    t_gen = time.perf_counter()
    cfgs = [synth.batch_stream_config(i, base_seed=base_seed, n_scans=n_scans) for i in range(n_streams)]
    scans, encs, decs, outs, planes, attrs_l = [], [], [], [], [], []
    for c in cfgs:
        seq = synth.ScanSequence(c, device=dev)
        sc = [seq.scan(t, as_numpy=False) for t in range(n_scans)]
        at = synth.attr_descs(c)
        # one T x H x W tensor per attribute (the binding addresses planes by arithmetic)
        stk = [torch.stack([sc[t][a] for t in range(n_scans)]) for a in range(len(at))]
        scans.append(stk)
        attrs_l.append(at)
        encs.append(J.jiffy_stream_create(J.JIFFY_ENCODER, c.H, c.W, at, device=local))
        decs.append(J.jiffy_stream_create(J.JIFFY_DECODER, c.H, c.W, at, device=local))
        outs.append(torch.empty(J.jiffy_max_encoded_size(c.H, c.W, at, n_scans), dtype=torch.uint8, device=dev))
        planes.append(J.empty_planes(decs[-1], n_scans))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    px = sum(c.H * c.W * n_scans for c in cfgs)
    raw = sum(p.numel() * p.element_size() for stk in scans for p in stk)
    b = J.jiffy_batch_create(local)
    J.jiffy_batch_set_graphs(b, True)
    J.jiffy_batch_set_autotune(b, True)
    stream = torch.cuda.current_stream()
    res = {}

    def step():
        for h in encs + decs:
            J.jiffy_stream_reset(h)
        r = J.jiffy_encode_batch(b, encs, scans, outs, stream)
        J.jiffy_decode_batch(b, decs, outs, [n for n, _ in r], [o for _, o in r], planes, stream)
        res["r"] = r

    for _ in range(warmup):
        step()
    # round trip of every stream (outside the timed region)
    for c, sc, pl, at in zip(cfgs, scans, planes, attrs_l):
        for a, (sz, P) in enumerate(at):
            m = (1 << (8 * sz)) - 1
            v = sc[a].to(torch.int64) & m
            q = torch.clamp((v + P // 2) // P, max=m // P)
            if not torch.equal(pl[a].to(torch.int64) & m, q * P):
                raise SystemExit("batched round trip mismatch")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    info = J.jiffy_batch_info(b)
    # the same steps on the automatic launch configuration (no tuner)
    J.jiffy_batch_set_autotune(b, False)
    step()
    step()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_auto = e0.elapsed_time(e1) / steps
    info_auto = J.jiffy_batch_info(b)
    J.jiffy_batch_set_autotune(b, True)
    stream_bytes = sum(n for n, _ in res["r"])
    # kernel split of one batched step (graphs off while profiling)
    J.jiffy_batch_set_profiling(b, True)
    for h in encs + decs:
        J.jiffy_stream_reset(h)
    r = J.jiffy_encode_batch(b, encs, scans, outs, stream)
    ke = J.jiffy_batch_kernel_times(b)
    J.jiffy_decode_batch(b, decs, outs, [n for n, _ in r], [o for _, o in r], planes, stream)
    kd = J.jiffy_batch_kernel_times(b)
    J.jiffy_batch_set_profiling(b, False)

    # the same scans, one scan per launch
    def per_launch():
        frames = []
        for h in encs + decs:
            J.jiffy_stream_reset(h)
        for i, (c, sc) in enumerate(zip(cfgs, scans)):
            pos = 0
            for t in range(n_scans):
                n = J.jiffy_encode(encs[i], [p[t] for p in sc], outs[i][pos:], stream)
                frames.append((i, pos, n))
                pos += (n + 15) // 16 * 16
        for i, pos, n in frames:
            J.jiffy_decode(decs[i], outs[i][pos:], n, [p[0] for p in planes[i]], stream)
    per_launch()
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    per_launch()
    p1.record(stream)
    torch.cuda.synchronize()
    ms_pl = p0.elapsed_time(p1)

    # the same scans, one enqueue-only call per stream and direction
    # (jiffy_encode_seq_async / jiffy_decode_seq_async: each stream's 8 scans
    # in one call, its launch sequence replayed from the stream's graph)
    d_offs = [torch.zeros(n_scans + 1, dtype=torch.int64, device=dev) for _ in encs]

    def per_stream():
        for i in range(len(encs)):
            J.jiffy_stream_reset(encs[i])
            J.jiffy_stream_reset(decs[i])
            J.jiffy_encode_seq_async(encs[i], scans[i], outs[i], d_offs[i], stream)
            J.jiffy_decode_seq_async(decs[i], outs[i], d_offs[i], planes[i], stream)
        for h in encs + decs:
            J.jiffy_stream_wait(h)
    per_stream()
    per_stream()  # both segment-table slots of every stream warm
    torch.cuda.synchronize()
    p0.record(stream)
    for _ in range(3):
        per_stream()
    p1.record(stream)
    torch.cuda.synchronize()
    ms_seq = p0.elapsed_time(p1) / 3
    peak, _ = peaks()
    rows_frac = None
    if len(ke) == 3 and kd:
        rows_frac = ((raw + stream_bytes) / ke[1] / 1e6 / peak, (raw + stream_bytes) / kd[0] / 1e6 / peak)
    return {"workload": "%d streams x %d scans, shapes from %s, attribute sets from %s" % (
                n_streams, n_scans, list(synth.BATCH_SHAPES), [list(a) for a in synth.BATCH_ATTR_SETS]),
            "gpoints_s": px / (ms / 1e3) / 1e9, "ms_per_step": ms, "points_per_step": px, "raw_bytes": raw,
            "stream_bytes": stream_bytes, "ratio": raw / stream_bytes,
            "seq_gpoints_s": px / (ms_seq / 1e3) / 1e9, "seq_ms_per_step": ms_seq, "speedup_vs_seq": ms_seq / ms,
            "encode_rows_frac": rows_frac[0] if rows_frac else None,
            "decode_rows_frac": rows_frac[1] if rows_frac else None,
            "one_scan_per_launch_gpoints_s": px / (ms_pl / 1e3) / 1e9, "speedup_vs_one_scan_per_launch": ms_pl / ms,
            "kernels_ms": {"trial": ke[0], "encode_rows": ke[1], "placement": ke[2], "decode_rows": kd[0]}
            if len(ke) == 3 and kd else None,
            "launch": {k: info[k] for k in ("warps_per_cta", "ctas_per_sm", "items_per_ticket", "grid")},
            "auto_launch_gpoints_s": px / (ms_auto / 1e3) / 1e9,
            "auto_launch": {k: info_auto[k] for k in ("warps_per_cta", "ctas_per_sm", "items_per_ticket", "grid")},
            "graph_replays": info["graph_replays"], "tunings": info["tunings"], "gen_s": t_gen,
            "launches_per_step": 5}


def serve_leg(J, torch, dev, local, seconds, sat_seconds, n_sensors=512, base_seed=5000):
    """Serving loop: n_sensors sensors (shapes and attribute sets of the
    many-stream set) with Poisson arrivals at 10-20 Hz, replayed in real time
    for `seconds`, 10 % decode requests, 40 GB HBM budget; then the same
    sensors with every scan available at once (saturation) for capacity."""
    import numpy as np
    from paper_2209_08196_gb300 import serve, synth
    rng = np.random.default_rng(base_seed)
    classes = [(sh, at) for sh in synth.BATCH_SHAPES for at in synth.BATCH_ATTR_SETS]
    t_gen = time.perf_counter()
    pools, descs = [], []
    for k, ((H, W), at) in enumerate(classes):
        prec = tuple(10 if a in (synth.RANGE, synth.RANGE2) else 1 for a in at)
        c = synth.SensorConfig(H=H, W=W, attrs=at, precisions=prec, n_scans=8, dropout=0.0,
                               target_zero_frac=0.12, wall=True, seed=base_seed + k)
        seq = synth.ScanSequence(c, device=dev)
        pools.append([seq.scan(t, as_numpy=False) for t in range(8)])
        descs.append(synth.attr_descs(c))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    sensors = []
    for i in range(n_sensors):
        ci = int(rng.integers(len(classes)))
        (H, W), _ = classes[ci]
        sensors.append(serve.Sensor(i, H, W, descs[ci], float(rng.uniform(10, 20)), pool=ci,
                                    pool_offset=int(rng.integers(8))))
    max_px = sum(s.H * s.W for s in sensors)
    # the serving backend runs the automatic launch configuration: the tuner
    # times every candidate on the first batch of each new shape class, and
    # serving batches (any mix of sensors and backlogs) keep meeting new ones
    sat = {}
    for graphs in (True, False):
        be = serve.GpuBackend(pools, device=local, graphs=graphs, max_batch_px=max_px)
        # warm-up: tune, build the handles' scratch and the handle cache on a short saturated run
        serve.Server(be, sensors, budget_bytes=40e9).run(
            serve.poisson_arrivals(sensors, 0.5, 0.1, seed=base_seed + 1), realtime=False)
        sat[graphs] = serve.Server(be, sensors, budget_bytes=40e9).run(
            serve.poisson_arrivals(sensors, sat_seconds, 0.1, seed=base_seed + 3), realtime=False).summary()
        if graphs:
            del be
    # real time without graphs: every batch is a new composition, so a graph
    # would be captured for it and never replayed, which costs latency
    use_graphs = False
    rt = serve.Server(be, sensors, budget_bytes=40e9).run(
        serve.poisson_arrivals(sensors, seconds, 0.1, seed=base_seed + 2), realtime=True).summary()
    return {"workload": "%d sensors, Poisson 10-20 Hz, %g s real time, 10%% decode requests, 40 GB budget"
                        % (n_sensors, seconds),
            "p50_ms": rt["p50_ms"], "p99_ms": rt["p99_ms"], "decode_p50_ms": rt["decode_p50_ms"],
            "decode_p99_ms": rt["decode_p99_ms"], "gpoints_s": rt["gpoints_s"], "graphs": use_graphs,
            "realtime": rt, "saturated": max(sat.values(), key=lambda x: x["gpoints_s"]),
            "saturated_graphs_on_gpoints_s": sat[True]["gpoints_s"],
            "saturated_graphs_off_gpoints_s": sat[False]["gpoints_s"],
            "max_group": be.max_group, "autotune": False, "gen_s": t_gen}


def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time: replicas run independently (no collective on
    the data path); only this reduction joins them."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sweep_leg(J, torch, dev, local, max_mib=4096, reps=3, seed=7):
    """Encode and decode throughput against total stream size on the
    high-sparsity, low-coherence workload: 128 x 2048 range (u32 mm, 1 mm
    precision) + reflectivity (u8), 40 % zeros in random discs, random yaw
    (+-30 deg/s) and 3 m/s translation in a random direction, so I frames are
    chosen often. One random walk is continued until its raw planes reach each
    size (64 MiB, doubling up to max_mib); each size is one encode call over
    its scans and one decode call over their stream, both enqueue-only on one
    CUDA stream, timed with CUDA events after two warm-up pairs, with a 256 MiB
    write between calls so that no input starts in L2. Precision 1 makes the
    round trip the identity: the decoded planes must equal the input."""
    from paper_2209_08196_gb300 import synth
    H, W = 128, 2048
    raw_scan = H * W * (4 + 1)
    sizes, mib = [], 64
    while mib <= max_mib:
        sizes.append(mib)
        mib *= 2
    if not sizes:
        return None
    n_of = {m: -(-m * 2**20 // raw_scan) for m in sizes}
    n_max = n_of[sizes[-1]]
    cfg = synth.config_low_coherence(seed=seed, n_scans=n_max)
    attrs = synth.attr_descs(cfg)
    t_gen = time.perf_counter()
    seq = synth.ScanSequence(cfg, device=dev)
    planes = [torch.empty((n_max, H, W), dtype=torch.int32, device=dev),
              torch.empty((n_max, H, W), dtype=torch.uint8, device=dev)]
    for t in range(n_max):
        for a, p in enumerate(seq.scan(t, as_numpy=False)):
            planes[a][t].copy_(p)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, device=local)
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs, device=local)
    J.jiffy_stream_set_profiling(enc, True)
    J.jiffy_stream_set_profiling(dec, True)
    out = torch.empty(J.jiffy_max_encoded_size(H, W, attrs, n_max), dtype=torch.uint8, device=dev)
    outs = J.empty_planes(dec, n_max)
    d_offs = torch.zeros(n_max + 1, dtype=torch.int64, device=dev)
    flush = torch.empty(64 * 2**20, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    peak, _ = peaks()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    rows = []
    for m in sizes:
        n = n_of[m]
        src = [p[:n] for p in planes]
        dst = [o[:n] for o in outs]
        raw = n * raw_scan
        t_enc, t_dec, k_enc, k_dec = [], [], [], []
        for rep in range(reps + 2):  # two warm-up pairs: calls alternate between two segment-table slots
            J.jiffy_stream_reset(enc)
            J.jiffy_stream_reset(dec)
            flush.fill_(rep)
            ev[0].record(stream)
            J.jiffy_encode_seq_async(enc, src, out, d_offs, stream)
            ev[1].record(stream)
            flush.fill_(rep + 1)
            ev[2].record(stream)
            J.jiffy_decode_seq_async(dec, out, d_offs, dst, stream)
            ev[3].record(stream)
            J.jiffy_stream_wait(enc)
            J.jiffy_stream_wait(dec)
            if rep >= 2:
                t_enc.append(ev[0].elapsed_time(ev[1]))
                t_dec.append(ev[2].elapsed_time(ev[3]))
                k_enc.append(J.jiffy_stream_kernel_times(enc)[1])
                k_dec.append(J.jiffy_stream_kernel_times(dec)[0])
        nb = int(d_offs[n])
        exact = all(torch.equal(d, s_) for d, s_ in zip(dst, src))
        # share of I sections, from the frame headers (mode byte of each attribute)
        idx = d_offs[:n, None] + 8 + 12 * torch.arange(2, device=dev)[None, :]
        i_share = float((out[idx.reshape(-1)] == 0).float().mean())
        te, td = statistics.mean(t_enc), statistics.mean(t_dec)
        ke, kd = statistics.mean(k_enc), statistics.mean(k_dec)
        moved = raw + nb  # algorithmic bytes of either direction: raw planes + stream
        rows.append({"MiB": m, "scans": n, "stream_bytes": nb, "ratio": raw / nb, "i_share": i_share,
                     "encode_gpoints_s": n * H * W / te / 1e6, "decode_gpoints_s": n * H * W / td / 1e6,
                     "encode_ms": te, "decode_ms": td, "k_encode_ms": ke, "k_decode_ms": kd,
                     "k_encode_frac": moved / ke / 1e6 / peak, "k_decode_frac": moved / kd / 1e6 / peak,
                     "exact": bool(exact)})
    J.jiffy_stream_destroy(enc)
    J.jiffy_stream_destroy(dec)
    del planes, out, outs, flush
    torch.cuda.empty_cache()
    return {"workload": "low-coherence 128x2048 range u32 (P=1) + reflectivity u8, 40%% zeros in discs, "
                        "random yaw +-30 deg/s and 3 m/s; seed %d" % seed,
            "l2": "256 MiB write before each timed call", "reps": reps, "generate_s": t_gen,
            "peak_GBps": peak, "sizes": rows}


def small_stream_leg(J, torch, dev, local, steps=200, warmup=5):
    """The small single-stream case: 16 consecutive scans of 64 x 1024, range
    only (u32 mm at 10 mm precision, 8 % dropouts), about 1 M points. Its
    kernels are short, so the launch sequence of each call is replayed from a
    CUDA graph captured by the stream on its first call of this shape. A step
    is the encode of the 16 scans and the decode of their stream, enqueue-only
    on one CUDA stream. Timed two ways with CUDA events: steps one at a time
    after a 256 MiB write that evicts L2 (cold), and steps back to back with
    the 4 MB of inputs left in L2 (hot). With profiling on (no graph for the
    timed enqueue-only calls) the per-kernel times show how much of a step
    the kernels fill."""
    from paper_2209_08196_gb300 import synth
    cfg = synth.config_small_range(seed=0)
    attrs = synth.attr_descs(cfg)
    T, H, W = cfg.n_scans, cfg.H, cfg.W
    seq = synth.ScanSequence(cfg, device=dev)
    planes = [torch.stack([seq.scan(t, as_numpy=False)[0] for t in range(T)])]
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, device=local)
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs, device=local)
    out = torch.empty(J.jiffy_max_encoded_size(H, W, attrs, T), dtype=torch.uint8, device=dev)
    outs = J.empty_planes(dec, T)
    d_offs = torch.zeros(T + 1, dtype=torch.int64, device=dev)
    flush = torch.empty(64 * 2**20, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        J.jiffy_stream_reset(enc)
        J.jiffy_stream_reset(dec)
        J.jiffy_encode_seq_async(enc, planes, out, d_offs, stream)
        J.jiffy_decode_seq_async(dec, out, d_offs, outs, stream)

    for _ in range(warmup):
        step()
    J.jiffy_stream_wait(enc)
    J.jiffy_stream_wait(dec)
    m = 0xFFFFFFFF
    q = torch.clamp(((planes[0].to(torch.int64) & m) + 5) // 10, max=m // 10) * 10
    exact = torch.equal(outs[0].to(torch.int64) & m, q)
    nb = int(d_offs[T])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cold = []
    for i in range(steps // 4):
        flush.fill_(i)
        e0.record(stream)
        step()
        e1.record(stream)
        J.jiffy_stream_wait(enc)
        J.jiffy_stream_wait(dec)
        cold.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    J.jiffy_stream_wait(enc)
    J.jiffy_stream_wait(dec)
    hot = e0.elapsed_time(e1) / steps
    # per-kernel device time of the same step
    J.jiffy_stream_set_profiling(enc, True)
    J.jiffy_stream_set_profiling(dec, True)
    for _ in range(warmup):
        step()
    J.jiffy_stream_wait(enc)
    J.jiffy_stream_wait(dec)
    for _ in range(steps // 4):
        step()
    J.jiffy_stream_wait(enc)
    J.jiffy_stream_wait(dec)
    ke, kd = J.jiffy_stream_kernel_times(enc), J.jiffy_stream_kernel_times(dec)
    px = T * H * W
    cold_ms = statistics.median(cold)
    J.jiffy_stream_destroy(enc)
    J.jiffy_stream_destroy(dec)
    return {"workload": "16 scans x 64 x 1024, range u32 (10 mm), 8% dropouts", "points_per_step": px,
            "stream_bytes": nb, "ratio": px * 4 / nb, "exact": bool(exact),
            "cold_gpoints_s": px / cold_ms / 1e6, "cold_us_per_step": 1e3 * cold_ms,
            "hot_gpoints_s": px / hot / 1e6, "hot_us_per_step": 1e3 * hot,
            "kernels_us_per_step": 1e3 * (sum(ke) + sum(kd)),
            "kernel_us": {"k_trial": 1e3 * ke[0], "k_encode": 1e3 * ke[1], "k_finalize": 1e3 * ke[2],
                          "k_decode": 1e3 * kd[0]},
            "graphs": "each call's launch sequence replayed from a CUDA graph (not with profiling on)",
            "l2": "cold: 256 MiB write before each step; hot: back-to-back steps, inputs in L2",
            "launches_per_step": 5}


def _zstd():
    """libzstd through ctypes (compress, decompress, error check), or None."""
    import ctypes
    import ctypes.util
    path = ctypes.util.find_library("zstd")
    if path is None:
        return None
    z = ctypes.CDLL(path)
    sz, vp = ctypes.c_size_t, ctypes.c_void_p
    z.ZSTD_compressBound.restype, z.ZSTD_compressBound.argtypes = sz, [sz]
    z.ZSTD_compress.restype, z.ZSTD_compress.argtypes = sz, [vp, sz, vp, sz, ctypes.c_int]
    z.ZSTD_decompress.restype, z.ZSTD_decompress.argtypes = sz, [vp, sz, vp, sz]
    z.ZSTD_isError.restype, z.ZSTD_isError.argtypes = ctypes.c_uint, [sz]
    z.ZSTD_versionNumber.restype = ctypes.c_uint
    return z


def mask_codec_leg(J, torch, dev, local, levels=(1, 3, 19)):
    """The zero-mask part of the stream (Sec. III-C: the mask of zero samples,
    for P XORed with the previous scan's, Sec. III-D) in this codec's per-row
    class/literal form against the paper's form: the section's mask packed
    into bytes (one bit per sample, row-major) and compressed with Zstd
    (libzstd through ctypes, on the host). Our bytes are read from the GPU's
    own stream; every Zstd frame is decompressed and checked."""
    import ctypes

    import numpy as np

    from paper_2209_08196_gb300 import streaminfo, synth
    z = _zstd()
    if z is None:
        return {"unavailable": "libzstd is not installed on this host"}
    cases = [("16 x 64x1024 range, 8% dropouts", synth.config_small_range(seed=0)),
             ("20 x 128x2048 five attributes, 12% zeros in range", synth.config_multi_attr(seed=0, n_scans=20)),
             ("50 x 128x2048 range + reflectivity, 40% zeros in discs", synth.config_low_coherence(seed=7, n_scans=50))]
    rows = []
    for name, cfg in cases:
        attrs = synth.attr_descs(cfg)
        T, H, W, A = cfg.n_scans, cfg.H, cfg.W, len(attrs)
        seq = synth.ScanSequence(cfg, device=dev)
        sc = [seq.scan(t, as_numpy=False) for t in range(T)]
        planes = [torch.stack([sc[t][a] for t in range(T)]) for a in range(A)]
        del sc
        enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, device=local)
        out = torch.empty(J.jiffy_max_encoded_size(H, W, attrs, T), dtype=torch.uint8, device=dev)
        n, _ = J.jiffy_encode_seq(enc, planes, out)
        _, secs = streaminfo.sections(out[:n].cpu().numpy().tobytes())
        # the zero masks of the quantized samples, packed 8 per byte (LSB first)
        wts = torch.tensor([1, 2, 4, 8, 16, 32, 64, 128], dtype=torch.int32, device=dev)
        packed = []
        for a, (s_, P) in enumerate(attrs):
            m = (1 << (8 * s_)) - 1
            q = torch.clamp(((planes[a].to(torch.int64) & m) + P // 2) // P, max=m // P)
            bits = (q == 0).to(torch.int32).reshape(T, H * W // 8, 8)
            packed.append((bits * wts).sum(-1).to(torch.uint8).cpu().numpy())
            del q, bits
        zb = {lv: 0 for lv in levels}
        for sinfo in secs:
            src = packed[sinfo.attr][sinfo.frame]
            if sinfo.mode == 1:
                src = src ^ packed[sinfo.attr][sinfo.frame - 1]
            src = np.ascontiguousarray(src)
            cap = z.ZSTD_compressBound(src.nbytes)
            dst = np.empty(cap, dtype=np.uint8)
            back = np.empty(src.nbytes, dtype=np.uint8)
            for lv in levels:
                k = z.ZSTD_compress(dst.ctypes.data, cap, src.ctypes.data, src.nbytes, lv)
                if z.ZSTD_isError(k):
                    raise SystemExit("ZSTD_compress failed")
                r = z.ZSTD_decompress(back.ctypes.data, back.nbytes, dst.ctypes.data, k)
                if z.ZSTD_isError(r) or r != src.nbytes or not np.array_equal(back, src):
                    raise SystemExit("Zstd round trip failed")
                zb[lv] += k
        ours = sum(x.mask_bytes for x in secs)
        rows.append({"workload": name, "scans": T, "sections": len(secs),
                     "p_share": sum(x.mode for x in secs) / len(secs),
                     "packed_mask_bytes_per_scan": H * W * A / 8,
                     "class_literal_bytes_per_scan": ours / T,
                     "zstd_bytes_per_scan": {str(lv): zb[lv] / T for lv in levels},
                     "mask_share_of_stream": ours / n,
                     "stream_bytes_per_scan": n / T})
        del planes, out, enc
    v = z.ZSTD_versionNumber()
    return {"zstd_version": "%d.%d.%d" % (v // 10000, v // 100 % 100, v % 100), "levels": list(levels),
            "bit_order": "row-major, least significant bit first", "cases": rows}


def zstd_mask_leg(J, torch, dev, local, planes_in, attrs, steps, warmup, base, info_scans=10):
    """The paper's mask coding as the stream option (Sec. III-C: the zero
    bitmask packed into bytes and compressed with Zstd; Sec. III-D: XORed with
    the previous scan's for P): every section's mask one Zstandard frame,
    written and read by the GPU kernels, on the benchmark's workload and step
    (enqueue-only encode and decode of all scans on one CUDA stream). Against
    the class-coded step of the headline: step time, stream bytes, mask bytes
    per scan (read back by the stream inspector) and the device time of the
    encoder's placement phase (which holds the Zstandard writer) and of the
    decode (which holds the reader)."""
    from paper_2209_08196_gb300 import streaminfo
    T, H, W = (int(x) for x in planes_in[0].shape)
    Z = J.STAGE_ZSTD_MASK
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, device=local, stages=Z)
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs, device=local, stages=Z)
    out = torch.empty(J.jiffy_max_encoded_size(H, W, attrs, T), dtype=torch.uint8, device=dev)
    outs = J.empty_planes(dec, T)
    d_offs = torch.zeros(T + 1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        J.jiffy_stream_reset(enc)
        J.jiffy_stream_reset(dec)
        J.jiffy_encode_seq_async(enc, planes_in, out, d_offs, stream)
        J.jiffy_decode_seq_async(dec, out, d_offs, outs, stream)

    for _ in range(warmup):
        step()
    J.jiffy_stream_wait(enc)
    J.jiffy_stream_wait(dec)
    exact = True
    for a, (s_, P) in enumerate(attrs):
        m = (1 << (8 * s_)) - 1
        q = torch.clamp(((planes_in[a].to(torch.int64) & m) + P // 2) // P, max=m // P)
        exact = exact and torch.equal(outs[a].to(torch.int64) & m, q * P)
        del q
    nz = int(d_offs[T])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    J.jiffy_stream_wait(enc)
    J.jiffy_stream_wait(dec)
    ms = e0.elapsed_time(e1) / steps
    J.jiffy_stream_set_profiling(enc, True)
    J.jiffy_stream_set_profiling(dec, True)
    for _ in range(steps):
        step()
    J.jiffy_stream_wait(enc)
    J.jiffy_stream_wait(dec)
    ke, kd = J.jiffy_stream_kernel_times(enc), J.jiffy_stream_kernel_times(dec)
    # mask bytes of the first scans, both mask codings, from the streams themselves
    n_i = min(info_scans, T)
    sub = [p[:n_i] for p in planes_in]
    per = {}
    for name, st in (("zstd", Z), ("class_words", 0)):
        e = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, device=local, stages=st)
        b = torch.empty(J.jiffy_max_encoded_size(H, W, attrs, n_i), dtype=torch.uint8, device=dev)
        nb, _ = J.jiffy_encode_seq(e, sub, b, stream)
        _, secs = streaminfo.sections(b[:nb].cpu().numpy().tobytes())
        per[name] = {"mask_bytes_per_scan": sum(x.mask_bytes for x in secs) / n_i, "stream_bytes_per_scan": nb / n_i}
        del e, b
    raw = sum(p.numel() * p.element_size() for p in planes_in)
    px = T * H * W
    J.jiffy_stream_destroy(enc)
    J.jiffy_stream_destroy(dec)
    return {"stages": "JIFFY_STAGE_ZSTD_MASK", "exact": bool(exact), "steps": steps,
            "gpoints_s": px / ms / 1e6, "ms_per_step": ms, "class_words_ms_per_step": base["ms_per_step"],
            "stream_bytes": nz, "class_words_stream_bytes": base["stream_bytes"],
            "ratio": raw / nz, "class_words_ratio": raw / base["stream_bytes"],
            "first_scans": n_i, "per_scan": per,
            "kernel_ms": {"k_trial": ke[0], "k_encode": ke[1], "k_finalize_with_zstd_writer": ke[2],
                          "k_decode_with_zstd_reader": kd[0]},
            "class_words_kernel_ms": {"k_finalize": base["k_finalize"], "k_decode": base["k_decode"]},
            "zstd_writer_ms": ke[2] - base["k_finalize"], "zstd_reader_ms": kd[0] - base["k_decode"],
            "blocks": "one per 8192 mask bytes: RLE, Raw, or Huffman literals (1 or 4 streams) with direct or "
                      "FSE-coded weights and no sequences; every frame is a standard Zstandard frame"}


def whole_job_gpoints(px_per_rank: int, world: int, ms: float) -> float:
    """All ranks' pixels over the slowest rank's time, in Gpoints/s."""
    return px_per_rank * world / (ms / 1e3) / 1e9


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--scans", type=int, default=100, help="scans per step (100 = the benchmark workload)")
    ap.add_argument("--no-batched", action="store_true", help="skip the many-stream leg")
    ap.add_argument("--no-heuristic", action="store_true", help="skip the trial-vs-brute-force leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-ablation", action="store_true", help="skip the ablated-codec leg")
    ap.add_argument("--no-standardize", action="store_true", help="skip the point-cloud standardization leg")
    ap.add_argument("--kernel-repeats", type=int, default=100,
                    help="steps over which the per-kernel averages are taken once more after the timed region")
    ap.add_argument("--no-sweep", action="store_true", help="skip the stream-size sweep leg")
    ap.add_argument("--no-small", action="store_true", help="skip the 16 x 64 x 1024 single-stream leg")
    ap.add_argument("--no-mask-codec", action="store_true", help="skip the Zstd mask comparison leg")
    ap.add_argument("--no-zstd-mask", action="store_true", help="skip the leg run with the Zstandard mask option")
    ap.add_argument("--sweep-max-mib", type=int, default=4096, help="largest raw size of the sweep")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-sat-seconds", type=float, default=5.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        # replicas: the scaling figure is the main step's; the other legs
        # measure single-GPU properties and run in the one-GPU invocation
        for leg in ("small", "sweep", "batched", "serve", "heuristic", "ablation", "standardize", "mask_codec",
                    "zstd_mask"):
            setattr(args, "no_" + leg, True)

    import torch
    import torch.distributed as dist
    from paper_2209_08196_gb300 import build as jbuild
    from paper_2209_08196_gb300 import jiffy as J

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    jbuild.build()
    dev = "cuda:%d" % local
    cfg, attrs, scans = make_workload(dev, seed=0 + rank, n_scans=args.scans)
    T, H, W, A = cfg.n_scans, cfg.H, cfg.W, len(attrs)
    raw_bytes = sum(p.numel() * p.element_size() for s in scans for p in s)
    # one T x H x W tensor per attribute: the binding addresses its planes by arithmetic
    planes_in = [torch.stack([scans[t][a] for t in range(T)]) for a in range(A)]
    del scans
    enc = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, device=local)
    dec = J.jiffy_stream_create(J.JIFFY_DECODER, H, W, attrs, device=local)
    J.jiffy_stream_set_profiling(enc, True)
    J.jiffy_stream_set_profiling(dec, True)
    cap = J.jiffy_max_encoded_size(H, W, attrs, T)
    out = torch.empty(cap, dtype=torch.uint8, device=dev)
    outs = J.empty_planes(dec, T)
    stream = torch.cuda.current_stream()
    ktimes = {"k_trial": [], "k_encode": [], "k_finalize": [], "k_decode": []}
    state = {}
    d_offs = torch.zeros(T + 1, dtype=torch.int64, device=dev)  # frame offsets, left on the device

    # one step: the encode of the T scans and the decode of their stream,
    # both enqueue-only on one CUDA stream (the frame offsets pass from the
    # encoder to the decoder in device memory: no host round trip)
    def step():
        J.jiffy_stream_reset(enc)
        J.jiffy_stream_reset(dec)
        J.jiffy_encode_seq_async(enc, planes_in, out, d_offs, stream)
        J.jiffy_decode_seq_async(dec, out, d_offs, outs, stream)

    def settle(record):
        # waits for the enqueued steps; the kernel times are the averages over them
        J.jiffy_stream_wait(enc)
        J.jiffy_stream_wait(dec)
        te = J.jiffy_stream_kernel_times(enc)
        td = J.jiffy_stream_kernel_times(dec)
        if record:
            ktimes["k_trial"].append(te[0])
            ktimes["k_encode"].append(te[1])
            ktimes["k_finalize"].append(te[2])
            ktimes["k_decode"].append(td[0])
        offs = [int(x) for x in d_offs.cpu()]
        state["n"], state["offs"] = offs[-1], offs

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    settle(False)
    # bit-exact check of the benchmarked configuration (outside the timed region)
    for a, (s, P) in enumerate(attrs):
        m = (1 << (8 * s)) - 1
        v = planes_in[a].to(torch.int64) & m
        q = torch.clamp((v + P // 2) // P, max=m // P)
        if not torch.equal(outs[a].to(torch.int64) & m, q * P):
            raise SystemExit("round trip mismatch on attribute %d" % a)
        del v, q

    clk = Clocks(local)
    barrier()
    clk.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    barrier()
    settle(True)
    clocks = clk.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    ms_step = ms / args.steps
    px_step = T * H * W
    value = whole_job_gpoints(px_step, world, ms_step)
    n = state["n"]
    # the per-kernel averages once more over many steps (after the timed
    # region; the roofline keeps the timed region's own averages)
    long_k = None
    if args.kernel_repeats > 0:
        for _ in range(args.kernel_repeats):
            step()
        J.jiffy_stream_wait(enc)
        J.jiffy_stream_wait(dec)
        te, td = J.jiffy_stream_kernel_times(enc), J.jiffy_stream_kernel_times(dec)
        long_k = {"steps": args.kernel_repeats, "k_trial_ms": te[0], "k_encode_ms": te[1], "k_finalize_ms": te[2],
                  "k_decode_ms": td[0]}

    # e2e through host buffers, every step: H2D of the scans, encode, D2H of
    # the stream, H2D of the stream, decode, D2H of the decoded scans. The
    # steps are software-pipelined the way a streaming user would run them:
    # while the (synchronous) encode of step i+1 and decode of step i run on
    # the compute stream, copy streams upload step i+2's scans, move step
    # i+1's stream to the host and back, and download step i-1's planes; all
    # device and host buffers are double-buffered and ordered by events. All
    # K steps' copies fall inside the timed region.
    scap = (n + (1 << 20)) // 256 * 256 + 256  # the stream of these scans, with room to spare
    host_in = [p.cpu().pin_memory() for p in planes_in]
    host_stream = [torch.empty(scap, dtype=torch.uint8).pin_memory() for _ in range(2)]
    host_out = [[torch.empty_like(o, device="cpu").pin_memory() for o in outs] for _ in range(2)]
    dev_in = [[torch.empty_like(p) for p in planes_in] for _ in range(2)]
    enc_out = [torch.empty(scap, dtype=torch.uint8, device=dev) for _ in range(2)]
    dec_in = [torch.empty(scap, dtype=torch.uint8, device=dev) for _ in range(2)]
    dev_out = [outs, J.empty_planes(dec, T)]
    up, down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)

    def evs():
        return [torch.cuda.Event(), torch.cuda.Event()]
    ev_in, ev_d2h, ev_h2d, ev_dec, ev_out = evs(), evs(), evs(), evs(), evs()
    for ev in ev_d2h + ev_h2d + ev_out:
        ev.record(stream)
    meta = {}

    def upload(i):
        s = i % 2
        with torch.cuda.stream(up):
            for h, d in zip(host_in, dev_in[s]):
                d.copy_(h, non_blocking=True)
            ev_in[s].record(up)

    def encode(i):
        s = i % 2
        stream.wait_event(ev_in[s])
        stream.wait_event(ev_d2h[s])  # step i-2's stream has left enc_out[s]
        J.jiffy_stream_reset(enc)
        meta[i] = J.jiffy_encode_seq(enc, dev_in[s], enc_out[s], stream)

    def round_trip(i):
        s, nn = i % 2, meta[i][0]
        with torch.cuda.stream(down):
            down.wait_event(ev_h2d[s])  # step i-2's stream has left host_stream[s]
            host_stream[s][:nn].copy_(enc_out[s][:nn], non_blocking=True)
            ev_d2h[s].record(down)
        with torch.cuda.stream(up):
            up.wait_event(ev_d2h[s])
            dec_in[s][:nn].copy_(host_stream[s][:nn], non_blocking=True)
            ev_h2d[s].record(up)

    def decode(i):
        s = i % 2
        nn, offs = meta.pop(i)
        stream.wait_event(ev_h2d[s])
        stream.wait_event(ev_out[s])  # step i-2's planes have left dev_out[s]
        J.jiffy_stream_reset(dec)
        J.jiffy_decode_seq(dec, dec_in[s], nn, offs, dev_out[s], stream)
        ev_dec[s].record(stream)
        with torch.cuda.stream(down):
            down.wait_event(ev_dec[s])
            for h, o in zip(host_out[s], dev_out[s]):
                h.copy_(o, non_blocking=True)
            ev_out[s].record(down)
        return nn

    def e2e_run(k):
        upload(0)
        if k > 1:
            upload(1)
        encode(0)
        round_trip(0)
        nn = 0
        for i in range(k):
            if i + 1 < k:
                encode(i + 1)
                if i + 2 < k:
                    upload(i + 2)
                round_trip(i + 1)
            nn = decode(i)
        for ev in ev_out:
            stream.wait_event(ev)
        return nn

    e2e = None
    if not args.no_e2e:
        e2e_run(3)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        up.wait_event(e0)
        down.wait_event(e0)
        nn = e2e_run(args.steps)
        e1.record(stream)
        barrier()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
        # the pipelined run decoded every step: check the last one bit-exactly
        for a, (s_, P) in enumerate(attrs):
            m = (1 << (8 * s_)) - 1
            q = torch.clamp(((planes_in[a].to(torch.int64) & m) + P // 2) // P, max=m // P)
            if not torch.equal(dev_out[(args.steps - 1) % 2][a].to(torch.int64) & m, q * P):
                raise SystemExit("e2e round trip mismatch on attribute %d" % a)
            del q
        e2e = {"value": whole_job_gpoints(px_step, world, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": raw_bytes + nn, "d2h_bytes_per_step": nn + raw_bytes,
               "pipelined": "encode of step i+1 and decode of step i overlap the uploads of step i+2, "
                            "the stream round trip of step i+1 and the download of step i-1"}
        del host_stream, host_out, dev_in, enc_out, dec_in

    # roofline of the dominant kernel: algorithmic bytes / CUDA-event duration
    avg = {k: statistics.mean(v) for k, v in ktimes.items()}
    algo = {"k_encode": raw_bytes + n, "k_decode": n + raw_bytes}
    dom = max(("k_encode", "k_decode"), key=lambda k: avg[k])
    peak, src = peaks()
    achieved = algo[dom] / (avg[dom] / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": src, "traffic": traffic(dom, T),
                "algorithmic_bytes_per_launch": algo[dom],
                "frac_of_nominal_8000GBps": achieved / 8000.0}
    kernels = {k: {"avg_ms": avg[k], "GBps": (algo[k] / (avg[k] / 1e3) / 1e9) if k in algo else None,
                   "frac_of_peak": (algo[k] / (avg[k] / 1e3) / 1e9 / peak) if k in algo else None}
               for k in avg}

    # trial heuristic (4 test lines) against the brute-force choice (every row a
    # test row), Sec. IV-E: per-section modes, stream bytes, encode time
    heuristic = None
    if not args.no_heuristic:
        bfe = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, test_lines=H, device=local)
        J.jiffy_stream_set_profiling(bfe, True)
        out_bf = torch.empty(cap, dtype=torch.uint8, device=dev)
        tb = []
        for _ in range(3):
            J.jiffy_stream_reset(bfe)
            n_bf, offs_bf = J.jiffy_encode_seq(bfe, planes_in, out_bf, stream)
            tb.append(sum(J.jiffy_stream_kernel_times(bfe)))

        def modes_of(buf, offs):
            idx = torch.tensor([offs[t] + 8 + 12 * a for t in range(1, T) for a in range(A)], device=dev)
            return buf[idx].cpu().tolist()
        mh = modes_of(out, state["offs"])
        mb = modes_of(out_bf, offs_bf)
        ns = len(mh)
        t_heur = statistics.mean(ktimes["k_trial"]) + statistics.mean(ktimes["k_encode"]) + \
            statistics.mean(ktimes["k_finalize"])
        heuristic = {
            "sections": ns, "agree_pct": 100.0 * sum(x == y for x, y in zip(mh, mb)) / ns,
            "suboptimal_i_pct": 100.0 * sum(x == 0 and y == 1 for x, y in zip(mh, mb)) / ns,
            "suboptimal_p_pct": 100.0 * sum(x == 1 and y == 0 for x, y in zip(mh, mb)) / ns,
            "p_pct_heuristic": 100.0 * sum(mh) / ns, "p_pct_brute_force": 100.0 * sum(mb) / ns,
            "stream_bytes_heuristic": n, "stream_bytes_brute_force": n_bf,
            "encode_ms_heuristic": t_heur, "encode_ms_brute_force": min(tb),
            "paper": "96 % agreement on 22,877 range scans (0.5 % sub-optimal I, 3.5 % sub-optimal P)"}
        del out_bf

    # the same scene seen from a parked sensor (the paper's ablation data is a
    # fixed infrastructure-monitoring sensor): 90 % of the dropouts hit the
    # same pixels every scan and the range has 10 mm of Gaussian noise
    parked = None
    if not (args.no_heuristic and args.no_ablation):
        from paper_2209_08196_gb300 import synth
        n_t = min(T, 20)
        scfg = synth.config_multi_attr(seed=0, n_scans=n_t)
        scfg.speed_mps = 0.0
        scfg.persistent_dropout = 0.9
        scfg.range_noise_mm = 10.0
        sseq = synth.ScanSequence(scfg, device=dev)
        sscans = [sseq.scan(t, as_numpy=False) for t in range(n_t)]
        parked = [torch.stack([sscans[t][a] for t in range(n_t)]) for a in range(A)]
        del sscans

    # precision sweep on the range plane (Fig. 4, Sec. IV-G): bits per sample as
    # the quantization precision doubles, on the noise-free moving scene and on
    # the parked scene with 10 mm range noise (the paper: about one bit saved
    # per doubling once the precision exceeds the sensor noise)
    precision = None
    if not args.no_heuristic:
        n_t = min(T, 20)
        precs = (1, 2, 4, 8, 16, 32, 64, 128, 256, 512, 1024)
        precision = {"scans": n_t, "attribute": "range (uint32 mm)", "precisions_mm": list(precs)}
        for scene, rng_planes in (("moving", [planes_in[0][:n_t]]), ("parked_10mm_noise", [parked[0]])):
            bits = []
            for P in precs:
                pe = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, [(4, P)], device=local)
                pbuf = torch.empty(J.jiffy_max_encoded_size(H, W, [(4, P)], n_t), dtype=torch.uint8, device=dev)
                nb_p, _ = J.jiffy_encode_seq(pe, rng_planes, pbuf, stream)
                bits.append(8.0 * nb_p / (n_t * H * W))
                del pe, pbuf
            # bits saved per doubling, from 16 mm and from 32 mm up to 1024 mm
            precision[scene] = {"bits_per_sample": bits,
                                "bits_saved_per_doubling_16_to_1024mm": (bits[4] - bits[-1]) / 6.0,
                                "bits_saved_per_doubling_32_to_1024mm": (bits[5] - bits[-1]) / 5.0,
                                "bits_saved_per_doubling_1_to_16mm": (bits[0] - bits[4]) / 4.0}

    # ablated codecs (Sec. IV-H, Table IV) on the first scans of the workload
    # and on the parked scene: compression ratio and encode time of each
    # stage set
    ablation = None
    if not args.no_ablation:
        n_t = min(T, 20)
        ladder = [("SIMD-PFOR", 7, 0), ("Delta -> SIMD-PFOR", 5, 0), ("Delta -> ZigZag -> SIMD-PFOR", 1, 0),
                  ("Mask -> Delta -> ZigZag -> SIMD-PFOR", 0, 0),
                  ("Mask -> Predict -> Delta -> ZigZag -> SIMD-PFOR (Jiffy)", 0, -1)]
        scenes = {"moving (10 m/s)": [p[:n_t] for p in planes_in], "parked": parked}
        abuf = torch.empty(J.jiffy_max_encoded_size(H, W, attrs, n_t), dtype=torch.uint8, device=dev)
        raw_t = sum(p.numel() * p.element_size() for p in scenes["parked"])
        ablation = {"scans": n_t, "attributes": list(cfg.attrs), "codecs": []}
        for name, stages, force in ladder:
            row = {"codec": name, "stages": stages, "force_mode": force}
            for scene, pl in scenes.items():
                ae = J.jiffy_stream_create(J.JIFFY_ENCODER, H, W, attrs, force_mode=force, device=local,
                                           stages=stages)
                J.jiffy_stream_set_profiling(ae, True)
                tms = []
                for _ in range(2):
                    J.jiffy_stream_reset(ae)
                    nb_a, _ = J.jiffy_encode_seq(ae, pl, abuf, stream)
                    tms.append(sum(J.jiffy_stream_kernel_times(ae)))
                row[scene] = {"ratio": raw_t / nb_a, "encode_gpoints_s": n_t * H * W / min(tms) / 1e6}
                del ae
            ablation["codecs"].append(row)
        ablation["paper"] = "Table IV (infrastructure monitoring data): 3.2, 2.2, 3.8, 5.4, 6.2"
        del abuf, scenes

    # input standardization (Sec. III-A) of the same scans given as points:
    # each scan's valid pixels as float32 x y z (metres) plus three float
    # attributes, converted back to the range and attribute images, all scans
    # in one call (two kernels: points, then pixels)
    standardize = None
    if not args.no_standardize:
        n_s = T
        alt = torch.linspace(22.5, -22.5, H, dtype=torch.float64, device=dev) * (math.pi / 180.0)
        clouds = []
        for t in range(n_s):
            rr = planes_in[0][t]
            rows_, cols_ = torch.nonzero(rr != 0, as_tuple=True)
            r_m = rr[rows_, cols_].to(torch.float64) / 1000.0
            el_, az_ = alt[rows_], (cols_.to(torch.float64) + 0.5) * (2 * math.pi / W)
            xyz = torch.stack([r_m * torch.cos(el_) * torch.cos(az_), r_m * torch.cos(el_) * torch.sin(az_),
                               r_m * torch.sin(el_)], 1).to(torch.float32).contiguous()
            vals = [(planes_in[a][t][rows_, cols_].to(torch.int64) & 0xFFFF).to(torch.float32) for a in (2, 3, 4)]
            clouds.append((xyz, vals))
        std = J.jiffy_standardizer_create(H, W, alt.cpu().tolist(), device=local)
        s_offs = [0]
        for c in clouds:
            s_offs.append(s_offs[-1] + c[0].shape[0])
        s_xyz = torch.cat([c[0] for c in clouds])
        s_vals = [torch.cat([c[1][a] for c in clouds]) for a in range(3)]
        del clouds
        s_range = torch.empty((n_s, H, W), dtype=torch.int32, device=dev)
        s_attr = [torch.empty((n_s, H, W), dtype=d, device=dev) for d in (torch.int16, torch.uint8, torch.int16)]

        def std_run():
            J.jiffy_standardize_seq(std, s_xyz, s_offs, s_range, [(s_vals[a], s_attr[a], 1.0) for a in range(3)],
                                    stream)
        std_run()
        torch.cuda.synchronize()
        ok = int((s_range.to(torch.int64) - planes_in[0][:n_s].to(torch.int64)).abs().max()) <= 1
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            std_run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / (reps * n_s)
        npts = s_offs[-1] / n_s
        moved = npts * (12 + 12) + H * W * (4 + 2 + 1 + 2)  # points + attributes in, images out
        peak_s, _ = peaks()
        standardize = {"scans": n_s, "points_per_scan": npts, "attributes": 3, "ms_per_scan": ms,
                       "gpoints_s": npts / ms / 1e6, "algorithmic_bytes_per_scan": moved,
                       "achieved_GBps": moved / ms / 1e6, "frac_of_hbm": moved / ms / 1e6 / peak_s,
                       "launches_per_call": 2, "scans_per_call": n_s, "all_scans_within_1_unit": bool(ok)}
        del s_xyz, s_vals, s_range, s_attr, std

    small = None
    if not args.no_small:
        small = small_stream_leg(J, torch, dev, local)

    mask_codec = None
    if not args.no_mask_codec:
        mask_codec = mask_codec_leg(J, torch, dev, local)

    zstd_mask = None
    if not args.no_zstd_mask:
        zstd_mask = zstd_mask_leg(J, torch, dev, local, planes_in, attrs, args.steps, args.warmup,
                                  {"ms_per_step": ms_step, "stream_bytes": n, "k_finalize": avg["k_finalize"],
                                   "k_decode": avg["k_decode"]})

    sweep = None
    if not args.no_sweep:
        sweep = sweep_leg(J, torch, dev, local, args.sweep_max_mib)

    batched = served = None
    if not args.no_batched:
        batched = batched_leg(J, torch, dev, local, args.steps, args.warmup)
    if not args.no_serve:
        served = serve_leg(J, torch, dev, local, args.serve_seconds, args.serve_sat_seconds)

    if rank == 0:
        cpu = cpu_n = cpu_cfg = None
        if not args.no_cpu_baseline and world == 1:
            host_scans = [[planes_in[a][t] for a in range(A)] for t in range(T)]
            cpu = cpu_baseline(cfg, attrs, host_scans)
            try:
                cpu_n = cpu_baseline_ncore(cfg, attrs, host_scans)
            except Exception as ex:  # a reported extra; the run goes on without it
                cpu_n = {"value": None, "error": "%s: %s" % (type(ex).__name__, ex)}
            cpu_cfg = cpu_baseline_configs()
        modes = {"ratio": raw_bytes / n}
        if long_k is not None:
            roofline["kernel_avgs_over_more_steps"] = long_k
        # compact copies of the other legs' headline figures inside the keys the
        # contract defines (the full legs follow as their own keys)
        if sweep is not None:
            roofline["sweep"] = {
                "columns": ["MiB", "encode_gpoints_s", "decode_gpoints_s", "k_encode_frac", "k_decode_frac", "exact"],
                "rows": [[r["MiB"], round(r["encode_gpoints_s"], 2), round(r["decode_gpoints_s"], 2),
                          round(r["k_encode_frac"], 3), round(r["k_decode_frac"], 3), r["exact"]]
                         for r in sweep["sizes"]]}
        if batched is not None:
            roofline["batched"] = {"gpoints_s": batched["gpoints_s"], "seq_gpoints_s": batched.get("seq_gpoints_s"),
                                   "encode_rows_frac": batched.get("encode_rows_frac"),
                                   "decode_rows_frac": batched.get("decode_rows_frac")}
        if zstd_mask is not None:
            roofline["zstd_mask"] = {"gpoints_s": zstd_mask["gpoints_s"], "ratio": zstd_mask["ratio"],
                                     "class_words_ratio": zstd_mask["class_words_ratio"], "exact": zstd_mask["exact"],
                                     "mask_bytes_per_scan": zstd_mask["per_scan"]["zstd"]["mask_bytes_per_scan"],
                                     "class_words_mask_bytes_per_scan":
                                         zstd_mask["per_scan"]["class_words"]["mask_bytes_per_scan"]}
        if small is not None:
            roofline["small_stream"] = {"cold_gpoints_s": small["cold_gpoints_s"], "hot_gpoints_s": small["hot_gpoints_s"],
                                        "kernels_us_per_step": small["kernels_us_per_step"]}
        if e2e is not None and served is not None:
            e2e["served"] = {"p50_ms": served["p50_ms"], "p99_ms": served["p99_ms"], "gpoints_s": served["gpoints_s"],
                             "saturated_gpoints_s": served["saturated"]["gpoints_s"]}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "scans": T, "H": H, "W": W, "attributes": A, "seed": rank,
                           "raw_bytes_per_step": raw_bytes, "l2": "inputs larger than L2 (no flush)",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_n,
                "cpu_baseline_configs": cpu_cfg, "e2e": e2e,
                "clocks": clocks,
                "gpu_launches": 5 * args.steps * (2 if e2e else 1),
                "batched": batched, "served": served, "heuristic": heuristic, "precision": precision,
                "ablation": ablation, "standardize": standardize, "small_stream": small, "mask_codec": mask_codec,
                "zstd_mask": zstd_mask,
                "sweep": None if sweep is None else roofline["sweep"]["rows"], "sweep_detail": sweep,
                "batched_gpoints_s": None if batched is None else batched["gpoints_s"],
                "served_p50_ms": None if served is None else served["p50_ms"],
                "served_p99_ms": None if served is None else served["p99_ms"],
                "detail": {"kernels": kernels, "compression": modes, "stream_bytes": n,
                           "gsamples_s": value * A,
                           "encode_gpoints_s": px_step / (avg["k_trial"] + avg["k_encode"] + avg["k_finalize"]) / 1e6,
                           "decode_gpoints_s": px_step / avg["k_decode"] / 1e6,
                           "paper_context": "65 M points/s on one core of an i7-1250U @ 1.9 GHz (paper abstract)"}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
