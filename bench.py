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

--impl reference times the oracle alone (the reference arm).
Multi-GPU (torchrun): independent replicas, one stream per GPU, no collective
on the data path; value = all ranks' pixels / max time.
"""
from __future__ import annotations

import argparse
import json
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


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", "clocks_rank%d.csv" % device_index)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [x for x in sm if x >= 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--scans", type=int, default=100, help="scans per step (100 = the benchmark workload)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

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

    def step(record):
        J.jiffy_stream_reset(enc)
        J.jiffy_stream_reset(dec)
        n, offs = J.jiffy_encode_seq(enc, scans, out, stream)
        te = J.jiffy_stream_kernel_times(enc)
        J.jiffy_decode_seq(dec, out, n, offs, outs, stream)
        td = J.jiffy_stream_kernel_times(dec)
        if record:
            ktimes["k_trial"].append(te[0])
            ktimes["k_encode"].append(te[1])
            ktimes["k_finalize"].append(te[2])
            ktimes["k_decode"].append(td[0])
        state["n"], state["offs"] = n, offs

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(False)
    # bit-exact check of the benchmarked configuration (outside the timed region)
    for a, (s, P) in enumerate(attrs):
        m = (1 << (8 * s)) - 1
        v = torch.stack([scans[t][a] for t in range(T)]).to(torch.int64) & m
        q = torch.clamp((v + P // 2) // P, max=m // P)
        if not torch.equal(outs[a].to(torch.int64) & m, q * P):
            raise SystemExit("round trip mismatch on attribute %d" % a)

    clk = Clocks(local)
    barrier()
    clk.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(True)
    ev1.record(stream)
    barrier()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    ms_step = ms / args.steps
    px_step = T * H * W
    value = px_step * world / (ms_step / 1e3) / 1e9
    n = state["n"]

    # e2e through host buffers: H2D scans, encode, D2H stream, H2D stream, decode, D2H scans
    host_in = [[p.cpu().pin_memory() for p in s] for s in scans]
    host_stream = torch.empty(cap, dtype=torch.uint8).pin_memory()
    host_out = [torch.empty_like(o, device="cpu").pin_memory() for o in outs]
    dev_in = [[torch.empty_like(p) for p in s] for s in scans]
    dev_stream = torch.empty(cap, dtype=torch.uint8, device=dev)

    def e2e_step():
        for hs, ds in zip(host_in, dev_in):
            for h, d in zip(hs, ds):
                d.copy_(h, non_blocking=True)
        J.jiffy_stream_reset(enc)
        J.jiffy_stream_reset(dec)
        nn, offs = J.jiffy_encode_seq(enc, dev_in, out, stream)
        host_stream[:nn].copy_(out[:nn], non_blocking=True)
        dev_stream[:nn].copy_(host_stream[:nn], non_blocking=True)
        J.jiffy_decode_seq(dec, dev_stream, nn, offs, outs, stream)
        for h, o in zip(host_out, outs):
            h.copy_(o, non_blocking=True)
        return nn

    e2e = None
    if not args.no_e2e:
        for _ in range(2):
            e2e_step()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            nn = e2e_step()
        e1.record(stream)
        barrier()
        e2e_ms = e0.elapsed_time(e1) / args.steps
        if world > 1:
            t = torch.tensor([e2e_ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())
        e2e = {"value": px_step * world / (e2e_ms / 1e3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": raw_bytes + nn, "d2h_bytes_per_step": nn + raw_bytes}

    # roofline of the dominant kernel: algorithmic bytes / CUDA-event duration
    avg = {k: statistics.mean(v) for k, v in ktimes.items()}
    algo = {"k_encode": raw_bytes + n, "k_decode": n + raw_bytes}
    dom = max(("k_encode", "k_decode"), key=lambda k: avg[k])
    peak, src = peaks()
    achieved = algo[dom] / (avg[dom] / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": src, "traffic": None,
                "algorithmic_bytes_per_launch": algo[dom]}
    kernels = {k: {"avg_ms": avg[k], "GBps": (algo[k] / (avg[k] / 1e3) / 1e9) if k in algo else None,
                   "frac_of_peak": (algo[k] / (avg[k] / 1e3) / 1e9 / peak) if k in algo else None}
               for k in avg}

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline(cfg, attrs, scans)
        modes = {"ratio": raw_bytes / n}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "scans": T, "H": H, "W": W, "attributes": A,
                           "raw_bytes_per_step": raw_bytes, "l2": "inputs larger than L2 (no flush)",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": 4 * args.steps * (2 if e2e else 1),
                "detail": {"kernels": kernels, "compression": modes, "stream_bytes": n,
                           "encode_gpoints_s": px_step / (avg["k_trial"] + avg["k_encode"] + avg["k_finalize"]) / 1e6,
                           "decode_gpoints_s": px_step / avg["k_decode"] / 1e6,
                           "paper_context": "65 M points/s on one core of an i7-1250U @ 1.9 GHz (paper abstract)"}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
