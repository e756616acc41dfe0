"""Benchmark of the B300 sector tracker.

Default workload: one central Pb-Pb-like event (36 sectors, 8000 primaries +
1600 secondaries, seed 1, ~1.0 M clusters).  A step is one pass of the whole
hot path (load from a device-resident buffer, grid, CA links, tracklets,
Kalman following, selection, refit) over that event.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "clusters/s tracked on 1 B300"
UNIT = "clusters/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_reference(args):
    """The oracle (plain FP64 C, all host cores) on the same workload."""
    import numpy as np

    import oracle
    import synth
    ev = synth.central_event(seed=1)
    n = len(ev.clusters)
    threads = os.cpu_count() or 1
    oracle.run(ev.clusters, threads=threads)  # build + warm
    for _ in range(args.warmup):
        pass
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(ev.clusters, threads=threads)
        times.append(time.perf_counter() - t0)
    v = n * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "central Pb-Pb-like event, 36 sectors, seed 1",
                                            "clusters": n},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"full event ({n} clusters) x {args.steps} runs"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import numpy as np
    import torch

    import paper_1709_00618_b300 as tpc
    import synth

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ev = synth.central_event(seed=1 + rank)
    cl = ev.clusters
    n = len(cl)
    stream = torch.cuda.Stream()
    trk = tpc.Tracker(device=local, stream=stream, arena="torch", arena_clusters=n)
    dev_in = torch.from_numpy(cl.view(np.uint8)).to(f"cuda:{local}")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=f"cuda:{local}")

    def step_device():
        trk.load(dev_in)
        trk.run_graph()

    for _ in range(max(args.warmup, 3)):
        step_device()
    trk.sync()
    torch.cuda.synchronize()
    times = []
    with ClockSampler(local) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step_device()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        torch.cuda.synchronize()
    t_step = sum(times) / len(times)
    if world > 1:
        tt = torch.tensor([t_step], device=f"cuda:{local}")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_step = float(tt.item())
    counts = trk.counts()
    tracks, ct, _ = trk.get()

    # end to end through the public API: pinned host input -> tracks + assignment on the host
    pinned = torch.from_numpy(cl.view(np.uint8)).pin_memory()
    host_in = pinned.numpy().view(synth.CLUSTER_DTYPE)
    e2e = []
    for i in range(max(args.warmup, 3) + args.steps):
        t0 = time.perf_counter()
        trk.load(host_in)
        trk.run_graph()
        tr, c2, _ = trk.get()
        if i >= max(args.warmup, 3):
            e2e.append(time.perf_counter() - t0)
    e2e_t = sum(e2e) / len(e2e)

    peaks, src = _peaks()
    line = {"metric": METRIC, "value": world * n / t_step, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "central Pb-Pb-like event, 36 sectors, 8000+1600 tracks, seed 1",
                       "clusters": n, "tracklets": counts["n_tracklets"], "tracks": counts["n_tracks"],
                       "l2": "flushed (256 MB write) between steps", "graph": True},
            "clocks": clk.summary(),
            "e2e": {"value": world * n / e2e_t, "unit": UNIT, "h2d_bytes_per_step": 16 * n,
                    "d2h_bytes_per_step": 128 * len(tr) + 4 * n},
            "peaks_source": src}
    if rank == 0:
        print(json.dumps(line))
    trk.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
