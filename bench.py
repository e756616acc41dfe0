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


# Kernels launched per step (tpc_run_graph): grid 7 + 3 scans x 3 kernels,
# neighbours 1, links/tracklets 2 + 1 scan, follow 1, selection 5 + 1 scan,
# refit 3 + 1 scan.
KERNELS_PER_STEP = 7 + 9 + 1 + 2 + 3 + 1 + 5 + 3 + 3 + 3

# Algorithmic FP32 work of the Kalman kernels (counted from the source, per
# unit of the device work counters): a propagation with covariance transport
# (helix step, Jacobian, J C J^T on the packed triangle, compensated adds) is
# 170 flop, an FP32 update (gain, state, covariance, residuals) 150 flop, a
# candidate examined by the pick-up 10 flop.
FLOP_PROP, FLOP_UPD, FLOP_CAND = 170, 150, 10
# Algorithmic DRAM bytes per cluster of the memory-bound stages: grid 88
# (16 B read twice, 4 B rs, 8 B bin/slot written and read, scatter 4 B,
# order 16 B gather + 16 B writes), neighbours 33 (8 B own y/z, 8 B candidate
# re-reads, 8 B links + 1 B tie written, ~8 B bin starts).
BYTES_GRID, BYTES_NEIGH = 88, 33


def roofline(stages, work, counts, n):
    peaks, src = _peaks()
    dom = max(stages, key=stages.get)
    t = stages[dom] / 1e3
    if dom in ("follow", "refit"):
        flop = FLOP_PROP * work["prop"] + FLOP_UPD * work["upd32"] + FLOP_CAND * work["cand"]
        sm = 148
        peak = sm * 128 * 2 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
        ach = flop / t / 1e12
        return {"kernel": f"k_{dom}", "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None,
                "note": f"FP32 FMA peak 148 SM x 128 lanes x 2 x {peaks.get('sm_max_mhz', 2032.0)} MHz ({src} clock); "
                        "work counted by device counters; the follow stage includes both Kalman kernels' FP64 zones"}
    b = (BYTES_GRID if dom == "grid" else BYTES_NEIGH) * n
    ach = b / t / 1e9
    peak = peaks["hbm_gbs"]
    return {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "traffic": None}


def cpu_baseline(cl):
    """The FP64 oracle timed on this host's cores over the same event."""
    import oracle
    threads = os.cpu_count() or 1
    oracle.run(cl[:1000], threads=threads)
    times = []
    t_end = time.perf_counter() + 15.0
    while time.perf_counter() < t_end or not times:
        t0 = time.perf_counter()
        oracle.run(cl, threads=threads)
        times.append(time.perf_counter() - t0)
    return {"value": len(cl) * len(times) / sum(times), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"the full event ({len(cl)} clusters) x {len(times)} runs, all stages a2-a8"}


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

    # per-stage device time (CUDA events recorded by the library on its stream)
    trk.set_profiling(True)
    runs = []
    for _ in range(5):
        with torch.cuda.stream(stream):
            flush.zero_()
        trk.load(dev_in)
        trk.find().fit()
        trk.sync()
        runs.append(trk.stage_times())
    trk.set_profiling(False)
    stages = {k: statistics.median(r[k] for r in runs) for k in runs[0]}
    work = trk.work()
    roof = roofline(stages, work, counts, n)

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
            "gpu_launches": KERNELS_PER_STEP,
            "roofline": roof,
            "stages_ms": {k: round(v, 4) for k, v in stages.items()},
            "work": work,
            "peaks_source": src}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cl)
    if rank == 0:
        print(json.dumps(line))
    trk.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
