"""Benchmark of the B300 sector tracker.

Default workload: a 10 ms continuous-readout timeframe at 50 kHz (about 500
Pb-Pb collisions, z from drift time, seed 2, ~90 M clusters), the largest
configuration that fits one GPU.  A step is one pass of the whole hot path
(load from a device-resident buffer, grid, CA links, tracklets, Kalman
following, selection, refit) over that timeframe.  Prints one JSON line;
the central Pb-Pb-like event, tracking time against input size, batching
and serving legs and the oracle's CPU baseline are extra keys of it.
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


# Algorithmic work of the Kalman kernels, counted from the source per unit of
# the device work counters (an FMA counts 2, an add, multiply, divide or
# square root 1):
#   helix step of the state with its Jacobian, binary32        67
#   covariance transport J C J^T (42 FMA on the packed triangle)  84
#   Kalman update, gain and covariance, binary32 (2x2 inverse)  99
#   Kalman update, gain and covariance, binary64 (a y and a z
#     scalar downdate: 2 adds, 2 reciprocals, 10 mul, 30 FMA)     74
#   Kalman update, residuals, state and chi2 (binary32)          56
#   candidate cluster examined by the gated pick-up              10
# FP32-zone work is all binary32; in the FP64 zone the transport and the
# covariance part of the update run in binary64.
FLOP_STATE, FLOP_TRANSPORT, FLOP_UPD_COV, FLOP_UPD_COV64, FLOP_UPD_STATE, FLOP_CAND = 67, 84, 99, 74, 56, 10
# Algorithmic DRAM bytes per cluster of the memory-bound stages: grid 44
# (the 16 B record read, 16 B of sorted output -- y/z, row-sector, input
# index -- written, a 4 B bin index written and half of the records read
# again), neighbours 45 (own y/z 8 B and row-sector 4 B, the two
# neighbouring rows' y/z read once each 16 B, about two bin starts 8 B, up,
# down and tie written 9 B).
BYTES_GRID, BYTES_NEIGH = 44, 45
# Nominal issue rates per SM and clock: 128 FP32 lanes (an FMA is 2 flop)
# and, on B300, 2 FP64 FMA units; the roofline uses the measured probe.
FP32_FLOP_PER_CLK_SM, FP64_FLOP_PER_CLK_SM, N_SM = 256, 4, 148


# The sources of the tracking path's kernels (the ones the traffic capture covers).
PATH_KERNEL_SOURCES = ("common.cuh", "scan.cuh", "grid.cuh", "links.cuh", "kalman.cuh", "order.cuh", "follow.cuh",
                       "select.cuh")


def _source_hash():
    """sha256 of the path's kernel sources with their comments and blank
    lines left out, so that a traffic file taken on them stays valid across
    edits of the comments alone."""
    import hashlib
    import re
    m = hashlib.sha256()
    for f in PATH_KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1709_00618_b300", "csrc", f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        lines = (re.sub(r"//.*$", "", ln).rstrip() for ln in src.splitlines())
        m.update("\n".join(ln for ln in lines if ln).encode())
    return m.hexdigest()


TRAFFIC_FILES = {"central": "kernel_traffic_central_event.txt", "timeframe": "kernel_traffic_timeframe_10ms.txt"}


def ncu_traffic(workload: str):
    """DRAM bytes per launch of each profiled kernel from the committed ncu
    summary of this workload, or {} when there is none or the kernels changed
    since it was taken."""
    if workload == CONFIG2:
        key = "central"
    elif workload == CONFIG3:
        key = "timeframe"
    else:
        return {}
    path = os.path.join(ROOT, "profiles", TRAFFIC_FILES[key])
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return {}
    tag = next((ln for ln in lines if ln.startswith("# sources:")), "")
    if not tag.endswith(_source_hash()):
        return {}
    out = {}
    for ln in lines:
        if ln and not ln.startswith("#"):
            name, rd, wr = ln.split()[:3]
            out[name] = (float(rd) + float(wr)) * 1e6
    return out


def kalman_flops(w):
    """(binary32 flop, binary64 flop) of one Kalman kernel's work counters."""
    p32 = w["prop"] - w["prop64"]
    f32 = (FLOP_STATE + FLOP_TRANSPORT) * p32 + FLOP_STATE * w["prop64"] + \
        (FLOP_UPD_COV + FLOP_UPD_STATE) * w["upd32"] + FLOP_UPD_STATE * w["upd64"] + FLOP_CAND * w["cand"]
    f64 = FLOP_TRANSPORT * w["prop64"] + FLOP_UPD_COV64 * w["upd64"]
    return f32, f64


def kernel_rooflines(stages, kalman, n, alu):
    """Roofline entry per timed kernel (Kalman kernels one by one, the
    neighbour kernel, the grid stage as a whole); the largest is the
    dominant kernel.  alu: the measured FMA-pipe rates (TFLOP/s)."""
    peaks, src = _peaks()
    p32, p64 = alu["fp32_tflops"], alu["fp64_tflops"]
    out = {}
    import paper_1709_00618_b300 as tpc
    for name, d in kalman.items():
        if d["prop"] == 0 or d["ms"] <= 0:
            continue  # not launched at this input size
        t = d["ms"] / 1e3
        f32, f64 = kalman_flops(d)
        zone = name in tpc.Tracker.ZONE_KERNELS
        if zone:
            ach = f64 / t / 1e12
            e = {"bound": "alu", "achieved": ach, "peak": p64, "unit": "TFLOP/s (FP64)", "frac": ach / p64,
                 "fp32_tflops": f32 / t / 1e12}
        else:
            ach = f32 / t / 1e12
            e = {"bound": "alu", "achieved": ach, "peak": p32, "unit": "TFLOP/s (FP32)", "frac": ach / p32}
        e["ms"] = d["ms"]
        e["work"] = {k: d[k] for k in ("prop", "upd32", "upd64", "cand", "prop64")}
        out[name] = e
    for name, ms, per in (("k_neighbours", stages["neighbours"], BYTES_NEIGH), ("grid stage", stages["grid"],
                                                                                  BYTES_GRID)):
        ach = per * n / (ms / 1e3) / 1e9
        out[name] = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": ach / peaks["hbm_gbs"], "ms": ms, "bytes_per_cluster": per}
    return out, src


def roofline(stages, kalman, n, alu, clocks, traffic=None):
    table, src = kernel_rooflines(stages, kalman, n, alu)
    dom = max((k for k in table if k != "grid stage"), key=lambda k: table[k]["ms"])
    e = dict(table[dom])
    mhz = clocks.get("sm_mhz") or 2032.0
    line = {"kernel": dom, "bound": e["bound"], "achieved": e["achieved"], "peak": e["peak"], "unit": e["unit"],
            "frac": e["frac"], "traffic": (traffic or {}).get(dom), "ms": e["ms"],
            "peak_source": f"ALU: measured FMA-pipe probe (tpc_measure_alu_peaks: FP32 {alu['fp32_tflops']:.1f}, "
                           f"FP64 {alu['fp64_tflops']:.2f} TFLOP/s; nominal at the sampled {mhz:.0f} MHz: FP32 "
                           f"{N_SM * FP32_FLOP_PER_CLK_SM * mhz * 1e6 / 1e12:.1f}, FP64 "
                           f"{N_SM * FP64_FLOP_PER_CLK_SM * mhz * 1e6 / 1e12:.2f}); HBM: {src} copy bandwidth"}
    return line, table


def cpu_sample(cl, workload):
    """A bounded sample of the workload for the oracle: the whole input up
    to 1.5 M clusters, else the clusters of sectors 0 and 18 (one sector per
    side), a labelled subset."""
    import numpy as np
    if len(cl) <= 1_500_000:
        return cl, f"the whole input ({len(cl)} clusters)"
    sub = cl[np.isin(cl["sector"], (0, 18))]
    return sub, f"sectors 0 and 18 of the {workload} ({len(sub)} of {len(cl)} clusters), all stages a2-a8"


def cpu_baseline(cl, workload, seconds=15.0):
    """The FP64 oracle, as it stands, timed on this host's cores over a
    bounded sample of the same workload (repeated for about `seconds`), and
    on one core over part of it."""
    import numpy as np

    import oracle
    threads = os.cpu_count() or 1
    sub, label = cpu_sample(cl, workload)
    oracle.run(sub[:1000], threads=threads)
    times = []
    t_end = time.perf_counter() + seconds
    while time.perf_counter() < t_end or not times:
        t0 = time.perf_counter()
        oracle.run(sub, threads=threads)
        times.append(time.perf_counter() - t0)
    one = sub[np.isin(sub["sector"], (0, 1, 2, 18, 19, 20))][:500_000]
    t0 = time.perf_counter()
    oracle.run(one, threads=1)
    one_rate = len(one) / (time.perf_counter() - t0)
    return {"value": len(sub) * len(times) / sum(times), "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{label} x {len(times)} runs",
            "one_core": {"value": one_rate, "sample": f"{len(one)} clusters of that sample, 1 thread"}}


def _entropy(v):
    """Shannon entropy (bits per symbol) of an integer sample."""
    import numpy as np
    if len(v) == 0:
        return 0.0
    _, c = np.unique(v, return_counts=True)
    p = c / c.sum()
    return float(-(p * np.log2(p)).sum())


def all_configs(local):
    """Per-config table (one sector, central event, 10 ms timeframe): GPU
    device throughput (graph, inputs resident, L2 flushed), per-call latency
    through the public API from page-locked host memory to results on the
    host, and the oracle on one core and on all cores (the timeframe on a
    subset of its sectors)."""
    import numpy as np
    import torch

    import oracle
    import paper_1709_00618_b300 as tpc
    import synth
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")
    cores = os.cpu_count() or 1
    rows = {}
    cases = [("config 1: one sector, 400 tracks, seed 0", lambda: synth.one_sector(seed=0).clusters, 50, None),
             ("config 2: central Pb-Pb-like event, seed 1", lambda: synth.central_event(seed=1).clusters, 20,
              None),
             ("config 3: 10 ms timeframe at 50 kHz, seed 2", lambda: synth.timeframe(seed=2, length_ms=10.0).clusters,
              3, (0, 18))]
    for name, gen, reps, subset in cases:
        cl = gen()
        n = len(cl)
        stream = torch.cuda.Stream()
        trk = tpc.Tracker(device=local, stream=stream)
        dev = torch.from_numpy(cl.view(np.uint8)).to(f"cuda:{local}")
        for _ in range(3):
            trk.load(dev).run_graph()
        trk.sync()
        dt = []
        for _ in range(reps):
            with torch.cuda.stream(stream):
                flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            trk.load(dev).run_graph()
            e1.record(stream)
            e1.synchronize()
            dt.append(e0.elapsed_time(e1))
        counts = trk.counts()
        vtx = None
        if subset is not None:  # a timeframe: vertex finding in the drift time on its tracks
            trk.find_vertices().vertices()
            vt = []
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                trk.find_vertices()
                e1.record(stream)
                e1.synchronize()
                vt.append(e0.elapsed_time(e1))
            vres = trk.vertices()
            vms = statistics.median(vt)
            # algorithmic bytes per track: the 128-byte track read twice (time
            # estimate, conversion) and 24 B of per-track outputs and scratch
            vtx = {"ms": vms, "vertices": int(len(vres["vertices"])),
                   "tracks_with_vertex": int((vres["track_vertex"] >= 0).sum()),
                   "tracks_per_s": counts["n_tracks"] / (vms / 1e3),
                   "hbm_gbs": counts["n_tracks"] * (2 * 128 + 24) / (vms / 1e3) / 1e9}
        merged = None
        if n > 100_000:  # second tracking phase: merging sector segments
            trk.merge()
            mt = []
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                trk._ck(trk._lib.tpc_merge_tracks(trk._ctx, None))
                e1.record(stream)
                e1.synchronize()
                mt.append(e0.elapsed_time(e1))
            mg = trk.merge()
            merged = {"ms": statistics.median(mt), "merged_tracks": int(len(mg["merged"])),
                      "segments_merged": int((mg["chain"] >= 0).sum()), "segments": int(counts["n_tracks"])}
        codec = None
        if n > 100_000:  # track-model compression of the event / timeframe
            trk.compress(0.01)
            ct_ms = []
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                trk._ck(trk._lib.tpc_compress(trk._ctx, 0.01))
                e1.record(stream)
                e1.synchronize()
                ct_ms.append(e0.elapsed_time(e1))
            c = trk.compress(0.01)
            t0 = time.perf_counter()
            qy, qz = trk.decompress(c["heads"], c["rows"], c["res_y"], c["res_z"], 0.01)
            dec_s = time.perf_counter() - t0
            ok = np.repeat(c["heads"]["ok"].astype(bool), c["heads"]["n_clusters"])
            first = np.zeros(len(ok), bool)
            first[np.concatenate([[0], np.cumsum(c["heads"]["n_clusters"])[:-1]])[c["heads"]["n_clusters"] > 0]] = True
            steps = (c["rows"][:-1].astype(np.int64) - c["rows"][1:])[~first[1:]]
            coded = _entropy(c["res_y"][ok]) + _entropy(c["res_z"][ok]) + _entropy(steps)
            fixed = _entropy(c["q_y"][ok]) + _entropy(c["q_z"][ok])
            head_bits = 32 * 5 + 8 + 8  # state, first row, cluster count per track
            n_ok = int(ok.sum())
            codec = {"encode_ms": statistics.median(ct_ms), "decode_api_ms": 1e3 * dec_s,
                     "round_trip_exact": bool(np.array_equal(qy, c["q_y"]) and np.array_equal(qz, c["q_z"])),
                     "track_clusters": int(len(ok)), "coded_clusters": n_ok,
                     "bits_per_cluster_coded": coded + head_bits * int(c["heads"]["ok"].sum()) / max(n_ok, 1),
                     "bits_per_cluster_fixed_point": fixed,
                     "unit_cm": 0.01}
            codec["factor"] = codec["bits_per_cluster_fixed_point"] / codec["bits_per_cluster_coded"]
        host = torch.from_numpy(cl.view(np.uint8)).pin_memory().numpy().view(synth.CLUSTER_DTYPE)
        tr_buf = torch.zeros(counts["n_tracks"] + 1024, 128, dtype=torch.uint8).pin_memory()
        ct_buf = torch.zeros(n, dtype=torch.int32).pin_memory()
        lat = []
        for i in range(reps + 2):
            t0 = time.perf_counter()
            trk.load(host).run_graph()
            trk.get_into(tr_buf, ct_buf)
            if i >= 2:
                lat.append(1e3 * (time.perf_counter() - t0))
        trk.close()
        del dev
        sub = cl if subset is None else cl[np.isin(cl["sector"], subset)]
        t0 = time.perf_counter()
        oracle.run(sub, threads=cores)
        t_all = time.perf_counter() - t0
        one = sub if subset is None else sub[sub["sector"] == subset[0]]
        one = one[: min(len(one), 500_000)]
        t0 = time.perf_counter()
        oracle.run(one, threads=1)
        t_one = time.perf_counter() - t0
        rows[name] = {"clusters": n, "tracks": counts["n_tracks"], "tracklets": counts["n_tracklets"],
                      "gpu_device_clusters_per_s": n / (statistics.median(dt) / 1e3),
                      "gpu_device_ms": statistics.median(dt),
                      "gpu_api_latency_ms_p50": _pct(lat, 50), "gpu_api_latency_ms_p99": _pct(lat, 99),
                      "oracle_all_cores_clusters_per_s": len(sub) / t_all, "oracle_cores": cores,
                      "oracle_all_cores_sample": "all sectors" if subset is None else f"sectors {subset}",
                      "oracle_one_core_clusters_per_s": len(one) / t_one,
                      "oracle_one_core_sample": f"{len(one)} clusters"}
        if vtx is not None:
            rows[name]["vertex_finding"] = vtx
        if codec is not None:
            rows[name]["track_model_compression"] = codec
        if merged is not None:
            rows[name]["sector_merging"] = merged
    rows["cluster rejection: central event with loopers, seed 1"] = cluster_rejection(local, flush)
    print(json.dumps({"all_configs": rows}))


def events_through_server(host_in, n, local, events=16, slots=4):
    """The same event as a stream through the serving API (tpc_server_*):
    `slots` events in flight, each copied in from page-locked host memory
    and its tracks and cluster assignment copied back into page-locked
    buffers; wall time from the first submission to the last result.  One
    event alone is bound by its longest tracklet; several in flight fill the
    GPU (the paper runs several events at once for the same reason)."""
    import numpy as np
    import torch

    import paper_1709_00618_b300 as tpc
    ring = slots + 2
    with tpc.Server(device=local, max_slots=slots) as srv:
        bufs = [(torch.zeros(n // 10 + 4096, 128, dtype=torch.uint8).pin_memory(),
                 torch.zeros(n, dtype=torch.int32).pin_memory()) for _ in range(ring)]

        def run(first, count):
            nxt, done, inflight, tracks = 0, 0, [], 0
            while done < count:
                while nxt < count and len(inflight) < ring:
                    if srv.submit(first + nxt, host_in, *bufs[nxt % ring]) != 0:
                        break
                    inflight.append(first + nxt)
                    nxt += 1
                r = srv.result(inflight[0])
                if r is None:
                    time.sleep(5e-5)
                    continue
                tracks = len(r[0])
                inflight.pop(0)
                done += 1
            return tracks

        run(0, ring)  # warm-up: arenas, graphs
        t0 = time.perf_counter()
        tracks = run(1000, events)
        dt = time.perf_counter() - t0
    return {"value": events * n / dt, "unit": UNIT, "events": events, "slots": slots,
            "ms_per_event": 1e3 * dt / events, "h2d_bytes_per_event": 16 * n,
            "d2h_bytes_per_event": 128 * tracks + 4 * n}


def cluster_rejection(local, flush):
    """Cluster rejection on the central event with loopers (|eta| < 1.5,
    pT from 40 MeV/c, low-momentum secondaries, loopers over four
    half-turns): time of tpc_reject_clusters on the fitted tracks, the
    rejected fractions, and the entropy-coded size of the track clusters
    (track-model residuals, row steps and headers) with and without the
    rejected tracks."""
    import numpy as np
    import torch

    import paper_1709_00618_b300 as tpc
    import synth
    cl = synth.looper_event(seed=1).clusters
    stream = torch.cuda.Stream()
    trk = tpc.Tracker(device=local, stream=stream)
    dev = torch.from_numpy(cl.view(np.uint8)).to(f"cuda:{local}")
    trk.load(dev).run_graph()
    res = trk.reject()
    rt = []
    for _ in range(5):
        with torch.cuda.stream(stream):
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        trk._ck(trk._lib.tpc_reject_clusters(trk._ctx, None))
        e1.record(stream)
        e1.synchronize()
        rt.append(e0.elapsed_time(e1))
    c = trk.compress(0.01)
    counts = trk.counts()
    trk.close()
    h = c["heads"]
    nc = h["n_clusters"].astype(np.int64)
    kept_track = res["track_class"][: len(h)] == 0
    first = np.zeros(int(nc.sum()), bool)
    first[np.concatenate([[0], np.cumsum(nc)[:-1]])[nc > 0]] = True
    steps = np.zeros(len(first), np.int64)
    steps[1:] = c["rows"][:-1].astype(np.int64) - c["rows"][1:]

    def bits(track_mask):
        cm = np.repeat(track_mask, nc)
        ok = cm & np.repeat(h["ok"].astype(bool), nc)
        raw = cm & ~ok
        coded = (_entropy(c["res_y"][ok]) + _entropy(c["res_z"][ok]) + _entropy(steps[ok & ~first])) * ok.sum()
        fixed = (_entropy(c["q_y"][raw]) + _entropy(c["q_z"][raw])) * raw.sum()
        return coded + fixed + (32 * 5 + 8 + 8) * int(track_mask.sum())

    b_all, b_kept = bits(np.ones(len(h), bool)), bits(kept_track)
    cnt = res["counts"]
    n = len(cl)
    return {"clusters": n, "tracks": int(counts["n_tracks"]), "reject_ms": statistics.median(rt),
            "tracks_per_s": counts["n_tracks"] / (statistics.median(rt) / 1e3),
            "rejected_fraction": cnt["all"] / n,
            "rejected_fraction_of_track_clusters": cnt["all"] / max(int(nc.sum()), 1),
            "by_class_fraction": {k: cnt[k] / n for k in ("low_p", "inclined", "looper_leg")},
            "coded_bits_track_clusters": b_all, "coded_bits_after_rejection": b_kept,
            "compression_gain_from_rejection": b_all / max(b_kept, 1.0)}


def run_reference(args):
    """The reference arm: the FP64 oracle (plain C, all host cores), as it
    stands, on the main line's workload; each step runs it over the same
    bounded sample as the CPU baseline (the oracle over 90 M clusters would
    take minutes per step)."""
    import oracle
    ev, workload = workload_of(args, 0)
    cl = ev.clusters
    sub, label = cpu_sample(cl, workload)
    threads = os.cpu_count() or 1
    oracle.run(sub[:1000], threads=threads)
    for _ in range(args.warmup):
        oracle.run(sub[:20000], threads=threads)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.run(sub, threads=threads)
        times.append(time.perf_counter() - t0)
    v = len(sub) * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload, "clusters": len(cl)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{label}, one oracle run per step x {args.steps} steps"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def combine_ranks(t_step, n_clusters, world, device):
    """Replicas: the job's step time is the slowest rank's, its work the sum
    of every rank's clusters (each rank tracks its own event).  Returns
    (max step time, total clusters)."""
    if world <= 1:
        return t_step, n_clusters
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_step], dtype=torch.float64, device=device)
    c = torch.tensor([float(n_clusters)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(c.item())


def _pct(v, q):
    import numpy as np
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else None


def batching_leg(local, flush, n_requests=256, reps=3):
    """256 independent requests of uneven size (1-36 sectors of events with
    50-8000 tracks, log-uniform) as one batch in one graph launch, against
    the same requests as separate plain launches one after the other.
    Inputs are resident on the device; the L2 is flushed before each run.
    Latency of a request: from the start of the run to the completion of its
    results on the device (all requests are there at the start)."""
    import numpy as np
    import torch

    import paper_1709_00618_b300 as tpc
    import synth
    reqs = synth.batch_requests(seed=3, n_requests=n_requests)
    sizes = np.array([len(r.clusters) for r in reqs], np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    cl = np.concatenate([r.clusters for r in reqs])
    dev = torch.from_numpy(cl.view(np.uint8)).to(f"cuda:{local}")
    views = [dev[16 * off[i]:16 * off[i + 1]] for i in range(n_requests)]
    stream = torch.cuda.Stream()
    out = {"workload": f"{n_requests} requests, 1-36 sectors of events with 50-8000 tracks (log-uniform), seed 3",
           "clusters": int(off[-1]), "request_clusters_p50": int(np.median(sizes)),
           "request_clusters_max": int(sizes.max())}

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.zero_()

    # batched: one context, one load, one graph launch; shapes by the autotuner
    bt = tpc.Tracker(device=local, stream=stream)
    bt.load(dev, off)
    choice, tuned_ms = bt.autotune(reps=3)
    out["autotuned"] = dict(choice, ms=tuned_ms)
    for _ in range(3):
        bt.load(dev, off)
        bt.run_graph()
    bt.sync()
    times = []
    for _ in range(reps):
        flush_l2()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.load(dev, off)
        bt.run_graph()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    bt.sync()
    t_b = statistics.median(times)
    out["batched"] = {"clusters_per_s": off[-1] / (t_b / 1e3), "ms": t_b, "launches": 1,
                      "kernels": bt.graph_kernels(), "latency_ms_p50": t_b, "latency_ms_p99": t_b}
    bt.close()

    # plain: one context, each request loaded, found and fitted on its own
    pt = tpc.Tracker(device=local, stream=stream)
    pt.reserve(n_clusters=int(sizes.max()), n_requests=1)
    for i in range(min(8, n_requests)):
        pt.load(views[i]).find().fit()
    pt.sync()
    tot, lat_all = [], []
    for _ in range(reps):
        flush_l2()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_requests + 1)]
        ev[0].record(stream)
        for i in range(n_requests):
            pt.load(views[i]).find().fit()
            ev[i + 1].record(stream)
        ev[-1].synchronize()
        lat = [ev[0].elapsed_time(ev[i + 1]) for i in range(n_requests)]
        tot.append(lat[-1])
        lat_all.append(lat)
    pt.sync()
    k = int(np.argsort(tot)[len(tot) // 2])
    t_p = tot[k]
    out["plain"] = {"clusters_per_s": off[-1] / (t_p / 1e3), "ms": t_p, "launches": n_requests,
                    "latency_ms_p50": _pct(lat_all[k], 50), "latency_ms_p99": _pct(lat_all[k], 99)}
    pt.close()
    out["batched_over_plain"] = out["batched"]["clusters_per_s"] / out["plain"]["clusters_per_s"]
    return out


def _generate_pool(seed, n_distinct, min_ms, max_ms, out_dir):
    """Child process: the serving pool's timeframes, saved as .npy files."""
    import numpy as np

    import synth
    rng = np.random.default_rng(seed)
    lengths = [float(rng.uniform(min_ms, max_ms)) for _ in range(n_distinct)]
    for i, ms in enumerate(lengths):
        cl = synth.timeframe(seed=seed * 1000 + i, length_ms=ms).clusters
        np.save(os.path.join(out_dir, f"tf{i:03d}.npy"), cl)
        with open(os.path.join(out_dir, f"tf{i:03d}.ms"), "w") as f:
            f.write(repr(ms))


class ServingPool:
    """Distinct seeded timeframes (lengths uniform in [min_ms, max_ms], the
    config-5 generator) made by a spawned child process while the bench's
    GPU legs run; load() waits for them."""

    def __init__(self, seed=4, n_distinct=16, min_ms=1.0, max_ms=20.0):
        import multiprocessing as mp
        import tempfile
        self.seed, self.n = seed, n_distinct
        base = "/dev/shm" if os.path.isdir("/dev/shm") else None
        self.dir = tempfile.mkdtemp(prefix="tpc_pool_", dir=base)
        self.proc = mp.get_context("spawn").Process(target=_generate_pool,
                                                    args=(seed, n_distinct, min_ms, max_ms, self.dir))
        self.proc.start()
        self.t0 = time.perf_counter()

    def load(self):
        """[(clusters, length_ms)] in pool order; removes the files."""
        import shutil

        import numpy as np
        self.proc.join()
        if self.proc.exitcode != 0:
            raise RuntimeError("timeframe pool generation failed")
        gen_s = time.perf_counter() - self.t0
        out = []
        for i in range(self.n):
            cl = np.load(os.path.join(self.dir, f"tf{i:03d}.npy"))
            with open(os.path.join(self.dir, f"tf{i:03d}.ms")) as f:
                out.append((cl, float(f.read())))
        shutil.rmtree(self.dir, ignore_errors=True)
        return out, gen_s


def serving_leg(local, pool, n_arrivals=500, loads=(0.5, 0.8, 1.0), headline=0.8, other_arrivals=64, slots=6,
                budget_gb=120.0, ring=8, seed=4):
    """Poisson stream of continuous-readout timeframes (lengths uniform in
    1-20 ms at 50 kHz) through the continuous-batching server, against
    sequential plain processing of the same stream, at several offered
    loads (arrival rate = load x the sequential plain capacity, measured
    first).  Arrivals replay a pool of distinct seeded timeframes (a
    ServingPool); the headline load takes n_arrivals arrivals, the others
    other_arrivals.  Inputs and result buffers are page-locked host memory in
    both arms (`ring` result buffers for the server: a request waits for a
    free one).  Latency: arrival to results (tracks and cluster assignment)
    in host memory."""
    import numpy as np
    import torch

    import paper_1709_00618_b300 as tpc
    import synth
    tfs, gen_s = pool.load()
    pinned = [torch.from_numpy(cl.view(np.uint8)).pin_memory() for cl, _ in tfs]
    lengths = [ms for _, ms in tfs]
    del tfs
    host = [p.numpy().view(synth.CLUSTER_DTYPE) for p in pinned]
    sizes = [len(h) for h in host]
    npool = len(host)

    # sequential plain service time of each pool entry (after one warm run)
    trk = tpc.Tracker(device=local)
    trk.reserve(n_clusters=max(sizes), n_requests=1)
    n_tracks, serv = [], []
    big_ct = torch.zeros(max(sizes), dtype=torch.int32).pin_memory()
    tr_buf = torch.zeros(max(sizes) // 10 + 1, 128, dtype=torch.uint8).pin_memory()
    for h in host:
        tr, _ = trk.track_into(h, tr_buf, big_ct[:len(h)])
        n_tracks.append(len(tr))
        t0 = time.perf_counter()
        trk.track_into(h, tr_buf, big_ct[:len(h)])
        serv.append(time.perf_counter() - t0)
    cap = int(1.25 * max(n_tracks)) + 1024
    bufs = [(torch.zeros(cap, 128, dtype=torch.uint8).pin_memory(),
             torch.zeros(max(sizes), dtype=torch.int32).pin_memory()) for _ in range(ring)]

    def plain_arm(order, arrivals):
        lat = []
        t_start = time.perf_counter()
        for k in range(len(order)):
            now = time.perf_counter() - t_start
            if now < arrivals[k]:
                time.sleep(arrivals[k] - now)
            h = host[order[k]]
            trk.track_into(h, tr_buf, big_ct[:len(h)])
            lat.append(time.perf_counter() - t_start - arrivals[k])
        return lat, time.perf_counter() - t_start

    def served_arm(order, arrivals):
        # latency = (submission - arrival) + the server's submission-to-results time
        free = list(range(ring))
        srv = tpc.Server(device=local, max_slots=slots, hbm_budget=int(budget_gb * 2**30))
        lat, late, owner, pending = [], {}, {}, set()
        t_start = time.perf_counter()
        k, m = 0, len(order)
        while k < m or pending:
            now = time.perf_counter() - t_start
            while k < m and arrivals[k] <= now and free:
                b = free.pop()
                h = host[order[k]]
                if srv.submit(k, pinned[order[k]], tracks_out=bufs[b][0], cluster_track_out=bufs[b][1][:len(h)]):
                    free.append(b)
                    break
                late[k] = time.perf_counter() - t_start - arrivals[k]
                owner[k] = b
                pending.add(k)
                k += 1
            for j in sorted(pending):
                r = srv.result(j)
                if r is not None:
                    lat.append(late[j] + r[2][2] / 1e3)
                    pending.discard(j)
                    free.append(owner.pop(j))
            time.sleep(0.0002)
        span = time.perf_counter() - t_start
        st = srv.stats()
        srv.close()
        return lat, span, st

    by_load = {}
    for li, load in enumerate(loads):
        m = n_arrivals if load == headline else other_arrivals
        rng = np.random.default_rng(seed + 1 + li)
        order = rng.integers(0, npool, size=m)
        mean_s = float(np.mean([serv[i] for i in order]))
        arrivals = np.cumsum(rng.exponential(1.0, size=m)) * (mean_s / load)
        arrivals -= arrivals[0]
        total = int(sum(sizes[i] for i in order))
        lat_p, span_p = plain_arm(order, arrivals)
        lat_s, span_s, st = served_arm(order, arrivals)
        by_load[str(load)] = {
            "arrivals": m, "arrival_rate_hz": load / mean_s, "clusters": total,
            "plain": {"latency_ms_p50": 1e3 * _pct(lat_p, 50), "latency_ms_p99": 1e3 * _pct(lat_p, 99),
                      "clusters_per_s": total / span_p, "samples": len(lat_p)},
            "served": {"latency_ms_p50": 1e3 * _pct(lat_s, 50), "latency_ms_p99": 1e3 * _pct(lat_s, 99),
                       "clusters_per_s": total / span_s, "peak_running": st["peak_running"],
                       "arena_gb": st["arena_bytes"] / 2**30, "samples": len(lat_s)}}
    trk.close()
    head = by_load[str(headline)]
    return {"workload": f"Poisson stream of timeframes drawn from {npool} distinct seeded timeframes of 1-20 ms "
                        f"at 50 kHz (seed {seed}); {n_arrivals} arrivals at the headline load {headline} of the "
                        f"sequential plain capacity, {other_arrivals} at the other loads {list(loads)}; {slots} "
                        f"slots, {budget_gb:g} GB HBM budget; page-locked inputs and outputs in both arms",
            "deviation": f"config 5 runs 2000 timeframes; this replays {npool} distinct ones {n_arrivals} times at "
                         f"the headline load",
            "pool_generation_s": gen_s,
            "timeframe_clusters": sizes, "timeframe_ms": [round(v, 3) for v in lengths],
            "timeframe_tracks": n_tracks, "service_ms_plain": [round(1e3 * v, 2) for v in serv],
            "headline_load": headline, "plain": head["plain"], "served": head["served"], "by_load": by_load}


CONFIG3 = "10 ms continuous-readout timeframe at 50 kHz, 36 sectors, drift-time z, seed 2"
CONFIG2 = "central Pb-Pb-like event, 36 sectors, 8000+1600 tracks, seed 1"


def workload_of(args, rank):
    """(event, workload name) of the bench's main line: the 10 ms timeframe
    (the largest configuration that fits one GPU), or a timeframe of another
    length, or the central event."""
    import synth
    if args.workload == "central":
        return synth.central_event(seed=1 + rank), CONFIG2 if rank == 0 else CONFIG2.replace("seed 1", f"seed {1 + rank}")
    ms = args.timeframe_ms if args.timeframe_ms > 0 else 10.0
    name = CONFIG3 if ms == 10.0 else CONFIG3.replace("10 ms", f"{ms:g} ms")
    return synth.timeframe(seed=2 + rank, length_ms=ms), name.replace("seed 2", f"seed {2 + rank}")


def measure(cl, local, args, flush, world=1, clocks=True, e2e_steps=None):
    """One workload through the whole path: W warm-up steps, K timed steps
    (load from a device-resident copy + one graph replay of a2-a8, L2 flushed
    before each, CUDA events on the library's stream, max over ranks), then
    profiled plain runs for per-stage and per-Kalman-kernel times, and the
    same metric end to end through the public API (page-locked host input ->
    tracks and cluster assignment in page-locked host buffers)."""
    import numpy as np
    import torch

    import paper_1709_00618_b300 as tpc
    import synth
    n = len(cl)
    stream = torch.cuda.Stream()
    trk = tpc.Tracker(device=local, stream=stream, arena="torch", arena_clusters=n)
    if getattr(args, "zone_rows", 0) > 0:
        trk.set_tuning(zone_rows=args.zone_rows)
    dev_in = torch.from_numpy(cl.view(np.uint8)).to(f"cuda:{local}")

    def step_device():
        trk.load(dev_in)
        trk.run_graph()

    warm = max(args.warmup, 3)
    for _ in range(warm):
        step_device()
    trk.sync()
    kernels_per_step = trk.graph_kernels()
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
    t_step, total_clusters = combine_ranks(sum(times) / len(times), n, world, f"cuda:{local}")
    counts = trk.counts()

    # per-stage and per-Kalman-kernel device time: CUDA events recorded by the
    # library on its stream between the launches of plain (non-graph) runs of
    # the same kernels, L2 flushed before each run; median of 5
    trk.set_profiling(True)
    runs, kruns = [], []
    for _ in range(5):
        with torch.cuda.stream(stream):
            flush.zero_()
        trk.load(dev_in)
        trk.find().fit()
        trk.sync()
        runs.append(trk.stage_times())
        kruns.append(trk.kalman_profile())
    trk.set_profiling(False)
    stages = {k: statistics.median(r[k] for r in runs) for k in runs[0]}
    kalman = {}
    for name in kruns[0]:
        d = dict(kruns[-1][name])
        d["ms"] = statistics.median(r[name]["ms"] for r in kruns)
        kalman[name] = d
    work = trk.work()

    # end to end through the public API: pinned host input -> tracks + assignment in pinned host buffers
    pinned = torch.from_numpy(cl.view(np.uint8)).pin_memory()
    host_in = pinned.numpy().view(synth.CLUSTER_DTYPE)
    tr_buf = torch.zeros(counts["n_tracks"] + 4096, 128, dtype=torch.uint8).pin_memory()
    ct_buf = torch.zeros(n, dtype=torch.int32).pin_memory()
    e2e = []
    k_e2e = e2e_steps if e2e_steps is not None else args.steps
    for i in range(warm + k_e2e):
        t0 = time.perf_counter()
        tr, _ = trk.track_host(host_in, tr_buf, ct_buf)  # tpc_track_host: one call, host to host
        if i >= warm:
            e2e.append(time.perf_counter() - t0)
    e2e_t, _ = combine_ranks(sum(e2e) / len(e2e), n, world, f"cuda:{local}")
    trk.close()
    del dev_in
    return {"n": n, "t_step": t_step, "total_clusters": total_clusters, "counts": counts, "stages": stages,
            "kalman": kalman, "work": work, "kernels_per_step": kernels_per_step, "clocks": clk.summary(),
            "e2e": {"value": total_clusters / e2e_t, "unit": UNIT, "h2d_bytes_per_step": 16 * n,
                    "d2h_bytes_per_step": 128 * len(tr) + 4 * n, "steps": k_e2e},
            "host_in": host_in, "pinned": pinned}


def time_vs_size(local, flush, known=(), reps=3):
    """Tracking time against input size (Sec. 2: linear in the input size;
    Sec. 5 for timeframes): device time of one graph replay (inputs resident,
    L2 flushed, median of `reps`) for one sector, the central event and
    timeframes of 0.3, 1 and 3 ms, plus the points in `known` ((name,
    clusters, ms) measured by the caller); least-squares fit ms = a + b N and
    the log-log slope over the inputs of 1 M clusters and more."""
    import numpy as np
    import torch

    import paper_1709_00618_b300 as tpc
    import synth
    cases = [("one sector, 400 tracks, seed 0", lambda: synth.one_sector(seed=0).clusters),
             (CONFIG2, lambda: synth.central_event(seed=1).clusters)]
    for ms in (0.3, 1.0, 3.0):
        cases.append((CONFIG3.replace("10 ms", f"{ms:g} ms"), lambda ms=ms: synth.timeframe(seed=2, length_ms=ms).clusters))
    pts = []
    for name, gen in cases:
        cl = gen()
        stream = torch.cuda.Stream()
        with tpc.Tracker(device=local, stream=stream) as trk:
            dev = torch.from_numpy(cl.view(np.uint8)).to(f"cuda:{local}")
            for _ in range(3):
                trk.load(dev).run_graph()
            trk.sync()
            dt = []
            for _ in range(reps):
                with torch.cuda.stream(stream):
                    flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                trk.load(dev).run_graph()
                e1.record(stream)
                e1.synchronize()
                dt.append(e0.elapsed_time(e1))
            pts.append({"workload": name, "clusters": len(cl), "ms": statistics.median(dt)})
            del dev
    for name, n, ms in known:
        pts.append({"workload": name, "clusters": n, "ms": ms})
    pts.sort(key=lambda p: p["clusters"])
    N = np.array([p["clusters"] for p in pts], np.float64)
    T = np.array([p["ms"] for p in pts], np.float64)
    b, a = np.polyfit(N, T, 1)
    pred = a + b * N
    r2 = 1.0 - float(((T - pred) ** 2).sum() / ((T - T.mean()) ** 2).sum())
    big = N >= 1e6
    k = float(np.polyfit(np.log(N[big]), np.log(T[big]), 1)[0]) if big.sum() >= 2 else None
    for p, q in zip(pts, pred):
        p["fit_ms"] = float(q)
        p["clusters_per_s"] = p["clusters"] / (p["ms"] / 1e3)
    return {"points": pts, "fit": {"intercept_ms": float(a), "slope_ns_per_cluster": float(b * 1e6), "r2": r2,
                                   "loglog_slope_from_1M_clusters": k},
            "reading": "device time of one graph replay (inputs resident, L2 flushed, median of 3) against "
                       "input clusters; linear in the input size means a log-log slope near 1 once the GPU is full"}


def link_skip_leg(local, flush, cases, reps=5):
    """The next-row variant of the links (link_skip = 1) against the default
    reading on the same inputs: tracklets per track and the device time of
    one graph replay (inputs resident, L2 flushed, median of reps)."""
    import numpy as np
    import torch

    import paper_1709_00618_b300 as tpc
    out = {}
    for name, cl in cases:
        dev = torch.from_numpy(cl.view(np.uint8)).to(f"cuda:{local}")
        row = {"clusters": len(cl)}
        for skip in (0, 1):
            stream = torch.cuda.Stream()
            with tpc.Tracker(device=local, stream=stream, cfg=tpc.default_config(link_skip=skip)) as trk:
                for _ in range(3):
                    trk.load(dev).run_graph()
                trk.sync()
                dt = []
                for _ in range(reps):
                    with torch.cuda.stream(stream):
                        flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    trk.load(dev).run_graph()
                    e1.record(stream)
                    e1.synchronize()
                    dt.append(e0.elapsed_time(e1))
                c = trk.counts()
            row["variant" if skip else "default"] = {
                "ms": statistics.median(dt), "clusters_per_s": len(cl) / (statistics.median(dt) / 1e3),
                "tracklets": c["n_tracklets"], "tracks": c["n_tracks"],
                "tracklets_per_track": c["n_tracklets"] / max(c["n_tracks"], 1)}
        out[name] = row
        del dev
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300")
    ap.add_argument("--workload", choices=("timeframe", "central"), default="timeframe",
                    help="the main line's workload: the 10 ms continuous-readout timeframe (default) or the "
                         "central event")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batching", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="main line only (no central-event line, size sweep or server stream)")
    ap.add_argument("--serving-arrivals", type=int, default=500,
                    help="arrivals of the serving leg at its headline load")
    ap.add_argument("--serving-pool", type=int, default=16, help="distinct timeframes the serving leg replays")
    ap.add_argument("--timeframe-ms", type=float, default=0.0,
                    help="length of the main line's timeframe (default 10 ms, seed 2 + rank)")
    ap.add_argument("--zone-rows", type=int, default=0,
                    help="zone rows in step before the zone tail kernels (tpc_tuning.zone_rows; 0: the library's "
                         "default by input size); a launch shape, results unchanged")
    ap.add_argument("--all-configs", action="store_true",
                    help="print the per-config table (one sector, central event, 10 ms timeframe) instead")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    # the serving leg's timeframes are generated by a spawned process while
    # the GPU legs run
    pool = ServingPool(n_distinct=args.serving_pool) if world == 1 and not args.no_serving and \
        not args.all_configs else None

    import torch

    import paper_1709_00618_b300 as tpc

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if args.all_configs:
        if rank == 0:
            all_configs(local)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    ev, workload = workload_of(args, rank)
    cl = ev.clusters
    n = len(cl)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=f"cuda:{local}")
    m = measure(cl, local, args, flush, world)
    alu = tpc.measure_alu_peaks(local)
    clocks = m["clocks"]
    traffic = ncu_traffic(workload)
    roof, kernel_table = roofline(m["stages"], m["kalman"], n, alu, clocks, traffic if world == 1 else None)
    for k, v in kernel_table.items():
        v["traffic"] = traffic.get(k)
    peaks, src = _peaks()
    counts = m["counts"]
    line = {"metric": METRIC, "value": m["total_clusters"] / m["t_step"], "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * m["t_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "clusters": n},
            "workload_detail": {"tracklets": counts["n_tracklets"], "tracks": counts["n_tracks"],
                                "tracklets_per_track": counts["n_tracklets"] / max(counts["n_tracks"], 1),
                                "l2": "inputs larger than L2, and L2 flushed (256 MB write) between steps",
                                "graph": True, "kernels_per_step": m["kernels_per_step"],
                                **({"zone_rows": args.zone_rows} if args.zone_rows > 0 else {})},
            "clocks": clocks,
            "alu_peaks_measured": alu,
            "e2e": m["e2e"],
            "gpu_launches": m["kernels_per_step"] * args.steps,
            "roofline": roof,
            "kernels": kernel_table,
            "stages_ms": {k: round(v, 4) for k, v in m["stages"].items()},
            "work": m["work"],
            "peaks_source": src}
    if world == 1 and not args.no_extras:
        host_in = m.pop("host_in")
        line["e2e_server"] = events_through_server(host_in, n, local, events=8 if n > 4_000_000 else 16,
                                                   slots=3 if n > 4_000_000 else 4)
        del host_in
        m.pop("pinned")
        import synth
        synth_central = synth.central_event(seed=1).clusters
        mc = measure(synth_central, local, args, flush, world)
        rc, tc = roofline(mc["stages"], mc["kalman"], len(synth_central), alu, mc["clocks"],
                          ncu_traffic(CONFIG2))
        ce = {"workload": CONFIG2, "clusters": len(synth_central), "value": mc["total_clusters"] / mc["t_step"],
              "ms_per_step": 1e3 * mc["t_step"], "steps": args.steps, "e2e": mc["e2e"], "roofline": rc,
              "stages_ms": {k: round(v, 4) for k, v in mc["stages"].items()},
              "tracks": mc["counts"]["n_tracks"], "clocks": mc["clocks"]}
        line["central_event"] = ce
        line["time_vs_size"] = time_vs_size(local, flush, known=((workload, n, 1e3 * m["t_step"]),))
        line["link_skip_variant"] = link_skip_leg(local, flush, ((CONFIG2, synth_central), (workload, cl)))
    else:
        m.pop("host_in", None)
        m.pop("pinned", None)
    if world == 1 and not args.no_batching:
        line["batching"] = batching_leg(local, flush)
    if world == 1 and not args.no_serving:
        del flush
        torch.cuda.empty_cache()
        line["serving"] = serving_leg(local, pool, n_arrivals=args.serving_arrivals)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cl, workload)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
