"""Serving loop, autotuner and capacity retry on the GPU.

The serving loop runs several requests at once on separate streams; each
request's result must be the one it gets alone (the same kernels on the same
data), and the first of them must also match the FP64 oracle."""
import time

import numpy as np
import pytest

import oracle
import synth
from parity import full_parity

pytestmark = pytest.mark.gpu


def _alone(tpc, clusters):
    with tpc.Tracker(device=0) as t:
        tracks, ct, _ = t.track(clusters, graph=True)
    return tracks, ct


def _mixed_requests():
    reqs = [r.clusters for r in synth.batch_requests(seed=21, n_requests=10, max_tracks=3000)]
    reqs.append(synth.timeframe(seed=22, length_ms=0.3).clusters)  # a larger, uneven one
    reqs.append(np.zeros(0, synth.CLUSTER_DTYPE))                    # an empty one
    return reqs


def test_server_result_equals_alone_in_the_mix():
    import paper_1709_00618_b300 as tpc
    reqs = _mixed_requests()
    alone = [_alone(tpc, c) for c in reqs]
    with tpc.Server(device=0, max_slots=4) as srv:
        for i, c in enumerate(reqs):
            assert srv.submit(i, c) == 0
        srv.drain(timeout_s=300)
        st = srv.stats()
        got = [srv.result(i) for i in range(len(reqs))]
    assert st["completed"] == len(reqs) and st["peak_running"] >= 2, st
    for (ta, ca), (tb, cb, times) in zip(alone, got):
        assert ta.tobytes() == tb.tobytes()
        assert np.array_equal(ca, cb)
        assert times[2] >= times[1] >= 0 and times[0] >= 0
    # the first request against the FP64 oracle, through a context of its own
    with tpc.Tracker(device=0) as t:
        stats = full_parity(t, reqs[0], oracle.run(reqs[0]))
    assert stats["tracks_compared"] > 0


def test_server_admits_by_budget():
    """A budget that holds one request's arena at a time serialises the
    requests; one that exceeds it alone is refused at submission."""
    import paper_1709_00618_b300 as tpc
    reqs = [r.clusters for r in synth.batch_requests(seed=23, n_requests=4, min_tracks=500, max_tracks=600)]
    lib = tpc.load_library()
    need = max(lib.tpc_arena_bytes(len(c), 1) for c in reqs)
    big = synth.central_event(seed=1).clusters
    with tpc.Server(device=0, max_slots=4, hbm_budget=int(need * 1.5)) as srv:
        with pytest.raises(tpc.TpcError):
            srv.submit(99, big)
        for i, c in enumerate(reqs):
            assert srv.submit(i, c) == 0
        srv.drain(timeout_s=300)
        st = srv.stats()
        for i, c in enumerate(reqs):
            tb, cb, _ = srv.result(i)
            ta, ca = _alone(tpc, c)
            assert ta.tobytes() == tb.tobytes() and np.array_equal(ca, cb)
    assert st["completed"] == 4 and st["arena_bytes"] <= need * 1.5


def test_server_poll_and_unknown_ids():
    import paper_1709_00618_b300 as tpc
    c = synth.one_sector(seed=0).clusters
    with tpc.Server(device=0, max_slots=1) as srv:
        assert srv.poll(5) == "unknown"
        assert srv.submit(5, c) == 0
        with pytest.raises(tpc.TpcError):
            srv.submit(5, c)  # id in use
        deadline = time.time() + 120
        while srv.poll(5) not in ("finished", "failed") and time.time() < deadline:
            time.sleep(0.01)
        assert srv.poll(5) == "finished"
        tracks, ct, _ = srv.result(5)
        assert srv.poll(5) == "unknown"
        # too small an output buffer: the request fails with the count found
        assert srv.submit(6, c, tracks_out=np.zeros(3, tpc.TRACK_DTYPE)) == 0
        srv.drain(timeout_s=120)
        with pytest.raises(tpc.TpcError) as e:
            srv.result(6)
        assert e.value.code == tpc.TPC_EOVERFLOW and f"({len(tracks)} tracks found)" in str(e.value)
    assert len(tracks) > 50 and (ct >= 0).sum() > 0


def test_server_pinned_buffers_and_plain_get_into():
    """Page-locked inputs and outputs (asynchronous copies) give the same
    bytes as the plain path writing into caller buffers."""
    import torch

    import paper_1709_00618_b300 as tpc
    reqs = [r.clusters for r in synth.batch_requests(seed=25, n_requests=6, max_tracks=4000)]
    pins = [torch.from_numpy(c.view(np.uint8)).pin_memory() for c in reqs]
    outs = [(torch.zeros(len(c) // 10 + 1, 128, dtype=torch.uint8).pin_memory(),
             torch.zeros(len(c), dtype=torch.int32).pin_memory()) for c in reqs]
    with tpc.Server(device=0, max_slots=3) as srv:
        for i, (p, (to, co)) in enumerate(zip(pins, outs)):
            assert srv.submit(i, p, tracks_out=to, cluster_track_out=co) == 0
        srv.drain(timeout_s=300)
        got = [srv.result(i) for i in range(len(reqs))]
    with tpc.Tracker(device=0) as t:
        for c, (tb, cb, _) in zip(reqs, got):
            t.load(c).find().fit()
            tr = np.zeros(len(c) // 10 + 1, tpc.TRACK_DTYPE)
            ct = np.zeros(len(c), np.int32)
            ta, ca = t.get_into(tr, ct)
            assert ta.tobytes() == tb.tobytes() and np.array_equal(ca, cb)


def test_autotuned_shapes_give_the_same_result():
    import paper_1709_00618_b300 as tpc
    ev = synth.GenParams(seed=11, n_primaries=1500, n_secondaries=300, sectors=(0, 1, 2, 18, 19, 20))
    cl = synth.generate(ev).clusters
    with tpc.Tracker(device=0) as t:
        ref_tracks, ref_ct, _ = t.track(cl)
        choice, ms = t.autotune(cl, reps=1)
        assert choice["block_clusters"] in (128, 256, 512)
        assert choice["block_follow"] in (64, 96, 128)
        assert choice["ctas_per_sm_zone"] in (2, 3, 4)
        assert choice["ctas_per_sm_follow"] in (2, 3, 64)
        assert choice["refill"] in (1, 4, 8, 16)
        assert choice["chunks"] in (1, 2)
        assert t.tuning() == choice
        assert ms > 0
        tracks, ct, _ = t.track(cl)
        g_tracks, g_ct, _ = t.track(cl, graph=True)
        names = ("block_clusters", "block_follow", "ctas_per_sm_zone", "ctas_per_sm_follow", "refill", "chunks")
        for shape in ((512, 64, 3, 2, 1, 1), (128, 128, 1, 8, 32, 2), (256, 96, 2, 1, 5, 2)):
            t.set_tuning(**dict(zip(names, shape)))
            s_tracks, s_ct, _ = t.track(cl)
            assert s_tracks.tobytes() == ref_tracks.tobytes() and np.array_equal(s_ct, ref_ct)
            s_tracks, s_ct, _ = t.track(cl, graph=True)
            assert s_tracks.tobytes() == ref_tracks.tobytes() and np.array_equal(s_ct, ref_ct)
    assert tracks.tobytes() == ref_tracks.tobytes() and np.array_equal(ct, ref_ct)
    assert g_tracks.tobytes() == ref_tracks.tobytes() and np.array_equal(g_ct, ref_ct)


def _stubs():
    """Straight lines (100 per sector, all 36 sectors) with rows 5 and 6 of
    every 7 left out.  The neighbour finder sees 5-row stubs whose end
    clusters have no pair, so every stub yields one 3-cluster tracklet (one
    per 4.95 clusters, more than the default capacity of n/6 + 1024); the
    Kalman follow bridges the 2-row gaps, so each line still becomes a track."""
    xr = 85.2 + np.arange(159) * ((245.8 - 85.2) / 158.0)
    rows = np.array([r for r in range(159) if r % 7 < 5])
    k_y, k_z = np.meshgrid(np.arange(5), np.arange(20), indexing="ij")
    y0 = (-12.0 + 6.0 * k_y).ravel()
    z0 = (10.0 + 9.0 * k_z).ravel()
    dx = xr[rows] - xr[0]
    parts = []
    for s in range(36):
        c = np.zeros((len(y0), len(rows)), synth.CLUSTER_DTYPE)
        c["y"] = y0[:, None] + 0.02 * dx[None, :]
        c["z"] = z0[:, None] + 0.3 * dx[None, :]
        c["row"] = rows[None, :]
        c["sector"] = s
        parts.append(c.ravel())
    cl = np.concatenate(parts)
    cl["id"] = np.arange(len(cl))
    return cl


def test_tracklet_overflow_is_retried_not_truncated():
    import paper_1709_00618_b300 as tpc
    cl = _stubs()
    n = len(cl)
    with tpc.Tracker(device=0) as big:
        big.reserve(n_clusters=n, n_requests=1, n_tracklets=n)
        ref_tracks, ref_ct, _ = big.track(cl)
        assert big.counts()["n_tracklets"] > n // 6 + 1024  # beyond the default capacity
    assert len(ref_tracks) == 3600  # one per line, as the FP64 oracle finds
    with tpc.Tracker(device=0) as t:
        tracks, ct, _ = t.track(cl)
    assert tracks.tobytes() == ref_tracks.tobytes() and np.array_equal(ct, ref_ct)
    with tpc.Server(device=0, max_slots=2) as srv:
        srv.submit(0, cl)
        srv.drain(timeout_s=300)
        tb, cb, _ = srv.result(0)
    assert tb.tobytes() == ref_tracks.tobytes() and np.array_equal(cb, ref_ct)


def test_kernel_profile_adds_up():
    """Per-Kalman-kernel counters sum to the totals; per-kernel times fit in
    their stages; the captured graph's kernel count is stable."""
    import paper_1709_00618_b300 as tpc
    p = synth.GenParams(seed=11, n_primaries=1500, n_secondaries=300, sectors=(0, 1, 2, 18, 19, 20))
    cl = synth.generate(p).clusters
    with tpc.Tracker(device=0) as t:
        t.set_profiling(True)
        t.load(cl).find().fit().sync()
        st = t.stage_times()
        kp = t.kalman_profile()
        work = t.work()
        t.set_profiling(False)
        t.load(cl).run_graph().sync()
        nk = t.graph_kernels()
        t.load(cl).run_graph().sync()
        assert t.graph_kernels() == nk
    for key in ("prop", "upd32", "upd64", "cand", "prop64"):
        assert sum(d[key] for d in kp.values()) == work[key], key
    assert kp["k_follow_p1"]["upd64"] > 0 and kp["k_follow_p2"]["upd32"] > 0 and kp["k_refit_p2"]["upd32"] > 0
    assert kp["k_follow_p2"]["upd64"] == 0 and kp["k_follow_p4"]["upd64"] == 0 and kp["k_refit_p2"]["upd64"] == 0
    assert kp["k_follow_p4r"]["upd64"] == 0
    follow = sum(v["ms"] for k, v in kp.items() if k.startswith("k_follow"))
    assert abs(follow - st["follow"]) < 1e-3 + 1e-3 * st["follow"]
    assert sum(v["ms"] for k, v in kp.items() if k.startswith("k_refit")) <= st["refit"] + 1e-3
    assert 30 <= nk <= 60
