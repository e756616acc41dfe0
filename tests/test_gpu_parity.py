"""Parity of the CUDA path (through the C ABI) with the FP64 oracle."""

import numpy as np
import pytest

import oracle
import synth
from parity import full_parity, record_stats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trk():
    import paper_1709_00618_b300 as tpc
    t = tpc.Tracker(device=0)
    yield t
    t.close()


def test_one_sector(trk, sector_event, sector_oracle):
    stats = full_parity(trk, sector_event.clusters, sector_oracle)
    record_stats("one_sector", stats)
    assert stats["tracks_compared"] > 50


def test_six_sectors_both_sides(trk, small_event, small_oracle):
    stats = full_parity(trk, small_event.clusters, small_oracle)
    record_stats("six_sectors", stats)
    assert stats["tracks_compared"] > 200


def test_central_event_full_size(trk):
    ev = synth.central_event(seed=1)
    ref = oracle.run(ev.clusters)
    stats = full_parity(trk, ev.clusters, ref)
    record_stats("central_event", stats)
    assert stats["tracks_compared"] > 0.9 * stats["tracks_ref"]


def test_central_event_graph_equals_plain(trk):
    ev = synth.central_event(seed=1)
    a, ca, _ = trk.track(ev.clusters)
    b, cb, _ = trk.track(ev.clusters, graph=True)
    c, cc, _ = trk.track(ev.clusters, graph=True)
    assert np.array_equal(ca, cb) and np.array_equal(cb, cc)
    assert a.tobytes() == b.tobytes() == c.tobytes()


def test_twenty_repeats_are_byte_identical(trk):
    """Determinism: 20 runs of the central event (graph and plain launches
    alternating) give byte-identical tracks, cluster assignments, links,
    tracklets and follow outputs, so no atomic or scatter order leaks into
    a result."""
    ev = synth.central_event(seed=1)
    names = ("perm", "up", "dn", "tie", "tl_start", "tl_len", "f_n", "f_hits", "f_par", "f_cov", "f_chi2",
             "tl_track")
    ref = None
    for k in range(20):
        tracks, ct, _ = trk.track(ev.clusters, graph=bool(k % 2))
        got = [tracks.tobytes(), ct.tobytes()] + [trk.stage(nm).tobytes() for nm in names]
        if ref is None:
            ref = got
            assert len(tracks) > 20000
        else:
            for nm, a, b in zip(("tracks", "cluster_track") + names, ref, got):
                assert a == b, f"run {k}: {nm} differs"


def test_rerun_without_reload_repeats_every_kernel(trk):
    """A second find + fit on the same loaded batch (as the autotuner's
    trials and repeated tpc_find_tracks calls make) starts from the state of
    a load: every Kalman kernel does the same work again (its work counter
    and tallies are reset per run) and the results are the same bytes."""
    ev = synth.central_event(seed=1)
    trk.load(ev.clusters)
    runs = []
    for k in range(3):
        if k < 2:
            trk.find().fit()
        else:
            trk.run_graph()
        trk.sync()
        tracks, ct, _ = trk.get()
        runs.append((trk.kalman_profile(times=False), trk.work(), tracks.tobytes(), ct.tobytes()))
    for name, w in runs[0][0].items():
        # below 16 Mi clusters no zone tail kernel runs, below 4 Mi no p4r
        assert w["prop"] > 0 or name in ("k_follow_p2", "k_follow_p1t", "k_follow_p3t", "k_follow_p4r",
                                         "k_refit_p1t"), name
    for prof, work, tb, cb in runs[1:]:
        assert prof == runs[0][0]
        assert work == runs[0][1]
        assert tb == runs[0][2] and cb == runs[0][3]


def test_large_batch_shapes_give_the_same_bytes():
    """From 4 Mi clusters the Kalman stage runs its large-input shapes (index
    order, the backward refit rows in a kernel of their own, four zone CTAs
    per SM, zones finished by the zone tail kernels); split in two chunks on
    two streams, with one zone CTA per SM, with refilling at once, or with
    other zone rows in step (1: most zones parked, the tail lists full and
    the rest finished in place; 159: no tail kernels), it must give the same
    bytes."""
    import paper_1709_00618_b300 as tpc
    ev = synth.timeframe(seed=2, length_ms=0.6)
    assert len(ev.clusters) >= 4 << 20
    names = ("f_n", "f_hits", "f_par", "f_cov", "f_chi2", "tl_track")
    with tpc.Tracker(device=0) as t:
        ref_tracks, ref_ct, _ = t.track(ev.clusters, graph=True)
        ref = [t.stage(nm).tobytes() for nm in names]
        for shape in (dict(chunks=2), dict(chunks=2, ctas_per_sm_zone=1, refill=1), dict(ctas_per_sm_follow=3),
                      dict(zone_rows=1), dict(zone_rows=4, chunks=1), dict(zone_rows=159)):
            t.set_tuning(**shape)
            for graph in (False, True):
                tracks, ct, _ = t.track(ev.clusters, graph=graph)
                assert tracks.tobytes() == ref_tracks.tobytes(), shape
                assert np.array_equal(ct, ref_ct), shape
                assert [t.stage(nm).tobytes() for nm in names] == ref, shape


def test_zone_tails_on_small_batches_give_the_same_bytes():
    """Below 4 Mi clusters the zones run to their ends in the zone kernels;
    with zone tail kernels (tracklets filed for the longest-first order by
    the tail kernel that ends their zone) the results must not change."""
    import paper_1709_00618_b300 as tpc
    cl = synth.central_event(seed=1).clusters
    names = ("f_n", "f_hits", "f_par", "f_cov", "f_chi2", "tl_track")
    with tpc.Tracker(device=0) as t:
        ref_tracks, ref_ct, _ = t.track(cl)
        ref = [t.stage(nm).tobytes() for nm in names]
        for rows in (1, 3, 9):
            t.set_tuning(zone_rows=rows)
            for graph in (False, True):
                tracks, ct, _ = t.track(cl, graph=graph)
                assert tracks.tobytes() == ref_tracks.tobytes(), rows
                assert np.array_equal(ct, ref_ct), rows
                assert [t.stage(nm).tobytes() for nm in names] == ref, rows


def test_link_skip_variant_parity():
    """The next-row variant of the links (link_skip = 1 on both sides):
    links, tracklets, follow, selection and refit against the FP64 oracle
    run with the same setting, on the central event (plain launches) and a
    1 ms timeframe (the graph)."""
    import paper_1709_00618_b300 as tpc
    cases = (("central_event", synth.central_event(seed=1).clusters, False),
             ("timeframe_1ms", synth.timeframe(seed=2, length_ms=1.0).clusters, True))
    for name, cl, graph in cases:
        ref = oracle.run(cl, cfg=oracle.default_config(link_skip=1))
        with tpc.Tracker(device=0, cfg=tpc.default_config(link_skip=1)) as t:
            stats = full_parity(t, cl, ref, graph=graph)
        stats["tracklets_per_track"] = len(ref["tl_start"]) / max(int(ref["n_tracks"]), 1)
        record_stats(f"link_skip_{name}", stats)
        assert stats["tracks_compared"] > 0.9 * stats["tracks_ref"]


def test_timeframe_slice(trk):
    """Continuous read-out: z is the drift coordinate up to ~2.5e3 cm here."""
    ev = synth.timeframe(seed=2, length_ms=1.0)
    ref = oracle.run(ev.clusters)
    stats = full_parity(trk, ev.clusters, ref)
    record_stats("timeframe_1ms", stats)
    assert stats["tracks_compared"] > 0.8 * stats["tracks_ref"]


def test_batch_of_requests(trk):
    reqs = synth.batch_requests(seed=3, n_requests=12, max_tracks=2000)
    cl = np.concatenate([r.clusters for r in reqs])
    off = np.concatenate([[0], np.cumsum([len(r.clusters) for r in reqs])])
    ref = oracle.run(cl, req_offsets=off)
    stats = full_parity(trk, cl, ref, req_offsets=off)
    record_stats("batch12", stats)


def test_batch_result_equals_alone(trk):
    reqs = synth.batch_requests(seed=5, n_requests=6, max_tracks=1500)
    cl = np.concatenate([r.clusters for r in reqs])
    off = np.concatenate([[0], np.cumsum([len(r.clusters) for r in reqs])])
    tb, ctb, _ = trk.track(cl, off)
    for q, r in enumerate(reqs):
        ta, cta, _ = trk.track(r.clusters)
        sel = tb[tb["request"] == q]
        assert len(sel) == len(ta)
        for k in ("par", "cov", "chi2", "n_clusters", "first_row", "last_row", "sector", "flags"):
            assert np.array_equal(sel[k], ta[k]), k
        m = ctb[off[q]:off[q + 1]]
        base = np.nonzero(tb["request"] == q)[0]
        expect = np.where(cta >= 0, base[np.maximum(cta, 0)] if len(base) else -1, -1)
        assert np.array_equal(m, expect)


def test_edge_cases(trk):
    import paper_1709_00618_b300 as tpc
    empty = np.zeros(0, synth.CLUSTER_DTYPE)
    t, ct, _ = trk.track(empty)
    assert len(t) == 0 and len(ct) == 0
    one = np.zeros(1, synth.CLUSTER_DTYPE)
    one["row"], one["sector"], one["y"], one["z"] = 5, 3, 1.0, 2.0
    t, ct, _ = trk.track(one)
    assert len(t) == 0 and ct[0] == -1
    # empty requests inside a batch
    ev = synth.one_sector(seed=0)
    off = [0, 0, len(ev.clusters), len(ev.clusters)]
    ref = oracle.run(ev.clusters, req_offsets=off)
    full_parity(trk, ev.clusters, ref, req_offsets=off)
    # duplicated clusters (exact distance ties) and a degenerate row: many
    # clusters at one point
    dup = np.concatenate([ev.clusters, ev.clusters[::3]])
    blob = np.zeros(3000, synth.CLUSTER_DTYPE)
    blob["row"], blob["sector"], blob["y"], blob["z"] = 80, 0, 3.0, 40.0
    cl = np.concatenate([dup, blob])
    # every third cluster duplicated: exact ties by construction, so the
    # tie-tainted shadow is large on purpose and its bound is lifted here
    full_parity(trk, cl, oracle.run(cl), shadow_max=1.0)
    # invalid cluster -> EINVAL, and the context stays usable
    bad = ev.clusters.copy()
    bad["row"][7] = 200
    with pytest.raises(tpc.TpcError) as e:
        trk.track(bad)
    assert e.value.code == tpc.TPC_EINVAL
    bad = ev.clusters.copy()
    bad["z"][3] = np.nan
    with pytest.raises(tpc.TpcError):
        trk.track(bad)
    full_parity(trk, ev.clusters, oracle.run(ev.clusters))


def test_fp64_zone_keeps_assignments_of_the_fp64_oracle(trk):
    """The precision pattern (FP32 with FP64 covariance over the first
    updates after each seed) must not change which clusters go to which
    track: with it, no untainted tracklet differs from the FP64 oracle
    (asserted by the full-size test above); the same event followed in
    FP32 only is recorded for comparison -- there the cancellation of the
    first updates does change cluster choices."""
    import paper_1709_00618_b300 as tpc
    from parity import TAINT, follow_result
    ev = synth.central_event(seed=1)
    ref = oracle.run(ev.clusters)
    counts = {}
    for zone in (0, tpc.default_config().fp64_updates):
        t0 = tpc.Tracker(device=0, cfg=tpc.default_config(fp64_updates=zone))
        try:
            t0.track(ev.clusters)
            g = follow_result(t0)
        finally:
            t0.close()
        taint = ((g["f_flags"] & TAINT) != 0) | ((ref["f_flags"] & TAINT) != 0)
        same = (g["f_n"] == ref["f_n"]) & (g["f_nf"] == ref["f_nf"])
        for t in np.nonzero(same & ~taint)[0]:
            n = g["f_n"][t]
            if not np.array_equal(g["f_hits"][t, :n], ref["f_hits"][t, :n]):
                same[t] = False
        counts[zone] = int((~same & ~taint).sum())
    record_stats("fp64_zone_effect", {"untainted_divergent_fp32_only": counts[0],
                                 "untainted_divergent_with_zone": counts[max(counts)]})
    assert counts[max(counts)] == 0


def test_fp64_zone_length():
    """The FP64 zone holds fp64_updates updates after each seed in the
    forward pass, and from fp64_updates up to twice as many in the backward
    pass and the refit, whose covariances are outputs (further updates while
    the covariance is still converging).  Checked with the per-kernel work
    counters against the update counts of the outputs: the backward pass
    updates every forward hit and every hit it picks up (f_n), the refit
    every owned cluster."""
    import paper_1709_00618_b300 as tpc
    from parity import follow_result
    ev = synth.central_event(seed=1)
    N = tpc.default_config().fp64_updates
    with tpc.Tracker(device=0) as t:
        t.set_profiling(True)
        tracks, _, _ = t.track(ev.clusters)
        kp = t.kalman_profile(times=False)
        g = follow_result(t)
    f_n = g["f_n"].astype(np.int64)
    ok = (g["f_flags"] & (tpc.TF_SEED_FAIL | tpc.TF_BACK_FAIL)) == 0
    p3 = kp["k_follow_p3"]["upd64"] + kp["k_follow_p3t"]["upd64"]
    assert np.minimum(f_n[ok], N).sum() <= p3 <= np.minimum(f_n, 2 * N).sum()
    assert kp["k_follow_p1"]["upd64"] + kp["k_follow_p1t"]["upd64"] <= N * len(f_n)
    assert kp["k_follow_p2"]["upd64"] == kp["k_follow_p4r"]["upd64"] == kp["k_follow_p4"]["upd64"] == 0
    assert kp["k_refit_p2"]["upd64"] == 0
    n = tracks["n_clusters"].astype(np.int64)
    rok = (tracks["flags"] & tpc.TF_REFIT_FAIL) == 0
    r1 = kp["k_refit_p1"]["upd64"] + kp["k_refit_p1t"]["upd64"]
    assert np.minimum(n[rok], N).sum() <= r1 <= np.minimum(n, 2 * N).sum()
    record_stats("fp64_zone_length", {"backward_fp64_updates": int(p3),
                                      "backward_fixed_zone_ok": int(np.minimum(f_n[ok], N).sum()),
                                      "refit_fp64_updates": int(r1),
                                      "refit_fixed_zone_ok": int(np.minimum(n[rok], N).sum())})
