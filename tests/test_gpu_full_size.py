"""Full-size workloads in the benchmark's launch configuration (the captured
graph), checked on samples the FP64 oracle can compute.  Sectors and
requests are tracked independently (Sec. 2), so the tracks and cluster
assignments of a few sectors of the full 10 ms timeframe (90 M clusters),
and of a few requests of the 256-request batch, must be exactly those of
the same sectors or requests tracked alone; those are then compared with
the oracle stage by stage."""

import numpy as np
import pytest

import oracle
import synth
from parity import full_parity, record_stats

pytestmark = pytest.mark.gpu


FIELDS = ("par", "cov", "chi2", "ndf", "n_clusters", "first_row", "last_row", "sector", "flags")


def _same_as_alone(tracks, ct, sel_tracks, sel_clusters, ta, cta):
    """The selected tracks of a large run equal a run on the selected part
    alone, and so do the assignments of the selected clusters."""
    part = tracks[sel_tracks]
    assert len(part) == len(ta)
    for k in FIELDS:
        assert np.array_equal(part[k], ta[k]), k
    idx = np.nonzero(sel_tracks)[0]
    local = np.full(len(tracks), -1, np.int64)
    local[idx] = np.arange(len(idx))
    got = ct[sel_clusters]
    got = np.where(got >= 0, local[np.maximum(got, 0)], -1)
    assert np.array_equal(got, cta)


def test_full_timeframe_sampled_sectors():
    import paper_1709_00618_b300 as tpc
    cl = synth.timeframe(seed=2, length_ms=10.0).clusters
    sectors = (5, 23)
    with tpc.Tracker(device=0) as t:
        tracks, ct, _ = t.track(cl, graph=True)
        # the zone tail kernels that run at this size change no result
        t.set_tuning(zone_rows=159)
        t2, ct2, _ = t.track(cl, graph=True)
        assert t2.tobytes() == tracks.tobytes() and np.array_equal(ct2, ct)
        sel = np.isin(cl["sector"], sectors)
        sub = cl[sel]
        ta, cta, _ = t.track(sub)
        _same_as_alone(tracks, ct, np.isin(tracks["sector"], sectors), sel, ta, cta)
        stats = full_parity(t, sub, oracle.run(sub))
    stats.update(clusters_full=int(len(cl)), tracks_full=int(len(tracks)), sectors=list(sectors))
    record_stats("timeframe_10ms_sectors_5_23", stats)
    assert len(tracks) > 2_000_000 and stats["tracks_compared"] > 0.8 * stats["tracks_ref"]


def test_full_batch_sampled_requests():
    import paper_1709_00618_b300 as tpc
    reqs = synth.batch_requests(seed=3, n_requests=256)
    cl = np.concatenate([r.clusters for r in reqs])
    off = np.concatenate([[0], np.cumsum([len(r.clusters) for r in reqs])])
    sizes = np.diff(off)
    sample = sorted({0, 97, 255, int(np.argmax(sizes)), int(np.argmin(sizes))})
    with tpc.Tracker(device=0) as t:
        tracks, ct, _ = t.track(cl, off, graph=True)
        for q in sample:
            ta, cta, _ = t.track(reqs[q].clusters)
            sel = np.zeros(len(cl), bool)
            sel[off[q]:off[q + 1]] = True
            _same_as_alone(tracks, ct, tracks["request"] == q, sel, ta, cta)
        for q in (int(np.argmax(sizes)), 97):
            stats = full_parity(t, reqs[q].clusters, oracle.run(reqs[q].clusters))
            stats.update(request=q, requests=256, clusters_batch=int(len(cl)))
            record_stats(f"batch256_request_{q}", stats)
            assert stats["tracks_compared"] > 0.8 * stats["tracks_ref"]
