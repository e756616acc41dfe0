"""Vertex finding in the drift-time coordinate (Sec. 5) on the GPU against the
FP64 oracle, on timeframe slices, through the C ABI."""

import numpy as np
import pytest

import oracle
import synth
from parity import full_parity, record_stats

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,length_ms", [(7, 0.3), (8, 1.0)])
def test_vertices_match_the_oracle(seed, length_ms):
    import paper_1709_00618_b300 as tpc
    ev = synth.timeframe(seed=seed, length_ms=length_ms)
    ref = oracle.run(ev.clusters)
    with tpc.Tracker(device=0) as t:
        stats = full_parity(t, ev.clusters, ref, vertices={})
    record_stats(f"vertices_tf_{length_ms}ms", stats)
    assert stats["vertices_compared"] >= 5
    assert stats["vertex_tracks_checked"] > 1000


def test_vertex_options_and_edge_cases():
    import paper_1709_00618_b300 as tpc
    ev = synth.timeframe(seed=9, length_ms=0.2)
    with tpc.Tracker(device=0) as t:
        t.track(ev.clusters)
        a = t.find_vertices().vertices()
        b = t.find_vertices(min_tracks=1000000).vertices()  # no vertex big enough
        c = t.find_vertices(dca_max_cm=0.0).vertices()      # no track close enough
        d = t.find_vertices().vertices()
        assert len(a["vertices"]) >= 3 and len(b["vertices"]) == 0 and len(c["vertices"]) == 0
        assert (b["track_vertex"] < 0).all() and np.isnan(b["track_z"]).all()
        assert a["vertices"].tobytes() == d["vertices"].tobytes()  # deterministic
        assert np.array_equal(a["track_vertex"], d["track_vertex"])
        assert np.all(np.diff(a["vertices"]["time_us"]) > 0.5)  # time order, cut at the gap
        # one request per call
        t.load(ev.clusters, [0, 10, len(ev.clusters)]).find().fit()
        with pytest.raises(tpc.TpcError):
            t.find_vertices()
        # an empty timeframe
        t.track(np.zeros(0, synth.CLUSTER_DTYPE))
        e = t.find_vertices().vertices()
        assert len(e["vertices"]) == 0
