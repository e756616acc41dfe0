"""tpc_track_host: one request host to host in one call (clusters in;
tracks and cluster assignment out, the assignment's copy overlapping the
refit) gives the bytes of tpc_load_clusters + tpc_find_tracks +
tpc_fit_tracks + tpc_get_tracks, with page-locked and with pageable output
buffers, and reports the same errors."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _reference(tpc, clusters):
    with tpc.Tracker(device=0) as t:
        tracks, ct, _ = t.track(clusters)
    return tracks, ct


@pytest.mark.parametrize("pinned,large", [(False, False), (True, False), (True, True)])
def test_track_host_equals_the_step_by_step_calls(pinned, large):
    """Below 4 Mi clusters the copies follow the refit; from 4 Mi clusters
    (a 0.6 ms timeframe) the assignment's copy overlaps it."""
    import torch

    import paper_1709_00618_b300 as tpc
    ev = synth.timeframe(seed=2, length_ms=0.6) if large else synth.central_event(seed=1)
    assert (len(ev.clusters) >= 4 << 20) == large
    ref_tracks, ref_ct = _reference(tpc, ev.clusters)
    n = len(ev.clusters)
    if pinned:
        tr_buf = torch.zeros(len(ref_tracks) + 100, 128, dtype=torch.uint8).pin_memory()
        ct_buf = torch.full((n,), 7, dtype=torch.int32).pin_memory()
    else:
        tr_buf = np.zeros(len(ref_tracks) + 100, tpc.TRACK_DTYPE)
        ct_buf = np.full(n, 7, np.int32)
    with tpc.Tracker(device=0) as t:
        for _ in range(2):  # a second call on the same context reuses its arena and streams
            tracks, ct = t.track_host(ev.clusters, tr_buf, ct_buf)
            assert tracks.tobytes() == ref_tracks.tobytes()
            assert np.array_equal(ct, ref_ct)


def test_track_host_empty_and_small_cap():
    import paper_1709_00618_b300 as tpc
    with tpc.Tracker(device=0) as t:
        tracks, ct = t.track_host(np.zeros(0, synth.CLUSTER_DTYPE), np.zeros(4, tpc.TRACK_DTYPE),
                                  np.zeros(0, np.int32))
        assert len(tracks) == 0
        ev = synth.one_sector(seed=0)
        ref_tracks, _ = _reference(tpc, ev.clusters)
        with pytest.raises(tpc.TpcError) as e:
            t.track_host(ev.clusters, np.zeros(len(ref_tracks) - 1, tpc.TRACK_DTYPE),
                         np.zeros(len(ev.clusters), np.int32))
        assert e.value.code == tpc.TPC_EOVERFLOW
        # the context stays usable
        tracks, ct = t.track_host(ev.clusters, np.zeros(len(ref_tracks), tpc.TRACK_DTYPE),
                                  np.zeros(len(ev.clusters), np.int32))
        assert tracks.tobytes() == ref_tracks.tobytes()


def test_track_host_rejects_invalid_clusters():
    import paper_1709_00618_b300 as tpc
    ev = synth.one_sector(seed=0)
    bad = ev.clusters.copy()
    bad["row"][5] = 200
    with tpc.Tracker(device=0) as t:
        with pytest.raises(tpc.TpcError) as e:
            t.track_host(bad, np.zeros(1000, tpc.TRACK_DTYPE), np.zeros(len(bad), np.int32))
        assert e.value.code == tpc.TPC_EINVAL
