"""The batched-request entry points tpc_submit_batch / tpc_poll on the GPU.

Several independent requests (events and timeframes of uneven size, one of
them empty) submitted as one batch on one context: each request's tracks
and cluster assignment, copied into its own host buffers, must equal what
the request gets alone (Sec. 2 runs several events at once to fill a GPU;
requests never share tracks)."""
import time

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

# fields that depend on where the request sits in the batch
BATCH_FIELDS = ("request", "cluster_offset")


def _alone(tpc, clusters):
    with tpc.Tracker(device=0) as t:
        tracks, ct, _ = t.track(clusters, graph=True)
    return tracks, ct


def _wait(trk, ids, timeout_s=300):
    out, t_end = {}, time.time() + timeout_s
    while len(out) < len(ids):
        for i in ids:
            if i not in out:
                r = trk.poll(i)
                if r is not None:
                    out[i] = r
        assert time.time() < t_end, "batch did not finish"
        time.sleep(1e-4)
    return out


def _same_tracks(a, b):
    assert len(a) == len(b)
    for k in a.dtype.names:
        if k not in BATCH_FIELDS:
            assert np.array_equal(a[k], b[k]), k


def test_submit_batch_results_equal_alone():
    import paper_1709_00618_b300 as tpc
    reqs = [r.clusters for r in synth.batch_requests(seed=31, n_requests=9, max_tracks=3000)]
    reqs.insert(3, np.zeros(0, synth.CLUSTER_DTYPE))
    reqs.append(synth.timeframe(seed=32, length_ms=0.3).clusters)
    alone = [_alone(tpc, c) for c in reqs]
    ids = [1000 + 7 * i for i in range(len(reqs))]
    with tpc.Tracker(device=0) as trk:
        for rep in range(2):  # a second batch on the same context reuses its arena
            trk.submit_batch([(i, c) for i, c in zip(ids, reqs)])
            got = _wait(trk, ids)
            for q, (i, (ta, ca)) in enumerate(zip(ids, alone)):
                tb, cb = got[i]
                _same_tracks(ta, tb)
                assert np.all(tb["request"] == q)
                assert np.array_equal(ca, cb)
            # the whole batch stays readable through tpc_get_tracks
            tall, call, _ = trk.get()
            assert len(tall) == sum(len(a[0]) for a in alone)
        with pytest.raises(tpc.TpcError) as e:
            trk.poll(12345)
        assert e.value.code == tpc.TPC_EINVAL


def test_submit_batch_small_cap_fails_only_that_request():
    import paper_1709_00618_b300 as tpc
    reqs = [r.clusters for r in synth.batch_requests(seed=33, n_requests=3, min_tracks=800, max_tracks=1000)]
    alone = [_alone(tpc, c) for c in reqs]
    small = np.zeros(max(len(alone[1][0]) - 1, 0), tpc.TRACK_DTYPE)
    with tpc.Tracker(device=0) as trk:
        trk.submit_batch([(0, reqs[0]), (1, reqs[1], small), (2, reqs[2])])
        t_end = time.time() + 300
        while True:
            try:
                r1 = trk.poll(1)
            except tpc.TpcError as e:
                assert e.code == tpc.TPC_EOVERFLOW
                break
            assert r1 is None, "a request whose cap is too small must fail"
            assert time.time() < t_end
            time.sleep(1e-4)
        got = _wait(trk, [0, 2])
        for q in (0, 2):
            _same_tracks(alone[q][0], got[q][0])
            assert np.array_equal(alone[q][1], got[q][1])


def test_submit_batch_retries_a_tracklet_overflow():
    """More tracklets than the default capacity: the batch reruns once with
    the worst-case capacity and nothing is truncated."""
    import paper_1709_00618_b300 as tpc
    from test_gpu_serving import _stubs
    cl = _stubs()
    ref_tracks, ref_ct = _alone(tpc, cl)
    other = synth.batch_requests(seed=34, n_requests=1, max_tracks=500)[0].clusters
    ref_o = _alone(tpc, other)
    with tpc.Tracker(device=0) as trk:
        trk.submit_batch([(5, other), (6, cl)])
        got = _wait(trk, [5, 6])
    _same_tracks(ref_tracks, got[6][0])
    assert np.array_equal(ref_ct, got[6][1])
    _same_tracks(ref_o[0], got[5][0])
    assert np.array_equal(ref_o[1], got[5][1])
