"""Cluster rejection on the GPU against the FP64 oracle (the compression
section's classes: low momentum, inclined, further looper legs).  Classes
are compared on the tracks both sides keep outside the exclusion shadow,
except where a decision lies within its margin of a cut: momentum within
0.1% of p_min, |dz/ds_T| within 1e-3 of tgl_max, the circle's reach within
0.2 cm of the outermost row radius, the z distance within 0.2 cm of
dz_leg.  Keep flags are compared on the clusters of the compared tracks."""

import numpy as np
import pytest

import oracle
import synth
from oracle import reject, vertex
from parity import compare_follow, compare_selection, follow_result, record_stats

pytestmark = pytest.mark.gpu


def _compare(name, cl, g, tracks, ct, gr, ref, orj):
    stats = {}
    excl = compare_follow(g, ref, stats)
    excl2 = compare_selection(g, ct, ref, excl, stats)
    common = np.intersect1d(np.nonzero(g["tl_track"] >= 0)[0], ref["t_tracklet"])
    common = common[~excl2[common]]
    gi = g["tl_track"][common]
    ri = ref["tl_track"][common]
    mg = orj["margin"]
    clear = (mg["p"][ri] > 1e-3) & (mg["tgl"][ri] > 1e-3) & (mg["reach"][ri] > 0.2) & (mg["dz"][ri] > 0.2)
    clear |= np.isnan(mg["dz"][ri]) & (mg["p"][ri] > 1e-3) & (mg["tgl"][ri] > 1e-3) & (mg["reach"][ri] > 0.2)
    gb = gr["track_class"][gi[clear]].astype(np.int32)
    rb = orj["bits"][ri[clear]]
    mism = int((gb != rb).sum())
    # keep flags of the clusters of compared tracks (same track on both sides)
    g_of_r = np.full(ref["n_tracks"], -1, np.int64)
    g_of_r[ri[clear]] = gi[clear]
    rct = ref["cluster_track"].astype(np.int64)
    sel = (rct >= 0) & (g_of_r[np.maximum(rct, 0)] >= 0) & (ct == g_of_r[np.maximum(rct, 0)])
    keep_mism = int((gr["cluster_keep"][sel] != orj["keep"][sel]).sum())
    per = {f"n_{k}": int(((rb & b) != 0).sum()) for k, b in (("low_p", 1), ("inclined", 2), ("leg", 4))}
    stats.update(reject_tracks_checked=int(clear.sum()), reject_tracks_margin=int((~clear).sum()),
                 reject_class_mismatches=mism, reject_clusters_checked=int(sel.sum()),
                 reject_keep_mismatches=keep_mism, reject_fraction_gpu=float(1.0 - gr["cluster_keep"].mean()),
                 reject_fraction_oracle=float(1.0 - orj["keep"].mean()), **per)
    record_stats(name, stats)
    assert mism == 0 and keep_mism == 0, stats
    return stats


def test_rejection_matches_the_oracle_on_an_event_with_loopers():
    import paper_1709_00618_b300 as tpc
    cl = synth.looper_event(seed=7).clusters
    with tpc.Tracker(device=0) as t:
        tracks, ct, _ = t.track(cl)
        g = follow_result(t)
        gr = t.reject()
    ref = oracle.run(cl)
    orj = reject.from_oracle_run(ref, len(cl))
    st = _compare("reject_looper_event", cl, g, tracks, ct, gr, ref, orj)
    assert st["reject_tracks_checked"] > 10000 and st["n_leg"] > 1000 and st["n_inclined"] > 100 and \
        st["n_low_p"] > 100, st
    # the counts agree with the keep mask and the classes
    c = gr["counts"]
    assert c["all"] == int((gr["cluster_keep"] == 0).sum())
    assert c["looper_leg"] == int(tracks["n_clusters"][(gr["track_class"] & tpc.RJ_LOOPER_LEG) != 0].sum())


def test_rejection_with_vertices_in_a_timeframe():
    import paper_1709_00618_b300 as tpc
    p = synth.GenParams(seed=43, n_primaries=5, n_secondaries=1, timeframe=True, tf_length_us=300.0, legs=4,
                        eta_max=1.5, pt_min=0.04)
    cl = synth.generate(p).clusters
    with tpc.Tracker(device=0) as t:
        tracks, ct, _ = t.track(cl)
        g = follow_result(t)
        with pytest.raises(tpc.TpcError):
            t.reject(use_vertices=1)  # no vertices of this fit yet
        t.find_vertices(min_pt_gev=0.2)
        gv = t.vertices()
        gr = t.reject(use_vertices=1)
    ref = oracle.run(cl)
    vx = vertex.from_oracle_run(ref, {"min_pt": 0.2})
    assert len(gv["vertices"]) == len(vx["v_time"]) >= 5
    assert np.allclose(gv["vertices"]["time_us"], vx["v_time"], atol=1e-3)
    orj = reject.from_oracle_run(ref, len(cl), vertices=vx)
    st = _compare("reject_timeframe_vertices", cl, g, tracks, ct, gr, ref, orj)
    assert st["reject_tracks_checked"] > 3000 and st["n_leg"] > 300, st
