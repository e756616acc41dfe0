"""Track-model compression on the GPU: the decompression restores every
fixed-point cluster exactly (in the same and in a fresh context), and the
encoding matches the FP64 oracle's up to rounding flips of the prediction."""

import numpy as np
import pytest

import oracle
import synth
from parity import compare_follow, compare_selection, follow_result, record_stats

pytestmark = pytest.mark.gpu
UNIT = 0.01

def _fixed_point(v):
    return np.rint(np.asarray(v, np.float32) * np.float32(1.0 / UNIT)).astype(np.int32)


@pytest.mark.parametrize("which", ["central", "timeframe"])
def test_round_trip_is_exact_and_matches_the_oracle(which):
    import paper_1709_00618_b300 as tpc
    ev = synth.central_event(seed=1) if which == "central" else synth.timeframe(seed=2, length_ms=0.5)
    cl = ev.clusters
    with tpc.Tracker(device=0) as t:
        tracks, ct, tc = t.track(cl)
        tc = t.get(track_clusters=True)[2]
        c = t.compress(UNIT)
        qy, qz = t.decompress(c["heads"], c["rows"], c["res_y"], c["res_z"], UNIT)
        g = follow_result(t)
    # exact round trip, and the encoded clusters are the fixed-point input
    assert np.array_equal(qy, c["q_y"]) and np.array_equal(qz, c["q_z"])
    off = np.concatenate([[0], np.cumsum(c["heads"]["n_clusters"])])
    order = np.concatenate([tc[off[m]:off[m + 1]][::-1] for m in range(len(tracks))]) if len(tracks) else []
    assert np.array_equal(c["q_y"], _fixed_point(cl["y"][order]))
    assert np.array_equal(c["q_z"], _fixed_point(cl["z"][order]))
    assert np.array_equal(c["rows"], cl["row"][order])
    # a fresh context decodes the same stream
    with tpc.Tracker(device=0) as t2:
        qy2, qz2 = t2.decompress(c["heads"], c["rows"], c["res_y"], c["res_z"], UNIT)
    assert np.array_equal(qy2, qy) and np.array_equal(qz2, qz)
    # against the oracle, on tracks outside the exclusion shadow
    ref = oracle.run(cl)
    stats = {}
    excl = compare_follow(g, ref, stats)
    excl2 = compare_selection(g, ct, ref, excl, stats)
    inp = oracle.codec_input(ref, cl, UNIT)
    enc = oracle.codec(inp)
    common = np.intersect1d(np.nonzero(g["tl_track"] >= 0)[0], ref["t_tracklet"])
    common = common[~excl2[common]]
    gi, ri = g["tl_track"][common], ref["tl_track"][common]
    slim = ((tracks["flags"][gi] | ref["t_flags"][ri]) & 8) != 0  # a |sin phi| limit test within the margin
    gi, ri = gi[~slim], ri[~slim]
    assert np.array_equal(c["heads"]["ok"][gi].astype(bool), enc["ok"][ri].astype(bool))
    gi, ri = gi[c["heads"]["ok"][gi] == 1], ri[c["heads"]["ok"][gi] == 1]
    gsel = np.concatenate([np.arange(off[m], off[m + 1]) for m in gi])
    rsel = np.concatenate([np.arange(inp["off"][r], inp["off"][r + 1]) for r in ri])
    assert np.array_equal(c["q_y"][gsel], inp["qy"][rsel]) and np.array_equal(c["rows"][gsel], inp["rows"][rsel])
    dy = c["res_y"][gsel] - enc["ry"][rsel]
    dz = c["res_z"][gsel] - enc["rz"][rsel]
    flips = (dy != 0) | (dz != 0)
    # a flip is the two predictions rounding to neighbouring units
    assert np.abs(dy).max() <= 1 and np.abs(dz).max() <= 1
    assert flips.mean() < 0.01, flips.mean()
    assert not (flips & (enc["margin"][rsel] > 0.05)).any()  # only near a rounding boundary
    hp = np.abs(c["heads"]["par"][gi] - inp["head"][ri])
    stats.update(codec_tracks=int(len(gi)), codec_clusters=int(len(gsel)), codec_flips=int(flips.sum()),
                 codec_head_abs_err_max=[float(v) for v in hp.max(0)] if len(hp) else [])
    record_stats(f"codec_{which}", stats)


def test_malformed_streams_are_rejected():
    import paper_1709_00618_b300 as tpc
    ev = synth.one_sector(seed=0)
    with tpc.Tracker(device=0) as t:
        t.track(ev.clusters)
        c = t.compress(UNIT)
        heads = c["heads"].copy()
        heads["n_clusters"][0] += 1  # counts do not add up
        with pytest.raises(tpc.TpcError):
            t.decompress(heads, c["rows"], c["res_y"], c["res_z"], UNIT)
        rows = c["rows"].copy()
        k = int(np.nonzero(c["heads"]["ok"])[0][0])
        rows[int(np.sum(c["heads"]["n_clusters"][:k]))] = 158 if c["heads"]["row_out"][k] < 158 else 0
        if c["heads"]["row_out"][k] < 158:
            with pytest.raises(tpc.TpcError):  # a cluster above the track's first row
                t.decompress(c["heads"], rows, c["res_y"], c["res_z"], UNIT)
        with pytest.raises(tpc.TpcError):
            t.compress(0.0)
