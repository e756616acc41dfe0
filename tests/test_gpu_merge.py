"""Second tracking phase on the GPU (merging sector segments and the merged
refit) against the FP64 oracle.  Pairs are compared on segments outside the
exclusion shadow whose choices are clear (best chi2 not within 1e-3 of the
second best on either side of the pair, and not within 1% of the cut)."""

import numpy as np
import pytest

import oracle
import synth
from oracle import merge
from parity import (PAR_TOL, compare_follow, compare_selection, cov_rel_err, follow_result, par_rel_err,
                    record_stats)

pytestmark = pytest.mark.gpu


def _near(a, b):
    with np.errstate(invalid="ignore"):  # no second candidate: inf - inf
        return np.abs(a - b) <= 1e-3 * (1.0 + np.minimum(a, b))


@pytest.mark.parametrize("which", ["six_sectors", "central"])
def test_merging_matches_the_oracle(which):
    import paper_1709_00618_b300 as tpc
    if which == "central":
        cl = synth.central_event(seed=1).clusters
    else:
        cl = synth.generate(synth.GenParams(seed=31, n_primaries=1500, n_secondaries=0,
                                            sectors=(0, 1, 2, 18, 19, 20))).clusters
    with tpc.Tracker(device=0) as t:
        tracks, ct, _ = t.track(cl)
        g = follow_result(t)
        gm = t.merge()
    ref = oracle.run(cl)
    mo = merge.merge(ref, cl)
    stats = {}
    excl = compare_follow(g, ref, stats)
    excl2 = compare_selection(g, ct, ref, excl, stats)
    # track maps over tracklets both sides keep, outside the shadow
    common = np.intersect1d(np.nonzero(g["tl_track"] >= 0)[0], ref["t_tracklet"])
    common = common[~excl2[common]]
    g_of_r = np.full(ref["n_tracks"], -1, np.int64)
    g_of_r[ref["tl_track"][common]] = g["tl_track"][common]
    r_of_g = np.full(len(tracks), -1, np.int64)
    r_of_g[g["tl_track"][common]] = ref["tl_track"][common]
    ro_link, go_link = mo["link"], gm["link"]
    c_o, s_o, si_o = mo["pair_chi2"], mo["pair_second"], mo["pair_second_in"]
    checked = mism = 0
    for a in range(ref["n_tracks"]):
        ga = g_of_r[a]
        if ga < 0:
            continue
        b = ro_link[a]
        gb = go_link[ga]
        # the oracle's choice for a is clear
        if _near(c_o[a], s_o[a]) or abs(c_o[a] - 25.0) < 0.25:
            continue
        if b >= 0 and (g_of_r[b] < 0 or _near(c_o[a], si_o[b])):
            continue
        if gb >= 0 and r_of_g[gb] < 0:
            continue
        checked += 1
        exp = g_of_r[b] if b >= 0 else -1
        mism += int(gb != exp)
    assert checked > 100 and mism == 0, (checked, mism)
    # merged refits of the chains both sides form from mapped segments
    gch = {}
    for k, m in enumerate(gm["merged"]):
        segs = []
        h = int(m["cluster_offset"])
        while h >= 0:
            segs.append(h)
            h = int(go_link[h])
        gch[tuple(segs)] = k
    pe_all, ce_all, compared = [], [], 0
    for k, ch in enumerate(mo["chains"]):
        if not mo["ok"][k] or any(g_of_r[s] < 0 for s in ch):
            continue
        key = tuple(int(g_of_r[s]) for s in ch)
        if key not in gch:
            continue
        m = gm["merged"][gch[key]]
        if m["flags"] & 64:
            continue
        good = mo["chi2"][k] <= 10 * max(mo["ndf"][k], 1)
        if not good:
            continue
        assert m["n_clusters"] == mo["n"][k] and m["first_row"] == mo["row_in"][k]
        pe_all.append(par_rel_err(m["par"][None], mo["par"][k][None], mo["cov"][k][None]).max())
        ce_all.append(cov_rel_err(m["cov"][None], mo["cov"][k][None]).max())
        compared += 1
    assert compared > 30
    stats.update(merge_pairs_checked=checked, merge_pair_mismatches=mism, merge_chains_gpu=int(len(gm["merged"])),
                 merge_chains_ref=int(len(mo["chains"])), merge_chains_compared=compared,
                 merge_par_err_max=float(max(pe_all)), merge_cov_err_max=float(max(ce_all)))
    record_stats(f"merge_{which}", stats)
    # cov_rel_err is in units of each entry's bound (1e-3 relative, or 1e-4
    # in correlation units for weak correlations): <= 1 passes
    assert stats["merge_par_err_max"] <= PAR_TOL and stats["merge_cov_err_max"] <= 1.0, stats
