"""Pins of the sector-merging oracle (second tracking phase, Sec. 2): a
noiseless helix split over two sectors is refitted to its true parameters
across the frame turn; on a smeared event the segments of one track in
neighbouring sectors are merged (and of different tracks are not); the pair
chi2 of true pairs follows five degrees of freedom; the z window at the
partner's first row only prunes (it changes no choice)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import merge

SECTORS = (0, 1, 2, 18, 19, 20)


def _labels(ev, ref):
    ct = ref["cluster_track"].astype(np.int64)
    labels = ev.clusters["id"].astype(np.int64)
    m = ref["n_tracks"]
    lab = np.full(m, -1, np.int64)
    sel = (ct >= 0) & (labels != 0xFFFFFFFF)
    pairs, cnt = np.unique(np.stack([ct[sel], labels[sel]], 1), axis=0, return_counts=True)
    order = np.lexsort((-cnt, pairs[:, 0]))
    first = np.concatenate([[True], pairs[order][1:, 0] != pairs[order][:-1, 0]])
    lab[pairs[order][first, 0]] = pairs[order][first, 1]
    return lab


@pytest.fixture(scope="module")
def smeared():
    p = synth.GenParams(seed=31, n_primaries=1500, n_secondaries=0, sectors=SECTORS)
    ev = synth.generate(p, truth=True)
    ref = oracle.run(ev.clusters)
    return ev, ref, merge.merge(ref, ev.clusters)


def test_noiseless_helix_across_sectors_is_recovered():
    p = synth.GenParams(seed=32, n_primaries=400, n_secondaries=0, sectors=SECTORS, sigma_y=0.0, sigma_z=0.0,
                        row_eff=1.0, noise_frac=0.0)
    ev = synth.generate(p, truth=True)
    ref = oracle.run(ev.clusters)
    mg = merge.merge(ref, ev.clusters)
    lab = _labels(ev, ref)
    assert len(mg["chains"]) >= 20
    checked = 0
    for k, ch in enumerate(mg["chains"]):
        if not mg["ok"][k] or len({lab[g] for g in ch}) != 1:
            continue
        inner = ch[0]
        cl = np.nonzero(ref["cluster_track"] == inner)[0]
        c0 = cl[np.argmin(ev.clusters["row"][cl])]
        t = ev.truth[c0]
        truth = np.array([t["y"], t["z"], t["sphi"], t["tgl"], t["qpt"]])
        sig = np.sqrt(np.abs(mg["cov"][k][[0, 2, 5, 9, 14]]))
        assert np.all(np.abs(mg["par"][k] - truth) <= 0.05 * sig + 1e-9), (k, mg["par"][k], truth)
        assert mg["chi2"][k] <= 1e-6 * mg["ndf"][k]
        checked += 1
    assert checked >= 20


def test_split_tracks_are_merged_and_others_not(smeared):
    ev, ref, mg = smeared
    lab = _labels(ev, ref)
    seg = mg["segments"]
    ok = seg["refit_ok"] & (seg["n"] >= 10)
    # true split pairs: two segments of one track in neighbouring sectors
    true_pairs = set()
    by_lab = {}
    for g in np.nonzero(ok & (lab >= 0))[0]:
        by_lab.setdefault(int(lab[g]), []).append(int(g))
    for gs in by_lab.values():
        for a in gs:
            for b in gs:
                if a != b and merge.adjacent_sectors(seg["sector"][a], seg["sector"][b]) and \
                        seg["row_in"][a] < seg["row_in"][b] and seg["row_out"][a] <= seg["row_in"][b] + 10:
                    true_pairs.add((a, b))
    assert len(true_pairs) >= 30
    merged = {(a, int(b)) for a, b in enumerate(mg["link"]) if b >= 0}
    found = len(true_pairs & merged) / len(true_pairs)
    assert found >= 0.9, found
    wrong = [(a, b) for a, b in merged if lab[a] != lab[b]]
    assert len(wrong) <= 0.02 * len(merged), wrong
    # the pair chi2 of the true merged pairs: five degrees of freedom
    c2 = np.array([mg["pair_chi2"][a] for a, b in true_pairs & merged])
    assert 3.0 <= np.median(c2) <= 6.0, np.median(c2)


def test_merged_refit_matches_its_pieces(smeared):
    """The merged track has every cluster of its segments, and its fit at
    the innermost cluster agrees with the inner segment's own fit within
    the inner segment's errors (the outer clusters only add information)."""
    ev, ref, mg = smeared
    seg = mg["segments"]
    for k, ch in enumerate(mg["chains"]):
        if not mg["ok"][k]:
            continue
        assert mg["n"][k] == sum(seg["n"][g] for g in ch)
        inner = ch[0]
        sig = np.sqrt(np.abs(seg["cov"][inner][[0, 2, 5, 9, 14]]))
        assert np.all(np.abs(mg["par"][k] - seg["par"][inner]) <= 5 * sig + 1e-6)
        assert np.all(np.sqrt(np.abs(mg["cov"][k][[0, 2, 5, 9, 14]])) <= sig * (1 + 1e-6))


def test_z_window_only_prunes(smeared):
    """A pair within the chi2 cut has |dz| <= 5 sigma_z at the partner's
    first row, far inside the 10 cm window: pairing without the window, or
    with a window of 2 cm, makes the same choices with the same chi2."""
    ev, ref, mg = smeared
    seg = mg["segments"]
    wide = merge.pairs(seg, {"window_cm": 1e9})
    narrow = merge.pairs(seg, {"window_cm": 2.0})
    for other in (wide, narrow):
        assert np.array_equal(other["link"], mg["link"])
        assert np.array_equal(other["chi2"], mg["pair_chi2"])
    # and a window below the residuals does cut true pairs
    tiny = merge.pairs(seg, {"window_cm": 1e-3})
    assert (tiny["link"] >= 0).sum() < 0.1 * (mg["link"] >= 0).sum()
