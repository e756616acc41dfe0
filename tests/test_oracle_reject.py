"""Pins of the cluster-rejection oracle (the paper's compression section).

Exact helix states -- the generator's truth at every crossing, turned into
the tracker's outward convention -- are classified as the generator's own
geometry fixes them: momentum and dip from the drawn kinematics; for a
primary (a circle through the beam axis, so |c| + R = 2R) the z at the
beam axis is t * 2 pi R * ceil(k/2) on its k-th further leg.  On tracked
events the segments of further legs are rejected and first legs kept, with
z_ref for an event and the found vertices for continuous read-out.  A
planted sign error is caught."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import reject, vertex

K = 0.299792458e-3 * 5.0
SECTORS = (0, 1, 2, 18, 19, 20)


def _states(ev, p):
    """Truth states at every crossing in the tracker's convention (cos phi
    > 0: a crossing run inward is seen with sin phi, t and q/pT negated),
    with each crossing's track kinematics and leg."""
    tr = ev.truth
    sel = tr["track"] >= 0
    tr, cl = tr[sel], ev.clusters[sel]
    tt = synth.track_table(p)[tr["track"]]
    sg = np.where((tr["flags"] & 1) != 0, -1.0, 1.0)
    par = np.stack([tr["y"], tr["z"], sg * tr["sphi"], sg * tr["tgl"], sg * tr["qpt"]], 1)
    return vertex.row_x(cl["row"]), par, tt, tr["flags"] >> 1


def _leg_offset(tt, leg):
    """z at the beam axis of a primary on its leg: the nearest axis passage
    is after ceil(leg/2) full turns of length 2 pi R, R = pT / K."""
    R = tt["pt"] / K
    return tt["t"] * 2.0 * math.pi * R * np.ceil(leg / 2.0), 2.0 * R


def _check_truth(ev, p, prm):
    x, par, tt, leg = _states(ev, p)
    out = reject.classify(x, par, prm)
    bits = out["bits"]
    mom = tt["pt"] * np.sqrt(1.0 + tt["t"] ** 2)
    clear = np.abs(mom - prm["p_min"]) > 1e-9
    assert np.array_equal((bits[clear] & reject.LOW_P) != 0, mom[clear] < prm["p_min"])
    clear = np.abs(np.abs(tt["t"]) - prm["tgl_max"]) > 1e-9
    assert np.array_equal((bits[clear] & reject.INCLINED) != 0, np.abs(tt["t"][clear]) > prm["tgl_max"])
    prim = (tt["xv"] == 0.0) & (tt["yv"] == 0.0)
    z_exp, reach = _leg_offset(tt, leg)
    rho = np.hypot(x, par[:, 0])
    far = rho > reach * (1.0 - 1e-7)  # at the farthest point both axis passages are equally near
    ok = prim & ~far
    bad_z = np.abs(out["z_axis"][ok] - z_exp[ok]) > 1e-6 * (1.0 + np.abs(z_exp[ok]))
    bad_r = np.abs(out["reach"][ok] - reach[ok]) > 1e-6 * reach[ok]
    looper = reach < reject.X_OUT
    exp_leg = looper & (np.abs(z_exp) > prm["dz_leg"])
    clear = ok & (np.abs(reach - reject.X_OUT) > 1e-6) & (np.abs(np.abs(z_exp) - prm["dz_leg"]) > 1e-6)
    bad_leg = ((bits[clear] & reject.LOOPER_LEG) != 0) != exp_leg[clear]
    return {"z": int(bad_z.sum()), "reach": int(bad_r.sum()), "leg": int(bad_leg.sum()),
            "n_leg": int(exp_leg[clear].sum()), "n_first": int((clear & (leg == 0)).sum()),
            "n_low_p": int((mom < prm["p_min"]).sum()), "n_inclined": int((np.abs(tt["t"]) > prm["tgl_max"]).sum())}


@pytest.fixture(scope="module")
def looper_truth():
    p = synth.GenParams(seed=41, n_primaries=6000, n_secondaries=3000, eta_max=1.5, pt_min=0.04, sec_r_max=200.0,
                        legs=4, sectors=SECTORS)
    return synth.generate(p, truth=True), p


def test_truth_states_are_classified_by_the_generator_geometry(looper_truth):
    ev, p = looper_truth
    r = _check_truth(ev, p, reject.default_params())
    assert r["z"] == 0 and r["reach"] == 0 and r["leg"] == 0, r
    assert r["n_leg"] > 1000 and r["n_first"] > 1000 and r["n_low_p"] > 100 and r["n_inclined"] > 100, r


def test_a_planted_sign_error_is_caught(looper_truth, monkeypatch):
    ev, p = looper_truth
    real = vertex.dca_path

    def flipped(*a):
        path, dist = real(*a)
        return -path, dist

    monkeypatch.setattr(reject.vertex, "dca_path", flipped)
    r = _check_truth(ev, p, reject.default_params())
    assert r["z"] > 100 and r["leg"] > 100, r


def _segment_truth(ev, ref, p):
    """Per oracle track: its majority label, that label's kinematics and the
    majority leg of its clusters."""
    ct = ref["cluster_track"].astype(np.int64)
    sel = (ct >= 0) & (ev.truth["track"] >= 0)
    key = ct[sel] * 8 + (ev.truth["flags"][sel] >> 1).clip(0, 7)
    lab = ev.truth["track"][sel]
    m = ref["n_tracks"]
    pairs, cnt = np.unique(np.stack([key, lab], 1), axis=0, return_counts=True)
    best = np.full(m, -1, np.int64)
    best_leg = np.full(m, -1, np.int64)
    top = np.zeros(m, np.int64)
    for (k, l), c in zip(pairs, cnt):
        t = k // 8
        if c > top[t]:
            top[t], best[t], best_leg[t] = c, l, k % 8
    return best, best_leg


def test_tracked_event_rejects_further_legs_and_keeps_first_ones(looper_truth):
    ev, p = looper_truth
    ref = oracle.run(ev.clusters)
    prm = reject.default_params()
    out = reject.from_oracle_run(ref, len(ev.clusters), prm)
    lab, leg = _segment_truth(ev, ref, p)
    tt = synth.track_table(p)
    has = lab >= 0
    k = tt[np.maximum(lab, 0)]
    prim = has & (k["xv"] == 0.0) & (k["yv"] == 0.0)
    z_exp, reach = _leg_offset(k, np.maximum(leg, 0))
    clear = prim & (np.abs(reach - reject.X_OUT) > 2.0) & (np.abs(np.abs(z_exp) - prm["dz_leg"]) > 5.0)
    exp_leg = (reach < reject.X_OUT) & (np.abs(z_exp) > prm["dz_leg"])
    got = (out["bits"] & reject.LOOPER_LEG) != 0
    further = clear & exp_leg
    first = clear & ~exp_leg & (leg == 0)
    assert further.sum() > 200 and first.sum() > 300, (further.sum(), first.sum())
    assert got[further].mean() >= 0.95, got[further].mean()
    assert (~got[first]).mean() >= 0.98, (~got[first]).mean()
    # the keep mask follows the track classes
    ct = ref["cluster_track"].astype(np.int64)
    a = ct >= 0
    assert np.array_equal(out["keep"][a] == 0, out["bits"][ct[a]] != 0) and out["keep"][~a].all()
    # about half the clusters of this workload's mix go
    frac = 1.0 - out["keep"].mean()
    assert 0.25 <= frac <= 0.75, frac


def test_continuous_readout_uses_the_vertices():
    p = synth.GenParams(seed=42, n_primaries=5, n_secondaries=1, timeframe=True, tf_length_us=300.0, legs=4,
                        eta_max=1.5, pt_min=0.04)
    ev = synth.generate(p, truth=True)
    ref = oracle.run(ev.clusters)
    # the further legs of loopers pass the beam axis at times shifted by whole
    # turns: the vertices come from tracks above the looping momentum
    vx = vertex.from_oracle_run(ref, {"min_pt": 0.2})
    assert len(vx["v_time"]) >= 5
    prm = reject.default_params()
    out = reject.from_oracle_run(ref, len(ev.clusters), prm, vertices=vx)
    lab, leg = _segment_truth(ev, ref, p)
    tt = synth.track_table(p)
    k = tt[np.maximum(lab, 0)]
    prim = (lab >= 0) & (k["xv"] == 0.0) & (k["yv"] == 0.0)
    # collisions with a found vertex within 0.1 us
    near = np.array([np.abs(vx["v_time"] - tc).min() < 0.1 if len(vx["v_time"]) else False for tc in k["tc"]])
    z_exp, reach = _leg_offset(k, np.maximum(leg, 0))
    clear = prim & near & (np.abs(reach - reject.X_OUT) > 2.0) & (np.abs(np.abs(z_exp) - prm["dz_leg"]) > 5.0)
    exp_leg = (reach < reject.X_OUT) & (np.abs(z_exp) > prm["dz_leg"])
    got = (out["bits"] & reject.LOOPER_LEG) != 0
    first = clear & ~exp_leg & (leg == 0)
    further = clear & exp_leg
    assert first.sum() > 200 and further.sum() > 50, (first.sum(), further.sum())
    assert (~got[first]).mean() >= 0.97, (~got[first]).mean()
    # a further leg can land within dz_leg of another collision (one vertex
    # per ~75 cm of drift here: about a quarter of them); the rest are caught
    assert got[further].mean() >= 0.7, got[further].mean()
