"""Stage-by-stage comparison of the CUDA path with the FP64 oracle.

Bit-exact: grid (order, bin parameters, bin starts), links, tie flags,
tracklets.  Follow and selection: exact cluster lists and assignments except
for tracklets flagged as tainted on either side (a decision within the
divergence margin, taken in binary32 on the GPU and in FP64 in the oracle)
and the tracklets sharing clusters with them -- the exclusion shadow, which
is bounded per case (SHADOW_MAX).  Fitted parameters within 1e-4 relative to
max(|value|, floor) with floors (1 cm, 1 cm, 0.01, 0.01, 0.01 c/GeV); a
parameter whose own standard deviation exceeds both (an unmeasured
curvature) is compared at 1e-4 of that deviation, and such results are
counted.  Covariances within 1e-3 relative for the diagonal and for entries
whose correlation reaches 0.1, within 1e-4 in correlation units below that.
"""
from __future__ import annotations

import json
import os

import numpy as np

TAINT = 1 | 2 | 4 | 8
PAR_FLOOR = np.array([1.0, 1.0, 0.01, 0.01, 0.01])
PAR_TOL = 1e-4
COV_TOL = 1e-3
# Below this correlation an entry is compared in correlation units
# |dC_ij| / sqrt(C_ii C_jj) <= COV_CORR_TOL: an entry near zero carries no
# relative digits, and 1e-4 there is the 1e-3 relative bound of an entry at
# the threshold.  Measured worst: 1.3e-5 (1 ms timeframes); relative worst
# above the threshold 8.3e-5.
COV_CORR_MIN = 0.1
COV_CORR_TOL = 1e-4
NROW = 159
# A fit with chi2/ndf above this is not a track (its residuals are many
# sigma, e.g. a combinatorial candidate in a dense timeframe).  Refitted
# tracks are held to the same bars either way (measured ill-fit worst 5.7e-5
# plain).  The follow state of such a candidate -- an intermediate whose only
# downstream use is as the refit's starting point -- is held to
# FOLLOW_ILLFIT_TOL: the filter, pulled by residuals of tens of sigma,
# amplifies binary32 rounding (measured worst 2.1e-4 on a 1 ms timeframe).
GOOD_CHI2_NDF = 10.0
FOLLOW_ILLFIT_TOL = 1e-3
# Largest share of a case's clusters, and of its oracle tracks, that the
# exclusion shadow may take (measured at most 1.2% and 1.1% with the 1e-4
# divergence margin), so that over-set taint flags cannot hide divergences.
SHADOW_MAX = 0.03


def tri_diag_index():
    return [i * (i + 1) // 2 + i for i in range(5)]


def _sigma(ref_cov):
    return np.sqrt(np.abs(np.asarray(ref_cov, np.float64)[..., tri_diag_index()]))


def par_plain_err(gpu, ref):
    """|gpu - ref| / max(|ref|, floor): the parameter tolerance as stated."""
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    return np.abs(gpu - ref) / np.maximum(np.abs(ref), PAR_FLOOR)


def par_rel_err(gpu, ref, ref_cov=None):
    """|gpu - ref| / max(|ref|, floor, sigma_ref): the stated relative error,
    except for a parameter whose standard deviation exceeds its value and
    floor (a q/pT of 0.0015 with sigma 3 has no relative digits): that one is
    measured in units of its own deviation."""
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    scale = np.maximum(np.abs(ref), PAR_FLOOR)
    if ref_cov is not None:
        scale = np.maximum(scale, _sigma(ref_cov))
    return np.abs(gpu - ref) / scale


def par_sigma_reading_count(gpu, ref, ref_cov):
    """(results beyond the plain 1e-4 bar, of which undetermined: sigma above
    value and floor).  The tolerance holds only if the two are equal."""
    e = par_plain_err(gpu, ref)
    und = _sigma(ref_cov) > np.maximum(np.abs(np.asarray(ref, np.float64)), PAR_FLOOR)
    over = e > PAR_TOL
    return int(over.any(axis=-1).sum()), int((over & und).any(axis=-1).sum()), int((over & ~und).sum())


def cov_rel_err(gpu, ref):
    """Per entry the covariance error in units of its bound: |dC_ij| /
    (COV_TOL |C_ij|) for the diagonal and for |corr_ij| >= COV_CORR_MIN,
    |dC_ij| / (COV_CORR_TOL sqrt(C_ii C_jj)) below that; <= 1 passes."""
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    d = tri_diag_index()
    diag = np.abs(ref[..., d])
    err = np.zeros_like(ref)
    q = 0
    for i in range(5):
        for j in range(i + 1):
            s = np.sqrt(diag[..., i] * diag[..., j])
            e = np.abs(gpu[..., q] - ref[..., q])
            strong = (np.abs(ref[..., q]) >= COV_CORR_MIN * s) | (i == j)
            err[..., q] = np.where(strong, e / np.maximum(COV_TOL * np.abs(ref[..., q]), 1e-300),
                                   e / np.maximum(COV_CORR_TOL * s, 1e-300))
            q += 1
    return err


def cov_parts(gpu, ref):
    """(worst relative error of the entries compared relatively, worst error
    in correlation units of the others)."""
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    if gpu.size == 0:
        return 0.0, 0.0
    d = tri_diag_index()
    diag = np.abs(ref[..., d])
    rel, corr = 0.0, 0.0
    q = 0
    for i in range(5):
        for j in range(i + 1):
            s = np.sqrt(diag[..., i] * diag[..., j])
            e = np.abs(gpu[..., q] - ref[..., q])
            strong = (np.abs(ref[..., q]) >= COV_CORR_MIN * s) | (i == j)
            if strong.any():
                rel = max(rel, float((e[strong] / np.maximum(np.abs(ref[..., q][strong]), 1e-300)).max()))
            if (~strong).any():
                corr = max(corr, float((e[~strong] / np.maximum(s[~strong], 1e-300)).max()))
            q += 1
    return rel, corr


def cov_corr_err(gpu, ref):
    """|dC_ij| / sqrt(C_ii C_jj): the covariance error in correlation units."""
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    diag = np.abs(ref[..., tri_diag_index()])
    err = np.zeros_like(ref)
    q = 0
    for i in range(5):
        for j in range(i + 1):
            err[..., q] = np.abs(gpu[..., q] - ref[..., q]) / np.maximum(np.sqrt(diag[..., i] * diag[..., j]), 1e-300)
            q += 1
    return err


def compare_grid(trk, ref):
    perm = trk.stage("perm")
    assert np.array_equal(perm, ref["perm"]), "sorted order differs"
    assert np.array_equal(trk.stage("rs_of"), ref["rs_of"])
    assert np.array_equal(trk.stage("row_start"), ref["row_start"])
    p = trk.stage("rs_params")
    for k in ("z_lo", "z_hi"):
        assert np.array_equal(p[k], ref[k]), k
    for k in ("inv_y", "inv_z"):
        assert np.array_equal(p[k].view(np.uint32), ref[k].view(np.uint32)), k
    for k in ("n_y", "n_z"):
        assert np.array_equal(p[k], ref[k]), k
    assert np.array_equal(p["bin_base"], ref["bin_base"][:-1].astype(np.int32))
    assert np.array_equal(p["count"], np.diff(ref["row_start"]))
    assert np.array_equal(trk.stage("bin_start"), ref["bin_start"])


def compare_links(trk, ref):
    for k in ("up", "dn", "tie", "up_m", "dn_m"):
        assert np.array_equal(trk.stage(k), ref[k]), k


def compare_tracklets(trk, ref):
    assert np.array_equal(trk.stage("tl_start"), ref["tl_start"])
    assert np.array_equal(trk.stage("tl_len"), ref["tl_len"])


def follow_result(trk):
    return {k: trk.stage(k) for k in ("f_n", "f_nf", "f_nb", "f_flags", "f_row", "f_hits", "f_par", "f_cov",
                                      "f_chi2", "owner", "tl_track")}


def compare_follow(g, ref, stats):
    """Exact cluster lists for untainted tracklets, tolerances on their state."""
    T = len(ref["f_n"])
    assert len(g["f_n"]) == T
    taint = ((g["f_flags"] & TAINT) != 0) | ((ref["f_flags"] & TAINT) != 0)
    same = (g["f_n"] == ref["f_n"]) & (g["f_nf"] == ref["f_nf"]) & (g["f_nb"] == ref["f_nb"])
    for t in np.nonzero(same)[0]:
        n = g["f_n"][t]
        if not np.array_equal(g["f_hits"][t, :n], ref["f_hits"][t, :n]):
            same[t] = False
    bad = ~same & ~taint
    assert not bad.any(), f"{bad.sum()} untainted tracklets differ, e.g. {np.nonzero(bad)[0][:10]}"
    fail_mask = ((g["f_flags"] ^ ref["f_flags"]) & (16 | 32)) != 0
    assert not (fail_mask & ~taint).any(), "seed/backward failure flags differ"
    ok = same & ~taint & (g["f_n"] > 0)
    assert np.array_equal(g["f_row"][ok], ref["f_row"][ok])
    good = ok & (ref["f_chi2"] <= GOOD_CHI2_NDF * np.maximum(2 * ref["f_n"] - 5, 1))
    bad_fit = ok & ~good
    pe = par_rel_err(g["f_par"][good], ref["f_par"][good], ref["f_cov"][good])
    ce = cov_rel_err(g["f_cov"][good], ref["f_cov"][good])
    rel, corr = cov_parts(g["f_cov"][good], ref["f_cov"][good])
    n_over, n_und, n_det = par_sigma_reading_count(g["f_par"][good], ref["f_par"][good], ref["f_cov"][good])
    pb = par_rel_err(g["f_par"][bad_fit], ref["f_par"][bad_fit], ref["f_cov"][bad_fit])
    cb = cov_rel_err(g["f_cov"][bad_fit], ref["f_cov"][bad_fit])
    flags = g["f_flags"] | ref["f_flags"]
    stats.update(tracklets=T, tainted=int(taint.sum()), diverged=int((~same).sum()),
                 tainted_by={k: int(((flags & b) != 0).sum()) for k, b in (("tie", 1), ("gate", 2), ("edge", 4),
                                                                           ("slim", 8))},
                 follow_par_err_max=float(pe.max()) if pe.size else 0.0,
                 follow_par_plain_err_max=float(par_plain_err(g["f_par"][good], ref["f_par"][good]).max())
                 if pe.size else 0.0,
                 follow_par_beyond_plain=n_over, follow_par_beyond_plain_undetermined=n_und,
                 follow_cov_err_max=float(ce.max()) if ce.size else 0.0,
                 follow_cov_rel_err_max=rel, follow_cov_corr_err_max=corr,
                 follow_illfit=int(bad_fit.sum()),
                 follow_illfit_par_err_max=float(pb.max()) if pb.size else 0.0,
                 follow_illfit_cov_err_max=float(cb.max()) if cb.size else 0.0)
    # every result beyond the plain bar is an undetermined parameter
    assert n_det == 0, stats
    assert stats["follow_illfit_par_err_max"] <= FOLLOW_ILLFIT_TOL, stats
    assert stats["follow_illfit_cov_err_max"] <= 1.0, stats
    return taint | ~same


def _tracklet_of_cluster(tl_track, cluster_track):
    """Per cluster (load order) the tracklet id of the track that owns it, -1
    when unassigned."""
    tl_of = np.full(max(int(tl_track.max(initial=-1)) + 1, 1), -1)
    kept = np.nonzero(tl_track >= 0)[0]
    tl_of[tl_track[kept]] = kept
    return np.where(cluster_track >= 0, tl_of[np.maximum(cluster_track, 0)], -1)


def compare_selection(g, gct, ref, excluded_tl, stats, shadow_max=SHADOW_MAX):
    """Cluster -> tracklet-of-track assignment outside the divergence shadow;
    the shadow is bounded and the mismatches over all clusters are counted."""
    T = len(ref["f_n"])
    hits_g, hits_r = g["f_hits"], ref["f_hits"]
    n_g, n_r = g["f_n"], ref["f_n"]
    shadow_clusters = set()
    for t in np.nonzero(excluded_tl)[0]:
        shadow_clusters.update(hits_g[t, :n_g[t]].tolist())
        shadow_clusters.update(hits_r[t, :n_r[t]].tolist())
    # tracklets touching those clusters, then all of their clusters
    sc = np.zeros(len(ref["perm"]), bool)
    if shadow_clusters:
        sc[np.fromiter(shadow_clusters, np.int64)] = True
    touched = np.zeros(T, bool)
    for t in range(T):
        if (n_g[t] and sc[hits_g[t, :n_g[t]]].any()) or (n_r[t] and sc[hits_r[t, :n_r[t]]].any()):
            touched[t] = True
    sc2 = sc.copy()
    for t in np.nonzero(touched)[0]:
        sc2[hits_g[t, :n_g[t]]] = True
        sc2[hits_r[t, :n_r[t]]] = True
    perm = ref["perm"]
    a = _tracklet_of_cluster(g["tl_track"], gct)
    b = _tracklet_of_cluster(ref["tl_track"], ref["cluster_track"])
    shadow_load = np.zeros(len(perm), bool)
    shadow_load[perm[sc2]] = True
    diff = (a != b) & ~shadow_load
    assert not diff.any(), f"{diff.sum()} cluster assignments differ outside the divergence shadow"
    n = max(len(perm), 1)
    stats.update(clusters=len(perm), shadow_clusters=int(shadow_load.sum()),
                 shadow_cluster_frac=float(shadow_load.sum()) / n,
                 assigned_equal=int(((a == b) & ~shadow_load).sum()),
                 assign_mismatch_all=int((a != b).sum()))
    assert stats["shadow_cluster_frac"] <= shadow_max, stats
    return touched | excluded_tl


def compare_refit(tracks, ref, g, excluded, stats, shadow_max=SHADOW_MAX):
    g_tl = np.nonzero(g["tl_track"] >= 0)[0]
    r_tl = ref["t_tracklet"]
    common = np.intersect1d(g_tl, r_tl)
    common = common[~excluded[common]]
    gi = g["tl_track"][common]
    ri = ref["tl_track"][common]
    # the refit's own near-limit decisions (|sin phi| at the limit) taint too
    rt = ((tracks["flags"][gi] & TAINT) != 0) | ((ref["t_flags"][ri] & TAINT) != 0)
    stats["refit_tainted"] = int(rt.sum())
    common, gi, ri = common[~rt], gi[~rt], ri[~rt]
    tg, = (tracks[gi],)
    assert np.array_equal(tg["n_clusters"], ref["t_n"][ri])
    assert np.array_equal(tg["first_row"], np.where(ref["t_flags"][ri] & 64, tg["first_row"], ref["t_row_in"][ri]))
    assert np.array_equal(tg["last_row"], ref["t_row_out"][ri])
    assert np.array_equal(tg["ndf"], ref["t_ndf"][ri])
    okf = (tg["flags"] & 64) == (ref["t_flags"][ri] & 64)
    assert okf.all()
    # every refitted track, ill fits included, is held to the same bars
    pe = par_rel_err(tg["par"], ref["t_par"][ri], ref["t_cov"][ri])
    ce = cov_rel_err(tg["cov"], ref["t_cov"][ri])
    rel, corr = cov_parts(tg["cov"], ref["t_cov"][ri])
    n_over, n_und, n_det = par_sigma_reading_count(tg["par"], ref["t_par"][ri], ref["t_cov"][ri])
    chi = np.abs(tg["chi2"] - ref["t_chi2"][ri]) / np.maximum(ref["t_chi2"][ri], 1.0)
    good = ref["t_chi2"][ri] <= GOOD_CHI2_NDF * np.maximum(ref["t_ndf"][ri], 1)
    n_ref = max(len(r_tl), 1)
    stats.update(tracks_compared=int(len(common)), tracks_gpu=int(len(tracks)), tracks_ref=int(len(r_tl)),
                 shadow_track_frac=1.0 - len(common) / n_ref,
                 refit_par_err_max=float(pe.max()) if pe.size else 0.0,
                 refit_par_plain_err_max=float(par_plain_err(tg["par"], ref["t_par"][ri]).max()) if pe.size else 0.0,
                 refit_par_beyond_plain=n_over, refit_par_beyond_plain_undetermined=n_und,
                 refit_cov_err_max=float(ce.max()) if ce.size else 0.0,
                 refit_cov_rel_err_max=rel, refit_cov_corr_err_max=corr,
                 refit_chi2_err_max=float(chi.max()) if chi.size else 0.0,
                 refit_illfit=int((~good).sum()))
    assert n_det == 0, stats
    assert (pe <= PAR_TOL).all(), f"refit params beyond 1e-4: max {pe.max()}"
    assert (ce <= 1.0).all(), f"refit covariance beyond its bound: {rel} relative, {corr} correlation units"
    assert stats["shadow_track_frac"] <= shadow_max, stats


VERTEX_TRACK_DT = 2e-3   # us: per-track time estimate (binary32 state and extrapolation)
VERTEX_GAP_MARGIN = 1e-2  # us: a cut this close to the gap may fall either way
VERTEX_USE_MARGIN = 1e-2  # cm: participation decided this close to dca_max or ext_max


def compare_vertices(trk, tracks, ref, g, excluded, stats, **cfg):
    """Vertex finding in the drift time against the FP64 oracle run on the
    oracle's own tracks: per matched track the time estimate, participation
    and vertex, per vertex the time and membership, per track the spatial z.
    Tracks in the exclusion shadow, ill fits and decisions within the margins
    above are not compared; the numbers are recorded."""
    from oracle import vertex
    pmap = {"vdrift_cm_us": "vdrift", "zmax_cm": "zmax", "dca_max_cm": "dca_max", "ext_max_cm": "ext_max",
            "gap_us": "gap", "min_tracks": "min_tracks", "min_clusters": "min_clusters"}
    vr = vertex.from_oracle_run(ref, {pmap[k]: v for k, v in cfg.items()})
    gv = trk.find_vertices(**cfg).vertices()
    g_tl = np.nonzero(g["tl_track"] >= 0)[0]
    common = np.intersect1d(g_tl, ref["t_tracklet"])
    common = common[~excluded[common]]
    gi, ri = g["tl_track"][common], ref["tl_track"][common]
    good = ref["t_chi2"][ri] <= GOOD_CHI2_NDF * np.maximum(ref["t_ndf"][ri], 1)
    gi, ri = gi[good], ri[good]
    dt = np.abs(gv["track_time"][gi].astype(np.float64) - vr["t_est"][ri])
    fin = np.isfinite(vr["t_est"][ri])
    assert (dt[fin] <= VERTEX_TRACK_DT + 1e-6 * np.abs(vr["t_est"][ri][fin])).all(), dt[fin].max()
    g_use = gv["track_vertex"] >= 0
    # participation: the GPU keeps no per-track flag; a track with a vertex took part
    sure = vr["use_margin"][ri] > VERTEX_USE_MARGIN
    # vertex matching by time; vertices whose cut falls within the margin are skipped
    gt = gv["vertices"]["time_us"]
    taint_v = vr["v_margin"] <= VERTEX_GAP_MARGIN
    mapping = {}
    for k, t in enumerate(vr["v_time"]):
        if taint_v[k] or not len(gt):
            continue
        j = int(np.argmin(np.abs(gt - t)))
        mapping[k] = j
    assert len(set(mapping.values())) == len(mapping)  # one GPU vertex per oracle vertex
    # membership of matched tracks
    rv = vr["vertex"][ri]
    check = sure & (rv >= 0) & np.isin(rv, list(mapping.keys()))
    exp = np.array([mapping[int(v)] for v in rv[check]], dtype=np.int64)
    assert np.array_equal(gv["track_vertex"][gi][check], exp)
    # an oracle track without a vertex has none on the GPU either (if its
    # decisions are clear and its would-be vertex is not tainted)
    none = sure & (rv < 0) & (vr["use"][ri] == False)  # noqa: E712
    assert (gv["track_vertex"][gi][none] < 0).all()
    # vertex times: the common members agree to VERTEX_TRACK_DT; members only
    # one side has (shadow) move the mean by at most their share of 2 us
    n_g = np.bincount(gv["track_vertex"][gv["track_vertex"] >= 0], minlength=len(gt))
    worst = 0.0
    for k, j in mapping.items():
        n = vr["v_n"][k]
        diff = abs(int(n_g[j]) - int(n))
        tol = VERTEX_TRACK_DT + 2.0 * (diff + max(1, int(0.01 * n))) / n
        err = abs(gt[j] - vr["v_time"][k])
        worst = max(worst, err)
        assert err <= tol, (k, err, tol)
    # spatial z of matched tracks
    zc = check
    zg = gv["track_z"][gi][zc].astype(np.float64)
    zr = vr["z"][ri][zc]
    dvt = np.abs(gt[exp] - vr["v_time"][rv[check]])
    zerr = np.abs(zg - zr)
    assert (zerr <= 2.5 * dvt + 1e-4 * np.maximum(np.abs(zr), 1.0) + 2.5 * VERTEX_TRACK_DT).all(), zerr.max()
    assert np.allclose(gv["track_tgl"][gi][zc], vr["tgl"][ri][zc], rtol=1e-4, atol=1e-4)
    stats.update(vertices_gpu=int(len(gt)), vertices_ref=int(len(vr["v_time"])),
                 vertices_compared=int(len(mapping)), vertices_tainted=int(taint_v.sum()),
                 vertex_time_err_max=float(worst), vertex_track_dt_max=float(dt[fin].max()) if fin.any() else 0.0,
                 vertex_tracks_checked=int(check.sum()), vertex_z_err_max=float(zerr.max()) if zerr.size else 0.0)
    return gv, vr


def full_parity(trk, clusters, ref, req_offsets=None, graph=False, vertices=None, shadow_max=SHADOW_MAX):
    """Run the CUDA path and compare every stage; returns the statistics.
    vertices: a dict of tpc_vertex_config fields to also compare vertex
    finding in the drift time (one request).  shadow_max: bound on the
    exclusion shadow's share of clusters and tracks (lifted only for inputs
    built to tie, e.g. duplicated clusters)."""
    stats = {}
    tracks, gct, _ = trk.track(clusters, req_offsets, graph=graph)
    compare_grid(trk, ref)
    compare_links(trk, ref)
    compare_tracklets(trk, ref)
    g = follow_result(trk)
    excl = compare_follow(g, ref, stats)
    excl2 = compare_selection(g, gct, ref, excl, stats, shadow_max)
    if "follow_par_err_max" in stats:
        assert stats["follow_par_err_max"] <= PAR_TOL, stats
        assert stats["follow_cov_err_max"] <= 1.0, stats
    compare_refit(tracks, ref, g, excl2, stats, shadow_max)
    if vertices is not None:
        compare_vertices(trk, tracks, ref, g, excl2, stats, **vertices)
    return stats


# Where the GPU tests append their per-case error statistics (one JSON line
# per case): TPC_PARITY_STATS_DIR, or parity_stats/ at the top of the repo.
STATS_DIR = os.environ.get("TPC_PARITY_STATS_DIR",
                           os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "parity_stats"))


def record_stats(name, stats):
    os.makedirs(STATS_DIR, exist_ok=True)
    with open(os.path.join(STATS_DIR, "parity_stats.jsonl"), "a") as f:
        f.write(json.dumps({"case": name, **stats}) + "\n")
