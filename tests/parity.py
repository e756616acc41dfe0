"""Stage-by-stage comparison of the CUDA path with the FP64 oracle.

Bit-exact: grid (order, bin parameters, bin starts), links, tie flags,
tracklets.  Follow and selection: exact cluster lists and assignments except
for tracklets flagged as tainted on either side (a decision within the
divergence margin, taken in FP32 on the GPU and FP64 in the oracle) and the
tracklets sharing clusters with them; parameters within 1e-4 relative
(floors 1 cm, 1 cm, 0.01, 0.01, 0.01 c/GeV), covariances within 1e-3 relative
(to 0.1 sqrt(C_ii C_jj) where the entry is smaller than that).
"""
from __future__ import annotations

import json
import os

import numpy as np

TAINT = 1 | 2 | 4 | 8
PAR_FLOOR = np.array([1.0, 1.0, 0.01, 0.01, 0.01])
PAR_TOL = 1e-4
COV_TOL = 1e-3
NROW = 159
# A fit with chi2/ndf above this is not a track (its residuals are many
# sigma, e.g. a combinatorial candidate in a dense timeframe); the filter is
# then ill-conditioned and amplifies rounding, so its parameters are stated
# separately and held to ILLFIT_TOL.  Its clusters are compared exactly.
GOOD_CHI2_NDF = 10.0
ILLFIT_TOL = 1e-2


def tri_diag_index():
    return [i * (i + 1) // 2 + i for i in range(5)]


def par_rel_err(gpu, ref, ref_cov=None):
    """|gpu - ref| / max(|ref|, floor, sigma_ref): relative where the
    parameter is measured better than its value, in units of its own
    standard deviation where it is not (a q/pT of 0.01 with sigma 4 has no
    meaningful relative digits)."""
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    scale = np.maximum(np.abs(ref), PAR_FLOOR)
    if ref_cov is not None:
        scale = np.maximum(scale, np.sqrt(np.abs(np.asarray(ref_cov, np.float64)[..., tri_diag_index()])))
    return np.abs(gpu - ref) / scale


# Covariance tolerance (a reading of "covariances within 1e-3 relative"):
# relative to the entry for the diagonal and for entries whose correlation
# is at least 10%; for weaker correlations the entry itself is near zero and
# its natural scale is sqrt(C_ii C_jj), so the bound is 1e-4 in correlation
# units.  The binary32 transport and update over ~150 rows leave up to
# about 7e-5 in correlation units on short low-pT tracks.
COV_CORR_FLOOR = 1e-1


def cov_rel_err(gpu, ref):
    """|dC_ij| / max(|C_ij|, 0.1 sqrt(C_ii C_jj)): relative for every entry
    whose correlation reaches 10%, 1e-4 in correlation units below that."""
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    d = tri_diag_index()
    diag = np.abs(ref[..., d])
    err = np.zeros_like(ref)
    q = 0
    for i in range(5):
        for j in range(i + 1):
            scale = np.maximum(np.abs(ref[..., q]), COV_CORR_FLOOR * np.sqrt(diag[..., i] * diag[..., j]))
            err[..., q] = np.abs(gpu[..., q] - ref[..., q]) / np.maximum(scale, 1e-300)
            q += 1
    return err


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
    stats["follow_cov_corr_err_max"] = float(cov_corr_err(g["f_cov"][good], ref["f_cov"][good]).max()) \
        if good.any() else 0.0
    pb = par_rel_err(g["f_par"][bad_fit], ref["f_par"][bad_fit], ref["f_cov"][bad_fit])
    stats.update(tracklets=T, tainted=int(taint.sum()), diverged=int((~same).sum()),
                 follow_par_err_max=float(pe.max()) if pe.size else 0.0,
                 follow_cov_err_max=float(ce.max()) if ce.size else 0.0,
                 follow_par_err_p99=float(np.percentile(pe.max(1), 99)) if pe.size else 0.0,
                 follow_illfit=int(bad_fit.sum()),
                 follow_illfit_par_err_max=float(pb.max()) if pb.size else 0.0)
    assert stats["follow_illfit_par_err_max"] <= ILLFIT_TOL, stats
    return taint | ~same


def compare_selection(g, gct, ref, excluded_tl, stats):
    """Cluster -> tracklet-of-track assignment outside the divergence shadow."""
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
    # map track index -> tracklet id on both sides, then compare per cluster (load order)
    perm = ref["perm"]
    g_tl_of_track = np.full(max(int(g["tl_track"].max(initial=-1)) + 1, 1), -1)
    kept = np.nonzero(g["tl_track"] >= 0)[0]
    g_tl_of_track[g["tl_track"][kept]] = kept
    r_tl_of_track = np.full(max(int(ref["tl_track"].max(initial=-1)) + 1, 1), -1)
    kept_r = np.nonzero(ref["tl_track"] >= 0)[0]
    r_tl_of_track[ref["tl_track"][kept_r]] = kept_r
    a = np.where(gct >= 0, g_tl_of_track[np.maximum(gct, 0)], -1)
    b = np.where(ref["cluster_track"] >= 0, r_tl_of_track[np.maximum(ref["cluster_track"], 0)], -1)
    shadow_load = np.zeros(len(perm), bool)
    shadow_load[perm[sc2]] = True
    diff = (a != b) & ~shadow_load
    assert not diff.any(), f"{diff.sum()} cluster assignments differ outside the divergence shadow"
    stats.update(clusters=len(perm), shadow_clusters=int(shadow_load.sum()),
                 assigned_equal=int(((a == b) & ~shadow_load).sum()))
    return touched | excluded_tl


def compare_refit(tracks, ref, g, excluded, stats):
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
    good = ref["t_chi2"][ri] <= GOOD_CHI2_NDF * np.maximum(ref["t_ndf"][ri], 1)
    pe = par_rel_err(tg["par"][good], ref["t_par"][ri][good], ref["t_cov"][ri][good])
    ce = cov_rel_err(tg["cov"][good], ref["t_cov"][ri][good])
    cc = cov_corr_err(tg["cov"][good], ref["t_cov"][ri][good])
    pb = par_rel_err(tg["par"][~good], ref["t_par"][ri][~good], ref["t_cov"][ri][~good])
    chi = np.abs(tg["chi2"][good] - ref["t_chi2"][ri][good]) / np.maximum(ref["t_chi2"][ri][good], 1.0)
    stats.update(tracks_compared=int(len(common)), tracks_gpu=int(len(tracks)), tracks_ref=int(len(r_tl)),
                 refit_par_err_max=float(pe.max()) if pe.size else 0.0,
                 refit_cov_err_max=float(ce.max()) if ce.size else 0.0,
                 refit_cov_corr_err_max=float(cc.max()) if cc.size else 0.0,
                 refit_chi2_err_max=float(chi.max()) if chi.size else 0.0,
                 refit_illfit=int((~good).sum()),
                 refit_illfit_par_err_max=float(pb.max()) if pb.size else 0.0)
    assert stats["refit_illfit_par_err_max"] <= ILLFIT_TOL, stats
    assert (pe <= PAR_TOL).all(), f"refit params beyond 1e-4: max {pe.max()}"
    assert (ce <= COV_TOL).all(), f"refit covariance beyond 1e-3: max {ce.max()}"


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


def full_parity(trk, clusters, ref, req_offsets=None, graph=False, vertices=None):
    """Run the CUDA path and compare every stage; returns the statistics.
    vertices: a dict of tpc_vertex_config fields to also compare vertex
    finding in the drift time (one request)."""
    stats = {}
    tracks, gct, _ = trk.track(clusters, req_offsets, graph=graph)
    compare_grid(trk, ref)
    compare_links(trk, ref)
    compare_tracklets(trk, ref)
    g = follow_result(trk)
    excl = compare_follow(g, ref, stats)
    excl2 = compare_selection(g, gct, ref, excl, stats)
    if "follow_par_err_max" in stats:
        assert stats["follow_par_err_max"] <= PAR_TOL, stats
        assert stats["follow_cov_err_max"] <= COV_TOL, stats
    compare_refit(tracks, ref, g, excl2, stats)
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
