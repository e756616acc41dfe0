"""FP64 oracle of vertex finding in the drift-time coordinate (test infrastructure only).

Continuous read-out (Sec. 5): the time of a collision is unknown before
tracking, so the tracks are found and fitted with z replaced by the drift
coordinate z_t, the collision times are estimated from the tracks, and only
then is z_t converted to the spatial z.  The paper gives the order of these
steps and no details; this module writes out the reading used here, step by
step, in FP64 with numpy:

1. Time estimate of a track.  From its fitted state at the innermost row
   (x, y, z_t, sin phi, t = dz_t/ds_T, q/pT) the helix is followed to its
   point of closest approach to the beam axis in the transverse plane;
   z_t there is v_d * t_coll + z_max for a track from a collision at z = 0,
   so t_est = (z_t(dca) - z_max) / v_d.
2. A track takes part when |dca| <= dca_max, it has at least min_clusters
   clusters, its extrapolation moves z_t by at most ext_max (no track
   from the beam line crosses more than the drift length) and its pT is at
   least min_pt (0: no cut; a cut above the looping momentum keeps the
   further legs of loopers, whose times are shifted by whole turns, out).
3. The participating tracks of a request, sorted by t_est, are cut wherever
   two neighbours are more than `gap` apart; a run of at least min_tracks
   tracks is a vertex, its time the mean t_est of its tracks.
4. The tracks of a vertex get z = side * (z_max - (z_t - v_d * t_vertex))
   (side +1 for sectors 0..17, -1 for 18..35) and dz/ds_T = -side * t.

Only the tests, the package smoke check and the benchmark's CPU leg import it.
"""
from __future__ import annotations

import math

import numpy as np

NROW = 159
NSEC = 36


def default_params(**kw) -> dict:
    p = {"vdrift": 2.5, "zmax": 250.0, "dca_max": 2.0, "ext_max": 300.0, "gap": 0.5, "min_tracks": 3,
         "min_clusters": 20, "min_pt": 0.0, "bz_kg": 5.0}
    p.update(kw)
    return p


def row_x(row):
    """Row radii as the tracker uses them: the FP64 expression rounded to binary32."""
    return np.float32(85.2 + np.asarray(row, dtype=np.float64) * ((245.8 - 85.2) / 158.0)).astype(np.float64)


def dca_path(x, y, s, q, K):
    """Transverse path length from (x, y) with direction sin phi = s (cos phi
    > 0) and curvature kappa = -K q to the point of the helix closest to the
    beam axis, and the signed distance there.  Closed form: on the circle
    around c = (x - s/kappa, y + cos phi/kappa) the direction psi at the point
    of closest approach is perpendicular to c and the point is c minus
    1/|kappa| along c; the path length is (psi - phi)/kappa with psi - phi
    wrapped into (-pi, pi].  A straight track (kappa = 0) has path
    -(x cos phi + y sin phi)."""
    x, y, s, q = (np.asarray(a, dtype=np.float64) for a in (x, y, s, q))
    with np.errstate(invalid="ignore"):
        c = np.sqrt(1.0 - s * s)  # NaN for |s| >= 1: no estimate
    kappa = -K * q
    straight = np.abs(kappa) < 1e-12
    k = np.where(straight, 1.0, kappa)
    cx = x - s / k
    cy = y + c / k
    sg = np.sign(k)
    psi = np.arctan2(-sg * cx, sg * cy)
    phi = np.arctan2(s, c)
    dpsi = psi - phi
    dpsi = np.where(dpsi > math.pi, dpsi - 2 * math.pi, dpsi)
    dpsi = np.where(dpsi <= -math.pi, dpsi + 2 * math.pi, dpsi)
    path = np.where(straight, -(x * c + y * s), dpsi / k)
    dist = np.where(straight, np.abs(x * s - y * c), np.abs(np.hypot(cx, cy) - 1.0 / np.abs(k)))
    return path, dist


def track_times(x, par, p: dict):
    """Step 1: t_est, |dca| and the z_t change of the extrapolation of
    tracks with state par (n x 5) at radii x."""
    K = 0.299792458e-3 * p["bz_kg"]
    with np.errstate(invalid="ignore", divide="ignore"):
        path, dist = dca_path(x, par[:, 0], par[:, 2], par[:, 4], K)
        dzt = par[:, 3] * path
    return ((par[:, 1] - p["zmax"]) + dzt) / p["vdrift"], dist, dzt


def find_vertices(x, par, n_clusters, sector, request, p: dict | None = None) -> dict:
    """Steps 1-4 for tracks given by their innermost radius x, state par,
    cluster count, sector and request.  Returns per track t_est, dca, the
    vertex index (-1: none), spatial z and dz/ds_T (NaN without a vertex),
    and per vertex its request, time, track count and the smallest margin of
    its two boundary gaps to the cut (|gap - cut|)."""
    p = default_params(**(p or {}))
    par = np.asarray(par, dtype=np.float64)
    m = len(par)
    t_est, dca, dzt = track_times(np.asarray(x, dtype=np.float64), par, p)
    with np.errstate(invalid="ignore"):
        use = (dca <= p["dca_max"]) & (np.asarray(n_clusters) >= p["min_clusters"]) & np.isfinite(t_est)
        use &= np.abs(dzt) <= p["ext_max"]
        if p["min_pt"] > 0:
            use &= np.abs(par[:, 4]) * p["min_pt"] <= 1.0
    vid = np.full(m, -1, np.int64)
    v_req, v_time, v_n, v_margin = [], [], [], []
    request = np.asarray(request)
    for r in np.unique(request[use]) if m else []:
        idx = np.nonzero(use & (request == r))[0]
        order = idx[np.argsort(t_est[idx], kind="stable")]
        ts = t_est[order]
        gaps = np.diff(ts)
        cuts = np.nonzero(gaps > p["gap"])[0]
        starts = np.concatenate([[0], cuts + 1])
        ends = np.concatenate([cuts + 1, [len(ts)]])
        for a, b in zip(starts, ends):
            if b - a < p["min_tracks"]:
                continue
            left = abs(gaps[a - 1] - p["gap"]) if a > 0 else np.inf
            right = abs(gaps[b - 1] - p["gap"]) if b < len(ts) else np.inf
            vid[order[a:b]] = len(v_time)
            v_req.append(int(r))
            v_time.append(float(ts[a:b].mean()))
            v_n.append(int(b - a))
            v_margin.append(float(min(left, right)))
    v_time = np.asarray(v_time, dtype=np.float64)
    side = np.where(np.asarray(sector) < NSEC // 2, 1.0, -1.0)
    tv = np.where(vid >= 0, v_time[np.maximum(vid, 0)] if len(v_time) else 0.0, np.nan)
    z = side * (p["zmax"] - (par[:, 1] - p["vdrift"] * tv))
    tgl = -side * par[:, 3]
    z = np.where(vid >= 0, z, np.nan)
    tgl = np.where(vid >= 0, tgl, np.nan)
    with np.errstate(invalid="ignore"):
        use_margin = np.minimum(np.abs(dca - p["dca_max"]), np.abs(np.abs(dzt) - p["ext_max"]))
        if p["min_pt"] > 0:  # relative distance of pT from the cut
            use_margin = np.minimum(use_margin, np.abs(np.abs(par[:, 4]) * p["min_pt"] - 1.0))
    return {"t_est": t_est, "dca": dca, "use": use, "use_margin": use_margin, "vertex": vid, "z": z, "tgl": tgl,
            "v_request": np.asarray(v_req, np.int64), "v_time": v_time, "v_n": np.asarray(v_n, np.int64),
            "v_margin": np.asarray(v_margin, np.float64)}


def from_oracle_run(ref: dict, p: dict | None = None) -> dict:
    """Vertices of the oracle's own refitted tracks (oracle.run output)."""
    tl = ref["t_tracklet"]
    rs = ref["rs_of"][ref["tl_start"][tl]] if len(tl) else np.zeros(0, np.int64)
    sector = (rs // NROW) % NSEC
    request = rs // (NROW * NSEC)
    return find_vertices(row_x(ref["t_row_in"]), ref["t_par"], ref["t_n"], sector, request, p)
