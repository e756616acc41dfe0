"""FP64 oracle of cluster rejection (test infrastructure only).

The paper's compression section: compression alone leaves a factor of about
two to the target, so the online reconstruction identifies the tracks that
physics does not use -- momentum below 50 MeV/c, the further legs of
looping tracks, segments at a high inclination -- and drops their clusters
(about half of all clusters).  The paper names the three classes and no
rules; the reading written out here, per fitted sector track (its state at
the innermost row, in its sector's frame; t = dz/ds_T), is:

1. LOW_P: momentum p = sqrt(1 + t^2) / |q/pT| below p_min (0.05 GeV/c).
2. INCLINED: |t| above tgl_max (2.0).
3. LOOPER_LEG: the track's circle stays inside the radius of the outermost
   pad row (|c| + R below it: a looper, whose particle spirals on inside
   the chamber), and at its point of closest approach to the beam axis
   (the vertex module's closed form) its z lies more than dz_leg (10 cm)
   from the collision.  Every leg of a helix from the collision passes the
   beam axis again after each full turn, with z moved by 2 pi R t, so only
   the first outgoing leg (or the leg running into it, for t near 0)
   points back to the collision.  The collision is z_ref for an event; for
   continuous read-out the nearest vertex of the request in time (vertex
   module): the distance is then v_drift * |t_est - t_vertex|.

A track is rejected when any class holds; so are its clusters.  Only the
tests, the package smoke check and the benchmark's CPU leg import it.
"""
from __future__ import annotations

import numpy as np

from . import vertex

LOW_P = 1
INCLINED = 2
LOOPER_LEG = 4

X_OUT = float(vertex.row_x(158))  # radius of the outermost pad row (binary32)


def default_params(**kw) -> dict:
    p = {"p_min": 0.05, "tgl_max": 2.0, "dz_leg": 10.0, "z_ref": 0.0, "bz_kg": 5.0, "vdrift": 2.5, "zmax": 250.0}
    p.update(kw)
    return p


def circle_reach(x, y, s, q, K):
    """Farthest distance of the track's circle from the beam axis, |c| + R
    (infinite for a straight track)."""
    x, y, s, q = (np.asarray(a, dtype=np.float64) for a in (x, y, s, q))
    with np.errstate(invalid="ignore", divide="ignore"):
        c = np.sqrt(1.0 - s * s)
        kappa = -K * q
        cx = x - s / kappa
        cy = y + c / kappa
        return np.where(kappa == 0.0, np.inf, np.hypot(cx, cy) + 1.0 / np.abs(kappa))


def classify(x, par, p: dict | None = None, vertices: dict | None = None, request=None) -> dict:
    """Class bits of tracks with state par (n x 5) at radii x.  vertices: the
    vertex module's output for continuous read-out (then request gives each
    track's request); else the collision is at z_ref.  Also returns, per
    track, the distance of each decision from its boundary (for the
    comparison with a binary32 implementation)."""
    p = default_params(**(p or {}))
    par = np.asarray(par, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    K = 0.299792458e-3 * p["bz_kg"]
    t, q = par[:, 3], par[:, 4]
    with np.errstate(divide="ignore", invalid="ignore"):
        mom = np.sqrt(1.0 + t * t) / np.abs(q)
    low_p = mom < p["p_min"]
    inclined = np.abs(t) > p["tgl_max"]
    reach = circle_reach(x, par[:, 0], par[:, 2], q, K)
    looper = reach < X_OUT
    with np.errstate(invalid="ignore"):
        path, _ = vertex.dca_path(x, par[:, 0], par[:, 2], q, K)
        z_axis = par[:, 1] + t * path
    if vertices is None:
        dz = np.abs(z_axis - p["z_ref"])
    else:
        t_est = (z_axis - p["zmax"]) / p["vdrift"]
        dz = np.full(len(par), np.inf)
        request = np.asarray(request)
        for r in np.unique(vertices["v_request"]):
            tv = np.sort(vertices["v_time"][vertices["v_request"] == r])
            sel = request == r
            dt = np.abs(t_est[sel][:, None] - tv[None, :]).min(axis=1) if len(tv) else np.full(sel.sum(), np.inf)
            dz[sel] = p["vdrift"] * dt
    with np.errstate(invalid="ignore"):
        leg = looper & (dz > p["dz_leg"])
    bits = np.where(low_p, LOW_P, 0) | np.where(inclined, INCLINED, 0) | np.where(leg, LOOPER_LEG, 0)
    with np.errstate(invalid="ignore"):
        margin = {"p": np.abs(mom - p["p_min"]) / p["p_min"], "tgl": np.abs(np.abs(t) - p["tgl_max"]),
                  "reach": np.abs(reach - X_OUT), "dz": np.abs(dz - p["dz_leg"])}
    return {"bits": bits.astype(np.int32), "p": mom, "reach": reach, "z_axis": z_axis, "dz": dz, "margin": margin}


def from_oracle_run(ref: dict, n_clusters: int, p: dict | None = None, vertices: dict | None = None) -> dict:
    """Classes of the oracle's own refitted tracks (oracle.run output) and
    the keep mask of the n_clusters input clusters (a cluster is dropped
    when its track is rejected; unassigned clusters are kept)."""
    rs = ref["rs_of"][ref["tl_start"][ref["t_tracklet"]]] if len(ref["t_tracklet"]) else np.zeros(0, np.int64)
    request = rs // (vertex.NROW * vertex.NSEC)
    out = classify(vertex.row_x(ref["t_row_in"]), ref["t_par"], p, vertices, request)
    ct = np.asarray(ref["cluster_track"]).astype(np.int64)
    keep = np.ones(n_clusters, np.uint8)
    sel = ct >= 0
    keep[sel] = (out["bits"][ct[sel]] == 0).astype(np.uint8)
    out["keep"] = keep
    return out
