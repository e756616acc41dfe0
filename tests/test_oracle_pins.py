"""Pins of the FP64 oracle against what the method and the mathematics fix.

None of these re-derives the oracle's own formula: each checks the oracle
against an independent fact -- an all-triplet brute force, the generator's
global-frame helix, a least-squares normal-equation solve, invariants of the
link/chain/ownership structures, or pull statistics.
"""
import math

import numpy as np
import pytest

import oracle
import synth

WY = np.float32(2.0 * ((245.8 - 85.2) / 158.0) + 0.5)
WZ = np.float32(2.5 * ((245.8 - 85.2) / 158.0) + 0.5)


# ------------------------------------------------------------------ grid (a2)
def _rs_of_input(cl, n_req=1, req_off=None):
    return (cl["sector"].astype(np.int64)) * 159 + cl["row"]


def test_grid_partition_and_order(small_event, small_oracle):
    cl, r = small_event.clusters, small_oracle
    n = len(cl)
    perm = r["perm"]
    assert np.array_equal(np.sort(perm), np.arange(n))
    rs_in = _rs_of_input(cl)
    counts = np.bincount(rs_in, minlength=r["n_rs"])
    assert np.array_equal(np.diff(r["row_start"]), counts)
    assert np.array_equal(r["rs_of"], rs_in[perm])
    assert np.array_equal(r["sy"], cl["y"][perm]) and np.array_equal(r["sz"], cl["z"][perm])
    # z range per row-sector is the exact min/max
    for rs in np.nonzero(counts)[0][:200]:
        zz = cl["z"][rs_in == rs]
        assert r["z_lo"][rs] == zz.min() and r["z_hi"][rs] == zz.max()
    # bins: bin_start is monotone, covers [0, n], and inside a bin input indices ascend
    bs = r["bin_start"]
    assert bs[0] == 0 and bs[-1] == n and np.all(np.diff(bs) >= 0)
    for rs in range(r["n_rs"]):
        a, b = r["row_start"][rs], r["row_start"][rs + 1]
        g0, g1 = r["bin_base"][rs], r["bin_base"][rs + 1]
        assert bs[g0] == a and bs[g1] == b
    pos_bin = np.searchsorted(bs, np.arange(n), side="right") - 1
    same = pos_bin[1:] == pos_bin[:-1]
    assert np.all(perm[1:][same] > perm[:-1][same])


def test_grid_cluster_inside_its_bin(small_event, small_oracle):
    r = small_oracle
    n = r["n"]
    x, yhi = oracle.tables()
    pos_bin = np.searchsorted(r["bin_start"], np.arange(n), side="right") - 1
    rs = r["rs_of"]
    local = pos_bin - r["bin_base"][rs]
    ny, nz = r["n_y"][rs], r["n_z"][rs]
    iy, iz = local % ny, local // ny
    assert np.all(local < ny * nz)
    ylo = -yhi[rs % 159].astype(np.float64)
    wy = 1.0 / r["inv_y"][rs].astype(np.float64)
    wz = 1.0 / r["inv_z"][rs].astype(np.float64)
    y, z = r["sy"].astype(np.float64), r["sz"].astype(np.float64)
    zlo = r["z_lo"][rs].astype(np.float64)
    tol = 1e-5
    assert np.all((iy == 0) | (y >= ylo + iy * wy - tol * (1 + np.abs(y))))
    assert np.all((iy == ny - 1) | (y <= ylo + (iy + 1) * wy + tol * (1 + np.abs(y))))
    assert np.all((iz == 0) | (z >= zlo + iz * wz - tol * (1 + np.abs(z))))
    assert np.all((iz == nz - 1) | (z <= zlo + (iz + 1) * wz + tol * (1 + np.abs(z))))


def test_grid_bin_count_scales_with_occupancy(small_oracle):
    """The bin edge sqrt(2 A / n) gives more than n/2 bins (mean occupancy
    below two) wherever no clamp binds."""
    r = small_oracle
    cnt = np.diff(r["row_start"])
    nb = r["n_y"].astype(np.int64) * r["n_z"]
    dz = r["z_hi"] - r["z_lo"]
    free = (cnt > 8) & (dz >= 1.0) & (r["n_y"] < 256) & (r["n_z"] < 4096)
    assert free.sum() > 50
    assert np.all(nb[free] > cnt[free] / 2)


# ---------------------------------------------------------- neighbours (a3)
def _brute_links(r, d_max=1.0):
    """All-triplet straight-line search in binary32, no grid."""
    x, _ = oracle.tables()
    n = r["n"]
    up = np.full(n, -1, np.int32)
    dn = np.full(n, -1, np.int32)
    tie = np.zeros(n, np.uint8)
    sy, sz, rs = r["sy"], r["sz"], r["rs_of"]
    for c in range(n):
        row = rs[c] % 159
        if row < 1 or row > 157:
            continue
        f = np.float32((x[row] - x[row - 1]) / (x[row + 1] - x[row - 1]))
        d = np.nonzero((rs == rs[c] - 1) & (np.abs(sy - sy[c]) <= WY) & (np.abs(sz - sz[c]) <= WZ))[0]
        u = np.nonzero((rs == rs[c] + 1) & (np.abs(sy - sy[c]) <= WY) & (np.abs(sz - sz[c]) <= WZ))[0]
        if len(d) == 0 or len(u) == 0:
            continue
        yd, zd, yu, zu = sy[d][:, None], sz[d][:, None], sy[u][None, :], sz[u][None, :]
        dy = (yd - sy[c]) + (yu - yd) * f
        dz = (zd - sz[c]) + (zu - zd) * f
        D = (dy * dy + dz * dz).astype(np.float32)
        dd, uu = np.meshgrid(d, u, indexing="ij")
        order = np.lexsort((uu.ravel(), dd.ravel(), D.ravel()))
        best = order[0]
        if D.ravel()[best] <= np.float32(d_max):
            up[c], dn[c] = uu.ravel()[best], dd.ravel()[best]
            if len(order) > 1:
                d1, d2 = D.ravel()[best], D.ravel()[order[1]]
                tie[c] = np.abs(d2 - d1) <= np.float32(1e-6) * max(d1, np.float32(1e-12))
    return up, dn, tie


def test_neighbours_equal_all_triplet_brute_force():
    for seed in (21, 22, 23):
        ev = synth.generate(synth.GenParams(seed=seed, n_primaries=12, n_secondaries=0, sectors=(5,),
                                            phi_min=math.radians(100), phi_max=math.radians(120),
                                            phi_radius=85.2, noise_frac=0.1))
        assert 30 < len(ev.clusters) <= 400
        # duplicate every fifth cluster: exact distance ties must go to the
        # lower sorted index of d, then of u
        cl = np.concatenate([ev.clusters, ev.clusters[::5]])
        r = oracle.run(cl, stop_after="neighbours")
        up, dn, tie = _brute_links(r)
        assert np.array_equal(r["up"], up) and np.array_equal(r["dn"], dn) and np.array_equal(r["tie"], tie)
        assert (up >= 0).sum() > 10 and tie.sum() > 0


def test_neighbours_grid_equals_oracle_brute_mode(sector_event, small_event):
    for ev in (sector_event, small_event):
        a = oracle.run(ev.clusters, stop_after="neighbours")
        b = oracle.run(ev.clusters, stop_after="neighbours", brute=True)
        for k in ("up", "dn", "tie"):
            assert np.array_equal(a[k], b[k])


def test_straight_lines_link_along_the_line():
    ev = synth.straight_lines(seed=3, n_lines=6, spacing=4.0, max_slope=0.05)
    assert len(ev.clusters) == 6 * 159
    r = oracle.run(ev.clusters, stop_after="tracklets")
    lab = ev.clusters["id"][r["perm"]]
    has = r["up_m"] >= 0
    assert has.sum() > 0
    assert np.array_equal(lab[has], lab[r["up_m"][has]])
    # one chain per line over rows 1..157
    assert r["n_tracklets"] == 6 and np.all(r["tl_len"] == 157)


# ------------------------------------------------------- link cleaning (a4)
def test_link_symmetry(small_oracle):
    r = small_oracle
    up_m, dn_m, up, dn = r["up_m"], r["dn_m"], r["up"], r["dn"]
    c = np.nonzero(up_m >= 0)[0]
    assert len(c) > 1000
    assert np.array_equal(dn_m[up_m[c]], c)
    c = np.nonzero(dn_m >= 0)[0]
    assert np.array_equal(up_m[dn_m[c]], c)
    m = up_m >= 0
    assert np.array_equal(up_m[m], up[m]) and np.array_equal(dn[up_m[m]], np.nonzero(m)[0])


# ----------------------------------------------------------- tracklets (a5)
def test_chains_disjoint_consecutive_and_complete(small_oracle):
    r = small_oracle
    seen = np.zeros(r["n"], np.int32)
    for s, L in zip(r["tl_start"], r["tl_len"]):
        assert r["dn_m"][s] < 0 and L >= 3
        k = s
        for i in range(L):
            seen[k] += 1
            nxt = r["up_m"][k]
            if i < L - 1:
                assert r["rs_of"][nxt] == r["rs_of"][k] + 1
            k = nxt
        assert k == -1
    assert seen.max() <= 1
    # every chain of three or more appears, in start order
    starts = np.nonzero((r["up_m"] >= 0) & (r["dn_m"] < 0))[0]
    lens = []
    for s in starts:
        L, k = 0, s
        while k >= 0:
            L, k = L + 1, r["up_m"][k]
        lens.append(L)
    assert np.array_equal(starts[np.array(lens) >= 3], r["tl_start"])


# -------------------------------------------------------- Kalman (a6, a8)
def _segments(ev, min_len=12):
    t, c = ev.truth, ev.clusters
    for lab in np.unique(t["track"][t["track"] >= 0]):
        m = np.nonzero(t["track"] == lab)[0]
        for sec in np.unique(c["sector"][m]):
            mm = m[c["sector"][m] == sec]
            mm = mm[np.argsort(c["row"][mm])]
            rows = c["row"][mm].astype(np.int32)
            if len(mm) < min_len or (t["flags"][mm] != 0).any() or (np.diff(rows) <= 0).any():
                continue
            yield rows, t[mm]


@pytest.fixture(scope="module")
def noiseless():
    p = synth.GenParams(seed=5, n_primaries=200, n_secondaries=40, sectors=tuple(range(36)), sigma_y=0.0,
                        sigma_z=0.0, row_eff=1.0, noise_frac=0.0, pt_min=0.3)
    return synth.generate(p, truth=True)


def _truth_state(tr):
    return np.stack([tr["y"], tr["z"], tr["sphi"], tr["tgl"], tr["qpt"]], axis=-1)


def test_helix_propagation_reproduces_global_frame_crossings(noiseless):
    """State-only propagation from the true state at the first crossing lands
    on the generator's independent circle/plane intersections."""
    n = 0
    for rows, tr in _segments(noiseless):
        truth = _truth_state(tr)
        try:
            out = oracle.propagate_rows(rows, truth[0])
        except ValueError:
            continue
        err = np.abs(out - truth) / np.maximum(np.abs(truth), 1.0)
        assert err.max() < 1e-11, err.max()
        n += 1
    assert n >= 30


def test_exact_helix_fit_has_zero_chi2(noiseless):
    """Fitting exact helix points from the true seed leaves the state on the
    helix: chi2 ~ 0 and the innermost state equals the truth."""
    n = 0
    for rows, tr in _segments(noiseless):
        truth = _truth_state(tr)
        try:
            p, cov, chi2 = oracle.kalman_fit(rows[::-1], tr["y"][::-1], tr["z"][::-1], truth[-1])
        except ValueError:
            continue
        assert chi2 < 1e-18
        assert np.all(np.abs(p - truth[0]) <= 1e-9 * np.maximum(np.abs(truth[0]), 1.0))
        C = oracle.unpack_cov(cov)
        assert np.all(np.linalg.eigvalsh(C) > 0)
        n += 1
    assert n >= 30


def test_noiseless_event_is_tracked_exactly(noiseless):
    """Without noise, smearing or inefficiency every found track is one true
    segment with all of its clusters, chi2/ndf ~ 0, and its parameters are
    far inside their own error."""
    ev, r = noiseless, oracle.run(noiseless.clusters)
    c, t = ev.clusters, ev.truth
    ct = r["cluster_track"]
    assert r["n_tracks"] > 100
    for k in range(r["n_tracks"]):
        idx = np.nonzero(ct == k)[0]
        labs = np.unique(t["track"][idx])
        assert len(labs) == 1
        seg = np.nonzero((t["track"] == labs[0]) & (c["sector"] == c["sector"][idx[0]]))[0]
        assert len(seg) == len(idx)
        assert r["t_chi2"][k] / r["t_ndf"][k] < 1e-4
        j = idx[c["row"][idx] == r["t_row_in"][k]]
        truth = _truth_state(t[j[0]])
        sig = np.sqrt(np.diag(oracle.unpack_cov(r["t_cov"][k])))
        assert np.all(np.abs(r["t_par"][k] - truth) <= 0.05 * sig)


def test_kalman_equals_least_squares_when_bz_is_zero():
    """Bz = 0 and a flat prior: the filter reproduces the weighted straight-
    line least-squares covariance (normal equations) exactly on noiseless
    lines, where every linearisation point is the true line, and the
    least-squares solution, chi2 and covariance on smeared lines up to the
    filter's linearisation at its running estimate."""
    x, _ = oracle.tables()
    x = x.astype(np.float64)
    rng = np.random.default_rng(1)
    cfg = oracle.default_config(bz_kg=0.0, c0=(1e6, 1e6, 1e2, 1e2, 1.0))
    for noise, tol, ctol in ((0.0, 1e-9, 1e-7), (0.1, 0.25, 0.01)):
        for _ in range(20):
            rows = np.arange(20, 140)
            b, a = rng.uniform(-0.5, 0.5), rng.uniform(-5, 5)
            e, z0 = rng.uniform(-1, 1), rng.uniform(-50, 50)
            xi = x[rows]
            y = a + b * (xi - xi[0]) + noise * rng.normal(0, 1, len(rows))
            z = z0 + e * (xi - xi[0]) + noise * rng.normal(0, 1, len(rows))
            L = math.hypot(xi[-1] - xi[0], y[-1] - y[0])
            p0 = [y[-1], z[-1], (y[-1] - y[0]) / L, (z[-1] - z[0]) / L, 0.0]
            p, _, _ = oracle.kalman_fit(rows[::-1], y[::-1], z[::-1], p0, cfg)
            pout = oracle.propagate_rows(np.array([rows[0], rows[-1]]), p, cfg)[1]
            p, cov, chi2 = oracle.kalman_fit(rows[::-1], y[::-1], z[::-1], pout, cfg)
            X = np.stack([np.ones_like(xi), xi - xi[0]], 1)
            N = X.T @ X
            Ay, Az = np.linalg.solve(N, X.T @ y), np.linalg.solve(N, X.T @ z)
            cphi = 1.0 / math.sqrt(1.0 + Ay[1] ** 2)
            ref = np.array([Ay[0], Az[0], Ay[1] * cphi, Az[1] * cphi])
            V = np.linalg.inv(N) * 0.01
            C = oracle.unpack_cov(cov)
            sig = np.sqrt([V[0, 0], V[0, 0], cphi ** 6 * V[1, 1], cphi ** 2 * V[1, 1]])
            if noise == 0.0:
                assert np.all(np.abs(p[:4] - ref) <= tol * np.maximum(np.abs(ref), 1.0))
                assert chi2 < 1e-12
            else:
                assert np.all(np.abs(p[:4] - ref) <= tol * sig)
                chi_ref = (np.sum((y - X @ Ay) ** 2) + np.sum((z - X @ Az) ** 2)) / 0.01
                assert abs(chi2 / chi_ref - 1) < 0.01
            assert abs(C[0, 0] / V[0, 0] - 1) < ctol and abs(C[1, 1] / V[0, 0] - 1) < ctol
            assert abs(C[2, 2] / (cphi ** 6 * V[1, 1]) - 1) < ctol
            assert abs(C[0, 2] / (cphi ** 3 * V[0, 1]) - 1) < ctol


def test_pulls_and_chi2_are_standard():
    """With Gaussian smearing the pulls of the refit parameters at the
    innermost row are centred and of unit width (robust estimates), and
    chi2/ndf ~ 1: this pins the covariance propagation."""
    p = synth.GenParams(seed=11, n_primaries=4000, n_secondaries=0, sectors=(0, 1, 2, 18, 19, 20))
    ev = synth.generate(p, truth=True)
    r = oracle.run(ev.clusters)
    c, t = ev.clusters, ev.truth
    pulls, chi = [], []
    for k in range(r["n_tracks"]):
        idx = np.nonzero(r["cluster_track"] == k)[0]
        labs = np.unique(t["track"][idx])
        if len(labs) != 1 or labs[0] < 0 or len(idx) < 40 or r["t_flags"][k] & oracle.F_REFIT_FAIL:
            continue
        j = idx[c["row"][idx] == r["t_row_in"][k]]
        truth = _truth_state(t[j[0]])
        pulls.append((r["t_par"][k] - truth) / np.sqrt(np.diag(oracle.unpack_cov(r["t_cov"][k]))))
        chi.append(r["t_chi2"][k] / r["t_ndf"][k])
    pulls = np.array(pulls)
    assert len(pulls) > 300
    med = np.median(pulls, 0)
    mad = 1.4826 * np.median(np.abs(pulls - med), 0)
    assert np.all(np.abs(med) < 0.12), med
    assert np.all((mad > 0.85) & (mad < 1.25)), mad
    assert 0.9 < np.median(chi) < 1.1


# ----------------------------------------------------------- selection (a7)
def test_selection_matches_cluster_centric_brute_force(small_oracle):
    """Each cluster goes to the highest (cluster count, lower id) candidate
    among all tracklets with >= 10 clusters; a tracklet survives if it owns
    >= 10.  Computed here per cluster, not per tracklet."""
    r = small_oracle
    nt, n = r["n_tracklets"], r["n"]
    cands = [[] for _ in range(n)]
    for t in range(nt):
        if r["f_n"][t] >= 10:
            for h in r["f_hits"][t, :r["f_n"][t]]:
                cands[h].append((int(r["f_n"][t]), -t))
    owner_t = np.full(n, -1)
    for h in range(n):
        if cands[h]:
            owner_t[h] = -max(cands[h])[1]
    kept = [t for t in range(nt) if r["f_n"][t] >= 10 and (owner_t[r["f_hits"][t, :r["f_n"][t]]] == t).sum() >= 10]
    assert np.array_equal(np.nonzero(r["tl_track"] >= 0)[0], np.array(kept, dtype=np.int64))
    assert np.array_equal(r["tl_track"][kept], np.arange(len(kept)))
    expect = np.full(n, -1, np.int32)
    for k, t in enumerate(kept):
        hh = r["f_hits"][t, :r["f_n"][t]]
        expect[r["perm"][hh[owner_t[hh] == t]]] = k
    assert np.array_equal(r["cluster_track"], expect)


def test_each_cluster_at_most_one_track(small_oracle):
    r = small_oracle
    ct = r["cluster_track"]
    counts = np.bincount(ct[ct >= 0], minlength=r["n_tracks"])
    assert np.all(counts >= 10)
    assert np.array_equal(counts, r["t_n"])
    assert np.all(r["t_ndf"] == 2 * r["t_n"] - 5)


def test_findable_efficiency_reported(small_event, small_oracle):
    """Findable (Sec. 2, Fig. 3 caption): >= 70 cm through the TPC, pT >=
    200 MeV/c, |eta| <= 0.9; here per sector segment.  The paper's level is
    in a missing figure, so this is a regression guard only."""
    ev, r = small_event, small_oracle
    c, t = ev.clusters, ev.truth
    x, _ = oracle.tables()
    found = 0
    findable = 0
    ct = r["cluster_track"]
    for lab in np.unique(t["track"][t["track"] >= 0]):
        m = np.nonzero(t["track"] == lab)[0]
        if abs(1.0 / t["qpt"][m[0]]) < 0.2:
            continue
        for sec in np.unique(c["sector"][m]):
            mm = m[c["sector"][m] == sec]
            if x[c["row"][mm].max()] - x[c["row"][mm].min()] < 70.0:
                continue
            findable += 1
            tr = ct[mm]
            if (tr >= 0).any():
                k = np.bincount(tr[tr >= 0]).argmax()
                if (tr == k).sum() >= 0.5 * len(mm):
                    found += 1
    eff = found / findable
    print(f"findable segments {findable}, efficiency {eff:.3f}")
    assert findable > 30 and eff > 0.8


# ------------------------------------- stopping rules of the extension (a6)
def _row_x():
    return np.array([float(np.float32(85.2 + r * ((245.8 - 85.2) / 158.0))) for r in range(159)])


def _line_clusters(rows, y_of_x, z_of_x, sector=0, ident=0):
    x = _row_x()
    rows = np.asarray(sorted(rows), dtype=np.int64)
    c = np.zeros(len(rows), synth.CLUSTER_DTYPE)
    c["y"], c["z"] = y_of_x(x[rows]), z_of_x(x[rows])
    c["row"], c["sector"], c["id"] = rows, sector, ident
    return c


def _tracks_of(r, cl):
    """Sets of rows of every found track (input order of the clusters)."""
    out = []
    for k in range(r["n_tracks"]):
        out.append(sorted(cl["row"][r["cluster_track"] == k].tolist()))
    return sorted(out)


@pytest.mark.parametrize("max_miss,gap", [(5, 4), (5, 5), (3, 2), (3, 3), (5, 1)])
def test_extension_bridges_fewer_than_max_miss_empty_rows(max_miss, gap):
    """A track with `gap` consecutive empty rows: the extension ends after
    max_miss consecutive rows without a cluster (Sec. 2 track following;
    MAX_MISS is the reading's constant), so a gap shorter than max_miss is
    bridged -- one track holds every cluster -- and a gap of max_miss rows
    splits the track in two at the gap.  Noiseless straight tracks in the
    default field; the inner piece's outward extension and the outer
    piece's inward extension both meet the gap, and each tracklet's own
    cluster list is checked as well as the selected tracks."""
    cfg = oracle.default_config(max_miss=max_miss)
    g0 = 60
    rows = [r for r in range(159) if not g0 < r <= g0 + gap]
    lines = [(-6.0, 0.02, 10.0, 0.3), (5.0, -0.03, 30.0, 0.5)]
    for sec, (y0, b, z0, e) in enumerate(lines):
        cl = _line_clusters(rows, lambda x: y0 + b * (x - 85.2), lambda x: z0 + e * (x - 85.2), sector=sec)
        r = oracle.run(cl, cfg=cfg)
        tracks = _tracks_of(r, cl)
        inner = [q for q in rows if q <= g0]
        outer = [q for q in rows if q > g0]
        # two tracklets (the chains on either side of the gap), inner first;
        # each one's own extension must bridge the gap, or stop at it
        assert r["n_tracklets"] == 2
        rows_sorted = cl["row"][r["perm"]]
        held = [sorted(rows_sorted[r["f_hits"][t, :r["f_n"][t]]].tolist()) for t in range(2)]
        if gap < max_miss:
            assert held == [sorted(rows), sorted(rows)], (max_miss, gap, [len(h) for h in held])
            assert tracks == [sorted(rows)], (max_miss, gap, [len(t) for t in tracks])
        else:
            assert held == [inner, outer], (max_miss, gap, [(h[0], h[-1]) for h in held])
            assert tracks == sorted([inner, outer]), (max_miss, gap, [(t[0], t[-1]) for t in tracks])


def _edge_lim(x):
    return x * 0.17632698070846498 + 2.0


def test_extension_stops_beyond_the_sector_edge_outward():
    """A straight track leaving the wedge: full rows up to row 40 (the
    chain), then a cluster on every other row (no chain there: links need
    rows r-1 and r+1), past the edge and on to row 158.  The outward
    extension takes every cluster while the predicted |y| is within x tan 10
    + 2 cm and stops at the first row beyond it; no cluster there lies
    within 0.05 cm of that limit."""
    x = _row_x()
    b, ra = 0.35, 40
    ya = _edge_lim(x[ra]) - 3.0
    rows = list(range(10, ra + 1)) + list(range(ra + 2, 159, 2))

    def y_of(xx):
        return ya + b * (xx - x[ra])
    over = y_of(x) - _edge_lim(x)
    assert np.all(np.abs(over[rows]) > 0.05) and over[158] > 5.0
    cl = _line_clusters(rows, y_of, lambda xx: 20.0 + 0.4 * (xx - 85.2))
    r = oracle.run(cl)
    first_out = int(np.nonzero(over > 0)[0][0])
    expect = [q for q in rows if q < first_out]
    assert first_out > ra + 8 and len(expect) < len(rows) - 20
    assert _tracks_of(r, cl) == [expect]


def test_extension_stops_beyond_the_sector_edge_inward():
    """The same for the inward extension of the backward pass: a track at
    constant y = 20 cm is inside the wedge from row ~28 outward (the chain:
    full rows 40..158) and beyond x tan 10 + 2 cm below row ~17; on every
    other row below the chain it is picked up down to the last row within
    the limit."""
    x = _row_x()
    y = 20.0
    rows = list(range(0, 40, 2)) + list(range(40, 159))
    over = y - _edge_lim(x)
    assert np.all(np.abs(over[rows]) > 0.05)
    cl = _line_clusters(rows, lambda xx: np.full_like(xx, y), lambda xx: 15.0 + 0.6 * (xx - 85.2))
    r = oracle.run(cl)
    last_out = int(np.nonzero(over > 0)[0][-1])
    expect = [q for q in rows if q > last_out]
    assert 10 < last_out < 30 and len(expect) < len(rows) - 5
    assert _tracks_of(r, cl) == [expect]


# ------------------------------------------------ chi2 increment r^T S^-1 r
@pytest.mark.parametrize("sphi,tgl,res", [(0.8, 2.0, (0.7, -0.9)), (-0.6, -1.5, (0.3, 0.4)),
                                          (0.2, 0.1, (-1.0, 0.5))])
def test_chi2_equals_least_squares_minimum_of_the_linear_model(sphi, tgl, res):
    """Bz = 0 makes the transport linear in the state deviations, so the
    filter is exact for the linear Gaussian model: the accumulated chi2 (sum
    of r^T S^-1 r over the updates) equals the minimum of the batch
    least-squares objective (prior term plus measurement terms), and the
    filtered state and covariance at the last row equal the least-squares
    solution carried there.  A first measurement on the seed (zero residual)
    and a second one offset by `res` ten rows further; with large |sin phi|
    and dz/ds_T the predicted y and z errors are strongly correlated, so the
    y-z term of S^-1 carries most of the chi2.  The least-squares side uses
    the straight-line geometry y' = y + dx tan(phi), z' = z + dz/ds_T dx/cos(phi)
    and its derivative, and numpy's solver."""
    cfg = oracle.default_config(bz_kg=0.0)
    x = _row_x()
    r0, r1 = 30, 40
    dx = x[r1] - x[r0]
    p0 = np.array([3.0, 40.0, sphi, tgl, 0.0])
    c = math.sqrt(1 - sphi ** 2)
    f = p0 + np.array([dx * sphi / c, tgl * dx / c, 0, 0, 0])
    m0 = p0[:2]
    m1 = f[:2] + np.array(res)
    p, cov, chi2 = oracle.kalman_fit([r0, r1], [m0[0], m1[0]], [m0[1], m1[1]], p0, cfg)
    # linear model around p0: state deviation d at row r0, carried by J
    J = np.eye(5)
    J[0, 2] = dx / c ** 3
    J[1, 2] = tgl * dx * sphi / c ** 3
    J[1, 3] = dx / c
    H = np.zeros((2, 5))
    H[0, 0] = H[1, 1] = 1.0
    V = cfg.sigma ** 2
    C0inv = np.diag(1.0 / np.array(cfg.c0[:]))
    N = C0inv + H.T @ H / V + (H @ J).T @ (H @ J) / V
    rhs = (H @ J).T @ (m1 - f[:2]) / V
    d = np.linalg.solve(N, rhs)
    obj = d @ C0inv @ d + np.sum((H @ d) ** 2) / V + np.sum((m1 - f[:2] - H @ J @ d) ** 2) / V
    assert abs(chi2 - obj) <= 1e-9 * obj, (chi2, obj)
    assert np.allclose(p, f + J @ d, rtol=1e-9, atol=1e-9)
    C = J @ np.linalg.inv(N) @ J.T
    assert np.allclose(oracle.unpack_cov(cov), C, rtol=1e-8, atol=1e-12 * np.abs(C).max())
    # the y-z correlation of the prediction matters: without its S^-1 term
    # the chi2 would be far off (guards the test's own sensitivity)
    Sp = H @ J @ np.linalg.inv(C0inv + H.T @ H / V) @ J.T @ H.T + V * np.eye(2)
    r = m1 - f[:2]
    diag_only = r[0] ** 2 / Sp[0, 0] + r[1] ** 2 / Sp[1, 1]
    if abs(sphi * tgl) > 0.5:
        assert abs(diag_only - obj) > 0.1 * obj


# ------------------------------------- next-row variant of the links (a3)
WY2 = np.float32(2 * 2.0 * ((245.8 - 85.2) / 158.0) + 0.5)
WZ2 = np.float32(2 * 2.5 * ((245.8 - 85.2) / 158.0) + 0.5)


def _brute_links_skip(r, d_max=1.0):
    """All-triplet search with the next-row variant, in binary32, no grid:
    the r-1/r+1 pairs first; a cluster on rows 2..156 without an accepted
    one takes the lexicographic minimum of (D, d, u) over the one-sided
    skips (r-2, r+1), (r-1, r+2), and without an accepted one of those over
    (r-2, r+2); windows scaled by the row distance."""
    x, _ = oracle.tables()
    up, dn, tie = _brute_links(r, d_max)
    sy, sz, rs = r["sy"], r["sz"], r["rs_of"]
    win = {1: (WY, WZ), 2: (WY2, WZ2)}
    for c in range(r["n"]):
        row = rs[c] % 159
        if up[c] >= 0 or row < 2 or row > 156:
            continue
        best = None
        Ds = []
        for dr, ur in ((-2, 1), (-1, 2), (-2, 2)):
            if ur - dr == 4:  # both sides skipped
                if best is not None and best[0] <= np.float32(d_max):
                    break
                best, Ds = None, []
            wd, wu = win[-dr], win[ur]
            d = np.nonzero((rs == rs[c] + dr) & (np.abs(sy - sy[c]) <= wd[0]) & (np.abs(sz - sz[c]) <= wd[1]))[0]
            u = np.nonzero((rs == rs[c] + ur) & (np.abs(sy - sy[c]) <= wu[0]) & (np.abs(sz - sz[c]) <= wu[1]))[0]
            if len(d) == 0 or len(u) == 0:
                continue
            f = np.float32((x[row] - x[row + dr]) / (x[row + ur] - x[row + dr]))
            for dd in d:
                for uu in u:
                    ey = (sy[dd] - sy[c]) + (sy[uu] - sy[dd]) * f
                    ez = (sz[dd] - sz[c]) + (sz[uu] - sz[dd]) * f
                    D = np.float32(ey * ey + ez * ez)
                    Ds.append(D)
                    if best is None or (D, dd, uu) < best:
                        best = (D, dd, uu)
        if best is not None and best[0] <= np.float32(d_max):
            dn[c], up[c] = best[1], best[2]
            Ds.sort()
            second = Ds[1] if len(Ds) > 1 else None
            tie[c] = second is not None and abs(second - best[0]) <= np.float32(1e-6) * max(best[0], np.float32(1e-12))
    return up, dn, tie


def test_link_skip_equals_all_triplet_brute_force():
    cfg = oracle.default_config(link_skip=1)
    for seed in (31, 32, 33):
        ev = synth.generate(synth.GenParams(seed=seed, n_primaries=14, n_secondaries=0, sectors=(5,),
                                            phi_min=math.radians(100), phi_max=math.radians(120),
                                            phi_radius=85.2, noise_frac=0.1, row_eff=0.8))
        cl = np.concatenate([ev.clusters, ev.clusters[::7]])  # exact ties
        r = oracle.run(cl, stop_after="neighbours", cfg=cfg)
        up, dn, tie = _brute_links_skip(r)
        assert np.array_equal(r["up"], up) and np.array_equal(r["dn"], dn) and np.array_equal(r["tie"], tie)
        rows = r["rs_of"] % 159
        skipped = (up >= 0) & (rows[np.maximum(up, 0)] - rows == 2) | (dn >= 0) & (rows - rows[np.maximum(dn, 0)] == 2)
        assert skipped.sum() > 5  # the variant is exercised
        base = oracle.run(cl, stop_after="neighbours")
        # clusters with an accepted adjacent pair keep it
        keep = base["up"] >= 0
        assert np.array_equal(r["up"][keep], base["up"][keep]) and np.array_equal(r["dn"][keep], base["dn"][keep])


def test_link_skip_chains_bridge_single_missing_rows():
    """Straight tracks with every seventh row missing: with the variant each
    track is one chain over all its clusters on rows 1..157; without it the
    chains break at every gap (runs of six rows: chains of four)."""
    rows = [q for q in range(159) if q % 7 != 3]
    ev = synth.straight_lines(seed=4, n_lines=5, spacing=5.0, max_slope=0.05, rows=rows)
    lab = ev.clusters["id"]
    for skip in (0, 1):
        r = oracle.run(ev.clusters, stop_after="tracklets", cfg=oracle.default_config(link_skip=skip))
        lab_sorted = lab[r["perm"]]
        if skip:
            assert r["n_tracklets"] == 5
            for s0, L in zip(r["tl_start"], r["tl_len"]):
                inside = [q for q in rows if 1 <= q <= 157]
                assert L == len(inside) and (lab_sorted == lab_sorted[s0]).sum() >= L
        else:
            assert r["n_tracklets"] >= 5 * 20 and np.all(r["tl_len"] <= 4)


def test_link_skip_cuts_duplicate_tracklets_on_noiseless_tracks():
    """Noiseless tracks at 90% row efficiency, where every missing row
    breaks an r-1/r+1 chain: with the variant the follow stage starts from
    less than half as many tracklets per track, and still at least 98% of
    the found tracks are exactly one true segment with all its clusters
    (without it: all of them; a wider two-row window occasionally carries a
    chain across a neighbouring track at a gap)."""
    p = synth.GenParams(seed=6, n_primaries=200, n_secondaries=0, sectors=tuple(range(36)), sigma_y=0.0,
                        sigma_z=0.0, row_eff=0.9, noise_frac=0.0, pt_min=0.3)
    ev = synth.generate(p, truth=True)
    c, t = ev.clusters, ev.truth
    res, whole = {}, {}
    for skip in (0, 1):
        r = oracle.run(c, cfg=oracle.default_config(link_skip=skip))
        ct = r["cluster_track"]
        assert r["n_tracks"] > 100
        good = 0
        for k in range(r["n_tracks"]):
            idx = np.nonzero(ct == k)[0]
            labs = np.unique(t["track"][idx])
            seg = np.nonzero((t["track"] == labs[0]) & (c["sector"] == c["sector"][idx[0]]))[0]
            good += len(labs) == 1 and len(seg) == len(idx)
        whole[skip] = good / r["n_tracks"]
        res[skip] = r["n_tracklets"] / r["n_tracks"]
    assert whole[0] == 1.0 and whole[1] >= 0.98, whole
    assert res[1] < 0.5 * res[0], res
