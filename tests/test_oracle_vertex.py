"""Pins of the vertex-finding oracle (drift-time coordinate, Sec. 5): the
closed-form point of closest approach against a brute-force minimisation
along the helix, its straight-line limit, and the recovery of the true
collision times and spatial z on a generated timeframe."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import vertex

K = 0.299792458e-3 * 5.0


def _helix_xy(x, y, s, q, sigma):
    kappa = -K * q
    phi = math.atan2(s, math.sqrt(1 - s * s))
    if kappa == 0.0:
        return x + sigma * math.cos(phi), y + sigma * math.sin(phi)
    return (x + (math.sin(phi + kappa * sigma) - math.sin(phi)) / kappa,
            y - (math.cos(phi + kappa * sigma) - math.cos(phi)) / kappa)


def _brute(x, y, s, q):
    """Closest approach to the beam axis by dense sampling of the path
    length over one full turn (or +-600 cm for a straight track) and golden
    section refinement."""
    kappa = -K * q
    span = math.pi / abs(kappa) if kappa != 0 else 600.0
    grid = np.linspace(-span, span, 20001)
    r2 = [sum(v * v for v in _helix_xy(x, y, s, q, g)) for g in grid]
    i = int(np.argmin(r2))
    a, b = grid[max(i - 1, 0)], grid[min(i + 1, len(grid) - 1)]
    g = (math.sqrt(5) - 1) / 2
    for _ in range(200):
        c, d = b - g * (b - a), a + g * (b - a)
        fc = sum(v * v for v in _helix_xy(x, y, s, q, c))
        fd = sum(v * v for v in _helix_xy(x, y, s, q, d))
        if fc < fd:
            b = d
        else:
            a = c
    sig = 0.5 * (a + b)
    return sig, math.sqrt(sum(v * v for v in _helix_xy(x, y, s, q, sig)))


def test_closest_approach_matches_brute_force():
    rng = np.random.default_rng(5)
    n = 60
    x = rng.uniform(85, 246, n)
    y = rng.uniform(-0.17, 0.17, n) * x
    s = rng.uniform(-0.9, 0.9, n)
    q = rng.choice([-1, 1], n) / np.exp(rng.uniform(np.log(0.1), np.log(10), n))
    q[:3] = 0.0  # straight tracks
    path, dist = vertex.dca_path(x, y, s, q, K)
    for i in range(n):
        sig, d = _brute(x[i], y[i], s[i], q[i])
        assert path[i] == pytest.approx(sig, rel=1e-6, abs=1e-6), i
        assert dist[i] == pytest.approx(d, rel=1e-6, abs=1e-6), i


def test_straight_limit_is_continuous_and_is_the_projection():
    x, y, s = np.array([120.0, 200.0]), np.array([3.0, -10.0]), np.array([0.2, -0.4])
    p0, d0 = vertex.dca_path(x, y, s, np.zeros(2), K)
    c = np.sqrt(1 - s * s)
    assert np.allclose(p0, -(x * c + y * s), rtol=0, atol=1e-12)  # projection onto the direction
    p1, d1 = vertex.dca_path(x, y, s, np.full(2, 1e-7), K)
    assert np.allclose(p0, p1, rtol=1e-6) and np.allclose(d0, d1, atol=1e-6)


@pytest.fixture(scope="module")
def tf_case():
    ev = synth.timeframe(seed=7, length_ms=0.3, truth=True)
    ref = oracle.run(ev.clusters)
    return ev, ref


def _truth_of_tracks(ev, ref):
    """Per oracle track: the majority generator label of its clusters, its
    collision time and whether it is a primary."""
    ct = ref["cluster_track"].astype(np.int64)
    labels = ev.clusters["id"].astype(np.int64)
    m = ref["n_tracks"]
    lab = np.full(m, -1, np.int64)
    sel = (ct >= 0) & (labels != 0xFFFFFFFF)
    pairs, cnt = np.unique(np.stack([ct[sel], labels[sel]], 1), axis=0, return_counts=True)
    order = np.lexsort((-cnt, pairs[:, 0]))  # per track, the most frequent label first
    first = np.concatenate([[True], pairs[order][1:, 0] != pairs[order][:-1, 0]])
    lab[pairs[order][first, 0]] = pairs[order][first, 1]
    table = synth.track_table(ev.params)
    ok = lab >= 0
    tc = np.where(ok, table["tc"][np.maximum(lab, 0)], np.nan)
    prim = ok & (table["xv"][np.maximum(lab, 0)] == 0.0) & (table["yv"][np.maximum(lab, 0)] == 0.0)
    return lab, tc, prim


def test_vertices_recover_collision_times_and_z(tf_case):
    ev, ref = tf_case
    v = vertex.from_oracle_run(ref)
    lab, tc, prim = _truth_of_tracks(ev, ref)
    use = v["use"]
    assert v["v_time"].size >= 5
    # every collision with at least 10 usable primary tracks and no other
    # collision within 1 us (closer ones cannot be told apart in time) is a
    # vertex within 0.25 us that holds at least 80% of those tracks
    true_t = np.unique(tc[np.isfinite(tc)])
    colls, counts = np.unique(tc[use & prim], return_counts=True)
    alone = np.array([np.sort(np.abs(true_t - t))[1] > 1.0 if len(true_t) > 1 else True for t in colls])
    big = colls[(counts >= 10) & alone]
    assert big.size >= 5
    for t in big:
        k = int(np.argmin(np.abs(v["v_time"] - t)))
        assert abs(v["v_time"][k] - t) < 0.25, t
        mine = use & prim & (tc == t)
        assert np.mean(v["vertex"][mine] == k) >= 0.8, t
    # 99% of the tracks given to vertices are in vertices on a true collision
    # (the rest: secondaries that pass the distance cut form small vertices
    # offset in time from their collision)
    on = np.array([np.min(np.abs(true_t - t)) < 0.25 for t in v["v_time"]])
    assert v["v_n"][on].sum() >= 0.99 * v["v_n"].sum()
    # spatial z at the innermost row, for tracks whose vertex is their collision
    ok = (v["vertex"] >= 0) & prim
    ok &= np.abs(v["v_time"][np.maximum(v["vertex"], 0)] - tc) < 0.1
    side = np.where(np.asarray(ref["rs_of"][ref["tl_start"][ref["t_tracklet"]]] // 159 % 36) < 18, 1.0, -1.0)
    # truth of the innermost cluster: drift z converted with the true time
    ct = ref["cluster_track"].astype(np.int64)
    cl = np.nonzero(ct >= 0)[0]
    cl = cl[np.lexsort((ev.clusters["row"][cl], ct[cl]))]
    first = np.concatenate([[True], ct[cl][1:] != ct[cl][:-1]])
    inner = np.full(ref["n_tracks"], -1, np.int64)
    inner[ct[cl][first]] = cl[first]
    t_ok = np.nonzero(ok & (inner >= 0))[0]
    z_true = side[t_ok] * (250.0 - (ev.truth["z"][inner[t_ok]] - 2.5 * tc[t_ok]))
    dz = np.abs(v["z"][t_ok] - z_true)
    assert len(dz) > 100
    assert np.median(dz) < 0.2 and np.percentile(dz, 95) < 1.0
    # dz/ds_T flips sign on the A side only
    assert np.allclose(v["tgl"][ok], -side[ok] * ref["t_par"][ok, 3])


def test_a_planted_sign_error_is_caught(tf_case, monkeypatch):
    """The pins see a wrong direction of the extrapolation to the beam."""
    ev, ref = tf_case
    orig = vertex.dca_path
    monkeypatch.setattr(vertex, "dca_path", lambda *a: (lambda p, d: (-p, d))(*orig(*a)))
    v = vertex.from_oracle_run(ref)
    lab, tc, prim = _truth_of_tracks(ev, ref)
    colls, counts = np.unique(tc[v["use"] & prim], return_counts=True)
    big = colls[counts >= 10]
    found = [v["v_time"].size and np.min(np.abs(v["v_time"] - t)) < 0.25 for t in big]
    assert np.mean(found) < 0.8
