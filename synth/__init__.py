"""Seeded synthetic TPC input (test and benchmark infrastructure).

Builds the five workloads the tracker is measured on: one sector of 400
tracks, one central Pb-Pb-like event over 36 sectors, a 10 ms continuous
read-out timeframe at 50 kHz (z from drift time, Sec. 5), batches of
independent requests of uneven size, and a stream of timeframes for the
serving loop.  The helix simulation is the C file beside this module; no
tracking arithmetic lives here.  Both the oracle tests and the CUDA tests
draw their inputs from this module only.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpcgen.c")
_LIB = os.path.join(_HERE, "libtpcgen.so")

CLUSTER_DTYPE = np.dtype([("y", "<f4"), ("z", "<f4"), ("row", "<u2"), ("sector", "<u2"), ("id", "<u4")])
TRUTH_DTYPE = np.dtype([("track", "<i4"), ("flags", "<i4"), ("y", "<f8"), ("z", "<f8"),
                        ("sphi", "<f8"), ("tgl", "<f8"), ("qpt", "<f8")])
assert CLUSTER_DTYPE.itemsize == 16 and TRUTH_DTYPE.itemsize == 48


class _Params(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("n_primaries", ctypes.c_int32), ("n_secondaries", ctypes.c_int32),
                ("pt_min", ctypes.c_double), ("pt_max", ctypes.c_double), ("eta_max", ctypes.c_double),
                ("phi_min", ctypes.c_double), ("phi_max", ctypes.c_double), ("phi_radius", ctypes.c_double),
                ("sec_r_max", ctypes.c_double),
                ("sector_mask", ctypes.c_uint64), ("sigma_y", ctypes.c_double), ("sigma_z", ctypes.c_double),
                ("row_eff", ctypes.c_double), ("noise_frac", ctypes.c_double), ("bz_kg", ctypes.c_double),
                ("timeframe", ctypes.c_int32), ("tf_length_us", ctypes.c_double), ("rate_khz", ctypes.c_double),
                ("vdrift", ctypes.c_double), ("mb_offset", ctypes.c_double), ("mb_max", ctypes.c_double),
                ("n_threads", ctypes.c_int32), ("legs", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile the generator into a shared library beside this file."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.gen_run.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(ctypes.c_void_p),
                                ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64),
                                ctypes.POINTER(ctypes.c_int64)]
        lib.gen_run.restype = ctypes.c_int
        lib.gen_free.argtypes = [ctypes.c_void_p]
        lib.gen_track_info.argtypes = [ctypes.POINTER(_Params), ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]
        lib.gen_track_info.restype = ctypes.c_int
        lib.gen_track_table.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_int64)]
        lib.gen_track_table.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class GenParams:
    """Knobs of one generated event or timeframe (defaults: central Pb-Pb event)."""
    seed: int = 1
    n_primaries: int = 8000
    n_secondaries: int = 1600
    pt_min: float = 0.1
    pt_max: float = 10.0
    eta_max: float = 0.9
    phi_min: float = 0.0
    phi_max: float = 2.0 * math.pi
    phi_radius: float = 0.0
    sec_r_max: float = 30.0
    sectors: tuple = tuple(range(36))
    sigma_y: float = 0.1
    sigma_z: float = 0.1
    row_eff: float = 0.95
    noise_frac: float = 0.02
    bz_kg: float = 5.0
    timeframe: bool = False
    tf_length_us: float = 10000.0
    rate_khz: float = 50.0
    vdrift: float = 2.5
    mb_offset: float = 50.0
    mb_max: float = 8000.0
    n_threads: int = field(default_factory=lambda: min(os.cpu_count() or 1, 32))
    legs: int = 1  # half-turns of a looper (1: only the first outgoing one)

    def _c(self) -> _Params:
        mask = 0
        for s in self.sectors:
            mask |= 1 << int(s)
        return _Params(self.seed, self.n_primaries, self.n_secondaries, self.pt_min, self.pt_max, self.eta_max,
                       self.phi_min, self.phi_max, self.phi_radius, self.sec_r_max, mask, self.sigma_y, self.sigma_z, self.row_eff,
                       self.noise_frac, self.bz_kg, int(self.timeframe), self.tf_length_us, self.rate_khz,
                       self.vdrift, self.mb_offset, self.mb_max, self.n_threads, self.legs)


@dataclass
class Event:
    """Clusters (16-byte records in input order) plus optional MC truth."""
    clusters: np.ndarray
    truth: np.ndarray | None
    n_tracks: int
    params: GenParams


def generate(p: GenParams, truth: bool = False) -> Event:
    lib = _load()
    cp = p._c()
    pc, pt = ctypes.c_void_p(), ctypes.c_void_p()
    n, ntr = ctypes.c_int64(), ctypes.c_int64()
    rc = lib.gen_run(ctypes.byref(cp), ctypes.byref(pc), ctypes.byref(pt) if truth else None,
                     ctypes.byref(n), ctypes.byref(ntr))
    if rc != 0:
        raise RuntimeError("generator failed")
    try:
        cl = np.frombuffer((ctypes.c_char * (n.value * 16)).from_address(pc.value), dtype=CLUSTER_DTYPE).copy() \
            if n.value else np.zeros(0, CLUSTER_DTYPE)
        tr = None
        if truth:
            tr = np.frombuffer((ctypes.c_char * (n.value * 48)).from_address(pt.value), dtype=TRUTH_DTYPE).copy() \
                if n.value else np.zeros(0, TRUTH_DTYPE)
    finally:
        lib.gen_free(pc)
        if truth:
            lib.gen_free(pt)
    return Event(cl, tr, int(ntr.value), p)


TRACK_TABLE_DTYPE = np.dtype([("xv", "<f8"), ("yv", "<f8"), ("phi0", "<f8"), ("pt", "<f8"), ("q", "<f8"),
                              ("t", "<f8"), ("tc", "<f8")])


def track_table(p: GenParams) -> np.ndarray:
    """Kinematics of every track drawn with `p`, indexed by label (cluster
    id): vertex (xv, yv), phi0, pT, charge, t = sinh(eta) and the collision
    time tc in us (timeframes; 0 for events)."""
    lib = _load()
    cp = p._c()
    n = ctypes.c_int64()
    if lib.gen_track_table(ctypes.byref(cp), None, 0, ctypes.byref(n)) != 0:
        raise RuntimeError("generator failed")
    out = np.zeros(n.value, TRACK_TABLE_DTYPE)
    if n.value and lib.gen_track_table(ctypes.byref(cp), out.ctypes.data, n.value, ctypes.byref(n)) != 0:
        raise RuntimeError("generator failed")
    return out


def track_info(p: GenParams, label: int) -> dict:
    """Kinematics of track `label` of an event generated with `p`."""
    lib = _load()
    out = (ctypes.c_double * 7)()
    if lib.gen_track_info(ctypes.byref(p._c()), label, out) != 0:
        raise IndexError(label)
    return dict(zip(("xv", "yv", "phi0", "pt", "q", "t", "tc"), list(out)))


# ---------------------------------------------------------------- workloads

def one_sector(seed: int = 0, n_tracks: int = 400, truth: bool = False, **kw) -> Event:
    """Plain method, one sector: 20-degree wedge, one z side, `n_tracks`
    primaries whose azimuth at the first pad row (85.2 cm) is uniform inside
    the wedge of sector 0 (only eta>0 ones leave clusters on that side)."""
    p = GenParams(seed=seed, n_primaries=n_tracks, n_secondaries=0, phi_min=0.0,
                  phi_max=math.radians(20.0), phi_radius=85.2, sectors=(0,))
    for k, v in kw.items():
        setattr(p, k, v)
    return generate(p, truth=truth)


def central_event(seed: int = 1, n_primaries: int = 8000, n_secondaries: int = 1600, truth: bool = False,
                  **kw) -> Event:
    """Plain method, full TPC: one central Pb-Pb-like event (~1.3M clusters)."""
    p = GenParams(seed=seed, n_primaries=n_primaries, n_secondaries=n_secondaries)
    for k, v in kw.items():
        setattr(p, k, v)
    return generate(p, truth=truth)


def looper_event(seed: int = 1, n_primaries: int = 16000, n_secondaries: int = 4000, truth: bool = False,
                 **kw) -> Event:
    """A central event in full acceptance for cluster rejection (~1.06M
    clusters): |eta| < 1.5, pT from 40 MeV/c (the p^-3 spectrum), secondaries
    born anywhere inside the outermost row radius (low-momentum ones among
    them), and loopers followed for four half-turns; about half of the
    clusters sit on further looper legs, below 50 MeV/c or at |dz/ds_T| > 2."""
    p = GenParams(seed=seed, n_primaries=n_primaries, n_secondaries=n_secondaries, eta_max=1.5, pt_min=0.04,
                  sec_r_max=200.0, legs=4)
    for k, v in kw.items():
        setattr(p, k, v)
    return generate(p, truth=truth)


def timeframe(seed: int = 2, length_ms: float = 10.0, truth: bool = False, **kw) -> Event:
    """Continuous read-out timeframe at 50 kHz with z taken from drift time
    (v_drift 2.5 cm/us, 250 cm drift).  Per-collision track counts follow the
    minimum-bias density ~1/(N+50) on [0, 8000]; secondaries at the same 1:5
    ratio as the central event."""
    p = GenParams(seed=seed, n_primaries=5, n_secondaries=1, timeframe=True, tf_length_us=length_ms * 1000.0)
    for k, v in kw.items():
        setattr(p, k, v)
    return generate(p, truth=truth)


@dataclass
class Request:
    request_id: int
    clusters: np.ndarray
    n_tracks: int
    sectors: tuple


def batch_requests(seed: int = 3, n_requests: int = 256, min_tracks: int = 50, max_tracks: int = 8000) -> list:
    """Independent requests of uneven size: each is an event with a
    log-uniform track count on [min_tracks, max_tracks] (20% extra
    secondaries) whose clusters are kept in k sectors, k uniform on 1..36."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_requests):
        nt = int(round(math.exp(rng.uniform(math.log(min_tracks), math.log(max_tracks)))))
        k = int(rng.integers(1, 37))
        secs = tuple(sorted(int(s) for s in rng.choice(36, size=k, replace=False)))
        ev = generate(GenParams(seed=seed * 100003 + i, n_primaries=nt, n_secondaries=nt // 5, sectors=secs))
        out.append(Request(i, ev.clusters, nt + nt // 5, secs))
    return out


def timeframe_stream(seed: int = 4, n_distinct: int = 8, min_ms: float = 1.0, max_ms: float = 20.0) -> list:
    """A pool of distinct seeded timeframes with lengths uniform in
    [min_ms, max_ms] for the serving loop (replayed with Poisson arrivals)."""
    rng = np.random.default_rng(seed)
    return [timeframe(seed=seed * 1000 + i, length_ms=float(rng.uniform(min_ms, max_ms))) for i in range(n_distinct)]


def straight_lines(seed: int = 0, n_lines: int = 10, sector: int = 0, sigma: float = 0.0, rows=range(159),
                   max_slope: float = 0.3, spacing: float = 6.0) -> Event:
    """Straight tracks (the Bz -> 0 limit) in one sector's local frame:
    y = y0 + b*x, z = z0 + e*x at every listed row, optionally smeared.
    Lines are spaced `spacing` cm apart in y at the first row and share one
    slope, so they never come within a link window of each other."""
    rng = np.random.default_rng(seed)
    rows = np.asarray(list(rows), dtype=np.int64)
    xr = np.array([float(np.float32(85.2 + r * ((245.8 - 85.2) / 158.0))) for r in range(159)])
    b = rng.uniform(-max_slope, max_slope)
    e = rng.uniform(0.05, 0.8)
    out, tru = [], []
    for k in range(n_lines):
        y_first = -0.5 * spacing * (n_lines - 1) + spacing * k - b * xr[0]
        z0 = rng.uniform(5.0, 50.0)
        for r in rows:
            x = xr[r]
            y, z = y_first + b * x, z0 + e * x
            if abs(y) > x * 0.17632698070846498 or z > 250.0:
                continue
            c = np.zeros(1, CLUSTER_DTYPE)
            c["y"], c["z"] = y + sigma * rng.normal(), z + sigma * rng.normal()
            c["row"], c["sector"], c["id"] = r, sector, k
            t = np.zeros(1, TRUTH_DTYPE)
            cphi = 1.0 / math.sqrt(1.0 + b * b)
            t["track"], t["y"], t["z"], t["sphi"], t["tgl"], t["qpt"] = k, y, z, b * cphi, e * cphi, 0.0
            out.append(c)
            tru.append(t)
    cl = np.concatenate(out) if out else np.zeros(0, CLUSTER_DTYPE)
    tr = np.concatenate(tru) if tru else np.zeros(0, TRUTH_DTYPE)
    return Event(cl, tr, n_lines, GenParams(seed=seed, bz_kg=0.0))
