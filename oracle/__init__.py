"""FP64 CPU oracle of the sector tracker (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package.  The arithmetic lives in tpc_oracle.c (plain C,
FP64); this module only marshals numpy arrays in and out of it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# The mutation tests plant a mistake in a copy of the oracle source and check
# that the pins catch it; they point this variable at the mutated copy.
if os.environ.get("TPC_ORACLE_MUTANT_SRC"):
    _SRC = os.environ["TPC_ORACLE_MUTANT_SRC"]
    _LIB = _SRC[:-2] + ".so"

NROW = 159
NSEC = 36
# follow / refit flags
F_TAINT_TIE, F_TAINT_GATE, F_TAINT_EDGE, F_TAINT_SLIM = 1, 2, 4, 8
F_SEED_FAIL, F_BACK_FAIL, F_REFIT_FAIL = 16, 32, 64
F_TAINT_ANY = F_TAINT_TIE | F_TAINT_GATE | F_TAINT_EDGE | F_TAINT_SLIM


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -ffp-contract=off so binary32 steps round once per operation)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class Config(ctypes.Structure):
    _fields_ = [("bz_kg", ctypes.c_double), ("sigma", ctypes.c_double), ("d_max", ctypes.c_float),
                ("min_chain", ctypes.c_int), ("max_miss", ctypes.c_int), ("n_min_track", ctypes.c_int),
                ("gate", ctypes.c_double), ("c0", ctypes.c_double * 5), ("s_max", ctypes.c_double),
                ("edge", ctypes.c_double), ("taint_rel", ctypes.c_double), ("trace_t", ctypes.c_int),
                ("link_skip", ctypes.c_int)]


_P = ctypes.c_void_p


class _Result(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("n_req", ctypes.c_int32), ("n_rs", ctypes.c_int32),
                ("n_bins", ctypes.c_int64), ("n_tracklets", ctypes.c_int32), ("n_tracks", ctypes.c_int32)] + \
               [(name, _P) for name in (
                   "row_start", "z_lo", "z_hi", "inv_y", "inv_z", "n_y", "n_z", "bin_base", "bin_start", "perm",
                   "rs_of", "sy", "sz", "up", "dn", "up_m", "dn_m", "tie", "tl_start", "tl_len",
                   "f_n", "f_nf", "f_nb", "f_flags", "f_row", "f_hits", "f_par", "f_cov", "f_chi2",
                   "owner", "tl_track", "cluster_track",
                   "t_tracklet", "t_n", "t_ndf", "t_flags", "t_row_in", "t_row_out", "t_par", "t_cov", "t_chi2",
                   "trace")] + [("n_trace", ctypes.c_int32)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_codec.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int32] + [ctypes.c_void_p] * 9 + \
            [ctypes.c_double, ctypes.c_void_p]
        lib.orc_codec.restype = ctypes.c_int
        lib.orc_quantise.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p]
        lib.orc_quantise.restype = None
        lib.orc_default_config.argtypes = [ctypes.POINTER(Config)]
        lib.orc_run.argtypes = [ctypes.POINTER(Config), ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                ctypes.c_int32, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_Result)]
        lib.orc_run.restype = ctypes.c_int
        lib.orc_free.argtypes = [ctypes.POINTER(_Result)]
        lib.orc_kalman_fit.argtypes = [ctypes.POINTER(Config), ctypes.c_int] + [ctypes.c_void_p] * 7
        lib.orc_kalman_fit.restype = ctypes.c_int
        lib.orc_propagate_rows.argtypes = [ctypes.POINTER(Config), ctypes.c_int] + [ctypes.c_void_p] * 3
        lib.orc_propagate_rows.restype = ctypes.c_int
        lib.orc_tables.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


def default_config(**overrides) -> Config:
    cfg = Config()
    _load().orc_default_config(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k == "c0":
            for i in range(5):
                cfg.c0[i] = v[i]
        else:
            setattr(cfg, k, v)
    return cfg


def _arr(ptr, dtype, count):
    if not ptr or count <= 0:
        return np.zeros(0, dtype)
    nbytes = int(count) * np.dtype(dtype).itemsize
    return np.frombuffer((ctypes.c_char * nbytes).from_address(ptr), dtype=dtype).copy()


STAGES = {"grid": 2, "neighbours": 3, "links": 4, "tracklets": 5, "follow": 6, "select": 7, "refit": 8}


def run(clusters: np.ndarray, req_offsets=None, stop_after: str = "refit", brute: bool = False,
        threads: int | None = None, cfg: Config | None = None) -> dict:
    """Run the oracle on a 16-byte cluster array (one request unless
    req_offsets [0, ..., n] splits it into independent requests)."""
    lib = _load()
    clusters = np.ascontiguousarray(clusters)
    n = len(clusters)
    if req_offsets is None:
        req_offsets = [0, n]
    off = np.ascontiguousarray(np.asarray(req_offsets, dtype=np.int64))
    nreq = len(off) - 1
    res = _Result()
    thr = threads if threads is not None else (os.cpu_count() or 1)
    rc = lib.orc_run(ctypes.byref(cfg) if cfg is not None else None, clusters.ctypes.data if n else None, n,
                     off.ctypes.data, nreq, STAGES[stop_after], int(brute), thr, ctypes.byref(res))
    try:
        if rc != 0:
            raise ValueError(f"oracle returned {rc}")
        out = {"n": n, "n_req": nreq, "n_rs": res.n_rs, "n_bins": res.n_bins}
        nrs, nb = res.n_rs, res.n_bins
        out.update(row_start=_arr(res.row_start, np.int32, nrs + 1), z_lo=_arr(res.z_lo, np.float32, nrs),
                   z_hi=_arr(res.z_hi, np.float32, nrs), inv_y=_arr(res.inv_y, np.float32, nrs),
                   inv_z=_arr(res.inv_z, np.float32, nrs), n_y=_arr(res.n_y, np.int32, nrs),
                   n_z=_arr(res.n_z, np.int32, nrs), bin_base=_arr(res.bin_base, np.int64, nrs + 1),
                   bin_start=_arr(res.bin_start, np.int32, nb + 1), perm=_arr(res.perm, np.int32, n),
                   rs_of=_arr(res.rs_of, np.int32, n), sy=_arr(res.sy, np.float32, n),
                   sz=_arr(res.sz, np.float32, n))
        if STAGES[stop_after] >= 3:
            out.update(up=_arr(res.up, np.int32, n), dn=_arr(res.dn, np.int32, n), tie=_arr(res.tie, np.uint8, n))
        if STAGES[stop_after] >= 4:
            out.update(up_m=_arr(res.up_m, np.int32, n), dn_m=_arr(res.dn_m, np.int32, n))
        if STAGES[stop_after] >= 5:
            nt = res.n_tracklets
            out.update(n_tracklets=nt, tl_start=_arr(res.tl_start, np.int32, nt), tl_len=_arr(res.tl_len, np.int32, nt))
        if STAGES[stop_after] >= 6:
            nt = res.n_tracklets
            out.update(f_n=_arr(res.f_n, np.int32, nt), f_nf=_arr(res.f_nf, np.int32, nt),
                       f_nb=_arr(res.f_nb, np.int32, nt), f_flags=_arr(res.f_flags, np.int32, nt),
                       f_row=_arr(res.f_row, np.int32, nt),
                       f_hits=_arr(res.f_hits, np.int32, nt * NROW).reshape(nt, NROW),
                       f_par=_arr(res.f_par, np.float64, nt * 5).reshape(nt, 5),
                       f_cov=_arr(res.f_cov, np.float64, nt * 15).reshape(nt, 15),
                       f_chi2=_arr(res.f_chi2, np.float64, nt))
        if STAGES[stop_after] >= 7:
            nt = res.n_tracklets
            out.update(owner=_arr(res.owner, np.uint64, n), tl_track=_arr(res.tl_track, np.int32, nt),
                       cluster_track=_arr(res.cluster_track, np.int32, n), n_tracks=res.n_tracks)
        if STAGES[stop_after] >= 8:
            m = res.n_tracks
            out.update(t_tracklet=_arr(res.t_tracklet, np.int32, m), t_n=_arr(res.t_n, np.int32, m),
                       t_ndf=_arr(res.t_ndf, np.int32, m), t_flags=_arr(res.t_flags, np.int32, m),
                       t_row_in=_arr(res.t_row_in, np.int32, m), t_row_out=_arr(res.t_row_out, np.int32, m),
                       t_par=_arr(res.t_par, np.float64, m * 5).reshape(m, 5),
                       t_cov=_arr(res.t_cov, np.float64, m * 15).reshape(m, 15),
                       t_chi2=_arr(res.t_chi2, np.float64, m))
        if res.trace:
            out["trace"] = _arr(res.trace, np.float64, 16 * res.n_trace).reshape(-1, 16)
        return out
    finally:
        lib.orc_free(ctypes.byref(res))


def quantise(v, unit: float) -> np.ndarray:
    """Fixed-point coordinate rint(v * (1/unit)) in binary32 (the lossy
    format conversion ahead of the track-model compression)."""
    lib = _load()
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float32))
    q = np.zeros(len(v), np.int32)
    if len(v):
        lib.orc_quantise(len(v), v.ctypes.data, unit, q.ctypes.data)
    return q


def codec_input(ref: dict, clusters: np.ndarray, unit: float = 0.01, cfg: Config | None = None) -> dict:
    """The oracle's compression input: per track the header -- the follow
    state carried to the outermost owned row, as the refit starts -- and its
    owned clusters outermost first (rows, fixed-point y and z)."""
    m = ref["n_tracks"]
    ct = ref["cluster_track"].astype(np.int64)
    idx = np.nonzero(ct >= 0)[0]
    rows_all = clusters["row"].astype(np.int64)
    idx = idx[np.lexsort((-rows_all[idx], ct[idx]))]  # by track, outermost first
    off = np.zeros(m + 1, np.int64)
    np.add.at(off, ct[idx] + 1, 1)
    off = np.cumsum(off)
    head = np.zeros((m, 5), np.float64)
    ok = np.ones(m, np.int32)
    for tr in range(m):
        t = ref["t_tracklet"][tr]
        fr, ro = int(ref["f_row"][t]), int(ref["t_row_out"][tr])
        step = 1 if ro >= fr else -1
        path = np.arange(fr, ro + step, step, dtype=np.int32)
        try:
            head[tr] = propagate_rows(path, ref["f_par"][t], cfg)[-1]
        except ValueError:
            ok[tr] = 0
    return {"row_out": ref["t_row_out"].astype(np.int32), "head": head, "ok": ok, "off": off,
            "cluster": idx, "rows": rows_all[idx].astype(np.int32),
            "qy": quantise(clusters["y"][idx], unit), "qz": quantise(clusters["z"][idx], unit), "unit": unit}


def codec(inp: dict, decode: bool = False, ry=None, rz=None, cfg: Config | None = None) -> dict:
    """Track-model compression (decode=False: residuals from the clusters) or
    decompression (decode=True: clusters from the residuals) of codec_input
    tracks.  Also returns, per cluster, the distance of the prediction (in
    units) from the rounding boundary, and per track whether it ran."""
    lib = _load()
    m = len(inp["row_out"])
    n = int(inp["off"][-1])
    qy = inp["qy"].copy() if not decode else np.zeros(n, np.int32)
    qz = inp["qz"].copy() if not decode else np.zeros(n, np.int32)
    ry = np.zeros(n, np.int32) if not decode else np.ascontiguousarray(ry, dtype=np.int32)
    rz = np.zeros(n, np.int32) if not decode else np.ascontiguousarray(rz, dtype=np.int32)
    margin = np.zeros(n, np.float64)
    ok = np.zeros(m, np.int32)
    row_out = np.ascontiguousarray(inp["row_out"], dtype=np.int32)
    head = np.ascontiguousarray(inp["head"], dtype=np.float64)
    off = np.ascontiguousarray(inp["off"], dtype=np.int64)
    rows = np.ascontiguousarray(inp["rows"], dtype=np.int32)
    lib.orc_codec(ctypes.byref(cfg) if cfg is not None else None, int(decode), m, row_out.ctypes.data,
                  head.ctypes.data, off.ctypes.data, rows.ctypes.data, qy.ctypes.data, qz.ctypes.data,
                  ry.ctypes.data, rz.ctypes.data, margin.ctypes.data, inp["unit"], ok.ctypes.data)
    ok &= inp["ok"]
    return {"qy": qy, "qz": qz, "ry": ry, "rz": rz, "margin": margin, "ok": ok}


def kalman_fit(rows, my, mz, p0, cfg: Config | None = None):
    """Direct Kalman fit over measurements at `rows` (monotone), seeded with
    p0 at rows[0] and the seed covariance.  Returns (p, packed cov, chi2)."""
    lib = _load()
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    my = np.ascontiguousarray(my, dtype=np.float64)
    mz = np.ascontiguousarray(mz, dtype=np.float64)
    p0 = np.ascontiguousarray(p0, dtype=np.float64)
    p = np.zeros(5)
    cov = np.zeros(15)
    chi2 = np.zeros(1)
    ok = lib.orc_kalman_fit(ctypes.byref(cfg) if cfg is not None else None, len(rows), rows.ctypes.data,
                            my.ctypes.data, mz.ctypes.data, p0.ctypes.data, p.ctypes.data, cov.ctypes.data,
                            chi2.ctypes.data)
    if not ok:
        raise ValueError("propagation failed")
    return p, cov, float(chi2[0])


def propagate_rows(rows, p0, cfg: Config | None = None) -> np.ndarray:
    """State-only propagation of p0 (at rows[0]) to each of `rows`."""
    lib = _load()
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    p0 = np.ascontiguousarray(p0, dtype=np.float64)
    out = np.zeros((len(rows), 5))
    if not lib.orc_propagate_rows(ctypes.byref(cfg) if cfg is not None else None, len(rows), rows.ctypes.data,
                                  p0.ctypes.data, out.ctypes.data):
        raise ValueError("propagation failed")
    return out


def tables():
    """Row radii and active half-widths (binary32) as the oracle uses them."""
    x = np.zeros(NROW, np.float32)
    yhi = np.zeros(NROW, np.float32)
    _load().orc_tables(x.ctypes.data, yhi.ctypes.data)
    return x, yhi


def unpack_cov(c15) -> np.ndarray:
    """Packed lower triangle (row-major) -> symmetric 5x5."""
    c15 = np.asarray(c15)
    C = np.zeros(c15.shape[:-1] + (5, 5))
    q = 0
    for i in range(5):
        for j in range(i + 1):
            C[..., i, j] = c15[..., q]
            C[..., j, i] = c15[..., q]
            q += 1
    return C
