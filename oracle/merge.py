"""FP64 oracle of the second tracking phase: merging sector segments and
refitting the merged tracks (test infrastructure only).

Sec. 2: the second phase merges the track segments found in the individual
sectors into final tracks and refits them.  The arithmetic (the frame
turn of a state with its covariance, the pair chi2, the mutual-best
pairing and the chained refit) is in tpc_oracle.c (orc_merge_pairs,
orc_merge_refit); this module gathers the oracle's own segments and
clusters and marshals them.  Only the tests, the package smoke check and
the benchmark's CPU leg import it.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import NROW, NSEC, F_REFIT_FAIL, _load, codec_input

_bound = False


def _bind():
    global _bound
    lib = _load()
    if not _bound:
        P = ctypes.c_void_p
        lib.orc_merge_pairs.argtypes = [P, ctypes.c_int32] + [P] * 7 + [ctypes.c_double, ctypes.c_int32,
                                                                         ctypes.c_int32, ctypes.c_double, P, P, P, P]
        lib.orc_merge_pairs.restype = ctypes.c_int
        lib.orc_merge_refit.argtypes = [P, ctypes.c_int32, P, P, P, P, P, ctypes.c_int32, P, P, P, P, P]
        lib.orc_merge_refit.restype = ctypes.c_int
        _bound = True
    return lib


def default_params(**kw) -> dict:
    p = {"chi2_max": 25.0, "overlap": 10, "min_clusters": 10, "window_cm": 10.0}
    p.update(kw)
    return p


def segments(ref: dict) -> dict:
    """The oracle's refitted sector tracks as segments."""
    tl = ref["t_tracklet"]
    rs = ref["rs_of"][ref["tl_start"][tl]] if len(tl) else np.zeros(0, np.int64)
    return {"request": (rs // (NROW * NSEC)).astype(np.int32), "sector": ((rs // NROW) % NSEC).astype(np.int32),
            "row_in": ref["t_row_in"].astype(np.int32), "row_out": ref["t_row_out"].astype(np.int32),
            "n": ref["t_n"].astype(np.int32), "par": np.ascontiguousarray(ref["t_par"], np.float64),
            "cov": np.ascontiguousarray(ref["t_cov"], np.float64),
            "refit_ok": (ref["t_flags"] & F_REFIT_FAIL) == 0}


def pairs(seg: dict, p: dict | None = None) -> dict:
    """Mutual-best pairs of inner and outer segments in adjacent sectors."""
    p = default_params(**(p or {}))
    lib = _bind()
    n = len(seg["n"])
    ncl = np.where(seg["refit_ok"], seg["n"], 0).astype(np.int32)  # a failed refit takes no part
    link = np.zeros(n, np.int32)
    chi2 = np.zeros(n, np.float64)
    second = np.zeros(n, np.float64)
    second_in = np.zeros(n, np.float64)
    c = lambda a: np.ascontiguousarray(a).ctypes.data  # noqa: E731
    if n:
        lib.orc_merge_pairs(None, n, c(seg["request"]), c(seg["sector"]), c(seg["row_in"]), c(seg["row_out"]),
                            c(ncl), c(seg["par"]), c(seg["cov"]), p["chi2_max"], p["overlap"], p["min_clusters"],
                            p["window_cm"], link.ctypes.data, chi2.ctypes.data, second.ctypes.data, second_in.ctypes.data)
    return {"link": link, "chi2": chi2, "second": second, "second_in": second_in}


def chains(link: np.ndarray) -> list:
    """Chains of segments linked inner -> outer, innermost first."""
    n = len(link)
    has_inner = np.zeros(n, bool)
    has_inner[link[link >= 0]] = True
    out = []
    for a in range(n):
        if has_inner[a] or link[a] < 0:
            continue
        ch = [a]
        while link[ch[-1]] >= 0:
            ch.append(int(link[ch[-1]]))
        out.append(ch)
    return out


def merge(ref: dict, clusters: np.ndarray, p: dict | None = None) -> dict:
    """Pairs, chains and the refit of every merged chain: per chain its
    parameters and covariance at the innermost cluster (innermost segment's
    frame), chi2, ndf and cluster count."""
    lib = _bind()
    seg = segments(ref)
    pr = pairs(seg, p)
    ch = chains(pr["link"])
    inp = codec_input(ref, clusters)  # per track: the refit's seed and clusters outermost first
    m = len(ch)
    par = np.zeros((m, 5))
    cov = np.zeros((m, 15))
    chi2 = np.zeros(m)
    ok = np.zeros(m, bool)
    ncl = np.zeros(m, np.int64)
    row_in = np.zeros(m, np.int32)
    for k, c in enumerate(ch):
        order = c[::-1]  # outermost segment first
        sec = np.array([seg["sector"][g] for g in order], np.int32)
        off = np.concatenate([[0], np.cumsum([inp["off"][g + 1] - inp["off"][g] for g in order])]).astype(np.int64)
        idx = np.concatenate([inp["cluster"][inp["off"][g]:inp["off"][g + 1]] for g in order])
        rows = np.ascontiguousarray(clusters["row"][idx].astype(np.int32))
        y = np.ascontiguousarray(clusters["y"][idx].astype(np.float64))
        z = np.ascontiguousarray(clusters["z"][idx].astype(np.float64))
        seed = np.ascontiguousarray(inp["head"][order[0]])
        po, co, c2, ri = np.zeros(5), np.zeros(15), ctypes.c_double(), ctypes.c_int32()
        ok[k] = bool(inp["ok"][order[0]]) and bool(lib.orc_merge_refit(
            None, len(order), sec.ctypes.data, off.ctypes.data, rows.ctypes.data, y.ctypes.data, z.ctypes.data,
            int(inp["row_out"][order[0]]), seed.ctypes.data, po.ctypes.data, co.ctypes.data, ctypes.byref(c2),
            ctypes.byref(ri)))
        par[k], cov[k], chi2[k], ncl[k], row_in[k] = po, co, c2.value, len(idx), ri.value
    return {"segments": seg, "link": pr["link"], "pair_chi2": pr["chi2"], "pair_second": pr["second"],
            "pair_second_in": pr["second_in"],
            "chains": ch, "par": par, "cov": cov, "chi2": chi2, "ndf": 2 * ncl - 5, "n": ncl, "ok": ok,
            "row_in": row_in}


def adjacent_sectors(s1, s2) -> bool:
    """Neighbouring sectors on the same side (the pairing's sector test)."""
    if s1 // 18 != s2 // 18:
        return False
    d = ((s2 % 18) - (s1 % 18) + 18) % 18
    return d in (1, 17)
