"""B300-native per-sector TPC track finding (arXiv 1709.00618, Sec. 2).

Thin ctypes binding of libtpcca.so (declared in include/tpcca.h).  Every step
of the path runs in the library's CUDA kernels; this module only marshals
arguments.  PyTorch, when used, only provides device memory (the arena) and
the CUDA stream.  There is no CPU fallback: without the compiled library and
a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB_PATH, build  # noqa: F401

__all__ = ["Tracker", "Server", "TpcError", "TRACK_DTYPE", "CLUSTER_DTYPE", "build", "load_library", "default_config",
           "ITEMS"]

CLUSTER_DTYPE = np.dtype([("y", "<f4"), ("z", "<f4"), ("row", "<u2"), ("sector", "<u2"), ("id", "<u4")])
TRACK_DTYPE = np.dtype([("x", "<f4"), ("par", "<f4", (5,)), ("cov", "<f4", (15,)), ("reserved", "<i4"),
                        ("chi2", "<f8"), ("ndf", "<i4"), ("n_clusters", "<i4"), ("sector", "<i4"),
                        ("request", "<i4"), ("first_row", "<i4"), ("last_row", "<i4"),
                        ("cluster_offset", "<i4"), ("flags", "<i4")])
assert CLUSTER_DTYPE.itemsize == 16 and TRACK_DTYPE.itemsize == 128
RS_PARAMS_DTYPE = np.dtype([("z_lo", "<f4"), ("z_hi", "<f4"), ("inv_y", "<f4"), ("inv_z", "<f4"), ("n_y", "<i4"),
                            ("n_z", "<i4"), ("bin_base", "<i4"), ("count", "<i4")])

TPC_OK, TPC_EINVAL, TPC_ENOMEM, TPC_ECUDA, TPC_ETIMEOUT, TPC_EOVERFLOW, TPC_EBUSY = range(7)
_CODES = {1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EOVERFLOW", 6: "EBUSY"}
TF_TAINT_ANY = 1 | 2 | 4 | 8
TF_SEED_FAIL, TF_BACK_FAIL, TF_REFIT_FAIL = 16, 32, 64  # TPC_TF_* of tpcca.h

# item -> (numpy dtype, columns)
ITEMS = {"perm": (1, np.int32), "rs_of": (2, np.int32), "row_start": (3, np.int32), "rs_params": (4, RS_PARAMS_DTYPE),
         "bin_start": (5, np.int32), "up": (6, np.int32), "dn": (7, np.int32), "tie": (8, np.uint8),
         "up_m": (9, np.int32), "dn_m": (10, np.int32), "tl_start": (11, np.int32), "tl_len": (12, np.int32),
         "f_n": (13, np.int32), "f_nf": (14, np.int32), "f_nb": (15, np.int32), "f_flags": (16, np.int32),
         "f_row": (17, np.int32), "f_hits": (18, np.int32), "f_par": (19, np.float32), "f_cov": (20, np.float32),
         "f_chi2": (21, np.float64), "owner": (22, np.uint64), "tl_track": (23, np.int32), "sy": (24, np.float32),
         "sz": (25, np.float32)}


class TpcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"TPC_{_CODES.get(code, code)}: {msg}")
        self.code = code


class TpcTuning(ctypes.Structure):
    _fields_ = [("block_clusters", ctypes.c_int32), ("block_follow", ctypes.c_int32),
                ("ctas_per_sm_zone", ctypes.c_int32), ("ctas_per_sm_follow", ctypes.c_int32),
                ("refill", ctypes.c_int32), ("chunks", ctypes.c_int32), ("zone_rows", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class VertexConfig(ctypes.Structure):
    _fields_ = [("vdrift_cm_us", ctypes.c_double), ("zmax_cm", ctypes.c_double), ("dca_max_cm", ctypes.c_double),
                ("ext_max_cm", ctypes.c_double), ("gap_us", ctypes.c_double), ("min_tracks", ctypes.c_int32),
                ("min_clusters", ctypes.c_int32), ("min_pt_gev", ctypes.c_double)]


class RejectConfig(ctypes.Structure):
    _fields_ = [("p_min_gev", ctypes.c_double), ("tgl_max", ctypes.c_double), ("dz_leg_cm", ctypes.c_double),
                ("z_ref_cm", ctypes.c_double), ("use_vertices", ctypes.c_int32), ("reserved", ctypes.c_int32)]


RJ_LOW_P, RJ_INCLINED, RJ_LOOPER_LEG = 1, 2, 4


class MergeConfig(ctypes.Structure):
    _fields_ = [("chi2_max", ctypes.c_double), ("overlap_rows", ctypes.c_int32), ("min_clusters", ctypes.c_int32),
                ("window_cm", ctypes.c_double)]


CODEC_HEADER_DTYPE = np.dtype([("par", "<f4", (5,)), ("row_out", "<i4"), ("n_clusters", "<i4"), ("ok", "<i4")])
assert CODEC_HEADER_DTYPE.itemsize == 32

VERTEX_DTYPE = np.dtype([("time_us", "<f8"), ("n_tracks", "<i4"), ("request", "<i4")])


class TpcConfig(ctypes.Structure):
    _fields_ = [("bz_kg", ctypes.c_double), ("sigma", ctypes.c_double), ("d_max", ctypes.c_float),
                ("min_chain", ctypes.c_int32), ("max_miss", ctypes.c_int32), ("n_min_track", ctypes.c_int32),
                ("gate", ctypes.c_double), ("c0", ctypes.c_double * 5), ("s_max", ctypes.c_double),
                ("edge", ctypes.c_double), ("taint_rel", ctypes.c_double), ("fp64_updates", ctypes.c_int32),
                ("link_skip", ctypes.c_int32)]


_lib = None
_VP, _I64, _I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32


class TpcRequest(ctypes.Structure):
    """One request of tpc_submit_batch (pointers to host buffers)."""
    _fields_ = [("id", _I64), ("clusters", _VP), ("n", _I64), ("tracks_out", _VP), ("cap", _I64),
                ("cluster_track_out", _VP), ("n_tracks", _VP)]


def load_library(path: str | None = None):
    """Load libtpcca.so (built in-tree by build()).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: run paper_1709_00618_b300.build() (nvcc, sm_103a) first")
    lib = ctypes.CDLL(path)
    sig = {
        "tpc_default_config": ([_VP], ctypes.c_int),
        "tpc_create": ([_VP, _VP, ctypes.c_int, _VP, ctypes.c_size_t], ctypes.c_int),
        "tpc_create_with_arena": ([_VP, _VP, ctypes.c_int, _VP, _VP, ctypes.c_size_t], ctypes.c_int),
        "tpc_destroy": ([_VP], None),
        "tpc_last_error": ([_VP], ctypes.c_char_p),
        "tpc_arena_bytes": ([_I64, _I32], ctypes.c_size_t),
        "tpc_reserve": ([_VP, _I64, _I32, _I64, _I64], ctypes.c_int),
        "tpc_load_clusters": ([_VP, _VP, _I64, ctypes.c_int], ctypes.c_int),
        "tpc_load_batch": ([_VP, _VP, _VP, _I32, ctypes.c_int], ctypes.c_int),
        "tpc_find_tracks": ([_VP], ctypes.c_int),
        "tpc_fit_tracks": ([_VP], ctypes.c_int),
        "tpc_run_graph": ([_VP], ctypes.c_int),
        "tpc_get_tracks": ([_VP, _VP, _I64, _VP, _VP, _VP], ctypes.c_int),
        "tpc_sync": ([_VP], ctypes.c_int),
        "tpc_get_counts": ([_VP, _VP], ctypes.c_int),
        "tpc_get_stage": ([_VP, ctypes.c_int, _VP, _I64, _VP], ctypes.c_int),
        "tpc_set_tuning": ([_VP, _VP], ctypes.c_int),
        "tpc_get_tuning": ([_VP, _VP], ctypes.c_int),
        "tpc_set_profiling": ([_VP, ctypes.c_int], ctypes.c_int),
        "tpc_get_stage_times": ([_VP, _VP], ctypes.c_int),
        "tpc_get_work": ([_VP, _VP], ctypes.c_int),
        "tpc_get_kalman_profile": ([_VP, _VP, _VP], ctypes.c_int),
        "tpc_graph_kernels": ([_VP, _VP], ctypes.c_int),
        "tpc_measure_alu_peaks": ([ctypes.c_int, _VP, _VP], ctypes.c_int),
        "tpc_default_vertex_config": ([_VP], ctypes.c_int),
        "tpc_compress": ([_VP, ctypes.c_double], ctypes.c_int),
        "tpc_default_merge_config": ([_VP], ctypes.c_int),
        "tpc_default_reject_config": ([_VP], ctypes.c_int),
        "tpc_reject_clusters": ([_VP, _VP], ctypes.c_int),
        "tpc_get_rejection": ([_VP, _VP, _VP, _VP], ctypes.c_int),
        "tpc_merge_tracks": ([_VP, _VP], ctypes.c_int),
        "tpc_get_merged": ([_VP, _VP, _I64, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
        "tpc_get_compressed": ([_VP, _VP, _I64, _VP, _VP, _VP, _VP, _VP, _I64, _VP, _VP], ctypes.c_int),
        "tpc_decompress": ([_VP, _VP, _I64, _VP, _VP, _VP, _I64, ctypes.c_double, _VP, _VP], ctypes.c_int),
        "tpc_find_vertices": ([_VP, _VP], ctypes.c_int),
        "tpc_get_vertices": ([_VP, _VP, _I64, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
        "tpc_row_params_noalloc": ([_VP, _I64, _VP, _I32, _VP, _VP], ctypes.c_int),
        "tpc_autotune": ([_VP, _I32, _VP, _VP], ctypes.c_int),
        "tpc_set_trace": ([_VP, _I32], ctypes.c_int),
        "tpc_get_trace": ([_VP, _VP, _I32, _VP], ctypes.c_int),
        "tpc_server_create": ([_VP, _VP, ctypes.c_int, _I32, ctypes.c_size_t, _I32], ctypes.c_int),
        "tpc_server_submit": ([_VP, _I64, _VP, _I64, _VP, _I64, _VP], ctypes.c_int),
        "tpc_server_poll": ([_VP, _I64, _VP], ctypes.c_int),
        "tpc_server_result": ([_VP, _I64, _VP, _VP], ctypes.c_int),
        "tpc_get_tracks_async": ([_VP, _VP, _I64, _VP, _VP], ctypes.c_int),
        "tpc_track_host": ([_VP, _VP, _I64, _VP, _I64, _VP, _VP], ctypes.c_int),
        "tpc_get_arena_bytes": ([_VP, _VP], ctypes.c_int),
        "tpc_server_drain": ([_VP, ctypes.c_double], ctypes.c_int),
        "tpc_server_stats": ([_VP, _VP], ctypes.c_int),
        "tpc_server_destroy": ([_VP], None),
        "tpc_submit_batch": ([_VP, _VP, _I32], ctypes.c_int),
        "tpc_poll": ([_VP, _I64, _VP], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def default_config(**overrides) -> TpcConfig:
    cfg = TpcConfig()
    load_library().tpc_default_config(ctypes.byref(cfg))
    for k, v in overrides.items():
        if k == "c0":
            for i in range(5):
                cfg.c0[i] = v[i]
        else:
            setattr(cfg, k, v)
    return cfg


def _ptr(a) -> int:
    """Address of a numpy array or a torch tensor."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


class Tracker:
    """One tracking context on one CUDA device.

    arena: None (the library allocates within hbm_budget), "torch" (a torch
    uint8 tensor sized by tpc_arena_bytes for the first load), or a torch
    tensor to use as the arena.  stream: None (library-owned stream), a
    torch.cuda.Stream, or a raw cudaStream_t integer.
    """

    def __init__(self, device: int = 0, cfg: TpcConfig | None = None, stream=None, hbm_budget: int = 0,
                 arena=None, arena_clusters: int = 0, arena_requests: int = 1):
        self._lib = load_library()
        self._ctx = ctypes.c_void_p()
        self._cfg = cfg
        self._batch = {}
        self._arena_tensor = None
        self._stream_obj = stream
        sp = None
        if stream is not None:
            sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        if arena is None:
            rc = self._lib.tpc_create(ctypes.byref(self._ctx), ctypes.byref(cfg) if cfg else None, device, sp,
                                      hbm_budget)
        else:
            if isinstance(arena, str):
                import torch
                nbytes = self._lib.tpc_arena_bytes(max(arena_clusters, 1), max(arena_requests, 1))
                arena = torch.empty(nbytes + 256, dtype=torch.uint8, device=f"cuda:{device}")
            self._arena_tensor = arena
            base = arena.data_ptr()
            aligned = (base + 255) // 256 * 256
            nbytes = arena.numel() * arena.element_size() - (aligned - base)
            rc = self._lib.tpc_create_with_arena(ctypes.byref(self._ctx), ctypes.byref(cfg) if cfg else None, device,
                                                 sp, aligned, nbytes)
        if rc != 0:
            raise TpcError(rc, "tpc_create failed")
        self.n = 0

    # -- error plumbing
    def _ck(self, rc: int):
        if rc != 0:
            raise TpcError(rc, self._lib.tpc_last_error(self._ctx).decode())

    def close(self):
        if self._ctx:
            self._lib.tpc_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- the path
    def load(self, clusters, req_offsets=None):
        """clusters: numpy structured array (CLUSTER_DTYPE) on the host, or a
        CUDA torch tensor holding the same 16-byte records."""
        on_device = int(hasattr(clusters, "is_cuda") and clusters.is_cuda)
        if not on_device:
            clusters = np.ascontiguousarray(clusters)
            n = len(clusters)
        else:
            n = clusters.numel() * clusters.element_size() // 16
        self._keep_in = clusters
        if req_offsets is None:
            self._ck(self._lib.tpc_load_clusters(self._ctx, _ptr(clusters) if n else None, n, on_device))
        else:
            off = np.ascontiguousarray(np.asarray(req_offsets, dtype=np.int64))
            self._ck(self._lib.tpc_load_batch(self._ctx, _ptr(clusters) if n else None, off.ctypes.data,
                                              len(off) - 1, on_device))
        self.n = n
        return self

    def find(self):
        self._ck(self._lib.tpc_find_tracks(self._ctx))
        return self

    def fit(self):
        self._ck(self._lib.tpc_fit_tracks(self._ctx))
        return self

    def run_graph(self):
        self._ck(self._lib.tpc_run_graph(self._ctx))
        return self

    def sync(self):
        self._ck(self._lib.tpc_sync(self._ctx))
        return self

    def reserve(self, n_clusters=0, n_requests=0, n_bins=0, n_tracklets=0):
        self._ck(self._lib.tpc_reserve(self._ctx, n_clusters, n_requests, n_bins, n_tracklets))

    def set_tuning(self, **fields):
        """Launch shapes (tpc_tuning fields; omitted ones keep their value)."""
        t = TpcTuning()
        for k, v in fields.items():
            if not hasattr(t, k):
                raise TypeError(f"unknown tuning field {k}")
            setattr(t, k, int(v))
        self._ck(self._lib.tpc_set_tuning(self._ctx, ctypes.byref(t)))

    def tuning(self) -> dict:
        t = TpcTuning()
        self._ck(self._lib.tpc_get_tuning(self._ctx, ctypes.byref(t)))
        return t.as_dict()

    TRACE_FIELDS = ("pass", "row", "nupd", "y", "z", "sphi", "tgl", "qpt", "Cyy", "Czz", "Css", "Ctt", "Cqq",
                    "chi2", "ry", "rz")

    def set_trace(self, tracklet: int):
        """Record every Kalman update of one tracklet in the next find."""
        self._ck(self._lib.tpc_set_trace(self._ctx, tracklet))

    def trace(self) -> np.ndarray:
        n = ctypes.c_int32()
        out = np.zeros((2048, 16), np.float32)
        self._ck(self._lib.tpc_get_trace(self._ctx, out.ctypes.data, 2048, ctypes.byref(n)))
        return out[:min(n.value, 2048)]

    def autotune(self, clusters=None, req_offsets=None, reps: int = 3, cache: str | None = None, key: str = ""):
        """Choose launch shapes for the loaded (or given) batch with the
        library's autotuner; with `cache`, reuse or store the choice under
        `key` in that JSON file.  Returns (tuning dict, best ms)."""
        import json
        if cache and os.path.exists(cache):
            try:
                entry = json.load(open(cache)).get(key)
            except (OSError, ValueError):
                entry = None
            if entry:
                self.set_tuning(**entry["tuning"])
                return dict(entry["tuning"]), entry["ms"]
        if clusters is not None:
            self.load(clusters, req_offsets)
        best = TpcTuning()
        ms = ctypes.c_float()
        self._ck(self._lib.tpc_autotune(self._ctx, reps, ctypes.byref(best), ctypes.byref(ms)))
        choice = best.as_dict()
        if cache:
            data = {}
            if os.path.exists(cache):
                try:
                    data = json.load(open(cache))
                except (OSError, ValueError):
                    data = {}
            data[key] = {"tuning": choice, "ms": ms.value}
            with open(cache, "w") as f:
                json.dump(data, f, indent=1)
        return choice, ms.value

    def set_profiling(self, on: bool = True):
        self._ck(self._lib.tpc_set_profiling(self._ctx, int(on)))

    STAGES = ("grid", "neighbours", "links_tracklets", "follow", "select", "refit")

    def stage_times(self) -> dict:
        """Device ms per stage of the last profiled find + fit."""
        ms = np.zeros(6, np.float32)
        self._ck(self._lib.tpc_get_stage_times(self._ctx, ms.ctypes.data))
        return dict(zip(self.STAGES, (float(v) for v in ms)))

    def work(self) -> dict:
        w = np.zeros(5, np.uint64)
        self._ck(self._lib.tpc_get_work(self._ctx, w.ctypes.data))
        return dict(zip(("prop", "upd32", "upd64", "cand", "prop64"), (int(v) for v in w)))

    KALMAN_KERNELS = ("k_follow_p1", "k_follow_p1t", "k_follow_p2", "k_follow_p3", "k_follow_p3t", "k_follow_p4r",
                      "k_follow_p4", "k_refit_p1", "k_refit_p1t", "k_refit_p2")
    # the kernels whose covariance is in FP64 (the zone kernels and their tails)
    ZONE_KERNELS = ("k_follow_p1", "k_follow_p1t", "k_follow_p3", "k_follow_p3t", "k_refit_p1", "k_refit_p1t")

    def kalman_profile(self, times: bool = True) -> dict:
        """Per Kalman kernel: device ms of the last profiled run (when
        times) and its work counters (zero for a kernel the batch's size
        does not launch)."""
        ms = np.zeros(len(self.KALMAN_KERNELS), np.float32)
        w = np.zeros(5 * len(self.KALMAN_KERNELS), np.uint64)
        self._ck(self._lib.tpc_get_kalman_profile(self._ctx, ms.ctypes.data if times else None, w.ctypes.data))
        out = {}
        for k, name in enumerate(self.KALMAN_KERNELS):
            d = dict(zip(("prop", "upd32", "upd64", "cand", "prop64"), (int(v) for v in w[5 * k:5 * k + 5])))
            if times:
                d["ms"] = float(ms[k])
            out[name] = d
        return out

    def find_vertices(self, **cfg):
        """Vertex finding in the drift-time coordinate on the fitted tracks
        of the loaded timeframe (tpc_find_vertices; keyword arguments
        override tpc_vertex_config fields)."""
        c = VertexConfig()
        self._lib.tpc_default_vertex_config(ctypes.byref(c))
        for k, v in cfg.items():
            if not hasattr(c, k):
                raise TypeError(f"unknown vertex option {k}")
            setattr(c, k, v)
        self._ck(self._lib.tpc_find_vertices(self._ctx, ctypes.byref(c)))
        return self

    def reject(self, **cfg) -> dict:
        """Cluster rejection (tpc_reject_clusters; keyword arguments override
        tpc_reject_config fields): per track its class bits (RJ_*), per
        loaded cluster its keep flag, and the rejected-cluster counts (all,
        low momentum, inclined, further looper legs)."""
        c = RejectConfig()
        self._lib.tpc_default_reject_config(ctypes.byref(c))
        for k, v in cfg.items():
            if not hasattr(c, k) or k == "reserved":
                raise TypeError(f"unknown rejection option {k}")
            setattr(c, k, v)
        self._ck(self._lib.tpc_reject_clusters(self._ctx, ctypes.byref(c)))
        cnt = self.counts()
        cls = np.zeros(cnt["n_tracks"], np.uint8)
        keep = np.zeros(cnt["n"], np.uint8)
        counts = np.zeros(4, np.int64)
        self._ck(self._lib.tpc_get_rejection(self._ctx, cls.ctypes.data if len(cls) else None,
                                             keep.ctypes.data if len(keep) else None, counts.ctypes.data))
        return {"track_class": cls, "cluster_keep": keep,
                "counts": dict(zip(("all", "low_p", "inclined", "looper_leg"), (int(v) for v in counts)))}

    def vertices(self) -> dict:
        """Vertices (VERTEX_DTYPE, in time order) and per track: vertex index
        (-1: none), time estimate (us), spatial z (cm) and dz/ds_T."""
        nv = ctypes.c_int64()
        self._ck(self._lib.tpc_get_vertices(self._ctx, None, 0, ctypes.byref(nv), None, None, None, None))
        m = self.counts()["n_tracks"]
        out = np.zeros(nv.value, VERTEX_DTYPE)
        tv = np.zeros(m, np.int32)
        tt, tz, tg = (np.zeros(m, np.float32) for _ in range(3))
        self._ck(self._lib.tpc_get_vertices(self._ctx, out.ctypes.data if nv.value else None, nv.value,
                                            ctypes.byref(nv), tv.ctypes.data if m else None,
                                            tt.ctypes.data if m else None, tz.ctypes.data if m else None,
                                            tg.ctypes.data if m else None))
        return {"vertices": out, "track_vertex": tv, "track_time": tt, "track_z": tz, "track_tgl": tg}

    def merge(self, **cfg) -> dict:
        """Second tracking phase (tpc_merge_tracks): merged tracks and, per
        sector track, its merged outer partner, its merged track and the
        chi2 of its best and second-best outer candidates."""
        c = MergeConfig()
        self._lib.tpc_default_merge_config(ctypes.byref(c))
        for k, v in cfg.items():
            if not hasattr(c, k):
                raise TypeError(f"unknown merge option {k}")
            setattr(c, k, v)
        self._ck(self._lib.tpc_merge_tracks(self._ctx, ctypes.byref(c)))
        nm = ctypes.c_int64()
        self._ck(self._lib.tpc_get_merged(self._ctx, None, 0, ctypes.byref(nm), None, None, None, None))
        m = self.counts()["n_tracks"]
        out = np.zeros(nm.value, TRACK_DTYPE)
        link, chain = np.zeros(m, np.int32), np.zeros(m, np.int32)
        c2, c2s = np.zeros(m, np.float32), np.zeros(m, np.float32)
        p = lambda a: a.ctypes.data if len(a) else None  # noqa: E731
        self._ck(self._lib.tpc_get_merged(self._ctx, p(out), nm.value, ctypes.byref(nm), p(link), p(chain), p(c2),
                                          p(c2s)))
        return {"merged": out, "link": link, "chain": chain, "pair_chi2": c2, "pair_second": c2s}

    def compress(self, unit_cm: float = 0.01) -> dict:
        """Track-model compression of the fitted tracks (tpc_compress):
        headers (CODEC_HEADER_DTYPE), per cluster rows, residuals and the
        encoded fixed-point coordinates."""
        self._ck(self._lib.tpc_compress(self._ctx, unit_cm))
        m, n = ctypes.c_int64(), ctypes.c_int64()
        self._ck(self._lib.tpc_get_compressed(self._ctx, None, 0, None, None, None, None, None, 0,
                                              ctypes.byref(m), ctypes.byref(n)))
        heads = np.zeros(m.value, CODEC_HEADER_DTYPE)
        rows = np.zeros(n.value, np.uint8)
        ry, rz, qy, qz = (np.zeros(n.value, np.int32) for _ in range(4))
        p = lambda a: a.ctypes.data if len(a) else None  # noqa: E731
        self._ck(self._lib.tpc_get_compressed(self._ctx, p(heads), m.value, p(rows), p(ry), p(rz), p(qy), p(qz),
                                              n.value, ctypes.byref(m), ctypes.byref(n)))
        return {"heads": heads, "rows": rows, "res_y": ry, "res_z": rz, "q_y": qy, "q_z": qz, "unit": unit_cm}

    def decompress(self, heads, rows, res_y, res_z, unit_cm: float = 0.01):
        """Fixed-point clusters (q_y, q_z) restored from a compressed stream."""
        heads = np.ascontiguousarray(heads, dtype=CODEC_HEADER_DTYPE)
        rows = np.ascontiguousarray(rows, dtype=np.uint8)
        ry = np.ascontiguousarray(res_y, dtype=np.int32)
        rz = np.ascontiguousarray(res_z, dtype=np.int32)
        n = len(rows)
        qy, qz = np.zeros(n, np.int32), np.zeros(n, np.int32)
        p = lambda a: a.ctypes.data if len(a) else None  # noqa: E731
        self._ck(self._lib.tpc_decompress(self._ctx, p(heads), len(heads), p(rows), p(ry), p(rz), n, unit_cm,
                                          p(qy), p(qz)))
        return qy, qz

    def graph_kernels(self) -> int:
        n = ctypes.c_int32()
        self._ck(self._lib.tpc_graph_kernels(self._ctx, ctypes.byref(n)))
        return n.value

    def counts(self) -> dict:
        c = np.zeros(8, np.int64)
        self._ck(self._lib.tpc_get_counts(self._ctx, c.ctypes.data))
        return dict(zip(("n", "n_req", "n_rs", "n_bins", "n_tracklets", "n_tracks", "status", "n_track_clusters"),
                        (int(v) for v in c)))

    def submit_batch(self, requests):
        """Submit independent requests as one batch (tpc_submit_batch) and
        return at once.  requests: list of (id, clusters) or (id, clusters,
        tracks_out, cluster_track_out) -- host buffers (numpy arrays or pinned
        CPU torch tensors); missing result buffers are allocated.  Results
        with poll()."""
        reqs = (TpcRequest * len(requests))()
        keep = []
        n_min = max(self._n_min_track(), 1)
        for k, rq in enumerate(requests):
            rid, clusters = rq[0], rq[1]
            cl = _records(clusters, CLUSTER_DTYPE, 0)
            n = len(cl)
            tr = _records(rq[2] if len(rq) > 2 and rq[2] is not None else np.zeros(n // n_min + 1, TRACK_DTYPE),
                          TRACK_DTYPE, 0)
            ct = _records(rq[3] if len(rq) > 3 and rq[3] is not None else np.zeros(n, np.int32), np.int32, n)
            nt = np.full(1, -1, np.int64)
            reqs[k].id, reqs[k].n, reqs[k].cap = rid, n, len(tr)
            reqs[k].clusters = cl.ctypes.data if n else None
            reqs[k].tracks_out = tr.ctypes.data if len(tr) else None
            reqs[k].cluster_track_out = ct.ctypes.data if n else None
            reqs[k].n_tracks = nt.ctypes.data
            keep.append((rid, clusters, cl, tr, ct, nt))
        self._ck(self._lib.tpc_submit_batch(self._ctx, reqs, len(requests)))
        self._batch = {k[0]: k for k in keep}
        self.n = sum(len(k[2]) for k in keep)
        return self

    def poll(self, request_id: int):
        """(tracks, cluster_track) of a finished request of the submitted
        batch -- views of its buffers -- or None while it runs.  Raises
        TpcError when the request failed (e.g. TPC_EOVERFLOW: tracks_out too
        small)."""
        done = ctypes.c_int()
        rc = self._lib.tpc_poll(self._ctx, request_id, ctypes.byref(done))
        if rc != 0:
            raise TpcError(rc, self._lib.tpc_last_error(self._ctx).decode())
        if not done.value:
            return None
        _, _, _, tr, ct, nt = self._batch[request_id]
        return tr[:int(nt[0])], ct

    def _n_min_track(self) -> int:
        return self._cfg.n_min_track if self._cfg is not None else default_config().n_min_track

    def get_into(self, tracks_out, cluster_track_out=None):
        """Wait and copy the results into caller buffers (numpy arrays or
        pinned CPU torch tensors); returns (tracks view, cluster_track)."""
        tr = _records(tracks_out, TRACK_DTYPE, 0)
        ct = _records(cluster_track_out, np.int32, self.n)
        nout = ctypes.c_int64()
        self._ck(self._lib.tpc_get_tracks(self._ctx, tr.ctypes.data if len(tr) else None, len(tr),
                                          ctypes.byref(nout), ct.ctypes.data if ct is not None and self.n else None,
                                          None))
        return tr[:nout.value], ct

    def arena_bytes(self) -> int:
        b = ctypes.c_size_t()
        self._ck(self._lib.tpc_get_arena_bytes(self._ctx, ctypes.byref(b)))
        return b.value

    def get(self, cluster_track: bool = True, track_clusters: bool = False, cap: int | None = None):
        """Wait and copy out: (tracks, cluster_track, track_clusters)."""
        nout = ctypes.c_int64()
        if cap is None:
            rc = self._lib.tpc_get_tracks(self._ctx, None, 0, ctypes.byref(nout), None, None)
            if rc not in (0, TPC_EOVERFLOW):
                self._ck(rc)
            cap = nout.value
        tracks = np.zeros(cap, TRACK_DTYPE)
        ct = np.zeros(self.n, np.int32) if cluster_track else None
        tc = None
        if track_clusters:
            tc = np.zeros(max(self.counts()["n_track_clusters"], 1), np.int32)
        self._ck(self._lib.tpc_get_tracks(self._ctx, tracks.ctypes.data, cap, ctypes.byref(nout),
                                          ct.ctypes.data if ct is not None and self.n else None,
                                          tc.ctypes.data if tc is not None else None))
        return tracks[:nout.value], ct, tc

    def stage(self, name: str) -> np.ndarray:
        item, dtype = ITEMS[name]
        nb = ctypes.c_int64()
        self._ck(self._lib.tpc_get_stage(self._ctx, item, None, 0, ctypes.byref(nb)))
        out = np.zeros(nb.value // np.dtype(dtype).itemsize, dtype)
        if nb.value:
            self._ck(self._lib.tpc_get_stage(self._ctx, item, out.ctypes.data, nb.value, ctypes.byref(nb)))
        if name == "f_hits":
            out = out.reshape(-1, 159)
        elif name == "f_par":
            out = out.reshape(-1, 5)
        elif name == "f_cov":
            out = out.reshape(-1, 15)
        return out

    def track_into(self, clusters, tracks_out, cluster_track_out=None):
        """load + find + fit + get_into (one request), retrying a capacity
        overflow once with the worst-case capacities, as track()."""
        for attempt in range(2):
            self.load(clusters).find().fit()
            try:
                return self.get_into(tracks_out, cluster_track_out)
            except TpcError as e:
                if e.code != TPC_EOVERFLOW or attempt:
                    raise
                c = self.counts()
                if not c["status"] & 2:  # not a device capacity (the caller's buffer is too small)
                    raise
                self.reserve(n_clusters=self.n, n_requests=1, n_bins=max(2 * c["n_bins"], 0),
                             n_tracklets=self.n // 3 + 16)
        raise AssertionError("unreachable")

    def track_host(self, clusters, tracks_out, cluster_track_out=None):
        """tpc_track_host: host clusters (numpy structured array) in, tracks and
        cluster assignment out, in one call whose assignment copy overlaps the
        refit (page-locked output buffers keep the copies asynchronous);
        retries a device capacity overflow once with the worst-case
        capacities, as track_into.  Returns (tracks view, cluster_track)."""
        clusters = np.ascontiguousarray(clusters)
        n = len(clusters)
        tr = _records(tracks_out, TRACK_DTYPE, 0)
        ct = _records(cluster_track_out, np.int32, n)
        nout = ctypes.c_int64()
        for attempt in range(2):
            self._keep_in = clusters
            rc = self._lib.tpc_track_host(self._ctx, _ptr(clusters) if n else None, n,
                                          tr.ctypes.data if len(tr) else None, len(tr), ctypes.byref(nout),
                                          ct.ctypes.data if ct is not None and n else None)
            self.n = n
            if rc == TPC_EOVERFLOW and not attempt:
                c = self.counts()
                if c["status"] & 2:  # a device capacity, not the caller's buffer
                    self.reserve(n_clusters=n, n_requests=1, n_bins=max(2 * c["n_bins"], 0),
                                 n_tracklets=n // 3 + 16)
                    continue
            self._ck(rc)
            return tr[:nout.value], ct
        raise AssertionError("unreachable")

    def track(self, clusters, req_offsets=None, graph: bool = False):
        """load + find + fit (+ graph) + get.  A capacity overflow (more
        tracklets or grid bins than reserved; reported, never truncated) is
        retried once with the worst-case capacities."""
        for attempt in range(2):
            self.load(clusters, req_offsets)
            if graph:
                self.run_graph()
            else:
                self.find().fit()
            try:
                return self.get()
            except TpcError as e:
                if e.code != TPC_EOVERFLOW or attempt:
                    raise
                n = self.n
                nreq = 1 if req_offsets is None else len(req_offsets) - 1
                c = self.counts()
                self.reserve(n_clusters=n, n_requests=nreq, n_bins=max(2 * c["n_bins"], 0),
                             n_tracklets=n // 3 + 16)
        raise AssertionError("unreachable")


def _records(buf, dtype, n):
    """A numpy view of n `dtype` records over a numpy array or a (pinned)
    CPU torch tensor; None stays None."""
    if buf is None:
        return None
    if hasattr(buf, "data_ptr"):
        buf = buf.numpy()
    v = buf.view(np.uint8).reshape(-1).view(dtype)
    if len(v) < n:
        raise ValueError(f"buffer holds {len(v)} records, {n} needed")
    return v


class Server:
    """Continuous-batching request loop (tpc_server_*): up to max_slots
    requests run at once, each on its own context and stream, admitted in
    arrival order while their arenas fit hbm_budget and free device memory.

    Results are written straight into buffers given at submission (numpy
    arrays or pinned CPU torch tensors; page-locked ones let the copies
    overlap other requests' kernels); without them, numpy buffers are
    allocated.  Inputs and buffers are referenced until result() returns."""

    STATES = {-1: "unknown", 0: "queued", 1: "running", 2: "finished", 3: "failed"}

    def __init__(self, device: int = 0, cfg: TpcConfig | None = None, max_slots: int = 4, hbm_budget: int = 0,
                 queue_cap: int = 1 << 20):
        self._lib = load_library()
        self._srv = ctypes.c_void_p()
        self._n_min = (cfg or default_config()).n_min_track
        rc = self._lib.tpc_server_create(ctypes.byref(self._srv), ctypes.byref(cfg) if cfg else None, device,
                                         max_slots, hbm_budget, queue_cap)
        if rc != 0:
            raise TpcError(rc, "tpc_server_create failed")
        self._live = {}

    def close(self):
        if self._srv:
            self._lib.tpc_server_destroy(self._srv)
            self._srv = ctypes.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, request_id: int, clusters, tracks_out=None, cluster_track_out=None) -> int:
        """Queue one request (host clusters: CLUSTER_DTYPE records, numpy or
        a pinned CPU torch tensor).  Returns 0, or TPC_EBUSY when the queue
        is full."""
        cl = _records(clusters, CLUSTER_DTYPE, 0)
        n = len(cl)
        if tracks_out is None:
            tracks_out = np.zeros(n // max(self._n_min, 1) + 1, TRACK_DTYPE)
        if cluster_track_out is None:
            cluster_track_out = np.zeros(n, np.int32)
        tr = _records(tracks_out, TRACK_DTYPE, 0)
        ct = _records(cluster_track_out, np.int32, n)
        rc = self._lib.tpc_server_submit(self._srv, request_id, cl.ctypes.data if n else None, n,
                                         tr.ctypes.data if len(tr) else None, len(tr),
                                         ct.ctypes.data if n else None)
        if rc == 0:
            self._live[request_id] = (clusters, cl, tr, ct, tracks_out, cluster_track_out)
        elif rc != TPC_EBUSY:
            raise TpcError(rc, f"tpc_server_submit({request_id})")
        return rc

    def poll(self, request_id: int) -> str:
        st = ctypes.c_int()
        self._lib.tpc_server_poll(self._srv, request_id, ctypes.byref(st))
        return self.STATES[st.value]

    def result(self, request_id: int):
        """(tracks, cluster_track, times_ms) of a finished request -- views
        of the buffers given at submission -- or None while it is queued or
        running.  times_ms: queue wait, service and total latency in ms.
        Raises TpcError if the request failed."""
        nt = ctypes.c_int64()
        times = np.zeros(3, np.float64)
        rc = self._lib.tpc_server_result(self._srv, request_id, ctypes.byref(nt), times.ctypes.data)
        if rc == TPC_EBUSY:
            return None
        live = self._live.pop(request_id, None)
        if rc != 0:
            raise TpcError(rc, f"request {request_id} failed ({nt.value} tracks found)")
        _, _, tr, ct, _, _ = live
        return tr[:nt.value], ct, times

    def drain(self, timeout_s: float = 0.0):
        rc = self._lib.tpc_server_drain(self._srv, timeout_s)
        if rc != 0:
            raise TpcError(rc, "drain timed out")

    def stats(self) -> dict:
        st = np.zeros(5, np.int64)
        self._lib.tpc_server_stats(self._srv, st.ctypes.data)
        return dict(zip(("admitted", "completed", "queued", "arena_bytes", "peak_running"), (int(v) for v in st)))


def measure_alu_peaks(device: int = 0) -> dict:
    """Measured FP32 and FP64 FMA-pipe rates of the device in TFLOP/s."""
    f32, f64 = ctypes.c_double(), ctypes.c_double()
    rc = load_library().tpc_measure_alu_peaks(device, ctypes.byref(f32), ctypes.byref(f64))
    if rc != 0:
        raise TpcError(rc, "tpc_measure_alu_peaks failed")
    return {"fp32_tflops": f32.value, "fp64_tflops": f64.value}


def row_params_noalloc(d_clusters, req_offsets=None, out=None, stream=None) -> int:
    """Per-row-sector grid records of device-resident clusters without any
    device allocation by the library (tpc_row_params_noalloc): for callers
    that may not allocate, e.g. under a memory budget owned by their host
    framework.  d_clusters and out are contiguous CUDA tensors on the same
    device (out: n_req*36*159*32 bytes, caller-allocated).  The call runs
    with that device current and, without `stream`, on torch's current
    stream of it.  Returns the status code."""
    import torch
    lib = load_library()
    n = d_clusters.numel() * d_clusters.element_size() // 16
    off = np.ascontiguousarray(np.asarray(req_offsets if req_offsets is not None else [0, n], dtype=np.int64))
    n_req = len(off) - 1
    need = n_req * 36 * 159 * 32
    if not (d_clusters.is_cuda and out is not None and out.is_cuda):
        raise ValueError("d_clusters and out must be CUDA tensors")
    if d_clusters.device != out.device:
        raise ValueError(f"d_clusters on {d_clusters.device}, out on {out.device}: one device expected")
    if not (d_clusters.is_contiguous() and out.is_contiguous()):
        raise ValueError("d_clusters and out must be contiguous")
    if d_clusters.numel() * d_clusters.element_size() != 16 * n:
        raise ValueError("d_clusters must hold whole 16-byte cluster records")
    if out.numel() * out.element_size() < need:
        raise ValueError(f"out holds {out.numel() * out.element_size()} bytes, {need} needed")
    with torch.cuda.device(d_clusters.device):
        if stream is None:
            sp = torch.cuda.current_stream().cuda_stream
        else:
            sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        return lib.tpc_row_params_noalloc(d_clusters.data_ptr() if n else None, n, off.ctypes.data, n_req,
                                          out.data_ptr(), sp)
