"""CPU-side checks of the C ABI: the library builds, loads and exports every
symbol declared in include/tpcca.h, and its host logic fails cleanly."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1709_00618_b300 as tpc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "tpcca.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tpc_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    tpc.build()
    lib = ctypes.CDLL(tpc.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_default_config_is_the_reading():
    cfg = tpc.default_config()
    assert cfg.bz_kg == 5.0 and cfg.sigma == 0.1 and cfg.min_chain == 3 and cfg.max_miss == 5
    assert cfg.n_min_track == 10 and cfg.gate == 16.0 and list(cfg.c0) == [100, 100, 1, 1, 100]
    assert cfg.s_max == 0.95 and cfg.fp64_updates == 10 and abs(cfg.d_max - 1.0) < 1e-7


def test_binding_flags_match_the_header():
    txt = open(os.path.join(ROOT, "include", "tpcca.h")).read()
    val = {k: int(v) for k, v in re.findall(r"\b(TPC_TF_[A-Z_]+|TPC_RJ_[A-Z_]+)\s*=\s*(\d+)", txt)}
    assert val["TPC_TF_SEED_FAIL"] == tpc.TF_SEED_FAIL and val["TPC_TF_BACK_FAIL"] == tpc.TF_BACK_FAIL
    assert val["TPC_TF_REFIT_FAIL"] == tpc.TF_REFIT_FAIL
    assert tpc.TF_TAINT_ANY == sum(v for k, v in val.items() if k.startswith("TPC_TF_TAINT_"))


def test_arena_size_grows_with_input():
    lib = tpc.load_library()
    a, b, c = lib.tpc_arena_bytes(1000, 1), lib.tpc_arena_bytes(1_000_000, 1), lib.tpc_arena_bytes(1_000_000, 4)
    assert 0 < a < b < c
    assert b % 256 == 0


def test_bad_arguments_are_rejected_without_a_device():
    lib = tpc.load_library()
    assert lib.tpc_load_clusters(None, None, 0, 0) == tpc.TPC_EINVAL
    assert lib.tpc_find_tracks(None) == tpc.TPC_EINVAL
    assert lib.tpc_get_tracks(None, None, 0, None, None, None) == tpc.TPC_EINVAL
    bad = tpc.default_config(s_max=1.5)
    ctx = ctypes.c_void_p()
    assert lib.tpc_create(ctypes.byref(ctx), ctypes.byref(bad), 0, None, 0) == tpc.TPC_EINVAL


def test_create_without_gpu_reports_cuda_error():
    lib = tpc.load_library()
    ctx = ctypes.c_void_p()
    rc = lib.tpc_create(ctypes.byref(ctx), None, 0, None, 0)
    if rc == 0:
        lib.tpc_destroy(ctx)
        pytest.skip("a GPU is present")
    assert rc == tpc.TPC_ECUDA


def test_server_arguments_are_checked_without_a_device():
    lib = tpc.load_library()
    srv = ctypes.c_void_p()
    assert lib.tpc_server_create(ctypes.byref(srv), None, 0, 0, 0, 16) == tpc.TPC_EINVAL
    assert lib.tpc_server_create(ctypes.byref(srv), None, 0, 4, 0, 0) == tpc.TPC_EINVAL
    assert lib.tpc_server_create(None, None, 0, 4, 0, 16) == tpc.TPC_EINVAL
    assert lib.tpc_server_submit(None, 1, None, 0, None, 0, None) == tpc.TPC_EINVAL
    st = ctypes.c_int()
    assert lib.tpc_server_poll(None, 1, ctypes.byref(st)) == tpc.TPC_EINVAL
    assert lib.tpc_server_result(None, 1, None, None) == tpc.TPC_EINVAL
    assert lib.tpc_get_tracks_async(None, None, 0, None, None) == tpc.TPC_EINVAL
    assert lib.tpc_get_arena_bytes(None, None) == tpc.TPC_EINVAL
    assert lib.tpc_server_drain(None, 0.0) == tpc.TPC_EINVAL
    lib.tpc_server_destroy(None)
    rc = lib.tpc_server_create(ctypes.byref(srv), None, 0, 2, 0, 16)
    if rc == 0:
        lib.tpc_server_destroy(srv)
        pytest.skip("a GPU is present")
    assert rc == tpc.TPC_ECUDA


def test_binding_structs_match_the_header():
    """The binding's mirror of tpc_tuning has the header's fields in order,
    and its Kalman kernel names the header's count (tpc_get_kalman_profile
    fills TPC_KALMAN_KERNELS times and 5 counters each)."""
    txt = open(os.path.join(ROOT, "include", "tpcca.h")).read()
    end = txt.index("} tpc_tuning;")
    body = txt[txt.rindex("typedef struct {", 0, end):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"int32_t\s+([a-z_0-9]+)\s*;", body)
    assert fields == [name for name, _ in tpc.TpcTuning._fields_]
    n = int(re.search(r"#define TPC_KALMAN_KERNELS (\d+)", txt).group(1))
    assert n == len(tpc.Tracker.KALMAN_KERNELS)
    assert set(tpc.Tracker.ZONE_KERNELS) <= set(tpc.Tracker.KALMAN_KERNELS)
